// ws_device.cuh -- device-side types, memory-model primitives and hashing.
//
// Memory-model primitives (paper §3.1 "GPU memory model", §4.2 "Lock-free
// concurrent queries"): every access to shared table state is a morally
// strong .gpu-scope operation that is served by the coherent L2, never by a
// stale L1 line.  Slots are 16-byte {key, value} pairs read and written only
// with 128-bit accesses, so a reader sees either the whole old pair or the
// whole new pair (the paper requires reader and writer widths to match).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ws {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;
typedef unsigned char u8;

// Sentinel keys.  EMPTY slots were never used; TOMB marks an erased slot that
// inserts may reuse (§5.1 Erase leaves a tombstone; EMPTY never comes back, so
// a scan may stop at an EMPTY slot).  RESV is the reservation marker of §4.2,
// rejected as a user key; this build claims slots with one 128-bit CAS and so
// never writes it.
constexpr u64 KEY_EMPTY = 0ull;
constexpr u64 KEY_TOMB = ~0ull;
constexpr u64 KEY_RESV = ~0ull - 1ull;
constexpr u16 TAG_EMPTY = 0, TAG_TOMB = 1;

enum { ST_MISS = 0, ST_FOUND = 1, ST_INSERTED = 2, ST_FULL = 3, ST_BADKEY = 4, ST_TIMEOUT = 5 };
enum { OP_ADD = 0, OP_MAX = 1, OP_REPLACE = 2, OP_INSERT = 3 };
enum { MX_QUERY = 0, MX_INSERT = 1, MX_ADD = 2, MX_MAX = 3, MX_REPLACE = 4, MX_ERASE = 5 };
enum { KIND_QUERY = 0, KIND_UPSERT = 1, KIND_ERASE = 2, KIND_MIXED = 3, KIND_PROBE = 4 };
enum { SCHEME_DOUBLE = 0, SCHEME_P2 = 1, SCHEME_ICEBERG = 2 };

struct __align__(16) Slot {
  u64 key, val;
};

// Device counters of a table (one 64-byte line).
struct Counters {
  u64 count;      // live keys
  u64 n_full;     // inserts that found no free slot
  u64 n_timeout;  // ops that hit the lock spin limit
  u64 n_badkey;   // ops on sentinel keys / unknown op codes
  u64 ticket;     // work ticket of the running single-table launch
  u64 done;       // blocks of that launch that finished; the last one zeroes both
  u64 pad[2];
};

// What a kernel needs of a table, passed by value.
struct TableView {
  Slot* slots;    // nb * B slots
  u16* tags;      // nb * B tags (metadata tables) or null
  u32* locks;     // one bit per bucket
  Counters* ctr;
  u64 nb_mask;    // nb - 1
  u64 nb_front;   // iceberg: front-yard buckets [0, nb_front), backyard [nb_front, nb)
  u64 nb_back;    // iceberg: nb - nb_front (at least 2)
  u64 seed1, seed2;
  u32 pmax;       // double hashing: buckets a probe sequence may visit (<= nb)
  u32 spin_limit; // lock attempts before giving up
  int shortcut;   // P2: no erase ever ran, so the primary-fill shortcut is exact
  int preload;    // the lane path with cp.async snapshots (1), or every op to the tiles (0)
  int phased;     // bulk-synchronous mode: weak cacheable probe loads, no locks (see WS_OPT_PHASED)
  int lane_waves; // double hashing: buckets the lane path checks before the tiles (0 = default)
  int stream;     // single-table launches: streaming lanes (1) or 32-op chunks (0); see WS_OPT_STREAM
};

struct BatchArgs {
  const u64* keys;
  const u64* vals;
  const u8* ops;
  u64* vals_out;
  u8* status_out;
  u64 n;
  int op;          // upsert callback for KIND_UPSERT
  u32 key_stride;  // elements between consecutive keys / values (0 or 1: dense; 2: a slot array)
  u32 flags;       // BATCH_SKIP_SENTINELS, BATCH_HOST_INPUTS
};
// BATCH_SKIP_SENTINELS: sentinel keys are skipped silently (rehash of a slot
// array).  BATCH_HOST_INPUTS: keys and values are page-locked host memory
// read in place over the host link; streaming warps then copy each lane's
// next inputs into shared memory a wave ahead (cp.async), so the link's
// latency does not hold up the warp's waves.
enum { BATCH_SKIP_SENTINELS = 1, BATCH_HOST_INPUTS = 2 };

// -------------------------------------------------------------------------
// Hashing.  The paper does not fix its hash functions; this build uses the
// MurmurHash3 64-bit finaliser (Appleby, public domain) of key ^ seed for the
// two independent hashes h1, h2 (§2.2: double hashing uses two hash
// functions, two-choice hashing two bucket choices).
// -------------------------------------------------------------------------
__device__ __forceinline__ u64 fmix64(u64 x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// Fingerprint (§5 "Concurrency and metadata": the low 16 bits of the key),
// lifted out of the two reserved tag values.
__device__ __forceinline__ u16 key_tag(u64 k) {
  u16 t = (u16)(k & 0xffffu);
  return t < 2 ? (u16)(t + 2) : t;
}

__device__ __forceinline__ bool is_sentinel(u64 k) { return k == KEY_EMPTY || k >= KEY_RESV; }

// -------------------------------------------------------------------------
// PTX primitives (PTX ISA >= 8.3 for .b128; atom.cas.b128 needs sm_90+).
// -------------------------------------------------------------------------
namespace ptx {

__device__ __forceinline__ void ld_slot(const Slot* p, u64& k, u64& v) {
  asm volatile(
      "{\n\t.reg .b128 t;\n\t"
      "ld.relaxed.gpu.global.b128 t, [%2];\n\t"
      "mov.b128 {%0, %1}, t;\n\t}"
      : "=l"(k), "=l"(v)
      : "l"(p)
      : "memory");
}

// Weak (L1-cacheable) loads for the bulk-synchronous mode: valid only while
// nothing writes what they read during the launch.
__device__ __forceinline__ void ld_slot_weak(const Slot* p, u64& k, u64& v) {
  asm volatile("ld.global.v2.u64 {%0, %1}, [%2];" : "=l"(k), "=l"(v) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_tags16_weak(const u16* p, u64& a, u64& b) {
  asm volatile("ld.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

// 128-bit compare-and-swap of a whole slot (relaxed: the pair itself is the
// published datum; a lock release or a release store orders it where needed).
// Returns true on success.
__device__ __forceinline__ bool cas_slot(Slot* p, u64 ek, u64 ev, u64 nk, u64 nv) {
  u64 ok, ov;
  asm volatile(
      "{\n\t.reg .b128 d, c, s;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 s, {%4, %5};\n\t"
      "atom.relaxed.gpu.global.cas.b128 d, [%6], c, s;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(ok), "=l"(ov)
      : "l"(ek), "l"(ev), "l"(nk), "l"(nv), "l"(p)
      : "memory");
  return ok == ek && ov == ev;
}

// Tag claim (acquire: the claimer's later pair store must come after the
// eraser's tombstone of that slot, which the eraser released with the tag).
__device__ __forceinline__ u16 cas_tag(u16* p, u16 expect, u16 desired) {
  u16 old;
  asm volatile("atom.acquire.gpu.global.cas.b16 %0, [%1], %2, %3;"
               : "=h"(old)
               : "l"(p), "h"(expect), "h"(desired)
               : "memory");
  return old;
}

// The pair store of a metadata claim.  It follows the tag CAS, which has
// acquire semantics, so it cannot be performed before the claim; no earlier
// write of the thread needs to be published with it, so no release (a
// release store waits for all of them).
__device__ __forceinline__ void st_slot_relaxed(Slot* p, u64 k, u64 v) {
  asm volatile(
      "{\n\t.reg .b128 t;\n\t"
      "mov.b128 t, {%1, %2};\n\t"
      "st.relaxed.gpu.global.b128 [%0], t;\n\t}" ::"l"(p),
      "l"(k), "l"(v)
      : "memory");
}

__device__ __forceinline__ void st_tag_release(u16* p, u16 v) {
  asm volatile("st.release.gpu.global.b16 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}
// The TOMB tag of an erase in a launch where nothing claims slots (an
// erase-only call): no claimer can observe it before the launch ends.
__device__ __forceinline__ void st_tag_relaxed(u16* p, u16 v) {
  asm volatile("st.relaxed.gpu.global.b16 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}

__device__ __forceinline__ u32 ld_u32_relaxed(const u32* p) {
  u32 v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ u32 atom_or_acquire(u32* p, u32 m) {
  u32 old;
  asm volatile("atom.acquire.gpu.global.or.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(m) : "memory");
  return old;
}

__device__ __forceinline__ void red_and_release(u32* p, u32 m) {
  asm volatile("red.release.gpu.global.and.b32 [%0], %1;" ::"l"(p), "r"(m) : "memory");
}
// Unlock by a holder that wrote nothing under the lock (its key was present,
// or its claim lost): there is nothing to publish, so no release.
__device__ __forceinline__ void red_and_relaxed(u32* p, u32 m) {
  asm volatile("red.relaxed.gpu.global.and.b32 [%0], %1;" ::"l"(p), "r"(m) : "memory");
}

__device__ __forceinline__ void red_add_u64(u64* p, u64 v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_max_u64(u64* p, u64 v) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_u64_relaxed(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Asynchronous 16-byte global -> shared copy through L2 (cp.async.cg): an
// op's bucket snapshot lands in shared memory without holding registers, so
// a warp keeps all 32 of its ops' probes of a wave in flight.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const u32 d = (u32)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
// 8-byte asynchronous global -> shared copy (cp.async.ca: the .cg form
// copies 16 bytes only); used to fetch batch inputs a wave ahead.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const u32 d = (u32)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Tag loads of 16, 8, 4 or 2 bytes (one lane's share of a 64-byte tag line).
__device__ __forceinline__ void ld_tags16(const u16* p, u64& a, u64& b) {
  asm volatile(
      "{\n\t.reg .b128 t;\n\t"
      "ld.relaxed.gpu.global.b128 t, [%2];\n\t"
      "mov.b128 {%0, %1}, t;\n\t}"
      : "=l"(a), "=l"(b)
      : "l"(p)
      : "memory");
}
__device__ __forceinline__ u64 ld_tags8(const u16* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ u32 ld_tags4(const u16* p) {
  u32 v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ u16 ld_tags2(const u16* p) {
  u16 v;
  asm volatile("ld.relaxed.gpu.global.b16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace ptx
}  // namespace ws
