// ws_kernels.cuh -- batch kernels for bucketed open addressing.
//
// Two levels serve an op.  The lane path: each lane owns one op and follows
// its probe sequence one bucket (or one 128-byte line) per wave, from a
// snapshot that the warp copies into shared memory with cp.async -- four ops'
// lines per copy instruction, so up to 32 probes of a warp are in flight per
// wave.  Single-table calls run "streaming lanes": a warp serves shares of
// the batch that it takes from a per-launch ticket, and a lane takes the
// next op as soon as its op settles.  What a lane cannot settle alone goes to
// cooperative tiles of T lanes (T in {4, 8, 16, 32}, §3.2 / §5), which read
// a bucket in steps of T consecutive 16-byte slots and decide with warp
// votes, identically on all lanes of the tile: several tag matches, a lost
// CAS, an insert without the lock, the probe-count kernel.
//
// Probe schemes (§2.2):
//   double hashing  b_i = (h1 + i * (h2 | 1)) mod nb, i < max_probe; a scan
//                   ends at the first bucket holding an EMPTY slot.
//   two-choice      b_0 = h1 mod nb, b_1 = h2 mod nb (b_0 + 1 if equal); an
//                   insert goes to b_0 while it is below 3/4 full (the
//                   "shortcut" of §2.2), otherwise to the less loaded bucket
//                   (ties to b_0).
//   iceberg         a front-yard bucket by single hashing, then two backyard
//                   choices; a key goes to its front bucket while that has a
//                   free slot.
// Fingerprints (§4.3): with metadata, each 32-slot bucket has a 64-byte line
// of 16-bit tags.  A probe reads the tag line, and only slots whose tag
// matches are read and compared against the full key, so the result is exact.
//
// Snapshots stand in for lock-free reads only: a query answer may come from
// one (queried keys are not written in the same call), every write is a CAS
// against the current slot, and what decides an insert under a lock is read
// after the lock was taken.
//
// Concurrency (§4.1, §4.2):
//   * queries take no lock; each slot is read as one 16-byte pair;
//   * a present key is updated in place with a 64-bit atomic and no lock
//     (stability, §2.1: keys never move);
//   * plain insert / upsert calls on double-hashing tables need no lock at all
//     (no erase runs in the same call, see do_upsert);
//   * otherwise an absent key is inserted under the lock bit of its primary
//     bucket b_0 (one bit per bucket in an external array; iceberg: the front
//     bucket): insert-if-unique ops take it before probing, add / max /
//     replace only once the key is proven absent.  The holder re-reads and
//     claims a free slot with one 128-bit CAS that publishes key and value
//     together (metadata tables: a 16-bit CAS on the tag, then a 128-bit
//     store of the pair).  The lock makes same-key inserters agree on one location (the
//     adversarial case of Fig. 2);
//   * erase swaps the pair for {TOMB, 0} with a 128-bit CAS (then the tag
//     becomes TOMB).  A tombstone never turns back into EMPTY, which keeps
//     every early-exit rule valid.
// Every wait is bounded: after spin_limit attempts the op reports
// WS_FAIL_TIMEOUT.  A tile waiting for a lock keeps re-probing lock-free and
// finishes without the lock as soon as the key appears.
#pragma once
#include "ws_device.cuh"

namespace ws {

template <int T>
struct TileCtx {
  unsigned mask;  // this tile's lanes within the warp
  int tl;         // lane index inside the tile
  int base;       // first warp lane of the tile

  __device__ __forceinline__ unsigned ballot(bool p) const {
    constexpr unsigned kLow = (T >= 32) ? 0xffffffffu : ((1u << (T & 31)) - 1u);
    const unsigned b = __ballot_sync(mask, p);
    if (T == 32) return b;
    return (b >> base) & kLow;
  }
  __device__ __forceinline__ u64 shfl(u64 v, int src) const { return __shfl_sync(mask, v, src, T); }
  __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(mask, v, src, T); }
};

template <int T>
__device__ __forceinline__ TileCtx<T> make_tile(int lane) {
  TileCtx<T> c;
  c.tl = lane & (T - 1);
  c.base = lane & ~(T - 1);
  c.mask = (T == 32) ? 0xffffffffu : (((1u << (T & 31)) - 1u) << c.base);
  return c;
}

// Bucket snapshots of a warp's 32 ops, in shared memory, op-major with one
// spare slot per op (9 slots = 144 bytes): an asynchronous copy of an op's
// 128-byte line lands in contiguous shared memory (one wavefront per line),
// and 8 lanes reading slot s of their own ops hit distinct banks.  Plain
// tables: slots 0..7 of op j = the first line of its bucket.  Metadata
// tables: slots 0..3 = the bucket's 32 tags (eight per slot), slot 4 = the
// first tag-matching slot's pair, slot 5 .key = that slot's index (~0 when no
// tag matched).  The whole-bucket rounds view the same array flat: bucket q
// of a round at [32 q, 32 q + 32).
constexpr int kPreStride = 9;
struct __align__(16) PreWarp {
  Slot s[32 * kPreStride];
  __device__ __forceinline__ Slot& at(int j, int k) { return s[j * kPreStride + k]; }
  __device__ __forceinline__ const Slot& at(int j, int k) const { return s[j * kPreStride + k]; }
  __device__ __forceinline__ Slot& flat(int q, int lane) { return s[q * 32 + lane]; }
};
constexpr u64 kNoCand = ~0ull;

// One op's view of its warp's snapshots (w == nullptr: no snapshot).
struct PreRef {
  const PreWarp* w;
  int j;
  __device__ __forceinline__ bool ok() const { return w != nullptr; }
  __device__ __forceinline__ Slot slot(int k) const { return w->at(j, k); }
  __device__ __forceinline__ const u16* tagrow(int r) const { return reinterpret_cast<const u16*>(&w->at(j, r)); }
  __device__ __forceinline__ Slot cand() const { return w->at(j, 4); }
  __device__ __forceinline__ u64 cand_idx() const { return w->at(j, 5).key; }
};
__device__ __forceinline__ PreRef no_pre() { return PreRef{nullptr, 0}; }

template <int SCHEME, bool META, int B, int T>
struct TileOps {
  static_assert(B == 8 || B == 16 || B == 32, "bucket size");
  static_assert(T == 4 || T == 8 || T == 16 || T == 32, "tile size");
  static_assert(!META || B == 32, "metadata tables use 32-slot buckets (one 64-byte tag line)");
  static_assert(SCHEME != SCHEME_ICEBERG || META, "the iceberg scheme is built with metadata only");
  static constexpr int G = (T > B) ? (T / B) : 1;    // buckets covered by one step
  static constexpr int LPB = (T > B) ? B : T;        // lanes per bucket in a step
  static constexpr int SPB = (T > B) ? 1 : (B / T);  // steps per bucket
  static constexpr int TPL = 32 / T;                 // tags per lane (metadata)
  static constexpr u32 FILL_SHORTCUT = (3u * B) / 4u;
  static constexpr int PRE_SLOTS = B < 8 ? B : 8;    // slots of b_0 in the snapshot

  struct Hit {
    bool found;
    u64 idx, val;
  };
  struct Scan {
    bool found;
    u64 idx, val;      // where the key is (found)
    bool has_free;
    u64 fidx, fk, fv;  // free slot to claim and its observed content (tag in fk for META)
    bool stuck;        // a wait for a claimed slot's pair ran out
  };

  __device__ static __forceinline__ u32 nprobe(const TableView& tv) {
    if (SCHEME == SCHEME_DOUBLE) return tv.pmax;
    if (SCHEME == SCHEME_ICEBERG) return 3u;
    return tv.nb_mask == 0 ? 1u : 2u;
  }

  // Candidate bucket i of a key.  Iceberg (§2.2 front yard / backyard): i = 0
  // is the front-yard bucket by single hashing, i = 1, 2 the two backyard
  // choices; bucket counts are not powers of two there, so indices come from
  // multiply-high range reduction (h * n / 2^64, resp. / 2^32 on 32-bit halves).
  __device__ static __forceinline__ u64 bucket(const TableView& tv, u64 h1, u64 h2, u32 i) {
    if (SCHEME == SCHEME_DOUBLE) return (h1 + (u64)i * (h2 | 1ull)) & tv.nb_mask;
    if (SCHEME == SCHEME_ICEBERG) {
      if (i == 0) return __umul64hi(h1, tv.nb_front);
      const u64 c1 = ((h2 >> 32) * tv.nb_back) >> 32;
      if (i == 1) return tv.nb_front + c1;
      u64 c2 = ((h2 & 0xffffffffull) * tv.nb_back) >> 32;
      if (c2 == c1) c2 = (c1 + 1 == tv.nb_back) ? 0 : c1 + 1;
      return tv.nb_front + c2;
    }
    const u64 b0 = h1 & tv.nb_mask;
    if (i == 0) return b0;
    u64 b1 = h2 & tv.nb_mask;
    if (b1 == b0) b1 = (b0 + 1) & tv.nb_mask;
    return b1;
  }

  // ----------------------------------------------------------------------
  // Lane snapshots (one lane per op; see the file comment)
  // ----------------------------------------------------------------------
  // Summary of a snapshot's 32 tags, packed in one word (it stays live
  // across the candidate copy): bits 0-5 first tag equal to the key's (63:
  // none), 6-11 number of such tags, 12-17 first free tag (always 63 here:
  // see tag_free), 19 the bucket has an EMPTY slot, 20-25 occupancy as
  // FILL_SHORTCUT - 1 (below the 3/4 threshold) or FILL_SHORTCUT (not below).
  // Four tags per 64-bit word are tested at once: a field's bit 15 of
  // zero16(x) is set exactly when the field of x is zero.  EMPTY slots form
  // a suffix of a bucket (every claim takes the bucket's first free slot),
  // so tag 31 tells whether the bucket has one; and in a table that never saw
  // an erase (no tombstones: the only case the two-choice shortcut runs),
  // occupancy is below 3/4 exactly when tag 3B/4 - 1 is EMPTY.
  static constexpr u32 kTsNone = 63u;
  __device__ static __forceinline__ u64 zero16(u64 x) {
    constexpr u64 lo = 0x7fff7fff7fff7fffull, hi = 0x8000800080008000ull;
    return ~(((x & lo) + lo) | x) & hi;  // (f & 0x7fff) + 0x7fff <= 0xfffe: no carry between fields
  }
  __device__ static __forceinline__ u64 tag_word(const PreWarp* pw, int j, int i) {
    return reinterpret_cast<const u64*>(&pw->at(j, i >> 1))[i & 1];
  }
  __device__ static __forceinline__ u32 tag_scan(const PreWarp* pw, int j, u16 kt) {
    const u64 k4 = (u64)kt * 0x0001000100010001ull;
    u64 any = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) any |= zero16(tag_word(pw, j, i) ^ k4);
    u32 first = kTsNone, nmatch = 0;
    if (any) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const u64 me = zero16(tag_word(pw, j, i) ^ k4);
        nmatch += (u32)__popcll(me);
        if (first == kTsNone && me) first = 4u * i + (u32)(__ffsll((long long)me) >> 4) - 1u;
      }
    }
    const u16* t = reinterpret_cast<const u16*>(&pw->at(j, 0));
    const u32 empty = t[31] == TAG_EMPTY;
    const u32 occ = (t[FILL_SHORTCUT - 1] == TAG_EMPTY) ? FILL_SHORTCUT - 1 : FILL_SHORTCUT;
    return first | (nmatch << 6) | (kTsNone << 12) | (empty << 19) | (occ << 20);
  }

  // Metadata second copy of a wave: the first slot of bucket b whose tag
  // matches K, for op j.  Returns the snapshot's tag summary.
  __device__ static __forceinline__ u32 preload_candidate(const TableView& tv, u64 K, u64 b0, PreWarp* pw, int j) {
    const u32 ts = tag_scan(pw, j, key_tag(K));
    const u32 q = ts & 63u;
    if (q != kTsNone) {
      ptx::cp_async16(&pw->at(j, 4), tv.slots + b0 * 32 + (u64)q);
      pw->at(j, 5).key = b0 * 32 + (u64)q;
    } else {
      pw->at(j, 5).key = kNoCand;
    }
    return ts;
  }

  // ----------------------------------------------------------------------
  // Plain buckets (no metadata)
  // ----------------------------------------------------------------------
  // Probe cost of one step: LPB consecutive 16-byte slots of each active
  // bucket = LPB/2 DRAM sectors and ceil(LPB*16/128) cache lines.
  static constexpr u32 kStepSectors = LPB / 2;
  static constexpr u32 kStepLines = (LPB * 16 + 127) / 128;

  // Slot read of a probe step: from the snapshot when it holds the slot.
  __device__ static __forceinline__ void step_read(const TableView& tv, PreRef pre, bool first, int g,
                                                   int sl, u64 si, bool act, u64& k, u64& v) {
    k = KEY_RESV;
    v = 0;
    if (!act) return;
    if (pre.ok() && first && g == 0 && sl < PRE_SLOTS) {
      const Slot s = pre.slot(sl);
      k = s.key;
      v = s.val;
    } else {
      if (tv.phased)
        ptx::ld_slot_weak(tv.slots + si, k, v);
      else
        ptx::ld_slot(tv.slots + si, k, v);
    }
  }

  template <bool COUNT = false>
  __device__ static Hit find_plain(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                   PreRef pre = PreRef{nullptr, 0}, u32* sectors = nullptr, u32* lines = nullptr) {
    const u32 P = nprobe(tv);
    const int g = c.tl / LPB, j = c.tl % LPB;
    u32 occ0 = 0;
    for (u32 i = 0; i < P; i += G) {
      const bool act = (i + g) < P;
      const u64 b = bucket(tv, h1, h2, act ? i + g : i);
      bool ended = false;
#pragma unroll
      for (int s = 0; s < SPB; ++s) {
        const int sl = s * LPB + j;
        const u64 si = b * B + (u64)sl;
        u64 k, v;
        step_read(tv, pre, i == 0, g, sl, si, act, k, v);
        if (COUNT) {
          const u32 nact = (u32)((P - i) < (u32)G ? (P - i) : (u32)G);
          *sectors += nact * kStepSectors;
          *lines += nact * kStepLines;
        }
        const unsigned hit = c.ballot(k == K);
        if (hit) {
          const int src = __ffs(hit) - 1;
          return {true, c.shfl(si, src), c.shfl(v, src)};
        }
        if (SCHEME == SCHEME_P2 && G == 1 && i == 0) occ0 += __popc(c.ballot(k != KEY_EMPTY && k != KEY_TOMB));
        if (c.ballot(k == KEY_EMPTY)) {
          ended = true;
          break;
        }
      }
      if (SCHEME == SCHEME_DOUBLE) {
        if (ended) break;
      } else if (G == 1 && i == 0 && tv.shortcut && occ0 < FILL_SHORTCUT) {
        break;  // never erased and b_0 below 3/4: the key cannot be in b_1
      }
    }
    return {false, 0, 0};
  }

  __device__ static Scan scan_plain(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                    PreRef pre) {
    Scan r;
    r.stuck = false;
    r.found = false;
    r.has_free = false;
    r.idx = r.val = r.fidx = r.fk = r.fv = 0;
    const u32 P = nprobe(tv);
    const int g = c.tl / LPB, j = c.tl % LPB;
    if (SCHEME == SCHEME_DOUBLE) {
      for (u32 i = 0; i < P; i += G) {
        const bool act = (i + g) < P;
        const u64 b = bucket(tv, h1, h2, act ? i + g : i);
#pragma unroll
        for (int s = 0; s < SPB; ++s) {
          const int sl = s * LPB + j;
          const u64 si = b * B + (u64)sl;
          u64 k, v;
          step_read(tv, pre, i == 0, g, sl, si, act, k, v);
          const unsigned hit = c.ballot(k == K);
          if (hit) {
            const int src = __ffs(hit) - 1;
            r.found = true;
            r.idx = c.shfl(si, src);
            r.val = c.shfl(v, src);
            return r;
          }
          const unsigned fr = c.ballot(k == KEY_EMPTY || k == KEY_TOMB);
          if (fr && !r.has_free) {
            const int src = __ffs(fr) - 1;
            r.has_free = true;
            r.fidx = c.shfl(si, src);
            r.fk = c.shfl(k, src);
            r.fv = c.shfl(v, src);
          }
          if (c.ballot(k == KEY_EMPTY)) return r;
        }
      }
      return r;
    }
    // two-choice: occupancy and first free slot of each candidate bucket
    const u32 nbk = P;
    u32 occ[2] = {0, 0};
    bool hf[2] = {false, false};
    u64 fi[2] = {0, 0}, fk[2] = {0, 0}, fv[2] = {0, 0};
    bool decided0 = false;
    if (G == 1) {
      for (u32 bi = 0; bi < nbk; ++bi) {
        const u64 b = bucket(tv, h1, h2, bi);
#pragma unroll
        for (int s = 0; s < SPB; ++s) {
          const int sl = s * LPB + j;
          const u64 si = b * B + (u64)sl;
          u64 k, v;
          step_read(tv, pre, bi == 0, 0, sl, si, true, k, v);
          const unsigned hit = c.ballot(k == K);
          if (hit) {
            const int src = __ffs(hit) - 1;
            r.found = true;
            r.idx = c.shfl(si, src);
            r.val = c.shfl(v, src);
            return r;
          }
          const unsigned fr = c.ballot(k == KEY_EMPTY || k == KEY_TOMB);
          occ[bi] += (u32)(T - __popc(fr));
          if (fr && !hf[bi]) {
            const int src = __ffs(fr) - 1;
            hf[bi] = true;
            fi[bi] = c.shfl(si, src);
            fk[bi] = c.shfl(k, src);
            fv[bi] = c.shfl(v, src);
          }
          if (c.ballot(k == KEY_EMPTY)) break;  // the rest of the bucket is EMPTY
        }
        if (bi == 0 && tv.shortcut && occ[0] < FILL_SHORTCUT) {
          decided0 = true;
          break;
        }
      }
    } else {
      const bool act = g < (int)nbk;
      const u64 b = bucket(tv, h1, h2, act ? (u32)g : 0u);
      const u64 si = b * B + (u64)j;
      u64 k, v;
      step_read(tv, pre, true, g, j, si, act, k, v);
      const unsigned hit = c.ballot(k == K);
      if (hit) {
        const int src = __ffs(hit) - 1;
        r.found = true;
        r.idx = c.shfl(si, src);
        r.val = c.shfl(v, src);
        return r;
      }
      const unsigned fr = c.ballot(act && (k == KEY_EMPTY || k == KEY_TOMB));
#pragma unroll
      for (int gg = 0; gg < 2; ++gg) {
        constexpr unsigned kBucketBits = (B >= 32) ? 0xffffffffu : ((1u << (B & 31)) - 1u);
        const unsigned gm = kBucketBits << ((gg * B) & 31);
        occ[gg] = (u32)(B - __popc(fr & gm));
        if (fr & gm) {
          const int src = __ffs(fr & gm) - 1;
          hf[gg] = true;
          fi[gg] = c.shfl(si, src);
          fk[gg] = c.shfl(k, src);
          fv[gg] = c.shfl(v, src);
        }
      }
      if (nbk == 1) decided0 = true;
    }
    int ch = 0;
    if (!decided0 && nbk == 2) {
      ch = (occ[0] < FILL_SHORTCUT) ? 0 : (occ[1] < occ[0] ? 1 : 0);
      if (!hf[ch]) ch = 1 - ch;
    }
    if (hf[ch]) {
      r.has_free = true;
      r.fidx = fi[ch];
      r.fk = fk[ch];
      r.fv = fv[ch];
    }
    return r;
  }

  // ----------------------------------------------------------------------
  // Metadata buckets: 32 slots, 64-byte tag line, TPL tags per lane
  // ----------------------------------------------------------------------
  __device__ static __forceinline__ void tag_masks(const TableView& tv, const TileCtx<T>& c, u64 b, u16 kt,
                                                   PreRef pre, unsigned& mm, unsigned& me,
                                                   unsigned& mf) {
    const u16* tp = tv.tags + b * 32 + (u64)(c.tl * TPL);
    unsigned lm = 0, le = 0, lf = 0;
    u16 t[TPL];
    if (pre.ok()) {
      const int q0 = c.tl * TPL;  // TPL tags inside one row of eight
      const u16* sp = pre.tagrow(q0 >> 3) + (q0 & 7);
#pragma unroll
      for (int q = 0; q < TPL; ++q) t[q] = sp[q];
    } else if (TPL == 8) {
      u64 a0, a1;
      if (tv.phased)
        ptx::ld_tags16_weak(tp, a0, a1);
      else
        ptx::ld_tags16(tp, a0, a1);
#pragma unroll
      for (int q = 0; q < TPL; ++q) t[q] = (u16)(((q < 4) ? (a0 >> (16 * q)) : (a1 >> (16 * (q - 4)))) & 0xffffu);
    } else if (TPL == 4) {
      const u64 a = ptx::ld_tags8(tp);
#pragma unroll
      for (int q = 0; q < TPL; ++q) t[q] = (u16)((a >> (16 * q)) & 0xffffu);
    } else if (TPL == 2) {
      const u32 a = ptx::ld_tags4(tp);
#pragma unroll
      for (int q = 0; q < TPL; ++q) t[q] = (u16)((a >> (16 * q)) & 0xffffu);
    } else {
      t[0] = ptx::ld_tags2(tp);
    }
#pragma unroll
    for (int q = 0; q < TPL; ++q) {
      lm |= (unsigned)(t[q] == kt) << q;
      le |= (unsigned)(t[q] == TAG_EMPTY) << q;
      lf |= (unsigned)(t[q] < 2) << q;
    }
    const int sh = c.tl * TPL;
    mm = __reduce_or_sync(c.mask, lm << sh);
    me = __reduce_or_sync(c.mask, le << sh);
    mf = __reduce_or_sync(c.mask, lf << sh);
  }

  // One slot read by the leader lane, broadcast to the tile (tile-uniform).
  __device__ static __forceinline__ void read_pair(const TableView& tv, const TileCtx<T>& c, u64 si, u64& k,
                                                   u64& v) {
    k = 0;
    v = 0;
    if (c.tl == 0) {
      if (tv.phased)
        ptx::ld_slot_weak(tv.slots + si, k, v);
      else
        ptx::ld_slot(tv.slots + si, k, v);
    }
    k = c.shfl(k, 0);
    v = c.shfl(v, 0);
  }

  // Reads the candidate slots of a tag match mask; true if one holds K.
  // The leader lane reads each candidate and broadcasts the pair, so every
  // lane of the tile takes the same branch even while another tile rewrites
  // the slot (separate per-lane reads could disagree and split the tile).
  // The snapshot's candidate (same shared value on every lane) stands in for
  // the first read when it is that slot.  With WAIT (lock-free inserts, where
  // no erase runs concurrently) a slot whose tag is claimed but whose pair is
  // not stored yet (key EMPTY/TOMB) is re-read until the claimer's pair store
  // lands, so a same-key inserter cannot miss a copy being written.
  // *stuck reports a wait that ran out.
  template <bool WAIT = false, bool COUNT = false>
  __device__ static __forceinline__ bool verify(const TableView& tv, const TileCtx<T>& c, u64 b, unsigned mm,
                                                u64 K, PreRef pre, u64& idx, u64& val,
                                                bool* stuck = nullptr, u32* nread = nullptr) {
    while (mm) {
      const int q = __ffs(mm) - 1;
      mm &= mm - 1;
      const u64 si = b * 32 + (u64)q;
      u64 k, v;
      if (pre.ok() && pre.cand_idx() == si) {
        const Slot s = pre.cand();
        k = s.key;
        v = s.val;
      } else {
        read_pair(tv, c, si, k, v);
      }
      if (COUNT) ++*nread;
      if (WAIT) {
        for (u32 n = 0; k == KEY_EMPTY || k == KEY_TOMB; ++n) {
          if (n >= tv.spin_limit) {
            *stuck = true;
            break;
          }
          __nanosleep(64);
          read_pair(tv, c, si, k, v);
        }
      }
      if (k == K) {
        idx = si;
        val = v;
        return true;
      }
    }
    return false;
  }

  // Probe cost with metadata: a tag line read is 64 B (2 sectors, 1 line);
  // each candidate slot read is one 32-byte sector of one line.
  template <bool COUNT = false>
  __device__ static Hit find_meta(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                  PreRef pre = PreRef{nullptr, 0}, u32* sectors = nullptr, u32* lines = nullptr) {
    const u32 P = nprobe(tv);
    const u16 kt = key_tag(K);
    for (u32 i = 0; i < P; ++i) {
      const u64 b = bucket(tv, h1, h2, i);
      const PreRef p = (i == 0) ? pre : no_pre();
      unsigned mm, me, mf;
      tag_masks(tv, c, b, kt, p, mm, me, mf);
      u64 idx, val;
      u32 nc = 0;
      const bool got = verify<false, COUNT>(tv, c, b, mm, K, p, idx, val, nullptr, &nc);
      if (COUNT) {
        *sectors += 2 + nc;
        *lines += 1 + nc;
      }
      if (got) return {true, idx, val};
      if (SCHEME == SCHEME_DOUBLE) {
        if (me) break;
      } else if (SCHEME == SCHEME_ICEBERG) {
        if (i == 0 && me) break;  // a front bucket with an EMPTY slot never overflowed
      } else if (i == 0 && tv.shortcut && (u32)(32 - __popc(mf)) < FILL_SHORTCUT) {
        break;
      }
    }
    return {false, 0, 0};
  }

  template <bool WAIT = false>
  __device__ static Scan scan_meta(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                   PreRef pre) {
    Scan r;
    r.stuck = false;
    r.found = false;
    r.has_free = false;
    r.idx = r.val = r.fidx = r.fk = r.fv = 0;
    const u32 P = nprobe(tv);
    const u16 kt = key_tag(K);
    if (SCHEME == SCHEME_DOUBLE) {
      for (u32 i = 0; i < P; ++i) {
        const u64 b = bucket(tv, h1, h2, i);
        const PreRef p = (i == 0) ? pre : no_pre();
        unsigned mm, me, mf;
        tag_masks(tv, c, b, kt, p, mm, me, mf);
        if (verify<WAIT>(tv, c, b, mm, K, p, r.idx, r.val, &r.stuck)) {
          r.found = true;
          return r;
        }
        if (r.stuck) return r;
        if (mf && !r.has_free) {
          const int q = __ffs(mf) - 1;
          r.has_free = true;
          r.fidx = b * 32 + (u64)q;
          r.fk = ((me >> q) & 1u) ? TAG_EMPTY : TAG_TOMB;
        }
        if (me) return r;
      }
      return r;
    }
    if (SCHEME == SCHEME_ICEBERG) {
      // Front bucket first; its first free slot (EMPTY or TOMB) wins.  A
      // front bucket holding an EMPTY slot was never full, so the key cannot
      // be in the backyard.  Otherwise both backyard buckets are searched and,
      // with no free front slot, the key goes to the less loaded one (ties to
      // the first), or to the other one when that is full.
      u32 occ[3] = {0, 0, 0};
      bool hf[3] = {false, false, false};
      u64 fi[3] = {0, 0, 0}, ft[3] = {0, 0, 0};
      u32 nread = 0;
      for (u32 bi = 0; bi < 3; ++bi) {
        const u64 b = bucket(tv, h1, h2, bi);
        const PreRef p = (bi == 0) ? pre : no_pre();
        unsigned mm, me, mf;
        tag_masks(tv, c, b, kt, p, mm, me, mf);
        if (verify<WAIT>(tv, c, b, mm, K, p, r.idx, r.val, &r.stuck)) {
          r.found = true;
          return r;
        }
        if (r.stuck) return r;
        occ[bi] = (u32)(32 - __popc(mf));
        if (mf) {
          const int q = __ffs(mf) - 1;
          hf[bi] = true;
          fi[bi] = b * 32 + (u64)q;
          ft[bi] = ((me >> q) & 1u) ? TAG_EMPTY : TAG_TOMB;
        }
        nread = bi + 1;
        if (bi == 0 && me) break;
      }
      int ch = -1;
      if (hf[0]) {
        ch = 0;
      } else if (nread == 3) {
        ch = (occ[2] < occ[1]) ? 2 : 1;
        if (!hf[ch]) ch = 3 - ch;
        if (!hf[ch]) ch = -1;
      }
      if (ch >= 0) {
        r.has_free = true;
        r.fidx = fi[ch];
        r.fk = ft[ch];
      }
      return r;
    }
    u32 occ[2] = {0, 0};
    bool hf[2] = {false, false};
    u64 fi[2] = {0, 0}, ft[2] = {0, 0};
    bool decided0 = (P == 1);
    for (u32 bi = 0; bi < P; ++bi) {
      const u64 b = bucket(tv, h1, h2, bi);
      const PreRef p = (bi == 0) ? pre : no_pre();
      unsigned mm, me, mf;
      tag_masks(tv, c, b, kt, p, mm, me, mf);
      if (verify<WAIT>(tv, c, b, mm, K, p, r.idx, r.val, &r.stuck)) {
        r.found = true;
        return r;
      }
      if (r.stuck) return r;
      occ[bi] = (u32)(32 - __popc(mf));
      if (mf) {
        const int q = __ffs(mf) - 1;
        hf[bi] = true;
        fi[bi] = b * 32 + (u64)q;
        ft[bi] = ((me >> q) & 1u) ? TAG_EMPTY : TAG_TOMB;
      }
      if (bi == 0 && tv.shortcut && occ[0] < FILL_SHORTCUT) {
        decided0 = true;
        break;
      }
    }
    int ch = 0;
    if (!decided0) {
      ch = (occ[0] < FILL_SHORTCUT) ? 0 : (occ[1] < occ[0] ? 1 : 0);
      if (!hf[ch]) ch = 1 - ch;
    }
    if (hf[ch]) {
      r.has_free = true;
      r.fidx = fi[ch];
      r.fk = ft[ch];
    }
    return r;
  }

  // ----------------------------------------------------------------------
  // Shared pieces
  // ----------------------------------------------------------------------
  __device__ static __forceinline__ Hit find(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                             PreRef pre) {
    if constexpr (META) return find_meta(tv, c, K, h1, h2, pre);
    else return find_plain(tv, c, K, h1, h2, pre);
  }
  template <bool WAIT = false>
  __device__ static __forceinline__ Scan scan(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                              PreRef pre) {
    if constexpr (META) return scan_meta<WAIT>(tv, c, K, h1, h2, pre);
    else return scan_plain(tv, c, K, h1, h2, pre);
  }

  // Claim the scanned free slot for (K, V).  Leader lane writes; all learn the outcome.
  __device__ static __forceinline__ bool claim(const TableView& tv, const TileCtx<T>& c, const Scan& r, u64 K,
                                               u64 V) {
    int ok = 0;
    if (c.tl == 0) {
      if (META) {
        const u16 expect = (u16)r.fk;
        if (ptx::cas_tag(tv.tags + r.fidx, expect, key_tag(K)) == expect) {
          ptx::st_slot_relaxed(tv.slots + r.fidx, K, V);
          ok = 1;
        }
      } else {
        ok = ptx::cas_slot(tv.slots + r.fidx, r.fk, r.fv, K, V) ? 1 : 0;
      }
    }
    return c.shfl(ok, 0) != 0;
  }

  // Upsert callback on a present key (leader lane only).
  __device__ static __forceinline__ void apply(const TableView& tv, u64 idx, int op, u64 V) {
    u64* vp = &tv.slots[idx].val;
    if (op == OP_ADD)
      ptx::red_add_u64(vp, V);
    else if (op == OP_MAX)
      ptx::red_max_u64(vp, V);
    else if (op == OP_REPLACE)
      ptx::st_u64_relaxed(vp, V);
  }

  // One test-and-test-and-set attempt on the lock bit of bucket b by the
  // leader lane; the outcome is returned on every lane of the tile.
  __device__ static __forceinline__ bool try_lock(const TableView& tv, const TileCtx<T>& c, u64 b) {
    int ok = 0;
    if (c.tl == 0) {
      u32* w = tv.locks + (b >> 5);
      const u32 bit = 1u << (b & 31);
      ok = (!(ptx::ld_u32_relaxed(w) & bit) && !(ptx::atom_or_acquire(w, bit) & bit)) ? 1 : 0;
    }
    ok = c.shfl(ok, 0);
    __syncwarp(c.mask);
    return ok != 0;
  }

  // Back-off between lock attempts (leader sleeps, the tile waits for it).
  __device__ static __forceinline__ void backoff(const TileCtx<T>& c, u32& ns) {
    if (c.tl == 0) {
      ns = ns ? (ns < 1024u ? ns * 2u : 1024u) : 32u;
      __nanosleep(ns);
    }
    __syncwarp(c.mask);
  }

  // Unlock; with release semantics only when the holder claimed a slot (the
  // next holder must see it), relaxed when it wrote nothing under the lock.
  __device__ static __forceinline__ void unlock(const TableView& tv, const TileCtx<T>& c, u64 b, bool wrote = true) {
    __syncwarp(c.mask);
    if (c.tl == 0) {
      if (wrote)
        ptx::red_and_release(tv.locks + (b >> 5), ~(1u << (b & 31)));
      else
        ptx::red_and_relaxed(tv.locks + (b >> 5), ~(1u << (b & 31)));
    }
  }

  // One lock attempt by a single lane (no test first: one round trip).  A
  // lane that finds the bit set owns nothing and must not unlock.
  __device__ static __forceinline__ bool lane_lock(const TableView& tv, u64 b) {
    const u32 bit = 1u << (b & 31);
    return !(ptx::atom_or_acquire(tv.locks + (b >> 5), bit) & bit);
  }
  __device__ static __forceinline__ void lane_unlock(const TableView& tv, u64 b, bool wrote) {
    if (wrote)
      ptx::red_and_release(tv.locks + (b >> 5), ~(1u << (b & 31)));
    else
      ptx::red_and_relaxed(tv.locks + (b >> 5), ~(1u << (b & 31)));
  }

  // Two-choice placement (§4.2) from both buckets' loads and first free
  // slots: b_0 while it is below 3/4, else the less loaded bucket (ties to
  // b_0); the other bucket when the chosen one has no free slot.  Returns
  // 0 / 1, or -1 when both are full.  have1 = false: only b_0 was read (the
  // shortcut proved the key absent from b_1, or there is one bucket).
  __device__ static __forceinline__ int p2_choice(u32 occ0, bool free0, u32 occ1, bool free1, bool have1) {
    if (!have1) return free0 ? 0 : -1;
    int ch = (occ0 < FILL_SHORTCUT) ? 0 : (occ1 < occ0 ? 1 : 0);
    if (ch == 0 && !free0) ch = 1;
    else if (ch == 1 && !free1) ch = 0;
    return (ch == 0 ? free0 : free1) ? ch : -1;
  }

  // ----------------------------------------------------------------------
  // Operations (tile-uniform control flow; results valid on every lane).
  // pre: the op's snapshot of b_0, or null.
  // ----------------------------------------------------------------------
  __device__ static u8 do_query(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2, PreRef pre,
                                u64& out) {
    out = 0;
    if (is_sentinel(K)) return ST_BADKEY;
    const Hit h = find(tv, c, K, h1, h2, pre);
    if (!h.found) return ST_MISS;
    out = h.val;
    return ST_FOUND;
  }

  // Probe-count instrumentation (§5 "probe count"): the cost a query of K
  // pays on the current table, as (cache lines << 32) | DRAM sectors.
  __device__ static u8 do_probe(const TableView& tv, const TileCtx<T>& c, u64 K, u64& out) {
    out = 0;
    if (is_sentinel(K)) return ST_BADKEY;
    const u64 h1 = fmix64(K ^ tv.seed1), h2 = fmix64(K ^ tv.seed2);
    u32 sec = 0, lin = 0;
    Hit h;
    if constexpr (META)
      h = find_meta<true>(tv, c, K, h1, h2, no_pre(), &sec, &lin);
    else
      h = find_plain<true>(tv, c, K, h1, h2, no_pre(), &sec, &lin);
    out = ((u64)lin << 32) | (u64)sec;
    return h.found ? ST_FOUND : ST_MISS;
  }

  // LOCKFREE: the caller guarantees that no erase runs in the same launch (a
  // plain insert / upsert call is one phase).
  template <bool LOCKFREE>
  // Writes read the table through L2 even in bulk-synchronous mode: the
  // call's other inserts write the slots they probe, and a lost claim must
  // see the winner (weak, L1-cacheable loads could return the stale line on
  // every retry).  `tv` keeps the mode for the lock decisions.
  __device__ static u8 do_upsert(const TableView& tv_in, const TileCtx<T>& c, u64 K, u64 h1, u64 h2, u64 V, int op,
                                 PreRef pre, int& dcount) {
    TableView tv = tv_in;
    const bool phased = tv.phased != 0;
    tv.phased = 0;
    if (is_sentinel(K)) return ST_BADKEY;
    if (LOCKFREE && SCHEME == SCHEME_DOUBLE) {
      // Without erases, free slots only disappear, so every inserter of K
      // targets the first free slot of K's probe sequence: the CAS winner
      // places K and a loser's rescan finds it (with metadata, verify waits
      // out a claimed-but-unwritten slot).  No lock is needed; the lock of
      // §4.1 is for inserts racing erases (mixed batches) and for two-choice
      // placement, whose choice depends on the moment's bucket loads.  The
      // first scan may use the snapshot: a stale free slot only makes the
      // CAS fail, and the rescans read afresh.
      for (int attempt = 0; attempt < 256; ++attempt) {
        const Scan r = scan<true>(tv, c, K, h1, h2, attempt == 0 ? pre : no_pre());
        if (r.stuck) return ST_TIMEOUT;
        if (r.found) {
          if (c.tl == 0) apply(tv, r.idx, op, V);
          return ST_FOUND;
        }
        if (!r.has_free) {
          if (attempt == 0 && pre.ok()) continue;  // confirm a full sequence on fresh data
          return ST_FULL;
        }
        if (claim(tv, c, r, K, V)) {
          ++dcount;
          return ST_INSERTED;
        }
      }
      return ST_TIMEOUT;
    }
    const Hit h = find(tv, c, K, h1, h2, pre);
    if (h.found) {
      if (c.tl == 0) apply(tv, h.idx, op, V);
      return ST_FOUND;
    }
    // Absent: take the primary bucket's lock so that inserters of this key
    // agree on one slot (§4.1).  While another tile holds it -- often one
    // inserting this very key -- probe again lock-free: once the key is
    // present its slot never moves, so the update needs no lock.  This keeps
    // a batch's many copies of a hot key from queueing on one lock bit.
    const u64 b0 = bucket(tv, h1, h2, 0);
    // bulk-synchronous mode: distinct keys per call, nothing to serialise
    for (u32 tries = 0, ns = 0; !phased;) {
      if (try_lock(tv, c, b0)) break;
      const Hit again = find(tv, c, K, h1, h2, no_pre());
      if (again.found) {
        if (c.tl == 0) apply(tv, again.idx, op, V);
        return ST_FOUND;
      }
      if (++tries >= tv.spin_limit) return ST_TIMEOUT;
      backoff(c, ns);
    }
    u8 st = ST_TIMEOUT;
    for (int attempt = 0; attempt < 256; ++attempt) {
      const Scan r = scan(tv, c, K, h1, h2, no_pre());
      if (r.found) {
        if (c.tl == 0) apply(tv, r.idx, op, V);
        st = ST_FOUND;
        break;
      }
      if (!r.has_free) {
        st = ST_FULL;
        break;
      }
      if (claim(tv, c, r, K, V)) {
        st = ST_INSERTED;
        ++dcount;
        break;
      }
    }
    if (!phased) unlock(tv, c, b0, st == ST_INSERTED);
    return st;
  }

  // TOMB_RELEASE: publish the TOMB tag with release semantics, so that a
  // claimer of the freed tag in the same launch finds the pair's CAS ordered
  // before its own pair store.  An erase-only launch claims nothing (calls on
  // a table are ordered, and batched phases run their op kinds as separate,
  // stream-ordered kernels), so there a relaxed store suffices.
  template <bool TOMB_RELEASE = true>
  __device__ static u8 do_erase(const TableView& tv_in, const TileCtx<T>& c, u64 K, u64 h1, u64 h2, PreRef pre,
                                u64& out, int& dcount) {
    TableView tv = tv_in;  // through L2, as for do_upsert
    tv.phased = 0;
    out = 0;
    if (is_sentinel(K)) return ST_BADKEY;
    for (int attempt = 0; attempt < 256; ++attempt) {
      const Hit h = find(tv, c, K, h1, h2, attempt == 0 ? pre : no_pre());
      if (!h.found) return ST_MISS;
      int ok = 0;
      if (c.tl == 0) {
        ok = ptx::cas_slot(tv.slots + h.idx, K, h.val, KEY_TOMB, 0) ? 1 : 0;
        if (ok && META) {
          if (TOMB_RELEASE)
            ptx::st_tag_release(tv.tags + h.idx, TAG_TOMB);
          else
            ptx::st_tag_relaxed(tv.tags + h.idx, TAG_TOMB);
        }
      }
      if (c.shfl(ok, 0)) {
        out = h.val;
        --dcount;
        return ST_FOUND;
      }
    }
    return ST_TIMEOUT;
  }

  // One op of the mixed codes (queries, upserts under the locked path, erases).
  __device__ static __forceinline__ u8 do_mixed(const TableView& tv, const TileCtx<T>& c, u8 code, u64 K, u64 h1,
                                                u64 h2, u64 V, PreRef pre, u64& out, int& dcount) {
    out = 0;
    switch (code) {
      case MX_QUERY: return do_query(tv, c, K, h1, h2, pre, out);
      case MX_INSERT: return do_upsert<false>(tv, c, K, h1, h2, V, OP_INSERT, pre, dcount);
      case MX_ADD: return do_upsert<false>(tv, c, K, h1, h2, V, OP_ADD, pre, dcount);
      case MX_MAX: return do_upsert<false>(tv, c, K, h1, h2, V, OP_MAX, pre, dcount);
      case MX_REPLACE: return do_upsert<false>(tv, c, K, h1, h2, V, OP_REPLACE, pre, dcount);
      case MX_ERASE: return do_erase(tv, c, K, h1, h2, pre, out, dcount);
      default: return ST_BADKEY;
    }
  }

  // ----------------------------------------------------------------------
  // Lane fast path: one lane settles its own op from the snapshot alone --
  // a hit, a miss proven by an EMPTY slot (or the two-choice shortcut), or
  // a claim / erase by one 128-bit CAS.  Returns true when settled.
  // *fresh becomes false when the lane tried a CAS that failed: the table
  // moved on, so the tile path must not reuse the snapshot.
  // ----------------------------------------------------------------------
  struct Snap {
    int hit;         // slot of K in the snapshot, -1 if none
    int ffree;       // first free slot (plain) / first free tag (metadata), -1 if none
    bool ffree_empty;
    bool empty;      // an EMPTY slot / tag seen: no key sits past it in b_0
    u32 occ;         // occupied slots of b_0 (exact when `empty`)
    bool unsure;     // metadata: a tag match that the snapshot cannot settle
  };

  // ts: the tag summary of the snapshot (metadata tables; see tag_scan).
  __device__ static __forceinline__ Snap snap_of(PreRef p, u64 K, u32 ts) {
    Snap sn;
    sn.hit = -1;
    sn.ffree = -1;
    sn.ffree_empty = false;
    sn.empty = false;
    sn.occ = 0;
    sn.unsure = false;
    if (!META) {
#pragma unroll
      for (int s = 0; s < PRE_SLOTS; ++s) {
        const u64 k = p.slot(s).key;
        if (k == K && sn.hit < 0) sn.hit = s;
        const bool fr = (k == KEY_EMPTY || k == KEY_TOMB);
        if (fr && sn.ffree < 0) {
          sn.ffree = s;
          sn.ffree_empty = (k == KEY_EMPTY);
        }
        sn.empty |= (k == KEY_EMPTY);
        sn.occ += fr ? 0u : 1u;
      }
    } else {
      const u32 nmatch = (ts >> 6) & 63u, ff = (ts >> 12) & 63u;
      sn.ffree = ff == kTsNone ? -1 : (int)ff;
      sn.ffree_empty = (ts >> 18) & 1u;
      sn.empty = (ts >> 19) & 1u;
      sn.occ = (ts >> 20) & 63u;
      if (nmatch > 0) {
        const u64 ck = p.cand().key;
        if (ck == K)
          sn.hit = 0;  // the candidate pair is K's
        else if (nmatch > 1 || ck == KEY_EMPTY || ck == KEY_TOMB)
          sn.unsure = true;  // more candidates, or a claimed slot not written yet
      }
    }
    return sn;
  }

  // The free tags of a metadata snapshot, for a lane that may claim a slot
  // in it (the tag summary leaves them out): the first free tag (EMPTY or
  // TOMB), whether it is EMPTY, and the exact occupancy.
  __device__ static __forceinline__ void tag_free(PreRef p, Snap& sn) {
    u32 ffree = kTsNone, nfree = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const u64 mf = zero16(tag_word(p.w, p.j, i) & 0xfffefffefffefffeull);  // tag < 2
      nfree += (u32)__popcll(mf);
      if (ffree == kTsNone && mf) ffree = 4u * i + (u32)(__ffsll((long long)mf) >> 4) - 1u;
    }
    sn.occ = 32u - nfree;
    sn.ffree = ffree == kTsNone ? -1 : (int)ffree;
    sn.ffree_empty = ffree != kTsNone && p.tagrow(0)[ffree] == TAG_EMPTY;
  }

  // Slot index and pair of the snapshot hit.
  __device__ static __forceinline__ void hit_pair(PreRef p, const Snap& sn, u64 b0, u64& idx, u64& val) {
    if (META) {
      idx = p.cand_idx();
      val = p.cand().val;
    } else {
      idx = b0 * B + (u64)sn.hit;
      val = p.slot(sn.hit).val;
    }
  }

  // ----------------------------------------------------------------------
  // Lane waves: the lane owning an op settles it bucket by bucket from
  // snapshots of the probe sequence (wave w holds bucket w of every op still
  // open), the same rules as the tile probe.  lane_wave returns 1 when the op
  // is settled, 0 to go on to the next wave, -1 to hand it to the tile path
  // (more than the snapshot can tell, or a lost CAS), and -2 when an upsert
  // probed without the lock has proven its key absent: it must now take b_0's
  // lock and read again before it may insert.
  // ----------------------------------------------------------------------
  // LW_INSERT_FREE: lock-free first-free insert (double hashing, no erase
  // in the launch).  LW_INSERT_LOCKED: the lane holds b_0's lock (or the
  // launch is bulk-synchronous), so its snapshots are authoritative for K.
  enum { LW_QUERY = 0, LW_INSERT_FREE = 1, LW_UPDATE_ONLY = 2, LW_ERASE = 3, LW_INSERT_LOCKED = 4 };
  struct LaneState {
    bool ff_set;  // first free slot of the probe sequence seen so far
    u64 ff_idx, ff_k, ff_v;
    u32 occ0;     // two-choice: load of b_0 (wave 0)
    u32 occ1;     // iceberg: load and first free tag of the first backyard bucket (wave 1)
    bool f1_set;
    u64 f1_idx, f1_k;
    u64 f1_v;     // two-choice by lines: observed value of b_1's first free slot
    u32 cur_occ;  // two-choice by lines: occupied slots of the current bucket so far
    u32 next_w;   // two-choice by lines: the wave to run next
    u32 tsum;     // metadata: tag summary of the current snapshot (tag_scan)
  };

  // Two-choice tables whose buckets are wider than a snapshot line: wave w
  // reads line w % L of candidate bucket w / L (L = B / 8 lines per bucket),
  // so a lane stops at the key or at the first EMPTY slot instead of reading
  // whole buckets.  Occupancy and first free slot accumulate per bucket for
  // the placement rule.  Streaming lanes only (lanes sit at different waves).
  static constexpr bool kLines = (SCHEME == SCHEME_P2) && !META && PRE_SLOTS < B;
  static constexpr u32 kLinesPerBucket = (u32)(B / PRE_SLOTS);
  __device__ static __forceinline__ u32 wave_bucket(u32 w) { return kLines ? w / kLinesPerBucket : w; }
  __device__ static __forceinline__ u32 wave_line(u32 w) { return kLines ? w % kLinesPerBucket : 0u; }

  __device__ static __forceinline__ int lane_wave_lines(const TableView& tv, PreRef p, u64 K, u64 V, int op, int opk,
                                                        u32 w, u64 bw, LaneState& ls, u64& out, u8& st,
                                                        int& dcount, bool& fresh) {
    const u32 c = w / kLinesPerBucket, l = w % kLinesPerBucket;
    const u64 line0 = bw * B + (u64)l * PRE_SLOTS;
    const Snap sn = snap_of(p, K, 0u);
    if (sn.hit >= 0) {
      const u64 idx = line0 + (u64)sn.hit;
      const u64 v = p.slot(sn.hit).val;
      if (opk == LW_QUERY) {
        out = v;
        st = ST_FOUND;
        return 1;
      }
      if (opk != LW_ERASE) {
        apply(tv, idx, op, V);
        st = ST_FOUND;
        return 1;
      }
      if (!ptx::cas_slot(tv.slots + idx, K, v, KEY_TOMB, 0)) {
        fresh = false;
        return -1;
      }
      out = v;
      --dcount;
      st = ST_FOUND;
      return 1;
    }
    if (l == 0) ls.cur_occ = 0;
    ls.cur_occ += sn.occ;
    if (sn.ffree >= 0) {
      const Slot o = p.slot(sn.ffree);
      if (c == 0 && !ls.ff_set) {
        ls.ff_set = true;
        ls.ff_idx = line0 + (u64)sn.ffree;
        ls.ff_k = o.key;
        ls.ff_v = o.val;
      } else if (c == 1 && !ls.f1_set) {
        ls.f1_set = true;
        ls.f1_idx = line0 + (u64)sn.ffree;
        ls.f1_k = o.key;
        ls.f1_v = o.val;
      }
    }
    if (!sn.empty && l + 1 < kLinesPerBucket) {  // the bucket goes on
      ls.next_w = w + 1;
      return 0;
    }
    if (c == 0) {  // b_0 done (an EMPTY slot ends a bucket: EMPTY slots are a suffix)
      ls.occ0 = ls.cur_occ;
      if (!(nprobe(tv) == 1 || (tv.shortcut && ls.occ0 < FILL_SHORTCUT))) {
        ls.next_w = kLinesPerBucket;  // b_1, line 0
        return 0;
      }
    }
    // K is in neither bucket
    if (opk == LW_QUERY || opk == LW_ERASE) {
      out = 0;
      st = ST_MISS;
      return 1;
    }
    if (opk != LW_INSERT_LOCKED) return -2;  // absent, and this op holds no lock
    const int ch = p2_choice(ls.occ0, ls.ff_set, ls.cur_occ, ls.f1_set, c == 1);
    if (ch < 0) {
      st = ST_FULL;
      return 1;
    }
    const bool ok = ch == 0 ? ptx::cas_slot(tv.slots + ls.ff_idx, ls.ff_k, ls.ff_v, K, V)
                            : ptx::cas_slot(tv.slots + ls.f1_idx, ls.f1_k, ls.f1_v, K, V);
    if (!ok) {
      fresh = false;
      return -1;
    }
    ++dcount;
    st = ST_INSERTED;
    return 1;
  }

  __device__ static __forceinline__ int lane_wave(const TableView& tv, PreRef p, u64 K, u64 V, int op, int opk,
                                                  u32 w, u64 bw, LaneState& ls, u64& out, u8& st, int& dcount,
                                                  bool& fresh, bool tomb_release) {
    Snap sn = snap_of(p, K, ls.tsum);
    if (sn.unsure) return -1;
    if (sn.hit >= 0) {
      u64 idx, v;
      hit_pair(p, sn, bw, idx, v);
      if (opk == LW_QUERY) {
        out = v;
        st = ST_FOUND;
        return 1;
      }
      if (opk != LW_ERASE) {
        apply(tv, idx, op, V);
        st = ST_FOUND;
        return 1;
      }
      if (!ptx::cas_slot(tv.slots + idx, K, v, KEY_TOMB, 0)) {
        fresh = false;
        return -1;
      }
      if (META) {  // see do_erase
        if (tomb_release)
          ptx::st_tag_release(tv.tags + idx, TAG_TOMB);
        else
          ptx::st_tag_relaxed(tv.tags + idx, TAG_TOMB);
      }
      out = v;
      --dcount;
      st = ST_FOUND;
      return 1;
    }
    // no K in what the snapshot shows; with plain buckets wider than the
    // snapshot an EMPTY slot in it still settles the whole bucket (EMPTY
    // slots form a suffix of the bucket)
    if (!META && PRE_SLOTS < B && !sn.empty) return -1;
    const bool ins = (opk == LW_INSERT_FREE || opk == LW_INSERT_LOCKED);
    if (META && ins) tag_free(p, sn);  // K is not here: this lane may claim a slot
    if (SCHEME == SCHEME_P2 && w == 0) ls.occ0 = sn.occ;
    if (SCHEME == SCHEME_ICEBERG && w == 1) {
      ls.occ1 = sn.occ;
      ls.f1_set = sn.ffree >= 0;
      ls.f1_idx = bw * 32 + (u64)(sn.ffree >= 0 ? sn.ffree : 0);
      ls.f1_k = sn.ffree_empty ? TAG_EMPTY : TAG_TOMB;
    }
    if (ins && !ls.ff_set && sn.ffree >= 0 && (SCHEME == SCHEME_DOUBLE || w == 0)) {
      ls.ff_set = true;
      if (META) {
        ls.ff_idx = bw * 32 + (u64)sn.ffree;
        ls.ff_k = sn.ffree_empty ? TAG_EMPTY : TAG_TOMB;
      } else {
        const Slot o = p.slot(sn.ffree);
        ls.ff_idx = bw * B + (u64)sn.ffree;
        ls.ff_k = o.key;
        ls.ff_v = o.val;
      }
    }
    const u32 P = nprobe(tv);
    bool ends;
    if (SCHEME == SCHEME_DOUBLE)
      ends = sn.empty || w + 1 >= P;
    else if (SCHEME == SCHEME_ICEBERG)
      ends = (w == 0 && sn.empty) || w + 1 >= P;
    else
      ends = (w + 1 >= P) || (w == 0 && tv.shortcut && sn.occ < FILL_SHORTCUT);
    if (!ends) return 0;
    if (opk == LW_QUERY || opk == LW_ERASE) {
      if (SCHEME == SCHEME_DOUBLE && !sn.empty) return -1;  // probe cap reached: let the tiles confirm
      out = 0;
      st = ST_MISS;
      return 1;
    }
    if (!ins) return -2;  // absent, and this op holds no lock
    u64 fidx = ls.ff_idx, fk = ls.ff_k, fv = ls.ff_v;
    if (SCHEME == SCHEME_DOUBLE) {
      if (!sn.empty || !ls.ff_set) return -1;
    } else if (SCHEME == SCHEME_ICEBERG) {
      // a free front slot (recorded in wave 0) wins; else the backyard choice
      // between wave 1's bucket and this one (wave 2), ties to the first
      if (!ls.ff_set) {
        const bool free2 = sn.ffree >= 0;
        int ch = (sn.occ < ls.occ1) ? 2 : 1;
        if (ch == 2 && !free2) ch = 1;
        else if (ch == 1 && !ls.f1_set) ch = 2;
        if (ch == 2 ? !free2 : !ls.f1_set) {
          st = ST_FULL;
          return 1;
        }
        if (ch == 1) {
          fidx = ls.f1_idx;
          fk = ls.f1_k;
        } else {
          fidx = bw * 32 + (u64)sn.ffree;
          fk = sn.ffree_empty ? TAG_EMPTY : TAG_TOMB;
        }
      }
    } else {
      // K is absent from its buckets and the lane holds b_0's lock: place it
      const bool free0 = (w == 0) ? sn.ffree >= 0 : ls.ff_set;
      const int ch = p2_choice(ls.occ0, free0, sn.occ, sn.ffree >= 0, w > 0);
      if (ch < 0) {
        st = ST_FULL;
        return 1;
      }
      if (ch == (int)w) {  // the free slot of this wave's bucket
        if (META) {
          fidx = bw * 32 + (u64)sn.ffree;
          fk = sn.ffree_empty ? TAG_EMPTY : TAG_TOMB;
        } else {
          const Slot o = p.slot(sn.ffree);
          fidx = bw * B + (u64)sn.ffree;
          fk = o.key;
          fv = o.val;
        }
      }
    }
    bool ok;
    if (META) {
      const u16 expect = (u16)fk;
      ok = ptx::cas_tag(tv.tags + fidx, expect, key_tag(K)) == expect;
      if (ok) ptx::st_slot_relaxed(tv.slots + fidx, K, V);
    } else {
      ok = ptx::cas_slot(tv.slots + fidx, fk, fv, K, V);
    }
    if (!ok) {
      fresh = false;
      return -1;
    }
    ++dcount;
    st = ST_INSERTED;
    return 1;
  }
};

// Failure counters for a finished op (leader lane).
__device__ __forceinline__ void count_failure(const TableView& tv, u8 st) {
  if (st >= ST_FULL) {
    u64* ctr = st == ST_FULL ? &tv.ctr->n_full : st == ST_TIMEOUT ? &tv.ctr->n_timeout : &tv.ctr->n_badkey;
    atomicAdd((unsigned long long*)ctr, 1ull);
  }
}

// -------------------------------------------------------------------------
// One warp serves a chunk of up to 32 consecutive ops.
//  1. Stage: lane j loads op j's key (value, op code) with coalesced loads and
//     hashes it once; keys and hashes go to shared memory.
//  2. Lock: an op that may have to insert under the lock (two-choice
//     inserts, mixed batches) takes b_0's lock from its lane, one attempt.
//  3. Lane path: wave w copies bucket w of every open op into shared memory
//     (cp.async; four ops' 128-byte lines per instruction, so each copy
//     instruction is coalesced; with metadata the 64-byte tag line, then the
//     first tag-matching slot), and lane j settles op j from the snapshot
//     when it can.  Two-choice tables with plain 32-slot buckets instead
//     read whole buckets, eight per round, scanned by the warp's votes.
//  4. Tiles serve the ops left over, side by side, with the cooperative
//     probe (snapshot reused unless a lane CAS showed it stale).
//  5. Results leave through shared memory as coalesced stores.
// -------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLaneRestarts = 2;  // streaming lane: restarts of an op after a lost CAS before the tiles

struct WarpSmem {
  u64 key[32], val[32], out[32], h1[32], h2[32];
  u64 bw[32];  // bucket of each op in the current wave
  u8 op[32], st[32], fresh[32], list[32];  // list: open ops of a bucket pass
  u64 in_key[32], in_val[32];  // streaming lanes, host inputs: op i's key / value in slot i % 32
  PreWarp pre;
};

enum { FLAG_SNAP = 1, FLAG_DONE = 2 };

template <int SCHEME, bool META, int B, int T, int KIND>
__device__ __forceinline__ int warp_chunk(const TableView& tv, const BatchArgs& a, int upsert_op, bool lockfree,
                                          u64 base, WarpSmem& sm, int lane) {
  using Ops = TileOps<SCHEME, META, B, T>;
  const u64 ks = a.key_stride ? a.key_stride : 1;
  const u64 gi = base + lane;
  const bool inb = gi < a.n;
  const u64 K = inb ? a.keys[gi * ks] : 0;
  const u64 V = ((KIND == KIND_UPSERT || KIND == KIND_MIXED) && inb && a.vals) ? a.vals[gi * ks] : 0;
  const u8 code = (KIND == KIND_MIXED && inb) ? a.ops[gi] : 0;
  const u64 h1 = fmix64(K ^ tv.seed1), h2 = fmix64(K ^ tv.seed2);
  sm.key[lane] = K;
  sm.val[lane] = V;
  sm.op[lane] = code;
  sm.h1[lane] = h1;
  sm.h2[lane] = h2;
  const bool skip = (KIND == KIND_UPSERT) && (a.flags & BATCH_SKIP_SENTINELS) && is_sentinel(K);
  __syncwarp();

  // what the lane path may do for this op
  int dcount = 0;
  bool done = !inb;
  bool fresh = true;
  u64 out = 0;
  u8 st = ST_MISS;
  int opk = -1, op = upsert_op;
  if (inb && skip) {
    done = true;  // an empty / erased slot of a rehash source
  } else if (inb && is_sentinel(K)) {
    done = true;
    st = ST_BADKEY;
  } else if (inb) {
    int kind = KIND;
    if (KIND == KIND_MIXED) {
      kind = code == MX_QUERY ? KIND_QUERY : code == MX_ERASE ? KIND_ERASE : KIND_UPSERT;
      op = code == MX_INSERT ? OP_INSERT : code == MX_ADD ? OP_ADD : code == MX_MAX ? OP_MAX : OP_REPLACE;
      if (code > MX_ERASE) {
        done = true;
        st = ST_BADKEY;
      }
    }
    if (!done) {
      if (kind == KIND_QUERY)
        opk = Ops::LW_QUERY;
      else if (kind == KIND_ERASE)
        opk = Ops::LW_ERASE;
      else if (KIND == KIND_UPSERT && lockfree && SCHEME == SCHEME_DOUBLE)
        opk = Ops::LW_INSERT_FREE;
      else
        opk = Ops::LW_UPDATE_ONLY;
    }
  }

  bool lane_ok = (KIND != KIND_PROBE) && tv.preload && opk >= 0;
  // two-choice tables with plain 32-slot buckets read whole buckets instead
  // of first-line snapshots (below)
  constexpr bool kRounds = (SCHEME == SCHEME_P2) && !META && B == 32;
  // An insert-if-unique op that may insert under the lock (its key is most
  // likely new) takes b_0's lock from its own lane, one attempt, before its
  // first copy; the lane's reads after it are then authoritative for K (only
  // holders of b_0's lock insert K).  Add / max / replace probe lock-free
  // first: a present key -- a hot Zipf key above all -- needs no lock, and an
  // absent one goes to the tiles, which lock and rescan.  A lane that misses
  // the lock also leaves absent keys to the tiles, which wait for it.
  constexpr bool kLaneLock = (SCHEME == SCHEME_DOUBLE) || META || Ops::PRE_SLOTS == B || kRounds;
  const u64 b0 = Ops::bucket(tv, h1, h2, 0);
  bool locked = false;
  if (kLaneLock && lane_ok && !done && opk == Ops::LW_UPDATE_ONLY && (op == OP_INSERT || tv.phased)) {
    locked = tv.phased || Ops::lane_lock(tv, b0);  // bulk-synchronous: no locks
    if (locked) opk = Ops::LW_INSERT_LOCKED;
  }
  int snap_wave = -1;

  if (kRounds) {
    // Whole-bucket rounds: eight buckets per round, one op's bucket per copy
    // instruction (lane s copies slot s), each scanned with two votes.
    // Pass 0 reads b_0 of every open op, pass 1 b_1 of the ops still open;
    // the lane owning an op settles it.  An op that proved its key absent
    // without holding b_0's lock (its one attempt found the lock taken, or
    // an add / max / replace that probed lock-free) tries the lock once more
    // after the rounds and, holding it, reads its buckets again (now in L2)
    // and claims; only ops that still miss the lock, or lose a CAS, go to
    // the tiles.
    for (int attempt = 0; attempt < 2; ++attempt) {
      bool open = lane_ok && !done;
      if (attempt == 1) {
        const bool retry = open && kLaneLock && opk == Ops::LW_UPDATE_ONLY && fresh;
        const bool got = retry && Ops::lane_lock(tv, b0);
        if (got) {
          locked = true;
          opk = Ops::LW_INSERT_LOCKED;
        }
        open = got;
        if (!__any_sync(0xffffffffu, open)) break;
      }
      u32 occ0 = 0;
      int f0 = -1;
      u64 f0k = 0, f0v = 0;
      for (u32 c = 0; c < 2; ++c) {
        const unsigned om = __ballot_sync(0xffffffffu, open);
        if (!om) break;
        if (open) {
          sm.bw[lane] = Ops::bucket(tv, h1, h2, c);
          sm.list[__popc(om & ((1u << lane) - 1u))] = (u8)lane;
        }
        __syncwarp();
        const int n = __popc(om);
        int hs = -1, fs = -1;
        u32 occ = 0;
        u64 hv = 0, fk = 0, fv = 0;
        for (int r0 = 0; r0 < n; r0 += 8) {
          const int nr = (n - r0) < 8 ? (n - r0) : 8;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < nr) ptx::cp_async16(&sm.pre.flat(q, lane), tv.slots + sm.bw[sm.list[r0 + q]] * 32 + (u64)lane);
          ptx::cp_async_wait_all();
          __syncwarp();
          // the votes of bucket q go to the lane owning its op; the owners
          // then settle their snapshots together, not one after another
          unsigned own_k = 0, own_f = 0;
          int own_q = -1;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (q >= nr) break;  // warp-uniform
            const int j = sm.list[r0 + q];
            const u64 k = sm.pre.flat(q, lane).key;
            const unsigned mk = __ballot_sync(0xffffffffu, k == sm.key[j]);
            const unsigned mf = __ballot_sync(0xffffffffu, k == KEY_EMPTY || k == KEY_TOMB);
            own_k = lane == j ? mk : own_k;
            own_f = lane == j ? mf : own_f;
            own_q = lane == j ? q : own_q;
          }
          if (own_q >= 0) {
            occ = 32u - (u32)__popc(own_f);
            if (own_k) {
              hs = __ffs(own_k) - 1;
              hv = sm.pre.flat(own_q, hs).val;
            }
            if (own_f) {
              fs = __ffs(own_f) - 1;
              const Slot f = sm.pre.flat(own_q, fs);
              fk = f.key;
              fv = f.val;
            }
          }
          __syncwarp();  // the next round overwrites the rows
        }
        if (!open) continue;
        const u64 bc = sm.bw[lane];
        bool absent = false;
        if (hs >= 0) {
          const u64 idx = bc * 32 + (u64)hs;
          open = false;
          if (opk == Ops::LW_QUERY) {
            out = hv;
            st = ST_FOUND;
            done = true;
          } else if (opk == Ops::LW_ERASE) {
            if (ptx::cas_slot(tv.slots + idx, K, hv, KEY_TOMB, 0)) {
              out = hv;
              --dcount;
              st = ST_FOUND;
              done = true;
            }
          } else {
            Ops::apply(tv, idx, op, V);
            st = ST_FOUND;
            done = true;
          }
        } else if (c == 0) {
          occ0 = occ;
          f0 = fs;
          f0k = fk;
          f0v = fv;
          absent = Ops::nprobe(tv) == 1 || (tv.shortcut && occ < Ops::FILL_SHORTCUT);
        } else {
          absent = true;
        }
        if (absent) {
          open = false;
          if (opk == Ops::LW_QUERY || opk == Ops::LW_ERASE) {
            out = 0;
            st = ST_MISS;
            done = true;
          } else if (opk == Ops::LW_INSERT_LOCKED) {
            const int ch = Ops::p2_choice(occ0, f0 >= 0, occ, fs >= 0, c == 1);
            if (ch < 0) {
              st = ST_FULL;
              done = true;
            } else {
              const u64 idx = ch == 0 ? b0 * 32 + (u64)f0 : bc * 32 + (u64)fs;
              if (ptx::cas_slot(tv.slots + idx, ch == 0 ? f0k : fk, ch == 0 ? f0v : fv, K, V)) {
                ++dcount;
                st = ST_INSERTED;
                done = true;
              }
            }
          }
        }
      }
      if (locked && !tv.phased) Ops::lane_unlock(tv, b0, done && st == ST_INSERTED);  // after the claim
      locked = false;
    }
  }

  // lane waves: wave w copies bucket w of every op still open into shared
  // memory (16 bytes per lane per copy instruction, coalesced per bucket),
  // then each lane settles its own op if the snapshot allows
  typename Ops::LaneState ls;
  ls.ff_set = false;
  ls.ff_idx = ls.ff_k = ls.ff_v = 0;
  ls.occ0 = ls.occ1 = 0;
  ls.f1_set = false;
  ls.tsum = 0;
  ls.f1_idx = ls.f1_k = 0;
  // waves: a double-hashing sequence is followed for lane_waves buckets
  // (default 4); the other schemes have 2 or 3 candidate buckets
  const u32 max_waves = kRounds                    ? 0u
                        : (SCHEME == SCHEME_DOUBLE) ? (tv.lane_waves > 0 ? (u32)tv.lane_waves : 4u)
                        : (SCHEME == SCHEME_ICEBERG) ? 3u
                                                     : 2u;
  // Pass 0 follows every open op.  Pass 1 reads again, under b_0's lock, the
  // ops whose keys proved absent without it (a lane that missed the lock, or
  // an add / max / replace that probed lock-free): by then the lock's holder
  // has usually finished, and the lane settles the op from L2-resident lines
  // instead of handing it to a tile that would spin on the lock.
  bool relock = false;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      bool again = false;
      if (relock) {
        again = Ops::lane_lock(tv, b0);
        if (again) {
          locked = true;
          opk = Ops::LW_INSERT_LOCKED;
          ls.ff_set = false;
          ls.ff_idx = ls.ff_k = ls.ff_v = 0;
          ls.occ0 = ls.occ1 = 0;
          ls.f1_set = false;
          ls.tsum = 0;
          ls.f1_idx = ls.f1_k = 0;
        }
      }
      if (!__any_sync(0xffffffffu, again)) break;
      lane_ok = again;  // the other open ops (a sequence longer than the waves) go to the tiles
    }
    for (u32 w = 0; w < max_waves; ++w) {
      const bool want = lane_ok && !done;
      const unsigned wmask = __ballot_sync(0xffffffffu, want);
      if (!wmask) break;
      sm.bw[lane] = want ? Ops::bucket(tv, h1, h2, w) : 0;
      __syncwarp();
      if (META) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = i * 8 + (lane >> 2), part = lane & 3;
          if ((wmask >> j) & 1u) ptx::cp_async16(&sm.pre.at(j, part), tv.tags + sm.bw[j] * 32 + 8 * part);
        }
      } else {
        constexpr int PS = Ops::PRE_SLOTS;  // 8 slots = 128 B per op
#pragma unroll
        for (int i = 0; i < PS; ++i) {
          const int j = i * (32 / PS) + lane / PS, part = lane % PS;
          if ((wmask >> j) & 1u) ptx::cp_async16(&sm.pre.at(j, part), tv.slots + sm.bw[j] * B + (u64)part);
        }
      }
      ptx::cp_async_wait_all();
      __syncwarp();
      if (META) {
          if (want) ls.tsum = Ops::preload_candidate(tv, K, sm.bw[lane], &sm.pre, lane);
        ptx::cp_async_wait_all();
        __syncwarp();
      }
      if (want) {
        snap_wave = (int)w;
        const PreRef p{&sm.pre, lane};
        const int r =
            Ops::lane_wave(tv, p, K, V, op, opk, w, sm.bw[lane], ls, out, st, dcount, fresh, KIND != KIND_ERASE);
        if (r > 0) {
          done = true;
        } else if (r == -2 && kLaneLock && pass == 0 && !locked) {
          relock = true;  // absent, and this op holds no lock
          lane_ok = false;
        } else if (r < 0) {
          lane_ok = false;
        }
      }
      __syncwarp();  // the next wave overwrites the snapshots
    }
    if (locked && !tv.phased) Ops::lane_unlock(tv, b0, done && st == ST_INSERTED);  // after the claim
    locked = false;
  }
  // the tile path may reuse a snapshot only if it is still of b_0 and fresh
  const unsigned pre_mask = __ballot_sync(0xffffffffu, snap_wave == 0 && fresh);
  sm.out[lane] = out;
  sm.st[lane] = st;
  sm.fresh[lane] = 1;
  if (done && inb && st >= ST_FULL) count_failure(tv, st);
  const unsigned todo = __ballot_sync(0xffffffffu, !done);
  __syncwarp();

  // tiles take the leftovers round-robin (a tile's delta lives on its leader)
  int tile_d = 0;
  if (todo) {
    const TileCtx<T> c = make_tile<T>(lane);
    const int tile = lane / T;
    constexpr int NT = 32 / T;
    const int n_todo = __popc(todo);
    // round k: tile t takes the (k*NT + t)-th leftover op, so all tiles work
    // side by side
    for (int k = 0; k * NT < n_todo; ++k) {
      const int rank = k * NT + tile;
      if (rank >= n_todo) continue;
      const int j = (int)__fns(todo, 0, rank + 1);
      const u64 Kj = sm.key[j];
      const u64 h1j = sm.h1[j], h2j = sm.h2[j];
      const PreRef pre = (((pre_mask >> j) & 1u) && sm.fresh[j]) ? PreRef{&sm.pre, j} : no_pre();
      u64 o = 0;
      u8 sj;
      if (KIND == KIND_QUERY) {
        sj = Ops::do_query(tv, c, Kj, h1j, h2j, pre, o);
      } else if (KIND == KIND_PROBE) {
        sj = Ops::do_probe(tv, c, Kj, o);
      } else if (KIND == KIND_UPSERT) {
        sj = lockfree ? Ops::template do_upsert<true>(tv, c, Kj, h1j, h2j, sm.val[j], upsert_op, pre, tile_d)
                      : Ops::template do_upsert<false>(tv, c, Kj, h1j, h2j, sm.val[j], upsert_op, pre, tile_d);
      } else if (KIND == KIND_ERASE) {
        sj = Ops::template do_erase<false>(tv, c, Kj, h1j, h2j, pre, o, tile_d);  // an erase-only launch
      } else {
        sj = Ops::do_mixed(tv, c, sm.op[j], Kj, h1j, h2j, sm.val[j], pre, o, tile_d);
      }
      if (c.tl == 0) {
        sm.out[j] = o;
        sm.st[j] = sj;
        count_failure(tv, sj);
      }
    }
    if (c.tl != 0) tile_d = 0;
  }
  __syncwarp();
  if (inb) {
    if (a.vals_out) a.vals_out[gi] = sm.out[lane];
    if (a.status_out) a.status_out[gi] = sm.st[lane];
  }
  __syncwarp();
  return dcount + tile_d;
}

// -------------------------------------------------------------------------
// Streaming lanes: one warp serves a contiguous range of ops.  Each lane holds
// one op at a time and follows its probe sequence wave by wave (one bucket per
// wave, copied with cp.async like the chunk path); a lane whose op settles
// takes the next op of the range before the next wave, so every wave keeps
// up to 32 probes in flight however long the individual sequences are.  Ops
// the lane path cannot settle (a lost CAS, an unsure tag match, an insert
// without the lock, the probe-count kernel) are parked and served by the
// cooperative tiles, which run only when no lane of the warp is active -- so
// no lane of the warp holds a bucket lock a tile might wait for.  Refill
// pauses once enough ops are parked to fill the tiles.
// -------------------------------------------------------------------------
// Work shares: with `ticket` null the warp serves [begin, end); otherwise it
// takes shares of up to `share` ops (a multiple of 32) from the launch's
// ticket, which counts ops (begin / end unused), whenever its lanes run dry,
// so warps whose ops probe long keep fewer ops and all finish close
// together; `warps` is the launch's warp count.
template <int SCHEME, bool META, int B, int T, int KIND>
__device__ __forceinline__ int warp_stream(const TableView& tv, const BatchArgs& a, int upsert_op, bool lockfree,
                                           u64 begin, u64 end, WarpSmem& sm, int lane, u64* ticket = nullptr,
                                           u64 share = 0, u64 warps = 1) {
  using Ops = TileOps<SCHEME, META, B, T>;
  enum { L_EMPTY = 0, L_ACTIVE = 1, L_PARKED = 2 };
  constexpr int NT = 32 / T;
  constexpr unsigned kAll = 0xffffffffu;
  constexpr bool kLaneLock = (SCHEME == SCHEME_DOUBLE) || META || Ops::PRE_SLOTS == B || Ops::kLines;
  const u64 ks = a.key_stride ? a.key_stride : 1;
  const bool lane_path = (KIND != KIND_PROBE) && tv.preload;
  // a cap on the waves of one op (WS_OPT_LANE_WAVES); by default the whole sequence
  const u32 cap = (SCHEME == SCHEME_DOUBLE && tv.lane_waves > 0) ? (u32)tv.lane_waves : 0xffffffffu;
  // a lane's op (key, value, hashes, index) lives in its shared-memory
  // columns; registers hold only the probe state
  int state = L_EMPTY;
  int opk = -1, op = upsert_op;
  bool locked = false, fresh = true;
  u32 w = 0;
  int restarts = 0;  // restarts of the current op after a lost CAS
  typename Ops::LaneState ls;
  int dcount = 0, tile_d = 0;
  u64 next = begin;
  bool exhausted = ticket == nullptr;  // no more shares to take
  if (ticket) next = end = 0;
  // Input ring (host inputs read in place): slot s of in_key / in_val holds
  // the op i with i % 32 == s among the 32 ops from `next` on (shares start
  // at multiples of 32).  Lane s copies its slot's op when the share begins
  // and whenever its op is taken, so a lane that takes a new op finds its
  // inputs in shared memory: the copies complete during the wave between.
  const bool ring = (a.flags & BATCH_HOST_INPUTS) != 0 && ticket != nullptr;
  const bool want_v = (KIND == KIND_UPSERT || KIND == KIND_MIXED) && a.vals != nullptr;
  for (;;) {
    // 1. refill: empty lanes take the next ops of the range, in lane order
    unsigned parked = __ballot_sync(kAll, state == L_PARKED);
    const unsigned empty = __ballot_sync(kAll, state == L_EMPTY);
    if (!exhausted && empty && next >= end) {  // the share is used up: take the next one
      u64 first = 0;
      if (lane == 0) first = atomicAdd((unsigned long long*)ticket, (unsigned long long)share);
      first = __shfl_sync(kAll, first, 0);
      if (first < a.n) {
        next = first;
        end = (a.n - first < share) ? a.n : first + share;
        // guided shares: once fewer than four shares per warp are left, take
        // a quarter per warp of what is left (a multiple of 32, at least 32),
        // so that the warps run dry together at the end of the launch
        const u64 left = ((a.n - end) / (4 * warps) + 31) / 32 * 32;
        if (left < share) share = left < 32 ? 32 : left;
        if (ring && first + (u64)lane < end) {
          ptx::cp_async8(&sm.in_key[lane], a.keys + (first + lane) * ks);
          if (want_v) ptx::cp_async8(&sm.in_val[lane], a.vals + (first + lane) * ks);
        }
      } else {
        exhausted = true;
      }
    }
    if (empty && next < end && __popc(parked) < NT) {
      const u64 rank = (u64)__popc(empty & ((1u << lane) - 1u));
      if (ring) {  // the ring's copies (usually complete long ago) become visible to the warp
        ptx::cp_async_wait_all();
        __syncwarp();
      }
      if (state == L_EMPTY && next + rank < end) {
        const u64 gi = next + rank;
        const u64 K = ring ? sm.in_key[gi & 31u] : a.keys[gi * ks];
        const u64 V = want_v ? (ring ? sm.in_val[gi & 31u] : a.vals[gi * ks]) : 0;
        const u8 code = (KIND == KIND_MIXED) ? a.ops[gi] : 0;
        const u64 h1 = fmix64(K ^ tv.seed1), h2 = fmix64(K ^ tv.seed2);
        u8 st = ST_MISS;
        bool settled = false;
        op = upsert_op;
        opk = -1;
        if (KIND == KIND_UPSERT && (a.flags & BATCH_SKIP_SENTINELS) && is_sentinel(K)) {
          settled = true;  // an empty / erased slot of a rehash source: MISS
          if (a.vals_out) a.vals_out[gi] = 0;
          if (a.status_out) a.status_out[gi] = ST_MISS;
        } else if (is_sentinel(K) || (KIND == KIND_MIXED && code > MX_ERASE)) {
          settled = true;
          st = ST_BADKEY;
          count_failure(tv, st);
          if (a.vals_out) a.vals_out[gi] = 0;
          if (a.status_out) a.status_out[gi] = st;
        } else {
          int kind = KIND;
          if (KIND == KIND_MIXED) {
            kind = code == MX_QUERY ? KIND_QUERY : code == MX_ERASE ? KIND_ERASE : KIND_UPSERT;
            op = code == MX_INSERT ? OP_INSERT : code == MX_ADD ? OP_ADD : code == MX_MAX ? OP_MAX : OP_REPLACE;
          }
          opk = kind == KIND_QUERY ? Ops::LW_QUERY
                : kind == KIND_ERASE ? Ops::LW_ERASE
                : (KIND == KIND_UPSERT && lockfree && SCHEME == SCHEME_DOUBLE) ? Ops::LW_INSERT_FREE
                                                                                 : Ops::LW_UPDATE_ONLY;
        }
        if (!settled) {
          sm.key[lane] = K;
          sm.val[lane] = V;
          sm.op[lane] = code;
          sm.h1[lane] = h1;
          sm.h2[lane] = h2;
          sm.out[lane] = gi;  // the op's index
          w = 0;
          fresh = true;
          restarts = 0;
          ls.ff_set = false;
          ls.ff_idx = ls.ff_k = ls.ff_v = 0;
          ls.occ0 = ls.occ1 = ls.cur_occ = ls.next_w = 0;
          ls.f1_set = false;
          ls.tsum = 0;
          ls.f1_idx = ls.f1_k = ls.f1_v = 0;
          locked = false;
          if (!lane_path) {
            state = L_PARKED;
          } else {
            if (kLaneLock && opk == Ops::LW_UPDATE_ONLY && (op == OP_INSERT || tv.phased)) {
              locked = tv.phased || Ops::lane_lock(tv, Ops::bucket(tv, h1, h2, 0));
              if (locked) opk = Ops::LW_INSERT_LOCKED;
            }
            state = L_ACTIVE;
          }
        }
      }
      const u64 took = (u64)__popc(empty);
      const u64 ncons = (end - next < took) ? end - next : took;
      if (ring) {
        // the slots of the ops just taken receive the op 32 further on
        __syncwarp();  // every lane has read its slot
        const u64 off = ((u64)lane - next) & 31u;  // this lane's slot in the window from `next`
        if (off < ncons && next + off + 32 < end) {
          ptx::cp_async8(&sm.in_key[lane], a.keys + (next + off + 32) * ks);
          if (want_v) ptx::cp_async8(&sm.in_val[lane], a.vals + (next + off + 32) * ks);
        }
      }
      next += ncons;
    }
    // 2. one wave: copy each active lane's current bucket, then settle
    const unsigned act = __ballot_sync(kAll, state == L_ACTIVE);
    if (act) {
      sm.bw[lane] = (state == L_ACTIVE) ? Ops::bucket(tv, sm.h1[lane], sm.h2[lane], Ops::wave_bucket(w)) : 0;
      if (Ops::kLines) sm.fresh[lane] = (u8)Ops::wave_line(w);  // which line of the bucket
      __syncwarp();
      if (META) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = i * 8 + (lane >> 2), part = lane & 3;
          if ((act >> j) & 1u) ptx::cp_async16(&sm.pre.at(j, part), tv.tags + sm.bw[j] * 32 + 8 * part);
        }
      } else {
        constexpr int PS = Ops::PRE_SLOTS;
#pragma unroll
        for (int i = 0; i < PS; ++i) {
          const int j = i * (32 / PS) + lane / PS, part = lane % PS;
          const u64 line = Ops::kLines ? (u64)sm.fresh[j] * PS : 0;
          if ((act >> j) & 1u) ptx::cp_async16(&sm.pre.at(j, part), tv.slots + sm.bw[j] * B + line + (u64)part);
        }
      }
      ptx::cp_async_wait_all();
      __syncwarp();
      if (META) {
        if (state == L_ACTIVE) ls.tsum = Ops::preload_candidate(tv, sm.key[lane], sm.bw[lane], &sm.pre, lane);
        ptx::cp_async_wait_all();
        __syncwarp();
      }
      if (state == L_ACTIVE) {
        const PreRef p{&sm.pre, lane};
        u64 out = 0;
        u8 st = ST_MISS;
        int r;
        if constexpr (Ops::kLines)
          r = Ops::lane_wave_lines(tv, p, sm.key[lane], sm.val[lane], op, opk, w, sm.bw[lane], ls, out, st, dcount,
                                   fresh);
        else
          r = Ops::lane_wave(tv, p, sm.key[lane], sm.val[lane], op, opk, w, sm.bw[lane], ls, out, st, dcount, fresh,
                             KIND != KIND_ERASE);
        const bool wrote = r > 0 && st == ST_INSERTED;
        if (r > 0) {
          const u64 gi = sm.out[lane];
          if (a.vals_out) a.vals_out[gi] = out;
          if (a.status_out) a.status_out[gi] = st;
          if (st >= ST_FULL) count_failure(tv, st);
          state = L_EMPTY;
        } else if (r == -2 && kLaneLock && !locked &&
                   Ops::lane_lock(tv, Ops::bucket(tv, sm.h1[lane], sm.h2[lane], 0))) {
          // absent without the lock: now holding b_0's lock, follow the
          // sequence again from b_0 and insert from what it reads
          locked = true;
          opk = Ops::LW_INSERT_LOCKED;
          w = 0;
          ls.ff_set = false;
          ls.ff_idx = ls.ff_k = ls.ff_v = 0;
          ls.occ0 = ls.occ1 = ls.cur_occ = ls.next_w = 0;
          ls.f1_set = false;
          ls.tsum = 0;
          ls.f1_idx = ls.f1_k = ls.f1_v = 0;
        } else if (r == -1 && !fresh && restarts < kLaneRestarts) {
          // a lost CAS: the table moved under the snapshot (another claim
          // or erase in this bucket).  Follow the sequence again from b_0
          // -- its lines are in L2 now -- instead of handing the op to a
          // tile; a held lock stays held.
          ++restarts;
          fresh = true;
          w = 0;
          ls.ff_set = false;
          ls.ff_idx = ls.ff_k = ls.ff_v = 0;
          ls.occ0 = ls.occ1 = ls.cur_occ = ls.next_w = 0;
          ls.f1_set = false;
          ls.tsum = 0;
          ls.f1_idx = ls.f1_k = ls.f1_v = 0;
        } else if (r < 0 || w + 1 >= cap) {
          state = L_PARKED;
        } else {
          w = Ops::kLines ? ls.next_w : w + 1;
        }
        if (state != L_ACTIVE && locked) {
          if (!tv.phased) Ops::lane_unlock(tv, Ops::bucket(tv, sm.h1[lane], sm.h2[lane], 0), wrote);  // after the claim
          locked = false;
        }
      }
      __syncwarp();  // the next wave overwrites the snapshots
    }
    // 3. tiles: parked ops, once no lane is active (no lane holds a lock)
    const bool any_active = __any_sync(kAll, state == L_ACTIVE);
    parked = __ballot_sync(kAll, state == L_PARKED);
    if (parked && !any_active) {
      const TileCtx<T> c = make_tile<T>(lane);
      const int tile = lane / T;
      const int n_todo = __popc(parked);
      for (int k = 0; k * NT < n_todo; ++k) {
        const int rank = k * NT + tile;
        if (rank >= n_todo) continue;  // tile-uniform
        const int j = (int)__fns(parked, 0, rank + 1);
        const u64 Kj = sm.key[j], h1j = sm.h1[j], h2j = sm.h2[j], gj = sm.out[j];
        u64 o = 0;
        u8 sj;
        int rd = 0;
        if (KIND == KIND_QUERY) {
          sj = Ops::do_query(tv, c, Kj, h1j, h2j, no_pre(), o);
        } else if (KIND == KIND_PROBE) {
          sj = Ops::do_probe(tv, c, Kj, o);
        } else if (KIND == KIND_UPSERT) {
          sj = lockfree ? Ops::template do_upsert<true>(tv, c, Kj, h1j, h2j, sm.val[j], upsert_op, no_pre(), rd)
                        : Ops::template do_upsert<false>(tv, c, Kj, h1j, h2j, sm.val[j], upsert_op, no_pre(), rd);
        } else if (KIND == KIND_ERASE) {
          sj = Ops::template do_erase<false>(tv, c, Kj, h1j, h2j, no_pre(), o, rd);  // an erase-only launch
        } else {
          sj = Ops::do_mixed(tv, c, sm.op[j], Kj, h1j, h2j, sm.val[j], no_pre(), o, rd);
        }
        if (c.tl == 0) {
          if (a.vals_out) a.vals_out[gj] = o;
          if (a.status_out) a.status_out[gj] = sj;
          count_failure(tv, sj);
          tile_d += rd;
        }
      }
      __syncwarp();
      if (state == L_PARKED) state = L_EMPTY;
    } else if (!any_active && next >= end && exhausted) {
      break;  // nothing active, parked or left to take
    }
  }
  return dcount + tile_d;
}

constexpr u64 kChunkGroup = 4;     // 32-op chunks a warp takes per ticket
constexpr u64 kStreamShare = 256;  // ops a streaming warp takes per ticket

template <int SCHEME, bool META, int B, int T, int KIND>
__global__ void __launch_bounds__(kThreads, 4) batch_kernel(TableView tv, BatchArgs a) {
  __shared__ WarpSmem s_w[kWarps];
  __shared__ long long s_cnt;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const bool lockfree = (KIND == KIND_UPSERT);  // one call is one phase: no erase runs with it
  int dcount = 0;
  // Insert-if-unique calls on tables whose inserts lock (two-choice,
  // iceberg) take a lock for almost every op; streaming would pay that
  // acquire once per wave instead of once per 32-op chunk.  Plain
  // two-choice tables with 32-slot buckets read whole buckets in 32-op
  // chunks (rounds) for queries and erases too: a negative query or an
  // erase of a late key needs most of both buckets, which rounds fetch in
  // fewer dependent steps than streaming lanes reading a line per wave
  // (measured at 2^28 slots: negative queries 2.56 ms in rounds vs 3.54 by
  // lines, positive queries 1.51 vs 1.31, upserts 1.87 vs 1.66).
  constexpr bool kRounds = (SCHEME == SCHEME_P2) && !META && B == 32;
  const bool lock_bound = (KIND == KIND_UPSERT) && SCHEME != SCHEME_DOUBLE && a.op == OP_INSERT;
  // (WS_OPT_STREAM = 2 streams them too, by lines: fewer bytes for hits near
  // the front of b_0, more dependent steps for misses.)
  const bool rounds = kRounds && (KIND == KIND_QUERY || KIND == KIND_ERASE) && tv.stream != 2;
  // Work comes from the launch's ticket: warps that draw long probe
  // sequences take less of it.  Shares shrink with the batch so that a small
  // launch still spreads over every warp (about four shares per warp, 32 to
  // kStreamShare ops each; one to kChunkGroup chunks), and shrink again
  // towards the end of the launch (guided self-scheduling).
  u64* ticket = &tv.ctr->ticket;
  const u64 warps = (u64)gridDim.x * kWarps;
  if (!tv.stream || lock_bound || rounds) {
    const u64 nchunks = (a.n + 31) / 32;
    u64 group = nchunks / (4 * warps);
    group = group < 1 ? 1 : (group > kChunkGroup ? kChunkGroup : group);
    for (;;) {
      u64 c0 = 0;
      if (lane == 0) c0 = atomicAdd((unsigned long long*)ticket, (unsigned long long)group);
      c0 = __shfl_sync(0xffffffffu, c0, 0);
      if (c0 >= nchunks) break;
      const u64 c1 = (nchunks - c0 < group) ? nchunks : c0 + group;
      // guided: once fewer than four groups per warp are left, take a
      // quarter per warp of what is left (at least one chunk)
      const u64 left = (nchunks - c1) / (4 * warps);
      if (left < group) group = left < 1 ? 1 : left;
      for (u64 ch = c0; ch < c1; ++ch)
        dcount += warp_chunk<SCHEME, META, B, T, KIND>(tv, a, a.op, lockfree, ch * 32, s_w[w], lane);
    }
  } else {
    u64 share = (a.n / (4 * warps) + 31) / 32 * 32;
    share = share < 32 ? 32 : (share > kStreamShare ? kStreamShare : share);
    dcount += warp_stream<SCHEME, META, B, T, KIND>(tv, a, a.op, lockfree, 0, 0, s_w[w], lane, ticket, share,
                                                    warps);
  }
  if (KIND != KIND_QUERY && KIND != KIND_PROBE) {
    const int mine = __reduce_add_sync(0xffffffffu, dcount);
    if (lane == 0 && mine) atomicAdd((unsigned long long*)&s_cnt, (unsigned long long)(long long)mine);
  }
  __syncthreads();  // every warp of the block is done with the ticket
  if (threadIdx.x == 0) {
    if ((KIND != KIND_QUERY && KIND != KIND_PROBE) && s_cnt)
      atomicAdd((unsigned long long*)&tv.ctr->count, (unsigned long long)s_cnt);
    // the launch's last block returns the ticket to zero for the next launch
    // on this table (launches on one table are stream-ordered)
    __threadfence();
    if (atomicAdd((unsigned long long*)&tv.ctr->done, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch((unsigned long long*)&tv.ctr->ticket, 0ull);
      atomicExch((unsigned long long*)&tv.ctr->done, 0ull);
    }
  }
}

// Occupancy-sized launch (one full wave of blocks; the warps take their work
// from the table's ticket).  The kernel is a template argument so each
// instantiation caches its own occupancy.
template <void (*KERN)(TableView, BatchArgs)>
cudaError_t launch_sized(const TableView& tv, const BatchArgs& a, cudaStream_t s, int num_sms) {
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, KERN, kThreads, 0) != cudaSuccess || o < 1) o = 1;
    occ = o;
  }
  const u64 chunks = (a.n + 31) / 32;
  const u64 need = (chunks + kWarps - 1) / kWarps;
  const u64 cap = (u64)occ * (u64)(num_sms > 0 ? num_sms : 1);
  const unsigned grid = (unsigned)(need < cap ? need : cap);
  if (grid == 0) return cudaSuccess;
  KERN<<<grid, kThreads, 0, s>>>(tv, a);
  return cudaGetLastError();
}

template <int SCHEME, bool META, int B, int T>
cudaError_t launch_cfg(const TableView& tv, const BatchArgs& a, int kind, cudaStream_t s, int num_sms) {
  switch (kind) {
    case KIND_QUERY: return launch_sized<batch_kernel<SCHEME, META, B, T, KIND_QUERY>>(tv, a, s, num_sms);
    case KIND_UPSERT: return launch_sized<batch_kernel<SCHEME, META, B, T, KIND_UPSERT>>(tv, a, s, num_sms);
    case KIND_ERASE: return launch_sized<batch_kernel<SCHEME, META, B, T, KIND_ERASE>>(tv, a, s, num_sms);
    case KIND_MIXED: return launch_sized<batch_kernel<SCHEME, META, B, T, KIND_MIXED>>(tv, a, s, num_sms);
    case KIND_PROBE: return launch_sized<batch_kernel<SCHEME, META, B, T, KIND_PROBE>>(tv, a, s, num_sms);
  }
  return cudaErrorInvalidValue;
}

// Dispatchers defined in the instantiation units.
cudaError_t launch_double_plain(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_double_meta(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_p2_plain(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_p2_meta(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_iceberg_meta(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);

}  // namespace ws
