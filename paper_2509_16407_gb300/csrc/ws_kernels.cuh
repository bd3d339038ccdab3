// ws_kernels.cuh -- tile-cooperative batch kernels for bucketed open addressing.
//
// One cooperative tile of T lanes (T in {4, 8, 16, 32}, densely packed in a
// warp, §3.2 / §5) serves one operation at a time.  A bucket of B slots
// (16 B each) is read in steps of T consecutive slots, so for B = 8, T = 8 a
// step is one coalesced 128-byte line per tile; for T > B one step covers
// T/B buckets at once (the next buckets of a double-hashing sequence, or
// both choices of a two-choice key).  Key matches, empty slots and free
// slots are found with warp votes over the tile.
//
// Probe schemes (§2.2):
//   double hashing  b_i = (h1 + i * (h2 | 1)) mod nb, i < max_probe; a scan
//                   ends at the first bucket holding an EMPTY slot.
//   two-choice      b_0 = h1 mod nb, b_1 = h2 mod nb (b_0 + 1 if equal); an
//                   insert goes to b_0 while it is below 3/4 full (the
//                   "shortcut" of §2.2), otherwise to the less loaded bucket
//                   (ties to b_0).
// Fingerprints (§4.3): with metadata, each 32-slot bucket has a 64-byte line
// of 16-bit tags.  A probe reads the tag line, and only slots whose tag
// matches are read and compared against the full key, so the result is exact.
//
// Concurrency (§4.1, §4.2):
//   * queries take no lock; each slot is read with one 128-bit load;
//   * an upsert first probes lock-free; a present key is updated in place
//     with a 64-bit atomic (stability, §2.1: keys never move), so repeated
//     upserts of a hot key never serialise on a lock;
//   * an absent key takes the lock bit of its primary bucket b_0 (one bit
//     per bucket in an external array), re-scans, and claims a free slot with
//     one 128-bit CAS that publishes key and value together (metadata
//     tables: a 16-bit CAS on the tag, then a 128-bit release store of the
//     pair).  The lock makes same-key inserters agree on one location (the
//     adversarial case of Fig. 2);
//   * erase finds the key and swaps the pair for {TOMB, 0} with a 128-bit
//     CAS (then the tag becomes TOMB).  A tombstone never turns back into
//     EMPTY, which keeps every early-exit rule valid.
// Every lock wait is bounded: after spin_limit attempts the op reports
// WS_FAIL_TIMEOUT instead of spinning on.  A tile waiting for a lock keeps
// re-probing lock-free and finishes without the lock as soon as the key
// appears (a concurrent inserter of the same key got there first).
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

template <int SCHEME, bool META, int B, int T>
struct TileOps {
  static_assert(B == 8 || B == 16 || B == 32, "bucket size");
  static_assert(T == 4 || T == 8 || T == 16 || T == 32, "tile size");
  static_assert(!META || B == 32, "metadata tables use 32-slot buckets (one 64-byte tag line)");
  static constexpr int G = (T > B) ? (T / B) : 1;    // buckets covered by one step
  static constexpr int LPB = (T > B) ? B : T;        // lanes per bucket in a step
  static constexpr int SPB = (T > B) ? 1 : (B / T);  // steps per bucket
  static constexpr int TPL = 32 / T;                 // tags per lane (metadata)
  static constexpr u32 FILL_SHORTCUT = (3u * B) / 4u;

  struct Hit {
    bool found;
    u64 idx, val;
  };
  struct Scan {
    bool found;
    u64 idx, val;     // where the key is (found)
    bool has_free;
    u64 fidx, fk, fv; // free slot to claim and its observed content (tag in fk for META)
    bool stuck;       // a wait for a claimed slot's pair ran out
  };

  __device__ static __forceinline__ u32 nprobe(const TableView& tv) {
    if (SCHEME == SCHEME_DOUBLE) return tv.pmax;
    return tv.nb_mask == 0 ? 1u : 2u;
  }

  __device__ static __forceinline__ u64 bucket(const TableView& tv, u64 h1, u64 h2, u32 i) {
    if (SCHEME == SCHEME_DOUBLE) return (h1 + (u64)i * (h2 | 1ull)) & tv.nb_mask;
    const u64 b0 = h1 & tv.nb_mask;
    if (i == 0) return b0;
    u64 b1 = h2 & tv.nb_mask;
    if (b1 == b0) b1 = (b0 + 1) & tv.nb_mask;
    return b1;
  }

  // Bring the first bucket(s) of key K into L2 ahead of the tile that will
  // probe them (one lane per op, so a warp has 32 ops' lines in flight while
  // its tiles work through the ops one at a time).  Double hashing: b_0;
  // two-choice: b_0 and b_1.  Metadata tables: the 64-byte tag lines.
  __device__ static __forceinline__ void prefetch_one(const TableView& tv, u64 b, int method) {
    if (META) {
      const u16* tp = tv.tags + b * 32;
      if (method == 2)
        ptx::prefetch_bulk_l2(tp, 64);
      else
        ptx::prefetch_line_l2(tp);
    } else {
      const Slot* sp = tv.slots + b * B;
      if (method == 2) {
        ptx::prefetch_bulk_l2(sp, B * 16);
      } else {
#pragma unroll
        for (int l = 0; l < (B * 16) / 128; ++l) ptx::prefetch_line_l2(sp + l * 8);
      }
    }
  }
  __device__ static __forceinline__ void prefetch_key(const TableView& tv, u64 K, int method) {
    if (is_sentinel(K)) return;
    const u64 h1 = fmix64(K ^ tv.seed1);
    prefetch_one(tv, h1 & tv.nb_mask, method);
    if (SCHEME == SCHEME_P2 && tv.nb_mask) prefetch_one(tv, bucket(tv, h1, fmix64(K ^ tv.seed2), 1), method);
  }

  // ----------------------------------------------------------------------
  // Plain buckets (no metadata)
  // ----------------------------------------------------------------------
  // Probe cost of one step: LPB consecutive 16-byte slots of each active
  // bucket = LPB/2 DRAM sectors and ceil(LPB*16/128) cache lines.
  static constexpr u32 kStepSectors = LPB / 2;
  static constexpr u32 kStepLines = (LPB * 16 + 127) / 128;

  template <bool COUNT = false>
  __device__ static Hit find_plain(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                   u32* sectors = nullptr, u32* lines = nullptr) {
    const u32 P = nprobe(tv);
    const int g = c.tl / LPB, j = c.tl % LPB;
    u32 occ0 = 0;
    for (u32 i = 0; i < P; i += G) {
      const bool act = (i + g) < P;
      const u64 b = bucket(tv, h1, h2, act ? i + g : i);
      bool ended = false;
#pragma unroll
      for (int s = 0; s < SPB; ++s) {
        const u64 si = b * B + (u64)(s * LPB + j);
        u64 k = KEY_RESV, v = 0;
        if (act) ptx::ld_slot(tv.slots + si, k, v);
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
        if (SCHEME == SCHEME_P2 && G == 1 && i == 0)
          occ0 += __popc(c.ballot(k != KEY_EMPTY && k != KEY_TOMB));
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

  __device__ static Scan scan_plain(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2) {
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
          const u64 si = b * B + (u64)(s * LPB + j);
          u64 k = KEY_RESV, v = 0;
          if (act) ptx::ld_slot(tv.slots + si, k, v);
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
          const u64 si = b * B + (u64)(s * LPB + j);
          u64 k, v;
          ptx::ld_slot(tv.slots + si, k, v);
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
      u64 k = KEY_RESV, v = 0;
      if (act) ptx::ld_slot(tv.slots + si, k, v);
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
  __device__ static __forceinline__ void tag_masks(const TableView& tv, const TileCtx<T>& c, u64 b,
                                                   u16 kt, unsigned& mm, unsigned& me,
                                                   unsigned& mf) {
    const u16* tp = tv.tags + b * 32 + (u64)(c.tl * TPL);
    unsigned lm = 0, le = 0, lf = 0;
    if (TPL == 8) {
      u64 a0, a1;
      ptx::ld_tags16(tp, a0, a1);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const u16 t = (u16)(((q < 4) ? (a0 >> (16 * q)) : (a1 >> (16 * (q - 4)))) & 0xffffu);
        lm |= (unsigned)(t == kt) << q;
        le |= (unsigned)(t == TAG_EMPTY) << q;
        lf |= (unsigned)(t < 2) << q;
      }
    } else if (TPL == 4) {
      const u64 a = ptx::ld_tags8(tp);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const u16 t = (u16)((a >> (16 * q)) & 0xffffu);
        lm |= (unsigned)(t == kt) << q;
        le |= (unsigned)(t == TAG_EMPTY) << q;
        lf |= (unsigned)(t < 2) << q;
      }
    } else if (TPL == 2) {
      const u32 a = ptx::ld_tags4(tp);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const u16 t = (u16)((a >> (16 * q)) & 0xffffu);
        lm |= (unsigned)(t == kt) << q;
        le |= (unsigned)(t == TAG_EMPTY) << q;
        lf |= (unsigned)(t < 2) << q;
      }
    } else {
      const u16 t = ptx::ld_tags2(tp);
      lm = (t == kt);
      le = (t == TAG_EMPTY);
      lf = (t < 2);
    }
    const int sh = c.tl * TPL;
    mm = __reduce_or_sync(c.mask, lm << sh);
    me = __reduce_or_sync(c.mask, le << sh);
    mf = __reduce_or_sync(c.mask, lf << sh);
  }

  // Reads the candidate slots of a tag match mask; true if one holds K.
  // The leader lane reads each candidate and broadcasts the pair, so every
  // lane of the tile takes the same branch even while another tile rewrites
  // the slot (separate per-lane reads could disagree and split the tile).
  // With WAIT (lock-free inserts, where no erase runs concurrently) a slot
  // whose tag is claimed but whose pair is not stored yet (key EMPTY/TOMB) is
  // re-read until the claimer's release store lands, so a same-key inserter
  // cannot miss a copy being written.  *stuck reports a wait that ran out.
  template <bool WAIT = false>
  __device__ static __forceinline__ bool verify(const TableView& tv, const TileCtx<T>& c, u64 b, unsigned mm,
                                                u64 K, u64& idx, u64& val, bool* stuck = nullptr) {
    while (mm) {
      const int q = __ffs(mm) - 1;
      mm &= mm - 1;
      const u64 si = b * 32 + (u64)q;
      u64 k, v;
      read_pair(tv, c, si, k, v);
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

  // One slot read by the leader lane, broadcast to the tile (tile-uniform).
  __device__ static __forceinline__ void read_pair(const TableView& tv, const TileCtx<T>& c, u64 si, u64& k,
                                                   u64& v) {
    k = 0;
    v = 0;
    if (c.tl == 0) ptx::ld_slot(tv.slots + si, k, v);
    k = c.shfl(k, 0);
    v = c.shfl(v, 0);
  }

  // Probe cost with metadata: a tag line read is 64 B (2 sectors, 1 line);
  // each candidate slot read is one 32-byte sector of one line.
  template <bool COUNT = false>
  __device__ static Hit find_meta(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2,
                                  u32* sectors = nullptr, u32* lines = nullptr) {
    const u32 P = nprobe(tv);
    const u16 kt = key_tag(K);
    for (u32 i = 0; i < P; ++i) {
      const u64 b = bucket(tv, h1, h2, i);
      unsigned mm, me, mf;
      tag_masks(tv, c, b, kt, mm, me, mf);
      if (COUNT) {
        // candidates read until the key is found (at most all of them)
        unsigned seen = mm;
        u32 nc = 0;
        while (seen) {
          const int q = __ffs(seen) - 1;
          seen &= seen - 1;
          ++nc;
          u64 kk, vv;
          read_pair(tv, c, b * 32 + (u64)q, kk, vv);
          if (kk == K) break;
        }
        *sectors += 2 + nc;
        *lines += 1 + nc;
      }
      u64 idx, val;
      if (verify(tv, c, b, mm, K, idx, val)) return {true, idx, val};
      if (SCHEME == SCHEME_DOUBLE) {
        if (me) break;
      } else if (i == 0 && tv.shortcut && (u32)(32 - __popc(mf)) < FILL_SHORTCUT) {
        break;
      }
    }
    return {false, 0, 0};
  }

  template <bool WAIT = false>
  __device__ static Scan scan_meta(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1, u64 h2) {
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
        unsigned mm, me, mf;
        tag_masks(tv, c, b, kt, mm, me, mf);
        if (verify<WAIT>(tv, c, b, mm, K, r.idx, r.val, &r.stuck)) {
          r.found = true;
          return r;
        }
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
    u32 occ[2] = {0, 0};
    bool hf[2] = {false, false};
    u64 fi[2] = {0, 0}, ft[2] = {0, 0};
    bool decided0 = (P == 1);
    for (u32 bi = 0; bi < P; ++bi) {
      const u64 b = bucket(tv, h1, h2, bi);
      unsigned mm, me, mf;
      tag_masks(tv, c, b, kt, mm, me, mf);
      if (verify<WAIT>(tv, c, b, mm, K, r.idx, r.val, &r.stuck)) {
        r.found = true;
        return r;
      }
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
  __device__ static __forceinline__ Hit find(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1,
                                             u64 h2) {
    if (META) return find_meta(tv, c, K, h1, h2);
    return find_plain(tv, c, K, h1, h2);
  }
  template <bool WAIT = false>
  __device__ static __forceinline__ Scan scan(const TableView& tv, const TileCtx<T>& c, u64 K, u64 h1,
                                              u64 h2) {
    if (META) return scan_meta<WAIT>(tv, c, K, h1, h2);
    return scan_plain(tv, c, K, h1, h2);
  }

  // Claim the scanned free slot for (K, V).  Leader lane writes; all learn the outcome.
  __device__ static __forceinline__ bool claim(const TableView& tv, const TileCtx<T>& c, const Scan& r,
                                               u64 K, u64 V) {
    int ok = 0;
    if (c.tl == 0) {
      if (META) {
        const u16 expect = (u16)r.fk;
        if (ptx::cas_tag(tv.tags + r.fidx, expect, key_tag(K)) == expect) {
          ptx::st_slot_release(tv.slots + r.fidx, K, V);
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

  __device__ static __forceinline__ void unlock(const TableView& tv, const TileCtx<T>& c, u64 b) {
    __syncwarp(c.mask);
    if (c.tl == 0) ptx::red_and_release(tv.locks + (b >> 5), ~(1u << (b & 31)));
  }

  // ----------------------------------------------------------------------
  // Operations (tile-uniform control flow; results valid on every lane)
  // ----------------------------------------------------------------------
  __device__ static u8 do_query(const TableView& tv, const TileCtx<T>& c, u64 K, u64& out) {
    out = 0;
    if (is_sentinel(K)) return ST_BADKEY;
    const u64 h1 = fmix64(K ^ tv.seed1), h2 = fmix64(K ^ tv.seed2);
    const Hit h = find(tv, c, K, h1, h2);
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
    if (META)
      h = find_meta<true>(tv, c, K, h1, h2, &sec, &lin);
    else
      h = find_plain<true>(tv, c, K, h1, h2, &sec, &lin);
    out = ((u64)lin << 32) | (u64)sec;
    return h.found ? ST_FOUND : ST_MISS;
  }

  // LOCKFREE: the caller guarantees that no erase runs in the same launch (a
  // plain insert / upsert call is one phase).
  template <bool LOCKFREE>
  __device__ static u8 do_upsert(const TableView& tv, const TileCtx<T>& c, u64 K, u64 V, int op,
                                 int& dcount) {
    if (is_sentinel(K)) return ST_BADKEY;
    const u64 h1 = fmix64(K ^ tv.seed1), h2 = fmix64(K ^ tv.seed2);
    if (LOCKFREE && SCHEME == SCHEME_DOUBLE) {
      // Without erases, free slots only disappear, so every inserter of K
      // targets the first free slot of K's probe sequence: the CAS winner
      // places K and a loser's rescan finds it (with metadata, verify waits
      // out a claimed-but-unwritten slot).  No lock is needed; the lock of
      // §4.1 is for inserts racing erases (mixed batches) and for two-choice
      // placement, whose choice depends on the moment's bucket loads.
      for (int attempt = 0; attempt < 256; ++attempt) {
        const Scan r = scan<true>(tv, c, K, h1, h2);
        if (r.stuck) return ST_TIMEOUT;
        if (r.found) {
          if (c.tl == 0) apply(tv, r.idx, op, V);
          return ST_FOUND;
        }
        if (!r.has_free) return ST_FULL;
        if (claim(tv, c, r, K, V)) {
          ++dcount;
          return ST_INSERTED;
        }
      }
      return ST_TIMEOUT;
    }
    const Hit h = find(tv, c, K, h1, h2);
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
    for (u32 tries = 0, ns = 0;;) {
      if (try_lock(tv, c, b0)) break;
      const Hit again = find(tv, c, K, h1, h2);
      if (again.found) {
        if (c.tl == 0) apply(tv, again.idx, op, V);
        return ST_FOUND;
      }
      if (++tries >= tv.spin_limit) return ST_TIMEOUT;
      backoff(c, ns);
    }
    u8 st = ST_TIMEOUT;
    for (int attempt = 0; attempt < 256; ++attempt) {
      const Scan r = scan(tv, c, K, h1, h2);
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
    unlock(tv, c, b0);
    return st;
  }

  __device__ static u8 do_erase(const TableView& tv, const TileCtx<T>& c, u64 K, u64& out,
                                int& dcount) {
    out = 0;
    if (is_sentinel(K)) return ST_BADKEY;
    const u64 h1 = fmix64(K ^ tv.seed1), h2 = fmix64(K ^ tv.seed2);
    for (int attempt = 0; attempt < 256; ++attempt) {
      const Hit h = find(tv, c, K, h1, h2);
      if (!h.found) return ST_MISS;
      int ok = 0;
      if (c.tl == 0) {
        ok = ptx::cas_slot(tv.slots + h.idx, K, h.val, KEY_TOMB, 0) ? 1 : 0;
        if (ok && META) ptx::st_tag_release(tv.tags + h.idx, TAG_TOMB);
      }
      if (c.shfl(ok, 0)) {
        out = h.val;
        --dcount;
        return ST_FOUND;
      }
    }
    return ST_TIMEOUT;
  }
};

// -------------------------------------------------------------------------
// The batch kernel.  Each warp takes chunks of 32 consecutive ops (grid
// stride); the chunk's keys/values/op codes are staged through shared memory
// with coalesced loads, tile t of the warp serves ops t*T .. t*T+T-1 of the
// chunk one after another, and results go back through shared memory as
// coalesced stores.  Count deltas are summed per block and added with one
// atomic per block.
// -------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int SCHEME, bool META, int B, int T, int KIND>
__global__ void __launch_bounds__(kThreads, 4) batch_kernel(TableView tv, BatchArgs a) {
  using Ops = TileOps<SCHEME, META, B, T>;
  __shared__ u64 s_key[kWarps][32];
  __shared__ u64 s_val[kWarps][32];
  __shared__ u64 s_out[kWarps][32];
  __shared__ u8 s_op[kWarps][32];
  __shared__ u8 s_st[kWarps][32];
  __shared__ long long s_cnt;

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  TileCtx<T> c;
  c.tl = lane & (T - 1);
  c.base = lane & ~(T - 1);
  c.mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << c.base);
  const int tile = lane / T;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();

  int dcount = 0;
  const u64 nchunks = (a.n + 31) / 32;
  const u64 stride = (u64)gridDim.x * kWarps;
  const int pf_method = (KIND == KIND_PROBE) ? 0 : (tv.prefetch & 3);
  const bool pf_lead = (tv.prefetch & 4) != 0;
  u64 ch = (u64)blockIdx.x * kWarps + w;
  const u64 ks = a.key_stride ? a.key_stride : 1;
  // keys of the chunk about to be staged (prefetched one chunk ahead with pf_lead)
  u64 next_key = 0;
  if (ch < nchunks) {
    const u64 gi0 = ch * 32 + lane;
    next_key = gi0 < a.n ? a.keys[gi0 * ks] : 0;
    if (pf_method && gi0 < a.n) Ops::prefetch_key(tv, next_key, pf_method);
  }
  for (; ch < nchunks; ch += stride) {
    const u64 base = ch * 32;
    const u64 gi = base + lane;
    const bool inb = gi < a.n;
    s_key[w][lane] = next_key;
    if (KIND == KIND_UPSERT || KIND == KIND_MIXED) s_val[w][lane] = (inb && a.vals) ? a.vals[gi * ks] : 0;
    if (KIND == KIND_MIXED) s_op[w][lane] = inb ? a.ops[gi] : 0;
    {
      const u64 nch = ch + stride;
      const u64 ngi = nch * 32 + lane;
      next_key = (nch < nchunks && ngi < a.n) ? a.keys[ngi * ks] : 0;
      if (pf_method && pf_lead && nch < nchunks && ngi < a.n) Ops::prefetch_key(tv, next_key, pf_method);
    }
    __syncwarp();
    const int cnt = (a.n - base) < 32 ? (int)(a.n - base) : 32;
    for (int jj = 0; jj < T; ++jj) {
      const int j = tile * T + jj;
      if (j >= cnt) break;
      const u64 K = s_key[w][j];
      u64 out = 0;
      u8 st;
      if (KIND == KIND_QUERY) {
        st = Ops::do_query(tv, c, K, out);
      } else if (KIND == KIND_PROBE) {
        st = Ops::do_probe(tv, c, K, out);
      } else if (KIND == KIND_UPSERT) {
        if ((a.flags & BATCH_SKIP_SENTINELS) && is_sentinel(K))
          st = ST_MISS;  // an empty / erased slot of the source table
        else
          st = Ops::template do_upsert<true>(tv, c, K, s_val[w][j], a.op, dcount);
      } else if (KIND == KIND_ERASE) {
        st = Ops::do_erase(tv, c, K, out, dcount);
      } else {
        const u8 code = s_op[w][j];
        switch (code) {
          case MX_QUERY: st = Ops::do_query(tv, c, K, out); break;
          case MX_INSERT: st = Ops::template do_upsert<false>(tv, c, K, s_val[w][j], OP_INSERT, dcount); break;
          case MX_ADD: st = Ops::template do_upsert<false>(tv, c, K, s_val[w][j], OP_ADD, dcount); break;
          case MX_MAX: st = Ops::template do_upsert<false>(tv, c, K, s_val[w][j], OP_MAX, dcount); break;
          case MX_REPLACE: st = Ops::template do_upsert<false>(tv, c, K, s_val[w][j], OP_REPLACE, dcount); break;
          case MX_ERASE: st = Ops::do_erase(tv, c, K, out, dcount); break;
          default: st = ST_BADKEY; break;
        }
      }
      if (c.tl == 0) {
        s_out[w][j] = out;
        s_st[w][j] = st;
        if (st >= ST_FULL) {
          u64* ctr = st == ST_FULL ? &tv.ctr->n_full : st == ST_TIMEOUT ? &tv.ctr->n_timeout : &tv.ctr->n_badkey;
          atomicAdd((unsigned long long*)ctr, 1ull);
        }
      }
    }
    __syncwarp();
    if (inb) {
      if (a.vals_out) a.vals_out[gi] = s_out[w][lane];
      if (a.status_out) a.status_out[gi] = s_st[w][lane];
    }
    __syncwarp();
  }
  if (KIND != KIND_QUERY && KIND != KIND_PROBE) {
    int mine = (c.tl == 0) ? dcount : 0;
    mine = __reduce_add_sync(0xffffffffu, mine);
    if (lane == 0 && mine) atomicAdd((unsigned long long*)&s_cnt, (unsigned long long)(long long)mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd((unsigned long long*)&tv.ctr->count, (unsigned long long)s_cnt);
  }
}

// Occupancy-sized grid-stride launch.  The kernel is a template argument so
// each instantiation caches its own occupancy.
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

}  // namespace ws
