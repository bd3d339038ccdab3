// ws_oracle.cpp -- the CPU oracle for the batched hash-table path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
// this file; only the tests, __graft_entry__.smoke() and bench.py's CPU
// baseline leg load it.  It shares no code, header, constant generator or
// helper with the CUDA path.
//
// What it computes.  The method of the paper (WarpSpeed, §5.1 "Hash table
// API") is a concurrent map: Upsert(key, value, callback), Query(key, &value)
// and Erase(key).  Whatever the bucket layout, probe scheme, tile size or
// metadata, the map contents after a batch are fixed by the map semantics
// alone, so the oracle is that plain definition: a std::unordered_map applied
// batch by batch, single-threaded, with these per-batch phase rules:
//
//   * insert(k, v): insert-if-unique, i.e. Upsert with the empty callback
//     (§5.1): if k is absent, M[k] = v; otherwise nothing changes.
//   * upsert add/max/replace: absent -> M[k] = v; present -> callback
//     (add = the atomicAdd callback of §5.1, wrapping mod 2^64; max; replace).
//   * query(k): (found, M[k]) -- §5.1 Query; a miss reports value 0.
//   * erase(k): returns whether k was present and removes it; a miss leaves
//     the map unchanged (§5.1 Erase).
//   * mixed batch: the query, erase and upsert classes of one batch touch
//     disjoint keys (the phase contract); queries observe the state at batch
//     start, then erases, then upserts/inserts apply, each class in index
//     order.
//   * Keys 0, 2^64-1 and 2^64-2 are reserved sentinel keys (empty, tombstone,
//     reservation marker of §4.2) and are rejected with status BAD_KEY.
//
// Per-op status codes (the documented values of the library's interface):
//   0 MISS, 1 FOUND (query hit / erase hit / upsert updated an existing key /
//   insert found the key present), 2 INSERTED (new key), 3 FULL, 4 BAD_KEY,
//   5 TIMEOUT.  The oracle never produces FULL or TIMEOUT: a map has no
//   capacity and no locks.
//
// The layout checker at the end is a separate routine that re-derives, from
// the written hash/probe specification only, where a key may legally sit in a
// dumped table, and checks the structural invariants the paper relies on:
// one copy per key (§4.1 adversarial benchmark), stability/legal placement
// (§2.1, §2.2), lossless metadata -- every tag equals the key's fingerprint
// (§4.3), and the double-hashing early-exit property.
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>
#include <algorithm>

namespace {

const uint64_t K_EMPTY = 0ull;
const uint64_t K_TOMB = ~0ull;
const uint64_t K_RESV = ~0ull - 1ull;

enum { ST_MISS = 0, ST_FOUND = 1, ST_INSERTED = 2, ST_FULL = 3, ST_BADKEY = 4, ST_TIMEOUT = 5 };
enum { UP_INSERT = -1, UP_ADD = 0, UP_MAX = 1, UP_REPLACE = 2 };
// mixed-batch op codes (documented interface values)
enum { MX_QUERY = 0, MX_INSERT = 1, MX_ADD = 2, MX_MAX = 3, MX_REPLACE = 4, MX_ERASE = 5 };

bool is_sentinel(uint64_t k) { return k == K_EMPTY || k == K_TOMB || k == K_RESV; }

struct Map {
  std::unordered_map<uint64_t, uint64_t> m;
};

uint8_t apply_upsert(Map* M, uint64_t k, uint64_t v, int op) {
  if (is_sentinel(k)) return ST_BADKEY;
  auto it = M->m.find(k);
  if (it == M->m.end()) {
    M->m.emplace(k, v);
    return ST_INSERTED;
  }
  switch (op) {
    case UP_INSERT: break;                                   // f(){return;}
    case UP_ADD: it->second = it->second + v; break;         // wraps mod 2^64
    case UP_MAX: if (v > it->second) it->second = v; break;
    case UP_REPLACE: it->second = v; break;
  }
  return ST_FOUND;
}

uint8_t apply_query(const Map* M, uint64_t k, uint64_t* out) {
  *out = 0;
  if (is_sentinel(k)) return ST_BADKEY;
  auto it = M->m.find(k);
  if (it == M->m.end()) return ST_MISS;
  *out = it->second;
  return ST_FOUND;
}

uint8_t apply_erase(Map* M, uint64_t k, uint64_t* out) {
  *out = 0;
  if (is_sentinel(k)) return ST_BADKEY;
  auto it = M->m.find(k);
  if (it == M->m.end()) return ST_MISS;
  *out = it->second;
  M->m.erase(it);
  return ST_FOUND;
}

}  // namespace

extern "C" {

void* ora_new(void) { return new Map(); }
void ora_free(void* h) { delete static_cast<Map*>(h); }
uint64_t ora_count(void* h) { return static_cast<Map*>(h)->m.size(); }
void ora_clear(void* h) { static_cast<Map*>(h)->m.clear(); }

// op: -1 insert-if-unique, 0 add, 1 max, 2 replace.  status may be null.
void ora_upsert(void* h, const uint64_t* keys, const uint64_t* vals, uint64_t n, int op,
                uint8_t* status) {
  Map* M = static_cast<Map*>(h);
  for (uint64_t i = 0; i < n; ++i) {
    uint8_t s = apply_upsert(M, keys[i], vals[i], op);
    if (status) status[i] = s;
  }
}

void ora_insert(void* h, const uint64_t* keys, const uint64_t* vals, uint64_t n, uint8_t* status) {
  ora_upsert(h, keys, vals, n, UP_INSERT, status);
}

// vals_out and status may be null.
void ora_query(void* h, const uint64_t* keys, uint64_t* vals_out, uint8_t* status, uint64_t n) {
  const Map* M = static_cast<const Map*>(h);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t v;
    uint8_t s = apply_query(M, keys[i], &v);
    if (vals_out) vals_out[i] = v;
    if (status) status[i] = s;
  }
}

void ora_erase(void* h, const uint64_t* keys, uint64_t* vals_out, uint8_t* status, uint64_t n) {
  Map* M = static_cast<Map*>(h);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t v;
    uint8_t s = apply_erase(M, keys[i], &v);
    if (vals_out) vals_out[i] = v;
    if (status) status[i] = s;
  }
}

// Mixed batch: queries see the batch-start state, then erases, then upserts.
// Unknown op codes get status BAD_KEY and do nothing (the library rejects them
// the same way).
void ora_mixed(void* h, const uint8_t* ops, const uint64_t* keys, const uint64_t* vals,
               uint64_t* vals_out, uint8_t* status, uint64_t n) {
  Map* M = static_cast<Map*>(h);
  for (uint64_t i = 0; i < n; ++i) {
    if (ops[i] != MX_QUERY) continue;
    uint64_t v;
    uint8_t s = apply_query(M, keys[i], &v);
    if (vals_out) vals_out[i] = v;
    if (status) status[i] = s;
  }
  for (uint64_t i = 0; i < n; ++i) {
    if (ops[i] != MX_ERASE) continue;
    uint64_t v;
    uint8_t s = apply_erase(M, keys[i], &v);
    if (vals_out) vals_out[i] = v;
    if (status) status[i] = s;
  }
  for (uint64_t i = 0; i < n; ++i) {
    int op;
    switch (ops[i]) {
      case MX_INSERT: op = UP_INSERT; break;
      case MX_ADD: op = UP_ADD; break;
      case MX_MAX: op = UP_MAX; break;
      case MX_REPLACE: op = UP_REPLACE; break;
      case MX_QUERY: case MX_ERASE: continue;
      default:
        if (vals_out) vals_out[i] = 0;
        if (status) status[i] = ST_BADKEY;
        continue;
    }
    uint8_t s = apply_upsert(M, keys[i], vals[i], op);
    if (vals_out) vals_out[i] = 0;
    if (status) status[i] = s;
  }
}

// Contents sorted by key; caller provides count() entries of room.
void ora_items(void* h, uint64_t* keys_out, uint64_t* vals_out) {
  Map* M = static_cast<Map*>(h);
  std::vector<std::pair<uint64_t, uint64_t>> v(M->m.begin(), M->m.end());
  std::sort(v.begin(), v.end());
  for (size_t i = 0; i < v.size(); ++i) {
    keys_out[i] = v[i].first;
    vals_out[i] = v[i].second;
  }
}

// Bulk-load from arrays (used to rebuild a state for a later batch).
void ora_load(void* h, const uint64_t* keys, const uint64_t* vals, uint64_t n) {
  Map* M = static_cast<Map*>(h);
  for (uint64_t i = 0; i < n; ++i) M->m[keys[i]] = vals[i];
}

// ---------------------------------------------------------------------------
// Layout checker.  Works on a host copy of the table's slot array (S slots of
// {key u64, val u64}) and, for fingerprint tables, its tag array (S x u16).
//
// Hash/probe specification it re-derives (written independently of the CUDA
// path from the specification in the design notes; the paper does not fix
// the hash functions):
//   fmix(x)  = MurmurHash3 64-bit finalizer: x ^= x>>33; x *= ff51afd7ed558ccd;
//              x ^= x>>33; x *= c4ceb9fe1a85ec53; x ^= x>>33.
//   h1 = fmix(k ^ seed1), h2 = fmix(k ^ seed2).
//   double hashing (§2.2):  b_i = (h1 + i*(h2|1)) mod nb,  i < P.
//   two choice (§2.2):      b_0 = h1 mod nb, b_1 = h2 mod nb, and b_1 = b_0+1
//                           mod nb when they coincide (nb > 1).
//   iceberg (§2.2 front yard / backyard; 83% / 17% as listed in §5):
//                           nb_back = max(2, floor((17 nb + 50) / 100)) buckets
//                           follow nb_front = nb - nb_back front buckets;
//                           front = floor(h1 nb_front / 2^64);
//                           back_j = nb_front + floor(x_j nb_back / 2^32) with
//                           x_1 = high 32 bits of h2, x_2 = low 32 bits; back_2
//                           moves to the next backyard bucket (cyclic) when the
//                           two coincide.  A key sits in the backyard only if
//                           its front bucket was full when it was placed, so a
//                           backyard key never has an EMPTY slot in its front.
//   tag(k) = k & 0xffff, moved up by 2 when below 2 (0 = empty, 1 = tombstone),
//   following §5 "Concurrency and metadata" (low 16 bits as the fingerprint).
// ---------------------------------------------------------------------------

namespace {
uint64_t fmix(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}
uint16_t spec_tag(uint64_t k) {
  uint16_t t = (uint16_t)(k & 0xffffu);
  return t < 2 ? (uint16_t)(t + 2) : t;
}
// Iceberg geometry: the three candidate buckets of a key (front, back_1, back_2).
struct IcebergBuckets {
  uint64_t front, back1, back2;
};
IcebergBuckets iceberg_buckets(uint64_t nb, uint64_t h1, uint64_t h2) {
  uint64_t n_back = (17 * nb + 50) / 100;
  if (n_back < 2) n_back = 2;
  const uint64_t n_front = nb - n_back;
  IcebergBuckets r;
  r.front = (uint64_t)(((unsigned __int128)h1 * n_front) >> 64);
  const uint64_t x1 = h2 >> 32, x2 = h2 & 0xffffffffull;
  const uint64_t c1 = (x1 * n_back) >> 32;
  uint64_t c2 = (x2 * n_back) >> 32;
  if (c2 == c1) c2 = (c1 + 1) % n_back;
  r.back1 = n_front + c1;
  r.back2 = n_front + c2;
  return r;
}
}  // namespace

struct ora_layout_report {
  uint64_t live, tomb, empty, resv;
  uint64_t bad_bucket;        // live key outside its legal buckets
  uint64_t duplicates;        // extra copies of a key
  uint64_t tag_mismatch;      // tag != fingerprint, or empty/tomb tag/key disagree
  uint64_t early_exit;        // double hashing: live key behind a bucket with an empty slot
  uint64_t empty_not_suffix;  // an occupied slot after an empty one inside a bucket
};

// scheme: 0 double hashing, 1 two-choice, 2 iceberg.  tags may be null (no metadata).
int ora_layout_check(const uint64_t* slots /* 2*S words */, const uint16_t* tags, uint64_t nb,
                     uint64_t B, int scheme, uint64_t pmax, uint64_t seed1, uint64_t seed2,
                     ora_layout_report* r) {
  std::memset(r, 0, sizeof(*r));
  if (nb == 0 || (nb & (nb - 1)) != 0 || B == 0) return -1;
  const uint64_t mask = nb - 1;
  std::unordered_set<uint64_t> seen;
  for (uint64_t b = 0; b < nb; ++b) {
    bool empty_seen = false;
    for (uint64_t j = 0; j < B; ++j) {
      const uint64_t s = b * B + j;
      const uint64_t k = slots[2 * s];
      // With metadata the tag array owns occupancy: tag 0 = empty, 1 = tomb.
      bool occupied;
      if (tags) {
        const uint16_t t = tags[s];
        if (t == 0) {
          occupied = false;
          ++r->empty;
          if (k != K_EMPTY) ++r->tag_mismatch;
          empty_seen = true;
          continue;
        }
        if (t == 1) {
          ++r->tomb;
          if (k != K_TOMB) ++r->tag_mismatch;
          if (empty_seen) ++r->empty_not_suffix;
          continue;
        }
        occupied = true;
        if (k == K_EMPTY || k == K_TOMB || k == K_RESV) { ++r->tag_mismatch; continue; }
        if (t != spec_tag(k)) ++r->tag_mismatch;
      } else {
        if (k == K_EMPTY) { ++r->empty; empty_seen = true; continue; }
        if (k == K_TOMB) { ++r->tomb; if (empty_seen) ++r->empty_not_suffix; continue; }
        if (k == K_RESV) { ++r->resv; if (empty_seen) ++r->empty_not_suffix; continue; }
        occupied = true;
      }
      (void)occupied;
      if (empty_seen) ++r->empty_not_suffix;
      ++r->live;
      if (!seen.insert(k).second) ++r->duplicates;
      const uint64_t h1 = fmix(k ^ seed1), h2 = fmix(k ^ seed2);
      bool legal = false;
      if (scheme == 0) {
        const uint64_t P = pmax < nb ? pmax : nb;
        const uint64_t step = h2 | 1ull;
        for (uint64_t i = 0; i < P; ++i) {
          const uint64_t bi = (h1 + i * step) & mask;
          if (bi == b) { legal = true; break; }
          // Every bucket before the key's bucket on its sequence must have
          // had no empty slot when the key was placed; empties never return.
          bool has_empty = false;
          for (uint64_t q = 0; q < B; ++q) {
            const uint64_t sq = bi * B + q;
            if (tags ? tags[sq] == 0 : slots[2 * sq] == K_EMPTY) { has_empty = true; break; }
          }
          if (has_empty) { ++r->early_exit; break; }
        }
      } else if (scheme == 2) {
        const IcebergBuckets ib = iceberg_buckets(nb, h1, h2);
        legal = (b == ib.front) || (b == ib.back1) || (b == ib.back2);
        if (legal && b != ib.front) {
          for (uint64_t q = 0; q < B; ++q) {
            const uint64_t sq = ib.front * B + q;
            if (tags ? tags[sq] == 0 : slots[2 * sq] == K_EMPTY) { ++r->early_exit; break; }
          }
        }
      } else {
        const uint64_t b0 = h1 & mask;
        uint64_t b1 = h2 & mask;
        if (b1 == b0) b1 = (b0 + 1) & mask;
        legal = (b == b0) || (b == b1);
      }
      if (!legal) ++r->bad_bucket;
    }
  }
  return 0;
}

// For each key, reports 1 if every slot of every bucket it may occupy is taken
// (live or reserved), 0 otherwise.  Used to validate inserts the table
// reported as FULL.
void ora_candidates_full(const uint64_t* slots, const uint16_t* tags, uint64_t nb, uint64_t B,
                         int scheme, uint64_t pmax, uint64_t seed1, uint64_t seed2,
                         const uint64_t* keys, uint64_t n, uint8_t* full_out) {
  const uint64_t mask = nb - 1;
  auto bucket_full = [&](uint64_t b) {
    for (uint64_t q = 0; q < B; ++q) {
      const uint64_t s = b * B + q;
      if (tags) {
        if (tags[s] < 2) return false;
      } else {
        const uint64_t k = slots[2 * s];
        if (k == K_EMPTY || k == K_TOMB) return false;
      }
    }
    return true;
  };
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = keys[i];
    const uint64_t h1 = fmix(k ^ seed1), h2 = fmix(k ^ seed2);
    bool all = true;
    if (scheme == 0) {
      const uint64_t P = pmax < nb ? pmax : nb;
      for (uint64_t j = 0; j < P && all; ++j) all = bucket_full((h1 + j * (h2 | 1ull)) & mask);
    } else if (scheme == 2) {
      const IcebergBuckets ib = iceberg_buckets(nb, h1, h2);
      all = bucket_full(ib.front) && bucket_full(ib.back1) && bucket_full(ib.back2);
    } else {
      const uint64_t b0 = h1 & mask;
      uint64_t b1 = h2 & mask;
      if (b1 == b0) b1 = (b0 + 1) & mask;
      all = bucket_full(b0) && bucket_full(b1);
    }
    full_out[i] = all ? 1 : 0;
  }
}

// Probe count (§5 "probe count", Table 1) recounted on a dumped table: the
// memory a query of each key touches, per the cost model the library
// documents for ws_probe_cost.  The query reads buckets along the key's
// candidate sequence in tile steps of `tile` consecutive 16-byte slots:
//   * plain buckets: a tile of T <= B lanes reads a bucket in B/T steps of T
//     slots (T/2 sectors, ceil(16T/128) lines each); a tile of T > B lanes
//     reads T/B buckets of the sequence side by side in one step (B/2
//     sectors and one line per bucket in range).  The scan of a key stops at
//     the step holding the key, and after a step in which some slot is EMPTY
//     it leaves the bucket (EMPTY slots form a suffix: nothing follows them);
//   * double hashing (§2.2) stops there for good -- an EMPTY slot means the
//     key was never placed further on -- and otherwise visits at most pmax
//     buckets (clamped to nb);
//   * two choice (§2.2) reads b_0, then b_1, except that a table that has
//     never seen an erase skips b_1 once b_0 holds fewer than 3B/4 live keys
//     (the placement shortcut makes b_1 unused then);
//   * fingerprint buckets (§4.3): the 64-byte tag line of the bucket (2
//     sectors, 1 line), then each slot whose tag equals tag(k), in slot order,
//     until the key (1 sector and 1 line each).  Double hashing stops after a
//     bucket with an EMPTY tag; iceberg after a front bucket with an EMPTY
//     tag; two choice as above with the occupancy counted on the tags.
// cost_out[i] = (lines << 32) | sectors; found_out[i] = 1 when k is present.
// Sentinel keys get cost 0 and found 0.  Returns -1 on a bad geometry.
int ora_probe_cost(const uint64_t* slots, const uint16_t* tags, uint64_t nb, uint64_t B, int scheme,
                   uint64_t pmax, uint64_t seed1, uint64_t seed2, uint64_t tile, int never_erased,
                   const uint64_t* keys, uint64_t n, uint64_t* cost_out, uint8_t* found_out) {
  if (nb == 0 || (nb & (nb - 1)) != 0 || B == 0 || tile == 0) return -1;
  if (tags && B != 32) return -1;
  const uint64_t mask = nb - 1;
  const uint64_t fill_shortcut = 3 * B / 4;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = keys[i];
    cost_out[i] = 0;
    if (found_out) found_out[i] = 0;
    if (is_sentinel(k)) continue;
    const uint64_t h1 = fmix(k ^ seed1), h2 = fmix(k ^ seed2);
    // the candidate buckets, in probe order
    std::vector<uint64_t> seq;
    if (scheme == 0) {
      const uint64_t P = pmax < nb ? pmax : nb;
      for (uint64_t j = 0; j < P; ++j) seq.push_back((h1 + j * (h2 | 1ull)) & mask);
    } else if (scheme == 2) {
      const IcebergBuckets ib = iceberg_buckets(nb, h1, h2);
      seq = {ib.front, ib.back1, ib.back2};
    } else {
      const uint64_t b0 = h1 & mask;
      seq.push_back(b0);
      if (nb > 1) {
        uint64_t b1 = h2 & mask;
        if (b1 == b0) b1 = (b0 + 1) & mask;
        seq.push_back(b1);
      }
    }
    uint64_t lines = 0, sectors = 0;
    bool found = false;
    if (tags) {
      const uint16_t kt = spec_tag(k);
      for (size_t j = 0; j < seq.size() && !found; ++j) {
        const uint64_t b = seq[j];
        sectors += 2;
        lines += 1;
        bool has_empty = false;
        uint64_t live = 0;
        for (uint64_t q = 0; q < 32; ++q) {
          const uint16_t t = tags[b * 32 + q];
          if (t == 0) has_empty = true;
          if (t >= 2) ++live;
        }
        for (uint64_t q = 0; q < 32 && !found; ++q) {
          if (tags[b * 32 + q] != kt) continue;
          sectors += 1;
          lines += 1;
          if (slots[2 * (b * 32 + q)] == k) found = true;
        }
        if (found) break;
        if (scheme == 0 && has_empty) break;
        if (scheme == 2 && j == 0 && has_empty) break;
        if (scheme == 1 && j == 0 && never_erased && live < fill_shortcut) break;
      }
    } else {
      const uint64_t G = tile > B ? tile / B : 1;          // buckets per step
      const uint64_t W = tile > B ? B : tile;              // slots of a bucket per step
      const uint64_t step_lines = (W * 16 + 127) / 128;
      for (size_t j = 0; j < seq.size() && !found; j += G) {
        const uint64_t nact = std::min<uint64_t>(G, seq.size() - j);
        bool ended = false;
        uint64_t live0 = 0;
        for (uint64_t s = 0; s * W < B; ++s) {
          sectors += nact * (W / 2);
          lines += nact * step_lines;
          bool empty_here = false;
          for (uint64_t g = 0; g < nact; ++g) {
            const uint64_t b = seq[j + g];
            for (uint64_t q = s * W; q < (s + 1) * W; ++q) {
              const uint64_t kq = slots[2 * (b * B + q)];
              if (kq == k) found = true;
              if (kq == K_EMPTY) empty_here = true;
              if (kq != K_EMPTY && kq != K_TOMB) ++live0;
            }
          }
          if (found) break;
          if (empty_here) {
            ended = true;
            break;
          }
        }
        if (found) break;
        if (scheme == 0 && ended) break;
        if (scheme == 1 && G == 1 && j == 0 && never_erased && live0 < fill_shortcut) break;
      }
    }
    cost_out[i] = (lines << 32) | sectors;
    if (found_out) found_out[i] = found ? 1 : 0;
  }
  return 0;
}

// Primary bucket (b_0) under the specification; the adversarial benchmark of
// §4.1 needs it on the host to build keys with a chosen primary bucket.
void ora_primary_bucket(const uint64_t* keys, uint64_t n, uint64_t nb, uint64_t seed1,
                        uint64_t* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = fmix(keys[i] ^ seed1) & (nb - 1);
}

// Iceberg candidate buckets (front, back_1, back_2) of each key, 3 per key.
void ora_iceberg_buckets(const uint64_t* keys, uint64_t n, uint64_t nb, uint64_t seed1, uint64_t seed2,
                         uint64_t* out) {
  for (uint64_t i = 0; i < n; ++i) {
    const IcebergBuckets ib = iceberg_buckets(nb, fmix(keys[i] ^ seed1), fmix(keys[i] ^ seed2));
    out[3 * i] = ib.front;
    out[3 * i + 1] = ib.back1;
    out[3 * i + 2] = ib.back2;
  }
}

}  // extern "C"
