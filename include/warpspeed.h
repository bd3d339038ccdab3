/*
 * warpspeed.h -- C ABI of a GB300-native (sm_103a) batched concurrent hash table.
 *
 * The operations follow the API of WarpSpeed (Pandey et al., arXiv 2509.16407),
 * §5.1 "Hash table API":
 *   Upsert(key, value, callback): insert the pair if the key is absent, otherwise
 *     run the callback on the stored value.  The empty callback is
 *     insert-if-unique; the atomicAdd callback accumulates.
 *   Query(key, &value): true and the value if the key is present.
 *   Erase(key): true if the key was present (and removes it); otherwise the
 *     table is unchanged.
 * Table designs (§2.2, §5): double hashing over 8-slot buckets (DoubleHT) and
 * power-of-two-choice over 32-slot buckets (P2HT), each optionally with a
 * 16-bit fingerprint per slot (the "(M)" metadata variants, §4.3).  Same-key
 * writers serialise on one lock bit of the key's primary bucket, held in an
 * external array (§4.1, §5 "Concurrency and metadata"); queries take no lock
 * and read each slot with one 128-bit load (§4.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Keys and values are uint64_t.  Keys 0 (EMPTY), 2^64-1 (TOMBSTONE) and
 *  2^64-2 (RESERVED) are sentinels: ops on them get the per-op status
 *  WS_FAIL_BADKEY and change nothing.
 *
 *  Batch buffers (keys, vals, ops, outputs) may be DEVICE pointers on the
 *  table's device (the fast path: kernels read them in place) or HOST pointers
 *  (pinned or pageable): the library then streams them through internal device
 *  staging buffers in chunks, overlapping copies with the kernels (see
 *  WS_OPT_HOST_DIRECT and WS_OPT_STAGE_CHUNK), and the
 *  outputs land in host memory once `stream` completes.  Buffers must be
 *  8-byte aligned (u64 arrays) and stay valid until `stream` completes.  The
 *  caller owns all batch buffers; the table owns its slot, tag, lock and
 *  staging memory and frees it in ws_destroy().
 *
 *  Every batch call is asynchronous on `stream` (a cudaStream_t; NULL = the
 *  legacy default stream).  One call is one phase: ops inside a call run
 *  concurrently; calls on one table must be ordered (same stream, or the
 *  caller synchronises).  Inside one call, queries observe the state at the
 *  start of the call for every key the call does not also write; for a
 *  mixed batch the keys of its query, erase and upsert classes must be
 *  disjoint (any overlap still leaves a valid linearisation for queries, but
 *  an erase and an upsert of one key in one batch is outside the contract).
 *
 *  Return value: argument and launch errors are reported immediately.
 *  Per-op failures (no free slot, lock timeout, sentinel key) do not fail
 *  the call: they are written to the optional per-op status array and
 *  counted in the table's device error counters (ws_last_error).
 *
 * Per-op status codes (uint8_t): WS_MISS 0, WS_FOUND 1, WS_INSERTED 2,
 *  WS_FAIL_FULL 3, WS_FAIL_BADKEY 4 (also an unknown mixed op code),
 *  WS_FAIL_TIMEOUT 5.
 */
#ifndef WARPSPEED_H
#define WARPSPEED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ws_table ws_table;       /* opaque; owned by the library */
typedef struct CUstream_st* ws_stream;  /* identical to cudaStream_t */

/* Probe schemes (§2.2): DOUBLE = double hashing over up to max_probe buckets;
 * P2 = two choices, primary bucket while below 3/4 full, else the less loaded;
 * ICEBERG = front yard / backyard (§2.2, split as in the table list of §5):
 * about 83% of the buckets form a front yard probed by single hashing, the
 * rest a backyard probed by two choices; a key goes to its front bucket while
 * that has a free slot, else to the less loaded of its two backyard buckets.
 * ICEBERG needs metadata (IcebergHT(M)) and at least 4 buckets. */
typedef enum { WS_DOUBLE = 0, WS_P2 = 1, WS_ICEBERG = 2 } ws_scheme;

/* Upsert callbacks of §5.1: ADD = atomicAdd (wrapping mod 2^64), MAX = u64 max,
 * REPLACE = overwrite, INSERT = the empty callback (insert-if-unique). */
typedef enum { WS_OP_ADD = 0, WS_OP_MAX = 1, WS_OP_REPLACE = 2, WS_OP_INSERT = 3 } ws_upsert_op;

/* Op codes of a mixed batch (ws_mixed). */
typedef enum {
  WS_MX_QUERY = 0, WS_MX_INSERT = 1, WS_MX_ADD = 2, WS_MX_MAX = 3, WS_MX_REPLACE = 4, WS_MX_ERASE = 5
} ws_mixed_op;

typedef enum {
  WS_OK = 0,
  WS_ERR_INVALID = 1,      /* bad argument (null table, bad size, misaligned, wrong device) */
  WS_ERR_INVALID_KEY = 2,  /* (ws_last_error) some op named a sentinel key */
  WS_ERR_OOM = 3,          /* device allocation failed */
  WS_ERR_FULL = 4,         /* (ws_last_error) some insert found no free slot */
  WS_ERR_TIMEOUT = 5,      /* (ws_last_error) some op hit the lock spin limit */
  WS_ERR_CUDA = 6          /* a CUDA call failed; see ws_cuda_error_string() */
} ws_status;

enum { WS_MISS = 0, WS_FOUND = 1, WS_INSERTED = 2, WS_FAIL_FULL = 3, WS_FAIL_BADKEY = 4,
       WS_FAIL_TIMEOUT = 5 };

/* Full configuration; ws_table_create() fills the paper's defaults (§5):
 *  DoubleHT: 8-slot buckets (one 128-byte line), tile 8; DoubleHT(M): 32-slot
 *  buckets, tile 4; P2HT: 32-slot buckets (four lines), tile 8; P2HT(M): 32,
 *  tile 4; IcebergHT(M): 32, tile 4.  bucket_slots in {8, 16, 32} (32 when
 *  metadata != 0); tile in {4, 8, 16, 32}.  max_probe = number of buckets a
 *  double-hashing probe sequence may visit (default 80, clamped to the bucket
 *  count); ignored by the other schemes.  The bucket count nb is capacity /
 *  bucket_slots rounded up to a power of two.  Iceberg splits it as
 *  nb_back = max(2, floor((17 nb + 50) / 100)) backyard buckets after
 *  nb_front = nb - nb_back front-yard buckets; a key's front bucket is
 *  floor(h1 nb_front / 2^64), its backyard buckets nb_front + floor(x nb_back /
 *  2^32) for x = the high and the low 32 bits of h2 (the second moved to the
 *  next backyard bucket, cyclically, when both coincide). */
typedef struct {
  uint64_t capacity;
  int32_t scheme;        /* ws_scheme */
  int32_t metadata;      /* 0 or 1 */
  int32_t bucket_slots;  /* 0 = default */
  int32_t tile;          /* 0 = default */
  uint32_t max_probe;    /* 0 = default (80) */
  uint32_t spin_limit;   /* lock attempts before WS_FAIL_TIMEOUT; 0 = default (65536, each a
                            lock-free re-probe plus <= 1 us back-off) */
  int32_t device;        /* -1 = current device */
  int32_t reserved;
} ws_config;

typedef struct {
  uint64_t slots;         /* total slots S = buckets * bucket_slots */
  uint64_t buckets;       /* nb (power of two) */
  uint64_t bucket_slots;  /* B */
  uint64_t tile;          /* T */
  uint64_t max_probe;     /* effective probe limit in buckets */
  uint64_t seed1, seed2;  /* hash seeds of h1, h2 */
  uint64_t bytes;         /* device bytes owned (slots + tags + locks + counters) */
  int32_t scheme, metadata, device, never_erased;
  uint64_t front_buckets; /* iceberg: front-yard buckets (the rest is the backyard); else nb */
} ws_table_info;

/* Create a table.  Slots start EMPTY.  Returns WS_ERR_OOM if device memory is
 * short (nothing is leaked), WS_ERR_INVALID for a bad configuration. */
ws_status ws_table_create(uint64_t capacity, ws_scheme scheme, int metadata, ws_table** out);
ws_status ws_table_create_ex(const ws_config* cfg, ws_table** out);
/* Frees all device memory of the table; synchronises the device first. */
ws_status ws_destroy(ws_table* t);
ws_status ws_table_info_get(const ws_table* t, ws_table_info* out);
/* Reset every slot to EMPTY (asynchronous on stream); counters are zeroed. */
ws_status ws_clear(ws_table* t, ws_stream stream);
/* Change the tile size used by later calls (4, 8, 16 or 32). */
ws_status ws_set_tile(ws_table* t, int tile);
ws_status ws_set_spin_limit(ws_table* t, uint32_t spins);

/* Tuning options (affect speed only, never results).
 *  WS_OPT_PRELOAD (default 1): the lane path -- each lane follows its op's
 *  probe sequence from bucket snapshots the warp copies into shared memory
 *  with asynchronous copies (the 128-byte line of a plain bucket, or the tag
 *  line and the first tag-matching slot), up to 32 probes per warp in flight
 *  per wave.  0 serves every op with the cooperative tiles and plain loads. */
/*  WS_OPT_PHASED (default 0): bulk-synchronous mode, the paper's "phased"
 *  tables of the concurrency-overhead benchmark (§6.2): query probes use weak
 *  L1-cacheable loads and absent-key inserts take no lock (inserts and erases
 *  still read through L2: they must see each other's claims).  Valid only for
 *  calls whose keys are distinct and whose probed slots nothing else writes
 *  during the call (e.g. a pure query batch, or inserts of distinct new
 *  keys); otherwise results are undefined. */
/*  WS_OPT_STREAM (default 1): single-table calls run "streaming lanes": each
 *  warp serves shares of the batch taken from a per-launch work ticket (so
 *  warps whose ops probe long take fewer; the shares shrink towards the end
 *  of the launch so the warps run dry together), a lane follows its op's probe
 *  sequence one bucket per wave and takes the next op as soon as its op
 *  settles; ops the lanes cannot settle go to the tiles.  0 serves 32-op
 *  chunks (lane waves, then tiles for what is left), as batched and serving
 *  launches always do, and as insert-if-unique calls on two-choice and
 *  iceberg tables do (their inserts lock: once per chunk beats once per wave).
 *  Queries and erases on two-choice tables with plain 32-slot buckets read
 *  whole buckets in 32-op chunks; 2 streams them too, reading a bucket line by
 *  line up to the key or the first EMPTY slot: fewer bytes for keys near the
 *  front of b_0, more dependent steps for misses (measured at 2^28 slots, 0.9
 *  load: positive queries 1.32 vs 1.47 ms, negative queries 3.53 vs 2.57 ms,
 *  erases 2.27 vs 1.66 ms per 2^24 ops), so it pays only for batches of hits.
 *  WS_OPT_LANE_WAVES (double hashing only; 0..255, 0 = default): buckets of a
 *  probe sequence the lane path follows, one per wave, before an op still
 *  open goes to the tiles.  Default: the whole sequence when streaming, 4 in
 *  32-op chunks. */
/*  WS_OPT_HOST_DIRECT (0..3, default 1): what a call does with host
 *  buffers that are page-locked and mapped into the device's address space
 *  (cudaHostAlloc / cudaMallocHost / cudaHostRegister memory with unified
 *  addressing).  0: every host buffer is staged through the table's device
 *  chunks (copy engines, eight chunk buffers rotating against the kernels).
 *  1: the kernels read keys, values and op codes in place over the host
 *  link; host result buffers are still staged.  2: results are written in
 *  place too.  3: 1 for insert-if-unique and erase calls (their probe
 *  sequences hide the host link's latency), 0 for queries, upserts and mixed
 *  batches (whose kernels are short per op and read inputs faster from
 *  device memory).  Pageable host memory is always staged.  The caller must
 *  not touch the buffers until the call's work on its stream has completed.
 *  Measured on a GB300 with its Grace host (2^28-slot tables, insert / query
 *  / upsert / erase of 13.4M / 2^24 ops per call, four designs, copies at
 *  about 200 GB/s each way): calls issued back to back run fastest with
 *  inputs read in place (9.26 Gops/s against 8.4-9.0 automatic and 8.6
 *  staged; device buffers 11.3), because staged copies then overlap the
 *  previous calls' kernels and compete with their memory traffic; calls
 *  timed one at a time run fastest automatic (a step of 30.2 ms against 34.0
 *  in place).  Results written in place cost most (scattered small writes
 *  over the host link). */
/*  WS_OPT_STAGE_CHUNK (16..24, default 22): log2 of the ops per chunk of the
 *  staging pipeline for host buffers (eight rotating chunk buffers per table,
 *  26 bytes per op each: 832 MiB at the default, allocated at the first
 *  host-buffer call; changing the size synchronises the table's last stream
 *  and frees them).  The staging copies of every table on a device run on
 *  one host-to-device and one device-to-host stream of that device, in the
 *  order the calls were issued. */
enum { WS_OPT_PRELOAD = 1, WS_OPT_PHASED = 2, WS_OPT_LANE_WAVES = 3, WS_OPT_STREAM = 4, WS_OPT_HOST_DIRECT = 5,
       WS_OPT_STAGE_CHUNK = 6 };
ws_status ws_set_option(ws_table* t, int option, int64_t value);

/* Insert-if-unique (§5.1 Upsert with the empty callback).  status_out: per-op
 * WS_INSERTED / WS_FOUND (already present, value kept) / WS_FAIL_*; nullable. */
ws_status ws_insert(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                    ws_stream stream);
ws_status ws_insert_ex(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                       uint8_t* status_out, ws_stream stream);

/* Upsert with callback op (§5.1).  Absent keys are inserted with their value;
 * present keys get the callback.  Duplicate keys in one batch: ADD and MAX
 * results are exact; REPLACE leaves one of the given values. */
ws_status ws_upsert(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                    ws_upsert_op op, ws_stream stream);
ws_status ws_upsert_ex(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                       ws_upsert_op op, uint8_t* status_out, ws_stream stream);

/* Query (§5.1).  vals_out[i] = value, or 0 on a miss; found_out (nullable) gets
 * the per-op status (WS_FOUND / WS_MISS / WS_FAIL_BADKEY).  Lock-free. */
ws_status ws_query(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint64_t n,
                   ws_stream stream);
ws_status ws_query_ex(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint8_t* found_out,
                      uint64_t n, ws_stream stream);

/* Erase (§5.1).  vals_out (nullable) gets the removed value (0 on a miss);
 * status_out (nullable) WS_FOUND / WS_MISS.  Duplicate keys in one batch:
 * exactly one reports WS_FOUND. */
ws_status ws_erase(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint64_t n,
                   ws_stream stream);
ws_status ws_erase_ex(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint8_t* status_out,
                      uint64_t n, ws_stream stream);

/* One kernel over an op-coded batch (ws_mixed_op per element), as in the
 * paper's aging benchmark where inserts, queries and removals of an iteration
 * run in one kernel (§6.4).  vals may be NULL when no op needs a value;
 * vals_out (nullable) gets query values / erased values (0 otherwise). */
ws_status ws_mixed(ws_table* t, const uint8_t* ops, const uint64_t* keys, const uint64_t* vals,
                   uint64_t* vals_out, uint8_t* status_out, uint64_t n, ws_stream stream);

/* Probe-count instrumentation (§5 "probe count", Table 1): for each key, the
 * memory a query of it touches on the current table, without changing the
 * table.  cost_out[i] = (cache lines << 32) | (32-byte DRAM sectors), counting
 * every bucket step (T slots of 16 B) and, with metadata, every 64-byte tag
 * read (2 sectors, 1 line) and every candidate slot read (1 sector, 1 line).
 * found_out (nullable) as in ws_query_ex.  Asynchronous on stream. */
ws_status ws_probe_cost(ws_table* t, const uint64_t* keys, uint64_t* cost_out, uint8_t* found_out, uint64_t n,
                        ws_stream stream);

/* Number of live keys.  Synchronises the table's last stream. */
ws_status ws_count(ws_table* t, uint64_t* out);

/* Per-op failure counters accumulated since creation/clear (synchronising).
 * Returns WS_OK if all are zero, else the most severe of WS_ERR_TIMEOUT,
 * WS_ERR_FULL, WS_ERR_INVALID_KEY.  Any pointer may be NULL. */
ws_status ws_last_error(ws_table* t, uint64_t* n_full, uint64_t* n_timeout, uint64_t* n_badkey);

/* Adversarial-benchmark hooks (§4.1): the bucket count, and each key's
 * primary bucket b_0 -- for iceberg its front-yard bucket -- computed on the
 * device (out: device or host u64[n]). */
ws_status ws_num_buckets(const ws_table* t, uint64_t* out);
ws_status ws_primary_bucket(ws_table* t, const uint64_t* keys, uint64_t* out, uint64_t n,
                            ws_stream stream);

/* Insert every live pair of src into dst (insert-if-unique), reading src's
 * slot array in place -- the growth step of a serving loop (allocate a larger
 * dst, rehash, destroy src).  src must not change meanwhile (its last stream
 * is synchronised first if it differs from stream).  status_out (nullable,
 * device u8[src slots]) gets WS_INSERTED / WS_FOUND / WS_FAIL_* per source slot
 * and WS_MISS for empty or erased source slots.  Asynchronous on stream. */
ws_status ws_rehash(ws_table* src, ws_table* dst, uint8_t* status_out, ws_stream stream);

/* Copy the slot array (S x {key, val}, 16 B each) and, for metadata tables,
 * the tag array (S x u16) to host memory.  Synchronising.  host_tags may be
 * NULL.  For layout checks and snapshots. */
ws_status ws_dump(ws_table* t, void* host_slots, void* host_tags);

/* Fault injection from the host: set (locked != 0) or clear every lock bit
 * with a memset.  With all bits set, ops that need a lock report
 * WS_FAIL_TIMEOUT after spin_limit attempts instead of hanging. */
ws_status ws_debug_fill_locks(ws_table* t, int locked, ws_stream stream);

/* ---------------------------------------------------------------------------
 * Batched mode: many tables and their op batches in one persistent kernel per
 * phase, captured once into a CUDA graph (a plan) and replayed with one launch.
 * Items of one phase run concurrently (the per-table phase contract holds per
 * phase); phases run in increasing order.  Every pointer must be a device
 * pointer on the tables' device (all tables on one device) and stay valid
 * while the plan exists; the plan copies the item list, so item arrays may be
 * rewritten in place between launches.  Tables whose (scheme, metadata, bucket,
 * tile) configuration is outside the compiled menu run as separate kernels in
 * the same graph (ws_batch_plan_info reports how many).  The plan owns its
 * descriptor, chunk and ticket arrays (allocated at create). */
typedef enum { WS_BK_INSERT = 0, WS_BK_UPSERT = 1, WS_BK_QUERY = 2, WS_BK_ERASE = 3 } ws_batch_kind;
typedef struct {
  ws_table* table;
  int32_t kind;   /* ws_batch_kind */
  int32_t op;     /* ws_upsert_op, for WS_BK_UPSERT */
  int32_t phase;  /* >= 0 */
  int32_t reserved;
  const uint64_t* keys;
  const uint64_t* vals;  /* insert / upsert */
  uint64_t* vals_out;    /* query / erase (nullable for erase) */
  uint8_t* status_out;   /* nullable */
  uint64_t n;
} ws_batch_item;
typedef struct ws_batch_plan ws_batch_plan;
ws_status ws_batch_plan_create(const ws_batch_item* items, uint64_t n_items, ws_batch_plan** out);
/* One graph launch on stream; asynchronous. */
ws_status ws_batch_plan_launch(ws_batch_plan* plan, ws_stream stream);
ws_status ws_batch_plan_info(const ws_batch_plan* plan, uint64_t* n_phases, uint64_t* n_chunks,
                             uint64_t* n_fallback_items);
/* Waits for the device, then frees the plan's device memory. */
ws_status ws_batch_plan_destroy(ws_batch_plan* plan);

/* Batched mode for callers that must not allocate device memory.  The paper
 * has no counterpart; this is an interface for callers that cannot call
 * cudaMalloc / cudaFree: code whose device memory is already held in full by a
 * caching allocator, code that reserved all memory up front, and latency-
 * critical loops that cannot take cudaFree's device-wide synchronisation.
 * Same items and semantics as a one-phase-at-a-time ws_batch_plan, run directly
 * (no graph), with the plan's scratch (descriptors, chunk map, work tickets)
 * kept in one fixed device array inside the library (~193 KiB on every GPU
 * that loads the library, held until exit) instead of allocated memory.
 * Limits: at most 1024 items and 16 distinct phases per call; larger calls
 * return WS_ERR_INVALID and ws_cuda_error_string() says why.  The first call
 * on a device looks up the array's device address.  Every call reuses the
 * array: calls whose work overlaps on the GPU race, so order them on one
 * stream.  Device pointers only. */
ws_status ws_batch_run_noalloc(const ws_batch_item* items, uint64_t n_items, ws_stream stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over device-resident tables.
 * A request is a mixed op batch (ws_mixed_op codes) on one table, with HOST
 * buffers (pinned recommended) that must stay valid until its completion is
 * polled.  A worker thread keeps up to max_inflight launches on the GPU; each
 * launch runs the waiting requests of distinct tables (per-table FIFO, oldest
 * first, at most one request per table in flight) in one persistent
 * multi-table kernel.  Each result therefore equals that of replaying its
 * table's requests alone in arrival order.  Tables are admitted only while
 * free device memory (counting memory the device's default stream-ordered
 * pool holds unused) stays above hbm_headroom of the total; a table about to
 * pass grow_at load is rehashed into one twice as large when memory admits
 * it.  Creating a server sets the default pool's release threshold to keep
 * freed memory (grown-out tables) pooled for later growth.  plain = 1 serves one request per launch, one launch at a time (the
 * per-request baseline). */
typedef struct ws_server ws_server;
typedef struct {
  int32_t device;           /* -1 = current */
  int32_t max_inflight;     /* launches in flight (default 4) */
  uint64_t max_batch_ops;   /* ops per launch and per request (default 2^22) */
  uint32_t max_batch_reqs;  /* requests per launch (default 256) */
  int32_t plain;            /* 1: per-request launches, one at a time */
  double hbm_headroom;      /* fraction of device memory kept free (default 0.05) */
  double grow_at;           /* load that triggers growth; 0 = never grow */
} ws_server_config;
typedef struct {
  uint32_t table;  /* id from ws_server_add_table */
  uint32_t reserved;
  const uint8_t* ops;
  const uint64_t* keys;
  const uint64_t* vals;  /* nullable: values 0 */
  uint64_t* vals_out;    /* nullable */
  uint8_t* status_out;   /* nullable */
  uint64_t n;
  uint64_t tag;          /* returned in the completion */
} ws_request;
typedef struct {
  uint64_t id, tag;
  double t_submit, t_start, t_done;  /* seconds on the steady clock */
  int32_t status;
  uint32_t table;
} ws_completion;
ws_status ws_server_create(const ws_server_config* cfg, ws_server** out);
/* WS_ERR_OOM when free device memory does not admit the table. */
ws_status ws_server_add_table(ws_server* s, uint64_t capacity, ws_scheme scheme, int metadata, int tile,
                              uint32_t* id);
/* Thread-safe; returns at once.  n <= max_batch_ops. */
ws_status ws_server_submit(ws_server* s, const ws_request* r, uint64_t* id);
/* Up to max completions (waits up to wait_ms for the first). */
ws_status ws_server_poll(ws_server* s, ws_completion* out, uint64_t max, uint64_t* n_out, int wait_ms);
/* Stop (paused != 0) or resume admitting requests into new launches; work
 * already on the GPU continues.  Lets a caller queue a burst first. */
ws_status ws_server_pause(ws_server* s, int paused);
/* Resumes a paused server, then blocks until every submitted request has
 * completed. */
ws_status ws_server_drain(ws_server* s);
/* The current table behind an id (changes when the table grows). */
ws_status ws_server_table(ws_server* s, uint32_t id, ws_table** out);
ws_status ws_server_stats(ws_server* s, uint64_t* submitted, uint64_t* completed, uint64_t* launches,
                          uint64_t* grows);
/* Finishes queued work, then frees the server and its tables. */
ws_status ws_server_destroy(ws_server* s);

/* ---------------------------------------------------------------------------
 * Measurement helper (not an operation of the paper): the read bandwidth of
 * the running GPU for the roofline's denominators -- for tables that fit in
 * L2 the relevant peak is L2 bandwidth, not HBM.  Allocates a buffer of
 * `bytes` (>= 1 MiB, a multiple of 128) on `device` (-1 = current), reads it
 * once to warm it, then times `passes` further reads with CUDA events, five
 * times, and stores the best rate in *gbs_out (10^9 bytes per second, bytes
 * moved / elapsed).  pattern 0: sequential 16-byte loads at a grid stride;
 * 1, 2, 3: random 128-, 64- and 32-byte blocks, each read by 8, 4 or 2 lanes
 * together as a bucket snapshot is (the probes' access pattern); 4, 5: random
 * 32- and 128-byte blocks written; 6, 7: a metadata probe's pair of dependent
 * reads, a random 64-byte tag line then a 16-byte slot chosen from its data,
 * with tags and slots in separate arrays (6) or each bucket's tag line and 32
 * slots in one 640-byte block (7), rated at 80 bytes per pair; 8-11: random
 * 128-byte reads confined to regions of 128 KiB, 512 KiB, 2 MiB or 8 MiB, each
 * block of threads reading 8 x depth lines per group of lanes in one region
 * before it moves to another.  depth (1, 2, 4 or 8): independent random
 * blocks (pairs) each group of lanes keeps in flight (ignored by pattern 0; 6
 * and 7 run 2 or 4).  Accesses
 * bypass L1 (.cg), so a buffer smaller than L2 measures L2.  Synchronous;
 * frees the buffer.  WS_ERR_OOM when the buffer cannot be allocated. */
ws_status ws_read_bandwidth(uint64_t bytes, int pattern, int depth, int passes, int device, double* gbs_out);

/* Text of the last CUDA error seen by this library on the calling thread. */
const char* ws_cuda_error_string(void);
const char* ws_status_string(ws_status s);
/* Library version, e.g. 0x000100 for 0.1.0. */
uint32_t ws_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WARPSPEED_H */
