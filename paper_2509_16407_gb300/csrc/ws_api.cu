// ws_api.cu -- the C ABI declared in include/warpspeed.h: table lifetime,
// argument checking, kernel dispatch, and the host-buffer staging pipeline.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "ws_internal.h"

namespace wsi {

thread_local char g_cuda_err[256] = "no error";

void note_cuda(cudaError_t e, const char* where) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
}

void note_text(const char* msg) { std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", msg); }

}  // namespace wsi

using namespace wsi;

namespace {

constexpr u64 kSeed1 = 0x243f6a8885a308d3ull;  // hex digits of pi: fixed, documented seeds
constexpr u64 kSeed2 = 0x13198a2e03707344ull;
constexpr uint32_t kDefaultProbe = 80;
constexpr uint32_t kDefaultSpin = 1u << 16;  // attempts; each costs a probe + <= 1 us back-off
constexpr int kDefaultPreload = 1;  // the lane path (see WS_OPT_PRELOAD)

}  // namespace

namespace {

void free_staging(Staging* s) {
  for (int b = 0; b < Staging::kBufs; ++b) {
    if (s->keys[b]) cudaFree(s->keys[b]);
    if (s->vals[b]) cudaFree(s->vals[b]);
    if (s->out[b]) cudaFree(s->out[b]);
    if (s->ops[b]) cudaFree(s->ops[b]);
    if (s->st[b]) cudaFree(s->st[b]);
    if (s->in_ready[b]) cudaEventDestroy(s->in_ready[b]);
    if (s->k_done[b]) cudaEventDestroy(s->k_done[b]);
    if (s->out_done[b]) cudaEventDestroy(s->out_done[b]);
  }
  delete s;  // the copy streams are the device's, shared by every table
}

// One H2D and one D2H copy stream per device, shared by every table's
// staging, so that copies run in the order the calls were issued.
bool shared_copy_streams(int device, cudaStream_t* h2d, cudaStream_t* d2h) {
  static std::mutex mu;
  static std::map<int, std::pair<cudaStream_t, cudaStream_t>> streams;
  std::lock_guard<std::mutex> lock(mu);
  auto it = streams.find(device);
  if (it == streams.end()) {
    cudaStream_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
      cudaStreamDestroy(a);
      return false;
    }
    it = streams.emplace(device, std::make_pair(a, b)).first;
  }
  *h2d = it->second.first;
  *d2h = it->second.second;
  return true;
}

ws_status free_table_memory(ws_table* t) {
  if (t->tv.slots) cudaFree(t->tv.slots);
  if (t->tv.tags) cudaFree(t->tv.tags);
  if (t->tv.locks) cudaFree(t->tv.locks);
  if (t->tv.ctr) cudaFree(t->tv.ctr);
  if (t->stage) {
    free_staging(t->stage);
    t->stage = nullptr;
  }
  t->tv.slots = nullptr;
  t->tv.tags = nullptr;
  t->tv.locks = nullptr;
  t->tv.ctr = nullptr;
  return WS_OK;
}

// Allocates the staging buffers on first use; on any failure nothing is kept.
ws_status ensure_staging(ws_table* t) {
  if (t->stage) return WS_OK;
  Staging* s = new (std::nothrow) Staging();
  if (!s) return WS_ERR_OOM;
  s->cap = 1ull << t->stage_log2;
  bool ok = true;
  for (int b = 0; b < Staging::kBufs && ok; ++b) {
    ok = cudaMalloc(&s->keys[b], s->cap * 8) == cudaSuccess && cudaMalloc(&s->vals[b], s->cap * 8) == cudaSuccess &&
         cudaMalloc(&s->out[b], s->cap * 8) == cudaSuccess && cudaMalloc(&s->ops[b], s->cap) == cudaSuccess &&
         cudaMalloc(&s->st[b], s->cap) == cudaSuccess;
    if (!ok) break;
    ok = cudaEventCreateWithFlags(&s->in_ready[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->k_done[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->out_done[b], cudaEventDisableTiming) == cudaSuccess;
  }
  if (ok) ok = shared_copy_streams(t->device, &s->h2d, &s->d2h);
  if (!ok) {
    const cudaError_t e = cudaGetLastError();
    free_staging(s);
    if (e == cudaErrorMemoryAllocation) return WS_ERR_OOM;
    note_cuda(e, "staging setup");
    return WS_ERR_CUDA;
  }
  t->stage = s;
  return WS_OK;
}

}  // namespace

int wsi::classify(const void* p, int device) {
  if (!p) return PTR_NULL;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
    return at.device == device ? PTR_DEVICE : PTR_OTHER_DEVICE;
  return PTR_HOST;
}

void* wsi::mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

namespace {

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// WS_OPT_HOST_DIRECT: replace a host pointer by the device's view of it when
// the memory is page-locked and mapped, so the kernel reads (and writes) it
// in place over the host link instead of through the staging copies.
template <typename P>
void go_direct(P& p, int& cls) {
  if (cls != wsi::PTR_HOST) return;
  void* d = wsi::mapped_host(p);
  if (!d) return;
  p = reinterpret_cast<P>(d);
  cls = wsi::PTR_DEVICE;
}

}  // namespace

cudaError_t wsi::dispatch(const ws_table* t, const ws::TableView& tv, const ws::BatchArgs& a, int kind,
                          cudaStream_t s) {
  const int B = (int)t->B, T = t->T;
  if (t->scheme == WS_DOUBLE)
    return t->meta ? ws::launch_double_meta(B, T, tv, a, kind, s, t->num_sms)
                   : ws::launch_double_plain(B, T, tv, a, kind, s, t->num_sms);
  if (t->scheme == WS_ICEBERG) return ws::launch_iceberg_meta(B, T, tv, a, kind, s, t->num_sms);
  return t->meta ? ws::launch_p2_meta(B, T, tv, a, kind, s, t->num_sms)
                 : ws::launch_p2_plain(B, T, tv, a, kind, s, t->num_sms);
}

namespace {

ws_status run_batch(ws_table* t, int kind, int op, const u8* ops, const uint64_t* keys_in,
                    const uint64_t* vals_in, uint64_t* vals_out_in, u8* status_out, u64 n, cudaStream_t s) {
  const u64* keys = reinterpret_cast<const u64*>(keys_in);
  const u64* vals = reinterpret_cast<const u64*>(vals_in);
  u64* vals_out = reinterpret_cast<u64*>(vals_out_in);
  if (!t) return WS_ERR_INVALID;
  if (n == 0) return WS_OK;
  if (!keys || !aligned8(keys) || !aligned8(vals) || !aligned8(vals_out)) return WS_ERR_INVALID;
  if ((kind == ws::KIND_UPSERT) && !vals) return WS_ERR_INVALID;
  if (kind == ws::KIND_MIXED && !ops) return WS_ERR_INVALID;
  DeviceGuard guard(t->device);

  int pk = classify(keys, t->device), pv = classify(vals, t->device), po = classify(ops, t->device);
  int pvo = classify(vals_out, t->device), pst = classify(status_out, t->device);
  if (pk == PTR_OTHER_DEVICE || pv == PTR_OTHER_DEVICE || po == PTR_OTHER_DEVICE ||
      pvo == PTR_OTHER_DEVICE || pst == PTR_OTHER_DEVICE)
    return WS_ERR_INVALID;

  // An erase anywhere in the table's history ends the two-choice shortcut
  // (with tombstones, a key can sit in b_1 while b_0 is below 3/4 full).
  if (kind == ws::KIND_ERASE || kind == ws::KIND_MIXED) t->never_erased = 0;
  ws::TableView tv = t->tv;
  tv.shortcut = t->never_erased;
  t->last_stream = s;

  // WS_OPT_HOST_DIRECT 3 (automatic): page-locked inputs are read in place
  // by calls whose kernels spend long per op (insert-if-unique, erase: the
  // host link's latency hides behind their probe sequences) and staged
  // through the copy engines for the others (queries, upserts, mixed).
  int hd = t->host_direct;
  if (hd == 3) hd = (kind == ws::KIND_ERASE || (kind == ws::KIND_UPSERT && op == ws::OP_INSERT)) ? 1 : 0;
  const int pk0 = pk, pv0 = pv;
  if (hd >= 1) {  // inputs read in place
    go_direct(keys, pk);
    go_direct(vals, pv);
    go_direct(ops, po);
  }
  // keys (and values) read in place from host memory
  const bool host_in = (pk0 == PTR_HOST && pk != PTR_HOST) && (vals == nullptr || (pv0 == PTR_HOST && pv != PTR_HOST));
  const u32 in_flags = host_in ? (u32)ws::BATCH_HOST_INPUTS : 0u;
  if (hd >= 2) {  // results written in place
    go_direct(vals_out, pvo);
    go_direct(status_out, pst);
  }
  const bool any_host = pk == PTR_HOST || pv == PTR_HOST || po == PTR_HOST || pvo == PTR_HOST || pst == PTR_HOST;
  if (!any_host) {
    ws::BatchArgs a{keys, vals, ops, vals_out, status_out, n, op, 1, in_flags};
    WS_CUDA(dispatch(t, tv, a, kind, s));
    return WS_OK;
  }

  ws_status rc = ensure_staging(t);
  if (rc != WS_OK) return rc;
  Staging& g = *t->stage;
  const bool host_out = pvo == PTR_HOST || pst == PTR_HOST;
  u64 chunk = 0;
  for (u64 off = 0; off < n; off += g.cap, ++chunk) {
    const u64 m = (n - off) < g.cap ? (n - off) : g.cap;
    const int b = (int)(chunk % Staging::kBufs);
    WS_CUDA(cudaStreamWaitEvent(g.h2d, g.k_done[b], 0));
    const u64* kp = keys + off;
    const u64* vp = vals ? vals + off : nullptr;
    const u8* op_p = ops ? ops + off : nullptr;
    if (pk == PTR_HOST) {
      WS_CUDA(cudaMemcpyAsync(g.keys[b], kp, m * 8, cudaMemcpyHostToDevice, g.h2d));
      kp = g.keys[b];
    }
    if (pv == PTR_HOST) {
      WS_CUDA(cudaMemcpyAsync(g.vals[b], vp, m * 8, cudaMemcpyHostToDevice, g.h2d));
      vp = g.vals[b];
    }
    if (po == PTR_HOST) {
      WS_CUDA(cudaMemcpyAsync(g.ops[b], op_p, m, cudaMemcpyHostToDevice, g.h2d));
      op_p = g.ops[b];
    }
    WS_CUDA(cudaEventRecord(g.in_ready[b], g.h2d));
    WS_CUDA(cudaStreamWaitEvent(s, g.in_ready[b], 0));
    WS_CUDA(cudaStreamWaitEvent(s, g.out_done[b], 0));
    u64* vo = vals_out ? (pvo == PTR_HOST ? g.out[b] : vals_out + off) : nullptr;
    u8* so = status_out ? (pst == PTR_HOST ? g.st[b] : status_out + off) : nullptr;
    ws::BatchArgs a{kp, vp, op_p, vo, so, m, op, 1, in_flags};
    WS_CUDA(dispatch(t, tv, a, kind, s));
    WS_CUDA(cudaEventRecord(g.k_done[b], s));
    if (host_out) {
      WS_CUDA(cudaStreamWaitEvent(g.d2h, g.k_done[b], 0));
      if (pvo == PTR_HOST) WS_CUDA(cudaMemcpyAsync(vals_out + off, g.out[b], m * 8, cudaMemcpyDeviceToHost, g.d2h));
      if (pst == PTR_HOST) WS_CUDA(cudaMemcpyAsync(status_out + off, g.st[b], m, cudaMemcpyDeviceToHost, g.d2h));
      WS_CUDA(cudaEventRecord(g.out_done[b], g.d2h));
    }
  }
  if (host_out)
    for (int b = 0; b < Staging::kBufs && (u64)b < chunk; ++b) WS_CUDA(cudaStreamWaitEvent(s, g.out_done[b], 0));
  return WS_OK;
}

// b_0 of each key (iceberg: the front-yard bucket, whose lock inserters take).
__global__ void primary_bucket_kernel(const u64* keys, u64* out, u64 n, u64 seed1, u64 mask, u64 nb_front,
                                      int iceberg) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const u64 h1 = ws::fmix64(keys[i] ^ seed1);
    out[i] = iceberg ? __umul64hi(h1, nb_front) : (h1 & mask);
  }
}

}  // namespace

// Shared constructor.  With a stream, memory comes from the stream-ordered
// allocator and is cleared on that stream (no device-wide synchronisation),
// so a serving loop can grow a table while other work is in flight.
ws_status wsi::table_create(const ws_config* cfg, cudaStream_t stream, ws_table** out) {
  if (!cfg || !out) return WS_ERR_INVALID;
  *out = nullptr;
  if (cfg->scheme != WS_DOUBLE && cfg->scheme != WS_P2 && cfg->scheme != WS_ICEBERG) return WS_ERR_INVALID;
  if (cfg->scheme == WS_ICEBERG && !cfg->metadata) return WS_ERR_INVALID;  // IcebergHT(M) only
  if (cfg->capacity == 0 || cfg->capacity > (1ull << 40)) return WS_ERR_INVALID;
  const int meta = cfg->metadata ? 1 : 0;
  int B = cfg->bucket_slots ? cfg->bucket_slots : ((cfg->scheme == WS_DOUBLE && !meta) ? 8 : 32);
  int T = cfg->tile ? cfg->tile : (meta ? 4 : 8);
  if (B != 8 && B != 16 && B != 32) return WS_ERR_INVALID;
  if (meta && B != 32) return WS_ERR_INVALID;
  if (T != 4 && T != 8 && T != 16 && T != 32) return WS_ERR_INVALID;

  int dev = cfg->device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
    note_cuda(cudaGetLastError(), "cudaGetDevice");
    return WS_ERR_CUDA;
  }
  DeviceGuard guard(dev);
  ws_table* t = new (std::nothrow) ws_table();
  if (!t) return WS_ERR_OOM;
  u64 nb = 1;
  const u64 want = (cfg->capacity + (u64)B - 1) / (u64)B;
  while (nb < want) nb <<= 1;
  if (cfg->scheme == WS_ICEBERG && nb < 4) nb = 4;  // a front yard and a two-bucket backyard
  t->nb = nb;
  t->B = (u64)B;
  t->S = nb * (u64)B;
  t->T = T;
  t->scheme = cfg->scheme;
  t->meta = meta;
  t->device = dev;
  t->pmax = cfg->max_probe ? cfg->max_probe : kDefaultProbe;
  if ((u64)t->pmax > nb) t->pmax = (uint32_t)nb;
  t->spin = cfg->spin_limit ? cfg->spin_limit : kDefaultSpin;
  t->stream_alloc = stream != nullptr;
  t->last_stream = stream;
  if (cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    note_cuda(cudaGetLastError(), "cudaDeviceGetAttribute");
    delete t;
    return WS_ERR_CUDA;
  }
  const u64 lock_words = (nb + 31) / 32;
  ws::TableView& tv = t->tv;
  std::memset(&tv, 0, sizeof(tv));
  auto alloc = [&](void** p, size_t bytes) {
    return (stream ? cudaMallocAsync(p, bytes, stream) : cudaMalloc(p, bytes)) == cudaSuccess;
  };
  bool ok = alloc(reinterpret_cast<void**>(&tv.slots), t->S * sizeof(ws::Slot));
  if (ok && meta) ok = alloc(reinterpret_cast<void**>(&tv.tags), t->S * sizeof(uint16_t));
  if (ok) ok = alloc(reinterpret_cast<void**>(&tv.locks), lock_words * 4);
  if (ok) ok = alloc(reinterpret_cast<void**>(&tv.ctr), sizeof(ws::Counters));
  if (!ok) {
    cudaGetLastError();
    free_table_memory(t);
    delete t;
    return WS_ERR_OOM;
  }
  t->bytes = t->S * sizeof(ws::Slot) + (meta ? t->S * 2 : 0) + lock_words * 4 + sizeof(ws::Counters);
  tv.nb_mask = nb - 1;
  tv.nb_front = nb;
  tv.nb_back = 0;
  if (cfg->scheme == WS_ICEBERG) {
    // backyard = 17% of the buckets, rounded to nearest, at least 2 (§5)
    tv.nb_back = (17 * nb + 50) / 100;
    if (tv.nb_back < 2) tv.nb_back = 2;
    tv.nb_front = nb - tv.nb_back;
  }
  tv.seed1 = kSeed1;
  tv.seed2 = kSeed2;
  tv.pmax = t->pmax;
  tv.spin_limit = t->spin;
  tv.shortcut = 1;
  tv.preload = kDefaultPreload;
  tv.stream = 1;  // streaming lanes in single-table launches (see WS_OPT_STREAM)
  auto clear = [&](void* p, size_t bytes) {
    return stream ? cudaMemsetAsync(p, 0, bytes, stream) : cudaMemset(p, 0, bytes);
  };
  cudaError_t e = clear(tv.slots, t->S * sizeof(ws::Slot));
  if (e == cudaSuccess && meta) e = clear(tv.tags, t->S * 2);
  if (e == cudaSuccess) e = clear(tv.locks, lock_words * 4);
  if (e == cudaSuccess) e = clear(tv.ctr, sizeof(ws::Counters));
  if (e == cudaSuccess && !stream) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    note_cuda(e, "table init");
    free_table_memory(t);
    delete t;
    return WS_ERR_CUDA;
  }
  *out = t;
  return WS_OK;
}

// Stream-ordered release of a table made with a stream (no device sync);
// a table made without one is released the ordinary way.
void wsi::table_free_async(ws_table* t, cudaStream_t stream) {
  if (!t) return;
  if (!t->stream_alloc) {
    ws_destroy(t);
    return;
  }
  DeviceGuard guard(t->device);
  void* ptrs[4] = {t->tv.slots, t->tv.tags, t->tv.locks, t->tv.ctr};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, stream);
  t->tv.slots = nullptr;
  t->tv.tags = nullptr;
  t->tv.locks = nullptr;
  t->tv.ctr = nullptr;
  if (t->stage) {
    free_staging(t->stage);
    t->stage = nullptr;
  }
  delete t;
}

extern "C" {

uint32_t ws_version(void) { return 0x000100u; }

const char* ws_cuda_error_string(void) { return g_cuda_err; }

const char* ws_status_string(ws_status s) {
  switch (s) {
    case WS_OK: return "ok";
    case WS_ERR_INVALID: return "invalid argument";
    case WS_ERR_INVALID_KEY: return "an op used a reserved sentinel key";
    case WS_ERR_OOM: return "out of device memory";
    case WS_ERR_FULL: return "an insert found no free slot";
    case WS_ERR_TIMEOUT: return "an op hit the lock spin limit";
    case WS_ERR_CUDA: return "CUDA error";
  }
  return "unknown status";
}

ws_status ws_table_create_ex(const ws_config* cfg, ws_table** out) { return wsi::table_create(cfg, nullptr, out); }

ws_status ws_table_create(uint64_t capacity, ws_scheme scheme, int metadata, ws_table** out) {
  ws_config c;
  std::memset(&c, 0, sizeof(c));
  c.capacity = capacity;
  c.scheme = scheme;
  c.metadata = metadata;
  c.device = -1;
  return ws_table_create_ex(&c, out);
}

ws_status ws_destroy(ws_table* t) {
  if (!t) return WS_ERR_INVALID;
  {
    DeviceGuard guard(t->device);
    cudaDeviceSynchronize();
    cudaGetLastError();
    free_table_memory(t);
  }
  delete t;
  return WS_OK;
}

ws_status ws_table_info_get(const ws_table* t, ws_table_info* o) {
  if (!t || !o) return WS_ERR_INVALID;
  o->slots = t->S;
  o->buckets = t->nb;
  o->bucket_slots = t->B;
  o->tile = (u64)t->T;
  o->max_probe = t->scheme == WS_DOUBLE ? t->pmax : t->scheme == WS_ICEBERG ? 3 : (t->nb > 1 ? 2 : 1);
  o->seed1 = t->tv.seed1;
  o->seed2 = t->tv.seed2;
  o->bytes = t->bytes;
  o->scheme = t->scheme;
  o->metadata = t->meta;
  o->device = t->device;
  o->never_erased = t->never_erased;
  o->front_buckets = t->tv.nb_front;
  return WS_OK;
}

ws_status ws_clear(ws_table* t, ws_stream stream) {
  if (!t) return WS_ERR_INVALID;
  DeviceGuard guard(t->device);
  cudaStream_t s = (cudaStream_t)stream;
  WS_CUDA(cudaMemsetAsync(t->tv.slots, 0, t->S * sizeof(ws::Slot), s));
  if (t->meta) WS_CUDA(cudaMemsetAsync(t->tv.tags, 0, t->S * 2, s));
  WS_CUDA(cudaMemsetAsync(t->tv.locks, 0, ((t->nb + 31) / 32) * 4, s));
  WS_CUDA(cudaMemsetAsync(t->tv.ctr, 0, sizeof(ws::Counters), s));
  t->never_erased = 1;
  t->last_stream = s;
  return WS_OK;
}

ws_status ws_set_tile(ws_table* t, int tile) {
  if (!t || (tile != 4 && tile != 8 && tile != 16 && tile != 32)) return WS_ERR_INVALID;
  t->T = tile;
  return WS_OK;
}

ws_status ws_set_option(ws_table* t, int option, int64_t value) {
  if (!t) return WS_ERR_INVALID;
  switch (option) {
    case WS_OPT_PRELOAD:
      if (value != 0 && value != 1) return WS_ERR_INVALID;
      t->tv.preload = (int)value;
      return WS_OK;
    case WS_OPT_PHASED:
      if (value != 0 && value != 1) return WS_ERR_INVALID;
      t->tv.phased = (int)value;
      return WS_OK;
    case WS_OPT_LANE_WAVES:
      if (value < 0 || value > 255) return WS_ERR_INVALID;
      t->tv.lane_waves = (int)value;
      return WS_OK;
    case WS_OPT_STREAM:
      if (value < 0 || value > 2) return WS_ERR_INVALID;
      t->tv.stream = (int)value;
      return WS_OK;
    case WS_OPT_STAGE_CHUNK:
      if (value < 16 || value > 24) return WS_ERR_INVALID;
      if (t->stage && t->stage->cap != (1ull << value)) {  // reallocated at the next host-buffer call
        DeviceGuard guard(t->device);
        WS_CUDA(cudaStreamSynchronize(t->last_stream));
        free_staging(t->stage);
        t->stage = nullptr;
      }
      t->stage_log2 = (int)value;
      return WS_OK;
    case WS_OPT_HOST_DIRECT:
      if (value < 0 || value > 3) return WS_ERR_INVALID;
      t->host_direct = (int)value;
      return WS_OK;
  }
  return WS_ERR_INVALID;
}

ws_status ws_set_spin_limit(ws_table* t, uint32_t spins) {
  if (!t || spins == 0) return WS_ERR_INVALID;
  t->spin = spins;
  t->tv.spin_limit = spins;
  return WS_OK;
}

ws_status ws_insert_ex(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                       uint8_t* status_out, ws_stream stream) {
  return run_batch(t, ws::KIND_UPSERT, ws::OP_INSERT, nullptr, keys, vals, nullptr, status_out, n,
                   (cudaStream_t)stream);
}
ws_status ws_insert(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n, ws_stream stream) {
  return ws_insert_ex(t, keys, vals, n, nullptr, stream);
}

ws_status ws_upsert_ex(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n,
                       ws_upsert_op op, uint8_t* status_out, ws_stream stream) {
  if (op != WS_OP_ADD && op != WS_OP_MAX && op != WS_OP_REPLACE && op != WS_OP_INSERT) return WS_ERR_INVALID;
  return run_batch(t, ws::KIND_UPSERT, (int)op, nullptr, keys, vals, nullptr, status_out, n,
                   (cudaStream_t)stream);
}
ws_status ws_upsert(ws_table* t, const uint64_t* keys, const uint64_t* vals, uint64_t n, ws_upsert_op op,
                    ws_stream stream) {
  return ws_upsert_ex(t, keys, vals, n, op, nullptr, stream);
}

ws_status ws_query_ex(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint8_t* found_out, uint64_t n,
                      ws_stream stream) {
  if (!vals_out && !found_out && n) return WS_ERR_INVALID;
  return run_batch(t, ws::KIND_QUERY, 0, nullptr, keys, nullptr, vals_out, found_out, n, (cudaStream_t)stream);
}
ws_status ws_query(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint64_t n, ws_stream stream) {
  return ws_query_ex(t, keys, vals_out, nullptr, n, stream);
}

ws_status ws_erase_ex(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint8_t* status_out, uint64_t n,
                      ws_stream stream) {
  return run_batch(t, ws::KIND_ERASE, 0, nullptr, keys, nullptr, vals_out, status_out, n, (cudaStream_t)stream);
}
ws_status ws_erase(ws_table* t, const uint64_t* keys, uint64_t* vals_out, uint64_t n, ws_stream stream) {
  return ws_erase_ex(t, keys, vals_out, nullptr, n, stream);
}

ws_status ws_mixed(ws_table* t, const uint8_t* ops, const uint64_t* keys, const uint64_t* vals,
                   uint64_t* vals_out, uint8_t* status_out, uint64_t n, ws_stream stream) {
  return run_batch(t, ws::KIND_MIXED, 0, ops, keys, vals, vals_out, status_out, n, (cudaStream_t)stream);
}

ws_status ws_probe_cost(ws_table* t, const uint64_t* keys, uint64_t* cost_out, uint8_t* found_out, uint64_t n,
                        ws_stream stream) {
  if (!cost_out && n) return WS_ERR_INVALID;
  return run_batch(t, ws::KIND_PROBE, 0, nullptr, keys, nullptr, cost_out, found_out, n, (cudaStream_t)stream);
}

ws_status ws_count(ws_table* t, uint64_t* out) {
  if (!t || !out) return WS_ERR_INVALID;
  DeviceGuard guard(t->device);
  WS_CUDA(cudaStreamSynchronize(t->last_stream));
  WS_CUDA(cudaMemcpy(out, &t->tv.ctr->count, sizeof(uint64_t), cudaMemcpyDeviceToHost));
  return WS_OK;
}

ws_status ws_last_error(ws_table* t, uint64_t* n_full, uint64_t* n_timeout, uint64_t* n_badkey) {
  if (!t) return WS_ERR_INVALID;
  DeviceGuard guard(t->device);
  WS_CUDA(cudaStreamSynchronize(t->last_stream));
  ws::Counters c;
  WS_CUDA(cudaMemcpy(&c, t->tv.ctr, sizeof(c), cudaMemcpyDeviceToHost));
  if (n_full) *n_full = c.n_full;
  if (n_timeout) *n_timeout = c.n_timeout;
  if (n_badkey) *n_badkey = c.n_badkey;
  if (c.n_timeout) return WS_ERR_TIMEOUT;
  if (c.n_full) return WS_ERR_FULL;
  if (c.n_badkey) return WS_ERR_INVALID_KEY;
  return WS_OK;
}

ws_status ws_num_buckets(const ws_table* t, uint64_t* out) {
  if (!t || !out) return WS_ERR_INVALID;
  *out = t->nb;
  return WS_OK;
}

ws_status ws_primary_bucket(ws_table* t, const uint64_t* keys, uint64_t* out, uint64_t n, ws_stream stream) {
  if (!t || (n && (!keys || !out))) return WS_ERR_INVALID;
  if (n == 0) return WS_OK;
  DeviceGuard guard(t->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int pk = classify(keys, t->device), po = classify(out, t->device);
  if (pk == PTR_OTHER_DEVICE || po == PTR_OTHER_DEVICE) return WS_ERR_INVALID;
  u64* dk = reinterpret_cast<u64*>(const_cast<uint64_t*>(keys));
  u64* dout = reinterpret_cast<u64*>(out);
  if (pk == PTR_HOST) {
    WS_CUDA(cudaMallocAsync(&dk, n * 8, s));
    WS_CUDA(cudaMemcpyAsync(dk, keys, n * 8, cudaMemcpyHostToDevice, s));
  }
  if (po == PTR_HOST) WS_CUDA(cudaMallocAsync(&dout, n * 8, s));
  const unsigned grid = (unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  primary_bucket_kernel<<<grid, 256, 0, s>>>(dk, dout, n, t->tv.seed1, t->tv.nb_mask, t->tv.nb_front,
                                             t->scheme == WS_ICEBERG ? 1 : 0);
  WS_CUDA(cudaGetLastError());
  if (po == PTR_HOST) {
    WS_CUDA(cudaMemcpyAsync(out, dout, n * 8, cudaMemcpyDeviceToHost, s));
    WS_CUDA(cudaFreeAsync(dout, s));
  }
  if (pk == PTR_HOST) WS_CUDA(cudaFreeAsync(dk, s));
  if (pk == PTR_HOST || po == PTR_HOST) WS_CUDA(cudaStreamSynchronize(s));
  return WS_OK;
}

ws_status ws_rehash(ws_table* src, ws_table* dst, uint8_t* status_out, ws_stream stream) {
  if (!src || !dst || src == dst || src->device != dst->device) return WS_ERR_INVALID;
  DeviceGuard guard(dst->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (src->last_stream != s) WS_CUDA(cudaStreamSynchronize(src->last_stream));
  // The source's slot array is the input: keys at stride 2, values right after.
  const u64* base = reinterpret_cast<const u64*>(src->tv.slots);
  ws::BatchArgs a{base, base + 1, nullptr, nullptr, status_out, src->S, ws::OP_INSERT, 2, ws::BATCH_SKIP_SENTINELS};
  ws::TableView tv = dst->tv;
  tv.shortcut = dst->never_erased;
  dst->last_stream = s;
  WS_CUDA(dispatch(dst, tv, a, ws::KIND_UPSERT, s));
  return WS_OK;
}

ws_status ws_dump(ws_table* t, void* host_slots, void* host_tags) {
  if (!t || !host_slots) return WS_ERR_INVALID;
  DeviceGuard guard(t->device);
  WS_CUDA(cudaDeviceSynchronize());
  WS_CUDA(cudaMemcpy(host_slots, t->tv.slots, t->S * sizeof(ws::Slot), cudaMemcpyDeviceToHost));
  if (host_tags && t->meta) WS_CUDA(cudaMemcpy(host_tags, t->tv.tags, t->S * 2, cudaMemcpyDeviceToHost));
  return WS_OK;
}

ws_status ws_debug_fill_locks(ws_table* t, int locked, ws_stream stream) {
  if (!t) return WS_ERR_INVALID;
  DeviceGuard guard(t->device);
  WS_CUDA(cudaMemsetAsync(t->tv.locks, locked ? 0xff : 0, ((t->nb + 31) / 32) * 4, (cudaStream_t)stream));
  t->last_stream = (cudaStream_t)stream;
  return WS_OK;
}

}  // extern "C"
