// ws_serve.cu -- a continuous-batching request loop over device-resident tables.
//
// Requests are mixed op batches (ws_mixed_op codes) against one table each,
// with host buffers.  A worker thread keeps up to `max_inflight` launch slots
// busy.  Each slot is a stream with its own device staging and descriptor
// buffers: the worker admits waiting requests into a free slot -- at most one
// request per table in flight, taken in per-table FIFO order, oldest head
// first -- copies their inputs in, runs them all in one persistent
// multi-table launch, copies the results out, and records an event.  Requests
// that arrive while other slots are on the GPU are admitted as soon as a slot
// frees up, and slots overlap on the device.  Because each table sees its
// requests one at a time in arrival order, every result equals the result of
// replaying that table's requests alone.
//
// Tables are added only when free device memory admits them (with a stated
// headroom), and a table that would pass `grow_at` load is replaced by one
// twice as large -- allocated and filled by rehash on the slot's stream --
// when memory admits it.  Plain mode (one request per launch, one launch at a
// time, single-table kernel) is the per-request baseline.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ws_internal.h"
#include "ws_multi.cuh"

using namespace wsi;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SReq {
  ws_request r;
  uint64_t id = 0;
  double t_submit = 0, t_start = 0;
  uint64_t n_write = 0;  // insert / upsert ops (growth estimate)
  bool has_erase = false;
};

struct STable {
  ws_table* t = nullptr;
  std::deque<uint64_t> pending;  // request ids in arrival order
  bool busy = false;
  uint64_t live = 0;             // exact live count after the last finished request
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  u64* d_keys = nullptr;
  u64* d_vals = nullptr;
  u64* d_out = nullptr;
  u8* d_ops = nullptr;
  u8* d_st = nullptr;
  ws::MultiItem* d_items = nullptr;
  ws::MultiChunk* d_chunks = nullptr;
  u32* d_ticket = nullptr;             // one work ticket per menu entry
  ws::MultiItem* h_items = nullptr;   // pinned
  ws::MultiChunk* h_chunks = nullptr; // pinned
  u64* h_counts = nullptr;            // pinned, one per request
  std::vector<uint64_t> reqs;
  std::vector<uint32_t> tabs;
  std::vector<ws_table*> retire;
  bool busy = false;
};

}  // namespace

struct ws_server {
  ws_server_config cfg;
  int device = 0, num_sms = 0;
  u64 max_chunks = 0;
  std::vector<STable> tables;
  std::vector<SReq> reqs;  // index = id (worker-owned once moved in from the inbox)
  std::vector<Slot> slots;
  std::vector<ws_completion> done;
  uint64_t n_completed = 0, n_launches = 0, n_grows = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  // Submissions go to an inbox under their own mutex, so a submit never waits
  // for the worker, which holds `mu` while it issues a slot's CUDA calls.
  std::mutex in_mu;
  std::condition_variable cv_in;  // wakes the worker: new requests or `wake`
  std::vector<SReq> inbox;
  bool wake = false;
  std::atomic<uint64_t> n_submitted{0};
  std::atomic<uint32_t> n_tables{0};
  std::thread worker;
  bool stop = false;
  bool paused = false;
  int error = 0;
};

namespace {

void slot_free(Slot& sl) {
  if (sl.s) cudaStreamSynchronize(sl.s);
  void* d[] = {sl.d_keys, sl.d_vals, sl.d_out, sl.d_ops, sl.d_st, sl.d_items, sl.d_chunks, sl.d_ticket};
  for (void* p : d)
    if (p) cudaFree(p);
  void* h[] = {sl.h_items, sl.h_chunks, sl.h_counts};
  for (void* p : h)
    if (p) cudaFreeHost(p);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.s) cudaStreamDestroy(sl.s);
  sl = Slot();
}

bool slot_alloc(Slot& sl, u64 cap, u64 max_items, u64 max_chunks) {
  bool ok = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc(&sl.d_keys, cap * 8) == cudaSuccess && cudaMalloc(&sl.d_vals, cap * 8) == cudaSuccess &&
            cudaMalloc(&sl.d_out, cap * 8) == cudaSuccess && cudaMalloc(&sl.d_ops, cap) == cudaSuccess &&
            cudaMalloc(&sl.d_st, cap) == cudaSuccess &&
            cudaMalloc(&sl.d_items, max_items * sizeof(ws::MultiItem)) == cudaSuccess &&
            cudaMalloc(&sl.d_chunks, max_chunks * sizeof(ws::MultiChunk)) == cudaSuccess &&
            cudaMalloc(&sl.d_ticket, ws::kMultiMenu * sizeof(u32)) == cudaSuccess &&
            cudaMallocHost(&sl.h_items, max_items * sizeof(ws::MultiItem)) == cudaSuccess &&
            cudaMallocHost(&sl.h_chunks, max_chunks * sizeof(ws::MultiChunk)) == cudaSuccess &&
            cudaMallocHost(&sl.h_counts, max_items * sizeof(u64)) == cudaSuccess;
  if (!ok) cudaGetLastError();
  return ok;
}

// Device memory a new table may take: free memory plus what the default pool
// holds but does not use (freed tables stay pooled, see ws_server_create).
bool avail_bytes(int dev, size_t* avail, size_t* total) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return false;
  cudaMemPool_t pool;
  uint64_t reserved = 0, used = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
    fr += (size_t)(reserved - used);
  cudaGetLastError();
  *avail = fr;
  *total = tot;
  return true;
}

// Replace table `ti` by one `factor` times larger if memory admits it; the
// rehash runs on stream s.  Returns true when grown.
bool try_grow(ws_server* sv, uint32_t ti, uint64_t need_live, Slot& sl) {
  ws_table* old = sv->tables[ti].t;
  uint64_t cap = old->S;
  while ((double)need_live > sv->cfg.grow_at * (double)cap) cap *= 2;
  if (cap == old->S) return false;
  size_t fr = 0, tot = 0;
  if (!avail_bytes(sv->device, &fr, &tot)) return false;
  const double bytes = (double)cap * (16.0 + (old->meta ? 2.0 : 0.0));
  if ((double)fr - bytes < sv->cfg.hbm_headroom * (double)tot) return false;  // not admitted
  ws_config c;
  std::memset(&c, 0, sizeof(c));
  c.capacity = cap;
  c.scheme = old->scheme;
  c.metadata = old->meta;
  c.bucket_slots = (int32_t)old->B;
  c.tile = old->T;
  c.device = sv->device;
  ws_table* nt = nullptr;
  if (table_create(&c, sl.s, &nt) != WS_OK) return false;
  const u64* base = reinterpret_cast<const u64*>(old->tv.slots);
  ws::BatchArgs a{base, base + 1, nullptr, nullptr, nullptr, old->S, ws::OP_INSERT, 2, ws::BATCH_SKIP_SENTINELS};
  ws::TableView tv = nt->tv;
  tv.shortcut = 1;
  if (dispatch(nt, tv, a, ws::KIND_UPSERT, sl.s) != cudaSuccess) {
    table_free_async(nt, sl.s);
    return false;
  }
  nt->never_erased = old->never_erased;
  sv->tables[ti].t = nt;
  sl.retire.push_back(old);
  ++sv->n_grows;
  return true;
}

// Admit waiting requests into a free slot and launch them.  Called by the
// worker with the lock held; returns true if something was launched.
bool launch_slot(ws_server* sv, Slot& sl) {
  // choose: one request per idle table, oldest head first, within budgets
  std::vector<uint32_t> cand;
  for (uint32_t ti = 0; ti < sv->tables.size(); ++ti)
    if (!sv->tables[ti].busy && !sv->tables[ti].pending.empty()) cand.push_back(ti);
  if (cand.empty()) return false;
  std::sort(cand.begin(), cand.end(), [&](uint32_t a, uint32_t b) {
    return sv->tables[a].pending.front() < sv->tables[b].pending.front();
  });
  const u64 cap = sv->cfg.max_batch_ops;
  const u64 max_items = sv->cfg.plain ? 1 : sv->cfg.max_batch_reqs;
  u64 ops = 0;
  sl.reqs.clear();
  sl.tabs.clear();
  for (uint32_t ti : cand) {
    const uint64_t id = sv->tables[ti].pending.front();
    const SReq& q = sv->reqs[id];
    if (!sl.reqs.empty() && (ops + q.r.n > cap || sl.reqs.size() >= max_items)) continue;
    sv->tables[ti].pending.pop_front();
    sv->tables[ti].busy = true;
    sl.reqs.push_back(id);
    sl.tabs.push_back(ti);
    ops += q.r.n;
    if (sl.reqs.size() >= max_items || ops >= cap) break;
  }
  const double t0 = now_s();
  cudaStream_t s = sl.s;
  u64 off = 0, nchunks = 0;
  bool ok = true;
  std::vector<int> fallback;
  for (size_t i = 0; i < sl.reqs.size() && ok; ++i) {
    SReq& q = sv->reqs[sl.reqs[i]];
    q.t_start = t0;
    STable& T = sv->tables[sl.tabs[i]];
    if (sv->cfg.grow_at > 0 && (double)(T.live + q.n_write) > sv->cfg.grow_at * (double)T.t->S)
      try_grow(sv, sl.tabs[i], T.live + q.n_write, sl);
    ws_table* t = T.t;
    if (q.has_erase) t->never_erased = 0;
    const u64 n = q.r.n;
    ok = cudaMemcpyAsync(sl.d_keys + off, q.r.keys, n * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(sl.d_ops + off, q.r.ops, n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         (q.r.vals ? cudaMemcpyAsync(sl.d_vals + off, q.r.vals, n * 8, cudaMemcpyHostToDevice, s)
                   : cudaMemsetAsync(sl.d_vals + off, 0, n * 8, s)) == cudaSuccess;
    ws::MultiItem& m = sl.h_items[i];
    std::memset(&m, 0, sizeof(m));
    m.tv = t->tv;
    m.tv.shortcut = t->never_erased;
    m.a = ws::BatchArgs{sl.d_keys + off, sl.d_vals + off, sl.d_ops + off, sl.d_out + off, sl.d_st + off, n, 0, 1, 0};
    m.kind = ws::KIND_MIXED;
    m.cfg = sv->cfg.plain ? -1 : ws::multi_menu_index(t->scheme, t->meta != 0, (int)t->B, t->T);
    if (m.cfg < 0) fallback.push_back((int)i);
    off += n;
  }
  // chunks grouped by menu entry (every request is a mixed batch): one
  // persistent launch per entry present
  u64 group_off[ws::kMultiMenu + 1] = {0};
  for (int cfg = 0; cfg < ws::kMultiMenu; ++cfg) {
    group_off[cfg] = nchunks;
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      if (sl.h_items[i].cfg != cfg) continue;
      for (u64 st = 0; st < sl.h_items[i].a.n; st += ws::kMultiChunk) {
        ws::MultiChunk c;
        c.item = (u32)i;
        c.pad = 0;
        c.start = st;
        sl.h_chunks[nchunks++] = c;
      }
    }
  }
  group_off[ws::kMultiMenu] = nchunks;
  if (ok && nchunks) {
    ok = cudaMemcpyAsync(sl.d_items, sl.h_items, sl.reqs.size() * sizeof(ws::MultiItem), cudaMemcpyHostToDevice,
                         s) == cudaSuccess &&
         cudaMemcpyAsync(sl.d_chunks, sl.h_chunks, nchunks * sizeof(ws::MultiChunk), cudaMemcpyHostToDevice, s) ==
             cudaSuccess &&
         cudaMemsetAsync(sl.d_ticket, 0, ws::kMultiMenu * sizeof(u32), s) == cudaSuccess;
    for (int cfg = 0; cfg < ws::kMultiMenu && ok; ++cfg) {
      const u64 n_c = group_off[cfg + 1] - group_off[cfg];
      if (!n_c) continue;
      ws::MultiGroup g{sl.d_items, sl.d_chunks + group_off[cfg], nullptr, 0, 0, (u32)n_c, sl.d_ticket + cfg};
      ok = ws::launch_multi(cfg, ws::KIND_MIXED, g, s, sv->num_sms) == cudaSuccess;
    }
  }
  for (size_t k = 0; k < fallback.size() && ok; ++k) {
    const ws::MultiItem& m = sl.h_items[fallback[k]];
    ok = dispatch(sv->tables[sl.tabs[fallback[k]]].t, m.tv, m.a, ws::KIND_MIXED, s) == cudaSuccess;
  }
  off = 0;
  for (size_t i = 0; i < sl.reqs.size() && ok; ++i) {
    SReq& q = sv->reqs[sl.reqs[i]];
    const u64 n = q.r.n;
    if (q.r.vals_out)
      ok = cudaMemcpyAsync(q.r.vals_out, sl.d_out + off, n * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok && q.r.status_out)
      ok = cudaMemcpyAsync(q.r.status_out, sl.d_st + off, n, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ws_table* t = sv->tables[sl.tabs[i]].t;
    if (ok) ok = cudaMemcpyAsync(&sl.h_counts[i], &t->tv.ctr->count, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    t->last_stream = s;
    off += n;
  }
  if (ok) ok = cudaEventRecord(sl.done, s) == cudaSuccess;
  if (!ok) {
    note_cuda(cudaGetLastError(), "server launch");
    sv->error = WS_ERR_CUDA;
  }
  sl.busy = true;
  ++sv->n_launches;
  return true;
}

void finish_slot(ws_server* sv, Slot& sl) {
  const double t1 = now_s();
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    SReq& q = sv->reqs[sl.reqs[i]];
    STable& T = sv->tables[sl.tabs[i]];
    T.busy = false;
    T.live = sl.h_counts[i];
    ws_completion c;
    c.id = q.id;
    c.tag = q.r.tag;
    c.t_submit = q.t_submit;
    c.t_start = q.t_start;
    c.t_done = t1;
    c.status = sv->error ? sv->error : WS_OK;
    c.table = q.r.table;
    sv->done.push_back(c);
    ++sv->n_completed;
  }
  for (ws_table* t : sl.retire) table_free_async(t, sl.s);
  sl.retire.clear();
  sl.reqs.clear();
  sl.tabs.clear();
  sl.busy = false;
}

void wake_worker(ws_server* sv) {
  {
    std::lock_guard<std::mutex> il(sv->in_mu);
    sv->wake = true;
  }
  sv->cv_in.notify_one();
}

// Moves submitted requests into the per-table queues (worker, `mu` held);
// counts each request's writes (growth estimate) and erases here, off the
// submitting thread.
void take_inbox(ws_server* sv) {
  std::vector<SReq> in;
  {
    std::lock_guard<std::mutex> il(sv->in_mu);
    in.swap(sv->inbox);
    sv->wake = false;
  }
  for (SReq& q : in) {
    for (uint64_t i = 0; i < q.r.n; ++i) {
      const uint8_t o = q.r.ops[i];
      q.n_write += (o >= WS_MX_INSERT && o <= WS_MX_REPLACE) ? 1 : 0;
      q.has_erase |= (o == WS_MX_ERASE);
    }
    sv->tables[q.r.table].pending.push_back(q.id);
    sv->reqs.push_back(q);  // ids are handed out in inbox order: index == id
  }
}

void worker_main(ws_server* sv) {
  DeviceGuard guard(sv->device);
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    take_inbox(sv);
    bool progress = false;
    for (Slot& sl : sv->slots) {
      if (sl.busy && cudaEventQuery(sl.done) != cudaErrorNotReady) {
        finish_slot(sv, sl);
        progress = true;
      }
    }
    if (progress) sv->cv_done.notify_all();
    for (Slot& sl : sv->slots) {
      if (sv->paused && !sv->stop) break;
      if (sl.busy) continue;
      if (!launch_slot(sv, sl)) break;
      progress = true;
      if (sv->cfg.plain) break;
    }
    bool any_busy = false, any_pending = false;
    for (const Slot& sl : sv->slots) any_busy |= sl.busy;
    for (const STable& t : sv->tables) any_pending |= !t.pending.empty();
    if (sv->stop && !any_busy && !any_pending && sv->reqs.size() == sv->n_submitted.load()) break;
    if (progress) continue;
    // launches in flight: look again shortly; idle: sleep until a request or
    // a state change (pause, drain, stop) arrives
    lk.unlock();
    {
      std::unique_lock<std::mutex> il(sv->in_mu);
      const auto dur = any_busy ? std::chrono::microseconds(20) : std::chrono::microseconds(2000);
      sv->cv_in.wait_for(il, dur, [&] { return !sv->inbox.empty() || sv->wake; });
    }
    lk.lock();
  }
}

}  // namespace

extern "C" {

ws_status ws_server_create(const ws_server_config* cfg, ws_server** out) {
  if (!out) return WS_ERR_INVALID;
  *out = nullptr;
  ws_server_config c;
  std::memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  if (c.max_inflight <= 0) c.max_inflight = 4;
  if (c.max_batch_ops == 0) c.max_batch_ops = 1ull << 22;
  if (c.max_batch_reqs == 0) c.max_batch_reqs = 256;
  if (c.hbm_headroom <= 0) c.hbm_headroom = 0.05;
  if (c.grow_at < 0) return WS_ERR_INVALID;
  if (c.plain) c.max_inflight = 1;
  int dev = c.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return WS_ERR_CUDA;
  DeviceGuard guard(dev);
  ws_server* sv = new (std::nothrow) ws_server();
  if (!sv) return WS_ERR_OOM;
  sv->cfg = c;
  sv->device = dev;
  if (cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    note_cuda(cudaGetLastError(), "server setup");
    delete sv;
    return WS_ERR_CUDA;
  }
  sv->max_chunks = c.max_batch_ops / ws::kMultiChunk + c.max_batch_reqs + 1;
  sv->slots.resize((size_t)c.max_inflight);
  for (Slot& sl : sv->slots) {
    if (!slot_alloc(sl, c.max_batch_ops, c.max_batch_reqs, sv->max_chunks)) {
      for (Slot& x : sv->slots) slot_free(x);
      delete sv;
      return WS_ERR_OOM;
    }
  }
  // Tables grow through the stream-ordered allocator.  With the default
  // release threshold (0) the pool hands freed memory back to the driver at
  // every synchronisation, and the next multi-gigabyte growth has to map it
  // again inside a launch slot; keep freed memory pooled instead.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return WS_OK;
}

ws_status ws_server_add_table(ws_server* sv, uint64_t capacity, ws_scheme scheme, int metadata, int tile,
                              uint32_t* id) {
  if (!sv || !id) return WS_ERR_INVALID;
  DeviceGuard guard(sv->device);
  size_t fr = 0, tot = 0;
  if (!avail_bytes(sv->device, &fr, &tot)) return WS_ERR_CUDA;
  const double bytes = (double)capacity * 1.25 * (16.0 + (metadata ? 2.0 : 0.0));  // up to pow2 rounding
  if ((double)fr - bytes < sv->cfg.hbm_headroom * (double)tot) return WS_ERR_OOM;  // not admitted
  ws_config c;
  std::memset(&c, 0, sizeof(c));
  c.capacity = capacity;
  c.scheme = scheme;
  c.metadata = metadata;
  c.tile = tile;
  c.device = sv->device;
  ws_table* t = nullptr;
  const ws_status rc = table_create(&c, nullptr, &t);
  if (rc != WS_OK) return rc;
  std::lock_guard<std::mutex> lk(sv->mu);
  STable st;
  st.t = t;
  sv->tables.push_back(st);
  sv->n_tables.store((uint32_t)sv->tables.size());
  *id = (uint32_t)(sv->tables.size() - 1);
  return WS_OK;
}

ws_status ws_server_submit(ws_server* sv, const ws_request* r, uint64_t* id) {
  if (!sv || !r || (r->n && (!r->ops || !r->keys))) return WS_ERR_INVALID;
  if (r->n > sv->cfg.max_batch_ops) return WS_ERR_INVALID;
  if (r->table >= sv->n_tables.load()) return WS_ERR_INVALID;
  SReq q;
  q.r = *r;
  q.t_submit = now_s();
  {
    std::lock_guard<std::mutex> il(sv->in_mu);
    q.id = sv->n_submitted.load();
    sv->inbox.push_back(q);
    sv->n_submitted.store(q.id + 1);
  }
  sv->cv_in.notify_one();
  if (id) *id = q.id;
  return WS_OK;
}

ws_status ws_server_poll(ws_server* sv, ws_completion* out, uint64_t max, uint64_t* n_out, int wait_ms) {
  if (!sv || !n_out || (max && !out)) return WS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (sv->done.empty() && wait_ms > 0)
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !sv->done.empty(); });
  const uint64_t n = std::min<uint64_t>(max, sv->done.size());
  for (uint64_t i = 0; i < n; ++i) out[i] = sv->done[i];
  sv->done.erase(sv->done.begin(), sv->done.begin() + (long)n);
  *n_out = n;
  return sv->error ? (ws_status)sv->error : WS_OK;
}

ws_status ws_server_pause(ws_server* sv, int paused) {
  if (!sv) return WS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->paused = paused != 0;
  }
  wake_worker(sv);
  return WS_OK;
}

ws_status ws_server_drain(ws_server* sv) {
  if (!sv) return WS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->paused = false;  // draining a paused server would wait forever
  lk.unlock();
  wake_worker(sv);
  lk.lock();
  sv->cv_done.wait(lk, [&] { return sv->n_completed == sv->n_submitted.load(); });
  return sv->error ? (ws_status)sv->error : WS_OK;
}

ws_status ws_server_table(ws_server* sv, uint32_t id, ws_table** out) {
  if (!sv || !out) return WS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (id >= sv->tables.size()) return WS_ERR_INVALID;
  *out = sv->tables[id].t;
  return WS_OK;
}

ws_status ws_server_stats(ws_server* sv, uint64_t* submitted, uint64_t* completed, uint64_t* launches,
                          uint64_t* grows) {
  if (!sv) return WS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (submitted) *submitted = sv->n_submitted.load();
  if (completed) *completed = sv->n_completed;
  if (launches) *launches = sv->n_launches;
  if (grows) *grows = sv->n_grows;
  return WS_OK;
}

ws_status ws_server_destroy(ws_server* sv) {
  if (!sv) return WS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  wake_worker(sv);
  if (sv->worker.joinable()) sv->worker.join();
  {
    DeviceGuard guard(sv->device);
    cudaDeviceSynchronize();
    for (Slot& sl : sv->slots) slot_free(sl);
    for (STable& t : sv->tables) ws_destroy(t.t);
  }
  delete sv;
  return WS_OK;
}

}  // extern "C"
