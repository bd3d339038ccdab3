// ws_batch.cu -- batched mode: many tables and their op batches in one
// persistent kernel per phase and (menu entry, op kind) group, captured once
// into a CUDA graph.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ws_internal.h"
#include "ws_multi.cuh"

using namespace wsi;

struct ws_batch_plan {
  struct Group {  // chunks of one menu entry and op kind, one persistent launch
    int cfg = 0, kind = 0;
    size_t chunk_off = 0, n_chunks = 0;
  };
  struct Phase {
    size_t item_off = 0, n_items = 0, chunk_off = 0, n_chunks = 0;
    std::vector<Group> groups;
  };
  int device = 0, num_sms = 0;
  std::vector<ws_batch_item> src;     // the caller's items, sorted by phase then size
  std::vector<int> src_phase_rank;    // dense phase index of each item
  std::vector<ws::MultiItem> items;   // device descriptors, one per menu item
  std::vector<int> menu_item_of;      // src index -> items index, or -1 (fallback)
  std::vector<Phase> phases;
  std::vector<ws::MultiChunk> chunks;
  std::vector<ws_table*> tables;      // distinct tables
  std::vector<int> erase_in_plan;     // per distinct table
  std::vector<int> shortcut_seen;     // never_erased of each table when the graph was built
  ws::MultiItem* d_items = nullptr;
  ws::MultiChunk* d_chunks = nullptr;
  u32* d_tickets = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

namespace {

void release(ws_batch_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_items) cudaFree(p->d_items);
  if (p->d_chunks) cudaFree(p->d_chunks);
  if (p->d_tickets) cudaFree(p->d_tickets);
  p->exec = nullptr;
  p->graph = nullptr;
  p->d_items = nullptr;
  p->d_chunks = nullptr;
  p->d_tickets = nullptr;
}

int table_index(const ws_batch_plan* p, const ws_table* t) {
  for (size_t i = 0; i < p->tables.size(); ++i)
    if (p->tables[i] == t) return (int)i;
  return -1;
}

ws::TableView view_for(const ws_batch_plan* p, const ws_table* t) {
  ws::TableView tv = t->tv;
  const int ti = table_index(p, t);
  tv.shortcut = (t->never_erased && !p->erase_in_plan[ti]) ? 1 : 0;
  return tv;
}

int kind_of(int bk) {
  return bk == WS_BK_QUERY ? ws::KIND_QUERY : bk == WS_BK_ERASE ? ws::KIND_ERASE : ws::KIND_UPSERT;
}

int op_of(const ws_batch_item& it) { return it.kind == WS_BK_INSERT ? ws::OP_INSERT : it.op; }

// Build descriptors and chunks, upload them, capture the phases into a graph.
ws_status build(ws_batch_plan* p) {
  release(p);
  p->items.clear();
  p->chunks.clear();
  p->menu_item_of.assign(p->src.size(), -1);
  p->phases.clear();
  p->shortcut_seen.clear();
  for (ws_table* t : p->tables) p->shortcut_seen.push_back(t->never_erased);
  int nph = p->src.empty() ? 0 : p->src_phase_rank.back() + 1;
  p->phases.resize((size_t)nph);
  // per phase: does a table see an erase in this phase?
  for (int ph = 0; ph < nph; ++ph) {
    std::vector<int> erased(p->tables.size(), 0);
    for (size_t i = 0; i < p->src.size(); ++i)
      if (p->src_phase_rank[i] == ph && p->src[i].kind == WS_BK_ERASE) erased[table_index(p, p->src[i].table)] = 1;
    ws_batch_plan::Phase& P = p->phases[(size_t)ph];
    P.item_off = p->items.size();
    P.chunk_off = p->chunks.size();
    // the phase's menu items grouped by (menu entry, kind), larger items first
    // inside a group (the src order): one persistent launch per group
    std::vector<size_t> sel;
    for (size_t i = 0; i < p->src.size(); ++i) {
      if (p->src_phase_rank[i] != ph || p->src[i].n == 0) continue;
      const ws_table* t = p->src[i].table;
      if (ws::multi_menu_index(t->scheme, t->meta != 0, (int)t->B, t->T) >= 0) sel.push_back(i);
    }
    auto key_of = [&](size_t i) {
      const ws_table* t = p->src[i].table;
      return ws::multi_menu_index(t->scheme, t->meta != 0, (int)t->B, t->T) * 8 + kind_of(p->src[i].kind);
    };
    std::stable_sort(sel.begin(), sel.end(), [&](size_t x, size_t y) { return key_of(x) < key_of(y); });
    for (size_t i : sel) {
      const ws_batch_item& s = p->src[i];
      const ws_table* t = s.table;
      const int cfg = ws::multi_menu_index(t->scheme, t->meta != 0, (int)t->B, t->T);
      ws::MultiItem m;
      std::memset(&m, 0, sizeof(m));
      m.tv = view_for(p, t);
      m.a.keys = reinterpret_cast<const u64*>(s.keys);
      m.a.vals = reinterpret_cast<const u64*>(s.vals);
      m.a.ops = nullptr;
      m.a.vals_out = reinterpret_cast<u64*>(s.vals_out);
      m.a.status_out = s.status_out;
      m.a.n = s.n;
      m.a.op = op_of(s);
      m.a.key_stride = 1;
      m.a.flags = 0;
      m.kind = kind_of(s.kind);
      m.cfg = cfg;
      m.lockfree = (m.kind == ws::KIND_UPSERT && !erased[table_index(p, t)]) ? 1 : 0;
      const u32 idx = (u32)p->items.size();
      p->menu_item_of[i] = (int)idx;
      p->items.push_back(m);
      if (P.groups.empty() || P.groups.back().cfg != cfg || P.groups.back().kind != m.kind) {
        ws_batch_plan::Group G;
        G.cfg = cfg;
        G.kind = m.kind;
        G.chunk_off = p->chunks.size();
        P.groups.push_back(G);
      }
      for (u64 st = 0; st < s.n; st += ws::kMultiChunk) {
        ws::MultiChunk c;
        c.item = idx;
        c.pad = 0;
        c.start = st;
        p->chunks.push_back(c);
        ++P.groups.back().n_chunks;
      }
    }
    P.n_items = p->items.size() - P.item_off;
    P.n_chunks = p->chunks.size() - P.chunk_off;
  }
  if (!p->items.empty()) {
    WS_CUDA(cudaMalloc(&p->d_items, p->items.size() * sizeof(ws::MultiItem)));
    WS_CUDA(cudaMemcpy(p->d_items, p->items.data(), p->items.size() * sizeof(ws::MultiItem), cudaMemcpyHostToDevice));
  }
  if (!p->chunks.empty()) {
    WS_CUDA(cudaMalloc(&p->d_chunks, p->chunks.size() * sizeof(ws::MultiChunk)));
    WS_CUDA(cudaMemcpy(p->d_chunks, p->chunks.data(), p->chunks.size() * sizeof(ws::MultiChunk),
                       cudaMemcpyHostToDevice));
  }
  size_t n_groups = 0;
  for (const ws_batch_plan::Phase& P : p->phases) n_groups += P.groups.size();
  WS_CUDA(cudaMalloc(&p->d_tickets, (n_groups > 0 ? n_groups : 1) * sizeof(u32)));

  WS_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  size_t gi = 0;
  for (int ph = 0; ph < nph && err == cudaSuccess; ++ph) {
    const ws_batch_plan::Phase& P = p->phases[(size_t)ph];
    for (const ws_batch_plan::Group& G : P.groups) {
      if (err != cudaSuccess) break;
      u32* ticket = p->d_tickets + gi++;
      err = cudaMemsetAsync(ticket, 0, sizeof(u32), p->cap);
      if (err == cudaSuccess) {
        ws::MultiGroup g{p->d_items, p->d_chunks + G.chunk_off, nullptr, 0, 0, (u32)G.n_chunks, ticket};
        err = ws::launch_multi(G.cfg, G.kind, g, p->cap, p->num_sms);
      }
    }
    for (size_t i = 0; i < p->src.size() && err == cudaSuccess; ++i) {
      if (p->src_phase_rank[i] != ph || p->menu_item_of[i] >= 0 || p->src[i].n == 0) continue;
      const ws_batch_item& s = p->src[i];
      ws::BatchArgs a{reinterpret_cast<const u64*>(s.keys), reinterpret_cast<const u64*>(s.vals), nullptr,
                      reinterpret_cast<u64*>(s.vals_out), s.status_out, s.n, op_of(s), 1, 0};
      // Fallback items run as their own kernels after the phase's persistent
      // kernel (stream order inside the graph), so they never race its erases.
      const int kind = kind_of(s.kind);
      err = dispatch(s.table, view_for(p, s.table), a, kind, p->cap);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(p->cap, &g);
  if (err == cudaSuccess) err = e2;
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    note_cuda(err, "batch plan capture");
    return WS_ERR_CUDA;
  }
  p->graph = g;
  WS_CUDA(cudaGraphInstantiate(&p->exec, p->graph, 0));
  return WS_OK;
}

}  // namespace

extern "C" {

ws_status ws_batch_plan_create(const ws_batch_item* items, uint64_t n_items, ws_batch_plan** out) {
  if (!out || (n_items && !items)) return WS_ERR_INVALID;
  *out = nullptr;
  if (n_items == 0) return WS_ERR_INVALID;
  const int dev = items[0].table ? items[0].table->device : -1;
  for (uint64_t i = 0; i < n_items; ++i) {
    const ws_batch_item& it = items[i];
    if (!it.table || it.table->device != dev) return WS_ERR_INVALID;
    if (it.kind < WS_BK_INSERT || it.kind > WS_BK_ERASE || it.phase < 0) return WS_ERR_INVALID;
    if (it.kind == WS_BK_UPSERT && (it.op < WS_OP_ADD || it.op > WS_OP_INSERT)) return WS_ERR_INVALID;
    if (it.n == 0) continue;
    if (!it.keys || ((reinterpret_cast<uintptr_t>(it.keys) | reinterpret_cast<uintptr_t>(it.vals) |
                      reinterpret_cast<uintptr_t>(it.vals_out)) & 7u))
      return WS_ERR_INVALID;
    if ((it.kind == WS_BK_INSERT || it.kind == WS_BK_UPSERT) && !it.vals) return WS_ERR_INVALID;
    if (it.kind == WS_BK_QUERY && !it.vals_out && !it.status_out) return WS_ERR_INVALID;
  }
  DeviceGuard guard(dev);
  for (uint64_t i = 0; i < n_items; ++i) {
    const ws_batch_item& it = items[i];
    if (it.n == 0) continue;
    const void* ptrs[5] = {it.keys, it.vals, it.vals_out, it.status_out, nullptr};
    for (const void* q : ptrs)
      if (q && classify(q, dev) != PTR_DEVICE) return WS_ERR_INVALID;  // batched mode is device-resident
  }
  ws_batch_plan* p = new (std::nothrow) ws_batch_plan();
  if (!p) return WS_ERR_OOM;
  p->device = dev;
  if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
    note_cuda(cudaGetLastError(), "batch plan setup");
    delete p;
    return WS_ERR_CUDA;
  }
  // phases in increasing order; inside a phase, larger items first (their
  // chunks are taken first, which shortens the tail of the persistent launch)
  std::vector<uint64_t> order(n_items);
  for (uint64_t i = 0; i < n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) {
    if (items[a].phase != items[b].phase) return items[a].phase < items[b].phase;
    return items[a].n > items[b].n;
  });
  int rank = -1, last = -1;
  for (uint64_t k = 0; k < n_items; ++k) {
    const ws_batch_item& it = items[order[k]];
    if (it.phase != last) {
      ++rank;
      last = it.phase;
    }
    p->src.push_back(it);
    p->src_phase_rank.push_back(rank);
    if (table_index(p, it.table) < 0) {
      p->tables.push_back(it.table);
      p->erase_in_plan.push_back(0);
    }
    if (it.kind == WS_BK_ERASE) p->erase_in_plan[(size_t)table_index(p, it.table)] = 1;
  }
  const ws_status rc = build(p);
  if (rc != WS_OK) {
    release(p);
    cudaStreamDestroy(p->cap);
    delete p;
    return rc;
  }
  *out = p;
  return WS_OK;
}

ws_status ws_batch_plan_launch(ws_batch_plan* p, ws_stream stream) {
  if (!p) return WS_ERR_INVALID;
  DeviceGuard guard(p->device);
  // A table erased since the graph was built has lost the two-choice
  // shortcut: rebuild so that no descriptor still allows it.
  for (size_t i = 0; i < p->tables.size(); ++i) {
    if (p->tables[i]->never_erased != p->shortcut_seen[i]) {
      const ws_status rc = build(p);
      if (rc != WS_OK) return rc;
      break;
    }
  }
  WS_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  for (size_t i = 0; i < p->tables.size(); ++i) {
    p->tables[i]->last_stream = (cudaStream_t)stream;
    if (p->erase_in_plan[i]) p->tables[i]->never_erased = 0;
  }
  for (size_t i = 0; i < p->tables.size(); ++i) p->shortcut_seen[i] = p->tables[i]->never_erased;
  return WS_OK;
}

ws_status ws_batch_plan_info(const ws_batch_plan* p, uint64_t* n_phases, uint64_t* n_chunks,
                             uint64_t* n_fallback_items) {
  if (!p) return WS_ERR_INVALID;
  if (n_phases) *n_phases = p->phases.size();
  if (n_chunks) *n_chunks = p->chunks.size();
  if (n_fallback_items) {
    uint64_t f = 0;
    for (size_t i = 0; i < p->src.size(); ++i)
      if (p->menu_item_of[i] < 0 && p->src[i].n) ++f;
    *n_fallback_items = f;
  }
  return WS_OK;
}

ws_status ws_batch_plan_destroy(ws_batch_plan* p) {
  if (!p) return WS_ERR_INVALID;
  {
    DeviceGuard guard(p->device);
    cudaStreamSynchronize(p->cap);
    cudaDeviceSynchronize();
    release(p);
    cudaStreamDestroy(p->cap);
  }
  delete p;
  return WS_OK;
}

}  // extern "C"
