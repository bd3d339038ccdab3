// ws_noalloc.cu -- ws_batch_run_noalloc: batched mode without any device
// allocation.
//
// Who needs it: code that must not call cudaMalloc / cudaFree -- a caller
// running inside a memory budget that a caching allocator (a framework's
// pool) already holds in full, a latency-critical loop that cannot afford
// cudaFree's implicit device-wide synchronisation, or a process that has
// reserved all device memory up front.  ws_batch_plan_create allocates its
// descriptor, chunk and ticket arrays; this entry point keeps the same
// scratch in one fixed, file-scope device array instead, so a call
// allocates nothing.
//
// The array (kScratchBytes, about 193 KiB) exists on every GPU that loads
// the library until the process exits.  Its device address is looked up once
// per device, on the first call that uses that device (cudaGetSymbolAddress
// with the device current).
// Every call reuses the same array and it keeps the last call's contents:
// each call rewrites the descriptors it uses and zeroes its work tickets.
// Calls whose work overlaps on the GPU race on the array -- order them on one
// stream or synchronise between them.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ws_internal.h"
#include "ws_multi.cuh"

using namespace wsi;

namespace {

constexpr uint32_t kMaxItems = 1024;  // items per call
constexpr uint32_t kMaxPhases = 16;   // distinct phases per call
constexpr int kMaxDevices = 64;

// Layout of the scratch array.
struct NoallocScratch {
  u32 tickets[kMaxItems];         // one work ticket per launch group, zeroed by every call
  u32 prefix[kMaxItems + 1];      // chunk prefix sums over the (phase, entry, kind)-sorted items
  u32 pad[(256 - ((kMaxItems + kMaxItems + 1) * 4) % 256) / 4];
  ws::MultiItem items[kMaxItems];
};
constexpr size_t kScratchBytes = sizeof(NoallocScratch);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
NoallocScratch* g_scratch_of[kMaxDevices] = {};

// Device address of the scratch array on `dev` (current device), looked up once.
cudaError_t scratch_for(int dev, NoallocScratch** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_of[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_of[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_scratch_of[dev];
  return cudaSuccess;
}

int kind_of(int bk) {
  return bk == WS_BK_QUERY ? ws::KIND_QUERY : bk == WS_BK_ERASE ? ws::KIND_ERASE : ws::KIND_UPSERT;
}

// Host-side staging of one call's descriptors (per thread, no heap).
constexpr uint32_t kTableSlots = 2 * kMaxItems;  // open-addressing set of the call's tables
struct HostStage {
  uint32_t order[kMaxItems];
  int64_t key[kMaxItems];          // sort key of each item (phase, menu entry, kind)
  uint32_t phase_idx[kMaxItems];   // index of the item's phase among the call's phases
  uint32_t table_slot[kMaxItems];  // slot of the item's table in `tables`
  ws_table* tables[kTableSlots];
  uint32_t erased_phases[kTableSlots];  // bit p: the table is erased in phase p of the call
  ws::MultiItem items[kMaxItems];
  u32 prefix[kMaxItems + 1];
  u32 phase_begin[kMaxPhases + 1];
  int phase_value[kMaxPhases];
};
thread_local HostStage t_stage;

}  // namespace

extern "C" ws_status ws_batch_run_noalloc(const ws_batch_item* items, uint64_t n_items, ws_stream stream) {
  if (n_items == 0) return WS_OK;
  if (!items) return WS_ERR_INVALID;
  if (n_items > kMaxItems) {
    char msg[128];
    std::snprintf(msg, sizeof(msg), "ws_batch_run_noalloc: %llu items exceed the maximum of %u per call",
                  (unsigned long long)n_items, kMaxItems);
    note_text(msg);
    return WS_ERR_INVALID;
  }
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
    const void* ptrs[4] = {it.keys, it.vals, it.vals_out, it.status_out};
    for (const void* q : ptrs)
      if (q && classify(q, dev) != PTR_DEVICE) return WS_ERR_INVALID;  // device-resident only
  }
  NoallocScratch* scratch = nullptr;
  WS_CUDA(scratch_for(dev, &scratch));
  int num_sms = 0;
  WS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));

  HostStage& hs = t_stage;
  // order by (phase, menu entry, kind), ties by position: the items of one
  // (entry, kind) run of a phase form one persistent launch.  Keys are
  // computed once; the sort works in place (no allocation).
  for (uint32_t i = 0; i < (uint32_t)n_items; ++i) {
    const ws_table* t = items[i].table;
    const int cfg = ws::multi_menu_index(t->scheme, t->meta != 0, (int)t->B, t->T);
    hs.key[i] = ((int64_t)items[i].phase * 16 + (cfg + 1)) * 8 + kind_of(items[i].kind);
    hs.order[i] = i;
  }
  std::sort(hs.order, hs.order + n_items, [&](uint32_t a, uint32_t b) {
    return hs.key[a] != hs.key[b] ? hs.key[a] < hs.key[b] : a < b;
  });
  // phases
  uint32_t n_ph = 0;
  for (uint32_t k = 0; k < (uint32_t)n_items; ++k) {
    const int ph = items[hs.order[k]].phase;
    if (n_ph == 0 || hs.phase_value[n_ph - 1] != ph) {
      if (n_ph == kMaxPhases) {
        char msg[128];
        std::snprintf(msg, sizeof(msg), "ws_batch_run_noalloc: more than %u distinct phases in one call", kMaxPhases);
        note_text(msg);
        return WS_ERR_INVALID;
      }
      hs.phase_value[n_ph] = ph;
      hs.phase_begin[n_ph] = k;
      ++n_ph;
    }
    hs.phase_idx[k] = n_ph - 1;
  }
  hs.phase_begin[n_ph] = (uint32_t)n_items;
  // tables erased anywhere in the call lose the two-choice shortcut for the
  // whole call, and a table erased in a phase takes the locked insert path
  // in that phase: one pass collects, per table, the phases that erase it
  std::memset(hs.tables, 0, sizeof(hs.tables));
  for (uint32_t k = 0; k < (uint32_t)n_items; ++k) {
    ws_table* t = items[hs.order[k]].table;
    uint32_t h = (uint32_t)((reinterpret_cast<uintptr_t>(t) >> 4) * 0x9E3779B1u) & (kTableSlots - 1);
    while (hs.tables[h] && hs.tables[h] != t) h = (h + 1) & (kTableSlots - 1);
    if (!hs.tables[h]) {
      hs.tables[h] = t;
      hs.erased_phases[h] = 0;
    }
    hs.table_slot[k] = h;
    if (items[hs.order[k]].kind == WS_BK_ERASE) hs.erased_phases[h] |= 1u << hs.phase_idx[k];
  }
  hs.prefix[0] = 0;
  uint64_t chunks = 0;
  for (uint32_t k = 0; k < (uint32_t)n_items; ++k) {
    const ws_batch_item& s = items[hs.order[k]];
    const ws_table* t = s.table;
    const uint32_t er = hs.erased_phases[hs.table_slot[k]];
    const bool erased_call = er != 0, erased_phase = ((er >> hs.phase_idx[k]) & 1u) != 0;
    ws::MultiItem& m = hs.items[k];
    std::memset(&m, 0, sizeof(m));
    m.tv = t->tv;
    m.tv.shortcut = (t->never_erased && !erased_call) ? 1 : 0;
    m.a.keys = reinterpret_cast<const u64*>(s.keys);
    m.a.vals = reinterpret_cast<const u64*>(s.vals);
    m.a.vals_out = reinterpret_cast<u64*>(s.vals_out);
    m.a.status_out = s.status_out;
    m.a.n = s.n;
    m.a.op = s.kind == WS_BK_INSERT ? ws::OP_INSERT : s.op;
    m.a.key_stride = 1;
    m.kind = kind_of(s.kind);
    m.cfg = ws::multi_menu_index(t->scheme, t->meta != 0, (int)t->B, t->T);
    m.lockfree = (m.kind == ws::KIND_UPSERT && !erased_phase) ? 1 : 0;
    // items outside the compiled menu run as single-table kernels below
    const u64 nc = (m.cfg >= 0) ? (s.n + ws::kMultiChunk - 1) / ws::kMultiChunk : 0;
    chunks += nc;
    if (chunks > 0xffffffffull) return WS_ERR_INVALID;
    hs.prefix[k + 1] = (u32)chunks;
  }
  // The call is valid from here on.  Tables it erases lose the shortcut
  // before anything is enqueued, so an error return below cannot leave a
  // table with tombstones that later calls would still read with the
  // shortcut.
  for (uint64_t i = 0; i < n_items; ++i)
    if (items[i].kind == WS_BK_ERASE) items[i].table->never_erased = 0;
  cudaStream_t st = (cudaStream_t)stream;
  WS_CUDA(cudaMemcpyAsync(scratch->prefix, hs.prefix, (n_items + 1) * sizeof(u32), cudaMemcpyHostToDevice, st));
  WS_CUDA(cudaMemcpyAsync(scratch->items, hs.items, n_items * sizeof(ws::MultiItem), cudaMemcpyHostToDevice, st));
  WS_CUDA(cudaMemsetAsync(scratch->tickets, 0, sizeof(scratch->tickets), st));
  uint32_t n_groups = 0;
  for (uint32_t p = 0; p < n_ph; ++p) {
    const uint32_t i0 = hs.phase_begin[p], i1 = hs.phase_begin[p + 1];
    for (uint32_t g0 = i0; g0 < i1;) {  // runs of one (menu entry, kind)
      uint32_t g1 = g0 + 1;
      while (g1 < i1 && hs.items[g1].cfg == hs.items[g0].cfg && hs.items[g1].kind == hs.items[g0].kind) ++g1;
      const u32 nch = hs.prefix[g1] - hs.prefix[g0];
      if (hs.items[g0].cfg >= 0 && nch) {
        ws::MultiGroup g{scratch->items, nullptr, scratch->prefix, g0, g1, nch, scratch->tickets + n_groups++};
        WS_CUDA(ws::launch_multi(hs.items[g0].cfg, hs.items[g0].kind, g, st, num_sms));
      }
      g0 = g1;
    }
    for (uint32_t k = i0; k < i1; ++k) {  // configurations outside the menu
      const ws::MultiItem& m = hs.items[k];
      if (m.cfg >= 0 || m.a.n == 0) continue;
      WS_CUDA(dispatch(items[hs.order[k]].table, m.tv, m.a, m.kind, st));
    }
  }
  for (uint64_t i = 0; i < n_items; ++i) items[i].table->last_stream = st;
  return WS_OK;
}
