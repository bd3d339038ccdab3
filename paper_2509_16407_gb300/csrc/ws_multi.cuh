// ws_multi.cuh -- one persistent launch over many tables (batched mode).
//
// A phase is a list of items (table, op kind, op arrays).  The host cuts every
// item into chunks of up to kMultiChunk ops; the persistent blocks take chunks
// in order from a ticket counter (dynamic scheduling: item sizes differ by
// four orders of magnitude) and each warp of a block serves 32 ops of the
// chunk with the same tile code as the single-table kernel.  The table
// configuration of an item selects one of a fixed menu of compiled tile
// configurations at run time.
#pragma once
#include "ws_kernels.cuh"

namespace ws {

constexpr int kMultiChunk = kWarps * 32;  // ops per chunk = one block iteration

struct MultiItem {
  TableView tv;
  BatchArgs a;
  int kind;      // KIND_QUERY / KIND_UPSERT / KIND_ERASE / KIND_MIXED (per-op codes in a.ops)
  int cfg;       // index into the menu
  int lockfree;  // no erase of this table in this phase
  int pad;
};

struct MultiChunk {
  u32 item;
  u32 pad;
  u64 start;
};

// Menu of compiled configurations (scheme, metadata, bucket slots, tile).
#define WS_MULTI_MENU(X)            \
  X(0, SCHEME_DOUBLE, false, 8, 4)  \
  X(1, SCHEME_DOUBLE, false, 8, 8)  \
  X(2, SCHEME_DOUBLE, true, 32, 4)  \
  X(3, SCHEME_DOUBLE, true, 32, 8)  \
  X(4, SCHEME_P2, false, 32, 8)     \
  X(5, SCHEME_P2, false, 32, 32)    \
  X(6, SCHEME_P2, true, 32, 4)      \
  X(7, SCHEME_P2, true, 32, 8)
constexpr int kMultiMenu = 8;

// Serves ops [base, base + 32) of one item with one warp (the single-table
// chunk routine, with the op kind chosen at run time); returns the warp's
// count delta.
template <int SCHEME, bool META, int B, int T>
__device__ __forceinline__ int multi_warp(const MultiItem& it, u64 base, WarpSmem& sm, int lane) {
  if (it.kind == KIND_QUERY)
    return warp_chunk<SCHEME, META, B, T, KIND_QUERY>(it.tv, it.a, 0, false, base, sm, lane);
  if (it.kind == KIND_UPSERT)
    return warp_chunk<SCHEME, META, B, T, KIND_UPSERT>(it.tv, it.a, it.a.op, it.lockfree != 0, base, sm, lane);
  if (it.kind == KIND_MIXED)
    return warp_chunk<SCHEME, META, B, T, KIND_MIXED>(it.tv, it.a, 0, false, base, sm, lane);
  return warp_chunk<SCHEME, META, B, T, KIND_ERASE>(it.tv, it.a, 0, false, base, sm, lane);
}

#ifndef WS_MULTI_NO_KERNEL  // units that only need the pieces above define this
__global__ void __launch_bounds__(kThreads, 2)
    multi_kernel(const MultiItem* __restrict__ items, const MultiChunk* __restrict__ chunks, u32 n_chunks,
                 u32* ticket) {
  __shared__ WarpSmem s_w[kWarps];
  __shared__ u32 s_chunk;
  __shared__ MultiChunk s_ch;
  __shared__ __align__(16) MultiItem s_it;
  static_assert(sizeof(MultiItem) % 8 == 0, "item copy");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  u32 cur_item = 0xffffffffu;
  for (;;) {
    if (threadIdx.x == 0) {
      s_chunk = atomicAdd(ticket, 1u);
      if (s_chunk < n_chunks) s_ch = chunks[s_chunk];
    }
    __syncthreads();
    const u32 ci = s_chunk;
    if (ci >= n_chunks) break;
    const MultiChunk ch = s_ch;
    if (ch.item != cur_item) {  // block-uniform: stage the item descriptor once
      const u64* src = reinterpret_cast<const u64*>(items + ch.item);
      u64* dst = reinterpret_cast<u64*>(&s_it);
      for (int q = threadIdx.x; q < (int)(sizeof(MultiItem) / 8); q += blockDim.x) dst[q] = src[q];
      cur_item = ch.item;
    }
    __syncthreads();
    const MultiItem& it = s_it;
    const u64 base = ch.start + (u64)w * 32;
    int d = 0;
    if (base < it.a.n) {
      switch (it.cfg) {
#define WS_MULTI_CASE(ID, SCH, MT, BB, TT)                                                      \
  case ID:                                                                                       \
    d = multi_warp<SCH, MT, BB, TT>(it, base, s_w[w], lane); \
    break;
        WS_MULTI_MENU(WS_MULTI_CASE)
#undef WS_MULTI_CASE
        default: break;
      }
    }
    if (it.kind != KIND_QUERY) {
      d = __reduce_add_sync(0xffffffffu, d);  // every lane reaches this: base is warp-uniform
      if (lane == 0 && d) atomicAdd((unsigned long long*)&it.tv.ctr->count, (unsigned long long)(long long)d);
    }
    __syncthreads();  // s_it / s_ch are rewritten by the next iteration
  }
}
#endif

// Menu index of a configuration, or -1.
inline int multi_menu_index(int scheme, bool meta, int B, int T) {
#define WS_MULTI_FIND(ID, SCH, MT, BB, TT) \
  if (scheme == SCH && meta == MT && B == BB && T == TT) return ID;
  WS_MULTI_MENU(WS_MULTI_FIND)
#undef WS_MULTI_FIND
  return -1;
}

}  // namespace ws
