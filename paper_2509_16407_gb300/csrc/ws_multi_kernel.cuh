// ws_multi_kernel.cuh -- the persistent multi-table kernel template, included
// only by the per-menu-entry translation units ws_multi_<entry>.cu.
#pragma once
#include "ws_multi.cuh"

namespace ws {

// One warp's share [begin, end) of a chunk of one item: streaming lanes, or
// -- for two-choice tables with plain 32-slot buckets -- 32-op chunks with
// whole-bucket rounds.  Returns the warp's count delta.
template <int SCHEME, bool META, int B, int T, int KIND>
__device__ __forceinline__ int multi_share(const MultiItem& it, u64 begin, u64 end, WarpSmem& sm, int lane) {
  constexpr bool kRounds = (SCHEME == SCHEME_P2) && !META && B == 32;
  const int op = (KIND == KIND_UPSERT) ? it.a.op : 0;
  const bool lockfree = (KIND == KIND_UPSERT) && it.lockfree != 0;
  if constexpr (kRounds) {
    int d = 0;
    for (u64 b = begin; b < end; b += 32)
      d += warp_chunk<SCHEME, META, B, T, KIND>(it.tv, it.a, op, lockfree, b, sm, lane);
    return d;
  } else {
    return warp_stream<SCHEME, META, B, T, KIND>(it.tv, it.a, op, lockfree, begin, end, sm, lane);
  }
}

template <int SCHEME, bool META, int B, int T, int KIND>
__global__ void __launch_bounds__(kThreads, 4) multi_kernel(MultiGroup g) {
  __shared__ WarpSmem s_w[kWarps];
  __shared__ u32 s_item;
  __shared__ u64 s_start;
  __shared__ int s_stop;
  __shared__ __align__(16) MultiItem s_it;
  static_assert(sizeof(MultiItem) % 8 == 0, "item copy");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  u32 cur_item = 0xffffffffu;
  for (;;) {
    if (threadIdx.x == 0) {
      const u32 c = atomicAdd(g.ticket, 1u);
      s_stop = c >= g.n_chunks;
      if (!s_stop) {
        if (g.chunks) {
          const MultiChunk ch = g.chunks[c];
          s_item = ch.item;
          s_start = ch.start;
        } else {
          const u32 gc = g.prefix[g.i0] + c;
          u32 lo = g.i0, hi = g.i1 - 1;  // largest item with prefix[item] <= gc
          while (lo < hi) {
            const u32 mid = (lo + hi + 1) / 2;
            if (g.prefix[mid] <= gc)
              lo = mid;
            else
              hi = mid - 1;
          }
          s_item = lo;
          s_start = (u64)(gc - g.prefix[lo]) * kMultiChunk;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const u32 item = s_item;
    const u64 start = s_start;
    if (item != cur_item) {  // block-uniform: stage the item descriptor once
      const u64* src = reinterpret_cast<const u64*>(g.items + item);
      u64* dst = reinterpret_cast<u64*>(&s_it);
      for (int q = threadIdx.x; q < (int)(sizeof(MultiItem) / 8); q += blockDim.x) dst[q] = src[q];
      cur_item = item;
    }
    __syncthreads();
    const MultiItem& it = s_it;
    const u64 base = start + (u64)w * kWarpShare;
    int d = 0;
    if (base < it.a.n) {
      const u64 end = (it.a.n - base < (u64)kWarpShare) ? it.a.n : base + kWarpShare;
      d = multi_share<SCHEME, META, B, T, KIND>(it, base, end, s_w[w], lane);
    }
    if (KIND != KIND_QUERY) {
      d = __reduce_add_sync(0xffffffffu, d);  // every lane reaches this: base is warp-uniform
      if (lane == 0 && d) atomicAdd((unsigned long long*)&it.tv.ctr->count, (unsigned long long)(long long)d);
    }
    __syncthreads();  // s_it is rewritten by the next iteration
  }
}

template <void (*KERN)(MultiGroup)>
cudaError_t launch_multi_one(const MultiGroup& g, cudaStream_t s, int num_sms) {
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, KERN, kThreads, 0) != cudaSuccess || o < 1) o = 1;
    occ = o;
  }
  const u64 cap = (u64)occ * (u64)(num_sms > 0 ? num_sms : 1);
  const unsigned grid = (unsigned)(g.n_chunks < cap ? g.n_chunks : cap);
  if (grid == 0) return cudaSuccess;
  KERN<<<grid, kThreads, 0, s>>>(g);
  return cudaGetLastError();
}

template <int SCHEME, bool META, int B, int T>
cudaError_t launch_multi_cfg(int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  switch (kind) {
    case KIND_QUERY: return launch_multi_one<multi_kernel<SCHEME, META, B, T, KIND_QUERY>>(g, s, num_sms);
    case KIND_UPSERT: return launch_multi_one<multi_kernel<SCHEME, META, B, T, KIND_UPSERT>>(g, s, num_sms);
    case KIND_ERASE: return launch_multi_one<multi_kernel<SCHEME, META, B, T, KIND_ERASE>>(g, s, num_sms);
    case KIND_MIXED: return launch_multi_one<multi_kernel<SCHEME, META, B, T, KIND_MIXED>>(g, s, num_sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
