// ws_peak.cu -- read-bandwidth probes: the denominators of the roofline for
// tables that fit in L2 (measured here, on the running GPU) beside the HBM
// copy bandwidth measured for tables that do not.
//
// Access patterns over a device buffer that the kernel touches `passes`
// times, through L2 only (.cg: no L1 reuse between passes):
//   0 sequential reads -- each thread reads 16-byte words at a grid stride,
//     the best case for any memory level;
//   1, 2, 3 random reads of 128, 64 and 32 bytes -- 8, 4 or 2 lanes read one
//     block together (16 bytes each, as a bucket snapshot is copied), the
//     block index drawn from a counter-based hash per (pass, group, step),
//     `depth` independent blocks in flight per group: the probes' pattern at
//     line, half-line and sector granularity;
//   4, 5 random writes of 32 and 128 bytes -- the same with stores: the
//     write-back traffic of slot updates;
//   6, 7 a metadata probe's dependent pair of reads -- a 64-byte tag line,
//     then one 16-byte slot chosen from the tag data -- with the tags in a
//     separate array (6, the tables' layout) or each bucket's tag line and
//     slots in one 640-byte block (7, a co-located layout);
//   8-11 random 128-byte reads confined to regions of 128 KiB, 512 KiB,
//     2 MiB or 8 MiB: each block of threads reads 8 x depth random lines
//     per group in one region, then moves to another.
// With a buffer smaller than L2 the second pass onwards is served by L2.
#include <cstdio>

#include "ws_internal.h"

using namespace wsi;

namespace {

__device__ __forceinline__ uint4 ld_cg16(const void* p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__global__ void __launch_bounds__(256) read_seq(uint4* __restrict__ p, uint64_t n16, int passes,
                                                unsigned int* sink) {
  uint32_t acc = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < passes; ++r) {
    uint64_t i = first;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = ld_cg16(p + i), b = ld_cg16(p + i + stride), c = ld_cg16(p + i + 2 * stride),
                  d = ld_cg16(p + i + 3 * stride);
      acc ^= a.x ^ b.y ^ c.z ^ d.w;
    }
    for (; i < n16; i += stride) acc ^= ld_cg16(p + i).x;
  }
  if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);  // keeps the loads
}

// splitmix64's finaliser as a counter-based index generator
__device__ __forceinline__ uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Random accesses of W bytes (W = 16 * LPG): LPG lanes read (or write) one
// W-byte block together, D independent blocks in flight per group.
template <int LPG, int D, bool WRITE>
__global__ void __launch_bounds__(256) random_blocks(uint4* __restrict__ p, uint64_t n_blocks, int steps,
                                                     int passes, unsigned int* sink) {
  uint32_t acc = 0;
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / LPG;
  const uint64_t group = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPG;
  const int part = threadIdx.x % LPG;
  for (int r = 0; r < passes; ++r) {
    const uint64_t ctr = ((uint64_t)r * groups + group) * (uint64_t)steps;
    for (int s = 0; s < steps; s += D) {
      // D independent blocks per step, the same for the group's lanes
      uint64_t l[D];
#pragma unroll
      for (int k = 0; k < D; ++k) l[k] = ((mix(ctr + (uint64_t)(s + k)) >> 32) * n_blocks) >> 32;
      if (WRITE) {
#pragma unroll
        for (int k = 0; k < D; ++k)
          asm volatile("st.global.cg.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p + l[k] * LPG + part), "r"(k),
                       "r"(s), "r"(r), "r"(part)
                       : "memory");
      } else {
        uint4 v[D];
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = ld_cg16(p + l[k] * LPG + part);
#pragma unroll
        for (int k = 0; k < D; ++k) acc ^= v[k].x ^ v[k].w;
      }
    }
  }
  if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);
}

// A metadata probe's two dependent reads: a 64-byte tag line (four lanes),
// then one 16-byte slot whose position depends on the tag data.  SPLIT: the
// tag lines and the slots live in separate halves of the buffer (tags in
// their own array, as the tables keep them); otherwise each 640-byte block
// holds one bucket's tag line followed by its 32 slots (a co-located layout),
// so the slot read falls in the block the tag line opened.  D pairs in
// flight per group of four lanes.
template <bool SPLIT, int D>
__global__ void __launch_bounds__(256) tag_then_slot(uint4* __restrict__ p, uint64_t n_buckets, int steps, int passes,
                                                    unsigned int* sink) {
  uint32_t acc = 0;
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / 4;
  const uint64_t group = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 4;
  const int part = threadIdx.x % 4;
  // 16-byte units: SPLIT -> tags [0, 4 nb), slots [4 nb, 4 nb + 32 nb);
  // co-located -> bucket b at 40 b (4 tag units + 32 slot units + 4 spare)
  for (int r = 0; r < passes; ++r) {
    const uint64_t ctr = ((uint64_t)r * groups + group) * (uint64_t)steps;
    for (int s = 0; s < steps; s += D) {
      uint64_t b[D];
      uint4 t[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        b[k] = ((mix(ctr + (uint64_t)(s + k)) >> 32) * n_buckets) >> 32;
        t[k] = ld_cg16(p + (SPLIT ? b[k] * 4 : b[k] * 40) + part);
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        // the slot index depends on the loaded tags (one lane's word, shared)
        const uint32_t w = __shfl_sync(0xffffffffu, t[k].x ^ t[k].y, (threadIdx.x & 31) & ~3);
        const uint64_t q = (mix(w ^ (ctr + (uint64_t)(s + k))) >> 59);  // 0..31
        const uint64_t unit = SPLIT ? 4 * n_buckets + b[k] * 32 + q : b[k] * 40 + 4 + q;
        if (part == 0) {
          const uint4 v = ld_cg16(p + unit);
          acc ^= v.x ^ v.w;
        }
      }
    }
  }
  if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);
}

// Random 128-byte reads confined to regions: every block of threads works
// in one region of `region_lines` lines at a time (its groups of eight lanes
// read random lines of it, `per_region` lines each), then moves to another
// random region -- the access pattern of a batch processed partition by
// partition when partitions follow the table's address order.
__global__ void __launch_bounds__(256) regional_lines(uint4* __restrict__ p, uint64_t n_lines, uint64_t region_lines,
                                                     int steps, int per_region, int passes, unsigned int* sink) {
  uint32_t acc = 0;
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / 8;
  const uint64_t group = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 8;
  const int part = threadIdx.x % 8;
  const uint64_t n_regions = n_lines / region_lines;
  for (int r = 0; r < passes; ++r) {
    const uint64_t ctr = ((uint64_t)r * groups + group) * (uint64_t)steps;
    for (int s = 0; s < steps; s += 4) {
      const uint64_t epoch = ((uint64_t)r * (uint64_t)steps + (uint64_t)s) / (uint64_t)per_region;
      const uint64_t reg = ((mix(((uint64_t)blockIdx.x << 32) ^ epoch ^ 0x5bd1e995ull) >> 32) * n_regions) >> 32;
      uint64_t l[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        l[k] = reg * region_lines + (((mix(ctr + (uint64_t)(s + k)) >> 32) * region_lines) >> 32);
      const uint4 a = ld_cg16(p + l[0] * 8 + part), b = ld_cg16(p + l[1] * 8 + part),
                  c = ld_cg16(p + l[2] * 8 + part), d = ld_cg16(p + l[3] * 8 + part);
      acc ^= a.x ^ b.y ^ c.z ^ d.w;
    }
  }
  if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);
}

template <int LPG, bool WRITE>
void launch_random(int depth, int grid, uint4* q, uint64_t n_blocks, int steps, int np, unsigned int* sink) {
  switch (depth) {
    case 1: random_blocks<LPG, 1, WRITE><<<grid, 256>>>(q, n_blocks, steps, np, sink); break;
    case 2: random_blocks<LPG, 2, WRITE><<<grid, 256>>>(q, n_blocks, steps, np, sink); break;
    case 4: random_blocks<LPG, 4, WRITE><<<grid, 256>>>(q, n_blocks, steps, np, sink); break;
    default: random_blocks<LPG, 8, WRITE><<<grid, 256>>>(q, n_blocks, steps, np, sink); break;
  }
}

}  // namespace

extern "C" ws_status ws_read_bandwidth(uint64_t bytes, int pattern, int depth, int passes, int device,
                                       double* gbs_out) {
  if (!gbs_out || bytes < (1u << 20) || (bytes & 127u) || passes < 1 || pattern < 0 || pattern > 11 ||
      (depth != 1 && depth != 2 && depth != 4 && depth != 8))
    return WS_ERR_INVALID;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return WS_ERR_CUDA;
  DeviceGuard guard(dev);
  int sms = 0;
  WS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* buf = nullptr;
  unsigned int* sink = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return WS_ERR_OOM;
  }
  if (cudaMalloc(&sink, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf);
    return WS_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ws_status rc = WS_OK;
  float best = 0.f;
  const uint64_t n16 = bytes / 16;
  // grid: 8 blocks of 256 threads per SM (a multiple of the SM count); each
  // group of eight lanes of the line pattern reads `steps` lines per pass
  const int grid = 8 * sms;
  // random patterns: 1 = 128-byte reads, 2 = 64-byte, 3 = 32-byte, 4 = 32-byte writes, 5 = 128-byte writes
  const int lpg = (pattern == 1 || pattern == 5 || pattern >= 8) ? 8 : (pattern == 2 || pattern >= 6) ? 4 : 2;
  // patterns 6, 7: buckets of 640 bytes (a tag line and 32 slots, plus
  // spare), counted as the 80 bytes a probe pair reads
  const uint64_t block_bytes = (pattern == 6 || pattern == 7) ? 640 : 16ull * (uint64_t)lpg;
  const uint64_t n_blocks = bytes / block_bytes;
  const uint64_t groups = (uint64_t)grid * 256 / (uint64_t)lpg;
  const int steps = (int)(((n_blocks + groups - 1) / groups + 7) / 8 * 8);  // a multiple of every depth
  auto launch = [&](int np) {
    uint4* q = static_cast<uint4*>(buf);
    switch (pattern) {
      case 0: read_seq<<<grid, 256>>>(q, n16, np, sink); break;
      case 1: launch_random<8, false>(depth, grid, q, n_blocks, steps, np, sink); break;
      case 2: launch_random<4, false>(depth, grid, q, n_blocks, steps, np, sink); break;
      case 3: launch_random<2, false>(depth, grid, q, n_blocks, steps, np, sink); break;
      case 4: launch_random<2, true>(depth, grid, q, n_blocks, steps, np, sink); break;
      case 5: launch_random<8, true>(depth, grid, q, n_blocks, steps, np, sink); break;
      case 6:
        if (depth <= 2) tag_then_slot<true, 2><<<grid, 256>>>(q, n_blocks, steps, np, sink);
        else tag_then_slot<true, 4><<<grid, 256>>>(q, n_blocks, steps, np, sink);
        break;
      case 7:
        if (depth <= 2) tag_then_slot<false, 2><<<grid, 256>>>(q, n_blocks, steps, np, sink);
        else tag_then_slot<false, 4><<<grid, 256>>>(q, n_blocks, steps, np, sink);
        break;
      default: {  // 8..11: regions of 2^(10 + 2 (pattern - 8)) lines: 128 KiB, 512 KiB, 2 MiB, 8 MiB
        const uint64_t rl = 1ull << (10 + 2 * (pattern - 8));
        if (rl > n_blocks) return cudaErrorInvalidValue;
        regional_lines<<<grid, 256>>>(q, n_blocks, rl, steps, 8 * depth, np, sink);
        break;
      }
    }
    return cudaGetLastError();
  };
  do {
    if (cudaMemset(buf, 0x5a, bytes) != cudaSuccess || cudaMemset(sink, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = WS_ERR_CUDA;
      break;
    }
    if (launch(1) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {  // warm: the buffer into L2
      rc = WS_ERR_CUDA;
      break;
    }
    for (int rep = 0; rep < 5 && rc == WS_OK; ++rep) {
      float ms = 0.f;
      if (cudaEventRecord(e0) != cudaSuccess || launch(passes) != cudaSuccess || cudaEventRecord(e1) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = WS_ERR_CUDA;
        break;
      }
      const double per = (pattern == 6 || pattern == 7) ? 80.0 : (double)block_bytes;  // a pair reads 64 + 16 bytes
      const double read = pattern == 0 ? (double)n16 * 16.0 : (double)groups * (double)steps * per;
      const float gbs = (float)(read * passes / (ms * 1e-3) / 1e9);
      if (gbs > best) best = gbs;
    }
  } while (false);
  if (rc == WS_ERR_CUDA) note_cuda(cudaGetLastError(), "ws_read_bandwidth");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(buf);
  *gbs_out = best;
  return rc;
}
