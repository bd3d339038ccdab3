// ws_peak.cu -- read-bandwidth probes: the denominators of the roofline for
// tables that fit in L2 (measured here, on the running GPU) beside the HBM
// copy bandwidth measured for tables that do not.
//
// Two access patterns over a device buffer that the kernel reads `passes`
// times, through L2 only (ld.global.cg: no L1 reuse between passes):
//   0 sequential -- each thread reads 16-byte words at a grid stride, the
//     best case for any memory level;
//   1 random lines -- eight lanes read one 128-byte line together (16 bytes
//     each, as a bucket snapshot is copied), the line index drawn from a
//     counter-based hash per (pass, group, step), four independent lines in
//     flight per group: the access pattern of the hash-table probes.
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

__global__ void __launch_bounds__(256) read_seq(const uint4* __restrict__ p, uint64_t n16, int passes,
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

__global__ void __launch_bounds__(256) read_lines(const uint4* __restrict__ p, uint64_t n_lines, int steps,
                                                  int passes, unsigned int* sink) {
  uint32_t acc = 0;
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) >> 3;
  const uint64_t group = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int part = threadIdx.x & 7;
  for (int r = 0; r < passes; ++r) {
    const uint64_t ctr = ((uint64_t)r * groups + group) * (uint64_t)steps;
    for (int s = 0; s < steps; s += 4) {
      // four independent lines per step, the same for the group's eight lanes
      uint64_t l[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) l[k] = ((mix(ctr + (uint64_t)(s + k)) >> 32) * n_lines) >> 32;
      const uint4 a = ld_cg16(p + l[0] * 8 + part), b = ld_cg16(p + l[1] * 8 + part),
                  c = ld_cg16(p + l[2] * 8 + part), d = ld_cg16(p + l[3] * 8 + part);
      acc ^= a.x ^ b.y ^ c.z ^ d.w;
    }
  }
  if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);
}

}  // namespace

extern "C" ws_status ws_read_bandwidth(uint64_t bytes, int pattern, int passes, int device, double* gbs_out) {
  if (!gbs_out || bytes < (1u << 20) || (bytes & 127u) || passes < 1 || (pattern != 0 && pattern != 1))
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
  const uint64_t n16 = bytes / 16, n_lines = bytes / 128;
  // grid: 8 blocks of 256 threads per SM (a multiple of the SM count); each
  // group of eight lanes of the line pattern reads `steps` lines per pass
  const int grid = 8 * sms;
  const uint64_t groups = (uint64_t)grid * 256 / 8;
  const int steps = (int)(((n_lines + groups - 1) / groups + 3) / 4 * 4);
  auto launch = [&](int np) {
    if (pattern == 0)
      read_seq<<<grid, 256>>>(static_cast<const uint4*>(buf), n16, np, sink);
    else
      read_lines<<<grid, 256>>>(static_cast<const uint4*>(buf), n_lines, steps, np, sink);
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
      const double read = pattern == 0 ? (double)n16 * 16.0 : (double)groups * (double)steps * 128.0;
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
