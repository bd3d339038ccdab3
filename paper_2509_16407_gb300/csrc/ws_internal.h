// ws_internal.h -- host-side table object shared by the C-ABI units.
#pragma once
#include <cstdint>
#include <cstdio>

#include "../../include/warpspeed.h"
#include "ws_kernels.cuh"

namespace wsi {

using ws::u64;
using ws::u8;
using ws::u32;

// Staging for host batch buffers: kBufs rotating chunk buffers, H2D copies on
// one stream, kernels on the caller's stream, D2H copies on a third, chained
// by events, so the copies of later chunks run while earlier chunks' kernels
// do.  The two copy streams belong to the device and are shared by every
// table on it, so copies run in the order the calls were issued (with a
// stream per table, the copies of the tables' next calls all started at
// once and starved the current call).
struct Staging {
  static constexpr int kBufs = 8;
  u64 cap = 0;  // ops per chunk
  u64* keys[kBufs] = {};
  u64* vals[kBufs] = {};
  u64* out[kBufs] = {};
  u8* ops[kBufs] = {};
  u8* st[kBufs] = {};
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t in_ready[kBufs] = {}, k_done[kBufs] = {}, out_done[kBufs] = {};
};

void note_cuda(cudaError_t e, const char* where);
// Replace the thread's error text (read back by ws_cuda_error_string).
void note_text(const char* msg);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev) {
      prev = cur;
      cudaSetDevice(dev);
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define WS_CUDA(call)                        \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) {                 \
      ::wsi::note_cuda(e_, #call);           \
      return WS_ERR_CUDA;                    \
    }                                        \
  } while (0)

}  // namespace wsi

struct ws_table {
  ws::TableView tv;
  wsi::u64 nb = 0, B = 0, S = 0;
  int T = 0, scheme = 0, meta = 0, device = 0, num_sms = 0;
  uint32_t pmax = 0, spin = 0;
  int never_erased = 1;
  int host_direct = 1;  // WS_OPT_HOST_DIRECT
  int stage_log2 = 22;  // WS_OPT_STAGE_CHUNK: ops per staging chunk, log2
  wsi::u64 bytes = 0;
  cudaStream_t last_stream = nullptr;
  wsi::Staging* stage = nullptr;
  bool stream_alloc = false;  // memory from the stream-ordered allocator
};

namespace wsi {
// Launch one single-table batch kernel for the table's configuration.
cudaError_t dispatch(const ws_table* t, const ws::TableView& tv, const ws::BatchArgs& a, int kind, cudaStream_t s);
// 1 device pointer on `device`, 2 host, 3 another device, 0 null.
int classify(const void* p, int device);
enum { PTR_NULL = 0, PTR_DEVICE = 1, PTR_HOST = 2, PTR_OTHER_DEVICE = 3 };
// The device's view of page-locked, mapped host memory, or null (pageable
// memory, or a pointer that is not host memory).
void* mapped_host(const void* p);
// Table constructor; with a non-null stream it allocates and clears on that
// stream without synchronising the device.
ws_status table_create(const ws_config* cfg, cudaStream_t stream, ws_table** out);
// Free a table on a stream (for tables made with a stream).
void table_free_async(ws_table* t, cudaStream_t stream);
}  // namespace wsi
