// ws_multi_1.cu -- persistent multi-table kernels of menu entry 1
// (SCHEME_DOUBLE, metadata false, 8-slot buckets, tile 8), one per op kind.
#include "ws_multi_kernel.cuh"

namespace ws {

cudaError_t launch_multi_1(int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  return launch_multi_cfg<SCHEME_DOUBLE, false, 8, 8>(kind, g, s, num_sms);
}

}  // namespace ws
