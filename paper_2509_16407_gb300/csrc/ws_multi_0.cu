// ws_multi_0.cu -- persistent multi-table kernels of menu entry 0
// (SCHEME_DOUBLE, metadata false, 8-slot buckets, tile 4), one per op kind.
#include "ws_multi_kernel.cuh"

namespace ws {

cudaError_t launch_multi_0(int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  return launch_multi_cfg<SCHEME_DOUBLE, false, 8, 4>(kind, g, s, num_sms);
}

}  // namespace ws
