// ws_multi_2.cu -- persistent multi-table kernels of menu entry 2
// (SCHEME_DOUBLE, metadata true, 32-slot buckets, tile 4), one per op kind.
#include "ws_multi_kernel.cuh"

namespace ws {

cudaError_t launch_multi_2(int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  return launch_multi_cfg<SCHEME_DOUBLE, true, 32, 4>(kind, g, s, num_sms);
}

}  // namespace ws
