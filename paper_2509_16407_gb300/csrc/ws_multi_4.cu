// ws_multi_4.cu -- persistent multi-table kernels of menu entry 4
// (SCHEME_P2, metadata false, 32-slot buckets, tile 8), one per op kind.
#include "ws_multi_kernel.cuh"

namespace ws {

cudaError_t launch_multi_4(int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  return launch_multi_cfg<SCHEME_P2, false, 32, 8>(kind, g, s, num_sms);
}

}  // namespace ws
