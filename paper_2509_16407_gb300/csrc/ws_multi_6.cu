// ws_multi_6.cu -- persistent multi-table kernels of menu entry 6
// (SCHEME_P2, metadata true, 32-slot buckets, tile 4), one per op kind.
#include "ws_multi_kernel.cuh"

namespace ws {

cudaError_t launch_multi_6(int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  return launch_multi_cfg<SCHEME_P2, true, 32, 4>(kind, g, s, num_sms);
}

}  // namespace ws
