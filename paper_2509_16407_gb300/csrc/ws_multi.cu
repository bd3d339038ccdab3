// ws_multi.cu -- dispatch of the persistent multi-table kernels by menu entry.
#include "ws_multi.cuh"

namespace ws {

cudaError_t launch_multi_0(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_1(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_2(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_3(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_4(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_5(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_6(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);
cudaError_t launch_multi_7(int kind, const MultiGroup& g, cudaStream_t s, int num_sms);

cudaError_t launch_multi(int cfg, int kind, const MultiGroup& g, cudaStream_t s, int num_sms) {
  switch (cfg) {
    case 0: return launch_multi_0(kind, g, s, num_sms);
    case 1: return launch_multi_1(kind, g, s, num_sms);
    case 2: return launch_multi_2(kind, g, s, num_sms);
    case 3: return launch_multi_3(kind, g, s, num_sms);
    case 4: return launch_multi_4(kind, g, s, num_sms);
    case 5: return launch_multi_5(kind, g, s, num_sms);
    case 6: return launch_multi_6(kind, g, s, num_sms);
    case 7: return launch_multi_7(kind, g, s, num_sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
