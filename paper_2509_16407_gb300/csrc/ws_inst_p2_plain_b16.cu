// ws_inst_p2_plain_b16.cu -- kernel instantiations: scheme SCHEME_P2, metadata false,
// 16-slot buckets.  (Split across translation units so the build compiles them in parallel.)
#include "ws_kernels.cuh"

namespace ws {

cudaError_t launch_p2_plain_b16(int B, int T, const TableView& tv, const BatchArgs& a, int kind, cudaStream_t s, int sms) {
  switch (B * 100 + T) {
    case 1604: return launch_cfg<SCHEME_P2, false, 16, 4>(tv, a, kind, s, sms);
    case 1608: return launch_cfg<SCHEME_P2, false, 16, 8>(tv, a, kind, s, sms);
    case 1616: return launch_cfg<SCHEME_P2, false, 16, 16>(tv, a, kind, s, sms);
    case 1632: return launch_cfg<SCHEME_P2, false, 16, 32>(tv, a, kind, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
