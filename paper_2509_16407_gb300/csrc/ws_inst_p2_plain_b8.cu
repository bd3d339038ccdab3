// ws_inst_p2_plain_b8.cu -- kernel instantiations: scheme SCHEME_P2, metadata false,
// 8-slot buckets.  (Split across translation units so the build compiles them in parallel.)
#include "ws_kernels.cuh"

namespace ws {

cudaError_t launch_p2_plain_b8(int B, int T, const TableView& tv, const BatchArgs& a, int kind, cudaStream_t s, int sms) {
  switch (B * 100 + T) {
    case 804: return launch_cfg<SCHEME_P2, false, 8, 4>(tv, a, kind, s, sms);
    case 808: return launch_cfg<SCHEME_P2, false, 8, 8>(tv, a, kind, s, sms);
    case 816: return launch_cfg<SCHEME_P2, false, 8, 16>(tv, a, kind, s, sms);
    case 832: return launch_cfg<SCHEME_P2, false, 8, 32>(tv, a, kind, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
