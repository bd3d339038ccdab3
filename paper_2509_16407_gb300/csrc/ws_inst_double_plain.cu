// ws_inst_double_plain.cu -- kernel instantiations: scheme SCHEME_DOUBLE, metadata false.
// (Split across translation units so the build compiles them in parallel.)
#include "ws_kernels.cuh"

namespace ws {

cudaError_t launch_double_plain(int B, int T, const TableView& tv, const BatchArgs& a, int kind,
                           cudaStream_t s, int sms) {
  switch (B * 100 + T) {
    case 804: return launch_cfg<SCHEME_DOUBLE, false, 8, 4>(tv, a, kind, s, sms);
    case 808: return launch_cfg<SCHEME_DOUBLE, false, 8, 8>(tv, a, kind, s, sms);
    case 816: return launch_cfg<SCHEME_DOUBLE, false, 8, 16>(tv, a, kind, s, sms);
    case 832: return launch_cfg<SCHEME_DOUBLE, false, 8, 32>(tv, a, kind, s, sms);
    case 1604: return launch_cfg<SCHEME_DOUBLE, false, 16, 4>(tv, a, kind, s, sms);
    case 1608: return launch_cfg<SCHEME_DOUBLE, false, 16, 8>(tv, a, kind, s, sms);
    case 1616: return launch_cfg<SCHEME_DOUBLE, false, 16, 16>(tv, a, kind, s, sms);
    case 1632: return launch_cfg<SCHEME_DOUBLE, false, 16, 32>(tv, a, kind, s, sms);
    case 3204: return launch_cfg<SCHEME_DOUBLE, false, 32, 4>(tv, a, kind, s, sms);
    case 3208: return launch_cfg<SCHEME_DOUBLE, false, 32, 8>(tv, a, kind, s, sms);
    case 3216: return launch_cfg<SCHEME_DOUBLE, false, 32, 16>(tv, a, kind, s, sms);
    case 3232: return launch_cfg<SCHEME_DOUBLE, false, 32, 32>(tv, a, kind, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
