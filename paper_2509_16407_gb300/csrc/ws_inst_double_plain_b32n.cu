// ws_inst_double_plain_b32n.cu -- kernel instantiations: scheme SCHEME_DOUBLE, metadata false,
// 32-slot buckets, tiles 4 and 8.  (Split across translation units so the build compiles them in parallel.)
#include "ws_kernels.cuh"

namespace ws {

cudaError_t launch_double_plain_b32n(int B, int T, const TableView& tv, const BatchArgs& a, int kind, cudaStream_t s, int sms) {
  switch (B * 100 + T) {
    case 3204: return launch_cfg<SCHEME_DOUBLE, false, 32, 4>(tv, a, kind, s, sms);
    case 3208: return launch_cfg<SCHEME_DOUBLE, false, 32, 8>(tv, a, kind, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
