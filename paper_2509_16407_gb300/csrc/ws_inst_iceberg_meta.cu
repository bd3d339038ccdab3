// ws_inst_iceberg_meta.cu -- kernel instantiations: scheme SCHEME_ICEBERG, metadata true.
// (Split across translation units so the build compiles them in parallel.)
#include "ws_kernels.cuh"

namespace ws {

cudaError_t launch_iceberg_meta(int B, int T, const TableView& tv, const BatchArgs& a, int kind,
                                cudaStream_t s, int sms) {
  switch (B * 100 + T) {
    case 3204: return launch_cfg<SCHEME_ICEBERG, true, 32, 4>(tv, a, kind, s, sms);
    case 3208: return launch_cfg<SCHEME_ICEBERG, true, 32, 8>(tv, a, kind, s, sms);
    case 3216: return launch_cfg<SCHEME_ICEBERG, true, 32, 16>(tv, a, kind, s, sms);
    case 3232: return launch_cfg<SCHEME_ICEBERG, true, 32, 32>(tv, a, kind, s, sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ws
