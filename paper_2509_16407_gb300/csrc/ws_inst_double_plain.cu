// ws_inst_double_plain.cu -- dispatcher of the SCHEME_DOUBLE plain instantiations, which
// live in ws_inst_double_plain_*.cu by bucket size (compiled in parallel).
#include "ws_kernels.cuh"

namespace ws {

cudaError_t launch_double_plain_b8(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_double_plain_b16(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_double_plain_b32n(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);
cudaError_t launch_double_plain_b32w(int B, int T, const TableView&, const BatchArgs&, int kind, cudaStream_t, int);

cudaError_t launch_double_plain(int B, int T, const TableView& tv, const BatchArgs& a, int kind, cudaStream_t s,
                              int sms) {
  if (B == 8) return launch_double_plain_b8(B, T, tv, a, kind, s, sms);
  if (B == 16) return launch_double_plain_b16(B, T, tv, a, kind, s, sms);
  if (B == 32) return (T <= 8) ? launch_double_plain_b32n(B, T, tv, a, kind, s, sms)
                               : launch_double_plain_b32w(B, T, tv, a, kind, s, sms);
  return cudaErrorInvalidValue;
}

}  // namespace ws
