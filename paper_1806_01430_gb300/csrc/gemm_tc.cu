// Tensor-core GEMM (placeholder until the tcgen05 path lands).
#include "gao_internal.h"

namespace gao {
size_t tc_scratch_bytes(int, int64_t, int64_t, int64_t) { return 0; }
cudaError_t launch_gemm_tc(int, float*, const float*, const float*, const float*, int64_t, int64_t, int64_t, float,
                           float, int, int, void*, size_t, int*, cudaStream_t, TcEvents&, std::string* why) {
    if (why) *why = "tensor-core path not built";
    return cudaErrorNotSupported;
}
}  // namespace gao
