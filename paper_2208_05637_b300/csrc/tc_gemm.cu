// BF16 tensor-core GEMM (placeholder until the tcgen05 kernel lands).
#include "nqs_internal.h"

namespace nqs {
int tc_gemm_bf16(const void*, const uint16_t*, const float*, void*, int64_t, int, int, int, cudaStream_t) {
    set_error("bf16 tensor-core GEMM not built yet");
    return NQS_ERR_UNSUPPORTED;
}
}  // namespace nqs
