// Tensor-core split-precision GEMM (tcgen05 / TMEM / TMA) -- see below.
#include "common.cuh"

namespace fpeps {

bool gemm_tc_supported(int64_t, int64_t, int64_t, int64_t, int64_t) { return false; }
size_t gemm_tc_scratch_bytes(int, int64_t, int64_t, int64_t) { return 0; }
void gemm_tc(cudaStream_t, int, int64_t, int64_t, int64_t, const float*, int64_t, const float*, int64_t, float*, OutMap,
             void*, size_t) {
  throw Error{FPEPS_ERR_UNSUPPORTED, "tensor-core GEMM not available"};
}

}  // namespace fpeps
