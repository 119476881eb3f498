// K2 instantiations for bf16 probabilities (see k_spmv.cuh).
#include "k_spmv.cuh"

namespace mdpk {

cudaError_t launch_arnoldi_spmv_bf16(const Mat& A, const int32_t* pi, float* basis, int64_t ld,
                                    int j, int restart, double* partials, DevState* st,
                                    cudaStream_t s) {
  (void)restart;
  return spmv_entry<__nv_bfloat16>(A, pi, basis, ld, j, partials, st, s);
}

}  // namespace mdpk
