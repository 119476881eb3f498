// K2 instantiations for bf16 probabilities (see k_spmv.cuh).
#include "k_spmv.cuh"

namespace mdpk {

cudaError_t launch_arnoldi_spmv_bf16(const Mat& A, const int32_t* pi, float* basis, int64_t ld,
                                    int j, float cdiag, double* partials, DevState* st,
                                    cudaStream_t s) {
  (void)partials;
  return arnoldi_spmv_tu<__nv_bfloat16>(A, pi, basis, ld, j, cdiag, st, s);
}

cudaError_t launch_richardson_bf16(const Mat& A, const int32_t* pi, const float* r,
                                   const float* d_in, float* d_out, double* partials,
                                   DevState* st, cudaStream_t s) {
  return richardson_tu<__nv_bfloat16>(A, pi, r, d_in, d_out, partials, st, s);
}

}  // namespace mdpk
