// K2 instantiations for f32 probabilities (see k_spmv.cuh) and the
// Gram-Schmidt dots (k_dots.cuh).
#include "k_dots.cuh"
#include "k_spmv.cuh"

namespace mdpk {

cudaError_t launch_arnoldi_spmv_f32(const Mat& A, const int32_t* pi, float* basis, int64_t ld,
                                    int j, float cdiag, double* partials, DevState* st,
                                    cudaStream_t s) {
  (void)partials;
  return arnoldi_spmv_tu<float>(A, pi, basis, ld, j, cdiag, st, s);
}

cudaError_t launch_richardson_f32(const Mat& A, const int32_t* pi, const float* r,
                                   const float* d_in, float* d_out, double* partials,
                                   DevState* st, cudaStream_t s) {
  return richardson_tu<float>(A, pi, r, d_in, d_out, partials, st, s);
}

cudaError_t launch_arnoldi_dots(const Mat& A, float* basis, int64_t ld, int j, int restart,
                                int out_h2, double* partials, DevState* st, cudaStream_t s) {
  return dots_entry(A, basis, ld, j, restart, out_h2, partials, st, s);
}

}  // namespace mdpk
