// Host-side launchers of the solver kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mdp_internal.cuh"

namespace mdpk {

// Device view of one handle's matrix, as the launchers need it.
struct Mat {
  int64_t n = 0, rows = 0, nnz = 0;
  int32_t m = 0;
  int32_t idx64 = 0;        // row pointers are int64
  const void* rp = nullptr;
  const int32_t* col = nullptr;  // packed layout (see k_rows.cuh), viewed as int32
  const float* val = nullptr;    // the same packed array, viewed as FP32
  const float* val_lo = nullptr;
  const float* g = nullptr;
  const float* g_lo = nullptr;
  const void* val16 = nullptr;
  const uint4* lpk = nullptr;  // [4 x int16 col - s | 4 x 16-bit value] groups (band < 2^15);
                               // in the action-major row order when am_len > 0
  // Action-major policy copy for short rows: row (s, a) at a*n + s, every row
  // padded to am_len entries with zero probabilities (column s) at its end, in
  // the packed 32-byte group format.  Read by the policy-row kernels (SpMV,
  // policy residual, Richardson): states that share an action read adjacent
  // rows.  am_len == 0: no copy.
  const uint32_t* pk_am = nullptr;
  int32_t am_len = 0;
  const float* row_scale = nullptr;
  int32_t store_t = 0;      // MDP_F32 / MDP_BF16 / MDP_F16 of val16
  int32_t uniform_len = 0;
  int32_t vec4 = 0;
  int32_t vw = 4;           // lanes per row
  int64_t band = 0;         // max |col - s| (measured at create)
  int32_t window = 0;       // 1: banded kernels stage V in a shared-memory ring
  int32_t screen = 0;       // 1: float-float backups screen actions in FP32 first
  double gamma = 0.0;
  int num_sms = 1;
};

// True when float-float backups of A take the FP32-screened windowed kernel.
bool bellman_screened(const Mat& A);
// K1 / K6: Bellman backup + greedy + residual.  ff selects float-float (V is
// float2 hi/lo) versus FP32 (V is float).  init_gmres: the last block also
// starts a GMRES cycle from r (target = eta*||r||_inf when st->target_rel).
cudaError_t launch_bellman(const Mat& A, bool ff, const void* V, void* V_out, int32_t* pi,
                           float* r, double* partials, DevState* st, int init_gmres,
                           cudaStream_t s);

// Policy residual in float-float: r = g_pi + gamma P_pi V - V, ||r||, and a
// GMRES cycle start (target kept as set on the device state).
cudaError_t launch_policy_residual(const Mat& A, const int32_t* pi, const float2* V, float* r,
                                   double* partials, DevState* st, cudaStream_t s);

// Arnoldi step j, SpMV half (K2): u_{j+1} = cdiag v_j - gamma P_pi v_j
// (cdiag = 1: w = A v_j; cdiag = 0: the s-step monomial basis (A - I) v_j).
// lp: use the 16-bit probabilities with row renormalisation.
cudaError_t launch_arnoldi_spmv(const Mat& A, bool lp, const int32_t* pi, float* basis,
                                int64_t ld, int j, float cdiag, double* partials, DevState* st,
                                cudaStream_t s);

// Richardson sweeps through the policy-row kernel (one per probability type).
cudaError_t launch_richardson_f32(const Mat& A, const int32_t* pi, const float* r,
                                  const float* d_in, float* d_out, double* partials,
                                  DevState* st, cudaStream_t s);
cudaError_t launch_richardson_bf16(const Mat& A, const int32_t* pi, const float* r,
                                   const float* d_in, float* d_out, double* partials,
                                   DevState* st, cudaStream_t s);
cudaError_t launch_richardson_f16(const Mat& A, const int32_t* pi, const float* r,
                                  const float* d_in, float* d_out, double* partials,
                                  DevState* st, cudaStream_t s);
cudaError_t launch_arnoldi_spmv_f32(const Mat& A, const int32_t* pi, float* basis, int64_t ld,
                                    int j, float cdiag, double* partials, DevState* st,
                                    cudaStream_t s);
cudaError_t launch_arnoldi_spmv_bf16(const Mat& A, const int32_t* pi, float* basis, int64_t ld,
                                    int j, float cdiag, double* partials, DevState* st,
                                     cudaStream_t s);
cudaError_t launch_arnoldi_spmv_f16(const Mat& A, const int32_t* pi, float* basis, int64_t ld,
                                    int j, float cdiag, double* partials, DevState* st,
                                    cudaStream_t s);
// Gram-Schmidt dots of u_{j+1} against v_0..v_j: into H(:, j) (out_h2 == 0)
// or st->h2 (second pass of CGS2).
cudaError_t launch_arnoldi_dots(const Mat& A, float* basis, int64_t ld, int j, int restart,
                                int out_h2, double* partials, DevState* st, cudaStream_t s);

// K3 (+K4 in its last block): w -= sum h_i v_i, ||w||, Givens, convergence.
cudaError_t launch_arnoldi_ortho(const Mat& A, float* basis, int64_t ld, int j, int restart,
                                 int cgs2, double* partials, DevState* st, cudaStream_t s);

// s-step GMRES (k_sstep.cu): the Gram pass of the block starting at step k
// (sb vectors in columns k+1..k+sb; its last block runs the block's FP64
// least-squares steps), and the update pass that orthonormalises the block in
// place and, on the block that ends the cycle, adds the solution update to V.
// s_blk is the cycle's block size (selects the kernel instantiation).
cudaError_t launch_block_dots(const Mat& A, const float* basis, int64_t ld, int k, int sb,
                              int s_blk, int restart, double* partials, DevState* st,
                              cudaStream_t s);
cudaError_t launch_block_update(const Mat& A, float* basis, int64_t ld, int k, int sb, int s_blk,
                                float2* V, DevState* st, cudaStream_t s);
// Doubles of the Gram pass's partials buffer for n states.
size_t block_partials_len(int num_sms, int64_t n);

// ---- many MDPs per launch (k_batch.cu) --------------------------------------
// One MDP of a fused batch, as the batched kernels see it (device copy).
struct BMdp {
  const void* rp;          // row pointers (int32 or int64 by idx64; unused when uniform_len)
  const int32_t* col;      // packed col/val groups (k_rows.cuh)
  const float* val;
  const float* val_lo;     // FP64 remainders or nullptr
  const float* g;
  const float* g_lo;
  float2* V;               // float-float iterate
  int32_t* pi;
  float* basis;
  DevState* st;
  double* part;            // per-unit residual partials (2 per unit)
  double* bpart;           // per-unit Gram partials (float-float pairs, kBlkMaxV * kSMax per unit)
  int64_t n, ld;
  int64_t u_bell, u_state, u_gram;  // units of the Bellman, state-range and Gram kernels
  int32_t m, idx64, uniform_len, vw, tb;
  int32_t maxlen;          // longest row (entries)
  int32_t grp;             // 1: short rows, a packed group (4 entries) per lane
  float gamma, gamma_hi, gamma_lo;
};
// The MDPs taking part in one batched launch: participant p is MDP mdp[p]
// and owns the global units [first[p], first[p + 1]); total = first[count].
struct BList {
  const int32_t* mdp;
  const int64_t* first;
  int32_t count;
  int64_t total;
};
cudaError_t launch_batch_bellman(const BMdp* mdps, const BList* list, int num_sms, cudaStream_t s);
cudaError_t launch_batch_policy_resid(const BMdp* mdps, const BList* list, int num_sms,
                                      cudaStream_t s);
cudaError_t launch_batch_spmv(const BMdp* mdps, const BList* list, int j, int num_sms,
                              cudaStream_t s);
cudaError_t launch_batch_gram(const BMdp* mdps, const BList* list, int k, int sb, int num_sms,
                              cudaStream_t s);
cudaError_t launch_batch_update(const BMdp* mdps, const BList* list, int k, int sb, int num_sms,
                                cudaStream_t s);
cudaError_t launch_batch_heads(const BMdp* mdps, int count, size_t head_bytes, unsigned char* out,
                               cudaStream_t s);
int batch_bellman_tile(int m);
int64_t batch_units_bellman(int64_t n, int m);
int64_t batch_units_state(int64_t n);
int64_t batch_units_gram(int64_t n);

// K5: V += sum_i y_i v_i over the completed steps (float-float V).
cudaError_t launch_gmres_update(const Mat& A, float* basis, int64_t ld, float2* V,
                                DevState* st, cudaStream_t s);

// Richardson sweep of the correction system (modified policy iteration):
// d_out = r + gamma P_pi d_in, ||d_out - d_in||_2 into st->res_2.
// Arm the device-side stop of a run of Richardson sweeps (target on res_2).
cudaError_t launch_richardson_begin(DevState* st, double target, cudaStream_t s);

cudaError_t launch_richardson(const Mat& A, bool lp, const int32_t* pi, const float* r,
                              const float* d_in, float* d_out, double* partials, DevState* st,
                              cudaStream_t s);

// V += d (float-float V, FP32 d).
cudaError_t launch_ff_axpy(int64_t n, float2* V, const float* d, int num_sms, cudaStream_t s);

// Conversions between caller vectors and the float-float iterate; neg = 1
// negates on the way (a maximising handle keeps -V internally).
cudaError_t launch_to_ff(int64_t n, const void* src, int src_f64, int neg, float2* dst,
                         int num_sms, cudaStream_t s);
cudaError_t launch_from_ff(int64_t n, const float2* src, void* dst, int dst_f64, int neg,
                           int num_sms, cudaStream_t s);
// BiCGStab on (I - gamma P_pi) x = r0 (FP32 vectors of n entries, scalars and
// status in DevState).  One iteration: bicg_spmv(mode 0: v = A p), bicg_s,
// bicg_spmv(mode 1: t = A s, s kept in r), bicg_r, bicg_p.
cudaError_t launch_bicg_spmv(const Mat& A, const int32_t* pi, const float* x, float* y,
                             const float* w, int mode, double* partials, DevState* st,
                             cudaStream_t s);
cudaError_t launch_bicg_begin(int64_t n, const float* r0, float* r, float* p, float* x,
                              double target, double* partials, DevState* st, int num_sms,
                              cudaStream_t s);
cudaError_t launch_bicg_s(int64_t n, const float* p, const float* v, float* r, float* x,
                          double* partials, DevState* st, int num_sms, cudaStream_t s);
cudaError_t launch_bicg_r(int64_t n, const float* rhat, const float* t, float* r, float* x,
                          double* partials, DevState* st, int num_sms, cudaStream_t s);
cudaError_t launch_bicg_p(int64_t n, const float* r, const float* v, float* p,
                          const DevState* st, int num_sms, cudaStream_t s);
// dst = -src (FP32 or FP64 vector of n entries); dst may equal src.
cudaError_t launch_negate(int64_t n, const void* src, void* dst, int f64, int num_sms,
                          cudaStream_t s);

// Matrix preparation (mdp_create).
struct PrepFlags {
  unsigned bad_csr;        // row pointer or column index invalid
  unsigned nonfinite;      // NaN / Inf in val or cost
  unsigned negative;       // a negative probability
  unsigned not_stochastic; // |row sum - 1| > tol or empty row
  unsigned not_aligned;    // some row start is not a multiple of 4
  int32_t min_len, max_len;
  unsigned long long band; // max |col - s|
  double max_sum_err;
};

// Point a policy-row kernel's view at the action-major copy, when there is one.
template <typename CsrT>
inline void use_policy_copy(CsrT& P, const Mat& A) {
  P.am = 0;
  if (A.am_len > 0) {
    P.col = reinterpret_cast<const int32_t*>(A.pk_am);
    P.val = reinterpret_cast<const float*>(A.pk_am);
    P.val_lo = nullptr;
    P.uniform_len = A.am_len;
    P.vec4 = 0;
    P.am = 1;
  }
}

// Build the action-major policy copy (rows padded to L entries) from the
// packed CSR of A.
cudaError_t launch_build_am(const Mat& A, uint32_t* pk_am, int32_t L, cudaStream_t s);

cudaError_t launch_prep_rows(int64_t n, int32_t m, int64_t nnz, const int64_t* rp_in,
                             const int32_t* col_in, const void* val_in, int val_f64,
                             const uint32_t* pk, const float* pk_lo, const void* g_in, int g_f64,
                             int g_neg, double tol, void* rp_out, int idx64, float* g_out,
                             float* g_lo_out, PrepFlags* flags, int num_sms, cudaStream_t s);
// Interleave col/val into the packed layout (groups of 4 entries, 32 bytes).
cudaError_t launch_pack(int64_t nnz, const int32_t* col_in, const void* val_in, int val_f64,
                        uint32_t* pk, float* val_lo_out, int num_sms, cudaStream_t s);
cudaError_t launch_prep_lowp(const Mat& A, void* val16, float* row_scale, int store_t,
                             cudaStream_t s);
// Packed 16-bit inner copy: per 4-entry group, 4 int16 column offsets from the
// entry's row state and the 4 rounded values, 16 bytes; plus row_scale.
cudaError_t launch_prep_lowp_packed(const Mat& A, uint4* lpk, float* row_scale, int store_t,
                                    cudaStream_t s);

}  // namespace mdpk
