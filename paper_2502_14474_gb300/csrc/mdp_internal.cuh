// Internal declarations of the GB300 MDP solver library (device + host).
//
// Conventions: state s, action a, row r = s*m + a of the (n*m) x n CSR matrix
// P; IdxT is the row-pointer type (int32 when nnz < 2^31, else int64).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdpk {

constexpr int kThreads = 256;     // threads per CTA for every streaming kernel
constexpr int kDotsMaxRuns = 256;  // dots kernel: at most 8 * 256 chunk slots
constexpr int kMaxRestart = 64;   // GMRES restart cap (basis holds restart+1 vectors)
constexpr int kMaxBasis = kMaxRestart + 1;
constexpr int kSMax = 8;                     // s-step GMRES: Krylov vectors per block
constexpr int kBlkMaxV = kMaxBasis + kSMax;  // vectors of one block Gram pass ([Q W])

// ---------------------------------------------------------------------------
// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2.  Error-free transforms:
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum and FMA-based TwoProd (Dekker
// 1971).  The explicit _rn intrinsics keep the compiler from contracting the
// error terms into FMAs.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_norm(float hi, float lo) {
  ff r;
  fast_two_sum(hi, lo, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_norm(s, e);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  return ff_norm(s, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_norm(p, e);
}

// s += p * (vhi + vlo) [+ plo * vhi], accumulating into an unnormalised pair
// (s_hi carries the TwoSum chain, s_lo collects every error term).
__device__ __forceinline__ void ff_acc(float& s_hi, float& s_lo, float p, float vhi, float vlo) {
  float ph = __fmul_rn(p, vhi);
  float pl = __fmaf_rn(p, vhi, -ph);
  pl = __fmaf_rn(p, vlo, pl);
  float t, e;
  two_sum(s_hi, ph, t, e);
  s_hi = t;
  s_lo = __fadd_rn(s_lo, __fadd_rn(e, pl));
}

// (ahi + alo) - (bhi + blo) rounded once to FP32: TwoSum makes the difference
// of the high parts exact before the low parts are added.
__device__ __forceinline__ float ff_diff_to_float(float ahi, float alo, float bhi, float blo) {
  float s, e;
  two_sum(ahi, -bhi, s, e);
  return __fadd_rn(s, __fadd_rn(e, __fsub_rn(alo, blo)));
}

__device__ __forceinline__ bool ff_less(ff a, ff b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int W>
__device__ __forceinline__ void group_sum_ff(float& hi, float& lo) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, ohi, s, e);
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
  }
}

__device__ __forceinline__ float warp_sum(float v) { return group_sum<32>(v); }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum / max of one double per thread (fixed order; result valid in
// thread 0).  `scratch` must hold kThreads/32 doubles.
__device__ __forceinline__ double block_sum_d(double v, double* scratch) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) r += scratch[i];
  return r;
}

__device__ __forceinline__ double block_max_d(double v, double* scratch) {
  v = warp_max_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) r = fmax(r, scratch[i]);
  return r;
}

template <int NT>
__device__ __forceinline__ double block_sum_nt(double v, double* scratch) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) r += scratch[i];
  return r;
}

template <int NT>
__device__ __forceinline__ double block_max_nt(double v, double* scratch) {
  v = warp_max_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) r = fmax(r, scratch[i]);
  return r;
}

// "Last block" ticket (threadFenceReduction pattern): every block publishes
// its partials, fences, then takes a ticket; the block that draws the last
// ticket sees every partial and reduces them in a fixed order, so results are
// deterministic without floating-point atomics.  No thread waits on another.
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// ---------------------------------------------------------------------------
// Device-resident solver state: residual norms and the GMRES cycle.
// H is stored column-major with leading dimension kMaxBasis.
// ---------------------------------------------------------------------------
enum : unsigned {
  kCntBellman = 0,
  kCntPolicy = 1,
  kCntDots = 2,
  kCntOrtho = 3,
  kCntDots2 = 4,
  kCntOrtho2 = 5,
  kCntMisc = 6,
  kCntBicg = 7,
  kNumCounters = 8
};

struct DevState {
  unsigned counter[kNumCounters];
  // outputs of the Bellman / residual reductions
  double res_inf;     // ||r||_inf
  double res_2;       // ||r||_2
  // GMRES cycle
  int active;         // 1 while Arnoldi steps remain in this cycle
  int jdone;          // Arnoldi steps completed in this cycle
  int converged;      // residual estimate <= target
  int breakdown;      // exact invariant subspace reached
  int restart;        // cycle length
  int target_rel;     // 1: target = eta * res_inf (set by the Bellman reduction)
  double eta;
  double target;      // absolute 2-norm target of the cycle
  double beta;        // ||r0||_2 of the cycle
  double est;         // current residual estimate |g_{j+1}|
  int nspmv;          // policy-row SpMVs the cycle ran (s-step: may exceed jdone)
  int bfin_k;         // s-step: first step of the block that ends the cycle, -1 before
  int dev_error;      // non-zero: a bounded device wait gave up (the kernel's code)
  int dev_error_pad;
  double H[kMaxBasis * kMaxRestart];
  double cs[kMaxRestart], sn[kMaxRestart];
  double gv[kMaxBasis];
  double y[kMaxRestart];
  double scale[kMaxBasis];  // v_i = u_i * scale[i]
  double h2[kMaxBasis];     // second Gram-Schmidt pass coefficients
  // tickets of the Gram-Schmidt dots kernel: per vector group, and per run of
  // eight chunk slots within a group (two-level fixed-order reduction)
  unsigned dots_group[kMaxBasis / 8 + 1];
  unsigned dots_run[kMaxBasis / 8 + 1][kDotsMaxRuns];
  // BiCGStab scalars (rho = <r^, r>, alpha, omega, beta of the recurrences)
  double bicg_rho, bicg_alpha, bicg_omega, bicg_beta;
  // the last finished GMRES cycle, kept for inspection: the Hessenberg matrix
  // as built (before the Givens rotations; column-major, leading dimension
  // kMaxBasis), its beta = ||r0||_2, step count and final residual estimate
  // (y above holds its least-squares solution until the next cycle ends)
  double Hraw[kMaxBasis * kMaxRestart];
  double last_beta, last_est;
  int last_J;
  // s-step GMRES block (k = first step of the block, sb its vectors w_1..w_sb
  // in basis columns k+1..k+sb): Gram pass results and the coefficients the
  // update pass applies
  unsigned blk_groups;           // ticket over the Gram pass's vector groups
  int bsb;                       // block columns kept (<= sb; fewer after a breakdown)
  double G[kBlkMaxV * kSMax];    // G[v * kSMax + i] = <x_v, w_{i+1}>, x = [u_0..u_k, W]
  float bC[kMaxBasis * kSMax];   // coefficient of raw column v in w_{i+1}'s projection
  float bRinv[kSMax * kSMax];    // R^{-1} (upper triangular), R^T R = W^T W - C^T C
  float bY[kBlkMaxV];            // coefficient of column v in the solution update
};

// Initialise a GMRES cycle from ||r0||_2 = beta (single thread).
__device__ __forceinline__ void gmres_begin(DevState* st, double beta) {
  st->beta = beta;
  st->jdone = 0;
  st->nspmv = 0;
  st->bfin_k = -1;
  st->breakdown = 0;
  st->est = beta;
  for (int i = 0; i < kMaxBasis; ++i) st->gv[i] = 0.0;
  st->gv[0] = beta;
  // v_0 = u_0 / beta; later columns start unscaled (the s-step SpMVs read
  // their block's vectors w_i with scale 1; Arnoldi sets its own scales)
  for (int i = 1; i < kMaxBasis; ++i) st->scale[i] = 1.0;
  st->scale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
  const bool done = !(beta > st->target);
  st->converged = done ? 1 : 0;
  st->active = done ? 0 : 1;
}

// ---------------------------------------------------------------------------
// Kernel argument blocks
// ---------------------------------------------------------------------------
template <typename IdxT>
struct Csr {
  const IdxT* rp;         // [rows + 1]
  const int32_t* col;     // [nnz]
  const float* val;       // [nnz] FP32 probabilities (defining values, rounded)
  const float* val_lo;    // [nnz] FP64 remainder val - (float)val, or nullptr
  const float* g;         // [rows]
  const float* g_lo;      // [rows] or nullptr
  const void* val16;      // [nnz] bf16/f16 copy or nullptr
  const uint4* lpk;       // packed 16-bit inner copy (16-byte groups) or nullptr
  const float* row_scale; // [rows] renormalisation of the 16-bit copy
  int64_t n;
  int32_t m;
  int32_t vec4;           // 1: 16-byte vector loads of col/val (rows long enough)
  int32_t uniform_len;    // > 0: every row has this many entries (rp unused)
  int32_t am;             // 1: policy rows action-major, row (s, a) at a*n + s
  float gamma;            // FP32 gamma
  float gamma_hi, gamma_lo;  // float-float gamma
};

// Row of P holding the transitions of state s under action a: s*m + a in the
// CSR as given, a*n + s in the action-major policy copy.
template <typename IdxT>
__device__ __forceinline__ int64_t policy_row(const Csr<IdxT>& P, int64_t s, int32_t a) {
  return P.am ? static_cast<int64_t>(a) * P.n + s : s * P.m + a;
}

struct Grid {
  int64_t n_tiles;
  int64_t tiles_per_block;
  int tile_states;
};

}  // namespace mdpk
