// Matrix preparation for mdp_create: validation, conversion, analysis and the
// 16-bit probability copy.
//
// Validation follows the problem definition (madupite, "Problem Setting and
// Solution Methods": P(.|s,a) is a probability distribution over the finite
// state space): every row non-empty, entries finite and non-negative, row sums
// within a tolerance of 1, column indices inside [0, n), costs finite.
#include <math.h>

#include "launch.h"

namespace mdpk {

__device__ __forceinline__ void atomic_max_double_pos(double* addr, double v) {
  // v >= 0: the IEEE bit pattern of non-negative doubles is ordered as integers
  atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

// One thread per row.  The entries come either from the caller's col/val or,
// when pk is given, from the packed copy that k_pack already wrote (FP32 value
// + FP32 remainder for FP64 inputs), so that inputs in host memory are read
// over the host link only once.
__global__ void k_prep_rows(int64_t n, int32_t m, int64_t nnz, const int64_t* __restrict__ rp_in,
                            const int32_t* __restrict__ col, const void* __restrict__ val,
                            int val_f64, const uint32_t* __restrict__ pk,
                            const float* __restrict__ pk_lo, const void* __restrict__ g_in,
                            int g_f64, int g_neg, double tol, void* __restrict__ rp_out, int idx64,
                            float* __restrict__ g_out, float* __restrict__ g_lo_out,
                            PrepFlags* __restrict__ flags) {
  const int64_t rows = n * m;
  unsigned bad_csr = 0, nonfinite = 0, negative = 0, not_stoch = 0, not_aligned = 0;
  int32_t mn = 0x7fffffff, mx = 0;
  unsigned long long band = 0;
  double max_err = 0.0;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = rp_in[r], e = rp_in[r + 1];
    if (r == 0 && b != 0) bad_csr = 1;
    if (e < b || b < 0 || e > nnz) {
      bad_csr = 1;
      continue;
    }
    if (idx64) {
      static_cast<int64_t*>(rp_out)[r] = b;
      if (r == rows - 1) static_cast<int64_t*>(rp_out)[rows] = e;
    } else {
      static_cast<int32_t*>(rp_out)[r] = static_cast<int32_t>(b);
      if (r == rows - 1) static_cast<int32_t*>(rp_out)[rows] = static_cast<int32_t>(e);
    }
    const int64_t len = e - b;
    if (len == 0) not_stoch = 1;
    if (b & 3) not_aligned = 1;
    const int32_t l32 = len > 0x7fffffff ? 0x7fffffff : static_cast<int32_t>(len);
    mn = min(mn, l32);
    mx = max(mx, l32);
    const int64_t s = r / m;
    double sum = 0.0;
    for (int64_t i = b; i < e; ++i) {
      const int64_t slot = ((i >> 2) << 3) + (i & 3);
      const int32_t c = pk ? static_cast<int32_t>(pk[slot]) : col[i];
      if (c < 0 || c >= n) {
        bad_csr = 1;
      } else {
        const unsigned long long d =
            static_cast<unsigned long long>(c > s ? c - s : s - c);
        band = d > band ? d : band;
      }
      double p;
      if (pk)
        p = static_cast<double>(__uint_as_float(pk[slot + 4])) +
            (pk_lo ? static_cast<double>(pk_lo[i]) : 0.0);
      else
        p = val_f64 ? static_cast<const double*>(val)[i]
                    : static_cast<double>(static_cast<const float*>(val)[i]);
      if (!isfinite(p)) nonfinite = 1;
      else if (p < 0.0) negative = 1;
      sum += p;
    }
    const double err = fabs(sum - 1.0);
    if (!(err <= tol)) not_stoch = 1;
    if (isfinite(err)) max_err = fmax(max_err, err);
    const double g_raw = g_f64 ? static_cast<const double*>(g_in)[r]
                               : static_cast<double>(static_cast<const float*>(g_in)[r]);
    const double gv = g_neg ? -g_raw : g_raw;  // rewards of a maximisation: g = -r, exact
    if (!isfinite(gv)) nonfinite = 1;
    const float ghi = static_cast<float>(gv);
    g_out[r] = ghi;
    if (g_lo_out) g_lo_out[r] = static_cast<float>(gv - static_cast<double>(ghi));
  }
  if (bad_csr) atomicOr(&flags->bad_csr, 1u);
  if (nonfinite) atomicOr(&flags->nonfinite, 1u);
  if (negative) atomicOr(&flags->negative, 1u);
  if (not_stoch) atomicOr(&flags->not_stochastic, 1u);
  if (not_aligned) atomicOr(&flags->not_aligned, 1u);
  if (mx > 0) {
    atomicMin(&flags->min_len, mn);
    atomicMax(&flags->max_len, mx);
  }
  if (band) atomicMax(&flags->band, band);
  if (max_err > 0.0) atomic_max_double_pos(&flags->max_sum_err, max_err);
}

// Pack col/val into groups of four entries, 32 bytes each:
// pk[8g .. 8g+3] = col(4g .. 4g+3), pk[8g+4 .. 8g+7] = val(4g .. 4g+3) as FP32
// bits; the tail of the last group is zero.  FP64 inputs also store the FP32
// remainder val - (float)val in val_lo (plain entry order).
__global__ void k_pack(int64_t nnz, const int32_t* __restrict__ col, const void* __restrict__ val,
                       int f64, uint32_t* __restrict__ pk, float* __restrict__ val_lo) {
  const int64_t padded = (nnz + 3) & ~int64_t(3);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < padded;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t slot = ((i >> 2) << 3) + (i & 3);
    if (i >= nnz) {
      pk[slot] = 0u;
      pk[slot + 4] = 0u;
      continue;
    }
    pk[slot] = static_cast<uint32_t>(col[i]);
    if (f64) {
      const double p = static_cast<const double*>(val)[i];
      const float hi = static_cast<float>(p);
      pk[slot + 4] = __float_as_uint(hi);
      val_lo[i] = static_cast<float>(p - static_cast<double>(hi));
    } else {
      pk[slot + 4] = __float_as_uint(static_cast<const float*>(val)[i]);
    }
  }
}

template <typename Q>
struct Round16;
template <>
struct Round16<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 q(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ float f(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <>
struct Round16<__half> {
  static __device__ __forceinline__ __half q(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ float f(__half v) { return __half2float(v); }
};

// 16-bit copy q_e = round(P_e) and per-row factor c_r = 1 / sum_e q_e, so that
// the inner operator c_r * q is stochastic to FP32 rounding.
template <typename IdxT, typename Q>
__global__ void k_prep_lowp(int64_t rows, const IdxT* __restrict__ rp, int32_t uniform_len,
                            const float* __restrict__ pk, Q* __restrict__ q,
                            float* __restrict__ scale) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = uniform_len > 0 ? r * uniform_len : static_cast<int64_t>(rp[r]);
    const int64_t e = uniform_len > 0 ? b + uniform_len : static_cast<int64_t>(rp[r + 1]);
    double sum = 0.0;
    for (int64_t i = b; i < e; ++i) {
      const Q v = Round16<Q>::q(pk[((i >> 2) << 3) + 4 + (i & 3)]);
      q[i] = v;
      sum += static_cast<double>(Round16<Q>::f(v));
    }
    scale[r] = sum > 0.0 ? static_cast<float>(1.0 / sum) : 0.f;
  }
}

// One thread per row: entry i of row r (state s = r / m) goes to group i/4,
// slot i%4: int16 (col - s) in the first 8 bytes, the rounded value in the
// last 8; row_scale[r] = 1 / sum of the rounded row.
template <typename IdxT, typename Q>
__global__ void k_prep_lowp_packed(int64_t rows, int32_t m, int64_t n, int am,
                                   const IdxT* __restrict__ rp, int32_t uniform_len,
                                   const float* __restrict__ pk, uint16_t* __restrict__ lpk,
                                   float* __restrict__ scale) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = uniform_len > 0 ? r * uniform_len : static_cast<int64_t>(rp[r]);
    const int64_t e = uniform_len > 0 ? b + uniform_len : static_cast<int64_t>(rp[r + 1]);
    const int64_t st = am ? r % n : r / m;  // the state whose transitions row r holds
    double sum = 0.0;
    for (int64_t i = b; i < e; ++i) {
      const int64_t slot = ((i >> 2) << 3) + (i & 3);
      const int32_t c = __float_as_int(pk[((i >> 2) << 3) + (i & 3)]);
      const Q v = Round16<Q>::q(pk[((i >> 2) << 3) + 4 + (i & 3)]);
      lpk[slot] = static_cast<uint16_t>(static_cast<int16_t>(c - st));
      lpk[slot + 4] = *reinterpret_cast<const uint16_t*>(&v);
      sum += static_cast<double>(Round16<Q>::f(v));
    }
    scale[r] = sum > 0.0 ? static_cast<float>(1.0 / sum) : 0.f;
  }
}

static unsigned grid_of(int64_t work, int num_sms) {
  int64_t b = (work + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 16;
  if (b > cap) b = cap;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t launch_prep_rows(int64_t n, int32_t m, int64_t nnz, const int64_t* rp_in,
                             const int32_t* col_in, const void* val_in, int val_f64,
                             const uint32_t* pk, const float* pk_lo, const void* g_in, int g_f64,
                             int g_neg, double tol, void* rp_out, int idx64, float* g_out,
                             float* g_lo_out, PrepFlags* flags, int num_sms, cudaStream_t s) {
  k_prep_rows<<<grid_of(n * m, num_sms), 256, 0, s>>>(n, m, nnz, rp_in, col_in, val_in, val_f64,
                                                      pk, pk_lo, g_in, g_f64, g_neg, tol, rp_out,
                                                      idx64, g_out, g_lo_out, flags);
  return cudaGetLastError();
}

cudaError_t launch_pack(int64_t nnz, const int32_t* col_in, const void* val_in, int val_f64,
                        uint32_t* pk, float* val_lo_out, int num_sms, cudaStream_t s) {
  k_pack<<<grid_of(nnz + 3, num_sms), 256, 0, s>>>(nnz, col_in, val_in, val_f64, pk, val_lo_out);
  return cudaGetLastError();
}

cudaError_t launch_prep_lowp(const Mat& A, void* val16, float* row_scale, int store_t,
                             cudaStream_t s) {
  const unsigned nb = grid_of(A.rows, A.num_sms);
  if (store_t == 3) {
    if (A.idx64)
      k_prep_lowp<int64_t, __half><<<nb, 256, 0, s>>>(A.rows, static_cast<const int64_t*>(A.rp),
                                                      A.uniform_len, A.val,
                                                      static_cast<__half*>(val16), row_scale);
    else
      k_prep_lowp<int32_t, __half><<<nb, 256, 0, s>>>(A.rows, static_cast<const int32_t*>(A.rp),
                                                      A.uniform_len, A.val,
                                                      static_cast<__half*>(val16), row_scale);
  } else {
    if (A.idx64)
      k_prep_lowp<int64_t, __nv_bfloat16><<<nb, 256, 0, s>>>(
          A.rows, static_cast<const int64_t*>(A.rp), A.uniform_len, A.val,
          static_cast<__nv_bfloat16*>(val16), row_scale);
    else
      k_prep_lowp<int32_t, __nv_bfloat16><<<nb, 256, 0, s>>>(
          A.rows, static_cast<const int32_t*>(A.rp), A.uniform_len, A.val,
          static_cast<__nv_bfloat16*>(val16), row_scale);
  }
  return cudaGetLastError();
}

}  // namespace mdpk

namespace mdpk {

cudaError_t launch_prep_lowp_packed(const Mat& A, uint4* lpk, float* row_scale, int store_t,
                                    cudaStream_t s) {
  const unsigned nb = grid_of(A.rows, A.num_sms);
  // from the action-major policy copy when there is one (the 16-bit copy is read
  // only by the policy-row kernels), else from the packed CSR
  const int am = A.am_len > 0 ? 1 : 0;
  const float* pk = am ? reinterpret_cast<const float*>(A.pk_am) : A.val;
  const int32_t ul = am ? A.am_len : A.uniform_len;
  uint16_t* out = reinterpret_cast<uint16_t*>(lpk);
  if (store_t == 3) {
    if (A.idx64)
      k_prep_lowp_packed<int64_t, __half><<<nb, 256, 0, s>>>(
          A.rows, A.m, A.n, am, static_cast<const int64_t*>(A.rp), ul, pk, out, row_scale);
    else
      k_prep_lowp_packed<int32_t, __half><<<nb, 256, 0, s>>>(
          A.rows, A.m, A.n, am, static_cast<const int32_t*>(A.rp), ul, pk, out, row_scale);
  } else {
    if (A.idx64)
      k_prep_lowp_packed<int64_t, __nv_bfloat16><<<nb, 256, 0, s>>>(
          A.rows, A.m, A.n, am, static_cast<const int64_t*>(A.rp), ul, pk, out, row_scale);
    else
      k_prep_lowp_packed<int32_t, __nv_bfloat16><<<nb, 256, 0, s>>>(
          A.rows, A.m, A.n, am, static_cast<const int32_t*>(A.rp), ul, pk, out, row_scale);
  }
  return cudaGetLastError();
}

// Action-major policy copy: original row r = s*m + a goes to row a*n + s of
// length L; its entries keep their order, and the row is padded with
// zero-probability entries pointing at s (they add exact zeros to every sum).
// The packed format is the CSR's: entry i sits at word ((i >> 2) << 3) + (i & 3)
// (column) and the same + 4 (value).
template <typename IdxT>
__global__ void k_build_am(int64_t rows, int32_t m, int64_t n, const IdxT* __restrict__ rp,
                           int32_t uniform_len, const uint32_t* __restrict__ pk, int32_t L,
                           uint32_t* __restrict__ pk_am) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = uniform_len > 0 ? r * uniform_len : static_cast<int64_t>(rp[r]);
    const int64_t e = uniform_len > 0 ? b + uniform_len : static_cast<int64_t>(rp[r + 1]);
    const int64_t st = r / m;
    const int64_t a = r - st * m;
    const int64_t base = (a * n + st) * L;
    for (int64_t k = 0; k < L; ++k) {
      const int64_t o = base + k;
      const int64_t wo = ((o >> 2) << 3) + (o & 3);
      if (b + k < e) {
        const int64_t i = b + k;
        const int64_t wi = ((i >> 2) << 3) + (i & 3);
        pk_am[wo] = pk[wi];
        pk_am[wo + 4] = pk[wi + 4];
      } else {
        pk_am[wo] = static_cast<uint32_t>(st);
        pk_am[wo + 4] = 0u;  // +0.0f
      }
    }
  }
}

cudaError_t launch_build_am(const Mat& A, uint32_t* pk_am, int32_t L, cudaStream_t s) {
  const unsigned nb = grid_of(A.rows, A.num_sms);
  const uint32_t* pk = reinterpret_cast<const uint32_t*>(A.val);
  if (A.idx64)
    k_build_am<int64_t><<<nb, 256, 0, s>>>(A.rows, A.m, A.n, static_cast<const int64_t*>(A.rp),
                                           A.uniform_len, pk, L, pk_am);
  else
    k_build_am<int32_t><<<nb, 256, 0, s>>>(A.rows, A.m, A.n, static_cast<const int32_t*>(A.rp),
                                           A.uniform_len, pk, L, pk_am);
  return cudaGetLastError();
}

}  // namespace mdpk
