// The small FP64 steps of an s-step GMRES block and the per-quad update of
// the block's orthonormalisation, shared by the single-MDP kernels
// (k_sstep.cu) and the kernels that run the blocks of many MDPs in one launch
// (k_batch.cu).  See k_sstep.cu for the method.
#pragma once

#include "k_rows.cuh"
#include "launch.h"

namespace mdpk {

constexpr int kBlkThreads = 256;
constexpr int kBlkChunk = 1024;             // at least this many states per Gram slot
constexpr int kBlkStride = kBlkMaxV * kSMax;           // doubles per partial slot
constexpr int kBlkRun = 8;                  // chunk slots per first-level reduction
constexpr double kPivotRel = 1e-9;          // dependence threshold on R_ii^2 / ||w_i||^2

// ---------------------------------------------------------------------------
// The small steps of a block (run by the whole last block of the Gram pass,
// FP64).  k: first step of the block, sb: block vectors; `scratch` holds
// kMaxRestart * kMaxRestart doubles of shared memory.
//
// FP64 instructions issue at a small fraction of the FP32 rate on this GPU and
// cost the same whether one lane or all 32 are active, so the sequential parts
// run on the lanes of warp 0 in parallel wherever the data allow: the Cholesky
// factor column by column (one lane per remaining column or pair), R^{-1} one
// column per lane, the earlier rotations applied to all new columns at once,
// and the back-solve one row per lane.
// ---------------------------------------------------------------------------
static __device__ void block_ls(DevState* st, int k, int sb, int restart, double* scratch) {
  __shared__ double C[kMaxBasis * kSMax];  // C[v * kSMax + i] = <q_v, w_{i+1}>
  __shared__ double Sm[kSMax * kSMax];     // W^T W - C^T C, then R (upper)
  __shared__ double Ri[kSMax * kSMax];     // R^{-1}
  __shared__ double rinv[kSMax];           // 1 / R_jj
  __shared__ double hc[kSMax][kBlkMaxV];   // new Hessenberg columns
  __shared__ double rcs[kMaxRestart], rsn[kMaxRestart], rgv[kMaxBasis];
  __shared__ double ys[kMaxRestart];
  __shared__ int s_ncol, s_nnew, s_J, s_end;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nq = k + 1;
  (void)restart;
  // C from the Gram block: dots with the raw columns times their scales
  for (int t = tid; t < nq * kSMax; t += blockDim.x) {
    const int v = t / kSMax, i = t % kSMax;
    C[t] = i < sb ? st->G[v * kSMax + i] * st->scale[v] : 0.0;
  }
  __syncthreads();
  for (int t = tid; t < kSMax * kSMax; t += blockDim.x) {
    const int i = t / kSMax, j = t % kSMax;
    double sij = 0.0;
    if (i < sb && j < sb) {
      sij = st->G[(nq + i) * kSMax + j];
      for (int v = 0; v < nq; ++v) sij -= C[v * kSMax + i] * C[v * kSMax + j];
    }
    Sm[t] = sij;
  }
  __syncthreads();
  if (warp == 0) {
    // right-looking Cholesky S = R^T R in place (upper triangle); a pivot
    // below kPivotRel of its column's squared norm is an exact dependence:
    // R_cc = 0 and the columns after c are dropped
    int nnew = sb, ncol = sb;
    for (int j = 0; j < sb; ++j) {
      const double d = Sm[j * kSMax + j];
      const double wn = st->G[(nq + j) * kSMax + j];  // ||w_{j+1}||^2
      if (!(d > kPivotRel * wn) || !(wn > 0.0)) {
        nnew = j;
        ncol = j + 1;
        break;
      }
      const double inv = rsqrt(d);
      if (lane > j && lane < sb) Sm[j * kSMax + lane] *= inv;  // R[j][l]
      __syncwarp();
      // trailing update S[p][q] -= R[j][p] R[j][q], j < p <= q < sb (<= 28 pairs)
      for (int pq = lane; pq < kSMax * kSMax; pq += 32) {
        const int pp = pq / kSMax, qq = pq % kSMax;
        if (pp > j && qq >= pp && qq < sb) Sm[pp * kSMax + qq] -= Sm[j * kSMax + pp] * Sm[j * kSMax + qq];
      }
      if (lane == 0) {
        Sm[j * kSMax + j] = d * inv;
        rinv[j] = inv;
      }
      __syncwarp();
    }
    // R: the upper triangle of the kept columns (column c = nnew keeps R[l][c],
    // l < c, with R_cc = 0 when the block broke down)
    for (int t = lane; t < kSMax * kSMax; t += 32) {
      const int i = t / kSMax, j = t % kSMax;
      if (i > j || j >= ncol || (j == nnew && i == j)) Sm[t] = 0.0;
    }
    __syncwarp();
    // R^{-1} of the leading nnew columns, one column per lane
    for (int t = lane; t < kSMax * kSMax; t += 32) Ri[t] = 0.0;
    __syncwarp();
    if (lane < nnew) {
      const int j = lane;
      Ri[j * kSMax + j] = rinv[j];
      for (int i = j - 1; i >= 0; --i) {
        double t = 0.0;
        for (int l = i + 1; l <= j; ++l) t += Sm[i * kSMax + l] * Ri[l * kSMax + j];
        Ri[i * kSMax + j] = -t * rinv[i];
      }
    }
    if (lane == 0) {
      s_ncol = ncol;
      s_nnew = nnew;
    }
  }
  __syncthreads();
  const int ncol = s_ncol, nnew = s_nnew;
  // New Hessenberg columns, one row per thread.  With z_0 = q_k and
  // z_j = w_j = sum_v C[v][j-1] q_v + sum_{l<j} R[l][j-1] q_{k+1+l}, the
  // basis relation A z_i = z_{i+1} + z_i gives
  //   A q_k     = z_1 + z_0
  //   A q_{k+i} = (z_{i+1} + z_i - sum_{v<k} C[v][i-1] A q_v - C[k][i-1] A q_k
  //                - sum_{l<i-1} R[l][i-1] A q_{k+1+l}) / R[i-1][i-1],
  // with A q_v (v < k) the earlier columns of the cycle (Hraw, unrotated).
  const int rows = k + ncol + 1;
  // the earlier raw columns (rows 0..k), staged: hs[v * kMaxRestart + m]
  double* hs = scratch;
  for (int t = tid; t < k * kMaxRestart; t += blockDim.x) {
    const int v = t / kMaxRestart, m = t % kMaxRestart;
    hs[t] = m <= v + 1 ? st->Hraw[static_cast<int64_t>(v) * kMaxBasis + m] : 0.0;
  }
  __syncthreads();
  for (int m = tid; m < rows; m += blockDim.x) {
    auto coefz = [&](int j) -> double {  // row m of z_j (j >= 1)
      if (m <= k) return C[m * kSMax + (j - 1)];
      const int l = m - k - 1;
      return l < j ? Sm[l * kSMax + (j - 1)] : 0.0;
    };
    hc[0][m] = coefz(1) + (m == k ? 1.0 : 0.0);
    for (int i = 1; i < ncol; ++i) {
      double t = coefz(i + 1) + coefz(i);
      for (int v = (m > 0 ? m - 1 : 0); v < k; ++v) t -= C[v * kSMax + (i - 1)] * hs[v * kMaxRestart + m];
      t -= C[k * kSMax + (i - 1)] * hc[0][m];
      for (int l = 0; l < i - 1; ++l) t -= Sm[l * kSMax + (i - 1)] * hc[l + 1][m];
      hc[i][m] = t * rinv[i - 1];
    }
  }
  __syncthreads();
  // store the raw columns (rows beyond the subdiagonal are zero by construction)
  for (int t = tid; t < ncol * kMaxBasis; t += blockDim.x) {
    const int i = t / kMaxBasis, m = t % kMaxBasis;
    const int j = k + i;
    st->Hraw[static_cast<int64_t>(j) * kMaxBasis + m] = m <= j + 1 && m < rows ? hc[i][m] : 0.0;
  }
  // the rotations so far and the right-hand side
  for (int t = tid; t < k; t += blockDim.x) {
    rcs[t] = st->cs[t];
    rsn[t] = st->sn[t];
  }
  for (int t = tid; t <= k; t += blockDim.x) rgv[t] = st->gv[t];
  __syncthreads();
  if (warp == 0) {
    // the earlier rotations on every new column at once (lane = column)
    if (lane < ncol) {
      double* h = hc[lane];
      for (int l = 0; l < k; ++l) {
        const double t = rcs[l] * h[l] + rsn[l] * h[l + 1];
        h[l + 1] = -rsn[l] * h[l] + rcs[l] * h[l + 1];
        h[l] = t;
      }
    }
    __syncwarp();
    if (lane == 0) {
      // the block's own rotations in order, and the convergence test per column
      bool end = false, conv = false, brk = false;
      int J = k + ncol;
      for (int i = 0; i < ncol && !end; ++i) {
        const int j = k + i;
        double* h = hc[i];
        for (int l = k; l < j; ++l) {
          const double t = rcs[l] * h[l] + rsn[l] * h[l + 1];
          h[l + 1] = -rsn[l] * h[l] + rcs[l] * h[l + 1];
          h[l] = t;
        }
        const double a = h[j], b = h[j + 1];
        const bool breakdown = !(b != 0.0);
        const double r2 = a * a + b * b;
        double c = 1.0, sn = 0.0, den = a;
        if (r2 > 0.0) {
          const double inv = rsqrt(r2);
          c = a * inv;
          sn = b * inv;
          den = r2 * inv;
        }
        rcs[j] = c;
        rsn[j] = sn;
        h[j] = den;
        h[j + 1] = 0.0;
        rgv[j + 1] = -sn * rgv[j];
        rgv[j] = c * rgv[j];
        const double est = fabs(rgv[j + 1]);
        st->est = est;
        if (breakdown || est <= st->target) {
          end = true;
          conv = true;
          brk = breakdown;
          J = j + 1;
        }
      }
      if (!end && k + ncol >= st->restart) end = true;
      st->jdone = J;
      st->bsb = nnew;
      st->nspmv = k + sb;
      if (end) {
        st->active = 0;
        st->converged = conv ? 1 : 0;
        st->breakdown = brk ? 1 : 0;
        st->bfin_k = k;
        st->last_J = J;
        st->last_beta = st->beta;
        st->last_est = st->est;
      }
      s_J = J;
      s_end = end ? 1 : 0;
    }
  }
  __syncthreads();
  const int J = s_J;
  // write back the columns the rotations reached (J - k of them), the
  // rotations, the right-hand side and the update coefficients
  for (int t = tid; t < (J - k) * kMaxBasis; t += blockDim.x) {
    const int i = t / kMaxBasis, m = t % kMaxBasis;
    st->H[static_cast<int64_t>(k + i) * kMaxBasis + m] = m <= k + i + 1 ? hc[i][m] : 0.0;
  }
  for (int t = tid; t < J; t += blockDim.x) {
    st->cs[t] = rcs[t];
    st->sn[t] = rsn[t];
  }
  for (int t = tid; t <= J; t += blockDim.x) st->gv[t] = rgv[t];
  for (int t = tid; t < nq * kSMax; t += blockDim.x)
    st->bC[t] = static_cast<float>(C[t] * st->scale[t / kSMax]);
  for (int t = tid; t < kSMax * kSMax; t += blockDim.x) st->bRinv[t] = static_cast<float>(Ri[t]);
  __syncthreads();  // the scales above were read before the new ones are set
  for (int i = tid; i < nnew; i += blockDim.x) st->scale[k + 1 + i] = 1.0;
  if (!s_end) return;
  // end of the cycle: back-solve R y = g over the J columns, R staged in the
  // scratch (column c at scratch[c * kMaxRestart], rows 0..c); lane l owns
  // rows l and l + 32
  for (int t = tid; t < J * kMaxRestart; t += blockDim.x) {
    const int c = t / kMaxRestart, r = t % kMaxRestart;
    if (r <= c) scratch[t] = c < k ? st->H[static_cast<int64_t>(c) * kMaxBasis + r] : hc[c - k][r];
  }
  __syncthreads();
  if (warp == 0) {
    double tr[2], dinv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      tr[h] = r < J ? rgv[r] : 0.0;
      const double d = r < J ? scratch[r * kMaxRestart + r] : 0.0;
      dinv[h] = d != 0.0 ? 1.0 / d : 0.0;
    }
    for (int i = J - 1; i >= 0; --i) {
      const int hi = i >> 5, li = i & 31;
      const double mine = (hi ? tr[1] * dinv[1] : tr[0] * dinv[0]);
      const double yi = __shfl_sync(0xffffffffu, mine, li);
      if (lane == li) ys[i] = yi;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        if (r < i) tr[h] -= scratch[i * kMaxRestart + r] * yi;
      }
    }
  }
  __syncthreads();
  for (int v = tid; v < kBlkMaxV; v += blockDim.x) {
    const double yv = v < J ? ys[v] : 0.0;
    if (v < J) st->y[v] = yv;
    st->bY[v] = v < J ? static_cast<float>(yv * (v <= k ? st->scale[v] : 1.0)) : 0.f;
  }
}

// ---------------------------------------------------------------------------
// One quad of the update pass: w_i <- (w_i - sum_v C[v][i] u_v) R^{-1} for the
// block's columns k+1.. (returned in w), and vacc += sum_{v < J} y_v u_v on the
// block that ends the cycle.
// ---------------------------------------------------------------------------
template <int S>
__device__ __forceinline__ void block_update_quad(const float* __restrict__ basis, int64_t ld,
                                                  int k, int nnew, int J, bool fin,
                                                  const float* cf, const float* ri,
                                                  const float* yc, int64_t s, float4* w,
                                                  float4& vacc) {
  auto fma4 = [](float4& a, float c, const float4& b) {
    a.x = fmaf(c, b.x, a.x);
    a.y = fmaf(c, b.y, a.y);
    a.z = fmaf(c, b.z, a.z);
    a.w = fmaf(c, b.w, a.w);
  };
#pragma unroll
  for (int i = 0; i < S; ++i)
    w[i] = i < nnew ? *reinterpret_cast<const float4*>(basis + static_cast<int64_t>(k + 1 + i) * ld + s)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int v = 0; v <= k; ++v) {
    const float4 u = __ldcs(reinterpret_cast<const float4*>(basis + static_cast<int64_t>(v) * ld + s));
#pragma unroll
    for (int i = 0; i < S; ++i) fma4(w[i], -cf[v * kSMax + i], u);
    if (fin && v < J) fma4(vacc, yc[v], u);
  }
  // in place, last column first: q_i needs w_0..w_i only
#pragma unroll
  for (int i = S - 1; i >= 0; --i) {
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int l = 0; l <= i; ++l) fma4(q, ri[l * kSMax + i], w[l]);
    w[i] = q;
  }
}

}  // namespace mdpk
