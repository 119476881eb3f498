// GMRES(k) for the policy-evaluation system (I - gamma P_pi) d = r.
//
// madupite ("Problem Setting and Solution Methods") evaluates each policy only
// approximately, with an inner Krylov solver, GMRES being the method of the
// inexact GMRES policy iteration it cites.  The Arnoldi process below is the
// classical Gram-Schmidt variant (Saad & Schultz 1986; Saad 2003, Alg. 6.9
// with CGS in place of MGS), with an optional second Gram-Schmidt pass, and
// the least-squares problem is solved by Givens rotations (Saad 2003, 6.5.3).
//
// Basis storage: u_0..u_k as FP32 columns of length n (leading dimension ld),
// with v_i = u_i * scale_i; the scale of a new vector is applied lazily by
// every reader, which saves a normalisation pass over the basis.
//
// Per Arnoldi step j the host enqueues:
//   K2  k_arnoldi_spmv : w = v_j - gamma P_pi v_j (row s*m+pi(s) gathered from
//                        the full CSR), stored in u_{j+1} (k_spmv.cuh);
//       k_gs_dots      : h_i = <w, v_i>, i <= j (k_dots.cuh);
//   K3  k_arnoldi_ortho: u_{j+1} = w - sum h_i v_i, ||u_{j+1}||_2; the last
//                        block appends column j of H, applies the Givens
//                        rotations, updates |g_{j+1}| and decides convergence
//                        (K4, a single thread in FP64).
// and at the end of a cycle
//   K5  k_gmres_update : V += sum_i y_i v_i in float-float.
// Every kernel of a step first reads st->active and returns at once when the
// cycle has ended, so a whole cycle can be enqueued without host round trips.
// Modified policy iteration's Richardson sweeps run through the policy-row
// kernel (its RICH form); this file holds their start kernel.
#include "k_rows.cuh"
#include "launch.h"

namespace mdpk {

static int64_t grid_blocks(const Grid& G) {
  int64_t b = (G.n_tiles + G.tiles_per_block - 1) / G.tiles_per_block;
  return b < 1 ? 1 : b;
}

static Grid grid_for(int64_t n_tiles, int max_blocks, int tile_states) {
  Grid G;
  G.tile_states = tile_states;
  G.n_tiles = n_tiles;
  int64_t blocks = n_tiles < max_blocks ? n_tiles : max_blocks;
  if (blocks < 1) blocks = 1;
  G.tiles_per_block = (n_tiles + blocks - 1) / blocks;
  if (G.tiles_per_block < 1) G.tiles_per_block = 1;
  return G;
}

template <typename K>
static int occ_of(K kernel) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, 0) != cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

// K4 (single thread): append ||w|| to column j, rotate, test convergence; at
// the end of the cycle back-solve R y = g.
__device__ void givens_step(DevState* st, int j, double nrm) {
  double* h = st->H + static_cast<int64_t>(j) * kMaxBasis;
  double colmax = 0.0;
  for (int i = 0; i <= j; ++i) colmax = fmax(colmax, fabs(h[i]));
  const bool breakdown = !(nrm > 1e-14 * colmax) || !(nrm > 1e-300);
  h[j + 1] = nrm;
  double* hr = st->Hraw + static_cast<int64_t>(j) * kMaxBasis;
  for (int i = 0; i <= j + 1; ++i) hr[i] = h[i];
  st->scale[j + 1] = breakdown ? 0.0 : 1.0 / nrm;
  for (int i = 0; i < j; ++i) {
    const double t = st->cs[i] * h[i] + st->sn[i] * h[i + 1];
    h[i + 1] = -st->sn[i] * h[i] + st->cs[i] * h[i + 1];
    h[i] = t;
  }
  const double a = h[j], b = breakdown ? 0.0 : h[j + 1];
  const double den = hypot(a, b);
  double c = 1.0, sn = 0.0;
  if (den > 0.0) {
    c = a / den;
    sn = b / den;
  }
  st->cs[j] = c;
  st->sn[j] = sn;
  h[j] = den > 0.0 ? den : a;
  h[j + 1] = 0.0;
  st->gv[j + 1] = -sn * st->gv[j];
  st->gv[j] = c * st->gv[j];
  const double est = fabs(st->gv[j + 1]);
  st->est = est;
  st->jdone = j + 1;
  st->nspmv = j + 1;
  const bool conv = breakdown || est <= st->target;
  if (conv || j + 1 >= st->restart) {
    st->active = 0;
    st->converged = conv ? 1 : 0;
    st->breakdown = breakdown ? 1 : 0;
    const int J = j + 1;
    for (int i = J - 1; i >= 0; --i) {
      double t = st->gv[i];
      for (int k = i + 1; k < J; ++k) t -= st->H[static_cast<int64_t>(k) * kMaxBasis + i] * st->y[k];
      const double d = st->H[static_cast<int64_t>(i) * kMaxBasis + i];
      st->y[i] = d != 0.0 ? t / d : 0.0;
    }
    st->last_J = J;
    st->last_beta = st->beta;
    st->last_est = est;
  }
}

// ---------------------------------------------------------------------------
// K3: u_{j+1} -= sum_i c_i u_i with c_i = h_i * scale_i, then ||u_{j+1}||_2.
// mode 0: CGS with H(:, j), then Givens.  mode 1: first pass of CGS2 (no norm).
// mode 2: second pass of CGS2 with st->h2 (added into H), then Givens.
// ---------------------------------------------------------------------------
// Subtract sum_i c_i u_i from one float4 quad of u_{j+1} (c_i = coef[i]).
__device__ __forceinline__ void ortho_fma(float4& w, float c, const float4& b) {
  w.x = fmaf(-c, b.x, w.x);
  w.y = fmaf(-c, b.y, w.y);
  w.z = fmaf(-c, b.z, w.z);
  w.w = fmaf(-c, b.w, w.w);
}

// wa, wb -= sum_{i <= j} coef_i v_i at the quads starting at states sa, sb:
// two basis vectors per step, so four 16-byte loads are in flight per thread.
// The basis is streamed once per pass (evict-first).
__device__ __forceinline__ void ortho_pair(const float* __restrict__ basis, int64_t ld, int j,
                                           const float* coef, int64_t sa, int64_t sb, float4& wa,
                                           float4& wb) {
  int i = 0;
  for (; i + 1 <= j; i += 2) {
    const float* b0 = basis + static_cast<int64_t>(i) * ld;
    const float* b1 = b0 + ld;
    const float4 a0 = __ldcs(reinterpret_cast<const float4*>(b0 + sa));
    const float4 c0 = __ldcs(reinterpret_cast<const float4*>(b0 + sb));
    const float4 a1 = __ldcs(reinterpret_cast<const float4*>(b1 + sa));
    const float4 c1 = __ldcs(reinterpret_cast<const float4*>(b1 + sb));
    ortho_fma(wa, coef[i], a0);
    ortho_fma(wb, coef[i], c0);
    ortho_fma(wa, coef[i + 1], a1);
    ortho_fma(wb, coef[i + 1], c1);
  }
  if (i <= j) {
    const float* b0 = basis + static_cast<int64_t>(i) * ld;
    ortho_fma(wa, coef[i], __ldcs(reinterpret_cast<const float4*>(b0 + sa)));
    ortho_fma(wb, coef[i], __ldcs(reinterpret_cast<const float4*>(b0 + sb)));
  }
}

// One quad on its own (ragged end of the vector), same order of operations.
__device__ __forceinline__ float4 ortho_quad(const float* __restrict__ basis, int64_t ld, int j,
                                             const float* coef, int64_t s, float4 w) {
  for (int i = 0; i <= j; ++i)
    ortho_fma(w, coef[i], *reinterpret_cast<const float4*>(basis + static_cast<int64_t>(i) * ld + s));
  return w;
}

// Warp tiles of 256 states: lane l owns the quads at states 256t + 4l and
// 256t + 128 + 4l of warp tile t, so a warp reads one contiguous kilobyte of
// every basis vector per tile (long DRAM runs).  Warps take tiles t = global
// warp index, + total warps, ... : every warp gets the same number of tiles
// to within one.
__global__ void __launch_bounds__(kThreads)
    k_arnoldi_ortho(int64_t n, float* __restrict__ basis, int64_t ld, int j, int mode,
                    double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  __shared__ float coef[kMaxBasis];
  __shared__ double red[kThreads / 32];
  const double* h = mode == 2 ? st->h2 : st->H + static_cast<int64_t>(j) * kMaxBasis;
  for (int i = threadIdx.x; i <= j; i += kThreads)
    coef[i] = static_cast<float>(h[i] * st->scale[i]);
  __syncthreads();
  float* uw = basis + static_cast<int64_t>(j + 1) * ld;
  float acc = 0.f;
  const int64_t n_wt = (n + 255) / 256;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kThreads / 32);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
       t < n_wt; t += nw) {
    const int64_t s_a = t * 256 + 4 * (threadIdx.x & 31);
    const int64_t s_b = s_a + 128;
    if (s_b + 3 < n) {
      float4 wa = *reinterpret_cast<const float4*>(uw + s_a);
      float4 wb = *reinterpret_cast<const float4*>(uw + s_b);
      ortho_pair(basis, ld, j, coef, s_a, s_b, wa, wb);
      *reinterpret_cast<float4*>(uw + s_a) = wa;
      *reinterpret_cast<float4*>(uw + s_b) = wb;
      acc = fmaf(wa.x, wa.x, fmaf(wa.y, wa.y, fmaf(wa.z, wa.z, fmaf(wa.w, wa.w, acc))));
      acc = fmaf(wb.x, wb.x, fmaf(wb.y, wb.y, fmaf(wb.z, wb.z, fmaf(wb.w, wb.w, acc))));
    } else {
      // ragged end of the vector: each quad on its own, scalar past the last full quad
      for (int64_t sq : {s_a, s_b}) {
        if (sq + 3 < n) {
          float4 w = *reinterpret_cast<const float4*>(uw + sq);
          w = ortho_quad(basis, ld, j, coef, sq, w);
          *reinterpret_cast<float4*>(uw + sq) = w;
          acc = fmaf(w.x, w.x, fmaf(w.y, w.y, fmaf(w.z, w.z, fmaf(w.w, w.w, acc))));
        } else {
          for (int64_t t2 = sq; t2 < n && t2 < sq + 4; ++t2) {
            float w = uw[t2];
            for (int i = 0; i <= j; ++i)
              w = fmaf(-coef[i], basis[static_cast<int64_t>(i) * ld + t2], w);
            uw[t2] = w;
            acc = fmaf(w, w, acc);
          }
        }
      }
    }
  }
  if (mode == 1) return;
  const double bs = block_sum_d(static_cast<double>(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = bs;
  if (last_block(&st->counter[mode == 2 ? kCntOrtho2 : kCntOrtho])) {
    double sq = 0.0;
    for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += kThreads)
      sq += __ldcg(partials + b);
    sq = block_sum_d(sq, red);
    if (threadIdx.x == 0) {
      st->counter[mode == 2 ? kCntOrtho2 : kCntOrtho] = 0;
      if (mode == 2) {
        double* hc = st->H + static_cast<int64_t>(j) * kMaxBasis;
        for (int i = 0; i <= j; ++i) hc[i] += st->h2[i];
      }
      givens_step(st, j, sqrt(sq));
    }
  }
}

// K5: V += sum_{i < jdone} y_i scale_i u_i  (FP32 correction, float-float V).
__global__ void __launch_bounds__(kThreads)
    k_gmres_update(int64_t n, Grid G, const float* __restrict__ basis, int64_t ld,
                   float2* __restrict__ V, const DevState* __restrict__ st) {
  __shared__ float coef[kMaxRestart];
  const int J = st->jdone;
  if (J == 0) return;
  for (int i = threadIdx.x; i < J; i += kThreads)
    coef[i] = static_cast<float>(st->y[i] * st->scale[i]);
  __syncthreads();
  const int64_t nq = (n + 3) / 4;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t q = tile * kThreads + threadIdx.x;
    if (q >= nq) continue;
    const int64_t s = 4 * q;
    if (s + 3 < n) {
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int i = 0; i < J; ++i) {
        const float4 b = *reinterpret_cast<const float4*>(basis + static_cast<int64_t>(i) * ld + s);
        const float c = coef[i];
        d.x = fmaf(c, b.x, d.x);
        d.y = fmaf(c, b.y, d.y);
        d.z = fmaf(c, b.z, d.z);
        d.w = fmaf(c, b.w, d.w);
      }
      float4* v4 = reinterpret_cast<float4*>(V + s);  // two float2 per float4
      float4 va = v4[0], vb = v4[1];
      ff r0 = ff_add_f(ff{va.x, va.y}, d.x), r1 = ff_add_f(ff{va.z, va.w}, d.y);
      ff r2 = ff_add_f(ff{vb.x, vb.y}, d.z), r3 = ff_add_f(ff{vb.z, vb.w}, d.w);
      v4[0] = make_float4(r0.hi, r0.lo, r1.hi, r1.lo);
      v4[1] = make_float4(r2.hi, r2.lo, r3.hi, r3.lo);
    } else {
      for (int64_t t = s; t < n; ++t) {
        float d = 0.f;
        for (int i = 0; i < J; ++i) d = fmaf(coef[i], basis[static_cast<int64_t>(i) * ld + t], d);
        const float2 v = V[t];
        const ff r = ff_add_f(ff{v.x, v.y}, d);
        V[t] = make_float2(r.hi, r.lo);
      }
    }
  }
}

// Start a run of Richardson sweeps toward the residual target.
__global__ void k_richardson_begin(DevState* st, double target) {
  st->active = 1;
  st->jdone = 0;
  st->target = target;
}

__global__ void k_ff_axpy(int64_t n, float2* __restrict__ V, const float* __restrict__ d) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float2 v = V[s];
    const ff r = ff_add_f(ff{v.x, v.y}, d[s]);
    V[s] = make_float2(r.hi, r.lo);
  }
}

// Caller vector -> float-float iterate.  neg: the handle maximises rewards and
// works on -V internally (negation is exact, so the split of -v is the negated
// split of v).
__global__ void k_to_ff(int64_t n, const void* __restrict__ src, int f64, int neg,
                        float2* __restrict__ dst) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (f64) {
      const double v0 = static_cast<const double*>(src)[s];
      const double v = neg ? -v0 : v0;
      const float hi = static_cast<float>(v);
      dst[s] = make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
    } else {
      const float v0 = static_cast<const float*>(src)[s];
      dst[s] = make_float2(neg ? -v0 : v0, 0.f);
    }
  }
}

// Float-float iterate -> caller vector; neg as in k_to_ff (the rounded sum is
// negated, which equals the rounded sum of the negated parts).
__global__ void k_from_ff(int64_t n, const float2* __restrict__ src, void* __restrict__ dst,
                          int f64, int neg) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float2 v = src[s];
    if (f64) {
      const double r = static_cast<double>(v.x) + static_cast<double>(v.y);
      static_cast<double*>(dst)[s] = neg ? -r : r;
    } else {
      const float r = __fadd_rn(v.x, v.y);
      static_cast<float*>(dst)[s] = neg ? -r : r;
    }
  }
}

// dst = -src elementwise (FP32 or FP64); dst may equal src.
__global__ void k_negate(int64_t n, const void* src, void* dst, int f64) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (f64) static_cast<double*>(dst)[s] = -static_cast<const double*>(src)[s];
    else static_cast<float*>(dst)[s] = -static_cast<const float*>(src)[s];
  }
}

// ---------------------------------------------------------------------------
// BiCGStab vector updates (van der Vorst 1992).  The policy SpMVs and the
// scalars alpha and omega come from k_bicg_spmv; each kernel here returns at
// once when the solve is over (DevState::active), so a batch of iterations can
// be enqueued without reading the status between them.  Reductions are fixed
// order (per-thread sums over a fixed grid-stride, block sums, last block).
// ---------------------------------------------------------------------------

// Shared tail: publish two block sums; the last block sums them in block order
// and hands the totals to `fin` (thread 0 only).
template <typename Fin>
__device__ __forceinline__ void bicg_reduce2(double a, double b, double* partials,
                                             DevState* st, Fin fin) {
  __shared__ double red[kThreads / 32];
  const double ba = block_sum_d(a, red);
  const double bb = block_sum_d(b, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = ba;
    partials[2 * blockIdx.x + 1] = bb;
  }
  if (last_block(&st->counter[kCntBicg])) {
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kThreads) {
      sa += __ldcg(partials + 2 * i);
      sb += __ldcg(partials + 2 * i + 1);
    }
    sa = block_sum_d(sa, red);
    sb = block_sum_d(sb, red);
    if (threadIdx.x == 0) {
      st->counter[kCntBicg] = 0;
      fin(sa, sb);
    }
  }
}

// r = p = r0, x = 0, rho = <r0, r0>; the solve starts unless ||r0||_2 <= target.
__global__ void k_bicg_begin(int64_t n, const float* __restrict__ r0, float* __restrict__ r,
                             float* __restrict__ p, float* __restrict__ x, double target,
                             double* __restrict__ partials, DevState* __restrict__ st) {
  double sq = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = r0[i];
    r[i] = v;
    p[i] = v;
    x[i] = 0.f;
    sq += static_cast<double>(v) * static_cast<double>(v);
  }
  bicg_reduce2(sq, 0.0, partials, st, [&](double rr, double) {
    st->bicg_rho = rr;
    st->res_2 = sqrt(rr);
    st->target = target;
    st->jdone = 0;
    st->breakdown = 0;
    const bool done = !(sqrt(rr) > target);
    st->converged = done ? 1 : 0;
    st->active = done ? 0 : 1;
  });
}

// x += alpha p;  s = r - alpha v (in place of r);  stop when ||s||_2 <= target.
__global__ void k_bicg_s(int64_t n, const float* __restrict__ p, const float* __restrict__ v,
                         float* __restrict__ r, float* __restrict__ x,
                         double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  const float alpha = static_cast<float>(st->bicg_alpha);
  double sq = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    x[i] = fmaf(alpha, p[i], x[i]);
    const float sv = fmaf(-alpha, v[i], r[i]);
    r[i] = sv;
    sq += static_cast<double>(sv) * static_cast<double>(sv);
  }
  bicg_reduce2(sq, 0.0, partials, st, [&](double ss, double) {
    st->res_2 = sqrt(ss);
    if (!(sqrt(ss) > st->target)) {
      st->jdone += 1;
      st->converged = 1;
      st->active = 0;
    }
  });
}

// x += omega s;  r = s - omega t;  rho' = <r^, r>;  beta = (rho'/rho)(alpha/omega).
__global__ void k_bicg_r(int64_t n, const float* __restrict__ rhat, const float* __restrict__ t,
                         float* __restrict__ r, float* __restrict__ x,
                         double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  const float omega = static_cast<float>(st->bicg_omega);
  double d = 0.0, sq = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float sv = r[i];
    x[i] = fmaf(omega, sv, x[i]);
    const float rv = fmaf(-omega, t[i], sv);
    r[i] = rv;
    d += static_cast<double>(rhat[i]) * static_cast<double>(rv);
    sq += static_cast<double>(rv) * static_cast<double>(rv);
  }
  bicg_reduce2(d, sq, partials, st, [&](double rho_new, double rr) {
    st->res_2 = sqrt(rr);
    st->jdone += 1;
    if (!(sqrt(rr) > st->target)) {
      st->converged = 1;
      st->active = 0;
      return;
    }
    const double beta = (rho_new / st->bicg_rho) * (st->bicg_alpha / st->bicg_omega);
    if (!(rho_new != 0.0 && isfinite(beta))) {
      st->breakdown = 1;
      st->active = 0;
      return;
    }
    st->bicg_beta = beta;
    st->bicg_rho = rho_new;
  });
}

// p = r + beta (p - omega v).
__global__ void k_bicg_p(int64_t n, const float* __restrict__ r, const float* __restrict__ v,
                         float* __restrict__ p, const DevState* __restrict__ st) {
  if (!st->active) return;
  const float beta = static_cast<float>(st->bicg_beta);
  const float omega = static_cast<float>(st->bicg_omega);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = fmaf(beta, fmaf(-omega, v[i], p[i]), r[i]);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_arnoldi_spmv(const Mat& A, bool lp, const int32_t* pi, float* basis,
                                int64_t ld, int j, float cdiag, double* partials, DevState* st,
                                cudaStream_t s) {
  if (!lp) return launch_arnoldi_spmv_f32(A, pi, basis, ld, j, cdiag, partials, st, s);
  if (A.store_t == 3) return launch_arnoldi_spmv_f16(A, pi, basis, ld, j, cdiag, partials, st, s);
  return launch_arnoldi_spmv_bf16(A, pi, basis, ld, j, cdiag, partials, st, s);
}

// Grid over thread-quads (4 states per thread) for the basis streams.
static Grid stream_grid(int64_t n, int num_sms, int occ) {
  const int64_t nq = (n + 3) / 4;
  return grid_for((nq + kThreads - 1) / kThreads, num_sms * occ, kThreads);
}

cudaError_t launch_arnoldi_ortho(const Mat& A, float* basis, int64_t ld, int j, int restart,
                                 int cgs2, double* partials, DevState* st, cudaStream_t s) {
  static int occ = occ_of(k_arnoldi_ortho);
  const int64_t warp_tiles = (A.n + 255) / 256;
  const int64_t want = (warp_tiles + kThreads / 32 - 1) / (kThreads / 32);
  const int64_t cap = static_cast<int64_t>(A.num_sms) * occ;
  const unsigned nb = static_cast<unsigned>(want < cap ? (want < 1 ? 1 : want) : cap);
  if (!cgs2) {
    k_arnoldi_ortho<<<nb, kThreads, 0, s>>>(A.n, basis, ld, j, 0, partials, st);
    return cudaGetLastError();
  }
  k_arnoldi_ortho<<<nb, kThreads, 0, s>>>(A.n, basis, ld, j, 1, partials, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_arnoldi_dots(A, basis, ld, j, restart, 1, partials, st, s);
  if (e != cudaSuccess) return e;
  k_arnoldi_ortho<<<nb, kThreads, 0, s>>>(A.n, basis, ld, j, 2, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_gmres_update(const Mat& A, float* basis, int64_t ld, float2* V, DevState* st,
                                cudaStream_t s) {
  static int occ = occ_of(k_gmres_update);
  const Grid G = stream_grid(A.n, A.num_sms, occ);
  k_gmres_update<<<static_cast<unsigned>(grid_blocks(G)), kThreads, 0, s>>>(A.n, G, basis, ld, V,
                                                                            st);
  return cudaGetLastError();
}

cudaError_t launch_richardson(const Mat& A, bool lp, const int32_t* pi, const float* r,
                              const float* d_in, float* d_out, double* partials, DevState* st,
                              cudaStream_t s) {
  if (!lp) return launch_richardson_f32(A, pi, r, d_in, d_out, partials, st, s);
  if (A.store_t == 3) return launch_richardson_f16(A, pi, r, d_in, d_out, partials, st, s);
  return launch_richardson_bf16(A, pi, r, d_in, d_out, partials, st, s);
}

static unsigned ew_blocks(int64_t n, int num_sms) {
  int64_t b = (n + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  if (b > cap) b = cap;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

cudaError_t launch_richardson_begin(DevState* st, double target, cudaStream_t s) {
  k_richardson_begin<<<1, 1, 0, s>>>(st, target);
  return cudaGetLastError();
}

cudaError_t launch_ff_axpy(int64_t n, float2* V, const float* d, int num_sms, cudaStream_t s) {
  k_ff_axpy<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, V, d);
  return cudaGetLastError();
}

cudaError_t launch_to_ff(int64_t n, const void* src, int src_f64, int neg, float2* dst,
                         int num_sms, cudaStream_t s) {
  k_to_ff<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, src, src_f64, neg, dst);
  return cudaGetLastError();
}

cudaError_t launch_from_ff(int64_t n, const float2* src, void* dst, int dst_f64, int neg,
                           int num_sms, cudaStream_t s) {
  k_from_ff<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, src, dst, dst_f64, neg);
  return cudaGetLastError();
}

cudaError_t launch_negate(int64_t n, const void* src, void* dst, int f64, int num_sms,
                          cudaStream_t s) {
  k_negate<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, src, dst, f64);
  return cudaGetLastError();
}

cudaError_t launch_bicg_begin(int64_t n, const float* r0, float* r, float* p, float* x,
                              double target, double* partials, DevState* st, int num_sms,
                              cudaStream_t s) {
  k_bicg_begin<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, r0, r, p, x, target, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_s(int64_t n, const float* p, const float* v, float* r, float* x,
                          double* partials, DevState* st, int num_sms, cudaStream_t s) {
  k_bicg_s<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, p, v, r, x, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_r(int64_t n, const float* rhat, const float* t, float* r, float* x,
                          double* partials, DevState* st, int num_sms, cudaStream_t s) {
  k_bicg_r<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, rhat, t, r, x, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_p(int64_t n, const float* r, const float* v, float* p,
                          const DevState* st, int num_sms, cudaStream_t s) {
  k_bicg_p<<<ew_blocks(n, num_sms), kThreads, 0, s>>>(n, r, v, p, st);
  return cudaGetLastError();
}

}  // namespace mdpk
