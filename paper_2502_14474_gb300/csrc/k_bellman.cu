// K1 / K6: fused Bellman backup, greedy improvement and Bellman residual.
//
//   Q(s,a)  = g(s,a) + gamma * sum_e P_e V(col_e)   over row r = s*m + a
//   V'(s)   = min_a Q(s,a),  pi(s) = lowest a attaining the minimum
//   r(s)    = V'(s) - V(s),  ||r||_inf and ||r||_2 (FP64, fixed-order)
//
// (madupite, "Problem Setting and Solution Methods": the improvement step of
// policy iteration; applied alone it is value iteration.)
//
// Work decomposition: a CTA owns a contiguous range of state tiles (T states
// = T*m rows each).  Within a tile, vectors of VW lanes compute the row sums
// (coalesced col/val streams, V gathered through L1/L2) and drop Q into a
// shared-memory tile stored action-major; then one thread per state takes the
// min/argmin over its m actions and writes V', pi, r.  Blocked tile ranges
// keep each CTA's V window (the band around its states) hot in L1.
//
// FF = float-float: V is float2 (hi, lo), the row sums are error-free
// TwoSum/TwoProd accumulations, gamma and g are float-float; this is the
// high-precision residual of the outer iteration.  Otherwise FP32 throughout.
#include <type_traits>

#include "k_rows.cuh"
#include "launch.h"

namespace mdpk {

// Row stride of the action-major Q tile (q[a * stride + state]).  A warp of
// the row passes writes the m actions of 32/m consecutive states at once; with
// stride = 32/m (mod 32) their 32 words fall in 32 different banks (a stride
// that is a multiple of 32 put the m actions of a state in one bank).
// Short tiles (many actions) keep the plain stride: the padding would add up
// to 31 words per action to a tile of a few states.
__host__ __device__ __forceinline__ int qtile_stride(int T, int m) {
  if (T < 64) return T;
  const int target = (32 % m == 0) ? (32 / m) & 31 : 1;
  return T + (((target - T) % 32) + 32) % 32;
}

// Fast path of one pass over the rows of a tile when every row holds 4*VW
// entries (16-byte aligned): the vector owns VW consecutive rows, each lane
// loads its slice of all of them before any gather, and a reduce-scatter
// leaves lane l with the sum of row lr0 + l, which it turns into Q(s, a).
template <bool FF, int VW, typename IdxT, typename GX>
__device__ __forceinline__ void bellman_pass_fast(const Csr<IdxT>& P, GX gx, int64_t r0, int lr0,
                                                  int64_t rows_here, int lane, int QS,
                                                  float* q_hi, float* q_lo) {
  int64_t b[VW];
  bool vd[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    vd[u] = lr0 + u < rows_here;
    b[u] = (r0 + lr0 + u) * P.uniform_len;
  }
  const int lr = lr0 + lane;
  float hi, lo = 0.f;
  if constexpr (FF) {
    float ph[VW], pl[VW];
    vec_rows_ff<VW>(P.col, P.val, gx, b, vd, lane, ph, pl);
    reduce_scatter_ff<VW>(ph, pl, lane, hi, lo);
  } else {
    float p[VW];
    vec_rows_f32<VW, float>(P.col, P.val, gx, b, vd, lane, p);
    hi = reduce_scatter<VW>(p, lane);
  }
  if (lr < rows_here) {
    const int a = lr % P.m;
    const int sl = lr / P.m;
    const int64_t r = r0 + lr;
    if constexpr (FF) {
      const ff sum = ff_norm(hi, lo);
      const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
      const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
      q_hi[a * QS + sl] = q.hi;
      q_lo[a * QS + sl] = q.lo;
    } else {
      q_hi[a * QS + sl] = fmaf(P.gamma, hi, __ldcs(P.g + r));
    }
  }
}

// The float-float sums of a thread's two short rows side by side in the packed
// FP32x2 instructions (ff_acc2).  Both rows walk the eight slots of their first
// two packed groups; a slot outside a row adds p = 0 times x = 0, which leaves
// the row's sum unchanged (TwoSum of s and +0 is s and 0), so each sum equals
// that of row_pre_dot_ff up to the sign of an exactly zero sum.  The slots of
// rows longer than two groups follow one row at a time, as there.
template <typename GX>
__device__ __forceinline__ void row_pre_dot_ff2(const int32_t* __restrict__ col,
                                                const float* __restrict__ val, GX V,
                                                const RowPre<float> (&R)[2], float (&hi)[2],
                                                float (&lo)[2]) {
  int o[2], end[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    o[u] = static_cast<int>(R[u].b & 3);
    end[u] = o[u] + static_cast<int>(R[u].e - R[u].b);
  }
  const int ca[8] = {R[0].c0.x, R[0].c0.y, R[0].c0.z, R[0].c0.w,
                     R[0].c1.x, R[0].c1.y, R[0].c1.z, R[0].c1.w};
  const int cb[8] = {R[1].c0.x, R[1].c0.y, R[1].c0.z, R[1].c0.w,
                     R[1].c1.x, R[1].c1.y, R[1].c1.z, R[1].c1.w};
  const float pa[8] = {R[0].v0.x, R[0].v0.y, R[0].v0.z, R[0].v0.w,
                       R[0].v1.x, R[0].v1.y, R[0].v1.z, R[0].v1.w};
  const float pb[8] = {R[1].v0.x, R[1].v0.y, R[1].v0.z, R[1].v0.w,
                       R[1].v1.x, R[1].v1.y, R[1].v1.z, R[1].v1.w};
  float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool va = q >= o[0] && q < end[0], vb = q >= o[1] && q < end[1];
    const float2 xa = V(ca[q]), xb = V(cb[q]);
    ff_acc2(h, l, make_float2(va ? pa[q] : 0.f, vb ? pb[q] : 0.f),
            make_float2(va ? xa.x : 0.f, vb ? xb.x : 0.f),
            make_float2(va ? xa.y : 0.f, vb ? xb.y : 0.f));
  }
  hi[0] = h.x;
  lo[0] = l.x;
  hi[1] = h.y;
  lo[1] = l.y;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int64_t e = R[u].e;
    for (int64_t g = (R[u].b >> 2) + 2; (g << 2) < e; ++g) {
      const int64_t j0 = g << 2;
      const int4 c = ldcol4(col, j0);
      const float4 p = Ld<float>::four(val, j0);
      const int cq[4] = {c.x, c.y, c.z, c.w};
      const float pq[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (j0 + q < e) {
          const float2 v = V(cq[q]);
          ff_acc(hi[u], lo[u], pq[q], v.x, v.y);
        }
      }
    }
  }
}

// One thread per row, two rows per thread in flight (short rows, VW == 1).
// PACKED: the float-float sums of the two rows in packed instructions
// (row_pre_dot_ff2; more registers, so only where the CTA has them).
template <bool FF, typename IdxT, typename GX, bool PACKED = false>
__device__ __forceinline__ void bellman_pass_g1x2(const Csr<IdxT>& P, GX gx, int64_t r0, int lr_a,
                                                  int lr_b, int64_t rows_here, int QS, float* q_hi,
                                                  float* q_lo) {
  int64_t b[2] = {0, 0}, e[2] = {0, 0};
  const int lr[2] = {lr_a, lr_b};
#pragma unroll
  for (int u = 0; u < 2; ++u)
    if (lr[u] < rows_here) row_bounds<IdxT>(P.rp, P.uniform_len, r0 + lr[u], b[u], e[u]);
  if constexpr (FF) {
    float hi[2], lo[2];
    if (!P.val_lo) {
      // both rows' first two packed groups in flight before any gather
      RowPre<float> R[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) row_pre<float>(P.col, P.val, b[u], e[u], R[u]);
      if constexpr (PACKED) {
        row_pre_dot_ff2(P.col, P.val, gx, R, hi, lo);
      } else {
#pragma unroll
        for (int u = 0; u < 2; ++u) row_pre_dot_ff(P.col, P.val, gx, R[u], hi[u], lo[u]);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 2; ++u)
        row_dot_ff_g1(P.col, P.val, P.val_lo, gx, b[u], e[u], hi[u], lo[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (lr[u] < rows_here) {
        const int a = lr[u] % P.m, sl = lr[u] / P.m;
        const int64_t r = r0 + lr[u];
        const ff sum = ff_norm(hi[u], lo[u]);
        const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
        const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
        q_hi[a * QS + sl] = q.hi;
        q_lo[a * QS + sl] = q.lo;
      }
    }
  } else {
    RowPre<float> R[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) row_pre<float>(P.col, P.val, b[u], e[u], R[u]);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (lr[u] < rows_here) {
        const int a = lr[u] % P.m, sl = lr[u] / P.m;
        const float d = row_pre_dot<float>(P.col, P.val, gx, R[u]);
        q_hi[a * QS + sl] = fmaf(P.gamma, d, __ldcs(P.g + r0 + lr[u]));
      }
    }
  }
}

template <bool FF, typename IdxT, int VW>
__global__ void __launch_bounds__(kThreads)
    k_bellman(Csr<IdxT> P, Grid G, const void* __restrict__ Vin, void* __restrict__ Vout,
              int32_t* __restrict__ pi_out, float* __restrict__ r_out,
              double* __restrict__ partials, DevState* __restrict__ st, int init_gmres) {
  extern __shared__ float smem[];
  __shared__ double red[kThreads / 32];
  constexpr int NV = kThreads / VW;
  const int lane = threadIdx.x % VW;
  const int vec = threadIdx.x / VW;
  const int m = P.m;
  const int T = G.tile_states;
  const int RT = T * m;
  const int QS = qtile_stride(T, m);
  float* q_hi = smem;
  float* q_lo = smem + m * QS;
  const float* Vf = static_cast<const float*>(Vin);
  const float2* Vff = static_cast<const float2*>(Vin);
  const bool vec4 = P.vec4 != 0;
  const bool fast = VW <= 4 && P.uniform_len == 4 * VW && vec4 && !P.val_lo;

  double my_max = 0.0, my_sq = 0.0;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s0 = tile * T;
    const int64_t r0 = s0 * m;
    const int64_t rows_here = min(static_cast<int64_t>(RT), (P.n - s0) * m);
    if (fast) {
      if constexpr (VW <= 4) {
        for (int base = 0; base < RT; base += kThreads) {
          if constexpr (FF)
            bellman_pass_fast<FF, VW>(P, GatherFF{Vff}, r0, base + vec * VW, rows_here, lane, QS,
                                      q_hi, q_lo);
          else
            bellman_pass_fast<FF, VW>(P, GatherF32{Vf}, r0, base + vec * VW, rows_here, lane, QS,
                                      q_hi, q_lo);
        }
      }
    } else if (VW == 1) {
      for (int base = 0; base < RT; base += 2 * kThreads) {
        if constexpr (FF)
          bellman_pass_g1x2<FF>(P, GatherFF{Vff}, r0, base + threadIdx.x,
                                base + kThreads + threadIdx.x, rows_here, QS, q_hi, q_lo);
        else
          bellman_pass_g1x2<FF>(P, GatherF32{Vf}, r0, base + threadIdx.x,
                                base + kThreads + threadIdx.x, rows_here, QS, q_hi, q_lo);
      }
    } else
    for (int base = 0; base < RT; base += NV) {
      const int lr = base + vec;
      int64_t b = 0, e = 0;
      if (lr < rows_here) row_bounds<IdxT>(P.rp, P.uniform_len, r0 + lr, b, e);
      float hi, lo = 0.f;
      if constexpr (FF) {
        row_dot_ff<VW>(P.col, P.val, P.val_lo, Vff, b, e, lane, vec4, hi, lo);
        group_sum_ff<VW>(hi, lo);
      } else {
        hi = row_dot_f32<VW, float>(P.col, P.val, Vf, b, e, lane, vec4);
        hi = group_sum<VW>(hi);
      }
      if (lane == 0 && lr < rows_here) {
        const int a = lr % m;
        const int sl = lr / m;
        const int64_t r = r0 + lr;
        if constexpr (FF) {
          const ff sum = ff_norm(hi, lo);
          const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
          const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
          q_hi[a * QS + sl] = q.hi;
          q_lo[a * QS + sl] = q.lo;
        } else {
          q_hi[a * QS + sl] = fmaf(P.gamma, hi, __ldcs(P.g + r));
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += kThreads) {
      const int64_t s = s0 + t;
      if (s < P.n) {
        float bh = q_hi[t], bl = FF ? q_lo[t] : 0.f;
        int arg = 0;
        for (int a = 1; a < m; ++a) {
          const float h = q_hi[a * QS + t];
          const float l = FF ? q_lo[a * QS + t] : 0.f;
          if (h < bh || (FF && h == bh && l < bl)) {
            bh = h;
            bl = l;
            arg = a;
          }
        }
        float r;
        if constexpr (FF) {
          const float2 v = Vff[s];
          r = ff_diff_to_float(bh, bl, v.x, v.y);
          if (Vout) static_cast<float2*>(Vout)[s] = make_float2(bh, bl);
        } else {
          r = bh - Vf[s];
          if (Vout) static_cast<float*>(Vout)[s] = bh;
        }
        if (pi_out) pi_out[s] = arg;
        if (r_out) r_out[s] = r;
        const double rd = static_cast<double>(r);
        my_max = fmax(my_max, fabs(rd));
        my_sq += rd * rd;
      }
    }
    __syncthreads();
  }

  const double bmax = block_max_d(my_max, red);
  const double bsq = block_sum_d(my_sq, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bmax;
    partials[2 * blockIdx.x + 1] = bsq;
  }
  if (last_block(&st->counter[kCntBellman])) {
    double mx = 0.0, sq = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kThreads) {
      mx = fmax(mx, __ldcg(partials + 2 * i));
      sq += __ldcg(partials + 2 * i + 1);
    }
    mx = block_max_d(mx, red);
    sq = block_sum_d(sq, red);
    if (threadIdx.x == 0) {
      st->res_inf = mx;
      st->res_2 = sqrt(sq);
      st->counter[kCntBellman] = 0;
      if (init_gmres) {
        if (st->target_rel) st->target = st->eta * mx;
        gmres_begin(st, sqrt(sq));
      }
    }
  }
}

// Policy residual in float-float: r(s) = g(s,pi) + gamma * sum P_pi V - V(s).
// One vector per state; a CTA owns a contiguous range of NV-state tiles.
template <typename IdxT, int VW>
__global__ void __launch_bounds__(kThreads)
    k_policy_residual(Csr<IdxT> P, Grid G, const int32_t* __restrict__ pi,
                      const float2* __restrict__ V, float* __restrict__ r_out,
                      double* __restrict__ partials, DevState* __restrict__ st) {
  __shared__ double red[kThreads / 32];
  constexpr int NV = kThreads / VW;
  const int lane = threadIdx.x % VW;
  const int vec = threadIdx.x / VW;
  const bool vec4 = P.vec4 != 0;
  double my_max = 0.0, my_sq = 0.0;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s = tile * NV + vec;
    int64_t b = 0, e = 0, r = 0;
    if (s < P.n) {
      const int32_t a = __ldg(pi + s);
      r = s * P.m + a;  // cost row
      row_bounds<IdxT>(P.rp, P.uniform_len, policy_row(P, s, a), b, e);
    }
    float hi, lo;
    row_dot_ff<VW>(P.col, P.val, P.val_lo, V, b, e, lane, vec4, hi, lo);
    group_sum_ff<VW>(hi, lo);
    if (lane == 0 && s < P.n) {
      const ff sum = ff_norm(hi, lo);
      const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
      const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
      const float2 v = V[s];
      const float rr = ff_diff_to_float(q.hi, q.lo, v.x, v.y);
      r_out[s] = rr;
      const double rd = static_cast<double>(rr);
      my_max = fmax(my_max, fabs(rd));
      my_sq += rd * rd;
    }
  }
  const double bmax = block_max_d(my_max, red);
  const double bsq = block_sum_d(my_sq, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bmax;
    partials[2 * blockIdx.x + 1] = bsq;
  }
  if (last_block(&st->counter[kCntPolicy])) {
    double mx = 0.0, sq = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kThreads) {
      mx = fmax(mx, __ldcg(partials + 2 * i));
      sq += __ldcg(partials + 2 * i + 1);
    }
    mx = block_max_d(mx, red);
    sq = block_sum_d(sq, red);
    if (threadIdx.x == 0) {
      st->res_inf = mx;
      st->res_2 = sqrt(sq);
      st->counter[kCntPolicy] = 0;
      gmres_begin(st, sqrt(sq));
    }
  }
}

// Fast form for rows of exactly 4*VW entries with 16-byte aligned starts (the
// layout of the policy SpMV's fast path): a thread per state, a vector of VW
// lanes owns VW consecutive states and each lane loads its 16-byte slice of
// all VW policy rows before any gather; a reduce-scatter leaves every lane
// with its own state's float-float row sum.
template <typename IdxT, int VW>
__global__ void __launch_bounds__(kThreads)
    k_policy_residual_fast(Csr<IdxT> P, Grid G, const int32_t* __restrict__ pi,
                           const float2* __restrict__ V, float* __restrict__ r_out,
                           double* __restrict__ partials, DevState* __restrict__ st) {
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x % VW;
  double my_max = 0.0, my_sq = 0.0;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s = tile * kThreads + threadIdx.x;
    const bool valid = s < P.n;
    const int32_t a = valid ? __ldg(pi + s) : 0;
    const int64_t rb = policy_row(P, s, a) * P.uniform_len;
    int64_t b[VW];
    bool vd[VW];
#pragma unroll
    for (int u = 0; u < VW; ++u) {
      b[u] = __shfl_sync(0xffffffffu, rb, u, VW);
      vd[u] = __shfl_sync(0xffffffffu, valid ? 1 : 0, u, VW) != 0;
    }
    float ph[VW], pl[VW], hi, lo;
    vec_rows_ff<VW>(P.col, P.val, GatherFF{V}, b, vd, lane, ph, pl);
    reduce_scatter_ff<VW>(ph, pl, lane, hi, lo);
    if (valid) {
      const int64_t r = s * P.m + a;  // cost row
      const ff sum = ff_norm(hi, lo);
      const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
      const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
      const float2 v = V[s];
      const float rr = ff_diff_to_float(q.hi, q.lo, v.x, v.y);
      r_out[s] = rr;
      const double rd = static_cast<double>(rr);
      my_max = fmax(my_max, fabs(rd));
      my_sq += rd * rd;
    }
  }
  const double bmax = block_max_d(my_max, red);
  const double bsq = block_sum_d(my_sq, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bmax;
    partials[2 * blockIdx.x + 1] = bsq;
  }
  if (last_block(&st->counter[kCntPolicy])) {
    double mx = 0.0, sq = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kThreads) {
      mx = fmax(mx, __ldcg(partials + 2 * i));
      sq += __ldcg(partials + 2 * i + 1);
    }
    mx = block_max_d(mx, red);
    sq = block_sum_d(sq, red);
    if (threadIdx.x == 0) {
      st->res_inf = mx;
      st->res_2 = sqrt(sq);
      st->counter[kCntPolicy] = 0;
      gmres_begin(st, sqrt(sq));
    }
  }
}

// ---------------------------------------------------------------------------
// Banded variant: the value vector is staged in a shared-memory ring.
//
// When every successor lies within `band` states of its source state, a CTA
// that walks a contiguous range of tiles needs only V[s0 - band, s0 + T + band)
// for the tile starting at s0.  That window lives in a ring of R >= 2*band + 2*T
// slots (entry c at slot c & (R-1)); while the tile's rows gather from the
// ring, the CTA already writes the next tile's leading edge
// [s0 + T + band, s0 + 2T + band), whose slots differ from every live slot
// because R exceeds the distance between them.  Gathers become shared-memory
// loads instead of scattered 32-byte L2 sectors.
// ---------------------------------------------------------------------------
// Screened float-float pass (rows of 4*VW aligned entries, m a power of two
// dividing 32, so that after the reduce-scatter thread base + i owns row
// base + i and a state's m rows sit on m aligned lanes of one warp).
//
// Every row is first summed in FP32 over the high parts of V, q32 =
// fl(gamma * sum p h + g), together with a bound E >= |q32 - q| on the
// distance to the float-float value q of the full pass:
//   |q32 - q| <= u (|q32| + (k + 2) gamma A + |g|) + O(u^2),  A = sum |p h|,
// for k entries per row, u = 2^-24 (the FP32 dot product's error (k+1) u A,
// the dropped low parts of V, gamma and g one u each, the final rounding u
// |q32|).  E doubles the constant, E = 2 (k + 3) u (gamma A + |g| + |q32|).
// A row whose lower bound q32 - E (rounded down) exceeds the smallest upper
// bound q32 + E (rounded up) among its state's actions has a float-float
// value strictly above the state's minimum, so it can neither attain the
// minimum nor tie with it.  Only the remaining candidates gather the low parts
// and repeat the row sum in float-float with exactly the operations of the
// full pass; the state's minimum and its lowest minimising action, hence V'
// and pi, are bitwise those of the full pass.  The winner of each state is
// left in b_hi / b_lo / b_arg at the state's tile slot.
template <int VW, typename IdxT>
__device__ __forceinline__ void bellman_pass_screened(const Csr<IdxT>& P,
                                                      const float* __restrict__ rh,
                                                      const float* __restrict__ rl, int mask,
                                                      int64_t r0, int lr0, int64_t rows_here,
                                                      int lane, float* b_hi, float* b_lo,
                                                      int* b_arg) {
  constexpr unsigned kAll = 0xffffffffu;
  int4 c[VW];
  float4 q[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    if (lr0 + u < rows_here) {
      const int64_t b = (r0 + lr0 + u) * P.uniform_len + 4 * lane;
      c[u] = ldcol4(P.col, b);
      q[u] = Ld<float>::four(P.val, b);
    } else {
      c[u] = make_int4(0, 0, 0, 0);
      q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  float p32[VW], a32[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    c[u] = make_int4(c[u].x & mask, c[u].y & mask, c[u].z & mask, c[u].w & mask);
    const float h0 = rh[c[u].x], h1 = rh[c[u].y], h2 = rh[c[u].z], h3 = rh[c[u].w];
    p32[u] = fmaf(q[u].w, h3, fmaf(q[u].z, h2, fmaf(q[u].y, h1, q[u].x * h0)));
    a32[u] = fmaf(fabsf(q[u].w), fabsf(h3),
                  fmaf(fabsf(q[u].z), fabsf(h2), fmaf(fabsf(q[u].y), fabsf(h1), fabsf(q[u].x * h0))));
  }
  const float s32 = reduce_scatter<VW>(p32, lane);
  const float sa = reduce_scatter<VW>(a32, lane);
  const int lr = lr0 + lane;
  const bool valid = lr < rows_here;
  const int64_t r = r0 + lr;
  float ghi = 0.f, glo = 0.f;
  if (valid) {
    ghi = __ldcs(P.g + r);
    if (P.g_lo) glo = __ldcs(P.g_lo + r);
  }
  const float inf = __int_as_float(0x7f800000);
  const float q32 = fmaf(P.gamma_hi, s32, ghi);
  const float cE = 2.f * static_cast<float>(P.uniform_len + 3) * 0x1p-24f;
  const float E = fmaf(cE, fmaf(P.gamma_hi, sa, fabsf(ghi)) + fabsf(q32), 1e-30f);
  float up = valid ? __fadd_ru(q32, E) : inf;
  const float dn = valid ? __fsub_rd(q32, E) : inf;
  for (int o = 1; o < P.m; o <<= 1) up = fminf(up, __shfl_xor_sync(kAll, up, o));
  const bool cand = valid && !(dn > up);  // NaN bounds keep the row
  float ph[VW], pl[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    float h = 0.f, l = 0.f;
    if (__shfl_sync(kAll, cand ? 1 : 0, u, VW)) {
      ff_acc(h, l, q[u].x, rh[c[u].x], rl[c[u].x]);
      ff_acc(h, l, q[u].y, rh[c[u].y], rl[c[u].y]);
      ff_acc(h, l, q[u].z, rh[c[u].z], rl[c[u].z]);
      ff_acc(h, l, q[u].w, rh[c[u].w], rl[c[u].w]);
    }
    ph[u] = h;
    pl[u] = l;
  }
  float hi, lo;
  reduce_scatter_ff<VW>(ph, pl, lane, hi, lo);
  float bh = inf, bl = 0.f;
  if (cand) {
    const ff qq = ff_add(ff_mul(ff_norm(hi, lo), ff{P.gamma_hi, P.gamma_lo}), ff_norm(ghi, glo));
    bh = qq.hi;
    bl = qq.lo;
  }
  // (value, action) minimum over the state's lanes: the full pass keeps the
  // first of equal values, i.e. the lowest action among them
  const int a = lr & (P.m - 1);
  int ba = a;
  for (int o = 1; o < P.m; o <<= 1) {
    const float oh = __shfl_xor_sync(kAll, bh, o);
    const float ol = __shfl_xor_sync(kAll, bl, o);
    const int oa = __shfl_xor_sync(kAll, ba, o);
    if (oh < bh || (oh == bh && (ol < bl || (ol == bl && oa < ba)))) {
      bh = oh;
      bl = ol;
      ba = oa;
    }
  }
  if (valid && a == 0) {
    const int sl = lr / P.m;
    b_hi[sl] = bh;
    b_lo[sl] = bl;
    b_arg[sl] = ba;
  }
}

template <int NT, typename VT>
__device__ __forceinline__ void ring_fill(VT* ring, int mask, const VT* __restrict__ src,
                                          int64_t lo, int64_t hi) {
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) ring[i & mask] = src[i];
}

template <int NT>
__device__ __forceinline__ void ring_fill_split(float* ring_hi, float* ring_lo, int mask,
                                                const float2* __restrict__ src, int64_t lo,
                                                int64_t hi) {
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
    const float2 v = src[i];
    ring_hi[i & mask] = v.x;
    ring_lo[i & mask] = v.y;
  }
}

// Bulk prefetch of `bytes` (a multiple of 16) from global memory into L2.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
constexpr int kPrefetchPasses = 2;
// Entries [e0, e1) of the packed array (32-byte groups of 4 entries) into L2.
__device__ __forceinline__ void prefetch_entries_l2(const int32_t* pk, int64_t e0, int64_t e1) {
  const int64_t g0 = e0 >> 2, g1 = (e1 + 3) >> 2;
  prefetch_l2_bulk(pk + g0 * 8, static_cast<unsigned>((g1 - g0) * 32));
}

// Shared memory: the ring (R float2 for the float-float pass; with SCREEN R
// high parts, then R low parts, so that the screen reads 4-byte words; R
// floats for FP32), then the tile: the Q tile q_hi[T*m] (and q_lo[T*m]) of
// the full pass, or with SCREEN each state's winner b_hi[T], b_lo[T], b_arg[T].
template <bool FF, typename IdxT, int VW, int NT, bool SCREEN>
__global__ void __launch_bounds__(NT, FF ? 1 : 2)
    k_bellman_win(Csr<IdxT> P, Grid G, int64_t band, int ring_log2, const void* __restrict__ Vin,
                  void* __restrict__ Vout, int32_t* __restrict__ pi_out,
                  float* __restrict__ r_out, double* __restrict__ partials,
                  DevState* __restrict__ st, int init_gmres) {
  static_assert(!SCREEN || (FF && VW <= 4), "screening is a float-float fast-path form");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  constexpr int NV = NT / VW;
  const int R = 1 << ring_log2;
  const int mask = R - 1;
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* ring_lo = ring + R;                            // SCREEN only
  float2* ring2 = reinterpret_cast<float2*>(smem_raw);  // FF without SCREEN
  const int lane = threadIdx.x % VW;
  const int vec = threadIdx.x / VW;
  const int m = P.m;
  const int T = G.tile_states;
  const int RT = T * m;
  const int QS = qtile_stride(T, m);
  float* q_hi = ring + (FF ? 2 * R : R);
  float* q_lo = q_hi + (SCREEN ? T : m * QS);
  int* b_arg = reinterpret_cast<int*>(q_lo + T);  // SCREEN only
  using GX = typename std::conditional<FF, RingFF, RingF32>::type;
  GX gx;
  if constexpr (FF)
    gx = RingFF{ring2, mask};
  else
    gx = RingF32{ring, mask};
  const bool vec4 = P.vec4 != 0;
  const bool fast = VW <= 4 && P.uniform_len == 4 * VW && vec4 && !P.val_lo;

  double my_max = 0.0, my_sq = 0.0;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  const int64_t row_end = min(t_end * T, P.n) * m;  // end of this CTA's rows
  int64_t pf_e0 = 0, pf_e1 = 0;                      // thread 0: entries to prefetch next
  auto fill = [&](int64_t lo, int64_t hi) {
    if constexpr (SCREEN)
      ring_fill_split<NT>(ring, ring_lo, mask, static_cast<const float2*>(Vin), lo, hi);
    else if constexpr (FF)
      ring_fill<NT>(ring2, mask, static_cast<const float2*>(Vin), lo, hi);
    else
      ring_fill<NT>(ring, mask, static_cast<const float*>(Vin), lo, hi);
  };
  if (t_begin < t_end) {
    const int64_t s_first = t_begin * T;
    fill(max(int64_t(0), s_first - band), min(P.n, s_first + T + band));
  }
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s0 = tile * T;
    const int64_t r0 = s0 * m;
    __syncthreads();  // window of this tile complete; tile area free
    if (tile + 1 < t_end) fill(s0 + T + band, min(P.n, s0 + 2 * T + band));
    const int64_t rows_here = min(static_cast<int64_t>(RT), (P.n - s0) * m);
    if constexpr (SCREEN) {
      for (int base = 0; base < RT; base += NT)
        bellman_pass_screened<VW>(P, ring, ring_lo, mask, r0, base + vec * VW, rows_here, lane,
                                  q_hi, q_lo, b_arg);
    } else if (fast) {
      if constexpr (VW <= 4) {
        for (int base = 0; base < RT; base += NT) {
          // the CTA's rows are one contiguous run of the packed array (a row
          // of 4*VW entries is VW groups of 32 bytes): ask L2 for the rows
          // kPrefetchPasses passes ahead with one bulk prefetch, so that the
          // row loads of those passes find their lines in L2
          if (threadIdx.x == 0) {
            const int64_t pr = r0 + base + kPrefetchPasses * NT;
            const int64_t pe = min(row_end, pr + NT);
            if (pr < pe)
              prefetch_l2_bulk(P.col + pr * 8 * VW, static_cast<unsigned>((pe - pr) * 32 * VW));
          }
          bellman_pass_fast<FF, VW>(P, gx, r0, base + vec * VW, rows_here, lane, QS, q_hi, q_lo);
        }
      }
    } else if (VW == 1) {
      for (int base = 0; base < RT; base += 2 * NT) {
        // rows of other lengths: thread 0 reads the entry bounds of the rows
        // kPrefetchPasses + 1 passes ahead during this pass (the loads overlap
        // it) and prefetches them into L2 at the start of the next
        if (threadIdx.x == 0) {
          if (pf_e1 > pf_e0) prefetch_entries_l2(P.col, pf_e0, pf_e1);
          const int64_t ra = r0 + base + (kPrefetchPasses + 1) * 2 * NT;
          const int64_t rb = min(row_end, ra + 2 * NT);
          pf_e0 = pf_e1 = 0;
          if (ra < rb) {
            int64_t e_dummy;
            row_bounds<IdxT>(P.rp, P.uniform_len, ra, pf_e0, e_dummy);
            row_bounds<IdxT>(P.rp, P.uniform_len, rb - 1, e_dummy, pf_e1);
          }
        }
        bellman_pass_g1x2<FF, IdxT, decltype(gx), true>(P, gx, r0, base + threadIdx.x,
                                                         base + NT + threadIdx.x, rows_here, QS,
                                                         q_hi, q_lo);
      }
    } else
    for (int base = 0; base < RT; base += NV) {
      const int lr = base + vec;
      int64_t b = 0, e = 0;
      if (lr < rows_here) row_bounds<IdxT>(P.rp, P.uniform_len, r0 + lr, b, e);
      float hi, lo = 0.f;
      if constexpr (FF) {
        row_dot_ff<VW>(P.col, P.val, P.val_lo, gx, b, e, lane, vec4, hi, lo);
        group_sum_ff<VW>(hi, lo);
      } else {
        hi = row_dot_f32<VW, float>(P.col, P.val, gx, b, e, lane, vec4);
        hi = group_sum<VW>(hi);
      }
      if (lane == 0 && lr < rows_here) {
        const int a = lr % m;
        const int sl = lr / m;
        const int64_t r = r0 + lr;
        if constexpr (FF) {
          const ff sum = ff_norm(hi, lo);
          const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
          const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
          q_hi[a * QS + sl] = q.hi;
          q_lo[a * QS + sl] = q.lo;
        } else {
          q_hi[a * QS + sl] = fmaf(P.gamma, hi, __ldcs(P.g + r));
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += NT) {
      const int64_t s = s0 + t;
      if (s < P.n) {
        float bh, bl = 0.f;
        int arg = 0;
        if constexpr (SCREEN) {
          bh = q_hi[t];
          bl = q_lo[t];
          arg = b_arg[t];
        } else {
          bh = q_hi[t];
          if (FF) bl = q_lo[t];
          for (int a = 1; a < m; ++a) {
            const float h = q_hi[a * QS + t];
            const float l = FF ? q_lo[a * QS + t] : 0.f;
            if (h < bh || (FF && h == bh && l < bl)) {
              bh = h;
              bl = l;
              arg = a;
            }
          }
        }
        float r;
        if constexpr (SCREEN) {
          r = ff_diff_to_float(bh, bl, ring[s & mask], ring_lo[s & mask]);
          if (Vout) static_cast<float2*>(Vout)[s] = make_float2(bh, bl);
        } else if constexpr (FF) {
          const float2 v = ring2[s & mask];
          r = ff_diff_to_float(bh, bl, v.x, v.y);
          if (Vout) static_cast<float2*>(Vout)[s] = make_float2(bh, bl);
        } else {
          r = bh - ring[s & mask];
          if (Vout) static_cast<float*>(Vout)[s] = bh;
        }
        if (pi_out) pi_out[s] = arg;
        if (r_out) r_out[s] = r;
        const double rd = static_cast<double>(r);
        my_max = fmax(my_max, fabs(rd));
        my_sq += rd * rd;
      }
    }
  }

  const double bmax = block_max_nt<NT>(my_max, red);
  const double bsq = block_sum_nt<NT>(my_sq, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bmax;
    partials[2 * blockIdx.x + 1] = bsq;
  }
  if (last_block(&st->counter[kCntBellman])) {
    double mx = 0.0, sq = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += NT) {
      mx = fmax(mx, __ldcg(partials + 2 * i));
      sq += __ldcg(partials + 2 * i + 1);
    }
    mx = block_max_nt<NT>(mx, red);
    sq = block_sum_nt<NT>(sq, red);
    if (threadIdx.x == 0) {
      st->res_inf = mx;
      st->res_2 = sqrt(sq);
      st->counter[kCntBellman] = 0;
      if (init_gmres) {
        if (st->target_rel) st->target = st->eta * mx;
        gmres_begin(st, sqrt(sq));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Policy residual with the value window in shared memory (banded matrices):
// the ring of k_bellman_win, a CTA walking contiguous tiles of NT states with
// one state per thread, for rows of 4*VW aligned entries in the vector form of
// k_policy_residual_fast (VW states per vector, a reduce-scatter).  The
// float-float row sums are those of the global kernel (same entries, same
// order, same operations).  (Short rows stay on the global kernel: there the
// action-major copy already makes neighbouring gathers hit L1/L2, and a window
// version measured slower, 0.528 against 0.478 ms on the 4096^2 grid.)
// ---------------------------------------------------------------------------
template <typename IdxT, int VW, int NT>
__global__ void __launch_bounds__(NT, 1)
    k_policy_residual_win(Csr<IdxT> P, Grid G, int64_t band, int ring_log2,
                          const int32_t* __restrict__ pi, const float2* __restrict__ V,
                          float* __restrict__ r_out, double* __restrict__ partials,
                          DevState* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  const int R = 1 << ring_log2;
  const int mask = R - 1;
  float2* ring = reinterpret_cast<float2*>(smem_raw);
  const RingFF gx{ring, mask};
  const int T = G.tile_states;  // == NT
  static_assert(VW <= 4, "rows of 4*VW aligned entries");
  const int lane = threadIdx.x % VW;
  double my_max = 0.0, my_sq = 0.0;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  if (t_begin < t_end) {
    const int64_t s_first = t_begin * T;
    ring_fill<NT>(ring, mask, V, max(int64_t(0), s_first - band), min(P.n, s_first + T + band));
  }
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s0 = tile * T;
    __syncthreads();  // window of this tile complete
    if (tile + 1 < t_end) ring_fill<NT>(ring, mask, V, s0 + T + band, min(P.n, s0 + 2 * T + band));
    const int64_t s = s0 + threadIdx.x;
    const bool valid = s < P.n;
    const int32_t a = valid ? __ldg(pi + s) : 0;
    float hi, lo;
    {
      const int64_t rb = policy_row(P, s, a) * P.uniform_len;
      int64_t b[VW];
      bool vd[VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        b[u] = __shfl_sync(0xffffffffu, rb, u, VW);
        vd[u] = __shfl_sync(0xffffffffu, valid ? 1 : 0, u, VW) != 0;
      }
      float ph[VW], pl[VW];
      vec_rows_ff<VW>(P.col, P.val, gx, b, vd, lane, ph, pl);
      reduce_scatter_ff<VW>(ph, pl, lane, hi, lo);
    }
    if (valid) {
      const int64_t r = s * P.m + a;  // cost row
      const ff sum = ff_norm(hi, lo);
      const ff gq = ff_norm(__ldcs(P.g + r), P.g_lo ? __ldcs(P.g_lo + r) : 0.f);
      const ff q = ff_add(ff_mul(sum, ff{P.gamma_hi, P.gamma_lo}), gq);
      const float2 v = ring[s & mask];
      const float rr = ff_diff_to_float(q.hi, q.lo, v.x, v.y);
      r_out[s] = rr;
      const double rd = static_cast<double>(rr);
      my_max = fmax(my_max, fabs(rd));
      my_sq += rd * rd;
    }
  }
  const double bmax = block_max_nt<NT>(my_max, red);
  const double bsq = block_sum_nt<NT>(my_sq, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bmax;
    partials[2 * blockIdx.x + 1] = bsq;
  }
  if (last_block(&st->counter[kCntPolicy])) {
    double mx = 0.0, sq = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += NT) {
      mx = fmax(mx, __ldcg(partials + 2 * i));
      sq += __ldcg(partials + 2 * i + 1);
    }
    mx = block_max_nt<NT>(mx, red);
    sq = block_sum_nt<NT>(sq, red);
    if (threadIdx.x == 0) {
      st->res_inf = mx;
      st->res_2 = sqrt(sq);
      st->counter[kCntPolicy] = 0;
      gmres_begin(st, sqrt(sq));
    }
  }
}

// ---------------------------------------------------------------------------
// BiCGStab (van der Vorst 1992) on (I - gamma P_pi) d = r: the policy SpMV
// y = x - gamma P_pi x over the FP32 probabilities (row s*m + pi(s) read from
// the CSR, or from the action-major copy), with <y, w> and <y, y> reduced in a
// fixed order; the last block turns them into a recurrence scalar:
//   mode 0: y = v = A p, w = r^  ->  alpha = rho / <r^, v>
//   mode 1: y = t = A s, w = s   ->  omega = <t, s> / <t, t>
// A zero or non-finite quotient ends the inner solve (breakdown).
// ---------------------------------------------------------------------------
template <typename IdxT, int VW>
__global__ void __launch_bounds__(kThreads)
    k_bicg_spmv(Csr<IdxT> P, Grid G, const int32_t* __restrict__ pi,
                const float* __restrict__ x, float* __restrict__ y,
                const float* __restrict__ w, int mode, double* __restrict__ partials,
                DevState* __restrict__ st) {
  if (!st->active) return;
  __shared__ double red[kThreads / 32];
  constexpr int NV = kThreads / VW;
  const int lane = threadIdx.x % VW;
  const int vec = threadIdx.x / VW;
  const bool vec4 = P.vec4 != 0;
  double d1 = 0.0, d2 = 0.0;
  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s = tile * NV + vec;
    int64_t b = 0, e = 0;
    if (s < P.n) row_bounds<IdxT>(P.rp, P.uniform_len, policy_row(P, s, __ldg(pi + s)), b, e);
    float acc = row_dot_f32<VW, float, GatherF32>(P.col, P.val, GatherF32{x}, b, e, lane, vec4);
    acc = group_sum<VW>(acc);
    if (lane == 0 && s < P.n) {
      const float yv = fmaf(-P.gamma, acc, x[s]);
      y[s] = yv;
      const double yd = static_cast<double>(yv);
      d1 += yd * static_cast<double>(w[s]);
      d2 += yd * yd;
    }
  }
  const double b1 = block_sum_d(d1, red);
  const double b2 = block_sum_d(d2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b1;
    partials[2 * blockIdx.x + 1] = b2;
  }
  if (last_block(&st->counter[kCntBicg])) {
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kThreads) {
      s1 += __ldcg(partials + 2 * i);
      s2 += __ldcg(partials + 2 * i + 1);
    }
    s1 = block_sum_d(s1, red);
    s2 = block_sum_d(s2, red);
    if (threadIdx.x == 0) {
      st->counter[kCntBicg] = 0;
      const double q = mode == 0 ? st->bicg_rho / s1 : s1 / s2;
      if (!(q != 0.0 && isfinite(q))) {
        st->breakdown = 1;
        st->active = 0;
      } else if (mode == 0) {
        st->bicg_alpha = q;
      } else {
        st->bicg_omega = q;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename IdxT>
static Csr<IdxT> make_csr(const Mat& A) {
  Csr<IdxT> P;
  P.rp = static_cast<const IdxT*>(A.rp);
  P.col = A.col;
  P.val = A.val;
  P.val_lo = A.val_lo;
  P.g = A.g;
  P.g_lo = A.g_lo;
  P.val16 = A.val16;
  P.lpk = A.lpk;
  P.row_scale = A.row_scale;
  P.n = A.n;
  P.m = A.m;
  P.vec4 = A.vec4;
  P.uniform_len = A.uniform_len;
  P.am = 0;
  P.gamma = static_cast<float>(A.gamma);
  P.gamma_hi = static_cast<float>(A.gamma);
  P.gamma_lo = static_cast<float>(A.gamma - static_cast<double>(P.gamma_hi));
  return P;
}

// Blocks resident per SM for a kernel at a given dynamic shared memory size.
template <typename K>
static int occupancy(K kernel, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, smem) != cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

static Grid make_grid(int64_t n_tiles, int max_blocks, int tile_states) {
  Grid G;
  G.tile_states = tile_states;
  G.n_tiles = n_tiles;
  int64_t blocks = n_tiles < max_blocks ? n_tiles : max_blocks;
  if (blocks < 1) blocks = 1;
  G.tiles_per_block = (n_tiles + blocks - 1) / blocks;
  if (G.tiles_per_block < 1) G.tiles_per_block = 1;
  return G;
}

static int64_t n_blocks(const Grid& G) {
  int64_t b = (G.n_tiles + G.tiles_per_block - 1) / G.tiles_per_block;
  return b < 1 ? 1 : b;
}

// Bellman tile: about 1024 rows, at least one state, at most kThreads states.
static int bellman_tile_states(int m) {
  int T = 1024 / m;
  if (T < 1) T = 1;
  if (T > kThreads) T = kThreads;
  return T;
}

// Ring slots needed for band B and tile T (power of two >= 2B + 2T), or 0 when
// the ring would not fit the shared-memory budget.
int window_log2(int64_t band, int T, size_t entry_bytes, size_t budget) {
  const int64_t need = 2 * band + 2 * static_cast<int64_t>(T);
  int lg = 0;
  while ((int64_t(1) << lg) < need) ++lg;
  if ((size_t(1) << lg) * entry_bytes > budget) return 0;
  return lg;
}

template <bool FF, typename IdxT, int VW, int NT, bool SCREEN>
static cudaError_t bellman_win(const Mat& A, int lg, int T, const void* V, void* V_out,
                               int32_t* pi, float* r, double* partials, DevState* st,
                               int init_gmres, cudaStream_t s) {
  const size_t entry = FF ? sizeof(float2) : sizeof(float);
  const size_t tile = SCREEN ? static_cast<size_t>(T) * 12
                             : static_cast<size_t>(qtile_stride(T, A.m)) * A.m * sizeof(float) *
                                   (FF ? 2 : 1);
  const size_t smem = (size_t(1) << lg) * entry + tile;
  auto kern = k_bellman_win<FF, IdxT, VW, NT, SCREEN>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int64_t n_tiles = (A.n + T - 1) / T;
  const Grid G = make_grid(n_tiles, A.num_sms * occ, T);
  Csr<IdxT> P = make_csr<IdxT>(A);
  kern<<<static_cast<unsigned>(n_blocks(G)), NT, smem, s>>>(P, G, A.band, lg, V, V_out, pi, r,
                                                            partials, st, init_gmres);
  return cudaGetLastError();
}

// The FP32 screen applies to float-float backups on the fast path (rows of
// 4*VW aligned entries, FP32 probabilities) when a state's actions fit in
// aligned lanes of one warp (m a power of two up to 32).
static bool screened(const Mat& A, int VW) {
  return A.screen && VW <= 4 && A.uniform_len == 4 * VW && A.vec4 && !A.val_lo && A.m <= 32 &&
         (A.m & (A.m - 1)) == 0;
}

// Ring geometry of the windowed float-float backup: NT threads, T states a tile.
static constexpr int kWinFFThreads = 1024;
// Passes of NT rows per tile: eight for the float-float backup (half the
// barriers and ring refills of four: 0.811 -> 0.755 ms per sweep on the banded
// 4M-state MDP), four for FP32 (eight measured 2% slower there).
static int win_tile(int NT, int m, bool ff) {
  int T = (ff ? 8 : 4) * NT / m;
  if (T < 1) T = 1;
  if (T > NT) T = NT;
  return T;
}

bool bellman_screened(const Mat& A) {
  return A.window && A.vw <= 4 && screened(A, A.vw) &&
         window_log2(A.band, win_tile(kWinFFThreads, A.m, true), 8, 128 * 1024) > 0;
}

template <bool FF, typename IdxT, int VW>
static cudaError_t bellman_vw(const Mat& A, const void* V, void* V_out, int32_t* pi, float* r,
                              double* partials, DevState* st, int init_gmres, cudaStream_t s) {
  if (A.window) {
    // 1024 threads per CTA for the float-float ring (one CTA per SM), 512 for FP32
    constexpr int NT = FF ? kWinFFThreads : 512;
    const int T = win_tile(NT, A.m, FF);
    const int lg = window_log2(A.band, T, FF ? 8 : 4, 128 * 1024);
    // the ring and the Q tile must fit one CTA's shared memory (227 KB)
    const size_t win_smem = (size_t(1) << lg) * (FF ? 8 : 4) +
                            static_cast<size_t>(qtile_stride(T, A.m)) * A.m * (FF ? 8 : 4);
    if (lg > 0 && win_smem <= 227 * 1024) {
      if constexpr (FF && VW <= 4) {
        if (screened(A, VW))
          return bellman_win<FF, IdxT, VW, NT, true>(A, lg, T, V, V_out, pi, r, partials, st,
                                                     init_gmres, s);
      }
      return bellman_win<FF, IdxT, VW, NT, false>(A, lg, T, V, V_out, pi, r, partials, st,
                                                  init_gmres, s);
    }
  }
  const int T = bellman_tile_states(A.m);
  const size_t smem =
      static_cast<size_t>(qtile_stride(T, A.m)) * A.m * sizeof(float) * (FF ? 2 : 1);
  auto kern = k_bellman<FF, IdxT, VW>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
  static int occ = occupancy(kern, smem);
  const int64_t n_tiles = (A.n + T - 1) / T;
  const Grid G = make_grid(n_tiles, A.num_sms * occ, T);
  Csr<IdxT> P = make_csr<IdxT>(A);
  kern<<<static_cast<unsigned>(n_blocks(G)), kThreads, smem, s>>>(P, G, V, V_out, pi, r, partials,
                                                                   st, init_gmres);
  return cudaGetLastError();
}

template <bool FF, typename IdxT>
static cudaError_t bellman_idx(const Mat& A, const void* V, void* V_out, int32_t* pi, float* r,
                               double* partials, DevState* st, int init_gmres, cudaStream_t s) {
  switch (A.vw) {
    case 1: return bellman_vw<FF, IdxT, 1>(A, V, V_out, pi, r, partials, st, init_gmres, s);
    case 2: return bellman_vw<FF, IdxT, 2>(A, V, V_out, pi, r, partials, st, init_gmres, s);
    case 4: return bellman_vw<FF, IdxT, 4>(A, V, V_out, pi, r, partials, st, init_gmres, s);
    case 8: return bellman_vw<FF, IdxT, 8>(A, V, V_out, pi, r, partials, st, init_gmres, s);
    case 16: return bellman_vw<FF, IdxT, 16>(A, V, V_out, pi, r, partials, st, init_gmres, s);
    default: return bellman_vw<FF, IdxT, 32>(A, V, V_out, pi, r, partials, st, init_gmres, s);
  }
}

cudaError_t launch_bellman(const Mat& A, bool ff, const void* V, void* V_out, int32_t* pi,
                           float* r, double* partials, DevState* st, int init_gmres,
                           cudaStream_t s) {
  if (A.idx64) {
    return ff ? bellman_idx<true, int64_t>(A, V, V_out, pi, r, partials, st, init_gmres, s)
              : bellman_idx<false, int64_t>(A, V, V_out, pi, r, partials, st, init_gmres, s);
  }
  return ff ? bellman_idx<true, int32_t>(A, V, V_out, pi, r, partials, st, init_gmres, s)
            : bellman_idx<false, int32_t>(A, V, V_out, pi, r, partials, st, init_gmres, s);
}

template <typename IdxT, int VW>
static cudaError_t presid_vw(const Mat& A, const int32_t* pi, const float2* V, float* r,
                             double* partials, DevState* st, cudaStream_t s) {
  if constexpr (VW <= 4) {
    // banded rows of 4*VW aligned entries: the window of V in shared memory
    const bool fast_rows = A.uniform_len == 4 * VW && A.vec4 && !A.val_lo && A.am_len == 0;
    if (A.window && fast_rows) {
      constexpr int NT = 1024;
      const int lg = window_log2(A.band, NT, 8, 128 * 1024);
      if (lg > 0) {
        auto kern = k_policy_residual_win<IdxT, VW, NT>;
        const size_t smem = (size_t(1) << lg) * sizeof(float2);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
        const Grid G = make_grid((A.n + NT - 1) / NT, A.num_sms, NT);
        Csr<IdxT> P = make_csr<IdxT>(A);
        use_policy_copy(P, A);
        kern<<<static_cast<unsigned>(n_blocks(G)), NT, smem, s>>>(P, G, A.band, lg, pi, V, r,
                                                                  partials, st);
        return cudaGetLastError();
      }
    }
  }
  if constexpr (VW <= 4) {
    if (A.uniform_len == 4 * VW && A.vec4 && !A.val_lo && A.am_len == 0) {
      auto kern = k_policy_residual_fast<IdxT, VW>;
      static int occ = occupancy(kern, 0);
      const Grid G = make_grid((A.n + kThreads - 1) / kThreads, A.num_sms * occ, kThreads);
      Csr<IdxT> P = make_csr<IdxT>(A);
      kern<<<static_cast<unsigned>(n_blocks(G)), kThreads, 0, s>>>(P, G, pi, V, r, partials, st);
      return cudaGetLastError();
    }
  }
  auto kern = k_policy_residual<IdxT, VW>;
  static int occ = occupancy(kern, 0);
  constexpr int NV = kThreads / VW;
  const int64_t n_tiles = (A.n + NV - 1) / NV;
  const Grid G = make_grid(n_tiles, A.num_sms * occ, NV);
  Csr<IdxT> P = make_csr<IdxT>(A);
  use_policy_copy(P, A);
  kern<<<static_cast<unsigned>(n_blocks(G)), kThreads, 0, s>>>(P, G, pi, V, r, partials, st);
  return cudaGetLastError();
}

template <typename IdxT>
static cudaError_t presid_idx(const Mat& A, const int32_t* pi, const float2* V, float* r,
                              double* partials, DevState* st, cudaStream_t s) {
  switch (A.vw) {
    case 1: return presid_vw<IdxT, 1>(A, pi, V, r, partials, st, s);
    case 2: return presid_vw<IdxT, 2>(A, pi, V, r, partials, st, s);
    case 4: return presid_vw<IdxT, 4>(A, pi, V, r, partials, st, s);
    case 8: return presid_vw<IdxT, 8>(A, pi, V, r, partials, st, s);
    case 16: return presid_vw<IdxT, 16>(A, pi, V, r, partials, st, s);
    default: return presid_vw<IdxT, 32>(A, pi, V, r, partials, st, s);
  }
}

cudaError_t launch_policy_residual(const Mat& A, const int32_t* pi, const float2* V, float* r,
                                   double* partials, DevState* st, cudaStream_t s) {
  return A.idx64 ? presid_idx<int64_t>(A, pi, V, r, partials, st, s)
                 : presid_idx<int32_t>(A, pi, V, r, partials, st, s);
}

template <typename IdxT, int VW>
static cudaError_t bicg_vw(const Mat& A, const int32_t* pi, const float* x, float* y,
                           const float* w, int mode, double* partials, DevState* st,
                           cudaStream_t s) {
  auto kern = k_bicg_spmv<IdxT, VW>;
  static int occ = occupancy(kern, 0);
  constexpr int NV = kThreads / VW;
  const int64_t n_tiles = (A.n + NV - 1) / NV;
  const Grid G = make_grid(n_tiles, A.num_sms * occ, NV);
  Csr<IdxT> P = make_csr<IdxT>(A);
  use_policy_copy(P, A);
  kern<<<static_cast<unsigned>(n_blocks(G)), kThreads, 0, s>>>(P, G, pi, x, y, w, mode, partials,
                                                               st);
  return cudaGetLastError();
}

template <typename IdxT>
static cudaError_t bicg_idx(const Mat& A, const int32_t* pi, const float* x, float* y,
                            const float* w, int mode, double* partials, DevState* st,
                            cudaStream_t s) {
  switch (A.vw) {
    case 1: return bicg_vw<IdxT, 1>(A, pi, x, y, w, mode, partials, st, s);
    case 2: return bicg_vw<IdxT, 2>(A, pi, x, y, w, mode, partials, st, s);
    case 4: return bicg_vw<IdxT, 4>(A, pi, x, y, w, mode, partials, st, s);
    case 8: return bicg_vw<IdxT, 8>(A, pi, x, y, w, mode, partials, st, s);
    case 16: return bicg_vw<IdxT, 16>(A, pi, x, y, w, mode, partials, st, s);
    default: return bicg_vw<IdxT, 32>(A, pi, x, y, w, mode, partials, st, s);
  }
}

cudaError_t launch_bicg_spmv(const Mat& A, const int32_t* pi, const float* x, float* y,
                             const float* w, int mode, double* partials, DevState* st,
                             cudaStream_t s) {
  return A.idx64 ? bicg_idx<int64_t>(A, pi, x, y, w, mode, partials, st, s)
                 : bicg_idx<int32_t>(A, pi, x, y, w, mode, partials, st, s);
}

}  // namespace mdpk
