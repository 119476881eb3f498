// K2: Arnoldi step j of GMRES on (I - gamma P_pi) -- the policy-row SpMV
// w = v_j - gamma P_pi v_j, gathering row s*m + pi(s) straight from the full
// CSR (no reassembly of P_pi), fused with the classical Gram-Schmidt dot
// products h_i = <w, v_i>, i <= j (Saad 2003, Alg. 6.9 with CGS).
//
// Tile = 4*NT states.  Phase A writes w for the tile straight to global
// memory.  Fast path (rows of exactly 4*VW entries, 16-byte aligned): a
// vector of VW lanes owns VW consecutive states, each lane loads its 16-byte
// slice of all VW policy rows before any gather (VW rows in flight per lane),
// and a reduce-scatter leaves every lane with its own state's row sum.
// Banded matrices gather v_j from a shared-memory ring window (see
// k_bellman.cu).  Phase B (after a block barrier): thread t owns states
// 4t..4t+3 of the tile and streams each basis vector once as float4; every
// warp reduces its partial dot with shuffles and accumulates it per warp in
// shared memory; the block's FP64 partials are reduced in a fixed order by the
// last block.  Included by one translation unit per probability type.
#pragma once

#include "k_rows.cuh"
#include "launch.h"

namespace mdpk {

template <int MAXB, int NT>
__device__ __forceinline__ void publish_dots_nt(int j, double* partials,
                                                const float (*wacc)[MAXB]) {
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += NT) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += static_cast<double>(wacc[k][i]);
    partials[static_cast<int64_t>(blockIdx.x) * MAXB + i] = s;
  }
}

// Last block: h_i = scale_i * sum over blocks of partial i, for i <= j.  Warp w
// reduces dots i = w, w + NT/32, ...: its lanes stride over the blocks and a
// fixed shuffle tree combines them (deterministic, no serial chain of loads).
template <int MAXB, int NT>
__device__ __forceinline__ void reduce_dots_nt(const double* partials, int j, double* out,
                                               const double* scale) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = static_cast<int>(gridDim.x);
  for (int i = warp; i <= j; i += NT / 32) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(partials + static_cast<int64_t>(b) * MAXB + i);
    s = warp_sum_d(s);
    if (lane == 0) out[i] = s * scale[i];
  }
}

template <int NT>
__device__ __forceinline__ void ring_fill_f32(float* ring, int mask, const float* __restrict__ src,
                                              int64_t lo, int64_t hi) {
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) ring[i & mask] = src[i];
}

// SPMV && DOTS: fused step; SPMV only: w into u_{j+1}; DOTS only: h_i = <u_{j+1}, v_i>
// into H(:, j) (out_h2 == 0) or into st->h2 (second Gram-Schmidt pass).
template <typename IdxT, int VW, typename PV, int MAXB, bool SPMV, bool DOTS, int NT, bool WIN>
__global__ void __launch_bounds__(NT, (NT == 512 ? 3 : 1))
    k_arnoldi_spmv(Csr<IdxT> P, Grid G, int64_t band, int ring_log2,
                   const int32_t* __restrict__ pi, float* __restrict__ basis, int64_t ld, int j,
                   int out_h2, double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  constexpr int TS = 4 * NT;  // states per tile (four passes of NT states)
  constexpr int NV = NT / VW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float wacc[NT / 32][MAXB];
  const int lane = threadIdx.x % VW;
  const int vec = threadIdx.x / VW;
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const bool vec4 = P.vec4 != 0;
  const float* uj = basis + static_cast<int64_t>(j) * ld;
  float* uw = basis + static_cast<int64_t>(j + 1) * ld;
  const float sj = static_cast<float>(st->scale[j]);
  const PV* val = SPMV ? (sizeof(PV) == 4 ? reinterpret_cast<const PV*>(P.val)
                                          : static_cast<const PV*>(P.val16))
                       : nullptr;
  const bool lp = sizeof(PV) != 4;
  float* ring = reinterpret_cast<float*>(smem_raw);
  const int mask = (1 << ring_log2) - 1;
  for (int i = threadIdx.x; i < (NT / 32) * MAXB; i += NT) (&wacc[0][0])[i] = 0.f;

  const int64_t t_begin = static_cast<int64_t>(blockIdx.x) * G.tiles_per_block;
  const int64_t t_end = min(G.n_tiles, t_begin + G.tiles_per_block);
  if (WIN && SPMV && t_begin < t_end) {
    const int64_t sf = t_begin * TS;
    ring_fill_f32<NT>(ring, mask, uj, max(int64_t(0), sf - band), min(P.n, sf + TS + band));
  }
  __syncthreads();
  // fast path: every row holds 4*VW entries, 16-byte aligned; a vector of VW
  // lanes owns VW consecutive states and each lane loads its slice of all VW
  // policy rows before any gather, then a reduce-scatter gives each lane the
  // row sum of its own state
  const bool fast = VW <= 4 && P.uniform_len == 4 * VW && vec4;
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const int64_t s0 = tile * TS;
    if constexpr (SPMV) {
      if (WIN && tile + 1 < t_end)  // next tile's leading edge; disjoint from live slots
        ring_fill_f32<NT>(ring, mask, uj, s0 + TS + band, min(P.n, s0 + 2 * TS + band));
      auto phase_a = [&](auto gx, auto xs) {
        if (fast) {
          if constexpr (VW <= 4) {
            int32_t act[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int64_t s = s0 + p * NT + threadIdx.x;
              act[p] = s < P.n ? __ldg(pi + s) : 0;
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int64_t s = s0 + p * NT + threadIdx.x;
              const bool valid = s < P.n;
              const int64_t r = s * P.m + act[p];
              const int64_t rb = r * P.uniform_len;
              int64_t b[VW];
              bool vd[VW];
#pragma unroll
              for (int u = 0; u < VW; ++u) {
                b[u] = __shfl_sync(0xffffffffu, rb, u, VW);
                vd[u] = __shfl_sync(0xffffffffu, valid ? 1 : 0, u, VW) != 0;
              }
              float part[VW];
              bool packed = false;
              float d = 0.f;
              if constexpr (sizeof(PV) == 2) {
                if (P.lpk) {
                  int64_t srow[VW];
                  float den[VW];
#pragma unroll
                  for (int u = 0; u < VW; ++u) srow[u] = s - lane + u;
                  vec_rows_lp<VW, PV>(P.lpk, gx, b, srow, vd, lane, part, den);
                  d = reduce_scatter<VW>(part, lane);
                  const float dd = reduce_scatter<VW>(den, lane);
                  d = dd > 0.f ? d / dd : 0.f;
                  packed = true;
                } else {
                  vec_rows_f32<VW, PV>(P.col, val, gx, b, vd, lane, part);
                }
              } else {
                vec_rows_f32<VW, PV>(P.col, val, gx, b, vd, lane, part);
              }
              if (!packed) d = reduce_scatter<VW>(part, lane);
              if (valid) {
                if (lp && !packed) d *= __ldcs(P.row_scale + r);
                uw[s] = sj * fmaf(-P.gamma, d, xs(s));
              }
            }
          }
        } else if (sizeof(PV) == 2 && P.lpk) {
          // packed 16-bit copy: lanes stride over the 16-byte groups of a row
          for (int base = 0; base < TS; base += NV) {
            const int64_t s = s0 + base + vec;
            int64_t b = 0, e = 0, r = 0;
            if (s < P.n) {
              r = s * P.m + __ldg(pi + s);
              row_bounds<IdxT>(P.rp, P.uniform_len, r, b, e);
            }
            float num = 0.f, den = 0.f;
            if constexpr (sizeof(PV) == 2) row_dot_lp<VW, PV>(P.lpk, gx, s, b, e, lane, num, den);
            num = group_sum<VW>(num);
            den = group_sum<VW>(den);
            if (lane == 0 && s < P.n) {
              const float d = den > 0.f ? num / den : 0.f;
              uw[s] = sj * fmaf(-P.gamma, d, xs(s));
            }
          }
        } else if (VW == 1) {
          // short rows: two states per thread with the actions, row pointers and
          // first two packed groups of both rows in flight together
          int32_t act[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int64_t s = s0 + p * NT + threadIdx.x;
            act[p] = s < P.n ? __ldg(pi + s) : 0;
          }
#pragma unroll
          for (int p = 0; p < 4; p += 2) {
            int64_t s2[2], r2[2];
            RowPre<PV> R[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              s2[u] = s0 + (p + u) * NT + threadIdx.x;
              int64_t b = 0, e = 0;
              r2[u] = s2[u] * P.m + act[p + u];
              if (s2[u] < P.n) row_bounds<IdxT>(P.rp, P.uniform_len, r2[u], b, e);
              row_pre<PV>(P.col, val, b, e, R[u]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if (s2[u] < P.n) {
                float d = row_pre_dot<PV>(P.col, val, gx, R[u]);
                if (lp) d *= __ldcs(P.row_scale + r2[u]);
                uw[s2[u]] = sj * fmaf(-P.gamma, d, xs(s2[u]));
              }
            }
          }
        } else {
          for (int base = 0; base < TS; base += NV) {
            const int64_t s = s0 + base + vec;
            int64_t b = 0, e = 0, r = 0;
            if (s < P.n) {
              r = s * P.m + __ldg(pi + s);
              row_bounds<IdxT>(P.rp, P.uniform_len, r, b, e);
            }
            float d = row_dot_f32<VW, PV>(P.col, val, gx, b, e, lane, vec4);
            d = group_sum<VW>(d);
            if (lane == 0 && s < P.n) {
              if (lp) d *= __ldcs(P.row_scale + r);
              uw[s] = sj * fmaf(-P.gamma, d, xs(s));
            }
          }
        }
      };
      if constexpr (WIN) {
        phase_a(RingF32{ring, mask}, [&](int64_t s) { return ring[s & mask]; });
      } else {
        phase_a(GatherF32{uj}, [&](int64_t s) { return uj[s]; });
      }
      __syncthreads();  // the tile's w (global) visible to the block; ring edge complete
    }
    if constexpr (!DOTS) continue;
    // phase B: thread t owns states s0 + 4t .. s0 + 4t + 3
    const int64_t sq = s0 + 4 * threadIdx.x;
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool full = sq + 3 < P.n;
    if (full) {
      w = *reinterpret_cast<const float4*>(uw + sq);
    } else if (sq < P.n) {
      w.x = uw[sq];
      if (sq + 1 < P.n) w.y = uw[sq + 1];
      if (sq + 2 < P.n) w.z = uw[sq + 2];
    }
#pragma unroll 4
    for (int i = 0; i <= j; ++i) {
      const float* bi = basis + static_cast<int64_t>(i) * ld;
      float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (full) {
        b4 = *reinterpret_cast<const float4*>(bi + sq);
      } else if (sq < P.n) {
        b4.x = bi[sq];
        if (sq + 1 < P.n) b4.y = bi[sq + 1];
        if (sq + 2 < P.n) b4.z = bi[sq + 2];
      }
      float p = fmaf(w.x, b4.x, fmaf(w.y, b4.y, fmaf(w.z, b4.z, w.w * b4.w)));
      p = warp_sum(p);
      if (wl == 0) wacc[warp][i] += p;
    }
  }
  if constexpr (DOTS) {
    publish_dots_nt<MAXB, NT>(j, partials, wacc);
    const unsigned cnt = out_h2 ? kCntDots2 : kCntDots;
    if (last_block(&st->counter[cnt])) {
      double* out = out_h2 ? st->h2 : st->H + static_cast<int64_t>(j) * kMaxBasis;
      reduce_dots_nt<MAXB, NT>(partials, j, out, st->scale);
      if (threadIdx.x == 0) st->counter[cnt] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <typename IdxT>
inline Csr<IdxT> csr_view(const Mat& A) {
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
  P.gamma = static_cast<float>(A.gamma);
  P.gamma_hi = P.gamma;
  P.gamma_lo = static_cast<float>(A.gamma - static_cast<double>(P.gamma));
  return P;
}

inline Grid tiles_grid(int64_t n_tiles, int max_blocks, int tile_states) {
  Grid G;
  G.tile_states = tile_states;
  G.n_tiles = n_tiles;
  int64_t blocks = n_tiles < max_blocks ? n_tiles : max_blocks;
  if (blocks < 1) blocks = 1;
  G.tiles_per_block = (n_tiles + blocks - 1) / blocks;
  if (G.tiles_per_block < 1) G.tiles_per_block = 1;
  return G;
}

inline int64_t tiles_blocks(const Grid& G) {
  int64_t b = (G.n_tiles + G.tiles_per_block - 1) / G.tiles_per_block;
  return b < 1 ? 1 : b;
}

// Power-of-two ring size >= 2*band + 2*tile, or 0 when it exceeds `budget` bytes.
inline int ring_log2_for(int64_t band, int64_t tile, size_t entry, size_t budget) {
  const int64_t need = 2 * band + 2 * tile;
  int lg = 0;
  while ((int64_t(1) << lg) < need) ++lg;
  if ((size_t(1) << lg) * entry > budget) return 0;
  return lg;
}

template <typename IdxT, int VW, typename PV, int MAXB, bool SPMV, bool DOTS, int NT, bool WIN>
cudaError_t spmv_launch(const Mat& A, const int32_t* pi, float* basis, int64_t ld, int j,
                        int out_h2, int lg, double* partials, DevState* st, cudaStream_t s) {
  auto kern = k_arnoldi_spmv<IdxT, VW, PV, MAXB, SPMV, DOTS, NT, WIN>;
  const size_t smem = WIN ? (size_t(1) << lg) * sizeof(float) : 0;
  if (smem > 0)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  constexpr int TS = 4 * NT;
  const Grid G = tiles_grid((A.n + TS - 1) / TS, A.num_sms * occ, TS);
  kern<<<static_cast<unsigned>(tiles_blocks(G)), NT, smem, s>>>(
      csr_view<IdxT>(A), G, A.band, lg, pi, basis, ld, j, out_h2, partials, st);
  return cudaGetLastError();
}

// SpMV only (w into u_{j+1}); the ring window for banded matrices.
template <typename IdxT, int VW, typename PV>
cudaError_t spmv_only(const Mat& A, const int32_t* pi, float* basis, int64_t ld, int j,
                      double* partials, DevState* st, cudaStream_t s) {
  if (A.window) {
    constexpr int NT = 512;
    const int lg = ring_log2_for(A.band, 4 * NT, sizeof(float), 64 * 1024);
    if (lg > 0)
      return spmv_launch<IdxT, VW, PV, 2, true, false, NT, true>(A, pi, basis, ld, j, 0, lg,
                                                                  partials, st, s);
  }
  return spmv_launch<IdxT, VW, PV, 2, true, false, 256, false>(A, pi, basis, ld, j, 0, 0,
                                                                partials, st, s);
}

// Lanes per row are 2, 4, 8 or 32 (the create-time choice is rounded to these).
template <typename IdxT, typename PV>
cudaError_t spmv_vw(const Mat& A, const int32_t* pi, float* basis, int64_t ld, int j,
                    double* partials, DevState* st, cudaStream_t s) {
  switch (A.vw) {
    case 1: return spmv_only<IdxT, 1, PV>(A, pi, basis, ld, j, partials, st, s);
    case 2: return spmv_only<IdxT, 2, PV>(A, pi, basis, ld, j, partials, st, s);
    case 4: return spmv_only<IdxT, 4, PV>(A, pi, basis, ld, j, partials, st, s);
    case 8:
    case 16: return spmv_only<IdxT, 8, PV>(A, pi, basis, ld, j, partials, st, s);
    default: return spmv_only<IdxT, 32, PV>(A, pi, basis, ld, j, partials, st, s);
  }
}

template <typename PV>
cudaError_t spmv_entry(const Mat& A, const int32_t* pi, float* basis, int64_t ld, int j,
                       double* partials, DevState* st, cudaStream_t s) {
  return A.idx64 ? spmv_vw<int64_t, PV>(A, pi, basis, ld, j, partials, st, s)
                 : spmv_vw<int32_t, PV>(A, pi, basis, ld, j, partials, st, s);
}

}  // namespace mdpk
