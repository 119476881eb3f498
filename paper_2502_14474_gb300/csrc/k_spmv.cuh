// K2: Arnoldi step j of GMRES on (I - gamma P_pi) -- the policy-row SpMV
// w = v_j - gamma P_pi v_j, gathering row s*m + pi(s) straight from the full
// CSR (no reassembly of P_pi) (Saad 2003, Alg. 6.9; the Gram-Schmidt dots and
// the orthogonalisation are separate streaming kernels, k_dots.cuh and
// k_gmres.cu).
//
// Work split: block b owns the contiguous states [b*S, (b+1)*S), S a multiple
// of 32 chosen so that every resident block gets the same share (no block
// owns a whole tile more than another), and walks them in tiles of 4*NT
// states (four passes of NT states).  Fast path (rows of exactly 4*VW
// entries, 16-byte aligned): a vector of VW lanes owns VW consecutive states,
// each lane loads its 16-byte slice of all VW policy rows before any gather
// (VW rows in flight per lane), and a reduce-scatter leaves every lane with
// its own state's row sum.  Banded matrices gather v_j from a shared-memory
// ring window (see k_bellman.cu).  Included by one translation unit per
// probability type.
#pragma once

#include "k_rows.cuh"
#include "launch.h"

namespace mdpk {

template <int NT>
__device__ __forceinline__ void ring_fill_f32(float* ring, int mask, const float* __restrict__ src,
                                              int64_t lo, int64_t hi) {
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) ring[i & mask] = src[i];
}

// RICH: the same policy-row product as a Richardson sweep of the correction
// system (modified policy iteration): xout = r + gamma P_pi xin, with
// ||xout - xin||_2 reduced in a fixed order into st->res_2 by the last block,
// st->jdone counting the sweeps that ran and st->active cleared once the
// residual meets st->target (later sweeps of the batch return at once).
// Otherwise xin = u_j, xout = scale_j (cdiag u_j - gamma P_pi u_j): with
// cdiag = 1 that is u_{j+1} = A v_j of the Arnoldi process, with cdiag = 0 the
// next vector (A - I) v_j = -gamma P_pi v_j of an s-step block's monomial basis.
template <typename IdxT, int VW, typename PV, int NT, bool WIN, bool RICH>
__global__ void __launch_bounds__(NT, (NT == 512 ? 2 : 1))
    k_arnoldi_spmv(Csr<IdxT> P, int64_t states_per_block, int64_t band, int ring_log2,
                   const int32_t* __restrict__ pi, const float* __restrict__ xin,
                   float* __restrict__ xout, int j, float cdiag, const float* __restrict__ rvec,
                   double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  constexpr int TS = 4 * NT;  // states per tile (four passes of NT states)
  constexpr int NV = NT / VW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % VW;
  const int vec = threadIdx.x / VW;
  const bool vec4 = P.vec4 != 0;
  const float* uj = xin;
  float* uw = xout;
  const float sj = RICH ? 1.f : static_cast<float>(st->scale[j]);
  double racc = 0.0;  // RICH: this thread's part of ||xout - xin||^2
  // the result of state s from its row product d and its own input xv
  auto emit = [&](int64_t s, float d, float xv) {
    if constexpr (RICH) {
      const float v = fmaf(P.gamma, d, rvec[s]);
      uw[s] = v;
      const double df = static_cast<double>(v - xv);
      racc += df * df;
    } else {
      uw[s] = sj * fmaf(-P.gamma, d, cdiag * xv);
    }
  };
  const PV* val = sizeof(PV) == 4 ? reinterpret_cast<const PV*>(P.val)
                                  : static_cast<const PV*>(P.val16);
  const bool lp = sizeof(PV) != 4;
  float* ring = reinterpret_cast<float*>(smem_raw);
  const int mask = (1 << ring_log2) - 1;

  const int64_t s_begin = static_cast<int64_t>(blockIdx.x) * states_per_block;
  const int64_t s_end = min(P.n, s_begin + states_per_block);
  if (WIN && s_begin < s_end)
    ring_fill_f32<NT>(ring, mask, uj, max(int64_t(0), s_begin - band),
                      min(P.n, s_begin + TS + band));
  __syncthreads();
  // fast path: every row holds 4*VW entries, 16-byte aligned; a vector of VW
  // lanes owns VW consecutive states and each lane loads its slice of all VW
  // policy rows before any gather, then a reduce-scatter gives each lane the
  // row sum of its own state
  const bool fast = VW <= 4 && P.uniform_len == 4 * VW && vec4;
  // The branches that take a thread's four states s0 + p*NT + t at once (the
  // fast path and the one-thread-per-row branches) read their actions one tile
  // ahead: the action load is then off the tile's dependent chain (action,
  // row, gather).
  const bool ahead = fast || VW == 1;
  int32_t act_nx[4] = {0, 0, 0, 0};
  auto load_act = [&](int64_t t0, int32_t(&a)[4]) {
    const int64_t lim = min(s_end, t0 + TS);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t s = t0 + p * NT + threadIdx.x;
      a[p] = s < lim ? __ldg(pi + s) : 0;
    }
  };
  if (ahead && s_begin < s_end) load_act(s_begin, act_nx);
  for (int64_t s0 = s_begin; s0 < s_end; s0 += TS) {
    const int64_t s_lim = min(s_end, s0 + TS);  // states of this tile: [s0, s_lim)
    int32_t act[4] = {act_nx[0], act_nx[1], act_nx[2], act_nx[3]};
    if (ahead && s0 + TS < s_end) load_act(s0 + TS, act_nx);
    {
      if (WIN && s0 + TS < s_end)  // next tile's leading edge; disjoint from live slots
        ring_fill_f32<NT>(ring, mask, uj, s0 + TS + band, min(P.n, s0 + 2 * TS + band));
      auto phase_a = [&](auto gx, auto xs) {
        if (fast) {
          if constexpr (VW <= 4) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int64_t s = s0 + p * NT + threadIdx.x;
              const bool valid = s < s_lim;
              const int64_t r = policy_row(P, s, act[p]);
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
                emit(s, d, xs(s));
              }
            }
          }
        } else if (VW == 1 && sizeof(PV) == 2 && P.lpk) {
          // packed 16-bit copy, short rows: two of a thread's four states at a
          // time have the first two groups of their rows in flight together (a
          // row of up to 5 entries spans at most two groups; longer rows load
          // the rest on the way); two, not four, to stay within 64 registers
          if constexpr (VW == 1 && sizeof(PV) == 2) {
#pragma unroll
            for (int p0 = 0; p0 < 4; p0 += 2) {
              int32_t oe[2];  // (row start & 3) | (row end - row start) << 2
              uint4 G0[2], G1[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int64_t s = s0 + (p0 + u) * NT + threadIdx.x;
                int64_t b = 0, e = 0;
                if (s < s_lim)
                  row_bounds<IdxT>(P.rp, P.uniform_len, policy_row(P, s, act[p0 + u]), b, e);
                const int32_t o = static_cast<int32_t>(b & 3), len = static_cast<int32_t>(e - b);
                oe[u] = o | (len << 2);
                G0[u] = len > 0 ? __ldcs(P.lpk + (b >> 2)) : make_uint4(0, 0, 0, 0);
                G1[u] = o + len > 4 ? __ldcs(P.lpk + (b >> 2) + 1) : make_uint4(0, 0, 0, 0);
              }
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int64_t s = s0 + (p0 + u) * NT + threadIdx.x;
                if (s < s_lim) {
                  const int32_t o = oe[u] & 3, len = oe[u] >> 2;
                  float num = 0.f, den = 0.f;
                  lp_group_dot_rel<PV>(G0[u], o, o + len, s, gx, num, den);
                  lp_group_dot_rel<PV>(G1[u], o - 4, o + len - 4, s, gx, num, den);
                  if (o + len > 8) {  // rows longer than two groups: the rest on the way
                    int64_t b = 0, e = 0;
                    row_bounds<IdxT>(P.rp, P.uniform_len, policy_row(P, s, act[p0 + u]), b, e);
                    for (int32_t k = 8; k < o + len; k += 4)
                      lp_group_dot_rel<PV>(__ldcs(P.lpk + (b >> 2) + (k >> 2)), o - k,
                                           o + len - k, s, gx, num, den);
                  }
                  const float d = den > 0.f ? __fdividef(num, den) : 0.f;
                  emit(s, d, xs(s));
                }
              }
            }
          }
        } else if (sizeof(PV) == 2 && P.lpk) {
          // packed 16-bit copy: lanes stride over the 16-byte groups of a row
          for (int base = 0; base < TS; base += NV) {
            const int64_t s = s0 + base + vec;
            int64_t b = 0, e = 0, r = 0;
            if (s < s_lim) {
              r = policy_row(P, s, __ldg(pi + s));
              row_bounds<IdxT>(P.rp, P.uniform_len, r, b, e);
            }
            float num = 0.f, den = 0.f;
            if constexpr (sizeof(PV) == 2) row_dot_lp<VW, PV>(P.lpk, gx, s, b, e, lane, num, den);
            num = group_sum<VW>(num);
            den = group_sum<VW>(den);
            if (lane == 0 && s < s_lim) {
              const float d = den > 0.f ? num / den : 0.f;
              emit(s, d, xs(s));
            }
          }
        } else if (VW == 1) {
          if constexpr (VW == 1 && sizeof(PV) == 2) {
            // unpacked 16-bit copy (bands too wide for the packed one): one row
            // at a time, so that this rare branch does not raise the register
            // budget of the packed branch compiled into the same kernel
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int64_t s = s0 + p * NT + threadIdx.x;
              if (s < s_lim) {
                int64_t b = 0, e = 0;
                const int64_t r = policy_row(P, s, act[p]);
                row_bounds<IdxT>(P.rp, P.uniform_len, r, b, e);
                float d = row_dot_f32<1, PV>(P.col, val, gx, b, e, 0, vec4);
                d *= __ldcs(P.row_scale + r);
                emit(s, d, xs(s));
              }
            }
          } else if constexpr (VW == 1) {
            // short rows: two states per thread with the actions, row pointers and
            // first two packed groups of both rows in flight together
#pragma unroll
            for (int p = 0; p < 4; p += 2) {
              int64_t s2[2], r2[2];
              RowPre<PV> R[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                s2[u] = s0 + (p + u) * NT + threadIdx.x;
                int64_t b = 0, e = 0;
                r2[u] = policy_row(P, s2[u], act[p + u]);
                if (s2[u] < s_lim) row_bounds<IdxT>(P.rp, P.uniform_len, r2[u], b, e);
                row_pre<PV>(P.col, val, b, e, R[u]);
              }
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                if (s2[u] < s_lim) {
                  float d = row_pre_dot<PV>(P.col, val, gx, R[u]);
                  if (lp) d *= __ldcs(P.row_scale + r2[u]);
                  emit(s2[u], d, xs(s2[u]));
                }
              }
            }
          }
        } else {
          for (int base = 0; base < TS; base += NV) {
            const int64_t s = s0 + base + vec;
            int64_t b = 0, e = 0, r = 0;
            if (s < s_lim) {
              r = policy_row(P, s, __ldg(pi + s));
              row_bounds<IdxT>(P.rp, P.uniform_len, r, b, e);
            }
            float d = row_dot_f32<VW, PV>(P.col, val, gx, b, e, lane, vec4);
            d = group_sum<VW>(d);
            if (lane == 0 && s < s_lim) {
              if (lp) d *= __ldcs(P.row_scale + r);
              emit(s, d, xs(s));
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
  }
  if constexpr (RICH) {
    __shared__ double red[NT / 32];
    const double bs = block_sum_nt<NT>(racc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    if (last_block(&st->counter[kCntMisc])) {
      double sq = 0.0;
      for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += NT)
        sq += __ldcg(partials + b);
      sq = block_sum_nt<NT>(sq, red);
      if (threadIdx.x == 0) {
        st->counter[kCntMisc] = 0;
        st->res_2 = sqrt(sq);
        st->jdone += 1;
        if (!(st->res_2 > st->target)) st->active = 0;
      }
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
  use_policy_copy(P, A);
  return P;
}

// Power-of-two ring size >= 2*band + 2*tile, or 0 when it exceeds `budget` bytes.
inline int ring_log2_for(int64_t band, int64_t tile, size_t entry, size_t budget) {
  const int64_t need = 2 * band + 2 * tile;
  int lg = 0;
  while ((int64_t(1) << lg) < need) ++lg;
  if ((size_t(1) << lg) * entry > budget) return 0;
  return lg;
}

// States per block: the smallest multiple of 32 that covers n with at most
// max_blocks blocks, so every resident block gets (nearly) the same share.
inline int64_t balanced_states_per_block(int64_t n, int64_t max_blocks) {
  if (max_blocks < 1) max_blocks = 1;
  int64_t per = (n + max_blocks - 1) / max_blocks;
  per = (per + 31) / 32 * 32;
  return per < 32 ? 32 : per;
}

// One launch of the policy-row kernel: xin/xout are u_j/u_{j+1} of the GMRES
// basis (RICH false) or the two Richardson iterates (RICH true, with the
// right-hand side rvec and one partial per block in `partials`).
struct SpmvArgs {
  const float* xin;
  float* xout;
  int j;
  const float* rvec;
  double* partials;
  float cdiag;
};

template <typename IdxT, int VW, typename PV, int NT, bool WIN, bool RICH>
cudaError_t spmv_launch(const Mat& A, const int32_t* pi, const SpmvArgs& a, int lg, DevState* st,
                        cudaStream_t s) {
  auto kern = k_arnoldi_spmv<IdxT, VW, PV, NT, WIN, RICH>;
  const size_t smem = WIN ? (size_t(1) << lg) * sizeof(float) : 0;
  if (smem > 0)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  // at most num_sms * 8 blocks (one Richardson partial each fits the partials
  // buffer), and at least NT states per block: a small matrix gets fewer blocks
  // with every thread busy, which leaves room for other streams' kernels
  const int64_t cap = static_cast<int64_t>(A.num_sms) * (occ < 8 ? occ : 8);
  int64_t per = balanced_states_per_block(A.n, cap);
  if (per < NT) per = NT;
  const int64_t blocks = (A.n + per - 1) / per;
  kern<<<static_cast<unsigned>(blocks < 1 ? 1 : blocks), NT, smem, s>>>(
      csr_view<IdxT>(A), per, A.band, lg, pi, a.xin, a.xout, a.j, a.cdiag, a.rvec, a.partials,
      st);
  return cudaGetLastError();
}

// The ring window for banded matrices, else gathers through L1/L2.
template <typename IdxT, int VW, typename PV, bool RICH>
cudaError_t spmv_only(const Mat& A, const int32_t* pi, const SpmvArgs& a, DevState* st,
                      cudaStream_t s) {
  if (A.window) {
    constexpr int NT = 512;
    const int lg = ring_log2_for(A.band, 4 * NT, sizeof(float), 64 * 1024);
    if (lg > 0) return spmv_launch<IdxT, VW, PV, NT, true, RICH>(A, pi, a, lg, st, s);
  }
  return spmv_launch<IdxT, VW, PV, 256, false, RICH>(A, pi, a, 0, st, s);
}

// Lanes per row are 1, 2, 4, 8 or 32 (the create-time choice is rounded to these).
template <typename IdxT, typename PV, bool RICH>
cudaError_t spmv_vw(const Mat& A, const int32_t* pi, const SpmvArgs& a, DevState* st,
                    cudaStream_t s) {
  switch (A.vw) {
    case 1: return spmv_only<IdxT, 1, PV, RICH>(A, pi, a, st, s);
    case 2: return spmv_only<IdxT, 2, PV, RICH>(A, pi, a, st, s);
    case 4: return spmv_only<IdxT, 4, PV, RICH>(A, pi, a, st, s);
    case 8:
    case 16: return spmv_only<IdxT, 8, PV, RICH>(A, pi, a, st, s);
    default: return spmv_only<IdxT, 32, PV, RICH>(A, pi, a, st, s);
  }
}

template <typename PV, bool RICH>
cudaError_t spmv_entry(const Mat& A, const int32_t* pi, const SpmvArgs& a, DevState* st,
                       cudaStream_t s) {
  return A.idx64 ? spmv_vw<int64_t, PV, RICH>(A, pi, a, st, s)
                 : spmv_vw<int32_t, PV, RICH>(A, pi, a, st, s);
}

// The two entry points every probability type's translation unit instantiates.
template <typename PV>
cudaError_t arnoldi_spmv_tu(const Mat& A, const int32_t* pi, float* basis, int64_t ld, int j,
                            float cdiag, DevState* st, cudaStream_t s) {
  const SpmvArgs a{basis + static_cast<int64_t>(j) * ld, basis + static_cast<int64_t>(j + 1) * ld,
                   j, nullptr, nullptr, cdiag};
  return spmv_entry<PV, false>(A, pi, a, st, s);
}

template <typename PV>
cudaError_t richardson_tu(const Mat& A, const int32_t* pi, const float* r, const float* d_in,
                          float* d_out, double* partials, DevState* st, cudaStream_t s) {
  const SpmvArgs a{d_in, d_out, 0, r, partials, 1.f};
  return spmv_entry<PV, true>(A, pi, a, st, s);
}

}  // namespace mdpk
