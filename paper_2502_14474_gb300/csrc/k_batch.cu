// Many MDPs in one launch per solve phase (the batching pattern): persistent
// kernels that walk a device-side work list of units (MDP, tile) over every
// MDP taking part in the phase.  The phases are those of inexact policy
// iteration with s-step GMRES (k_sstep.cu, k_bellman.cu):
//   kb_bellman       float-float Bellman backup, greedy policy, r = T V - V,
//                    the residual norms and the start of a GMRES cycle
//   kb_policy_resid  float-float policy residual between restart cycles
//   kb_spmv          an s-step basis vector w = -gamma P_pi x
//   kb_gram          the block's Gram matrix and its least-squares steps
//   kb_update        the block's orthonormalisation (+ the solution update)
// Each MDP's units are a fixed function of its own shape (not of the batch or
// the grid), and each MDP's reductions run in a fixed order over its own
// units, by the unit that draws its last ticket: an MDP's result is bitwise
// the same alone and in any batch.  The lanes per row (vw) of each MDP come
// from its handle (fixed at create, or chosen by the create-time autotuner).
#include "k_sstep.cuh"

namespace mdpk {

constexpr int kBT = 256;              // threads per block of every batched kernel
constexpr int kBStateUnit = 1024;     // states per unit of the residual, SpMV and update
constexpr int kBGramUnit = 1024;      // states per unit of the Gram pass
constexpr int kBRowTile = 2048;       // rows of a Bellman unit (states = max(32, 2048 / m))

int batch_bellman_tile(int m) {
  const int t = kBRowTile / m;
  return t < 32 ? 32 : t;
}

// Participant of unit u: the largest p with first[p] <= u.
__device__ __forceinline__ int find_part(const BList& L, int64_t u) {
  int lo = 0, hi = L.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.first[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The units of one block: chunks of kBChunk consecutive units, the chunks
// dealt round-robin to the blocks (chunk c to block c mod gridDim), so that at
// any time the grid works on a window of neighbouring units -- a few MDPs,
// whose gathered value vectors stay in L2 -- and a block meets a new MDP only
// at some chunk boundaries.  `walk_next` finds unit u's participant (moving
// forward from the last one) and, on a change of MDP, copies the descriptor to
// shared memory.
constexpr int kBChunk = 4;
struct UnitWalk {
  int64_t pend;
  int p;
};
__device__ __forceinline__ UnitWalk walk_begin(const BList& L) {
  (void)L;
  UnitWalk w;
  w.pend = -1;
  w.p = -1;
  return w;
}
__device__ __forceinline__ void walk_next(UnitWalk& w, const BList& L, const BMdp* mdps, int64_t u,
                                          BMdp& sm) {
  if (w.p >= 0 && u < w.pend) return;
  __syncthreads();  // every thread is done with the previous descriptor
  if (w.p < 0 || u >= L.first[w.p + 1] + 64) w.p = find_part(L, u);
  while (u >= L.first[w.p + 1]) ++w.p;
  w.pend = L.first[w.p + 1];
  if (threadIdx.x == 0) sm = mdps[L.mdp[w.p]];
  __syncthreads();
}
// for (unit u of this block): BATCH_UNITS(L, u) { ... }
#define BATCH_UNITS(L, u)                                                               \
  for (int64_t chunk_ = blockIdx.x; chunk_ * kBChunk < (L).total; chunk_ += gridDim.x) \
    for (int64_t u = chunk_ * kBChunk; u < min((L).total, (chunk_ + 1) * kBChunk); ++u)

// The block that draws the last of `total` tickets on `counter` (fixed order
// reductions of one MDP's units; the last one resets the counter).
__device__ __forceinline__ bool last_of(unsigned* counter, unsigned total) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    s_last = t == total - 1;
    if (s_last) *counter = 0;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

__device__ __forceinline__ void row_span(const BMdp& M, int64_t r, int64_t& b, int64_t& e) {
  if (M.uniform_len > 0) {
    b = r * M.uniform_len;
    e = b + M.uniform_len;
  } else if (M.idx64) {
    b = __ldcs(static_cast<const int64_t*>(M.rp) + r);
    e = __ldcs(static_cast<const int64_t*>(M.rp) + r + 1);
  } else {
    b = __ldcs(static_cast<const int32_t*>(M.rp) + r);
    e = __ldcs(static_cast<const int32_t*>(M.rp) + r + 1);
  }
}

// Sums over the vw lanes of a row (vw a power of two <= 32; every lane of
// the warp takes part).
__device__ __forceinline__ float gsum_rt(float v, int vw) {
  for (int o = vw >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ void gsum_ff_rt(float& hi, float& lo, int vw) {
  for (int o = vw >> 1; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_merge(hi, lo, ohi, olo);
  }
}

// Float-float row sum of P V over entries b + lane, b + lane + vw, ... < e.
__device__ __forceinline__ void row_ff(const BMdp& M, int64_t b, int64_t e, int lane, int vw,
                                       float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
  const GatherFF V{M.V};
  for (int64_t i = b + lane; i < e; i += vw) ff_elem(M.col, M.val, M.val_lo, V, i, hi, lo);
}

// Group mode (short rows): lane l of a row's vw lanes takes the packed groups
// (b >> 2) + l, + vw, ... of the row, so a row of up to 4 vw entries has all its
// loads in flight at once; within a group the entries are added in order, then
// the lanes' sums are combined by a fixed shuffle tree.
__device__ __forceinline__ void row_ff_groups(const BMdp& M, int64_t b, int64_t e, int lane,
                                              int vw, float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
  for (int64_t g = (b >> 2) + lane; (g << 2) < e; g += vw) {
    const int64_t i0 = g << 2;
    const int4 c = ldcol4(M.col, i0);
    const float4 p = Ld<float>::four(M.val, i0);
    const int cc[4] = {c.x, c.y, c.z, c.w};
    const float pp[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q;
      if (i >= b && i < e) {
        const float2 v = __ldg(M.V + cc[q]);
        ff_acc(hi, lo, pp[q], v.x, v.y);
      }
    }
  }
  gsum_ff_rt(hi, lo, vw);
}

__device__ __forceinline__ float row_f32_groups(const BMdp& M, const float* __restrict__ x,
                                                int64_t b, int64_t e, int lane, int vw) {
  float d = 0.f;
  for (int64_t g = (b >> 2) + lane; (g << 2) < e; g += vw) {
    const int64_t i0 = g << 2;
    const int4 c = ldcol4(M.col, i0);
    const float4 p = Ld<float>::four(M.val, i0);
    if (i0 >= b) d = fmaf(p.x, __ldg(x + c.x), d);
    if (i0 + 1 >= b && i0 + 1 < e) d = fmaf(p.y, __ldg(x + c.y), d);
    if (i0 + 2 >= b && i0 + 2 < e) d = fmaf(p.z, __ldg(x + c.z), d);
    if (i0 + 3 >= b && i0 + 3 < e) d = fmaf(p.w, __ldg(x + c.w), d);
  }
  return gsum_rt(d, vw);
}

// Per-unit partials (max |r|, sum r^2) and the MDP's fixed-order reduction.
__device__ __forceinline__ void unit_norms(const BMdp& M, int64_t lu, unsigned units,
                                           unsigned* counter, double my_max, double my_sq,
                                           bool set_target) {
  __shared__ double red[kBT / 32];
  const double bmax = block_max_d(my_max, red);
  const double bsq = block_sum_d(my_sq, red);
  if (threadIdx.x == 0) {
    M.part[2 * lu] = bmax;
    M.part[2 * lu + 1] = bsq;
  }
  if (last_of(counter, units)) {
    double mx = 0.0, sq = 0.0;
    for (int64_t q = threadIdx.x; q < units; q += kBT) {
      mx = fmax(mx, __ldcg(M.part + 2 * q));
      sq += __ldcg(M.part + 2 * q + 1);
    }
    mx = block_max_d(mx, red);
    sq = block_sum_d(sq, red);
    if (threadIdx.x == 0) {
      DevState* st = M.st;
      st->res_inf = mx;
      st->res_2 = sqrt(sq);
      if (set_target && st->target_rel) st->target = st->eta * mx;
      gmres_begin(st, sqrt(sq));
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Bellman backup (float-float): unit = a tile of tb states (tb * m <= 2048 rows)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT)
    kb_bellman(const BMdp* __restrict__ mdps, const BList* __restrict__ Lp) {
  __shared__ float qh[kBRowTile], ql[kBRowTile];
  __shared__ BMdp sm;
  const BList L = *Lp;
  UnitWalk wk = walk_begin(L);
  BATCH_UNITS(L, u) {
    walk_next(wk, L, mdps, u, sm);
    const BMdp& M = sm;
    const int64_t lu = u - L.first[wk.p];
    const int m = M.m, T = M.tb, vw = M.vw;
    const int64_t s0 = lu * T;
    const int ns = static_cast<int>(min(static_cast<int64_t>(T), M.n - s0));
    const int rows = ns * m;
    auto put_q = [&](int lr, float hi, float lo) {
      const int64_t r = s0 * m + lr;
      const ff sum = ff_norm(hi, lo);
      const ff gq = ff_norm(__ldcs(M.g + r), M.g_lo ? __ldcs(M.g_lo + r) : 0.f);
      const ff q = ff_add(ff_mul(sum, ff{M.gamma_hi, M.gamma_lo}), gq);
      const int a = lr % m, sl = lr / m;
      qh[a * T + sl] = q.hi;
      ql[a * T + sl] = q.lo;
    };
    const int lane = threadIdx.x % vw, vec = threadIdx.x / vw, nvec = kBT / vw;
    for (int base = 0; base < rows; base += nvec) {
      const int lr = base + vec;
      int64_t b = 0, e = 0;
      if (lr < rows) row_span(M, s0 * m + lr, b, e);
      float hi, lo;
      if (M.grp) {
        row_ff_groups(M, b, e, lane, vw, hi, lo);
      } else {
        row_ff(M, b, e, lane, vw, hi, lo);
        gsum_ff_rt(hi, lo, vw);
      }
      if (lane == 0 && lr < rows) put_q(lr, hi, lo);
    }
    __syncthreads();
    double my_max = 0.0, my_sq = 0.0;
    for (int t = threadIdx.x; t < ns; t += kBT) {
      float bh = qh[t], bl = ql[t];
      int arg = 0;
      for (int a = 1; a < m; ++a) {
        const float h = qh[a * T + t], l = ql[a * T + t];
        if (h < bh || (h == bh && l < bl)) {
          bh = h;
          bl = l;
          arg = a;
        }
      }
      const int64_t s = s0 + t;
      const float2 v = M.V[s];
      const float r = ff_diff_to_float(bh, bl, v.x, v.y);
      M.pi[s] = arg;
      M.basis[s] = r;  // u_0 of the next cycle
      const double rd = static_cast<double>(r);
      my_max = fmax(my_max, fabs(rd));
      my_sq += rd * rd;
    }
    unit_norms(M, lu, static_cast<unsigned>(M.u_bell), &M.st->counter[kCntBellman], my_max, my_sq,
               true);
  }
}

// ---------------------------------------------------------------------------
// Policy residual (float-float) r = g_pi + gamma P_pi V - V: unit = 1024 states
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT)
    kb_policy_resid(const BMdp* __restrict__ mdps, const BList* __restrict__ Lp) {
  const BList L = *Lp;
  __shared__ BMdp sm;
  UnitWalk wk = walk_begin(L);
  BATCH_UNITS(L, u) {
    walk_next(wk, L, mdps, u, sm);
    const BMdp& M = sm;
    const int64_t lu = u - L.first[wk.p];
    const int vw = M.vw;
    const int64_t s0 = lu * kBStateUnit;
    const int ns = static_cast<int>(min(static_cast<int64_t>(kBStateUnit), M.n - s0));
    double my_max = 0.0, my_sq = 0.0;
    auto emit = [&](int64_t s, int64_t r, float hi, float lo) {
      const ff sum = ff_norm(hi, lo);
      const ff gq = ff_norm(__ldcs(M.g + r), M.g_lo ? __ldcs(M.g_lo + r) : 0.f);
      const ff q = ff_add(ff_mul(sum, ff{M.gamma_hi, M.gamma_lo}), gq);
      const float2 v = M.V[s];
      const float rr = ff_diff_to_float(q.hi, q.lo, v.x, v.y);
      M.basis[s] = rr;
      const double rd = static_cast<double>(rr);
      my_max = fmax(my_max, fabs(rd));
      my_sq += rd * rd;
    };
    const int lane = threadIdx.x % vw, vec = threadIdx.x / vw, nvec = kBT / vw;
    for (int base = 0; base < ns; base += nvec) {
      const int t = base + vec;
      const int64_t s = s0 + t;
      int64_t b = 0, e = 0, r = 0;
      if (t < ns) {
        r = s * M.m + M.pi[s];
        row_span(M, r, b, e);
      }
      float hi, lo;
      if (M.grp) {
        row_ff_groups(M, b, e, lane, vw, hi, lo);
      } else {
        row_ff(M, b, e, lane, vw, hi, lo);
        gsum_ff_rt(hi, lo, vw);
      }
      if (lane == 0 && t < ns) emit(s, r, hi, lo);
    }
    unit_norms(M, lu, static_cast<unsigned>(M.u_state), &M.st->counter[kCntPolicy], my_max,
               my_sq, false);
  }
}

// ---------------------------------------------------------------------------
// s-step basis vector: column j+1 = -gamma P_pi (scale_j u_j): unit = 1024 states
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT, 4)
    kb_spmv(const BMdp* __restrict__ mdps, const BList* __restrict__ Lp, int j) {
  const BList L = *Lp;
  __shared__ BMdp sm;
  UnitWalk wk = walk_begin(L);
  BATCH_UNITS(L, u) {
    walk_next(wk, L, mdps, u, sm);
    const BMdp& M = sm;
    if (!M.st->active) continue;
    const int64_t lu = u - L.first[wk.p];
    const int vw = M.vw;
    const float sj = static_cast<float>(M.st->scale[j]);
    const float* x = M.basis + static_cast<int64_t>(j) * M.ld;
    float* w = M.basis + static_cast<int64_t>(j + 1) * M.ld;
    const int64_t s0 = lu * kBStateUnit;
    const int ns = static_cast<int>(min(static_cast<int64_t>(kBStateUnit), M.n - s0));
    const int lane = threadIdx.x % vw, vec = threadIdx.x / vw, nvec = kBT / vw;
    for (int base = 0; base < ns; base += nvec) {
      const int t = base + vec;
      const int64_t s = s0 + t;
      int64_t b = 0, e = 0;
      if (t < ns) row_span(M, s * M.m + M.pi[s], b, e);
      float d;
      if (M.grp) {
        d = row_f32_groups(M, x, b, e, lane, vw);
      } else {
        d = 0.f;
        for (int64_t i = b + lane; i < e; i += vw)
          d = fmaf(Ld<float>::one(M.val, i), __ldg(x + ldcol(M.col, i)), d);
        d = gsum_rt(d, vw);
      }
      if (lane == 0 && t < ns) w[s] = sj * (-M.gamma * d);
    }
  }
}

// ---------------------------------------------------------------------------
// Gram pass of the block at step k (sb vectors): unit = 1024 states of one
// MDP.  W's chunk is staged in shared memory; warp w streams the vectors
// v = w, w + 8, ... < k + 1 + sb over the chunk, sums each product column in
// FP32 over the lane's 32 terms, then in float-float across the warp, and
// writes one float-float partial per (unit, vector, column).  The MDP's last
// unit sums the partials over its units in order and runs block_ls.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT)
    kb_gram(const BMdp* __restrict__ mdps, const BList* __restrict__ Lp, int k, int sb) {
  constexpr int CQ = kBGramUnit / 4;
  __shared__ __align__(16) float4 wsm[kSMax * CQ];  // 32 KB; block_ls's scratch at the end
  static_assert(sizeof(wsm) >= sizeof(double) * kMaxRestart * kMaxRestart, "scratch");
  const BList L = *Lp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nv = k + 1 + sb;
  __shared__ BMdp sm;
  UnitWalk wk = walk_begin(L);
  BATCH_UNITS(L, u) {
    walk_next(wk, L, mdps, u, sm);
    const BMdp& M = sm;
    if (!M.st->active) continue;
    const int64_t lu = u - L.first[wk.p];
    const int64_t c0 = lu * kBGramUnit;
    const int len = static_cast<int>(min(static_cast<int64_t>(kBGramUnit), M.n - c0));
    __syncthreads();  // the previous unit's readers are done with wsm
    for (int q = threadIdx.x; q < kSMax * CQ; q += kBT) {
      const int i = q / CQ, e = 4 * (q % CQ);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < sb) {
        const float* src = M.basis + static_cast<int64_t>(k + 1 + i) * M.ld + c0;
        if (e + 3 < len) {
          v = *reinterpret_cast<const float4*>(src + e);
        } else if (e < len) {
          v.x = src[e];
          if (e + 1 < len) v.y = src[e + 1];
          if (e + 2 < len) v.z = src[e + 2];
        }
      }
      wsm[q] = v;
    }
    __syncthreads();
    float2* out = reinterpret_cast<float2*>(M.bpart) + lu * kBlkStride;
    for (int v = warp; v < nv; v += kBT / 32) {
      const float* xv = M.basis + static_cast<int64_t>(v) * M.ld + c0;
      float acc[kSMax];
#pragma unroll
      for (int i = 0; i < kSMax; ++i) acc[i] = 0.f;
      for (int qd = lane; qd < CQ; qd += 32) {
        const int e = 4 * qd;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e + 3 < len) {
          x = __ldcs(reinterpret_cast<const float4*>(xv + e));
        } else if (e < len) {
          x.x = xv[e];
          if (e + 1 < len) x.y = xv[e + 1];
          if (e + 2 < len) x.z = xv[e + 2];
        }
#pragma unroll
        for (int i = 0; i < kSMax; ++i) {
          const float4 w = wsm[i * CQ + qd];
          acc[i] = fmaf(x.x, w.x, fmaf(x.y, w.y, fmaf(x.z, w.z, fmaf(x.w, w.w, acc[i]))));
        }
      }
#pragma unroll
      for (int i = 0; i < kSMax; ++i) {
        if (i >= sb) break;  // the same for the whole block
        float h = acc[i], l = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          ff_merge(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
        if (lane == 0) out[v * kSMax + i] = make_float2(h, l);
      }
    }
    if (last_of(&M.st->dots_group[0], static_cast<unsigned>(M.u_gram))) {
      // the MDP's Gram block: float-float sums over its units in order
      const float2* all = reinterpret_cast<const float2*>(M.bpart);
      // one warp per (vector, column): lanes stride over the units, then a
      // fixed float-float shuffle tree
      for (int q = warp; q < nv * kSMax; q += kBT / 32) {
        const int v = q / kSMax, i = q % kSMax;
        if (i >= sb) continue;
        float h = 0.f, l = 0.f;
        for (int64_t c = lane; c < M.u_gram; c += 32) {
          const float2 t = __ldcg(all + c * kBlkStride + v * kSMax + i);
          ff_merge(h, l, t.x, t.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          ff_merge(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
        if (lane == 0) M.st->G[v * kSMax + i] = static_cast<double>(h) + static_cast<double>(l);
      }
      __syncthreads();
      block_ls(M.st, k, sb, M.st->restart, reinterpret_cast<double*>(wsm));
    }
  }
}

// ---------------------------------------------------------------------------
// Update pass of the block at step k: unit = 1024 states (a quad per thread)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT)
    kb_update(const BMdp* __restrict__ mdps, const BList* __restrict__ Lp, int k, int sb) {
  __shared__ float cf[kMaxBasis * kSMax];
  __shared__ float ri[kSMax * kSMax];
  __shared__ float yc[kBlkMaxV];
  const BList L = *Lp;
  (void)sb;
  __shared__ BMdp sm;
  UnitWalk wk = walk_begin(L);
  BATCH_UNITS(L, u) {
    walk_next(wk, L, mdps, u, sm);
    const BMdp& M = sm;
    const DevState* st = M.st;
    const bool fin = st->bfin_k == k;
    if (!st->active && !fin) continue;
    const int64_t lu = u - L.first[wk.p];
    const int nnew = st->bsb;
    const int J = fin ? st->jdone : 0;
    __syncthreads();  // the previous unit's readers are done with the coefficients
    for (int t = threadIdx.x; t < (k + 1) * kSMax; t += kBT) cf[t] = st->bC[t];
    for (int t = threadIdx.x; t < kSMax * kSMax; t += kBT) ri[t] = st->bRinv[t];
    for (int t = threadIdx.x; t < kBlkMaxV; t += kBT) yc[t] = fin ? st->bY[t] : 0.f;
    __syncthreads();
    const int64_t s = lu * kBStateUnit + 4 * threadIdx.x;
    if (s >= M.n) continue;
    if (s + 3 < M.n) {
      float4 w[kSMax];
      float4 vacc = make_float4(0.f, 0.f, 0.f, 0.f);
      block_update_quad<kSMax>(M.basis, M.ld, k, nnew, J, fin, cf, ri, yc, s, w, vacc);
#pragma unroll
      for (int i = 0; i < kSMax; ++i) {
        if (i < nnew) {
          *reinterpret_cast<float4*>(M.basis + static_cast<int64_t>(k + 1 + i) * M.ld + s) = w[i];
          if (fin && k + 1 + i < J) {
            const float c = yc[k + 1 + i];
            vacc.x = fmaf(c, w[i].x, vacc.x);
            vacc.y = fmaf(c, w[i].y, vacc.y);
            vacc.z = fmaf(c, w[i].z, vacc.z);
            vacc.w = fmaf(c, w[i].w, vacc.w);
          }
        }
      }
      if (fin) {
        float4* v4 = reinterpret_cast<float4*>(M.V + s);
        const float4 va = v4[0], vb = v4[1];
        const ff r0 = ff_add_f(ff{va.x, va.y}, vacc.x), r1 = ff_add_f(ff{va.z, va.w}, vacc.y);
        const ff r2 = ff_add_f(ff{vb.x, vb.y}, vacc.z), r3 = ff_add_f(ff{vb.z, vb.w}, vacc.w);
        v4[0] = make_float4(r0.hi, r0.lo, r1.hi, r1.lo);
        v4[1] = make_float4(r2.hi, r2.lo, r3.hi, r3.lo);
      }
    } else {
      // ragged end of the vector: state by state, same order of operations
      for (int64_t e = s; e < M.n; ++e) {
        float w[kSMax];
        float va = 0.f;
#pragma unroll
        for (int i = 0; i < kSMax; ++i)
          w[i] = i < nnew ? M.basis[static_cast<int64_t>(k + 1 + i) * M.ld + e] : 0.f;
        for (int v = 0; v <= k; ++v) {
          const float x = M.basis[static_cast<int64_t>(v) * M.ld + e];
#pragma unroll
          for (int i = 0; i < kSMax; ++i) w[i] = fmaf(-cf[v * kSMax + i], x, w[i]);
          if (fin && v < J) va = fmaf(yc[v], x, va);
        }
#pragma unroll
        for (int i = kSMax - 1; i >= 0; --i) {
          float q = 0.f;
#pragma unroll
          for (int l = 0; l <= i; ++l) q = fmaf(ri[l * kSMax + i], w[l], q);
          w[i] = q;
        }
#pragma unroll
        for (int i = 0; i < kSMax; ++i)
          if (i < nnew) {
            M.basis[static_cast<int64_t>(k + 1 + i) * M.ld + e] = w[i];
            if (fin && k + 1 + i < J) va = fmaf(yc[k + 1 + i], w[i], va);
          }
        if (fin) {
          const float2 v = M.V[e];
          const ff r = ff_add_f(ff{v.x, v.y}, va);
          M.V[e] = make_float2(r.hi, r.lo);
        }
      }
    }
  }
}

// Copy the status prefix of every MDP's device state into one array.
__global__ void kb_heads(const BMdp* __restrict__ mdps, int count, size_t head_bytes,
                         unsigned char* __restrict__ out) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const unsigned char* src = reinterpret_cast<const unsigned char*>(mdps[i].st);
    for (size_t b = threadIdx.x; b < head_bytes; b += blockDim.x) out[i * head_bytes + b] = src[b];
  }
}

// ---------------------------------------------------------------------------
// Launchers: one persistent wave (num_sms x resident blocks per SM)
// ---------------------------------------------------------------------------
template <typename K>
static unsigned waves_of(K kern, int num_sms, size_t smem = 0) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBT, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  return static_cast<unsigned>(num_sms * occ);
}

cudaError_t launch_batch_bellman(const BMdp* mdps, const BList* list, int num_sms, cudaStream_t s) {
  static const unsigned nb = waves_of(kb_bellman, num_sms);
  kb_bellman<<<nb, kBT, 0, s>>>(mdps, list);
  return cudaGetLastError();
}

cudaError_t launch_batch_policy_resid(const BMdp* mdps, const BList* list, int num_sms,
                                      cudaStream_t s) {
  static const unsigned nb = waves_of(kb_policy_resid, num_sms);
  kb_policy_resid<<<nb, kBT, 0, s>>>(mdps, list);
  return cudaGetLastError();
}

cudaError_t launch_batch_spmv(const BMdp* mdps, const BList* list, int j, int num_sms,
                              cudaStream_t s) {
  static const unsigned nb = waves_of(kb_spmv, num_sms);
  kb_spmv<<<nb, kBT, 0, s>>>(mdps, list, j);
  return cudaGetLastError();
}

cudaError_t launch_batch_gram(const BMdp* mdps, const BList* list, int k, int sb, int num_sms,
                              cudaStream_t s) {
  static const unsigned nb = waves_of(kb_gram, num_sms);
  kb_gram<<<nb, kBT, 0, s>>>(mdps, list, k, sb);
  return cudaGetLastError();
}

cudaError_t launch_batch_update(const BMdp* mdps, const BList* list, int k, int sb, int num_sms,
                                cudaStream_t s) {
  static const unsigned nb = waves_of(kb_update, num_sms);
  kb_update<<<nb, kBT, 0, s>>>(mdps, list, k, sb);
  return cudaGetLastError();
}

cudaError_t launch_batch_heads(const BMdp* mdps, int count, size_t head_bytes, unsigned char* out,
                               cudaStream_t s) {
  kb_heads<<<count < 1024 ? (count > 0 ? count : 1) : 1024, 128, 0, s>>>(mdps, count, head_bytes,
                                                                          out);
  return cudaGetLastError();
}

int64_t batch_units_bellman(int64_t n, int m) {
  const int t = batch_bellman_tile(m);
  return (n + t - 1) / t;
}
int64_t batch_units_state(int64_t n) { return (n + kBStateUnit - 1) / kBStateUnit; }
int64_t batch_units_gram(int64_t n) { return (n + kBGramUnit - 1) / kBGramUnit; }

}  // namespace mdpk
