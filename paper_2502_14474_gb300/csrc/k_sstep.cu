// s-step GMRES for the policy-evaluation system (I - gamma P_pi) d = r.
//
// Classical Gram-Schmidt Arnoldi streams the whole basis twice per step (the
// dots, then the subtraction).  The s-step form (Chronopoulos & Gear 1989;
// Hoemmen 2010, "Communication-avoiding Krylov subspace methods", ch. 3)
// builds a block of sb Krylov vectors with sb policy-row SpMVs first and
// orthogonalises the whole block against the basis at once, so the basis is
// streamed twice per block instead of twice per step.
//
// Block starting at step k (orthonormal q_0..q_k in basis columns 0..k, q_v =
// u_v * scale_v):
//   SpMVs   w_1 = (A - I) q_k, w_{i+1} = (A - I) w_i  (= -gamma P_pi w_i; the
//           monomial basis of A - I), w_i stored in column k+i (k_spmv.cuh,
//           cdiag = 0).
//   Gram    one pass over [Q W]: G = [Q W]^T W, C = Q^T W, and the block's own
//           Gram matrix W^T W; products are summed in FP32 over 32 terms per
//           lane, then in float-float, so that the Pythagorean form below keeps
//           its digits (k_block_dots).  Its last block runs the small FP64
//           steps (block_ls): R^T R = W^T W - C^T C (Cholesky; "BCGS-PIP",
//           Carson, Lund, Rozloznik & Thomas 2021), the new Hessenberg columns
//           from A [q_k, W] = [q_k, W] B (B: ones on the diagonal and the
//           subdiagonal), the Givens rotations and the convergence test of each
//           new column, and at the end of the cycle the back-solve R y = g.
//   Update  one pass: q_{k+1+i} = ((W - Q C) R^{-1})_i written over w_{i+1};
//           on the block that ends the cycle the same pass also adds the
//           solution update V += sum_v y_v q_v (it reads every q_v anyway),
//           so no separate update kernel runs (k_block_update).
// A pivot of the Cholesky factor below a relative 1e-9 of its column's norm
// is an exact dependence of the block (an invariant subspace): its Hessenberg
// column gets a zero subdiagonal and the cycle ends there, as an Arnoldi
// breakdown does.
#include <cstdlib>
#include <type_traits>

#include "k_async.cuh"
#include "k_sstep.cuh"

namespace mdpk {

// ---------------------------------------------------------------------------
// Gram pass: G[v][i] = <x_v, w_{i+1}> for x = [u_0..u_k, w_1..w_sb] (raw
// columns 0..k+sb), i < sb.  Grid (slots x groups): block (y, gx) owns the
// contiguous states of slot y and the group's vectors, split evenly over the
// groups and round-robin over the warps (up to VPW per warp).  The block walks
// its slot in chunks of 512 states: W's chunk is staged in shared memory by
// cp.async (double-buffered, so the copy of the next chunk overlaps the
// products of this one), and each warp loads its vectors one 128-state tile
// ahead in registers.  Products are summed in FP32 over eight tiles per lane
// (32 terms), then folded into float-float sums kept in shared memory.
// Partials: one FP64 value per (slot, v, i), reduced in two fixed-order levels
// (runs of eight slots, then the runs of a group); the last group runs
// block_ls.
// ---------------------------------------------------------------------------
template <int S>
struct GramVpw {  // vectors per warp: 8 * VPW vectors per group, FP32 accumulators VPW * S
  static constexpr int value = S <= 4 ? 6 : 4;
};
constexpr int kGramChunk = 512;  // states of W staged per chunk (4 tiles of 128)

// Dynamic shared memory of the Gram pass: the per-lane float-float sums
// (hi, lo) of every accumulator, thread-contiguous, then two W chunk buffers;
// the last block reuses the space as block_ls's scratch.
template <int S>
constexpr size_t gram_ff_bytes() {
  return 2ull * GramVpw<S>::value * S * kBlkThreads * sizeof(float);
}
template <int S>
constexpr size_t gram_smem_bytes() {
  constexpr size_t b = gram_ff_bytes<S>() + 2ull * S * kGramChunk * sizeof(float);
  constexpr size_t ls = sizeof(double) * kMaxRestart * kMaxRestart;
  return b > ls ? b : ls;
}

// 16-byte asynchronous copy global -> shared; bytes past `src_bytes` are zero.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int S>
__global__ void __launch_bounds__(kBlkThreads)
    k_block_dots(int64_t n, int64_t states_per_slot, const float* __restrict__ basis, int64_t ld,
                 int k, int sb, int restart, double* __restrict__ partials,
                 DevState* __restrict__ st) {
  if (!st->active) return;
  constexpr int VPW = GramVpw<S>::value;
  constexpr int NW = kBlkThreads / 32;
  constexpr int VPG = NW * VPW;  // vectors per group
  constexpr int NA = VPW * S;    // accumulators per lane
  constexpr int CQ = kGramChunk / 4;  // quads per staged column
  extern __shared__ __align__(16) unsigned char gram_dyn[];
  float* fhi = reinterpret_cast<float*>(gram_dyn);
  float* flo = fhi + NA * kBlkThreads;
  float4* wbuf = reinterpret_cast<float4*>(gram_dyn + gram_ff_bytes<S>());  // [2][S][CQ]
  double* scratch = reinterpret_cast<double*>(gram_dyn);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gx = static_cast<int>(blockIdx.y), vg = static_cast<int>(gridDim.y);
  const int64_t slot = blockIdx.x, slots = gridDim.x;
  const int nv = k + 1 + sb;
  // the vectors split evenly over the groups, then round-robin over the warps
  const int per_g = (nv + vg - 1) / vg;
  const int g0 = gx * per_g, g1 = min(nv, g0 + per_g);
  int vid[VPW];
  bool vok[VPW];
#pragma unroll
  for (int u = 0; u < VPW; ++u) {
    vid[u] = g0 + u * NW + warp;
    vok[u] = vid[u] < g1;
  }
#pragma unroll
  for (int a = 0; a < NA; ++a) fhi[a * kBlkThreads + threadIdx.x] = flo[a * kBlkThreads + threadIdx.x] = 0.f;
  float acc[VPW][S];
#pragma unroll
  for (int u = 0; u < VPW; ++u)
#pragma unroll
    for (int i = 0; i < S; ++i) acc[u][i] = 0.f;
  auto fold = [&]() {  // this lane's FP32 runs into its float-float sums
#pragma unroll
    for (int u = 0; u < VPW; ++u)
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const int a = (u * S + i) * kBlkThreads + threadIdx.x;
        float h = fhi[a], l = flo[a];
        ff_merge(h, l, acc[u][i], 0.f);
        fhi[a] = h;
        flo[a] = l;
        acc[u][i] = 0.f;
      }
  };
  const int64_t s_begin = slot * states_per_slot;
  const int64_t s_end = min(n, s_begin + states_per_slot);
  const float* wcol = basis + static_cast<int64_t>(k + 1) * ld;
  // W chunk c of this slot into buffer b (zero past the end of the vector)
  auto stage = [&](int64_t c0, int b) {
    for (int q = threadIdx.x; q < sb * CQ; q += kBlkThreads) {
      const int i = q / CQ, e4 = q % CQ;
      const int64_t e = c0 + 4 * e4;
      int64_t left = s_end - e;
      const int bytes = left >= 4 ? 16 : (left > 0 ? static_cast<int>(left) * 4 : 0);
      cp_async16(wbuf + (b * S + i) * CQ + e4, wcol + i * ld + (bytes > 0 ? e : s_begin), bytes);
    }
    cp_async_commit();
  };
  auto ldx = [&](int64_t e, float4 (&x)[VPW]) {  // the warp's vectors at quad e
#pragma unroll
    for (int u = 0; u < VPW; ++u) {
      x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (vok[u] && e < s_end) {
        const float* p = basis + vid[u] * ld;
        if (e + 3 < s_end) {
          x[u] = __ldcs(reinterpret_cast<const float4*>(p + e));
        } else {  // ragged end: past n reads as zero
          x[u].x = p[e];
          if (e + 1 < s_end) x[u].y = p[e + 1];
          if (e + 2 < s_end) x[u].z = p[e + 2];
        }
      }
    }
  };
  const int64_t nch = (s_end - s_begin + kGramChunk - 1) / kGramChunk;
  if (nch > 0) stage(s_begin, 0);
  float4 xc[VPW];
  ldx(s_begin + 4 * lane, xc);
  int frun = 0;
  for (int64_t c = 0; c < nch; ++c) {
    const int64_t c0 = s_begin + c * kGramChunk;
    if (c + 1 < nch) {
      stage(c0 + kGramChunk, static_cast<int>((c + 1) & 1));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // chunk c is in its buffer for every warp
    const float4* wb = wbuf + static_cast<int>(c & 1) * S * CQ;
#pragma unroll
    for (int t = 0; t < kGramChunk / 128; ++t) {
      float4 xn[VPW];
      ldx(c0 + 128 * (t + 1) + 4 * lane, xn);  // one tile ahead (the next chunk's first)
      if (vok[0]) {
#pragma unroll
        for (int i = 0; i < S; ++i) {
          if (i < sb) {
            const float4 w = wb[i * CQ + t * 32 + lane];
#pragma unroll
            for (int u = 0; u < VPW; ++u)
              acc[u][i] = fmaf(xc[u].x, w.x, fmaf(xc[u].y, w.y, fmaf(xc[u].z, w.z,
                                                                  fmaf(xc[u].w, w.w, acc[u][i]))));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < VPW; ++u) xc[u] = xn[u];
    }
    if (++frun == 2) {  // 8 tiles of FP32 products per lane, then float-float
      frun = 0;
      fold();
    }
    __syncthreads();  // every warp is done with this buffer before it is refilled
  }
  fold();
  // warp sums (float-float) and the slot's partials
#pragma unroll
  for (int u = 0; u < VPW; ++u)
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const int a = (u * S + i) * kBlkThreads + threadIdx.x;
      float h = fhi[a], l = flo[a];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        ff_merge(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
      if (lane == 0 && vok[u] && i < sb)
        partials[slot * kBlkStride + vid[u] * kSMax + i] =
            static_cast<double>(h) + static_cast<double>(l);
    }
  __shared__ bool s_last;
  const int t = threadIdx.x;
  // level 1: the last block of this run of slots sums the run in slot order
  const int64_t run = slot / kBlkRun, runs = (slots + kBlkRun - 1) / kBlkRun;
  const int64_t run_len = min(static_cast<int64_t>(kBlkRun), slots - run * kBlkRun);
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->dots_run[gx][run], 1u) == run_len - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = t; q < VPG * kSMax; q += kBlkThreads) {
    const int qv = g0 + q / kSMax, qi = q % kSMax;
    if (qv >= g1 || qi >= sb) continue;
    const double* pr = partials + run * kBlkRun * kBlkStride + qv * kSMax + qi;
    double sum = 0.0;
    for (int r = 0; r < run_len; ++r) sum += __ldcg(pr + r * kBlkStride);
    partials[run * kBlkRun * kBlkStride + qv * kSMax + qi] = sum;
  }
  if (t == 0) st->dots_run[gx][run] = 0;
  // level 2: the last run of this group sums the runs in order
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->dots_group[gx], 1u) == runs - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // one thread per (vector, column) value, the runs summed in order (the
  // loads are independent, so an unrolled loop keeps several in flight)
  for (int q = t; q < VPG * kSMax; q += kBlkThreads) {
    const int qv = g0 + q / kSMax, qi = q % kSMax;
    if (qv >= g1 || qi >= sb) continue;
    const double* pr = partials + qv * kSMax + qi;
    double sum = 0.0;
#pragma unroll 8
    for (int64_t r = 0; r < runs; ++r) sum += __ldcg(pr + r * kBlkRun * kBlkStride);
    st->G[qv * kSMax + qi] = sum;
  }
  if (t == 0) st->dots_group[gx] = 0;
  // level 3: the last group runs the block's small steps
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->blk_groups, 1u) == static_cast<unsigned>(vg) - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (t == 0) st->blk_groups = 0;
  __syncthreads();  // the float-float sums are no longer read: the space is block_ls's
  block_ls(st, k, sb, restart, scratch);
}

// ---------------------------------------------------------------------------
// Gram pass, bulk-copy form (the default): one CTA per SM owns a contiguous
// slot of states and walks it in stages of `stg` states.  A producer warp
// copies each stage of every vector of the CTA's group (and of W, when the
// group does not hold it) from HBM into shared memory with cp.async.bulk,
// completing on the stage's mbarrier; the copies of up to `nstages` stages are
// in flight at once, independent of the registers.  Eight consumer warps each
// own a few of the group's vectors: per 128-state tile a lane reads its quad
// of W's columns and of its vectors from the stage and accumulates the
// products in pairs with the packed FP32x2 FMA (two running sums per dot, of
// the quads' (x, y) and (z, w) entries), folds them into float-float sums held
// in registers every eight tiles, and releases the stage.  Partials and their
// fixed-order reduction are those of the register form above (runs of eight
// slots, then the runs, then block_ls).
// ---------------------------------------------------------------------------
constexpr int kGramCW = 8;                          // consumer warps
constexpr int kGramTh = 32 * (kGramCW + 1);         // + the producer warp
constexpr int kGramStageMax = 2048;                 // states per stage, at most
constexpr int kGramMaxStages = 16;
constexpr size_t kGramSmemBudget = 208 * 1024;      // stage buffers
constexpr int kGramErrTimeout = 1;                  // dev_error code of a wait that gave up
// vectors per consumer warp and per group.  A thread holds 2 * VPW * S FP32
// sums and as many float-float parts; with nine warps per SM (three on one of
// the four schedulers' register files) a thread has at most 168 registers.
constexpr int gram_vpw(int S) { return S <= 4 ? 6 : (S <= 6 ? 4 : 3); }
constexpr int gram_vpg(int S) { return kGramCW * gram_vpw(S); }

template <int S>
__global__ void __launch_bounds__(kGramTh, 1)
    k_block_gram(int64_t n, int64_t states_per_slot, const float* __restrict__ basis, int64_t ld,
                 int k, int sb, int restart, int nstages, int stg, int stall,
                 double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  constexpr int NW = kGramCW, VPW = gram_vpw(S);
  extern __shared__ __align__(128) unsigned char gram_stage_dyn[];
  __shared__ __align__(8) uint64_t full[kGramMaxStages], empty[kGramMaxStages];
  __shared__ int s_abort;
  __shared__ bool s_last;
  float* stages = reinterpret_cast<float*>(gram_stage_dyn);
  double* scratch = reinterpret_cast<double*>(gram_stage_dyn);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  const int gx = static_cast<int>(blockIdx.y), vg = static_cast<int>(gridDim.y);
  const int64_t slot = blockIdx.x, slots = gridDim.x;
  const int nv = k + 1 + sb;
  const int per_g = (nv + vg - 1) / vg;
  const int g0 = gx * per_g, g1 = min(nv, g0 + per_g);
  const int ng = g1 - g0;
  // W's columns inside the group's copies (the group holds the last vectors) or after them
  const bool w_in = g1 == nv && g0 <= k + 1;
  const int w_off = w_in ? k + 1 - g0 : ng;
  const int ncp = ng + (w_in ? 0 : sb);
  const int64_t s_begin = slot * states_per_slot;
  const int64_t s_end = min(n, s_begin + states_per_slot);
  const int64_t nch = s_end > s_begin ? (s_end - s_begin + stg - 1) / stg : 0;
  if (t == 0) {
    s_abort = 0;
    for (int b = 0; b < nstages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NW);
    }
    mbar_init_fence();
  }
  __syncthreads();

  float fh[VPW][S], fl[VPW][S];
  int vloc[VPW];
  bool vok[VPW];
#pragma unroll
  for (int u = 0; u < VPW; ++u) {
    vloc[u] = u * NW + warp;
    vok[u] = warp < NW && vloc[u] < ng;
  }
  if (warp == NW) {
    // ---- producer: stage c into buffer c % nstages once its last reader left
    // (`stall`, a test of the bounded waits: no stage is ever armed, so every
    // consumer's wait runs out and the launch reports it)
    int64_t issued = 0;
    for (int64_t c = 0; c < (stall ? 0 : nch); ++c) {
      const int b = static_cast<int>(c % nstages);
      if (c >= nstages &&
          !mbar_wait(&empty[b], static_cast<unsigned>((c / nstages - 1) & 1), &s_abort)) {
        s_abort = 1;
        break;
      }
      const int64_t c0 = s_begin + c * stg;
      const int64_t left = s_end - c0;
      // a short last stage rounds up to 16 bytes: the column's padding (ld >=
      // n rounded up to 64) or the next slot's states, masked by the consumers
      const unsigned bytes = left >= stg ? static_cast<unsigned>(stg) * 4u
                                                : static_cast<unsigned>((left * 4 + 15) & ~15);
      if (lane == 0) mbar_arrive_expect_tx(&full[b], bytes * static_cast<unsigned>(ncp));
      __syncwarp();
      float* dst = stages + static_cast<size_t>(b) * ncp * stg;
      for (int q = lane; q < ncp; q += 32) {
        const int v = q < ng ? g0 + q : k + 1 + (q - ng);
        bulk_g2s(dst + static_cast<size_t>(q) * stg, basis + v * ld + c0, bytes, &full[b]);
      }
      issued = c + 1;
    }
    // copies still in flight (only after an abort) land before the CTA leaves
    if (lane == 0 && s_abort) {
      const int none = 0;
      for (int64_t c = max(int64_t(0), issued - nstages); c < issued; ++c)
        mbar_wait(&full[c % nstages], static_cast<unsigned>((c / nstages) & 1), &none);
    }
  } else {
    // ---- consumers.  acc[u][i] holds two running sums, of the (x, y) and of
    // the (z, w) entries of the lane's quads
    float2 acc[VPW][S];
#pragma unroll
    for (int u = 0; u < VPW; ++u)
#pragma unroll
      for (int i = 0; i < S; ++i) {
        acc[u][i] = make_float2(0.f, 0.f);
        fh[u][i] = fl[u][i] = 0.f;
      }
    auto fold = [&]() {
#pragma unroll
      for (int u = 0; u < VPW; ++u)
#pragma unroll
        for (int i = 0; i < S; ++i) {
          ff_merge(fh[u][i], fl[u][i], acc[u][i].x, 0.f);
          ff_merge(fh[u][i], fl[u][i], acc[u][i].y, 0.f);
          acc[u][i] = make_float2(0.f, 0.f);
        }
    };
    // one 128-state tile of a stage; MASKED: the stage ends inside the slot
    // and its entries from `left` on are zero
    auto tile = [&](const float* sp, int tl, int64_t left, auto masked) {
      constexpr bool MASKED = decltype(masked)::value;
      const int e = tl * 128 + 4 * lane;
      int lim = 4;
      if constexpr (MASKED)
        lim = left - e >= 4 ? 4 : (left - e > 0 ? static_cast<int>(left - e) : 0);
      auto ld4 = [&](const float* p) {
        float4 x = *reinterpret_cast<const float4*>(p);
        if constexpr (MASKED) {
          if (lim < 1) x.x = 0.f;
          if (lim < 2) x.y = 0.f;
          if (lim < 3) x.z = 0.f;
          if (lim < 4) x.w = 0.f;
        }
        return x;
      };
      float2 wa[S], wb[S];
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const float4 w = i < sb ? ld4(sp + (w_off + i) * stg + e)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        wa[i] = make_float2(w.x, w.y);
        wb[i] = make_float2(w.z, w.w);
      }
#pragma unroll
      for (int u = 0; u < VPW; ++u) {
        if (vok[u]) {
          const float4 x = ld4(sp + vloc[u] * stg + e);
          const float2 xa = make_float2(x.x, x.y), xb = make_float2(x.z, x.w);
#pragma unroll
          for (int i = 0; i < S; ++i)
            acc[u][i] = __ffma2_rn(xb, wb[i], __ffma2_rn(xa, wa[i], acc[u][i]));
        }
      }
    };
    int ftiles = 0;
    for (int64_t c = 0; c < nch; ++c) {
      const int b = static_cast<int>(c % nstages);
      if (!mbar_wait(&full[b], static_cast<unsigned>((c / nstages) & 1), &s_abort)) {
        s_abort = 1;
        break;
      }
      const float* sp = stages + static_cast<size_t>(b) * ncp * stg;
      const int64_t left = s_end - (s_begin + c * stg);
      if (left >= stg) {
        // whole stage: groups of four tiles unrolled, so that a tile's loads
        // overlap the previous tile's products
        const int ntl = stg / 128;
        int tl = 0;
        for (; tl + 4 <= ntl; tl += 4) {
#pragma unroll
          for (int q = 0; q < 4; ++q) tile(sp, tl + q, left, std::integral_constant<bool, false>{});
          ftiles += 4;
          if (ftiles >= 8) {  // 16 products in each of the paired FP32 sums
            ftiles = 0;
            fold();
          }
        }
        for (; tl < ntl; ++tl) {
          tile(sp, tl, left, std::integral_constant<bool, false>{});
          if (++ftiles >= 8) {
            ftiles = 0;
            fold();
          }
        }
      } else {
        const int ntl = static_cast<int>((left + 127) / 128);
        for (int tl = 0; tl < ntl; ++tl) {
          tile(sp, tl, left, std::integral_constant<bool, true>{});
          if (++ftiles >= 8) {
            ftiles = 0;
            fold();
          }
        }
      }
      // this warp no longer reads the stage (__syncwarp orders the lanes'
      // reads before lane 0's release)
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
    fold();
    // warp sums (float-float) and the slot's partials
#pragma unroll
    for (int u = 0; u < VPW; ++u)
#pragma unroll
      for (int i = 0; i < S; ++i) {
        float h = fh[u][i], l = fl[u][i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          ff_merge(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
        if (lane == 0 && vok[u] && i < sb)
          partials[slot * kBlkStride + (g0 + vloc[u]) * kSMax + i] =
              static_cast<double>(h) + static_cast<double>(l);
      }
  }
  __syncthreads();
  // a wait gave up: report it (the solve reads the flag at its next status
  // check and fails the call) and still take part in the reduction, so that
  // the tickets return to zero
  if (s_abort && t == 0) atomicExch(&st->dev_error, kGramErrTimeout);

  // level 1: the last block of this run of slots sums the run in slot order
  const int64_t run = slot / kBlkRun, runs = (slots + kBlkRun - 1) / kBlkRun;
  const int64_t run_len = min(static_cast<int64_t>(kBlkRun), slots - run * kBlkRun);
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->dots_run[gx][run], 1u) == run_len - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = t; q < ng * kSMax; q += kGramTh) {
    const int qv = g0 + q / kSMax, qi = q % kSMax;
    if (qi >= sb) continue;
    const double* pr = partials + run * kBlkRun * kBlkStride + qv * kSMax + qi;
    double sum = 0.0;
    for (int r = 0; r < run_len; ++r) sum += __ldcg(pr + r * kBlkStride);
    partials[run * kBlkRun * kBlkStride + qv * kSMax + qi] = sum;
  }
  if (t == 0) st->dots_run[gx][run] = 0;
  // level 2: the last run of this group sums the runs in order
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->dots_group[gx], 1u) == runs - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = t; q < ng * kSMax; q += kGramTh) {
    const int qv = g0 + q / kSMax, qi = q % kSMax;
    if (qi >= sb) continue;
    const double* pr = partials + qv * kSMax + qi;
    double sum = 0.0;
#pragma unroll 8
    for (int64_t r = 0; r < runs; ++r) sum += __ldcg(pr + r * kBlkRun * kBlkStride);
    st->G[qv * kSMax + qi] = sum;
  }
  if (t == 0) st->dots_group[gx] = 0;
  // level 3: the last group runs the block's small steps
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->blk_groups, 1u) == static_cast<unsigned>(vg) - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (t == 0) st->blk_groups = 0;
  __syncthreads();  // the stages are no longer read: the space is block_ls's
  block_ls(st, k, sb, restart, scratch);
}

// ---------------------------------------------------------------------------
// Update pass: q_{k+1+i} = sum_{l <= i} (w_{l+1} - sum_v C[v][l] u_v) Rinv[l][i]
// over basis columns k+1.., in place; on the block that ends the cycle also
// V += sum_{v < J} y_v q_v (float-float V).  Warp tiles of 128 states: lane l
// owns the quad at 128 t + 4 l, so each warp reads one contiguous 512-byte run
// of every column per tile.
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(kBlkThreads)
    k_block_update(int64_t n, float* __restrict__ basis, int64_t ld, int k, int sb,
                   float2* __restrict__ V, const DevState* __restrict__ st) {
  const bool fin = st->bfin_k == k;
  if (!st->active && !fin) return;
  __shared__ float cf[kMaxBasis * kSMax];
  __shared__ float ri[kSMax * kSMax];
  __shared__ float yc[kBlkMaxV];
  const int nnew = st->bsb;
  const int J = fin ? st->jdone : 0;
  for (int t = threadIdx.x; t < (k + 1) * kSMax; t += blockDim.x) cf[t] = st->bC[t];
  for (int t = threadIdx.x; t < kSMax * kSMax; t += blockDim.x) ri[t] = st->bRinv[t];
  for (int t = threadIdx.x; t < kBlkMaxV; t += blockDim.x) yc[t] = fin ? st->bY[t] : 0.f;
  __syncthreads();
  (void)sb;
  const int64_t n_wt = (n + 127) / 128;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * (kBlkThreads / 32);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * (kBlkThreads / 32) + (threadIdx.x >> 5);
       t < n_wt; t += nw) {
    const int64_t s = t * 128 + 4 * (threadIdx.x & 31);
    if (s >= n) continue;
    if (s + 3 < n) {
      float4 w[S];
      float4 vacc = make_float4(0.f, 0.f, 0.f, 0.f);
      block_update_quad<S>(basis, ld, k, nnew, J, fin, cf, ri, yc, s, w, vacc);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        if (i < nnew) {
          *reinterpret_cast<float4*>(basis + static_cast<int64_t>(k + 1 + i) * ld + s) = w[i];
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
        float4* v4 = reinterpret_cast<float4*>(V + s);  // two float2 per float4
        const float4 va = v4[0], vb = v4[1];
        const ff r0 = ff_add_f(ff{va.x, va.y}, vacc.x), r1 = ff_add_f(ff{va.z, va.w}, vacc.y);
        const ff r2 = ff_add_f(ff{vb.x, vb.y}, vacc.z), r3 = ff_add_f(ff{vb.z, vb.w}, vacc.w);
        v4[0] = make_float4(r0.hi, r0.lo, r1.hi, r1.lo);
        v4[1] = make_float4(r2.hi, r2.lo, r3.hi, r3.lo);
      }
    } else {
      // ragged end of the vector: state by state, same order of operations
      for (int64_t e = s; e < n; ++e) {
        float w[S];
        float va = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i)
          w[i] = i < nnew ? basis[static_cast<int64_t>(k + 1 + i) * ld + e] : 0.f;
        for (int v = 0; v <= k; ++v) {
          const float u = basis[static_cast<int64_t>(v) * ld + e];
#pragma unroll
          for (int i = 0; i < S; ++i) w[i] = fmaf(-cf[v * kSMax + i], u, w[i]);
          if (fin && v < J) va = fmaf(yc[v], u, va);
        }
#pragma unroll
        for (int i = S - 1; i >= 0; --i) {
          float q = 0.f;
#pragma unroll
          for (int l = 0; l <= i; ++l) q = fmaf(ri[l * kSMax + i], w[l], q);
          w[i] = q;
        }
#pragma unroll
        for (int i = 0; i < S; ++i)
          if (i < nnew) {
            basis[static_cast<int64_t>(k + 1 + i) * ld + e] = w[i];
            if (fin && k + 1 + i < J) va = fmaf(yc[k + 1 + i], w[i], va);
          }
        if (fin) {
          const float2 v = V[e];
          const ff r = ff_add_f(ff{v.x, v.y}, va);
          V[e] = make_float2(r.hi, r.lo);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int64_t block_slots(int num_sms, int64_t n);

template <int S>
cudaError_t block_gram_launch(const Mat& A, const float* basis, int64_t ld, int k, int sb,
                              int restart, double* partials, DevState* st, cudaStream_t s) {
  const int nv = k + 1 + sb;
  const int vg = (nv + gram_vpg(S) - 1) / gram_vpg(S);
  // one CTA per SM in one wave; slot boundaries on whole stages
  int64_t slots = static_cast<int64_t>(A.num_sms) / vg;
  const int64_t cap = block_slots(A.num_sms, A.n);
  if (slots > cap) slots = cap;
  if (slots < 1) slots = 1;
  const int per_g = (nv + vg - 1) / vg;
  // copies per stage: the group's vectors, and W's when the group does not hold them
  const int ncp_max = vg == 1 ? nv : per_g + sb;
  // the largest stage (a multiple of 512 states) of which two fit: a bulk copy
  // costs about the same however long it is, so long copies stream faster
  int stg = static_cast<int>(kGramSmemBudget / (2 * sizeof(float) * ncp_max)) / 512 * 512;
  if (stg > kGramStageMax) stg = kGramStageMax;
  if (stg < 512) stg = 512;
  int64_t per = (A.n + slots - 1) / slots;
  per = (per + stg - 1) / stg * stg;
  const int64_t used = (A.n + per - 1) / per;  // <= slots
  const size_t stage_bytes = static_cast<size_t>(ncp_max) * stg * sizeof(float);
  int nstages = static_cast<int>(kGramSmemBudget / stage_bytes);
  if (nstages > kGramMaxStages) nstages = kGramMaxStages;
  size_t smem = static_cast<size_t>(nstages) * stage_bytes;
  const size_t ls = sizeof(double) * kMaxRestart * kMaxRestart;
  if (smem < ls) smem = ls;
  static bool attr = [] {
    cudaFuncSetAttribute(k_block_gram<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kGramSmemBudget));
    return true;
  }();
  (void)attr;
  // MDP_TEST_STALL_GRAM: the failure test of the bounded barrier waits
  const int stall = getenv("MDP_TEST_STALL_GRAM") ? 1 : 0;
  k_block_gram<S><<<dim3(static_cast<unsigned>(used), static_cast<unsigned>(vg)), kGramTh, smem,
                    s>>>(A.n, per, basis, ld, k, sb, restart, nstages, stg, stall, partials, st);
  return cudaGetLastError();
}

template <int S>
cudaError_t block_dots_launch(const Mat& A, const float* basis, int64_t ld, int k, int sb,
                              int restart, double* partials, DevState* st, cudaStream_t s) {
  // the register-staged form stays selectable for comparison (MDP_GRAM_REGS)
  static const bool regs = getenv("MDP_GRAM_REGS") != nullptr;
  if (!regs) return block_gram_launch<S>(A, basis, ld, k, sb, restart, partials, st, s);
  constexpr int VPG = (kBlkThreads / 32) * GramVpw<S>::value;
  const int nv = k + 1 + sb;
  const int vg = (nv + VPG - 1) / VPG;
  // about two blocks per SM in one wave (the register budget allows two):
  // each warp streams many tiles, and the reduction tail has few runs
  int64_t slots = static_cast<int64_t>(2 * A.num_sms) / vg;
  const int64_t cap = block_slots(A.num_sms, A.n);
  if (slots > cap) slots = cap;
  if (slots < 1) slots = 1;
  int64_t per = (A.n + slots - 1) / slots;
  per = (per + 127) / 128 * 128;
  const int64_t used = (A.n + per - 1) / per;  // <= slots
  constexpr size_t smem = gram_smem_bytes<S>();
  static bool attr = [] {
    cudaFuncSetAttribute(k_block_dots<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    return true;
  }();
  (void)attr;
  k_block_dots<S><<<dim3(static_cast<unsigned>(used), static_cast<unsigned>(vg)), kBlkThreads,
                    smem, s>>>(A.n, per, basis, ld, k, sb, restart, partials, st);
  return cudaGetLastError();
}

template <int S>
cudaError_t block_update_launch(const Mat& A, float* basis, int64_t ld, int k, int sb, float2* V,
                                DevState* st, cudaStream_t s) {
  static int occ = [] {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_block_update<S>, kBlkThreads, 0) !=
            cudaSuccess ||
        nb < 1)
      nb = 1;
    return nb;
  }();
  const int64_t warp_tiles = (A.n + 127) / 128;
  const int64_t want = (warp_tiles + kBlkThreads / 32 - 1) / (kBlkThreads / 32);
  const int64_t cap = static_cast<int64_t>(A.num_sms) * occ;
  const unsigned nb = static_cast<unsigned>(want < cap ? (want < 1 ? 1 : want) : cap);
  k_block_update<S><<<nb, kBlkThreads, 0, s>>>(A.n, basis, ld, k, sb, V, st);
  return cudaGetLastError();
}

// Chunk slots of the Gram pass: one per chunk, at most eight per SM (and
// kDotsMaxRuns runs of kBlkRun slots, the tickets of the two-level reduction).
int64_t block_slots(int num_sms, int64_t n) {
  const int64_t n_chunks = (n + kBlkChunk - 1) / kBlkChunk;
  const int64_t max_slots =
      static_cast<int64_t>(num_sms < kDotsMaxRuns ? num_sms : kDotsMaxRuns) * kBlkRun;
  return n_chunks < max_slots ? n_chunks : max_slots;
}

size_t block_partials_len(int num_sms, int64_t n) {
  return static_cast<size_t>(block_slots(num_sms, n)) * kBlkStride;
}

cudaError_t launch_block_dots(const Mat& A, const float* basis, int64_t ld, int k, int sb,
                              int s_blk, int restart, double* partials, DevState* st,
                              cudaStream_t s) {
  if (s_blk <= 4) return block_dots_launch<4>(A, basis, ld, k, sb, restart, partials, st, s);
  if (s_blk <= 6) return block_dots_launch<6>(A, basis, ld, k, sb, restart, partials, st, s);
  return block_dots_launch<8>(A, basis, ld, k, sb, restart, partials, st, s);
}

cudaError_t launch_block_update(const Mat& A, float* basis, int64_t ld, int k, int sb, int s_blk,
                                float2* V, DevState* st, cudaStream_t s) {
  if (s_blk <= 4) return block_update_launch<4>(A, basis, ld, k, sb, V, st, s);
  if (s_blk <= 6) return block_update_launch<6>(A, basis, ld, k, sb, V, st, s);
  return block_update_launch<8>(A, basis, ld, k, sb, V, st, s);
}

}  // namespace mdpk
