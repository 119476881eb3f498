// Gram-Schmidt dots h_i = <w, v_i>, i <= j, of the stored w = u_{j+1}
// (classical Gram-Schmidt, Saad 2003, Alg. 6.9): a pure stream over the j+2
// basis vectors of n floats each.
//
// Vector-major: a block stages one chunk of kDotsChunk states of w in shared
// memory, then each of its eight warps streams one basis vector (or 1/WPV of
// one when fewer than eight vectors remain, so that every warp has work) over
// that chunk with a register accumulator: no shuffle inside the streaming
// loop, one warp reduction per vector at the end.  Block b covers vectors
// [ (b % VG) * VPB, +VPB ) and chunks b / VG, b / VG + S, ... of the S chunk
// slots; consecutive blocks share a chunk, so w is fetched from DRAM once and
// served from L2 to the other vector groups.  The FP64 partial of slot y for
// vector i lands in partials[y * MAXB + i].  Two-level fixed-order reduction:
// the last block of each run of eight slots (a ticket per run and group) sums
// the run in slot order into the run's first slot, and the last run of each
// group (a ticket per group) sums the runs in order and scales the result.
// Results are deterministic, and no single block has to read every partial
// (at 1024 slots that read cost about 8 us of L2 round trips per launch).
// Included by one translation unit.
#pragma once

#include "launch.h"
#include "mdp_internal.cuh"

namespace mdpk {

constexpr int kDotsThreads = 256;
constexpr int kDotsChunk = 4096;  // states of w staged per block (16 KB)
constexpr int kDotsRun = 8;       // chunk slots per first-level reduction

template <int MAXB, int WPV>
__global__ void __launch_bounds__(kDotsThreads)
    k_gs_dots(int64_t n, int64_t n_chunks, int vg, const float* __restrict__ basis, int64_t ld,
              int j, int out_h2, double* __restrict__ partials, DevState* __restrict__ st) {
  if (!st->active) return;
  constexpr int NW = kDotsThreads / 32, VPB = NW / WPV, CH = kDotsChunk, STEP = 32 * WPV;
  __shared__ __align__(16) float wsm[CH];
  __shared__ float wred[NW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gx = static_cast<int>(blockIdx.x % vg);
  const int64_t slot = blockIdx.x / vg, slots = gridDim.x / vg;
  const int i = gx * VPB + warp / WPV;  // this warp's basis vector
  const int part = warp % WPV;          // and its share of the chunk
  const float* uw = basis + static_cast<int64_t>(j + 1) * ld;
  const float* bi = basis + static_cast<int64_t>(i <= j ? i : j) * ld;
  float acc = 0.f;
  for (int64_t c = slot; c < n_chunks; c += slots) {
    const int64_t c0 = c * CH;
    const int len = static_cast<int>(n - c0 < CH ? n - c0 : CH);
    __syncthreads();  // the previous chunk's readers are done with wsm
    for (int q = threadIdx.x; q < CH / 4; q += kDotsThreads) {
      const int e = 4 * q;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e + 3 < len) {
        v = *reinterpret_cast<const float4*>(uw + c0 + e);
      } else if (e < len) {
        v.x = uw[c0 + e];
        if (e + 1 < len) v.y = uw[c0 + e + 1];
        if (e + 2 < len) v.z = uw[c0 + e + 2];
      }
      reinterpret_cast<float4*>(wsm)[q] = v;
    }
    __syncthreads();
    if (i > j) continue;
    const float4* b4 = reinterpret_cast<const float4*>(bi + c0);
    const float4* w4 = reinterpret_cast<const float4*>(wsm);
    const int nq = len >> 2;
    int q = part * 32 + lane;
    for (; q + 3 * STEP < nq; q += 4 * STEP) {
      float4 b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = __ldcs(b4 + q + u * STEP);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 w = w4[q + u * STEP];
        acc = fmaf(w.x, b[u].x, fmaf(w.y, b[u].y, fmaf(w.z, b[u].z, fmaf(w.w, b[u].w, acc))));
      }
    }
    for (; q < nq; q += STEP) {
      const float4 b = __ldcs(b4 + q);
      const float4 w = w4[q];
      acc = fmaf(w.x, b.x, fmaf(w.y, b.y, fmaf(w.z, b.z, fmaf(w.w, b.w, acc))));
    }
    if (part == 0 && lane == 0)  // ragged tail of the last chunk, in state order
      for (int e = 4 * nq; e < len; ++e) acc = fmaf(wsm[e], bi[c0 + e], acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) wred[warp] = acc;
  __syncthreads();
  if (threadIdx.x < VPB) {
    const int ii = gx * VPB + threadIdx.x;
    if (ii <= j) {
      double s = 0.0;
      for (int p = 0; p < WPV; ++p) s += static_cast<double>(wred[threadIdx.x * WPV + p]);
      partials[slot * MAXB + ii] = s;
    }
  }
  __shared__ bool s_last;
  // level 1: the last block of this run of slots sums the run, in slot order
  const int64_t run = slot / kDotsRun, runs = (slots + kDotsRun - 1) / kDotsRun;
  const int64_t run_len = min(static_cast<int64_t>(kDotsRun), slots - run * kDotsRun);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->dots_run[gx][run], 1u) == run_len - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < VPB) {
    const int d = gx * VPB + threadIdx.x;
    if (d <= j) {
      const double* pr = partials + run * kDotsRun * MAXB + d;
      double v[kDotsRun];
#pragma unroll
      for (int k = 0; k < kDotsRun; ++k) v[k] = k < run_len ? __ldcg(pr + k * MAXB) : 0.0;
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < kDotsRun; ++k) s += v[k];
      partials[run * kDotsRun * MAXB + d] = s;  // the run's first slot
    }
  }
  if (threadIdx.x == 0) st->dots_run[gx][run] = 0;
  // level 2: the last run of this vector group sums the runs in order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->dots_group[gx], 1u) == runs - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double* out = out_h2 ? st->h2 : st->H + static_cast<int64_t>(j) * kMaxBasis;
  for (int v = warp; v < VPB; v += NW) {
    const int d = gx * VPB + v;
    if (d > j) break;
    // lanes stride over the runs; a fixed shuffle tree combines them
    double s = 0.0;
    for (int64_t r = lane; r < runs; r += 32) s += __ldcg(partials + r * kDotsRun * MAXB + d);
    s = warp_sum_d(s);
    if (lane == 0) out[d] = s * st->scale[d];
  }
  if (threadIdx.x == 0) st->dots_group[gx] = 0;
}

// Grid: ceil((j+1)/VPB) vector groups x S chunk slots, S bounded by the
// partials buffer (num_sms * 8 slots of MAXB doubles each, MAXB <= 65) and by
// the run tickets (kDotsMaxRuns runs of kDotsRun slots).
template <int MAXB, int WPV>
cudaError_t dots_launch_w(const Mat& A, float* basis, int64_t ld, int j, int out_h2,
                          double* partials, DevState* st, cudaStream_t s) {
  constexpr int VPB = (kDotsThreads / 32) / WPV;
  const int vg = (j + 1 + VPB - 1) / VPB;
  const int64_t n_chunks = (A.n + kDotsChunk - 1) / kDotsChunk;
  const int64_t max_slots =
      static_cast<int64_t>(A.num_sms < kDotsMaxRuns ? A.num_sms : kDotsMaxRuns) * kDotsRun;
  const int64_t slots = n_chunks < max_slots ? n_chunks : max_slots;
  k_gs_dots<MAXB, WPV><<<static_cast<unsigned>(slots * vg), kDotsThreads, 0, s>>>(
      A.n, n_chunks, vg, basis, ld, j, out_h2, partials, st);
  return cudaGetLastError();
}

template <int MAXB>
cudaError_t dots_launch(const Mat& A, float* basis, int64_t ld, int j, int out_h2,
                        double* partials, DevState* st, cudaStream_t s) {
  // eight warps per block: one vector each once j+1 >= 8, else split the chunk
  if (j + 1 >= 5) return dots_launch_w<MAXB, 1>(A, basis, ld, j, out_h2, partials, st, s);
  if (j + 1 >= 3) return dots_launch_w<MAXB, 2>(A, basis, ld, j, out_h2, partials, st, s);
  if (j + 1 == 2) return dots_launch_w<MAXB, 4>(A, basis, ld, j, out_h2, partials, st, s);
  return dots_launch_w<MAXB, 8>(A, basis, ld, j, out_h2, partials, st, s);
}

inline cudaError_t dots_entry(const Mat& A, float* basis, int64_t ld, int j, int restart,
                              int out_h2, double* partials, DevState* st, cudaStream_t s) {
  if (restart + 1 <= 32) return dots_launch<32>(A, basis, ld, j, out_h2, partials, st, s);
  return dots_launch<kMaxBasis>(A, basis, ld, j, out_h2, partials, st, s);
}

}  // namespace mdpk
