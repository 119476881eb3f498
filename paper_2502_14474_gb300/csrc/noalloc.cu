// mdp_bellman_noalloc: one FP32 Bellman backup on a caller's plain CSR that
// allocates no memory at all.
//
// Who needs it: a caller whose device memory is owned by somebody else -- a
// process that must stay inside a fixed memory budget accounted by its own
// allocator (a framework's caching allocator, or the admission budget of a
// request loop), or a latency-critical host thread that may not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device.
// Such a caller cannot create a handle (mdp_create allocates the converted
// matrix and work vectors), yet may still want one backup with its residual
// norms.  This entry point reads the caller's arrays as they are and keeps the
// only scratch it needs -- the per-tile partial norms and the completion
// ticket of the fixed-order reduction -- in a file-scope __device__ array.
//
// The scratch array is resolved once per device with cudaGetSymbolAddress (the
// array's name in host code is only a host-side stand-in, not a device
// address).  That happens on the first call on each device.  No call may be
// made on a stream that is being captured into a CUDA graph: every call reads
// its results back with a copy into host memory and a stream synchronisation,
// which capture does not allow, so a call on a capturing stream is rejected
// with MDP_ERR_ARG before anything is enqueued.  Every call on a device shares
// the one array: concurrent calls whose kernels overlap on the GPU race on it
// and must be serialised by the caller (one stream, or events).
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/mdp.h"
#include "mdp_internal.cuh"

// Sets the thread-local message returned by mdp_last_error (capi.cu).
void mdpk_set_last_error(const char* msg);

namespace {

constexpr int kTileStates = 256;      // one CTA of 256 threads per tile, a thread per state
constexpr int kMaxTiles = 16384;      // scratch holds one partial pair per tile
constexpr int kHeadBytes = 256;       // ticket, error flag, results; 256-byte aligned tail
constexpr size_t kScratchBytes = kHeadBytes + static_cast<size_t>(kMaxTiles) * 2 * sizeof(double);

struct Head {
  unsigned ticket;   // blocks done (must start at zero: cleared by every call)
  unsigned bad_csr;  // set when a row pointer or column index is invalid
  double res_inf;
  double res_2;
};

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The kernel's reduction helpers (mdpk::block_max_d / block_sum_d) reduce over
// mdpk::kThreads / 32 warps into `red`; the tile width must match them.
static_assert(kTileStates == mdpk::kThreads, "tile width must equal the reduction width");

__global__ void __launch_bounds__(kTileStates)
    k_bellman_plain(int64_t n, int32_t m, const int64_t* __restrict__ rp,
                    const int32_t* __restrict__ col, const float* __restrict__ val,
                    const float* __restrict__ g, float gamma, const float* __restrict__ V,
                    float* __restrict__ V_out, int32_t* __restrict__ pi_out,
                    float* __restrict__ r_out, unsigned char* __restrict__ scratch) {
  __shared__ double red[kTileStates / 32];
  Head* head = reinterpret_cast<Head*>(scratch);
  double* part = reinterpret_cast<double*>(scratch + kHeadBytes);
  const int64_t rows = n * m;
  const int64_t nnz = rp[rows];
  const int64_t s = static_cast<int64_t>(blockIdx.x) * kTileStates + threadIdx.x;
  double amax = 0.0, sq = 0.0;
  bool bad = false;
  if (s < n) {
    float best = 0.f;
    int arg = 0;
    for (int32_t a = 0; a < m; ++a) {
      const int64_t r = s * m + a;
      const int64_t b = rp[r], e = rp[r + 1];
      float acc = 0.f;
      if (b < 0 || e < b || e > nnz) {
        bad = true;
      } else {
        for (int64_t i = b; i < e; ++i) {
          const int32_t c = col[i];
          if (c < 0 || c >= n) {
            bad = true;
            continue;
          }
          acc = fmaf(val[i], V[c], acc);
        }
      }
      const float q = fmaf(gamma, acc, g[r]);
      if (a == 0 || q < best) {
        best = q;
        arg = a;
      }
    }
    const float rr = best - V[s];
    if (V_out) V_out[s] = best;
    if (pi_out) pi_out[s] = arg;
    if (r_out) r_out[s] = rr;
    amax = fabs(static_cast<double>(rr));
    sq = static_cast<double>(rr) * static_cast<double>(rr);
  }
  if (bad) atomicOr(&head->bad_csr, 1u);
  const double bmax = mdpk::block_max_d(amax, red);
  const double bsq = mdpk::block_sum_d(sq, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = bmax;
    part[2 * blockIdx.x + 1] = bsq;
  }
  if (mdpk::last_block(&head->ticket)) {
    double mx = 0.0, acc = 0.0;
    for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kTileStates) {
      mx = fmax(mx, __ldcg(part + 2 * i));
      acc += __ldcg(part + 2 * i + 1);
    }
    mx = mdpk::block_max_d(mx, red);
    acc = mdpk::block_sum_d(acc, red);
    if (threadIdx.x == 0) {
      head->res_inf = mx;
      head->res_2 = sqrt(acc);
    }
  }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_dev_ptr[kMaxDevices] = {nullptr};

mdp_status fail(mdp_status st, const char* msg) {
  mdpk_set_last_error(msg);
  return st;
}

}  // namespace

extern "C" mdp_status mdp_bellman_noalloc(int64_t n_states, int32_t n_actions,
                                          const int64_t* row_ptr, const int32_t* col,
                                          const float* val, const float* cost, double gamma,
                                          const float* V_in, float* V_out, int32_t* pi_out,
                                          float* r_out, double* res_inf, double* res_2,
                                          void* stream) {
  if (n_states <= 0 || n_actions <= 0)
    return fail(MDP_ERR_ARG, "mdp_bellman_noalloc: n_states and n_actions must be >= 1");
  if (!row_ptr || !col || !val || !cost || !V_in)
    return fail(MDP_ERR_ARG, "mdp_bellman_noalloc: NULL input array");
  if (V_out && V_out == V_in)
    return fail(MDP_ERR_ARG, "mdp_bellman_noalloc: V_out must not alias V_in");
  if (!(gamma >= 0.0 && gamma < 1.0))
    return fail(MDP_ERR_ARG, "mdp_bellman_noalloc: gamma must be in [0, 1)");
  const int64_t tiles = (n_states + kTileStates - 1) / kTileStates;
  if (tiles > kMaxTiles)
    return fail(MDP_ERR_ARG,
                "mdp_bellman_noalloc: n_states exceeds the static scratch limit of 4194304 states");
  if (n_states > INT64_MAX / n_actions)
    return fail(MDP_ERR_ARG, "mdp_bellman_noalloc: n_states * n_actions overflows");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess)
    return fail(MDP_ERR_CUDA, "mdp_bellman_noalloc: cudaStreamIsCapturing failed");
  if (cs != cudaStreamCaptureStatusNone)
    return fail(MDP_ERR_ARG, "mdp_bellman_noalloc: the stream is capturing a graph; this call "
                             "synchronises and cannot be captured");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(MDP_ERR_CUDA, "mdp_bellman_noalloc: no usable current device");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(MDP_ERR_CUDA, "mdp_bellman_noalloc: cudaGetSymbolAddress failed");
      }
      g_dev_ptr[dev] = p;
    }
    scratch = g_dev_ptr[dev];
  }
  // the ticket and the error flag must start at zero; results are rewritten
  if (cudaMemsetAsync(scratch, 0, kHeadBytes, s) != cudaSuccess)
    return fail(MDP_ERR_CUDA, "mdp_bellman_noalloc: clearing the scratch head failed");
  k_bellman_plain<<<static_cast<unsigned>(tiles), kTileStates, 0, s>>>(
      n_states, n_actions, row_ptr, col, val, cost, static_cast<float>(gamma), V_in, V_out,
      pi_out, r_out, static_cast<unsigned char*>(scratch));
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    // the message names the error, so a failure left pending by an earlier
    // unrelated call on this thread can be told apart from this launch failing
    static thread_local char msg[192];
    snprintf(msg, sizeof(msg), "mdp_bellman_noalloc: kernel launch reported %s (%s)",
             cudaGetErrorName(le), cudaGetErrorString(le));
    return fail(MDP_ERR_CUDA, msg);
  }
  Head head;
  if (cudaMemcpyAsync(&head, scratch, sizeof(Head), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(MDP_ERR_CUDA, "mdp_bellman_noalloc: reading the results failed");
  if (head.bad_csr)
    return fail(MDP_ERR_BAD_CSR,
                "mdp_bellman_noalloc: a row pointer or column index is out of range");
  if (res_inf) *res_inf = head.res_inf;
  if (res_2) *res_2 = head.res_2;
  return MDP_OK;
}
