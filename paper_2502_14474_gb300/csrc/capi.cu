// C ABI of the solver (include/mdp.h): handle management and the host-side
// drivers of policy evaluation (restarted GMRES) and inexact policy iteration.
//
// The host enqueues kernels asynchronously and synchronises only where a
// decision needs a scalar: once per outer iteration (the Bellman residual)
// and once per GMRES restart cycle (its step count and convergence flag).
// Within a cycle the kernels decide on the device (DevState::active).
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mdp.h"
#include "launch.h"

using namespace mdpk;

namespace {

thread_local std::string g_err;

mdp_status fail(mdp_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mdp_status fail(mdp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// NVTX range over a scope: the phases of a call appear by name in a profiler's
// timeline (nsys, ncu --nvtx); without a profiler attached the calls do nothing.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Prefix of DevState that the host reads back after a synchronisation.
struct StatusHead {
  unsigned counter[kNumCounters];
  double res_inf;
  double res_2;
  int active, jdone, converged, breakdown, restart, target_rel;
  double eta, target, beta, est;
  int nspmv, bfin_k;
  int dev_error, dev_error_pad;
};
static_assert(offsetof(StatusHead, est) == offsetof(DevState, est), "DevState prefix layout");
static_assert(offsetof(StatusHead, bfin_k) == offsetof(DevState, bfin_k), "DevState prefix layout");
static_assert(offsetof(StatusHead, dev_error) == offsetof(DevState, dev_error),
              "DevState prefix layout");
constexpr size_t kHeadBytes = sizeof(StatusHead);

struct ProfRec {
  int kind;
  int j;          // Arnoldi step of K2/K3 launches, -1 otherwise
  bool skipped;   // the launch returned at once (its GMRES cycle was over)
  double bytes;
  cudaEvent_t a, b;
};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> free_ev;
  std::vector<ProfRec> pending;
  mdp_profile_t agg;
  std::vector<float> samples[MDP_PROF_KINDS];  // per-launch durations of the timed launches
};

// Nearest-rank percentile q (0 < q <= 1) of v (reorders v).
double percentile(std::vector<float>& v, double q) {
  if (v.empty()) return 0.0;
  size_t k = static_cast<size_t>(std::ceil(q * static_cast<double>(v.size())));
  k = k < 1 ? 0 : k - 1;
  if (k >= v.size()) k = v.size() - 1;
  std::nth_element(v.begin(), v.begin() + static_cast<std::ptrdiff_t>(k), v.end());
  return v[k];
}

}  // namespace

// Message hook for entry points defined in other translation units.
void mdpk_set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct mdp_s {
  int device = 0;
  Mat A;
  bool broken = false;
  std::atomic<int> cancel{0};
  // owned device memory
  void* rp = nullptr;
  uint32_t* pk = nullptr;   // packed col/val (groups of 4 entries, 32 bytes)
  uint32_t* pk_am = nullptr;  // action-major policy copy (short rows), same format
  float* val_lo = nullptr;
  float* g = nullptr;
  float* g_lo = nullptr;
  void* val16 = nullptr;
  uint4* lpk = nullptr;     // packed 16-bit inner copy (band < 2^15)
  float* row_scale = nullptr;
  float2* V = nullptr;      // float-float iterate
  float2* W1 = nullptr;     // float-float scratch (mdp_bellman input)
  float2* W2 = nullptr;     // float-float scratch (mdp_bellman output)
  int32_t* pi = nullptr;    // policy buffer
  float* basis = nullptr;   // (restart_cap + 1) x ld
  int64_t ld = 0;
  int restart_cap = 0;
  float* d0 = nullptr;      // Richardson vectors (BiCGStab: x, r)
  float* d1 = nullptr;
  float* bt = nullptr;      // BiCGStab t = A s
  double* partials = nullptr;
  double* bpart = nullptr;  // s-step Gram pass partials (allocated on first use)
  size_t bpart_len = 0;     // doubles
  double* bnorm = nullptr;  // fused-batch residual partials (allocated on first use)
  size_t bnorm_len = 0;     // doubles
  DevState* st = nullptr;
  int* flag = nullptr;      // policy range check
  StatusHead* head = nullptr;  // pinned host mirror
  size_t bytes = 0;
  // analysis
  int64_t band = 0;
  int32_t min_len = 0, max_len = 0;
  int aligned = 0;
  int32_t store_t = MDP_F32;
  int neg = 0;  // MDP_FLAG_MAXIMIZE: costs are -rewards, V is kept as -V
  int32_t val_t = MDP_F32;
  Prof prof;
  int64_t launches = 0;
  cudaStream_t home = nullptr;   // stream of mdp_create: device memory is allocated in its order
  cudaEvent_t done_ev = nullptr; // recorded at the end of every call: destroy waits on it
  // captured GMRES restart cycles, replayed with one launch each
  struct CycleGraph {
    int steps;
    bool lp;
    int cgs2;
    int sblk;
    const int32_t* pi;
    cudaGraphExec_t exec;
  };
  std::vector<CycleGraph> graphs;
  int64_t eager_cycles = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

#define CK(h, call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      if (h) (h)->broken = true;                                                         \
      return fail(MDP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
    }                                                                                    \
  } while (0)

// Device memory comes from a stream-ordered pool that the library owns, one
// per device (cudaMemPoolCreate; cudaMallocFromPoolAsync / cudaFreeAsync):
// creating and destroying handles does not synchronise the device, so handles
// of concurrent solves (batch, serving) come and go while other streams keep
// running.  The pool keeps freed memory mapped (no release threshold): a
// handle created after another was destroyed reuses its pages instead of
// mapping new ones, which costs milliseconds per GB.  mdp_pool_trim hands
// cached memory back to the device.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {nullptr};

cudaMemPool_t device_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
      cudaGetLastError();
    g_pool[dev] = p;
  }
  return g_pool[dev];
}

cudaError_t pool_alloc(int dev, void** q, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = device_pool(dev);
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(q, bytes < 16 ? 16 : bytes, pool, s);
}

template <typename T>
cudaError_t dalloc(mdp_s* h, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = pool_alloc(h->device, &q, bytes, h->home);
  if (e == cudaSuccess) {
    *p = static_cast<T*>(q);
    h->bytes += bytes;
  }
  return e;
}

// One non-blocking stream per device on which handles are freed after their
// last call's completion event.
std::mutex g_free_mu;
cudaStream_t g_free_stream[64] = {nullptr};

cudaStream_t free_stream(int dev) {
  std::lock_guard<std::mutex> lk(g_free_mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!g_free_stream[dev]) {
    if (cudaStreamCreateWithFlags(&g_free_stream[dev], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g_free_stream[dev] = nullptr;
    }
  }
  return g_free_stream[dev];
}

// ---- profiling -------------------------------------------------------------
cudaEvent_t ev_get(mdp_s* h) {
  if (!h->prof.free_ev.empty()) {
    cudaEvent_t e = h->prof.free_ev.back();
    h->prof.free_ev.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Run one library launch call `f` (which issues `nlaunch` kernels) of the
// given kind; with timing on, bracket it by events on the same stream.
template <class F>
cudaError_t run(mdp_s* h, cudaStream_t s, int kind, int nlaunch, double bytes, int j, F f) {
  h->launches += nlaunch;
  if (!h->prof.on) return f();
  ProfRec r{kind, j, false, bytes, ev_get(h), ev_get(h)};
  if (!r.a || !r.b) return f();
  cudaEventRecord(r.a, s);
  cudaError_t e = f();
  cudaEventRecord(r.b, s);
  h->prof.pending.push_back(r);
  return e;
}

// Accumulate every pending record (their events must be complete).
void prof_flush(mdp_s* h) {
  for (ProfRec& r : h->prof.pending) {
    if (r.skipped) {
      h->prof.agg.skipped[r.kind] += 1;
    } else {
      float ms = 0.f;
      cudaEventSynchronize(r.b);
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        h->prof.agg.ms[r.kind] += ms;
        h->prof.agg.launches[r.kind] += 1;
        h->prof.samples[r.kind].push_back(ms);
        h->prof.agg.bytes[r.kind] += r.bytes;
      } else {
        cudaGetLastError();
      }
    }
    h->prof.free_ev.push_back(r.a);
    h->prof.free_ev.push_back(r.b);
  }
  h->prof.pending.clear();
}

// ---- algorithmic bytes per launch (gathers of the value vector excluded) ----
double rp_bytes(const Mat& A) { return A.uniform_len > 0 ? 0.0 : (A.idx64 ? 8.0 : 4.0); }
double policy_len(const Mat& A) {
  return A.uniform_len > 0 ? A.uniform_len : static_cast<double>(A.nnz) / A.rows;
}
// Row-pointer bytes and entries per policy row as the policy-row kernels read
// them (the action-major copy has uniform rows of am_len entries).
double prp_bytes(const Mat& A) { return A.am_len > 0 ? 0.0 : rp_bytes(A); }
double ppolicy_len(const Mat& A) { return A.am_len > 0 ? A.am_len : policy_len(A); }
double bytes_bellman(const Mat& A, bool ff, bool v_out) {
  const double n = A.n, rows = A.rows, nnz = A.nnz;
  const double vb = ff ? 8.0 : 4.0;
  return nnz * (8.0 + (A.val_lo ? 4.0 : 0.0)) + rows * (rp_bytes(A) + 4.0 + (A.g_lo ? 4.0 : 0.0)) +
         n * (vb + 4.0 + 4.0 + (v_out ? vb : 0.0));
}
double bytes_policy_resid(const Mat& A) {
  const double n = A.n;
  return n * (4.0 + 2.0 * prp_bytes(A) +
              ppolicy_len(A) * (8.0 + (A.val_lo && !A.am_len ? 4.0 : 0.0)) + 4.0 +
              (A.g_lo ? 4.0 : 0.0) + 8.0 + 4.0);
}
double bytes_spmv(const Mat& A, bool lp) {
  const double n = A.n;
  const double per_entry = lp ? (A.lpk ? 4.0 : 6.0) : 8.0;
  const double row_scale = (lp && !A.lpk) ? 4.0 : 0.0;  // the packed copy renormalises on the fly
  return n * (4.0 + 2.0 * prp_bytes(A) + ppolicy_len(A) * per_entry + row_scale + 4.0 + 4.0);
}
double bytes_dots(const Mat& A, int j) { return 4.0 * A.n * (j + 2); }
double bytes_ortho(const Mat& A, int j, int cgs2) {
  const double n = A.n;
  const double one = 4.0 * (j + 1) * n + 8.0 * n;
  return cgs2 ? 2.0 * one + 4.0 * (j + 2) * n : one;
}
double bytes_update(const Mat& A, int J) { return 4.0 * J * A.n + 16.0 * A.n; }
// s-step block at step k with sb vectors: the Gram pass reads u_0..u_k and
// w_1..w_sb once; the update pass reads them again and writes the sb new
// vectors (plus 16 bytes per state of V read and written on the last block).
double bytes_block_gram(const Mat& A, int k, int sb) { return 4.0 * A.n * (k + 1 + sb); }
double bytes_block_update(const Mat& A, int k, int sb, bool fin) {
  return 4.0 * A.n * (k + 1 + 2 * sb) + (fin ? 16.0 * A.n : 0.0);
}
double bytes_richardson(const Mat& A, bool lp) {
  const double n = A.n;
  return n * (4.0 + 2.0 * prp_bytes(A) + ppolicy_len(A) * (4.0 + (lp ? 2.0 : 4.0)) +
              (lp ? 4.0 : 0.0) + 12.0);
}

void free_all(mdp_s* h) {
  void* ptrs[] = {h->rp, h->pk, h->pk_am, h->val_lo, h->g, h->g_lo, h->val16, h->lpk, h->row_scale,
                  h->V, h->W1, h->W2, h->pi, h->basis, h->d0, h->d1, h->bt, h->partials, h->bpart,
                  h->bnorm, h->st, h->flag};
  cudaStream_t fs = free_stream(h->device);
  if (fs && h->done_ev) cudaStreamWaitEvent(fs, h->done_ev, 0);
  for (void* p : ptrs)
    if (p) {
      if (fs) cudaFreeAsync(p, fs);
      else cudaFree(p);
    }
  if (h->done_ev) cudaEventDestroy(h->done_ev);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  free(h->head);
  for (ProfRec& r : h->prof.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : h->prof.free_ev) cudaEventDestroy(e);
}

#define ALLOC(h, p, bytes)                                                                      \
  do {                                                                                          \
    cudaError_t e_ = dalloc((h), &(p), (bytes));                                                \
    if (e_ != cudaSuccess) {                                                                    \
      cudaGetLastError();                                                                       \
      return fail(MDP_ERR_OOM, "device allocation of %zu bytes failed: %s", (size_t)(bytes), \
                  cudaGetErrorString(e_));                                                      \
    }                                                                                           \
  } while (0)

// ---- autotuner -----------------------------------------------------------------
// Schedules of the CSR kernels: lanes per row (vw) and the shared-memory window
// for banded matrices.  Candidates are timed on the float-float Bellman kernel
// (CUDA events, best of 3 after 2 warm-up launches); the winner is cached per
// process by matrix shape so that similar matrices are not re-tuned.
struct TuneKey {
  int64_t n_bucket, mean_x4, band_bucket;
  int32_t m, uniform_len, vec4, idx64;
  bool operator<(const TuneKey& o) const {
    return std::tie(n_bucket, mean_x4, band_bucket, m, uniform_len, vec4, idx64) <
           std::tie(o.n_bucket, o.mean_x4, o.band_bucket, o.m, o.uniform_len, o.vec4, o.idx64);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

int64_t log2_bucket(int64_t x) {
  int64_t b = 0;
  while (x > 1) {
    x >>= 1;
    ++b;
  }
  return b;
}

size_t partials_len(int num_sms) { return static_cast<size_t>(num_sms) * 8 * (kMaxBasis + 1); }

// Growth of the work buffers happens in the calling stream's order.
mdp_status ensure_basis(mdp_s* h, int restart, cudaStream_t s) {
  if (restart <= h->restart_cap && h->basis) return MDP_OK;
  const cudaStream_t home = h->home;
  h->home = s;
  if (h->basis) {
    cudaFreeAsync(h->basis, s);
    h->bytes -= static_cast<size_t>(h->restart_cap + 1) * h->ld * sizeof(float);
    h->basis = nullptr;
  }
  cudaError_t e = dalloc(h, &h->basis, static_cast<size_t>(restart + 1) * h->ld * sizeof(float));
  h->home = home;
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->restart_cap = 0;
    return fail(MDP_ERR_OOM, "device allocation of the GMRES basis failed");
  }
  h->restart_cap = restart;
  return MDP_OK;
}

// Mark the end of a call on stream s (mdp_destroy waits for the last mark).
void mark_done(mdp_s* h, cudaStream_t s) {
  if (h->done_ev) cudaEventRecord(h->done_ev, s);
}

// Records the completion mark on every exit path of an entry point.
struct DoneMark {
  mdp_s* h;
  cudaStream_t s;
  ~DoneMark() { mark_done(h, s); }
};

cudaError_t autotune(mdp_s* h, float* scratch_r, cudaStream_t s) {
  Mat& A = h->A;
  TuneKey key{log2_bucket(A.n), static_cast<int64_t>(4.0 * A.nnz / A.rows), log2_bucket(A.band + 1),
              A.m, A.uniform_len, A.vec4, A.idx64};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      A.vw = it->second.first;
      A.window = it->second.second;
      return cudaSuccess;
    }
  }
  std::vector<std::pair<int, int>> cand;
  const int window0 = A.window;
  for (int vw : {1, 2, 4, 8, 32}) {
    // the uniform fast path needs rows of exactly 4*vw aligned entries
    if (A.vec4 && A.uniform_len > 0 && vw <= 4 && A.uniform_len != 4 * vw && vw != 1) continue;
    cand.push_back({vw, window0});
    if (window0) cand.push_back({vw, 0});
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaMemsetAsync(h->V, 0, static_cast<size_t>(A.n) * sizeof(float2), s);
  float best = 1e30f;
  std::pair<int, int> pick{A.vw, A.window};
  for (auto c : cand) {
    A.vw = c.first;
    A.window = c.second;
    float t_best = 1e30f;
    for (int it = 0; it < 5 && err == cudaSuccess; ++it) {
      cudaEventRecord(e0, s);
      err = launch_bellman(A, true, h->V, nullptr, h->pi, scratch_r, h->partials, h->st, 0, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (it >= 2) t_best = std::min(t_best, ms);
    }
    if (err != cudaSuccess) break;
    if (t_best < best) {
      best = t_best;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  A.vw = pick.first;
  A.window = pick.second;
  if (err == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = pick;
  }
  return err;
}

mdp_status ensure_richardson(mdp_s* h, cudaStream_t s) {
  if (h->d0) return MDP_OK;
  const cudaStream_t home = h->home;
  h->home = s;
  cudaError_t e = dalloc(h, &h->d0, static_cast<size_t>(h->A.n) * sizeof(float));
  if (e == cudaSuccess) e = dalloc(h, &h->d1, static_cast<size_t>(h->A.n) * sizeof(float));
  h->home = home;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_OOM, "device allocation of the Richardson vectors failed");
  }
  return MDP_OK;
}

// BiCGStab vectors: x and r in the Richardson pair, p and v in W2 (n float2 =
// 2n floats, free during a solve), r^ = r0 in W1, and t of its own.
mdp_status ensure_bicgstab(mdp_s* h, cudaStream_t s) {
  mdp_status rc = ensure_richardson(h, s);
  if (rc != MDP_OK || h->bt) return rc;
  const cudaStream_t home = h->home;
  h->home = s;
  cudaError_t e = dalloc(h, &h->bt, static_cast<size_t>(h->A.n) * sizeof(float));
  h->home = home;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_OOM, "device allocation of the BiCGStab vector failed");
  }
  return MDP_OK;
}

// The s-step Gram pass's partial sums: one slot of kBlkMaxV x kSMax doubles
// per chunk slot (at most one slot per 1024 states).
mdp_status ensure_sstep(mdp_s* h, cudaStream_t s, size_t min_doubles = 0) {
  const size_t want = std::max(block_partials_len(h->A.num_sms, h->A.n), min_doubles);
  if (h->bpart && h->bpart_len >= want) return MDP_OK;
  const cudaStream_t home = h->home;
  h->home = s;
  if (h->bpart) {
    cudaFreeAsync(h->bpart, s);
    h->bytes -= h->bpart_len * sizeof(double);
    h->bpart = nullptr;
    h->bpart_len = 0;
  }
  cudaError_t e = dalloc(h, &h->bpart, want * sizeof(double));
  h->home = home;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_OOM, "device allocation of the s-step partials failed");
  }
  h->bpart_len = want;
  return MDP_OK;
}

// Residual partials of the fused batch kernels (two doubles per unit).
mdp_status ensure_bnorm(mdp_s* h, cudaStream_t s, size_t doubles) {
  if (h->bnorm && h->bnorm_len >= doubles) return MDP_OK;
  const cudaStream_t home = h->home;
  h->home = s;
  if (h->bnorm) {
    cudaFreeAsync(h->bnorm, s);
    h->bytes -= h->bnorm_len * sizeof(double);
    h->bnorm = nullptr;
    h->bnorm_len = 0;
  }
  cudaError_t e = dalloc(h, &h->bnorm, doubles * sizeof(double));
  h->home = home;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_OOM, "device allocation of the batch partials failed");
  }
  h->bnorm_len = doubles;
  return MDP_OK;
}

// Read the status prefix of the device state (synchronises the stream).
mdp_status read_head(mdp_s* h, cudaStream_t s, bool flush = true) {
  CK(h, cudaMemcpyAsync(h->head, h->st, kHeadBytes, cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (flush) prof_flush(h);
  if (h->head->dev_error) {
    // a kernel's bounded wait gave up: the work of that launch is incomplete;
    // the flag is cleared so that the handle stays usable
    const int code = h->head->dev_error;
    CK(h, cudaMemsetAsync(reinterpret_cast<char*>(h->st) + offsetof(DevState, dev_error), 0,
                          sizeof(int), s));
    CK(h, cudaStreamSynchronize(s));
    return fail(MDP_ERR_TIMEOUT, "a device wait exceeded its bound (code %d)", code);
  }
  return MDP_OK;
}

__global__ void k_set_cycle(DevState* st, int restart, int target_rel, double eta, double target,
                            int set_target) {
  st->restart = restart;
  st->target_rel = target_rel;
  st->eta = eta;
  if (set_target) st->target = target;
}

__global__ void k_check_policy(int64_t n, int32_t m, const int32_t* __restrict__ pi, int* flag) {
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t a = pi[s];
    if (a < 0 || a >= m) atomicOr(flag, 1);
  }
}

mdp_status set_cycle(mdp_s* h, int restart, int target_rel, double eta, double target,
                     int set_target, cudaStream_t s) {
  CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
       k_set_cycle<<<1, 1, 0, s>>>(h->st, restart, target_rel, eta, target, set_target);
       return cudaGetLastError();
     }));
  return MDP_OK;
}

mdp_status check_policy(mdp_s* h, const int32_t* pi, cudaStream_t s) {
  CK(h, cudaMemsetAsync(h->flag, 0, sizeof(int), s));
  unsigned nb = static_cast<unsigned>(std::min<int64_t>((h->A.n + 255) / 256, h->A.num_sms * 8));
  CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
       k_check_policy<<<nb, 256, 0, s>>>(h->A.n, h->A.m, pi, h->flag);
       return cudaGetLastError();
     }));
  int f = 0;
  CK(h, cudaMemcpyAsync(&f, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  if (f) return fail(MDP_ERR_ARG, "policy has an action outside [0, %d)", h->A.m);
  return MDP_OK;
}

// Enqueue the kernels of one restart cycle: `steps` Arnoldi steps (policy-row
// SpMV, Gram-Schmidt dots, orthogonalisation + Givens) and the solution update.
// Arnoldi steps j0 .. j1-1 of a cycle of `steps` steps.
cudaError_t enqueue_steps(mdp_s* h, const int32_t* pi, int j0, int j1, int steps, bool lp,
                          int cgs2, cudaStream_t s) {
  for (int j = j0; j < j1; ++j) {
    cudaError_t e = run(h, s, MDP_PROF_ARNOLDI_SPMV, 1, bytes_spmv(h->A, lp), j, [&] {
      return launch_arnoldi_spmv(h->A, lp, pi, h->basis, h->ld, j, 1.f, h->partials, h->st, s);
    });
    if (e != cudaSuccess) return e;
    e = run(h, s, MDP_PROF_ARNOLDI_DOTS, 1, bytes_dots(h->A, j), j, [&] {
      return launch_arnoldi_dots(h->A, h->basis, h->ld, j, steps, 0, h->partials, h->st, s);
    });
    if (e != cudaSuccess) return e;
    e = run(h, s, MDP_PROF_ARNOLDI_ORTHO, cgs2 ? 3 : 1, bytes_ortho(h->A, j, cgs2), j, [&] {
      return launch_arnoldi_ortho(h->A, h->basis, h->ld, j, steps, cgs2, h->partials, h->st, s);
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t enqueue_update(mdp_s* h, cudaStream_t s) {
  return run(h, s, MDP_PROF_GMRES_UPDATE, 1, 0.0, -1, [&] {
    return launch_gmres_update(h->A, h->basis, h->ld, h->V, h->st, s);
  });
}

// Blocks b0 .. b1-1 of an s-step cycle of `steps` steps with blocks of sblk
// vectors (k_sstep.cu): per block sb policy-row SpMVs of the monomial basis,
// the Gram pass (with the block's least-squares steps) and the update pass
// (which adds the solution update on the block that ends the cycle).
cudaError_t enqueue_blocks(mdp_s* h, const int32_t* pi, int b0, int b1, int steps, bool lp,
                           int sblk, cudaStream_t s) {
  for (int b = b0; b < b1; ++b) {
    const int k = b * sblk;
    if (k >= steps) break;
    const int sb = std::min(sblk, steps - k);
    for (int i = 0; i < sb; ++i) {
      cudaError_t e = run(h, s, MDP_PROF_ARNOLDI_SPMV, 1, bytes_spmv(h->A, lp), k + i, [&] {
        return launch_arnoldi_spmv(h->A, lp, pi, h->basis, h->ld, k + i, 0.f, h->partials, h->st,
                                   s);
      });
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = run(h, s, MDP_PROF_BLOCK_GRAM, 1, bytes_block_gram(h->A, k, sb), k, [&] {
      return launch_block_dots(h->A, h->basis, h->ld, k, sb, sblk, steps, h->bpart, h->st, s);
    });
    if (e != cudaSuccess) return e;
    e = run(h, s, MDP_PROF_BLOCK_UPDATE, 1, bytes_block_update(h->A, k, sb, false), k, [&] {
      return launch_block_update(h->A, h->basis, h->ld, k, sb, sblk, h->V, h->st, s);
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int n_blocks(int steps, int sblk) { return (steps + sblk - 1) / sblk; }

cudaError_t enqueue_cycle(mdp_s* h, const int32_t* pi, int steps, bool lp, int cgs2, int sblk,
                          cudaStream_t s) {
  if (sblk > 0) return enqueue_blocks(h, pi, 0, n_blocks(steps, sblk), steps, lp, sblk, s);
  const cudaError_t e = enqueue_steps(h, pi, 0, steps, steps, lp, cgs2, s);
  return e != cudaSuccess ? e : enqueue_update(h, s);
}

int64_t cycle_launches(int steps, int cgs2, int sblk) {
  if (sblk > 0) return static_cast<int64_t>(steps) + 2 * n_blocks(steps, sblk);
  return static_cast<int64_t>(steps) * (cgs2 ? 5 : 3) + 1;
}

// Below this many states a GMRES step takes a few microseconds and the launches
// of the steps past the end of a cycle (which return at once, but still pass
// through the GPU's launch queue) outweigh a host check: such cycles are
// enqueued kChunkSteps steps at a time, with a status read between chunks.
constexpr int64_t kChunkedBelow = int64_t(1) << 20;
constexpr int kChunkSteps = 8;

// The captured graph of a cycle configuration (captured once the handle has
// run four eager cycles, which also initialised every launcher); nullptr when
// capture is not possible (legacy default stream, profiling, or a capture error).
cudaGraphExec_t cycle_graph(mdp_s* h, const int32_t* pi, int steps, bool lp, int cgs2, int sblk,
                            cudaStream_t s) {
  // capture pays off for handles that run many cycles (long or repeated
  // solves); short-lived handles stay eager (instantiation costs ~a cycle)
  if (h->prof.on || s == nullptr || h->eager_cycles < 4 || getenv("MDP_NO_GRAPHS"))
    return nullptr;
  for (auto& g : h->graphs)
    if (g.steps == steps && g.lp == lp && g.cgs2 == cgs2 && g.sblk == sblk && g.pi == pi)
      return g.exec;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;  // the caller is capturing: stay eager inside its graph
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const int64_t launches = h->launches;
  cudaError_t e = enqueue_cycle(h, pi, steps, lp, cgs2, sblk, s);
  h->launches = launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && e2 == cudaSuccess && graph &&
      cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
    if (h->graphs.size() >= 8) {
      cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back({steps, lp, cgs2, sblk, pi, exec});
  } else {
    exec = nullptr;
    cudaGetLastError();
  }
  if (graph) cudaGraphDestroy(graph);
  return exec;
}

// One GMRES restart cycle on the current device residual (already in u_0 with
// the cycle begun by the kernel that produced it): `steps` Arnoldi steps and
// the solution update, replayed from a captured graph when possible; then the
// cycle's outcome is read back.  sblk > 0 runs the cycle in s-step blocks of
// sblk vectors.  *jdone: the steps the solution update used; *nspmv: the
// policy-row SpMVs the cycle ran (s-step: up to sblk - 1 more than *jdone).
mdp_status gmres_cycle(mdp_s* h, const int32_t* pi, int steps, bool lp, int cgs2, int sblk,
                       cudaStream_t s, int* jdone, int* converged, int* nspmv) {
  const size_t first = h->prof.pending.size();
  const bool chunked =
      h->A.n < kChunkedBelow && steps > kChunkSteps && !getenv("MDP_NO_CYCLE_CHUNKS");
  cudaGraphExec_t g = chunked ? nullptr : cycle_graph(h, pi, steps, lp, cgs2, sblk, s);
  if (chunked && sblk > 0) {
    const int per = std::max(1, kChunkSteps / sblk), nb = n_blocks(steps, sblk);
    for (int b0 = 0; b0 < nb; b0 += per) {
      const int b1 = std::min(nb, b0 + per);
      CK(h, enqueue_blocks(h, pi, b0, b1, steps, lp, sblk, s));
      if (b1 == nb) break;
      mdp_status rc = read_head(h, s, false);
      if (rc != MDP_OK) return rc;
      if (!h->head->active) break;
    }
  } else if (chunked) {
    for (int j0 = 0; j0 < steps; j0 += kChunkSteps) {
      const int j1 = std::min(steps, j0 + kChunkSteps);
      CK(h, enqueue_steps(h, pi, j0, j1, steps, lp, cgs2, s));
      if (j1 == steps) break;
      mdp_status rc = read_head(h, s, false);
      if (rc != MDP_OK) return rc;
      if (!h->head->active) break;
    }
    CK(h, enqueue_update(h, s));
  } else if (g) {
    CK(h, cudaGraphLaunch(g, s));
    h->launches += cycle_launches(steps, cgs2, sblk);
  } else {
    CK(h, enqueue_cycle(h, pi, steps, lp, cgs2, sblk, s));
    h->eager_cycles += 1;
  }
  const size_t upd = h->prof.pending.empty() ? 0 : h->prof.pending.size() - 1;
  mdp_status rc = read_head(h, s, false);
  if (rc != MDP_OK) return rc;
  *jdone = h->head->jdone;
  *converged = h->head->converged;
  *nspmv = h->head->nspmv;
  // launches of steps past the end of the cycle returned at once
  const int fin_k = h->head->bfin_k;
  for (size_t i = first; i < h->prof.pending.size(); ++i) {
    ProfRec& r = h->prof.pending[i];
    if (r.kind == MDP_PROF_BLOCK_GRAM || r.kind == MDP_PROF_BLOCK_UPDATE) {
      r.skipped = r.j > fin_k;
      if (r.kind == MDP_PROF_BLOCK_UPDATE && r.j == fin_k) r.bytes += 16.0 * h->A.n;
    } else if (sblk > 0 && r.kind == MDP_PROF_ARNOLDI_SPMV) {
      r.skipped = r.j >= *nspmv;
    } else if (r.j >= *jdone) {
      r.skipped = true;
    }
    if (sblk == 0 && i == upd && r.kind == MDP_PROF_GMRES_UPDATE) {
      r.bytes = bytes_update(h->A, *jdone);
      r.skipped = *jdone == 0;
    }
  }
  prof_flush(h);
  return MDP_OK;
}

bool dtype_ok_vec(mdp_dtype t) { return t == MDP_F32 || t == MDP_F64; }

int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p *= 2;
  return p;
}

int pow2_floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

}  // namespace

extern "C" {

const char* mdp_last_error(void) { return g_err.c_str(); }

mdp_status mdp_pool_trim(int32_t device, uint64_t keep_bytes, uint64_t* reserved_after) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_CUDA, "mdp_pool_trim: no CUDA device");
  }
  if (device < 0 || device >= count || device >= 64)
    return fail(MDP_ERR_ARG, "mdp_pool_trim: device %d out of range", device);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    pool = g_pool[device];
  }
  uint64_t reserved = 0;
  if (pool) {
    DeviceGuard dg(device);
    // frees of destroyed handles are queued on the library's free stream
    cudaStream_t fs = free_stream(device);
    if (fs && cudaStreamSynchronize(fs) != cudaSuccess)
      return fail(MDP_ERR_CUDA, "mdp_pool_trim: waiting for pending frees failed");
    if (cudaMemPoolTrimTo(pool, static_cast<size_t>(keep_bytes)) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) !=
            cudaSuccess) {
      cudaGetLastError();
      return fail(MDP_ERR_CUDA, "mdp_pool_trim: trimming the pool failed");
    }
  }
  if (reserved_after) *reserved_after = reserved;
  return MDP_OK;
}

const char* mdp_version(void) { return "mdp-gb300 0.1 (sm_103a)"; }

void mdp_default_opts(mdp_solve_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-9;
  o->inner_rtol = 0.1;
  o->restart = 30;
  o->max_outer = 1000;
  o->max_inner = 10000;
  o->inner = MDP_INNER_GMRES;
  o->cgs2 = 0;
  o->low_precision_inner = 0;
  o->inner_norm = 0;
  o->s_step = 6;
}

size_t mdp_bytes_required(int64_t n, int32_t m, int64_t nnz, mdp_dtype val_t, mdp_dtype store_t,
                          int32_t restart) {
  if (n <= 0 || m <= 0 || nnz < 0) return 0;
  const int64_t rows = n * m;
  const bool idx64 = nnz >= (int64_t(1) << 31);
  const int64_t ld = static_cast<int64_t>(round_up(static_cast<size_t>(n), 64));
  size_t b = 0;
  b += static_cast<size_t>(rows + 1) * (idx64 ? 8 : 4);
  b += static_cast<size_t>(nnz) * (4 + 4 + (val_t == MDP_F64 ? 4 : 0));
  b += static_cast<size_t>(rows) * 4 * 2;  // g (+ g_lo bound)
  // 16-bit copy: packed groups take 4 bytes per entry (2 for the column offset),
  // in the action-major order of short rows up to 1.25 nnz entries; row scales
  if (store_t == MDP_BF16 || store_t == MDP_F16)
    b += static_cast<size_t>(nnz + nnz / 4 + 4) * 4 + static_cast<size_t>(rows) * 4;
  // action-major policy copy of short rows: at most 1.25 nnz padded entries
  if (nnz < 12 * rows) b += static_cast<size_t>(nnz + nnz / 4 + 4) * 8;
  b += static_cast<size_t>(n) * (8 * 3 + 4 + 8 + 4);  // V, W1, W2, pi; d0, d1; BiCGStab t
  b += static_cast<size_t>(restart + 1) * ld * 4;
  b += sizeof(DevState) + (1 << 20);
  return b;
}

mdp_status mdp_create(mdp_t* out, int64_t n, int32_t m, const int64_t* row_ptr,
                      const int32_t* col, const void* val, mdp_dtype val_t, const void* cost,
                      mdp_dtype cost_t, double gamma, mdp_dtype store_t, void* stream,
                      uint64_t flags) {
  Range nvtx("mdp_create");
  if (!out) return fail(MDP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || m <= 0) return fail(MDP_ERR_ARG, "n_states and n_actions must be >= 1");
  if (n > (int64_t(1) << 31) - 1) return fail(MDP_ERR_ARG, "n_states must fit int32 columns");
  if (n > INT64_MAX / m) return fail(MDP_ERR_ARG, "n_states * n_actions overflows");
  if (!row_ptr || !col || !val || !cost) return fail(MDP_ERR_ARG, "NULL array argument");
  if (!dtype_ok_vec(val_t) || !dtype_ok_vec(cost_t))
    return fail(MDP_ERR_ARG, "val_t and cost_t must be MDP_F32 or MDP_F64");
  if (store_t != MDP_F32 && store_t != MDP_BF16 && store_t != MDP_F16)
    return fail(MDP_ERR_ARG, "store_t must be MDP_F32, MDP_BF16 or MDP_F16");
  if (!(gamma >= 0.0 && gamma < 1.0)) return fail(MDP_ERR_ARG, "gamma must be in [0, 1)");
  const bool host_in = (flags & MDP_FLAG_HOST_INPUT) != 0;
  const int neg = (flags & MDP_FLAG_MAXIMIZE) ? 1 : 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t rows = n * m;

  mdp_s* h = new mdp_s();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(MDP_ERR_CUDA, "no CUDA device");
  }
  h->home = s;
  if (cudaEventCreateWithFlags(&h->done_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(MDP_ERR_CUDA, "event creation failed");
  }
  auto bail = [&](mdp_status st) {
    free_all(h);
    delete h;
    return st;
  };
  int num_sms = 1;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, h->device);

  // nnz from the last row pointer
  int64_t nnz = 0;
  if (host_in) {
    nnz = row_ptr[rows];
  } else {
    if (cudaMemcpy(&nnz, row_ptr + rows, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(MDP_ERR_ARG, "row_ptr is not a readable device pointer"));
    }
  }
  if (nnz < rows) return bail(fail(MDP_ERR_NOT_STOCHASTIC, "nnz < n*m: some row is empty"));
  const int idx64 = nnz >= (int64_t(1) << 31) ? 1 : 0;

  // staging of host inputs
  const int64_t* rp_in = row_ptr;
  const int32_t* col_in = col;
  const void* val_in = val;
  const void* g_in = cost;
  void* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  auto free_tmp = [&]() {
    for (void*& p : tmp)
      if (p) {
        cudaFreeAsync(p, s);
        p = nullptr;
      }
  };
  const size_t vbytes = static_cast<size_t>(nnz) * (val_t == MDP_F64 ? 8 : 4);
  const size_t gbytes = static_cast<size_t>(rows) * (cost_t == MDP_F64 ? 8 : 4);
  // Host inputs in page-locked memory are read by the kernels in place over the
  // host link (mapped through the unified address space): no staging copy, and
  // each byte crosses the link once.  Other host memory is staged on the device.
  auto mapped = [](const void* p) -> const void* {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
  };
  bool zero_copy = false;
  if (host_in && !getenv("MDP_STAGE_HOST_INPUT")) {
    const void* mp[4] = {mapped(row_ptr), mapped(col), mapped(val), mapped(cost)};
    if (mp[0] && mp[1] && mp[2] && mp[3]) {
      zero_copy = true;
      rp_in = static_cast<const int64_t*>(mp[0]);
      col_in = static_cast<const int32_t*>(mp[1]);
      val_in = mp[2];
      g_in = mp[3];
    }
  }
  if (host_in && !zero_copy) {
    const size_t sz[4] = {static_cast<size_t>(rows + 1) * 8, static_cast<size_t>(nnz) * 4, vbytes,
                          gbytes};
    const void* src[4] = {row_ptr, col, val, cost};
    for (int i = 0; i < 4; ++i) {
      if (pool_alloc(h->device, &tmp[i], sz[i], s) != cudaSuccess) {
        cudaGetLastError();
        free_tmp();
        return bail(fail(MDP_ERR_OOM, "staging allocation failed"));
      }
      if (cudaMemcpyAsync(tmp[i], src[i], sz[i], cudaMemcpyHostToDevice, s) != cudaSuccess) {
        free_tmp();
        return bail(fail(MDP_ERR_CUDA, "host to device copy failed"));
      }
    }
    rp_in = static_cast<const int64_t*>(tmp[0]);
    col_in = static_cast<const int32_t*>(tmp[1]);
    val_in = tmp[2];
    g_in = tmp[3];
  }

#define CALLOC(p, bytes)                                                          \
  do {                                                                            \
    if (dalloc(h, &(p), (bytes)) != cudaSuccess) {                               \
      cudaGetLastError();                                                         \
      free_tmp();                                                                 \
      return bail(fail(MDP_ERR_OOM, "device allocation of %zu bytes failed",      \
                       (size_t)(bytes)));                                         \
    }                                                                             \
  } while (0)
#define CCK(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      free_tmp();                                                                 \
      return bail(fail(MDP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)));   \
    }                                                                             \
  } while (0)

  CALLOC(h->rp, static_cast<size_t>(rows + 1) * (idx64 ? 8 : 4));
  const int64_t padded = (nnz + 3) & ~int64_t(3);
  CALLOC(h->pk, static_cast<size_t>(padded) * 8);
  if (val_t == MDP_F64) CALLOC(h->val_lo, static_cast<size_t>(nnz) * 4);
  CALLOC(h->g, static_cast<size_t>(rows) * 4);
  if (cost_t == MDP_F64) CALLOC(h->g_lo, static_cast<size_t>(rows) * 4);
  PrepFlags* dflags = nullptr;
  CALLOC(dflags, sizeof(PrepFlags));
  PrepFlags init;
  memset(&init, 0, sizeof(init));
  init.min_len = 0x7fffffff;
  CCK(cudaMemcpyAsync(dflags, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  const double tol = (flags & MDP_FLAG_NO_VALIDATE) ? INFINITY : 1e-5;
  if (zero_copy) {
    // pack first (the one pass over the host's col/val), then check the rows
    // against the packed copy
    CCK(launch_pack(nnz, col_in, val_in, val_t == MDP_F64, h->pk, h->val_lo, num_sms, s));
    CCK(launch_prep_rows(n, m, nnz, rp_in, nullptr, nullptr, val_t == MDP_F64, h->pk, h->val_lo,
                         g_in, cost_t == MDP_F64, neg, tol, h->rp, idx64, h->g, h->g_lo, dflags,
                         num_sms, s));
  } else {
    CCK(launch_prep_rows(n, m, nnz, rp_in, col_in, val_in, val_t == MDP_F64, nullptr, nullptr,
                         g_in, cost_t == MDP_F64, neg, tol, h->rp, idx64, h->g, h->g_lo, dflags,
                         num_sms, s));
    CCK(launch_pack(nnz, col_in, val_in, val_t == MDP_F64, h->pk, h->val_lo, num_sms, s));
  }
  PrepFlags fl;
  CCK(cudaMemcpyAsync(&fl, dflags, sizeof(fl), cudaMemcpyDeviceToHost, s));
  CCK(cudaStreamSynchronize(s));
  cudaFreeAsync(dflags, s);
  h->bytes -= sizeof(PrepFlags);
  free_tmp();
  if (fl.bad_csr)
    return bail(fail(MDP_ERR_BAD_CSR, "row_ptr not monotone from 0 or a column outside [0, n)"));
  if (fl.nonfinite) return bail(fail(MDP_ERR_NONFINITE, "NaN or Inf in probabilities or costs"));
  if (fl.negative) return bail(fail(MDP_ERR_NOT_STOCHASTIC, "negative probability"));
  if (fl.not_stochastic)
    return bail(fail(MDP_ERR_NOT_STOCHASTIC,
                     "a row of P is empty or sums to 1 +- %.3g (max error %.3g)", tol,
                     fl.max_sum_err));

  Mat& A = h->A;
  A.n = n;
  A.rows = rows;
  A.nnz = nnz;
  A.m = m;
  A.idx64 = idx64;
  A.rp = h->rp;
  A.col = reinterpret_cast<const int32_t*>(h->pk);
  A.val = reinterpret_cast<const float*>(h->pk);
  A.val_lo = h->val_lo;
  A.g = h->g;
  A.g_lo = h->g_lo;
  A.gamma = gamma;
  A.num_sms = num_sms;
  h->min_len = fl.min_len;
  h->max_len = fl.max_len;
  h->band = static_cast<int64_t>(fl.band);
  h->aligned = fl.not_aligned ? 0 : 1;
  h->val_t = val_t;
  A.uniform_len = (fl.min_len == fl.max_len) ? fl.min_len : 0;
  // lanes per row: about 4 entries per lane with 16-byte loads for rows of 12+
  // entries whose starts are all 16-byte aligned, one entry per lane otherwise.
  // (With aligned starts every row splits the same way, so a row's summation
  // order depends only on its entries: identical rows give identical sums and
  // exact ties resolve to the lowest action.)
  // Rows of uniform length 4*VW (VW <= 4) with aligned starts take the
  // VW-rows-per-vector fast path; other rows of fewer than 24 entries on
  // average are read by one thread each in whole packed groups; longer rows
  // are split over lanes.
  const double mean = static_cast<double>(nnz) / static_cast<double>(rows);
  A.vec4 = (mean >= 12.0 && h->aligned) ? 1 : 0;
  int vw = pow2_floor(std::max(1, static_cast<int>(std::lround(A.vec4 ? mean / 4.0 : mean))));
  A.vw = std::min(32, std::max(1, vw));
  const bool fast = A.vec4 && fl.min_len == fl.max_len && (fl.min_len == 8 || fl.min_len == 16);
  if (!fast && mean < 24.0) A.vw = 1;
  if (fast) A.vw = fl.min_len / 4;
  A.band = h->band;
  // stage V in shared memory when the band window fits (2*band + 2*tile <= 16384
  // float-float slots) and the matrix is large enough to amortise the fills
  A.window = (h->band <= 7680 && n >= 16 * (2 * h->band + 1)) ? 1 : 0;
  if (getenv("MDP_NO_WINDOW")) A.window = 0;
  A.screen = getenv("MDP_FF_SCREEN") ? 1 : 0;

  h->store_t = store_t;
  h->neg = neg;
  A.store_t = store_t;
  const bool lp_store = store_t == MDP_BF16 || store_t == MDP_F16;
  // Short rows (one thread per row, no aligned 16-byte slices) read by the
  // policy-row kernels come from an action-major copy padded to the longest
  // row, when padding costs at most a quarter more entries: states that share
  // an action then read adjacent rows instead of one short row per 128-byte
  // line.  Not for FP64 probabilities (the copy has no low parts) nor for a
  // 16-bit copy that cannot be packed.
  const int64_t am_entries = rows * static_cast<int64_t>(fl.max_len);
  if (A.vw == 1 && !A.vec4 && fl.max_len > 0 && fl.max_len <= 16 && !h->val_lo &&
      am_entries <= nnz + nnz / 4 &&
      (!lp_store || (h->band < 32768 && !getenv("MDP_NO_LP_PACK"))) &&
      !getenv("MDP_NO_POLICY_COPY")) {
    const int64_t am_padded = (am_entries + 3) & ~int64_t(3);
    CALLOC(h->pk_am, static_cast<size_t>(am_padded) * 8);
    CCK(cudaMemsetAsync(h->pk_am, 0, static_cast<size_t>(am_padded) * 8, s));
    CCK(launch_build_am(A, h->pk_am, fl.max_len, s));
    A.pk_am = h->pk_am;
    A.am_len = fl.max_len;
  }
  if (lp_store) {
    CALLOC(h->row_scale, static_cast<size_t>(rows) * 4);
    if (h->band < 32768 && !getenv("MDP_NO_LP_PACK")) {
      // 16-byte groups of int16 column offsets and 16-bit values
      const int64_t lp_padded =
          A.am_len > 0 ? ((rows * static_cast<int64_t>(A.am_len) + 3) & ~int64_t(3)) : padded;
      CALLOC(h->lpk, static_cast<size_t>(lp_padded) * 4);
      CCK(cudaMemsetAsync(h->lpk, 0, static_cast<size_t>(lp_padded) * 4, s));
      CCK(launch_prep_lowp_packed(A, h->lpk, h->row_scale, store_t, s));
      A.lpk = h->lpk;
    } else {
      CALLOC(h->val16, static_cast<size_t>(padded) * 2);  // group loads read whole quads
      CCK(cudaMemsetAsync(h->val16, 0, static_cast<size_t>(padded) * 2, s));
      CCK(launch_prep_lowp(A, h->val16, h->row_scale, store_t, s));
      A.val16 = h->val16;
    }
    A.row_scale = h->row_scale;
  }

  // work memory
  h->ld = static_cast<int64_t>(round_up(static_cast<size_t>(n), 64));
  CALLOC(h->V, static_cast<size_t>(n) * sizeof(float2));
  CALLOC(h->W1, static_cast<size_t>(n) * sizeof(float2));
  CALLOC(h->W2, static_cast<size_t>(n) * sizeof(float2));
  CALLOC(h->pi, static_cast<size_t>(n) * sizeof(int32_t));
  CALLOC(h->partials, partials_len(num_sms) * sizeof(double));
  CALLOC(h->st, sizeof(DevState));
  CALLOC(h->flag, sizeof(int));
  CCK(cudaMemsetAsync(h->st, 0, sizeof(DevState), s));
  h->head = static_cast<StatusHead*>(malloc(kHeadBytes));
  if (!h->head) return bail(fail(MDP_ERR_OOM, "host allocation failed"));
  if (ensure_basis(h, 30, s) != MDP_OK) return bail(MDP_ERR_OOM);
  if (flags & MDP_FLAG_AUTOTUNE) CCK(autotune(h, h->basis, s));
  mark_done(h, s);
  CCK(cudaStreamSynchronize(s));
#undef CALLOC
#undef CCK
  *out = h;
  return MDP_OK;
}

void mdp_destroy(mdp_t h) {
  if (!h) return;
  DeviceGuard g(h->device);
  free_all(h);  // frees after the handle's last call completes, without a device sync
  delete h;
}

void mdp_cancel(mdp_t h) {
  if (h) h->cancel.store(1);
}

mdp_status mdp_info(mdp_t h, mdp_info_t* info) {
  if (!h || !info) return fail(MDP_ERR_ARG, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->n_states = h->A.n;
  info->n_rows = h->A.rows;
  info->nnz = h->A.nnz;
  info->n_actions = h->A.m;
  info->vec_width = h->A.vw;
  info->uniform_len = h->A.uniform_len;
  info->idx64 = h->A.idx64;
  info->band = h->band;
  info->has_low_precision = (h->val16 != nullptr || h->lpk != nullptr) ? 1 : 0;
  info->store_t = h->store_t;
  info->maximize = h->neg;
  info->window = h->A.window;
  info->ff_screen = bellman_screened(h->A) ? 1 : 0;
  info->device_bytes = h->bytes;
  info->gamma = h->A.gamma;
  return MDP_OK;
}

mdp_status mdp_last_cycle(mdp_t h, mdp_gmres_cycle_t* out) {
  static_assert(MDP_MAX_RESTART == kMaxRestart, "ABI restart cap");
  if (!h || !out) return fail(MDP_ERR_ARG, "NULL argument");
  DeviceGuard dg(h->device);
  memset(out, 0, sizeof(*out));
  const char* base = reinterpret_cast<const char*>(h->st);
  int J = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&J, base + offsetof(DevState, last_J), sizeof(int), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemcpy(&out->beta, base + offsetof(DevState, last_beta), sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&out->est, base + offsetof(DevState, last_est), sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(out->H, base + offsetof(DevState, Hraw), sizeof(out->H),
                 cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(out->y, base + offsetof(DevState, y), sizeof(out->y), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_CUDA, "mdp_last_cycle: reading the cycle record failed");
  }
  out->J = J;
  return MDP_OK;
}

mdp_status mdp_bellman(mdp_t h, const void* V_in, mdp_dtype v_t, void* V_out, int32_t* pi_out,
                       float* r_out, double* res_inf, double* res_2, void* stream) {
  Range nvtx("mdp_bellman");
  if (!h) return fail(MDP_ERR_ARG, "NULL handle");
  if (h->broken) return fail(MDP_ERR_CUDA, "handle is broken by an earlier CUDA error");
  if (!V_in) return fail(MDP_ERR_ARG, "V_in is NULL");
  if (!dtype_ok_vec(v_t)) return fail(MDP_ERR_ARG, "v_t must be MDP_F32 or MDP_F64");
  if (V_out && V_out == V_in) return fail(MDP_ERR_ARG, "V_out must not alias V_in");
  DeviceGuard dg(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DoneMark dm{h, s};
  if (v_t == MDP_F32) {
    // a maximising handle backs up -V_in (kept in W1) and negates V_out, r_out
    const void* vin = V_in;
    if (h->neg) {
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
           return launch_negate(h->A.n, V_in, h->W1, 0, h->A.num_sms, s);
         }));
      vin = h->W1;
    }
    CK(h, run(h, s, MDP_PROF_BELLMAN_F32, 1, bytes_bellman(h->A, false, V_out != nullptr), -1, [&] {
         return launch_bellman(h->A, false, vin, V_out, pi_out, r_out, h->partials, h->st, 0, s);
       }));
    if (h->neg && V_out)
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
                [&] { return launch_negate(h->A.n, V_out, V_out, 0, h->A.num_sms, s); }));
  } else {
    CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
              [&] { return launch_to_ff(h->A.n, V_in, 1, h->neg, h->W1, h->A.num_sms, s); }));
    CK(h, run(h, s, MDP_PROF_BELLMAN_FF, 1, bytes_bellman(h->A, true, V_out != nullptr), -1, [&] {
         return launch_bellman(h->A, true, h->W1, V_out ? h->W2 : nullptr, pi_out, r_out,
                               h->partials, h->st, 0, s);
       }));
    if (V_out)
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
                [&] { return launch_from_ff(h->A.n, h->W2, V_out, 1, h->neg, h->A.num_sms, s); }));
  }
  if (h->neg && r_out)
    CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
              [&] { return launch_negate(h->A.n, r_out, r_out, 0, h->A.num_sms, s); }));
  mark_done(h, s);
  if (res_inf || res_2) {
    mdp_status rc = read_head(h, s);
    if (rc != MDP_OK) return rc;
    if (res_inf) *res_inf = h->head->res_inf;
    if (res_2) *res_2 = h->head->res_2;
  }
  return MDP_OK;
}

mdp_status mdp_policy_eval(mdp_t h, const int32_t* pi, void* v_inout, mdp_dtype v_t, double tol,
                           int32_t restart, int32_t max_iters, mdp_eval_stats* stats,
                           void* stream) {
  Range nvtx("mdp_policy_eval");
  if (!h) return fail(MDP_ERR_ARG, "NULL handle");
  if (h->broken) return fail(MDP_ERR_CUDA, "handle is broken by an earlier CUDA error");
  if (!pi || !v_inout) return fail(MDP_ERR_ARG, "NULL argument");
  if (!dtype_ok_vec(v_t)) return fail(MDP_ERR_ARG, "v_t must be MDP_F32 or MDP_F64");
  if (restart < 1 || restart > kMaxRestart) return fail(MDP_ERR_ARG, "restart must be in [1, 64]");
  if (!(tol >= 0.0)) return fail(MDP_ERR_ARG, "tol must be >= 0");
  if (max_iters < 0) return fail(MDP_ERR_ARG, "max_iters must be >= 0");
  DeviceGuard dg(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a cancel request made before this call started (a server may publish the
  // handle to its cancel path before it calls in) is honoured here, not dropped
  if (h->cancel.exchange(0)) return fail(MDP_ERR_CANCELLED, "cancelled before the call started");
  DoneMark dm{h, s};
  mdp_status rc = check_policy(h, pi, s);
  if (rc != MDP_OK) return rc;
  rc = ensure_basis(h, restart, s);
  if (rc != MDP_OK) return rc;
  CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
       return launch_to_ff(h->A.n, v_inout, v_t == MDP_F64, h->neg, h->V, h->A.num_sms, s);
     }));
  rc = set_cycle(h, restart, 0, 0.0, tol, 1, s);
  if (rc != MDP_OK) return rc;
  mdp_eval_stats es;
  memset(&es, 0, sizeof(es));
  CK(h, run(h, s, MDP_PROF_POLICY_RESID, 1, bytes_policy_resid(h->A), -1, [&] {
       return launch_policy_residual(h->A, pi, h->V, h->basis, h->partials, h->st, s);
     }));
  es.policy_sweeps = 1;
  rc = read_head(h, s);
  if (rc != MDP_OK) return rc;
  double res = h->head->res_2;
  mdp_status result = MDP_OK;
  while (!(res <= tol)) {
    if (es.iters >= max_iters) {
      result = fail(MDP_ERR_NOT_CONVERGED, "policy evaluation hit max_iters=%d (residual %.3e)",
                    max_iters, res);
      break;
    }
    if (h->cancel.exchange(0)) {  // the request is consumed by this call
      result = fail(MDP_ERR_CANCELLED, "cancelled");
      break;
    }
    const int steps = std::min(restart, max_iters - es.iters);
    rc = set_cycle(h, steps, 0, 0.0, tol, 1, s);
    if (rc != MDP_OK) return rc;
    int jdone = 0, conv = 0, nspmv = 0;
    rc = gmres_cycle(h, pi, steps, false, 0, 0, s, &jdone, &conv, &nspmv);
    if (rc != MDP_OK) return rc;
    es.iters += jdone;
    es.cycles += 1;
    es.policy_sweeps += jdone;
    // refinement residual of the updated iterate (also begins the next cycle)
    CK(h, run(h, s, MDP_PROF_POLICY_RESID, 1, bytes_policy_resid(h->A), -1, [&] {
         return launch_policy_residual(h->A, pi, h->V, h->basis, h->partials, h->st, s);
       }));
    es.policy_sweeps += 1;
    rc = read_head(h, s);
    if (rc != MDP_OK) return rc;
    const double prev = res;
    res = h->head->res_2;
    if (jdone == 0 && !(res < prev)) {
      result = fail(MDP_ERR_NOT_CONVERGED, "GMRES stagnated at residual %.3e", res);
      break;
    }
  }
  es.residual_2 = res;
  es.converged = res <= tol;
  CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
       return launch_from_ff(h->A.n, h->V, v_inout, v_t == MDP_F64, h->neg, h->A.num_sms, s);
     }));
  mark_done(h, s);
  CK(h, cudaStreamSynchronize(s));
  prof_flush(h);
  if (stats) *stats = es;
  return result;
}

mdp_status mdp_solve(mdp_t h, const mdp_solve_opts* opts_in, const void* V_init,
                     mdp_dtype vinit_t, double* V_out, int32_t* pi_out, mdp_solve_stats* stats,
                     void* stream) {
  Range nvtx("mdp_solve");
  if (!h) return fail(MDP_ERR_ARG, "NULL handle");
  if (h->broken) return fail(MDP_ERR_CUDA, "handle is broken by an earlier CUDA error");
  if (!V_out) return fail(MDP_ERR_ARG, "V_out is NULL");
  mdp_solve_opts o;
  if (opts_in) o = *opts_in;
  else mdp_default_opts(&o);
  if (V_init && !dtype_ok_vec(vinit_t)) return fail(MDP_ERR_ARG, "vinit_t must be F32 or F64");
  if (o.restart < 1 || o.restart > kMaxRestart) return fail(MDP_ERR_ARG, "restart in [1, 64]");
  if (!(o.tol >= 0.0) || !(o.inner_rtol > 0.0)) return fail(MDP_ERR_ARG, "bad tolerances");
  if (o.max_outer < 0 || o.max_inner < 1) return fail(MDP_ERR_ARG, "bad iteration limits");
  if (o.inner != MDP_INNER_GMRES && o.inner != MDP_INNER_RICHARDSON &&
      o.inner != MDP_INNER_BICGSTAB)
    return fail(MDP_ERR_ARG, "unknown inner solver");
  if (o.inner_norm != 0 && o.inner_norm != 1) return fail(MDP_ERR_ARG, "inner_norm is 0 or 1");
  if (o.s_step < 0 || o.s_step > kSMax) return fail(MDP_ERR_ARG, "s_step in [0, %d]", kSMax);
  if (o.s_step > 0 && o.cgs2) return fail(MDP_ERR_ARG, "cgs2 applies to s_step = 0 only");
  const bool lp = o.low_precision_inner != 0;
  if (lp && !h->val16 && !h->lpk)
    return fail(MDP_ERR_ARG, "low_precision_inner needs store_t BF16/F16");
  DeviceGuard dg(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->cancel.exchange(0)) return fail(MDP_ERR_CANCELLED, "cancelled before the call started");
  DoneMark dm{h, s};
  mdp_status rc = MDP_OK;
  if (o.inner == MDP_INNER_GMRES) {
    rc = ensure_basis(h, o.restart, s);
    if (rc == MDP_OK && o.s_step > 0) rc = ensure_sstep(h, s);
  } else if (o.inner == MDP_INNER_RICHARDSON) {
    rc = ensure_richardson(h, s);
  } else {
    rc = ensure_bicgstab(h, s);
  }
  if (rc != MDP_OK) return rc;
  const Mat& A = h->A;
  if (V_init)
    CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
         return launch_to_ff(A.n, V_init, vinit_t == MDP_F64, h->neg, h->V, A.num_sms, s);
       }));
  else CK(h, cudaMemsetAsync(h->V, 0, static_cast<size_t>(A.n) * sizeof(float2), s));
  rc = set_cycle(h, o.restart, 1, o.inner_rtol, 0.0, 0, s);
  if (rc != MDP_OK) return rc;

  mdp_solve_stats ss;
  memset(&ss, 0, sizeof(ss));
  const double policy_nnz =
      A.uniform_len > 0 ? static_cast<double>(A.n) * A.uniform_len
                        : static_cast<double>(A.nnz) / static_cast<double>(A.m);
  double transitions = 0.0;
  mdp_status result = MDP_OK;
  for (int k = 0;; ++k) {
    Range nvtx_outer("outer iteration");
    // improvement + high-precision residual (+ GMRES cycle start from r)
    float* r_dst = o.inner == MDP_INNER_GMRES ? h->basis : reinterpret_cast<float*>(h->W1);
    CK(h, run(h, s, MDP_PROF_BELLMAN_FF, 1, bytes_bellman(A, true, false), -1, [&] {
         return launch_bellman(A, true, h->V, nullptr, h->pi, r_dst, h->partials, h->st,
                               o.inner == MDP_INNER_GMRES ? 1 : 0, s);
       }));
    ss.bellman_sweeps += 1;
    transitions += static_cast<double>(A.nnz);
    rc = read_head(h, s);
    if (rc != MDP_OK) return rc;
    const double res = h->head->res_inf;
    if (ss.n_history < MDP_HISTORY) ss.residual_history[ss.n_history++] = res;
    ss.residual_inf = res;
    if (res <= o.tol) {
      ss.converged = 1;
      break;
    }
    if (!std::isfinite(res)) {
      result = fail(MDP_ERR_NOT_CONVERGED, "non-finite Bellman residual");
      break;
    }
    if (k >= o.max_outer) {
      result = fail(MDP_ERR_NOT_CONVERGED, "max_outer=%d reached (residual %.3e)", o.max_outer, res);
      break;
    }
    if (h->cancel.exchange(0)) {  // the request is consumed by this call
      result = fail(MDP_ERR_CANCELLED, "cancelled");
      break;
    }
    ss.outer_iters += 1;
    const double target = o.inner_rtol * res;
    int used = 0;
    Range nvtx_inner(o.inner == MDP_INNER_GMRES      ? "inner: gmres"
                     : o.inner == MDP_INNER_BICGSTAB ? "inner: bicgstab"
                                                     : "inner: richardson");
    if (o.inner == MDP_INNER_GMRES) {
      // the Bellman kernel began the first cycle: target = eta * res_inf
      for (;;) {
        const int steps = std::min(o.restart, o.max_inner - used);
        if (steps != o.restart) {
          rc = set_cycle(h, steps, 1, o.inner_rtol, 0.0, 0, s);
          if (rc != MDP_OK) return rc;
        }
        int jdone = 0, conv = 0, nspmv = 0;
        rc = gmres_cycle(h, h->pi, steps, lp, o.cgs2, o.s_step, s, &jdone, &conv, &nspmv);
        if (rc != MDP_OK) return rc;
        // work counts every policy SpMV the cycle ran (an s-step cycle that
        // ends inside a block ran the whole block's SpMVs)
        used += nspmv;
        ss.policy_sweeps += nspmv;
        transitions += policy_nnz * nspmv;
        if (conv || used >= o.max_inner || jdone == 0) break;
        if (h->cancel.load()) break;
        // refinement residual of the policy system, next cycle from it
        CK(h, run(h, s, MDP_PROF_POLICY_RESID, 1, bytes_policy_resid(A), -1, [&] {
             return launch_policy_residual(A, h->pi, h->V, h->basis, h->partials, h->st, s);
           }));
        ss.policy_sweeps += 1;
        transitions += policy_nnz;
        rc = read_head(h, s);
        if (rc != MDP_OK) return rc;
        if (!h->head->active) break;  // already below the target
        if (o.inner_norm == 1 && h->head->res_inf <= target) break;
      }
      if (o.restart != std::min(o.restart, o.max_inner)) {
        rc = set_cycle(h, o.restart, 1, o.inner_rtol, 0.0, 0, s);
        if (rc != MDP_OK) return rc;
      }
    } else if (o.inner == MDP_INNER_BICGSTAB) {
      // BiCGStab in correction form: (I - gamma P_pi) x = r from x = 0, then V += x,
      // stopping at ||r_k||_2 <= eta * ||T V - V||_inf.  Iterations (five launches
      // each) are enqueued eight at a time; every launch returns at once after the
      // solve met its target or broke down, so the host reads the status once per
      // batch.  A breakdown keeps the iterate reached so far.
      const float* rhat = reinterpret_cast<const float*>(h->W1);
      float* x = h->d0;
      float* r = h->d1;
      float* p = reinterpret_cast<float*>(h->W2);
      float* v = p + A.n;
      float* t = h->bt;
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
           return launch_bicg_begin(A.n, rhat, r, p, x, target, h->partials, h->st, A.num_sms,
                                    s);
         }));
      int executed = 0;
      while (used < o.max_inner) {
        const int batch = std::min(8, o.max_inner - used);
        const size_t first = h->prof.pending.size();
        for (int i = 0; i < batch; ++i) {
          const int k = executed + i;
          CK(h, run(h, s, MDP_PROF_BICGSTAB_SPMV, 1, bytes_richardson(A, false), k, [&] {
               return launch_bicg_spmv(A, h->pi, p, v, rhat, 0, h->partials, h->st, s);
             }));
          CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, k, [&] {
               return launch_bicg_s(A.n, p, v, r, x, h->partials, h->st, A.num_sms, s);
             }));
          CK(h, run(h, s, MDP_PROF_BICGSTAB_SPMV, 1, bytes_richardson(A, false), k, [&] {
               return launch_bicg_spmv(A, h->pi, r, t, r, 1, h->partials, h->st, s);
             }));
          CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, k, [&] {
               return launch_bicg_r(A.n, rhat, t, r, x, h->partials, h->st, A.num_sms, s);
             }));
          CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, k, [&] {
               return launch_bicg_p(A.n, r, v, p, h->st, A.num_sms, s);
             }));
        }
        rc = read_head(h, s, false);
        if (rc != MDP_OK) return rc;
        const int now = h->head->jdone;
        for (size_t i = first; i < h->prof.pending.size(); ++i)
          if (h->prof.pending[i].j >= now) h->prof.pending[i].skipped = true;
        prof_flush(h);
        ss.policy_sweeps += 2 * (now - executed);
        transitions += 2.0 * policy_nnz * (now - executed);
        used += now - executed;
        executed = now;
        if (!h->head->active) break;
        if (h->cancel.load()) break;
      }
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
                [&] { return launch_ff_axpy(A.n, h->V, x, A.num_sms, s); }));
    } else {
      // modified policy iteration in correction form: d_1 = r, d_{k+1} = r + gamma P_pi d_k;
      // V + d_k equals T_pi^k V, and ||d_{k+1} - d_k||_2 is the residual of d_k.
      // Sweeps are enqueued eight at a time; each returns at once once an earlier
      // one met the target, so the host reads the status once per batch.  Sweep k
      // reads d_(k&1) and writes d_((k+1)&1); the last one that ran wrote d_(e&1).
      const float* rsave = reinterpret_cast<const float*>(h->W1);
      float* dbuf[2] = {h->d0, h->d1};
      CK(h, cudaMemcpyAsync(dbuf[0], rsave, static_cast<size_t>(A.n) * sizeof(float),
                            cudaMemcpyDeviceToDevice, s));
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
                [&] { return launch_richardson_begin(h->st, target, s); }));
      used = 1;
      int executed = 0;
      while (used < o.max_inner) {
        const int batch = std::min(8, o.max_inner - used);
        const size_t first = h->prof.pending.size();
        for (int i = 0; i < batch; ++i) {
          const int k = executed + i;
          CK(h, run(h, s, MDP_PROF_RICHARDSON, 1, bytes_richardson(A, lp), k, [&] {
               return launch_richardson(A, lp, h->pi, rsave, dbuf[k & 1], dbuf[(k + 1) & 1],
                                        h->partials, h->st, s);
             }));
        }
        rc = read_head(h, s, false);
        if (rc != MDP_OK) return rc;
        const int now = h->head->jdone;
        for (size_t i = first; i < h->prof.pending.size(); ++i)
          if (h->prof.pending[i].j >= now) h->prof.pending[i].skipped = true;
        prof_flush(h);
        ss.policy_sweeps += now - executed;
        transitions += policy_nnz * (now - executed);
        used += now - executed;
        executed = now;
        if (!h->head->active) break;
        if (h->cancel.load()) break;
      }
      CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1, [&] {
           return launch_ff_axpy(A.n, h->V, dbuf[executed & 1], A.num_sms, s);
         }));
    }
    ss.inner_iters += used;
    if (ss.outer_iters - 1 < MDP_HISTORY) ss.inner_history[ss.outer_iters - 1] = used;
  }
  CK(h, run(h, s, MDP_PROF_OTHER, 1, 0.0, -1,
            [&] { return launch_from_ff(A.n, h->V, V_out, 1, h->neg, A.num_sms, s); }));
  if (pi_out)
    CK(h, cudaMemcpyAsync(pi_out, h->pi, static_cast<size_t>(A.n) * sizeof(int32_t),
                          cudaMemcpyDeviceToDevice, s));
  mark_done(h, s);
  CK(h, cudaStreamSynchronize(s));
  prof_flush(h);
  ss.transitions = transitions;
  if (stats) *stats = ss;
  return result;
}

mdp_status mdp_batch_solve(mdp_t const* hs, int32_t count, const mdp_solve_opts* opts,
                           double* const* V_out, int32_t* const* pi_out, mdp_solve_stats* stats,
                           mdp_status* status_out, int32_t n_streams) {
  Range nvtx("mdp_batch_solve");
  if (count < 0 || (count > 0 && (!hs || !V_out)))
    return fail(MDP_ERR_ARG, "mdp_batch_solve: bad arguments");
  if (n_streams == 0) n_streams = 8;
  if (n_streams < 1 || n_streams > 64)
    return fail(MDP_ERR_ARG, "mdp_batch_solve: n_streams must be in [1, 64]");
  for (int32_t i = 0; i < count; ++i)
    if (!hs[i] || !V_out[i]) return fail(MDP_ERR_ARG, "mdp_batch_solve: NULL handle or output");
  for (int32_t i = 0; i < count; ++i)
    for (int32_t k = i + 1; k < count && k < i + 1 + 4096; ++k)
      if (hs[i] == hs[k]) return fail(MDP_ERR_ARG, "mdp_batch_solve: a handle appears twice");
  std::vector<mdp_status> st(static_cast<size_t>(count), MDP_OK);
  std::vector<std::string> msg(static_cast<size_t>(count));
  // largest first (by nonzeros): a large MDP taken last would leave the other
  // workers idle while it runs alone; results do not depend on the order
  std::vector<int32_t> order(static_cast<size_t>(count));
  for (int32_t i = 0; i < count; ++i) order[static_cast<size_t>(i)] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return hs[a]->A.nnz > hs[b]->A.nnz; });
  std::atomic<int32_t> next{0};
  const int workers = std::min<int>(n_streams, std::max<int32_t>(count, 1));
  std::vector<std::thread> pool;
  std::vector<int> dev_err(static_cast<size_t>(workers), 0);
  int device = 0;
  cudaGetDevice(&device);
  for (int w = 0; w < workers; ++w) {
    pool.emplace_back([&, w]() {
      cudaSetDevice(device);
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        dev_err[w] = 1;
        return;
      }
      for (;;) {
        const int32_t k = next.fetch_add(1);
        if (k >= count) break;
        const int32_t i = order[static_cast<size_t>(k)];
        mdp_solve_stats one;
        st[i] = mdp_solve(hs[i], opts, nullptr, MDP_F64, V_out[i], pi_out ? pi_out[i] : nullptr,
                          &one, s);
        if (st[i] != MDP_OK) msg[i] = g_err;
        if (stats) stats[i] = one;
      }
      cudaStreamDestroy(s);
    });
  }
  for (auto& t : pool) t.join();
  for (int w = 0; w < workers; ++w)
    if (dev_err[w]) return fail(MDP_ERR_CUDA, "mdp_batch_solve: stream creation failed");
  mdp_status first = MDP_OK;
  for (int32_t i = 0; i < count; ++i) {
    if (status_out) status_out[i] = st[i];
    if (first == MDP_OK && st[i] != MDP_OK) {
      first = st[i];
      g_err = "mdp_batch_solve: MDP " + std::to_string(i) + ": " + msg[i];
    }
  }
  return first;
}

mdp_status mdp_batch_solve_fused(mdp_t const* hs, int32_t count, const mdp_solve_opts* opts_in,
                                 double* const* V_out, int32_t* const* pi_out,
                                 mdp_solve_stats* stats, mdp_status* status_out, void* stream) {
  Range nvtx("mdp_batch_solve_fused");
  if (count < 0 || (count > 0 && (!hs || !V_out)))
    return fail(MDP_ERR_ARG, "mdp_batch_solve_fused: bad arguments");
  if (count == 0) return MDP_OK;
  mdp_solve_opts o;
  if (opts_in) o = *opts_in;
  else mdp_default_opts(&o);
  if (o.restart < 1 || o.restart > kMaxRestart) return fail(MDP_ERR_ARG, "restart in [1, 64]");
  if (!(o.tol >= 0.0) || !(o.inner_rtol > 0.0)) return fail(MDP_ERR_ARG, "bad tolerances");
  if (o.max_outer < 0 || o.max_inner < 1) return fail(MDP_ERR_ARG, "bad iteration limits");
  if (o.inner != MDP_INNER_GMRES || o.cgs2 || o.low_precision_inner || o.s_step < 1 ||
      o.s_step > kSMax || (o.inner_norm != 0 && o.inner_norm != 1))
    return fail(MDP_ERR_ARG,
                "mdp_batch_solve_fused runs s-step GMRES (s_step 1..%d) on the FP32 probabilities",
                kSMax);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(MDP_ERR_CUDA, "no current device");
  std::unordered_set<mdp_t> seen;
  for (int32_t i = 0; i < count; ++i) {
    mdp_s* h = hs[i];
    if (!h || !V_out[i]) return fail(MDP_ERR_ARG, "mdp_batch_solve_fused: NULL handle or output");
    if (!seen.insert(h).second)
      return fail(MDP_ERR_ARG, "mdp_batch_solve_fused: a handle appears twice");
    if (h->device != dev)
      return fail(MDP_ERR_ARG, "mdp_batch_solve_fused: every handle must be on the current device");
    if (h->broken) return fail(MDP_ERR_CUDA, "mdp_batch_solve_fused: handle %d is broken", i);
    if (h->A.m > 64) return fail(MDP_ERR_ARG, "mdp_batch_solve_fused: at most 64 actions");
  }
  DeviceGuard dg(dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int R = o.restart, sblk = o.s_step;
  const int num_sms = hs[0]->A.num_sms;
  // per-MDP buffers, initial state and the device descriptors
  std::vector<BMdp> hd(static_cast<size_t>(count));
  std::vector<double> pnnz(static_cast<size_t>(count));
  for (int32_t i = 0; i < count; ++i) {
    mdp_s* h = hs[i];
    const Mat& A = h->A;
    BMdp& d = hd[static_cast<size_t>(i)];
    d.u_bell = batch_units_bellman(A.n, A.m);
    d.u_state = batch_units_state(A.n);
    d.u_gram = batch_units_gram(A.n);
    mdp_status rc = ensure_basis(h, R, s);
    if (rc == MDP_OK)
      rc = ensure_sstep(h, s, static_cast<size_t>(d.u_gram) * (kBlkMaxV * kSMax));
    if (rc == MDP_OK)
      rc = ensure_bnorm(h, s, 2 * static_cast<size_t>(std::max(d.u_bell, d.u_state)));
    if (rc == MDP_OK) rc = set_cycle(h, R, 1, o.inner_rtol, 0.0, 0, s);
    if (rc != MDP_OK) return rc;
    CK(h, cudaMemsetAsync(h->V, 0, static_cast<size_t>(A.n) * sizeof(float2), s));
    d.rp = A.rp;
    d.col = A.col;
    d.val = A.val;
    d.val_lo = A.val_lo;
    d.g = A.g;
    d.g_lo = A.g_lo;
    d.V = h->V;
    d.pi = h->pi;
    d.basis = h->basis;
    d.st = h->st;
    d.part = h->bnorm;
    d.bpart = h->bpart;
    d.n = A.n;
    d.ld = h->ld;
    d.m = A.m;
    d.idx64 = A.idx64;
    d.uniform_len = A.uniform_len;
    // rows of up to 64 entries: one packed group of 4 entries per lane, as many
    // lanes as the longest row has groups (2..16), so a row's loads are in
    // flight together; longer rows: the handle's lanes per row, entry by entry
    const int groups = (h->max_len + 3) / 4;
    d.grp = h->max_len <= 64 ? 1 : 0;
    d.vw = d.grp ? std::max(2, std::min(16, pow2_ceil(groups)))
                 : pow2_floor(std::min(32, std::max(1, A.vw)));
    d.tb = batch_bellman_tile(A.m);
    d.maxlen = h->max_len;
    d.gamma = static_cast<float>(A.gamma);
    d.gamma_hi = d.gamma;
    d.gamma_lo = static_cast<float>(A.gamma - static_cast<double>(d.gamma));
    pnnz[static_cast<size_t>(i)] =
        A.uniform_len > 0 ? static_cast<double>(A.n) * A.uniform_len
                          : static_cast<double>(A.nnz) / static_cast<double>(A.m);
  }
  // device buffers: descriptors, four work lists (Bellman, residual, and the
  // cycle's state-range and Gram units), the gathered status heads
  const size_t n4 = static_cast<size_t>(count);
  const size_t off_lists = round_up(n4 * sizeof(BMdp), 256);
  const size_t off_mdp = off_lists + round_up(4 * sizeof(BList), 256);
  const size_t off_first = off_mdp + round_up(4 * n4 * sizeof(int32_t), 256);
  const size_t off_heads = off_first + round_up(4 * (n4 + 1) * sizeof(int64_t), 256);
  const size_t total_bytes = off_heads + n4 * kHeadBytes;
  void* dbuf = nullptr;
  if (pool_alloc(dev, &dbuf, total_bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(MDP_ERR_OOM, "mdp_batch_solve_fused: device allocation failed");
  }
  unsigned char* db = static_cast<unsigned char*>(dbuf);
  const BMdp* d_mdps = reinterpret_cast<const BMdp*>(db);
  BList* d_lists = reinterpret_cast<BList*>(db + off_lists);
  std::vector<unsigned char> hbuf(off_heads);  // descriptors + lists, uploaded together
  std::vector<unsigned char> heads(n4 * kHeadBytes);
  memcpy(hbuf.data(), hd.data(), n4 * sizeof(BMdp));
  BList* hl = reinterpret_cast<BList*>(hbuf.data() + off_lists);
  int32_t* hmdp = reinterpret_cast<int32_t*>(hbuf.data() + off_mdp);
  int64_t* hfirst = reinterpret_cast<int64_t*>(hbuf.data() + off_first);
  for (int l = 0; l < 4; ++l) {
    hl[l].mdp = reinterpret_cast<const int32_t*>(db + off_mdp) + l * n4;
    hl[l].first = reinterpret_cast<const int64_t*>(db + off_first) + l * (n4 + 1);
    hl[l].count = 0;
    hl[l].total = 0;
  }
  mdp_status result = MDP_OK;
  cudaError_t ce = cudaSuccess;
  auto build = [&](int l, const std::vector<int32_t>& members, int kind) {
    int64_t t = 0;
    int32_t* mm = hmdp + l * n4;
    int64_t* ff = hfirst + l * (n4 + 1);
    for (size_t p = 0; p < members.size(); ++p) {
      const BMdp& d = hd[static_cast<size_t>(members[p])];
      mm[p] = members[p];
      ff[p] = t;
      t += kind == 0 ? d.u_bell : (kind == 1 ? d.u_state : d.u_gram);
    }
    ff[members.size()] = t;
    hl[l].count = static_cast<int32_t>(members.size());
    hl[l].total = t;
  };
  auto upload = [&]() {
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(db, hbuf.data(), off_heads, cudaMemcpyHostToDevice, s);
  };
  auto read_heads = [&]() {
    if (ce == cudaSuccess) ce = launch_batch_heads(d_mdps, count, kHeadBytes, db + off_heads, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(heads.data(), db + off_heads, n4 * kHeadBytes, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  };
  auto head = [&](int32_t i) -> const StatusHead& {
    return *reinterpret_cast<const StatusHead*>(heads.data() + static_cast<size_t>(i) * kHeadBytes);
  };
  // one restart cycle of every MDP in the inner phase: lists 2 (state units) and 3 (Gram units)
  auto enqueue_cycle_all = [&]() -> cudaError_t {
    for (int k = 0; k < R; k += sblk) {
      const int sb = std::min(sblk, R - k);
      for (int i = 0; i < sb; ++i) {
        cudaError_t e = launch_batch_spmv(d_mdps, d_lists + 2, k + i, num_sms, s);
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = launch_batch_gram(d_mdps, d_lists + 3, k, sb, num_sms, s);
      if (e != cudaSuccess) return e;
      e = launch_batch_update(d_mdps, d_lists + 2, k, sb, num_sms, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  cudaGraphExec_t cycle = nullptr;
  bool tried_graph = false;
  enum { kOuter = 0, kCont = 1, kInner = 2, kDone = 3 };
  std::vector<int> phase(n4, kOuter), outer(n4, 0), used(n4, 0);
  std::vector<double> target(n4, 0.0);
  std::vector<mdp_solve_stats> ss(n4);
  std::vector<mdp_status> st(n4, MDP_OK);
  std::vector<std::string> msg(n4);
  for (auto& x : ss) memset(&x, 0, sizeof(x));
  int remaining = count;
  auto finish_inner = [&](int32_t i) {
    mdp_solve_stats& q = ss[static_cast<size_t>(i)];
    q.inner_iters += used[static_cast<size_t>(i)];
    if (q.outer_iters - 1 < MDP_HISTORY) q.inner_history[q.outer_iters - 1] = used[static_cast<size_t>(i)];
    phase[static_cast<size_t>(i)] = kOuter;
  };
  while (remaining > 0 && ce == cudaSuccess) {
    std::vector<int32_t> bell, res, inner;
    for (int32_t i = 0; i < count; ++i) {
      if (phase[static_cast<size_t>(i)] == kOuter) bell.push_back(i);
      if (phase[static_cast<size_t>(i)] == kCont) res.push_back(i);
    }
    build(0, bell, 0);
    build(1, res, 1);
    upload();
    if (ce == cudaSuccess && !bell.empty()) ce = launch_batch_bellman(d_mdps, d_lists + 0, num_sms, s);
    if (ce == cudaSuccess && !res.empty())
      ce = launch_batch_policy_resid(d_mdps, d_lists + 1, num_sms, s);
    read_heads();
    if (ce != cudaSuccess) break;
    for (int32_t i : bell) {
      const size_t u = static_cast<size_t>(i);
      mdp_solve_stats& q = ss[u];
      const double r = head(i).res_inf;
      q.bellman_sweeps += 1;
      q.transitions += static_cast<double>(hs[i]->A.nnz);
      if (q.n_history < MDP_HISTORY) q.residual_history[q.n_history++] = r;
      q.residual_inf = r;
      if (r <= o.tol) {
        q.converged = 1;
        phase[u] = kDone;
      } else if (!std::isfinite(r)) {
        st[u] = MDP_ERR_NOT_CONVERGED;
        msg[u] = "non-finite Bellman residual";
        phase[u] = kDone;
      } else if (outer[u] >= o.max_outer) {
        st[u] = MDP_ERR_NOT_CONVERGED;
        msg[u] = "max_outer reached";
        phase[u] = kDone;
      } else {
        outer[u] += 1;
        q.outer_iters += 1;
        used[u] = 0;
        target[u] = o.inner_rtol * r;
        phase[u] = kInner;
      }
      if (phase[u] == kDone) --remaining;
    }
    for (int32_t i : res) {
      const size_t u = static_cast<size_t>(i);
      ss[u].policy_sweeps += 1;
      ss[u].transitions += pnnz[u];
      if (!head(i).active || (o.inner_norm == 1 && head(i).res_inf <= target[u])) finish_inner(i);
      else phase[u] = kInner;
    }
    for (int32_t i = 0; i < count; ++i)
      if (phase[static_cast<size_t>(i)] == kInner) inner.push_back(i);
    if (inner.empty()) continue;
    build(2, inner, 1);
    build(3, inner, 2);
    upload();
    if (ce != cudaSuccess) break;
    if (!tried_graph && s != nullptr && !getenv("MDP_NO_GRAPHS")) {
      tried_graph = true;
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
          cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaError_t e = enqueue_cycle_all();
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g ||
            cudaGraphInstantiate(&cycle, g, 0) != cudaSuccess)
          cycle = nullptr;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
    }
    ce = cycle ? cudaGraphLaunch(cycle, s) : enqueue_cycle_all();
    read_heads();
    if (ce != cudaSuccess) break;
    for (int32_t i : inner) {
      const size_t u = static_cast<size_t>(i);
      const StatusHead& hh = head(i);
      used[u] += hh.nspmv;
      ss[u].policy_sweeps += hh.nspmv;
      ss[u].transitions += pnnz[u] * hh.nspmv;
      if (hh.converged || used[u] >= o.max_inner || hh.jdone == 0) finish_inner(i);
      else phase[u] = kCont;
    }
  }
  if (cycle) cudaGraphExecDestroy(cycle);
  if (ce != cudaSuccess) {
    cudaFreeAsync(dbuf, s);
    for (int32_t i = 0; i < count; ++i) hs[i]->broken = true;
    return fail(MDP_ERR_CUDA, "mdp_batch_solve_fused: %s", cudaGetErrorString(ce));
  }
  for (int32_t i = 0; i < count; ++i) {
    mdp_s* h = hs[i];
    CK(h, launch_from_ff(h->A.n, h->V, V_out[i], 1, h->neg, h->A.num_sms, s));
    if (pi_out && pi_out[i])
      CK(h, cudaMemcpyAsync(pi_out[i], h->pi, static_cast<size_t>(h->A.n) * sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, s));
    mark_done(h, s);
  }
  cudaFreeAsync(dbuf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return fail(MDP_ERR_CUDA, "mdp_batch_solve_fused: the final synchronisation failed");
  for (int32_t i = 0; i < count; ++i) {
    const size_t u = static_cast<size_t>(i);
    if (stats) stats[u] = ss[u];
    if (status_out) status_out[u] = st[u];
    if (result == MDP_OK && st[u] != MDP_OK) {
      result = st[u];
      g_err = "mdp_batch_solve_fused: MDP " + std::to_string(i) + ": " + msg[u];
    }
  }
  return result;
}

mdp_status mdp_profile_enable(mdp_t h, int on) {
  if (!h) return fail(MDP_ERR_ARG, "NULL handle");
  DeviceGuard dg(h->device);
  for (ProfRec& r : h->prof.pending) cudaEventSynchronize(r.b);
  prof_flush(h);
  memset(&h->prof.agg, 0, sizeof(h->prof.agg));
  for (auto& v : h->prof.samples) v.clear();
  h->launches = 0;
  h->prof.on = on != 0;
  return MDP_OK;
}

mdp_status mdp_profile_read(mdp_t h, mdp_profile_t* out) {
  if (!h || !out) return fail(MDP_ERR_ARG, "NULL argument");
  DeviceGuard dg(h->device);
  for (ProfRec& r : h->prof.pending) cudaEventSynchronize(r.b);
  prof_flush(h);
  *out = h->prof.agg;
  out->total_launches = h->launches;
  for (int k = 0; k < MDP_PROF_KINDS; ++k) {
    std::vector<float> v = h->prof.samples[k];
    out->p50_ms[k] = percentile(v, 0.50);
    out->p99_ms[k] = percentile(v, 0.99);
  }
  return MDP_OK;
}

}  // extern "C"
