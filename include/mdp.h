/*
 * mdp.h -- C ABI of the GB300 (sm_103a) inexact-policy-iteration solver for
 * large discounted Markov decision processes with sparse transitions.
 *
 * Problem (madupite, "Problem Setting and Solution Methods"): an
 * infinite-horizon discounted MDP with n states and m actions; minimise the
 * expected discounted cost (or maximise a reward, MDP_FLAG_MAXIMIZE).  With
 * P(s'|s,a) and stage cost g(s,a):
 *
 *   Q(s,a)   = g(s,a) + gamma * sum_{s'} P(s'|s,a) V(s')          (Bellman backup)
 *   (T V)(s) = min_a Q(s,a),   greedy(V)(s) = lowest a attaining it
 *   V*       = the unique fixed point of T;  pi* = greedy(V*)
 *
 * Solution method (same section): inexact policy iteration (iPI), a variant of
 * policy iteration whose policy-evaluation step -- the linear system
 * (I - gamma P_pi) v = g_pi -- is solved only approximately, here by restarted
 * GMRES (the "inexact GMRES policy iteration" the paper cites), to a tolerance
 * tied to the current Bellman residual ("tuning the level of inexactness").
 *
 * Data layout (all calls):
 *   row r = s*m + a of an (n*m) x n CSR matrix holds P(.|s,a);
 *   row_ptr[n*m + 1] (int64, row_ptr[0] = 0), col[nnz] (int32 state index),
 *   val[nnz] (probabilities), cost[n*m] (g(s,a) at row r).
 *   Value vectors have n entries, policies are int32 action indices.
 *
 * Memory: every array argument is a DEVICE pointer on the handle's device
 * unless a flag below says otherwise.  mdp_create copies (and converts) its
 * inputs into library-owned device memory; the caller may free them as soon as
 * the call returns.  Outputs are caller-owned buffers.  All work is enqueued
 * on the given CUDA stream (NULL = the legacy default stream); calls that
 * return host scalars (residual norms, stats) synchronise that stream.
 *
 * Errors: every call returns an mdp_status and never throws or traps.
 * mdp_last_error() returns a thread-local message describing the last failure.
 * A CUDA error inside a call returns MDP_ERR_CUDA and marks the handle broken
 * (later calls on it return MDP_ERR_CUDA).
 *
 * Precision: probabilities are kept in FP32 (FP64 inputs also keep an FP32
 * remainder so that the defining values are represented to ~2^-48).  The
 * Bellman residual, the outer iterate of mdp_solve and the refinement residual
 * are evaluated in float-float arithmetic (an unevaluated sum hi + lo of two
 * FP32 numbers, ~48 significant bits); the GMRES inner solve runs in FP32 (or
 * BF16/FP16 probabilities renormalised per row); the GMRES
 * Hessenberg/Givens least-squares and all norms run in FP64.
 */
#ifndef MDP_GB300_MDP_H
#define MDP_GB300_MDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdp_s* mdp_t;

typedef enum { MDP_F32 = 0, MDP_F64 = 1, MDP_BF16 = 2, MDP_F16 = 3 } mdp_dtype;

typedef enum {
  MDP_OK = 0,
  MDP_ERR_ARG = 1,            /* bad argument (size, pointer, dtype, gamma, ...) */
  MDP_ERR_NOT_STOCHASTIC = 2, /* a row of P is empty, negative or does not sum to 1 */
  MDP_ERR_OOM = 3,            /* device allocation failed */
  MDP_ERR_CUDA = 4,           /* a CUDA call failed; the handle is now broken */
  MDP_ERR_NOT_CONVERGED = 5,  /* iteration limit hit; best iterate written */
  MDP_ERR_TIMEOUT = 6,        /* a device wait exceeded its bound */
  MDP_ERR_CANCELLED = 7,      /* cancelled through mdp_cancel */
  MDP_ERR_BAD_CSR = 8,        /* row_ptr not monotone / wrong length, col out of range */
  MDP_ERR_NONFINITE = 9       /* NaN or Inf in probabilities or costs */
} mdp_status;

/* mdp_create flags */
#define MDP_FLAG_HOST_INPUT 0x1ull   /* row_ptr, col, val, cost are host pointers; in
                                        page-locked memory they are read in place by the
                                        packing kernel (no device staging copy), otherwise
                                        staged on the device first */
#define MDP_FLAG_NO_VALIDATE 0x2ull  /* skip the stochasticity check (CSR checks stay) */
#define MDP_FLAG_AUTOTUNE 0x4ull     /* time the candidate lanes-per-row / shared-memory window
                                        schedules of the Bellman kernel at create and keep the
                                        fastest (cached per process by matrix shape) */
#define MDP_FLAG_MAXIMIZE 0x8ull     /* `cost` holds rewards r(s,a) to be maximised: V = max_a
                                        [r + gamma P V], pi = lowest maximising action.  Solved
                                        as the minimisation with g = -r; every value vector in
                                        or out of the handle (V_in, V_out, V_init, v_inout,
                                        r_out) is in reward terms.  Negation is exact, so the
                                        results are bitwise the negated values (same policy,
                                        same norms and statistics) of a minimising handle
                                        given cost -r and value vectors -V. */

/* Inner solver of the policy-evaluation step (madupite: "selecting among a wide
 * range of inner solvers for the approximate policy evaluation step"). */
typedef enum {
  MDP_INNER_GMRES = 0,      /* restarted GMRES(restart), the default */
  MDP_INNER_RICHARDSON = 1, /* v <- g_pi + gamma P_pi v sweeps: modified policy iteration */
  MDP_INNER_BICGSTAB = 2    /* BiCGStab (van der Vorst 1992) on the FP32 probabilities:
                               two policy SpMVs per iteration, no restart, no basis */
} mdp_inner;

typedef struct {
  double tol;           /* stop when ||T V - V||_inf <= tol (absolute), default 1e-9 */
  double inner_rtol;    /* eta: the inner solve stops when ||(I - gamma P_pi) v - g_pi||_2
                           <= eta * ||T V - V||_inf, default 0.1 */
  int32_t restart;      /* GMRES restart length, 1..64, default 30 */
  int32_t max_outer;    /* outer (improvement) iterations, default 1000 */
  int32_t max_inner;    /* inner iterations (Arnoldi steps, sweeps or BiCGStab
                           iterations) per outer, default 10000 */
  int32_t inner;        /* mdp_inner, default MDP_INNER_GMRES */
  int32_t cgs2;         /* 1 = re-orthogonalise once (classical Gram-Schmidt twice) */
  int32_t low_precision_inner; /* 1 = inner SpMV on the BF16/FP16 copy (needs store_t;
                                  GMRES and Richardson; BiCGStab always uses FP32) */
  int32_t inner_norm;   /* 0: stop the inner GMRES on its 2-norm residual estimate
                           <= eta * ||T V - V||_inf (default, conservative);
                           1: additionally stop after any restart cycle whose explicit
                           policy residual has ||.||_inf <= eta * ||T V - V||_inf */
  int32_t s_step;       /* GMRES in s-step form (default 6): 0 = classical Gram-Schmidt
                           Arnoldi (one orthogonalisation per step); 1..8 = blocks of s_step
                           Krylov vectors (monomial basis of A - I) orthogonalised
                           together, with the solution update fused into the last
                           block's pass; not combinable with cgs2 */
} mdp_solve_opts;

#define MDP_HISTORY 128

typedef struct {
  int32_t outer_iters;       /* improvement steps taken */
  int32_t inner_iters;       /* Arnoldi steps (or Richardson sweeps) in total */
  int32_t bellman_sweeps;    /* full-matrix Bellman backups */
  int32_t policy_sweeps;     /* policy-row SpMVs (inner steps + refinement residuals) */
  int32_t converged;         /* 1 when ||T V - V||_inf <= tol */
  int32_t n_history;
  double residual_inf;       /* final ||T V - V||_inf */
  double transitions;        /* nonzeros touched: sweeps * nnz + policy sweeps * policy nnz */
  double residual_history[MDP_HISTORY]; /* ||T V_k - V_k||_inf per outer iteration */
  int32_t inner_history[MDP_HISTORY];   /* inner iterations per outer iteration */
} mdp_solve_stats;

typedef struct {
  int32_t iters;        /* Arnoldi steps */
  int32_t cycles;       /* restart cycles */
  int32_t converged;
  int32_t policy_sweeps;
  double residual_2;    /* final ||(I - gamma P_pi) v - g_pi||_2, refinement precision */
} mdp_eval_stats;

typedef struct {
  int64_t n_states, n_rows, nnz;
  int32_t n_actions;
  int32_t vec_width;     /* lanes per row chosen for the CSR kernels */
  int32_t uniform_len;   /* nnz per row when every row has the same length, else 0 */
  int32_t idx64;         /* 1 when row pointers are kept as int64 */
  int64_t band;          /* max |col - s| over all entries */
  int32_t has_low_precision;
  int32_t store_t;       /* mdp_dtype of the inner-solve probabilities */
  size_t device_bytes;   /* library-owned device memory of this handle */
  double gamma;
  int32_t maximize;      /* 1 when created with MDP_FLAG_MAXIMIZE */
  int32_t window;        /* 1 when the banded kernels stage V in a shared-memory ring */
  int32_t ff_screen;     /* 1 when the float-float backups screen the actions in FP32
                            and repeat only the candidate rows in float-float (same
                            results bit for bit; opt-in: environment MDP_FF_SCREEN
                            at create, for banded rows of 16 aligned entries and a
                            power-of-two action count up to 32) */
} mdp_info_t;

/*
 * mdp_create -- build a solver handle from a CSR MDP (madupite: "create an MDP
 * by loading offline data"; problem as defined above).
 *   out       receives the handle (NULL on failure).
 *   n_states  n >= 1; n_actions m >= 1; n*m rows.
 *   row_ptr   int64[n*m + 1], row_ptr[0] = 0, non-decreasing, every row non-empty.
 *   col       int32[nnz], 0 <= col < n.
 *   val       MDP_F32 or MDP_F64 [nnz], each row non-negative, summing to 1 within 1e-5.
 *   cost      MDP_F32 or MDP_F64 [n*m], finite.
 *   gamma     discount factor, 0 <= gamma < 1.
 *   store_t   MDP_F32: inner solve on FP32 probabilities; MDP_BF16 / MDP_F16:
 *             also keep a 16-bit copy of the probabilities q(P_e) for the
 *             low-precision inner solve, renormalised per row: when the band
 *             fits int16 column offsets the packed copy divides each row sum
 *             by sum_e q(P_e) on the fly (no stored factor); otherwise a
 *             stored FP32 factor c_r = 1 / sum_e q(P_e) per row.
 *   stream    cudaStream_t (NULL = default stream); flags: MDP_FLAG_*.
 * Errors: MDP_ERR_ARG, MDP_ERR_BAD_CSR, MDP_ERR_NOT_STOCHASTIC, MDP_ERR_NONFINITE,
 * MDP_ERR_OOM, MDP_ERR_CUDA.  Synchronises the stream (validation result).
 */
mdp_status mdp_create(mdp_t* out, int64_t n_states, int32_t n_actions, const int64_t* row_ptr,
                      const int32_t* col, const void* val, mdp_dtype val_t, const void* cost,
                      mdp_dtype cost_t, double gamma, mdp_dtype store_t, void* stream,
                      uint64_t flags);

/* Release all device memory of the handle (NULL is a no-op). */
void mdp_destroy(mdp_t h);

/*
 * mdp_bellman -- one Bellman backup with greedy improvement (madupite, "Problem
 * Setting": the improvement step of policy iteration, the whole of value
 * iteration):  V_out = T V_in,  pi_out = greedy(V_in) (lowest index on ties),
 * r_out = T V_in - V_in.
 *   V_in, V_out  [n] of v_t: MDP_F32 (FP32 accumulation) or MDP_F64 (float-float
 *                accumulation over the defining probabilities; result to ~1e-13
 *                relative).  V_out may be NULL; V_out must not alias V_in.
 *   pi_out       int32[n] or NULL.   r_out  float[n] or NULL.
 *   res_inf, res_2  host doubles or NULL: ||r||_inf and ||r||_2 (FP64 reduction,
 *                fixed order, deterministic).  Non-NULL scalars synchronise the stream.
 */
mdp_status mdp_bellman(mdp_t h, const void* V_in, mdp_dtype v_t, void* V_out, int32_t* pi_out,
                       float* r_out, double* res_inf, double* res_2, void* stream);

/*
 * mdp_policy_eval -- approximate policy evaluation (madupite, "Problem Setting":
 * the inexact evaluation step of iPI): solve (I - gamma P_pi) v = g_pi by
 * restarted GMRES whose SpMV gathers row s*m + pi(s) of the CSR directly, with
 * float-float refinement residuals between restart cycles.
 *   pi        int32[n] actions in [0, m).
 *   v_inout   [n] of v_t (MDP_F32 or MDP_F64): initial guess in, solution out.
 *   tol       absolute target for ||(I - gamma P_pi) v - g_pi||_2.
 *   restart   GMRES restart length 1..64;  max_iters  cap on Arnoldi steps.
 *   st        host stats or NULL.
 * Returns MDP_ERR_NOT_CONVERGED (v holds the last iterate) when max_iters is hit.
 * Synchronises the stream.
 */
mdp_status mdp_policy_eval(mdp_t h, const int32_t* pi, void* v_inout, mdp_dtype v_t, double tol,
                           int32_t restart, int32_t max_iters, mdp_eval_stats* st, void* stream);

/* Fill opts with the defaults listed in mdp_solve_opts. */
void mdp_default_opts(mdp_solve_opts* opts);

/*
 * mdp_solve -- inexact policy iteration (madupite, "Problem Setting and
 * Solution Methods"):  repeat { Bellman backup on the float-float iterate V:
 * pi <- greedy(V), r = T V - V; stop if ||r||_inf <= tol; else solve
 * (I - gamma P_pi) d = r approximately (GMRES, ||residual||_2 <= eta ||r||_inf)
 * and set V <- V + d }.  Since pi is greedy for V, r = g_pi + gamma P_pi V - V,
 * so V + d approximates V_pi: the outer loop is also iterative refinement of
 * the low-precision inner solves.
 *   opts     NULL = defaults.   V_init  [n] of vinit_t (MDP_F32/MDP_F64) or NULL (V = 0).
 *   V_out    double[n] device;  pi_out int32[n] device or NULL;  st host stats or NULL.
 * Returns MDP_ERR_NOT_CONVERGED (best iterate written) when max_outer is hit.
 * Synchronises the stream.
 */
mdp_status mdp_solve(mdp_t h, const mdp_solve_opts* opts, const void* V_init, mdp_dtype vinit_t,
                     double* V_out, int32_t* pi_out, mdp_solve_stats* st, void* stream);

/*
 * mdp_batch_solve -- solve `count` independent MDPs (one handle each) with the
 * inexact policy iteration of mdp_solve, concurrently: `n_streams` host
 * workers each own a CUDA stream and take the next MDP, largest (by nonzeros)
 * first, from a shared counter, so the kernels of different (often small,
 * uneven) MDPs overlap on the GPU and no large MDP runs alone at the end.
 *   hs[count]      distinct handles (each solved once; not shared across calls).
 *   opts           NULL = defaults, used for every MDP.
 *   V_out[i]       double[n_i] device;  pi_out[i] int32[n_i] device or NULL
 *                  (pi_out itself may be NULL);  stats[count] host or NULL.
 *   n_streams      1..64 concurrent workers (0 = 8).
 * Every per-MDP result equals what mdp_solve returns for that MDP alone: the
 * handles share no state and every reduction has a fixed order.  Returns
 * MDP_OK when all converged, else the first non-OK status in index order
 * (per-MDP statuses in status_out[count] when it is not NULL).  Returns after
 * all work is complete.
 */
mdp_status mdp_batch_solve(mdp_t const* hs, int32_t count, const mdp_solve_opts* opts,
                           double* const* V_out, int32_t* const* pi_out, mdp_solve_stats* stats,
                           mdp_status* status_out, int32_t n_streams);

/*
 * mdp_batch_solve_fused -- solve `count` independent MDPs (one handle each) by
 * the inexact policy iteration of mdp_solve with every solve phase of all the
 * MDPs in one launch (madupite's solver applied to many problems at once; the
 * batching of many uneven MDPs is this implementation's).  Each phase kernel
 * is persistent (one wave of blocks) and walks a device-side work list of
 * units -- a tile of one MDP's states -- over the MDPs in that phase: the
 * float-float Bellman backup, the policy residual between restart cycles, and
 * the s-step GMRES cycle (SpMVs, Gram pass with the least squares, update).
 * Rounds advance every MDP by one phase; the host reads all MDPs' status with
 * one copy per phase and rebuilds the work lists; a restart cycle is captured
 * once as a CUDA graph and replayed (on a non-default stream).
 *   hs[count]      distinct handles on the current device, at most 64 actions.
 *   opts           NULL = defaults; needs the GMRES inner solver in s-step form
 *                  (s_step 1..8) on the FP32 probabilities (no cgs2, no
 *                  low_precision_inner).  Every cycle has `restart` steps, so the
 *                  max_inner cap is checked after each cycle.
 *   V_out[i]       double[n_i] device;  pi_out[i] int32[n_i] device or NULL
 *                  (pi_out may be NULL);  stats[count] host or NULL.
 *   stream         one stream for every launch (NULL = legacy default stream,
 *                  no graph capture).
 * Each MDP's units and reduction order depend only on that MDP, so its result
 * is bitwise the same when solved alone through this call and in any batch.
 * (It is not bitwise the same as mdp_solve, whose kernels are laid out for one
 * large MDP; both meet the same tolerance.)  mdp_cancel is not checked.
 * Returns MDP_OK when all converged, else the first non-OK status in index
 * order (per-MDP statuses in status_out[count] when not NULL); MDP_ERR_ARG for
 * options or handles it does not support.  Synchronises the stream.
 */
mdp_status mdp_batch_solve_fused(mdp_t const* hs, int32_t count, const mdp_solve_opts* opts,
                                 double* const* V_out, int32_t* const* pi_out,
                                 mdp_solve_stats* stats, mdp_status* status_out, void* stream);

/* Handle properties (layout chosen at create, memory held). */
mdp_status mdp_info(mdp_t h, mdp_info_t* info);

#define MDP_MAX_RESTART 64

/* The last finished GMRES restart cycle of a handle (the least-squares step of
 * GMRES, Saad 2003, 6.5.3: minimise ||beta e_1 - H y||_2 over y, H the
 * (J+1) x J upper Hessenberg matrix of the Arnoldi process, which the inner
 * policy evaluation of the paper's "Problem Setting and Solution Methods" runs
 * on (I - gamma P_pi)). */
typedef struct {
  int32_t J;        /* Arnoldi steps of the cycle (0 when no cycle has finished) */
  int32_t pad;
  double beta;      /* ||r_0||_2 of the cycle */
  double est;       /* |g_{J}|: the Givens residual estimate ||beta e_1 - H y||_2 */
  double H[(MDP_MAX_RESTART + 1) * MDP_MAX_RESTART]; /* H as built by the Arnoldi
                       process, before the rotations: entry (i, j) at H[j * 65 + i],
                       i <= j + 1 < J + 1; other entries unspecified */
  double y[MDP_MAX_RESTART];  /* the back-solved least-squares solution, y[0..J) */
} mdp_gmres_cycle_t;

/* Copy the last finished GMRES cycle of h (mdp_solve with the GMRES inner solver,
 * or mdp_policy_eval) into *out.  Synchronises the handle's last stream.  The
 * record is the one of the cycle that finished last: later cycles overwrite
 * it.  Returns MDP_ERR_ARG for a NULL argument, MDP_ERR_CUDA if the copy fails. */
mdp_status mdp_last_cycle(mdp_t h, mdp_gmres_cycle_t* out);

/*
 * Device bytes a handle of this shape needs (CSR copy, low-precision copy,
 * GMRES basis of `restart`+1 vectors, work vectors); used for admission control.
 */
size_t mdp_bytes_required(int64_t n_states, int32_t n_actions, int64_t nnz, mdp_dtype val_t,
                          mdp_dtype store_t, int32_t restart);

/* Request that the mdp_solve / mdp_policy_eval running on h stop at its next
 * host check (at most one GMRES restart cycle or one batch of eight inner
 * iterations later); it then returns MDP_ERR_CANCELLED with the iterate
 * reached so far in its outputs.  A request made while no call runs on h stays
 * pending: the next mdp_solve / mdp_policy_eval on h returns MDP_ERR_CANCELLED
 * at once, before it enqueues anything or writes its outputs.  Each request is consumed by the call that returns
 * MDP_ERR_CANCELLED for it; a request that arrives after a call's last check
 * therefore cancels the next call on h.  Thread-safe. */
void mdp_cancel(mdp_t h);

/* ---- per-kernel profiling (CUDA events on the launching stream) ---------- */
enum {
  MDP_PROF_BELLMAN_F32 = 0,  /* K1: FP32 Bellman backup */
  MDP_PROF_BELLMAN_FF = 1,   /* K6: float-float Bellman backup + residual */
  MDP_PROF_POLICY_RESID = 2, /* float-float policy residual (refinement) */
  MDP_PROF_ARNOLDI_SPMV = 3, /* K2: policy-row SpMV w = v_j - gamma P_pi v_j */
  MDP_PROF_ARNOLDI_ORTHO = 4,/* K3 + K4: orthogonalisation, norm, Givens */
  MDP_PROF_GMRES_UPDATE = 5, /* K5: V += sum y_i v_i */
  MDP_PROF_RICHARDSON = 6,   /* modified-PI sweep */
  MDP_PROF_OTHER = 7,        /* conversions, set-up kernels */
  MDP_PROF_ARNOLDI_DOTS = 8, /* Gram-Schmidt dots <w, v_i> */
  MDP_PROF_BICGSTAB_SPMV = 9,/* BiCGStab policy SpMV y = x - gamma P_pi x with its dots */
  MDP_PROF_BLOCK_GRAM = 10,  /* s-step GMRES: Gram pass of a block + its least squares */
  MDP_PROF_BLOCK_UPDATE = 11,/* s-step GMRES: block orthonormalisation (+ V update) */
  MDP_PROF_KINDS = 12
};

typedef struct {
  int64_t launches[MDP_PROF_KINDS]; /* timed launches that did work */
  int64_t skipped[MDP_PROF_KINDS];  /* launches that returned at once (GMRES cycle already over) */
  double ms[MDP_PROF_KINDS];        /* summed event-timed duration of the timed launches */
  double bytes[MDP_PROF_KINDS];     /* algorithmic DRAM bytes of the timed launches (gathers of
                                       the value vector excluded: they hit L2) */
  int64_t total_launches;           /* every kernel launch of the handle since the last reset,
                                       counted whether or not timing is on */
  double p50_ms[MDP_PROF_KINDS];    /* median duration of one timed launch (nearest rank) */
  double p99_ms[MDP_PROF_KINDS];    /* 99th percentile of the same (nearest rank) */
} mdp_profile_t;

/* Turn event timing of every kernel launch on (1) or off (0); resets the
 * counters.  Timing adds two event records per launch on the same stream. */
mdp_status mdp_profile_enable(mdp_t h, int on);

/* Aggregate the counters since the last enable (synchronises pending events). */
mdp_status mdp_profile_read(mdp_t h, mdp_profile_t* out);

/*
 * mdp_bellman_noalloc -- one FP32 Bellman backup (as mdp_bellman with v_t =
 * MDP_F32) computed directly on a caller's CSR, allocating no memory at all.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code whose device memory belongs to
 * another allocator or a fixed budget (a framework's caching allocator, a
 * request loop's admission budget), or a latency-critical thread that may not
 * call cudaMalloc/cudaFree because they can synchronise the whole device.
 *   n_states, n_actions, row_ptr (int64[n*m+1]), col (int32[nnz]), val
 *   (float[nnz]), cost (float[n*m]): the CSR as mdp_create takes it, device
 *   pointers, read in place (not validated for stochasticity; out-of-range row
 *   pointers or columns are skipped and reported as MDP_ERR_BAD_CSR).
 *   gamma in [0, 1).  V_in float[n]; V_out float[n] (not aliasing V_in),
 *   pi_out int32[n] and r_out float[n] may be NULL; res_inf, res_2 host
 *   doubles or NULL (FP64 fixed-order reduction).  Synchronises the stream.
 * Scratch: a file-scope device array of 262,400 bytes per device that loads
 * the library (held until exit), enough for n_states <= 4,194,304; larger
 * problems are rejected with MDP_ERR_ARG.  The first call on a device looks
 * the array up with cudaGetSymbolAddress.  The call reads its results back
 * through host memory and synchronises `stream`, so it must never be made on a
 * stream that is capturing a CUDA graph; such a call returns MDP_ERR_ARG
 * before it enqueues anything.  All calls on a device share the array: calls
 * whose kernels overlap on the GPU race and must be serialised by the caller.
 */
mdp_status mdp_bellman_noalloc(int64_t n_states, int32_t n_actions, const int64_t* row_ptr,
                               const int32_t* col, const float* val, const float* cost,
                               double gamma, const float* V_in, float* V_out, int32_t* pi_out,
                               float* r_out, double* res_inf, double* res_2, void* stream);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* mdp_last_error(void);

/* Hand device memory cached by the library back to the device.
 *
 * No counterpart in the paper: a memory-management call of this
 * implementation.  Handles take their device memory from a stream-ordered
 * pool that the library owns, one per device, and that keeps the memory of
 * destroyed handles mapped so that later handles reuse it without mapping new
 * pages.  This call waits for the frees of destroyed handles on `device` to
 * complete, then releases cached memory until at most `keep_bytes` stay
 * reserved (memory of live handles is never released).  `reserved_after`
 * (may be NULL) receives the bytes the pool still reserves.  Returns
 * MDP_ERR_ARG for a device index out of range, MDP_ERR_CUDA if a CUDA call
 * fails. */
mdp_status mdp_pool_trim(int32_t device, uint64_t keep_bytes, uint64_t* reserved_after);

/* Library version string. */
const char* mdp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MDP_GB300_MDP_H */
