/*
 * mdp_ingest.h -- building the host CSR that mdp_create takes, from the two
 * sources the madupite paper names (section "Implementation", last paragraph:
 * an MDP is created by loading offline data from earlier experiments or from
 * online simulation, with the simulation run in parallel), and from/to files
 * in PETSc's binary matrix format, the storage of the PETSc matrices that the
 * paper's library is built on (same section).
 *
 * Every call here is host-only: no CUDA call, no device memory.  The output
 * is an mdp_host_csr in the layout of mdp_create (row r = s*m + a of an
 * (n*m) x n matrix, columns ascending within a row, no repeated column), ready
 * for mdp_create(..., MDP_FLAG_HOST_INPUT) with val_t = cost_t = MDP_F64.
 *
 * Output memory: each function takes an allocator `alloc(bytes, alloc_user)`.
 * With alloc == NULL the library allocates with malloc and mdp_csr_free
 * releases the arrays.  With a caller allocator (for instance one returning
 * page-locked memory, which mdp_create then reads in place) the arrays belong
 * to the caller, also when the call fails; mdp_csr_free then only clears the
 * struct.  `alloc` is called only from the calling thread, at most four times
 * (row_ptr, col, val, cost), and must return memory aligned to 8 bytes or
 * NULL (the call then fails with MDP_ERR_OOM).
 *
 * Errors: the functions return an mdp_status and set mdp_last_error(); on
 * failure *out is cleared and library-allocated arrays are released.
 */
#ifndef MDP_GB300_MDP_INGEST_H
#define MDP_GB300_MDP_INGEST_H

#include "mdp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n_states;
  int32_t n_actions;
  int64_t nnz;
  int64_t* row_ptr; /* [n*m + 1], row_ptr[0] = 0 */
  int32_t* col;     /* [nnz], ascending within each row */
  double* val;      /* [nnz] */
  double* cost;     /* [n*m], cost (or reward) of row r = s*m + a */
  int32_t owned;    /* 1: arrays from malloc, released by mdp_csr_free */
} mdp_host_csr;

typedef void* (*mdp_alloc_fn)(size_t bytes, void* alloc_user);

/*
 * Row generator of mdp_csr_from_functions: write the successors of (s, a) --
 * at most `cap` of them -- into col[0..k) (states) and prob[0..k) (their
 * probabilities) and return k.  Return a k > cap to be called again for the
 * same (s, a) with cap >= k; a negative value aborts the build (MDP_ERR_ARG).
 * Repeated successors are summed; the order of the entries does not matter.
 */
typedef int32_t (*mdp_row_fn)(int64_t s, int32_t a, int32_t cap, int32_t* col, double* prob,
                              void* user);
/* Cost generator: g(s, a) (or the reward, for a handle created with MDP_FLAG_MAXIMIZE). */
typedef double (*mdp_cost_fn)(int64_t s, int32_t a, void* user);

/*
 * mdp_csr_from_functions -- evaluate the generators for every (s, a) and
 * assemble the CSR ("online simulation").
 *   n, m      states (1 <= n < 2^31) and actions (m >= 1).
 *   threads   host threads evaluating disjoint contiguous state ranges
 *             concurrently (<= 0: one per hardware thread); the generators
 *             must then be safe to call concurrently.  The result does not
 *             depend on the thread count.
 * Errors: MDP_ERR_ARG (bad size, NULL generator, aborted by the generator),
 * MDP_ERR_NOT_STOCHASTIC (an empty row or a negative probability),
 * MDP_ERR_BAD_CSR (a successor outside [0, n)), MDP_ERR_NONFINITE (NaN/Inf in
 * a probability or a cost), MDP_ERR_OOM.  Row sums are not checked here
 * (mdp_create checks them).
 */
mdp_status mdp_csr_from_functions(int64_t n, int32_t m, mdp_row_fn row, mdp_cost_fn cost,
                                  void* user, int32_t threads, mdp_alloc_fn alloc,
                                  void* alloc_user, mdp_host_csr* out);

/*
 * mdp_csr_from_rows -- assemble the CSR from raw rows: the entries of row
 * r = s*m + a are col/prob[offsets[r] .. offsets[r+1]), in any order and with
 * repeated successors; cost[r] is g(s, a).  Rows are sorted and repeats summed
 * in entry order, so the result is bitwise that of mdp_csr_from_functions on a
 * generator returning the same rows.  Checks and errors as there (the lowest
 * failing row is reported); offsets must start at 0 and never decrease
 * (MDP_ERR_BAD_CSR otherwise).  The inputs are only read.
 *   offsets  int64[n*m + 1];  col int32[offsets[n*m]];  prob, cost doubles.
 */
mdp_status mdp_csr_from_rows(int64_t n, int32_t m, const int64_t* offsets, const int32_t* col,
                             const double* prob, const double* cost, int32_t threads,
                             mdp_alloc_fn alloc, void* alloc_user, mdp_host_csr* out);

/* Handling of state-action pairs without a sample in mdp_csr_from_samples. */
typedef enum {
  MDP_UNSEEN_ERROR = 0,     /* fail with MDP_ERR_ARG, naming the first such (s, a) */
  MDP_UNSEEN_SELF_LOOP = 1  /* P(s|s,a) = 1 with cost unseen_cost */
} mdp_unseen;

/*
 * mdp_csr_from_samples -- the maximum-likelihood model of logged transitions
 * ("offline data"): sample i says that action a[i] in state s[i] led to state
 * s_next[i] at cost c[i].  P(s'|s,a) = N(s,a,s') / N(s,a) and g(s,a) = the mean
 * of the costs of the samples of (s, a), summed in sample order (so the
 * result is deterministic).  c may be NULL when only P is wanted (g = 0).
 *   count     number of samples (>= 0); s, a, s_next, c have `count` entries.
 *   unseen    mdp_unseen; unseen_cost is the cost of an unseen pair's self-loop.
 *   threads   as in mdp_csr_from_functions (for the per-row pass).
 * Errors: MDP_ERR_ARG (a state or action out of range, naming the sample; an
 * unseen pair under MDP_UNSEEN_ERROR), MDP_ERR_NONFINITE, MDP_ERR_OOM.
 */
mdp_status mdp_csr_from_samples(int64_t n, int32_t m, int64_t count, const int64_t* s,
                                const int32_t* a, const int64_t* s_next, const double* c,
                                int32_t unseen, double unseen_cost, int32_t threads,
                                mdp_alloc_fn alloc, void* alloc_user, mdp_host_csr* out);

/*
 * mdp_csr_read_petsc -- load P and g from PETSc binary files.
 *   p_path  the transition matrix: an (n*m) x n sparse (AIJ) matrix whose row
 *           s*m + a holds P(.|s,a).
 *   g_path  the costs: an n x m matrix, dense (MATRIX_BINARY_FORMAT_DENSE,
 *           values by rows) or sparse (missing entries are 0); NULL: all 0.
 * The file format: big-endian; a header of four integers {1211216 (the
 * matrix class id), rows, columns, nonzeros (-1: dense)}; for a sparse matrix
 * the row lengths, the column indices, then the values; for a dense one the
 * values.  Integers are 32-bit, or 64-bit in files of PETSc builds with 64-bit
 * indices (recognised from the header); values are IEEE doubles (real scalars).
 * n = columns of P, m = rows of P / n.  Columns are sorted within each row and
 * repeated columns summed.
 *   threads  host threads for the byte-order conversion (<= 0: all).
 * Errors: MDP_ERR_ARG (unreadable or truncated file, wrong class id, shapes that
 * disagree, a row length or column out of range), MDP_ERR_NONFINITE, MDP_ERR_OOM.
 */
mdp_status mdp_csr_read_petsc(const char* p_path, const char* g_path, int32_t threads,
                              mdp_alloc_fn alloc, void* alloc_user, mdp_host_csr* out);

/*
 * mdp_csr_write_petsc -- write csr as the two files mdp_csr_read_petsc reads
 * (32-bit integers when every count fits, else 64-bit; g dense).  Either path
 * may be NULL to skip that file.  Errors: MDP_ERR_ARG (NULL csr or array,
 * unwritable file).
 */
mdp_status mdp_csr_write_petsc(const mdp_host_csr* csr, const char* p_path, const char* g_path);

/* Release the arrays of a library-allocated csr (owned = 1) and clear it. */
void mdp_csr_free(mdp_host_csr* csr);

#ifdef __cplusplus
}
#endif

#endif /* MDP_GB300_MDP_INGEST_H */
