/*
 * A C99 program against include/mdp.h and include/mdp_ingest.h: the boundary
 * used from plain C, with no Python and no C++.
 *
 * Host part (any machine): build a ring-world MDP from C generator callbacks,
 * write it as PETSc binary files, read it back, check the arrays, and check the
 * host-only entry points (version, default options, size model, error text).
 * With the argument "gpu" (built with -DMDP_EXAMPLE_CUDA and the CUDA runtime,
 * which the program uses for its own device buffers) it also creates a handle
 * from the host CSR, solves it, and checks the Bellman residual and the closed
 * form of the solution (every step costs 1: V = 1 / (1 - gamma)).
 *
 * Prints "ok" and exits 0 on success; prints the failed check and exits 1.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mdp.h"
#include "mdp_ingest.h"

#ifdef MDP_EXAMPLE_CUDA
#include <cuda_runtime_api.h>
#endif

#define CHECK(c)                                                        \
  do {                                                                  \
    if (!(c)) {                                                         \
      printf("check failed at line %d: %s (%s)\n", __LINE__, #c,        \
             mdp_last_error());                                         \
      return 1;                                                         \
    }                                                                   \
  } while (0)

enum { N = 1000, M = 3 };

/* action 0: stay; action 1: step right; action 2: step left, each slipping
   to the two neighbours with probability 0.1 each */
static int32_t ring_row(int64_t s, int32_t a, int32_t cap, int32_t* col, double* prob,
                        void* user) {
  (void)user;
  if (cap < 3) return 3;
  const int32_t left = (int32_t)((s + N - 1) % N), right = (int32_t)((s + 1) % N);
  const int32_t target = a == 0 ? (int32_t)s : (a == 1 ? right : left);
  col[0] = target;
  prob[0] = 0.8;
  col[1] = left;
  prob[1] = 0.1;
  col[2] = right;
  prob[2] = 0.1;
  return 3;
}

static double unit_cost(int64_t s, int32_t a, void* user) {
  (void)s;
  (void)a;
  (void)user;
  return 1.0;
}

int main(int argc, char** argv) {
  const int gpu = argc > 1 && strcmp(argv[1], "gpu") == 0;
  const char* dir = argc > 2 ? argv[2] : ".";
  char p_path[4096], g_path[4096];
  snprintf(p_path, sizeof(p_path), "%s/ring_P.bin", dir);
  snprintf(g_path, sizeof(g_path), "%s/ring_g.bin", dir);

  CHECK(strncmp(mdp_version(), "mdp-gb300", 9) == 0);
  mdp_solve_opts o;
  mdp_default_opts(&o);
  CHECK(o.restart == 30 && o.tol == 1e-9 && o.inner == MDP_INNER_GMRES);
  CHECK(mdp_bytes_required(N, M, 3 * N * M, MDP_F64, MDP_F32, 30) > (size_t)N * M * 12);

  mdp_host_csr a, b;
  CHECK(mdp_csr_from_functions(N, M, ring_row, unit_cost, NULL, 4, NULL, NULL, &a) == MDP_OK);
  CHECK(a.n_states == N && a.n_actions == M && a.owned == 1);
  /* a stay row holds three states; a move's target is also a slip neighbour,
     and the two entries merge (0.8 + 0.1), leaving two; rows are sorted */
  CHECK(a.nnz == 7 * (int64_t)N);
  CHECK(a.row_ptr[1] == 3 && a.row_ptr[2] == 5 && a.row_ptr[3] == 7);
  CHECK(a.col[0] == 0 && a.col[1] == 1 && a.col[2] == N - 1);
  CHECK(a.val[0] == 0.8 && a.val[1] == 0.1 && a.val[2] == 0.1);
  CHECK(a.col[3] == 1 && a.col[4] == N - 1 && a.val[3] == 0.8 + 0.1 && a.val[4] == 0.1);

  CHECK(mdp_csr_write_petsc(&a, p_path, g_path) == MDP_OK);
  CHECK(mdp_csr_read_petsc(p_path, g_path, 2, NULL, NULL, &b) == MDP_OK);
  CHECK(b.n_states == N && b.n_actions == M && b.nnz == a.nnz);
  CHECK(memcmp(a.row_ptr, b.row_ptr, sizeof(int64_t) * (N * M + 1)) == 0);
  CHECK(memcmp(a.col, b.col, sizeof(int32_t) * (size_t)a.nnz) == 0);
  CHECK(memcmp(a.val, b.val, sizeof(double) * (size_t)a.nnz) == 0);
  CHECK(memcmp(a.cost, b.cost, sizeof(double) * N * M) == 0);

  /* errors come back as a status with a message, never as a crash */
  mdp_host_csr c;
  CHECK(mdp_csr_read_petsc("/nonexistent/P.bin", NULL, 1, NULL, NULL, &c) == MDP_ERR_ARG);
  CHECK(strstr(mdp_last_error(), "cannot open") != NULL);
  CHECK(c.row_ptr == NULL && c.nnz == 0);

  if (gpu) {
#ifdef MDP_EXAMPLE_CUDA
    mdp_t h = NULL;
    CHECK(mdp_create(&h, N, M, b.row_ptr, b.col, b.val, MDP_F64, b.cost, MDP_F64, 0.9, MDP_F32,
                     NULL, MDP_FLAG_HOST_INPUT) == MDP_OK);
    mdp_info_t info;
    CHECK(mdp_info(h, &info) == MDP_OK && info.nnz == b.nnz && info.maximize == 0);
    double* V = NULL;
    int32_t* pi = NULL;
    CHECK(cudaMalloc((void**)&V, sizeof(double) * N) == cudaSuccess);
    CHECK(cudaMalloc((void**)&pi, sizeof(int32_t) * N) == cudaSuccess);
    mdp_solve_stats st;
    CHECK(mdp_solve(h, &o, NULL, MDP_F64, V, pi, &st, NULL) == MDP_OK);
    CHECK(st.converged == 1 && st.residual_inf <= o.tol);
    static double Vh[N];
    static int32_t pih[N];
    CHECK(cudaMemcpy(Vh, V, sizeof(Vh), cudaMemcpyDeviceToHost) == cudaSuccess);
    CHECK(cudaMemcpy(pih, pi, sizeof(pih), cudaMemcpyDeviceToHost) == cudaSuccess);
    for (int s = 0; s < N; ++s) {
      /* every step costs 1: V* = 1 / (1 - gamma) = 10 */
      CHECK(fabs(Vh[s] - 10.0) <= o.tol / (1.0 - 0.9) * 1.05);
      CHECK(pih[s] >= 0 && pih[s] < M);
    }
    /* a bad argument is a status, and the handle stays usable */
    CHECK(mdp_solve(h, &o, V, (mdp_dtype)7, V, pi, &st, NULL) == MDP_ERR_ARG);
    CHECK(mdp_bellman(h, V, MDP_F64, NULL, pi, NULL, NULL, NULL, NULL) == MDP_OK);
    cudaFree(V);
    cudaFree(pi);
    mdp_destroy(h);
#else
    printf("built without MDP_EXAMPLE_CUDA\n");
    return 1;
#endif
  }

  mdp_csr_free(&a);
  mdp_csr_free(&b);
  CHECK(a.row_ptr == NULL && b.col == NULL);
  printf("ok\n");
  return 0;
}
