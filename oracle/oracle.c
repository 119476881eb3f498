/*
 * FP64 CPU oracle for the Bellman operator of a finite discounted MDP.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU path is checked against.  Only the tests, the package's smoke check and
 * the bench's CPU-baseline leg may load it; the solver never calls it.  It
 * shares no code with the CUDA library.
 *
 * Problem (madupite, "Problem Setting and Solution Methods"; Bertsekas 2007):
 * minimise expected discounted cost.  With P(s'|s,a) stored as a CSR matrix of
 * n*m rows (row r = s*m + a) and stage cost g(s,a):
 *
 *   Q(s,a)    = g(s,a) + gamma * sum_{s'} P(s'|s,a) V(s')
 *   (T V)(s)  = min_a Q(s,a)
 *   greedy(V) = the lowest action index a with Q(s,a) = (T V)(s)
 *   (T_pi V)(s) = g(s,pi(s)) + gamma * sum_{s'} P(s'|s,pi(s)) V(s')
 *
 * Every sum runs in FP64 in CSR order.  Probabilities and costs may be stored
 * as FP32 or FP64; FP32 values are read exactly (widened to FP64), so the
 * defined problem is the stored values.
 *
 * The states handled are [s0, s0 + n_local); row_ptr is local to that range
 * (n_local*m + 1 entries, first entry 0), col holds global state indices and
 * V is the full value vector of length n.
 */
#include <math.h>
#include <stdint.h>

static double load_val(const float* v32, const double* v64, int64_t i) {
  return v64 ? v64[i] : (double)v32[i];
}

/*
 * One application of T at the states [s0, s0 + n_local):
 * TV[i] = (T V)(s0 + i), pi[i] = greedy action, and, when the pointers are not
 * NULL, Q[i*m + a] = Q(s0 + i, a) and gap[i] = (second smallest Q) - (smallest Q)
 * (INFINITY when m == 1).
 */
void oracle_bellman(int64_t n_local, int32_t m, const int64_t* row_ptr, const int32_t* col,
                    const float* val32, const double* val64, const float* g32, const double* g64,
                    double gamma, const double* V, double* TV, int32_t* pi, double* Q,
                    double* gap) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_local; ++i) {
    double best = INFINITY, second = INFINITY;
    int32_t arg = 0;
    for (int32_t a = 0; a < m; ++a) {
      int64_t r = i * m + a;
      double sum = 0.0;
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) sum += load_val(val32, val64, e) * V[col[e]];
      double q = load_val(g32, g64, r) + gamma * sum;
      if (Q) Q[r] = q;
      if (q < best) {
        second = best;
        best = q;
        arg = a;
      } else if (q < second) {
        second = q;
      }
    }
    TV[i] = best;
    pi[i] = arg;
    if (gap) gap[i] = second - best;
  }
}

/*
 * One application of T_pi at the states [s0, s0 + n_local):
 * out[i] = g(s, pi(s)) + gamma * sum P(s'|s,pi(s)) V(s'),  s = s0 + i.
 */
void oracle_policy_apply(int64_t n_local, int32_t m, const int64_t* row_ptr, const int32_t* col,
                         const float* val32, const double* val64, const float* g32,
                         const double* g64, double gamma, const int32_t* pi, const double* V,
                         double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_local; ++i) {
    int64_t r = i * m + pi[i];
    double sum = 0.0;
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) sum += load_val(val32, val64, e) * V[col[e]];
    out[i] = load_val(g32, g64, r) + gamma * sum;
  }
}
