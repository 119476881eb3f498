// Host-side construction of the CSR MDP that mdp_create takes (mdp_ingest.h):
// from user generators (online simulation), from logged transitions (offline
// data: the maximum-likelihood model), and from/to PETSc binary matrix files.
// No CUDA call in this file; every entry point runs on a host without a GPU.
#include <errno.h>
#include <fcntl.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <exception>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/mdp_ingest.h"

void mdpk_set_last_error(const char* msg);  // the thread-local message of mdp_last_error

namespace {

mdp_status ifail(mdp_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mdp_status ifail(mdp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  mdpk_set_last_error(buf);
  return st;
}

constexpr int64_t kMaxStates = 0x7fffffff;  // columns are int32

int thread_count(int32_t threads, int64_t work) {
  int t = threads > 0 ? threads : static_cast<int>(std::thread::hardware_concurrency());
  if (t < 1) t = 1;
  if (t > 256) t = 256;
  if (work < t) t = static_cast<int>(work < 1 ? 1 : work);
  return t;
}

// f(block, begin, end) over t contiguous blocks of [0, count), one thread each.
// An exception thrown in a block (an allocation failure) is caught in its
// thread and the first one rethrown here after every thread has joined.
template <class F>
void parallel_blocks(int t, int64_t count, F&& f) {
  if (t <= 1) {
    f(0, int64_t(0), count);
    return;
  }
  std::vector<std::exception_ptr> thrown(static_cast<size_t>(t));
  std::vector<std::thread> ws;
  ws.reserve(t);
  try {
    for (int i = 0; i < t; ++i) {
      const int64_t b = count / t * i + std::min<int64_t>(i, count % t);
      const int64_t e = b + count / t + (i < count % t ? 1 : 0);
      ws.emplace_back([&f, &thrown, i, b, e] {
        try {
          f(i, b, e);
        } catch (...) {
          thrown[static_cast<size_t>(i)] = std::current_exception();
        }
      });
    }
  } catch (...) {  // a thread could not start: finish the ones that did, then report
    for (auto& w : ws) w.join();
    throw;
  }
  for (auto& w : ws) w.join();
  for (auto& x : thrown)
    if (x) std::rethrow_exception(x);
}

// Output arrays from the caller's allocator, or malloc (released on failure).
struct Outputs {
  mdp_alloc_fn alloc;
  void* user;
  mdp_host_csr c{};
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 8;  // keep every array non-NULL
    return alloc ? alloc(bytes, user) : malloc(bytes);
  }
  void release() {
    if (c.owned) {
      free(c.row_ptr);
      free(c.col);
      free(c.val);
      free(c.cost);
    }
    memset(&c, 0, sizeof(c));
  }
};

// Sort one row's entries by column (stable) and sum repeated columns in their
// original order; returns the new length.  Rows already strictly ascending
// are left as they are.
int64_t canon_row(int32_t* col, double* val, int64_t k,
                  std::vector<std::pair<int32_t, double>>& tmp) {
  bool ascending = true;
  for (int64_t i = 1; i < k; ++i)
    if (col[i] <= col[i - 1]) {
      ascending = false;
      break;
    }
  if (ascending) return k;
  if (k <= 64) {
    // short rows: stable insertion sort in place (no allocation)
    for (int64_t i = 1; i < k; ++i) {
      const int32_t c = col[i];
      const double v = val[i];
      int64_t j = i;
      for (; j > 0 && col[j - 1] > c; --j) {
        col[j] = col[j - 1];
        val[j] = val[j - 1];
      }
      col[j] = c;
      val[j] = v;
    }
  } else {
    tmp.resize(static_cast<size_t>(k));
    for (int64_t i = 0; i < k; ++i) tmp[i] = {col[i], val[i]};
    std::stable_sort(tmp.begin(), tmp.end(),
                     [](const std::pair<int32_t, double>& x,
                        const std::pair<int32_t, double>& y) { return x.first < y.first; });
    for (int64_t i = 0; i < k; ++i) {
      col[i] = tmp[i].first;
      val[i] = tmp[i].second;
    }
  }
  // sum repeated columns (now adjacent) in their original order
  int64_t w = 0;
  for (int64_t i = 0; i < k; ++i) {
    if (w > 0 && col[i] == col[w - 1]) {
      val[w - 1] += val[i];
    } else {
      col[w] = col[i];
      val[w] = val[i];
      ++w;
    }
  }
  return w;
}

// The first failure of a parallel pass, by row: a thread that fails at row r
// lowers `limit` to r, and every thread stops only past the limit, so the
// error reported is that of the lowest failing row whatever the timing.
struct RowError {
  int64_t row = INT64_MAX;
  mdp_status st = MDP_OK;
  std::string msg;
};

void lower_limit(std::atomic<int64_t>& limit, int64_t r) {
  int64_t cur = limit.load();
  while (r < cur && !limit.compare_exchange_weak(cur, r)) {
  }
}

mdp_status first_error(const std::vector<RowError>& errs) {
  const RowError* best = nullptr;
  for (const RowError& e : errs)
    if (e.st != MDP_OK && (!best || e.row < best->row)) best = &e;
  if (!best) return MDP_OK;
  mdpk_set_last_error(best->msg.c_str());
  return best->st;
}

std::string fmt(const char* f, ...) __attribute__((format(printf, 1, 2)));
std::string fmt(const char* f, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof(buf), f, ap);
  va_end(ap);
  return buf;
}

// Checks of one raw row of state s, action a (before sorting): non-empty,
// successors in [0, n), probabilities finite and non-negative.  Returns MDP_OK,
// or the status with its message in *msg.
mdp_status check_row(int64_t n, int64_t s, int32_t a, const int32_t* col, const double* val,
                     int64_t k, std::string* msg) {
  const long long sl = static_cast<long long>(s);
  if (k == 0) {
    *msg = fmt("row (s, a) = (%lld, %d) has no successor", sl, a);
    return MDP_ERR_NOT_STOCHASTIC;
  }
  for (int64_t i = 0; i < k; ++i) {
    if (col[i] < 0 || col[i] >= n) {
      *msg = fmt("successor %d of (s, a) = (%lld, %d) is outside [0, n)", col[i], sl, a);
      return MDP_ERR_BAD_CSR;
    }
    if (!std::isfinite(val[i])) {
      *msg = fmt("probability of (s, a) = (%lld, %d) is not finite", sl, a);
      return MDP_ERR_NONFINITE;
    }
    if (val[i] < 0.0) {
      *msg = fmt("negative probability in (s, a) = (%lld, %d)", sl, a);
      return MDP_ERR_NOT_STOCHASTIC;
    }
  }
  return MDP_OK;
}

mdp_status check_cost(int64_t s, int32_t a, double g, std::string* msg) {
  if (std::isfinite(g)) return MDP_OK;
  *msg = fmt("cost of (s, a) = (%lld, %d) is not finite", static_cast<long long>(s), a);
  return MDP_ERR_NONFINITE;
}

// row_ptr[1..rows] holds row lengths; turn it into offsets.  Returns nnz.
int64_t prefix_sum(int64_t* row_ptr, int64_t rows) {
  row_ptr[0] = 0;
  for (int64_t r = 0; r < rows; ++r) row_ptr[r + 1] += row_ptr[r];
  return row_ptr[rows];
}

}  // namespace

extern "C" {

void mdp_csr_free(mdp_host_csr* csr) {
  if (!csr) return;
  if (csr->owned) {
    free(csr->row_ptr);
    free(csr->col);
    free(csr->val);
    free(csr->cost);
  }
  memset(csr, 0, sizeof(*csr));
}

mdp_status mdp_csr_from_functions(int64_t n, int32_t m, mdp_row_fn row, mdp_cost_fn cost,
                                  void* user, int32_t threads, mdp_alloc_fn alloc,
                                  void* alloc_user, mdp_host_csr* out) {
  if (!out) return ifail(MDP_ERR_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  if (n < 1 || n > kMaxStates || m < 1)
    return ifail(MDP_ERR_ARG, "need 1 <= n_states < 2^31 and n_actions >= 1");
  if (!row || !cost) return ifail(MDP_ERR_ARG, "NULL generator");
  const int64_t rows = n * m;
  Outputs o{alloc, alloc_user};
  o.c.n_states = n;
  o.c.n_actions = m;
  o.c.owned = alloc ? 0 : 1;
  try {
    o.c.row_ptr = static_cast<int64_t*>(o.get(static_cast<size_t>(rows + 1) * sizeof(int64_t)));
    o.c.cost = static_cast<double*>(o.get(static_cast<size_t>(rows) * sizeof(double)));
    if (!o.c.row_ptr || !o.c.cost) {
      o.release();
      return ifail(MDP_ERR_OOM, "host allocation of %lld rows failed",
                   static_cast<long long>(rows));
    }
    const int T = thread_count(threads, n);
    struct Part {
      std::vector<int32_t> col;
      std::vector<double> val;
    };
    std::vector<Part> parts(T);
    std::vector<RowError> errs(T);
    std::vector<int64_t> first_state(T + 1, n);
    std::atomic<int64_t> limit{INT64_MAX};
    parallel_blocks(T, n, [&](int t, int64_t s0, int64_t s1) {
      first_state[t] = s0;
      Part& p = parts[t];
      RowError& err = errs[t];
      std::vector<int32_t> cb(64);
      std::vector<double> vb(64);
      std::vector<std::pair<int32_t, double>> tmp;
      auto stop = [&](int64_t r, mdp_status st, std::string msg) {
        err.row = r;
        err.st = st;
        err.msg = std::move(msg);
        lower_limit(limit, r);
      };
      try {
        for (int64_t s = s0; s < s1; ++s) {
          for (int32_t a = 0; a < m; ++a) {
            const int64_t r = s * m + a;
            if (r > limit.load(std::memory_order_relaxed)) return;
            const int32_t cap = static_cast<int32_t>(cb.size());
            int32_t k = row(s, a, cap, cb.data(), vb.data(), user);
            if (k > cap) {
              cb.resize(static_cast<size_t>(k));
              vb.resize(static_cast<size_t>(k));
              const int32_t k2 = row(s, a, k, cb.data(), vb.data(), user);
              if (k2 > k)
                return stop(r, MDP_ERR_ARG,
                            fmt("row generator of (s, a) = (%lld, %d) asked for %d entries, then "
                                "%d", static_cast<long long>(s), a, k, k2));
              k = k2;
            }
            if (k < 0)
              return stop(r, MDP_ERR_ARG,
                           fmt("row generator aborted at (s, a) = (%lld, %d) with %d",
                               static_cast<long long>(s), a, k));
            std::string msg;
            mdp_status cs = check_row(n, s, a, cb.data(), vb.data(), k, &msg);
            if (cs != MDP_OK) return stop(r, cs, std::move(msg));
            const int64_t kk = canon_row(cb.data(), vb.data(), k, tmp);
            const double g = cost(s, a, user);
            if ((cs = check_cost(s, a, g, &msg)) != MDP_OK) return stop(r, cs, std::move(msg));
            o.c.cost[r] = g;
            o.c.row_ptr[r + 1] = kk;
            p.col.insert(p.col.end(), cb.begin(), cb.begin() + kk);
            p.val.insert(p.val.end(), vb.begin(), vb.begin() + kk);
          }
        }
      } catch (const std::bad_alloc&) {
        stop(s0 * m, MDP_ERR_OOM, "host allocation failed while building rows");
      }
    });
    mdp_status st = first_error(errs);
    if (st != MDP_OK) {
      o.release();
      return st;
    }
    const int64_t nnz = prefix_sum(o.c.row_ptr, rows);
    o.c.nnz = nnz;
    o.c.col = static_cast<int32_t*>(o.get(static_cast<size_t>(nnz) * sizeof(int32_t)));
    o.c.val = static_cast<double*>(o.get(static_cast<size_t>(nnz) * sizeof(double)));
    if (!o.c.col || !o.c.val) {
      o.release();
      return ifail(MDP_ERR_OOM, "host allocation of %lld entries failed",
                   static_cast<long long>(nnz));
    }
    parallel_blocks(T, T, [&](int, int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        const int64_t off = o.c.row_ptr[first_state[t] * m];
        std::copy(parts[t].col.begin(), parts[t].col.end(), o.c.col + off);
        std::copy(parts[t].val.begin(), parts[t].val.end(), o.c.val + off);
      }
    });
  } catch (const std::bad_alloc&) {
    o.release();
    return ifail(MDP_ERR_OOM, "host allocation failed");
  } catch (const std::system_error& e) {
    o.release();
    return ifail(MDP_ERR_ARG, "could not start host threads: %s", e.what());
  }
  *out = o.c;
  return MDP_OK;
}

mdp_status mdp_csr_from_rows(int64_t n, int32_t m, const int64_t* offsets, const int32_t* col,
                             const double* prob, const double* cost, int32_t threads,
                             mdp_alloc_fn alloc, void* alloc_user, mdp_host_csr* out) {
  if (!out) return ifail(MDP_ERR_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  if (n < 1 || n > kMaxStates || m < 1)
    return ifail(MDP_ERR_ARG, "need 1 <= n_states < 2^31 and n_actions >= 1");
  if (!offsets || !col || !prob || !cost) return ifail(MDP_ERR_ARG, "NULL array argument");
  const int64_t rows = n * m;
  if (offsets[0] != 0) return ifail(MDP_ERR_BAD_CSR, "offsets[0] must be 0");
  for (int64_t r = 0; r < rows; ++r)
    if (offsets[r + 1] < offsets[r])
      return ifail(MDP_ERR_BAD_CSR, "offsets decrease at row %lld", static_cast<long long>(r));
  Outputs o{alloc, alloc_user};
  o.c.n_states = n;
  o.c.n_actions = m;
  o.c.owned = alloc ? 0 : 1;
  try {
    o.c.row_ptr = static_cast<int64_t*>(o.get(static_cast<size_t>(rows + 1) * sizeof(int64_t)));
    o.c.cost = static_cast<double*>(o.get(static_cast<size_t>(rows) * sizeof(double)));
    if (!o.c.row_ptr || !o.c.cost) {
      o.release();
      return ifail(MDP_ERR_OOM, "host allocation of %lld rows failed",
                   static_cast<long long>(rows));
    }
    const int T = thread_count(threads, rows / 1024 + 1);
    // the canonical form of row r, in the caller's scratch vectors; returns its length
    auto canon = [&](int64_t r, std::vector<int32_t>& cb, std::vector<double>& vb,
                     std::vector<std::pair<int32_t, double>>& tmp) {
      const int64_t b = offsets[r], k = offsets[r + 1] - b;
      cb.assign(col + b, col + b + k);
      vb.assign(prob + b, prob + b + k);
      return canon_row(cb.data(), vb.data(), k, tmp);
    };
    // pass 1: checks and canonical lengths
    std::vector<RowError> errs(T);
    std::atomic<int64_t> limit{INT64_MAX};
    parallel_blocks(T, rows, [&](int t, int64_t r0, int64_t r1) {
      std::vector<int32_t> cb;
      std::vector<double> vb;
      std::vector<std::pair<int32_t, double>> tmp;
      try {
        for (int64_t r = r0; r < r1; ++r) {
          if (r > limit.load(std::memory_order_relaxed)) return;
          const int64_t s = r / m;
          const int32_t a = static_cast<int32_t>(r % m);
          std::string msg;
          mdp_status cs = check_row(n, s, a, col + offsets[r], prob + offsets[r],
                                    offsets[r + 1] - offsets[r], &msg);
          if (cs == MDP_OK) cs = check_cost(s, a, cost[r], &msg);
          if (cs != MDP_OK) {
            errs[t] = RowError{r, cs, std::move(msg)};
            lower_limit(limit, r);
            return;
          }
          o.c.row_ptr[r + 1] = canon(r, cb, vb, tmp);
          o.c.cost[r] = cost[r];
        }
      } catch (const std::bad_alloc&) {
        errs[t] = RowError{r0, MDP_ERR_OOM, "host allocation failed while sorting rows"};
        lower_limit(limit, r0);
      }
    });
    mdp_status st = first_error(errs);
    if (st != MDP_OK) {
      o.release();
      return st;
    }
    const int64_t nnz = prefix_sum(o.c.row_ptr, rows);
    o.c.nnz = nnz;
    o.c.col = static_cast<int32_t*>(o.get(static_cast<size_t>(nnz) * sizeof(int32_t)));
    o.c.val = static_cast<double*>(o.get(static_cast<size_t>(nnz) * sizeof(double)));
    if (!o.c.col || !o.c.val) {
      o.release();
      return ifail(MDP_ERR_OOM, "host allocation of %lld entries failed",
                   static_cast<long long>(nnz));
    }
    // pass 2: the canonical rows into place
    parallel_blocks(T, rows, [&](int, int64_t r0, int64_t r1) {
      std::vector<int32_t> cb;
      std::vector<double> vb;
      std::vector<std::pair<int32_t, double>> tmp;
      for (int64_t r = r0; r < r1; ++r) {
        const int64_t kk = canon(r, cb, vb, tmp);
        std::copy(cb.begin(), cb.begin() + kk, o.c.col + o.c.row_ptr[r]);
        std::copy(vb.begin(), vb.begin() + kk, o.c.val + o.c.row_ptr[r]);
      }
    });
  } catch (const std::bad_alloc&) {
    o.release();
    return ifail(MDP_ERR_OOM, "host allocation failed");
  } catch (const std::system_error& e) {
    o.release();
    return ifail(MDP_ERR_ARG, "could not start host threads: %s", e.what());
  }
  *out = o.c;
  return MDP_OK;
}

mdp_status mdp_csr_from_samples(int64_t n, int32_t m, int64_t count, const int64_t* s,
                                const int32_t* a, const int64_t* s_next, const double* c,
                                int32_t unseen, double unseen_cost, int32_t threads,
                                mdp_alloc_fn alloc, void* alloc_user, mdp_host_csr* out) {
  if (!out) return ifail(MDP_ERR_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  if (n < 1 || n > kMaxStates || m < 1)
    return ifail(MDP_ERR_ARG, "need 1 <= n_states < 2^31 and n_actions >= 1");
  if (count < 0) return ifail(MDP_ERR_ARG, "count must be >= 0");
  if (count > 0 && (!s || !a || !s_next)) return ifail(MDP_ERR_ARG, "NULL sample array");
  if (unseen != MDP_UNSEEN_ERROR && unseen != MDP_UNSEEN_SELF_LOOP)
    return ifail(MDP_ERR_ARG, "unseen must be MDP_UNSEEN_ERROR or MDP_UNSEEN_SELF_LOOP");
  if (unseen == MDP_UNSEEN_SELF_LOOP && !std::isfinite(unseen_cost))
    return ifail(MDP_ERR_ARG, "unseen_cost must be finite");
  const int64_t rows = n * m;
  Outputs o{alloc, alloc_user};
  o.c.n_states = n;
  o.c.n_actions = m;
  o.c.owned = alloc ? 0 : 1;
  try {
    // samples grouped by row r = s*m + a, in sample order (a stable counting sort)
    std::vector<int64_t> start(static_cast<size_t>(rows + 1), 0);
    for (int64_t i = 0; i < count; ++i) {
      if (s[i] < 0 || s[i] >= n || a[i] < 0 || a[i] >= m || s_next[i] < 0 || s_next[i] >= n)
        return ifail(MDP_ERR_ARG,
                     "sample %lld: (s, a, s') = (%lld, %d, %lld) is outside the %lld x %d MDP",
                     static_cast<long long>(i), static_cast<long long>(s[i]), a[i],
                     static_cast<long long>(s_next[i]), static_cast<long long>(n), m);
      if (c && !std::isfinite(c[i]))
        return ifail(MDP_ERR_NONFINITE, "sample %lld: the cost is not finite",
                     static_cast<long long>(i));
      ++start[static_cast<size_t>(s[i] * m + a[i] + 1)];
    }
    if (unseen == MDP_UNSEEN_ERROR)
      for (int64_t r = 0; r < rows; ++r)
        if (start[r + 1] == 0)
          return ifail(MDP_ERR_ARG, "no sample of (s, a) = (%lld, %d)",
                       static_cast<long long>(r / m), static_cast<int>(r % m));
    for (int64_t r = 0; r < rows; ++r) start[r + 1] += start[r];
    std::vector<int32_t> next(static_cast<size_t>(count));
    std::vector<double> csum(static_cast<size_t>(rows), 0.0);
    {
      std::vector<int64_t> fill(start.begin(), start.end() - 1);
      for (int64_t i = 0; i < count; ++i) {
        const int64_t r = s[i] * m + a[i];
        next[static_cast<size_t>(fill[r]++)] = static_cast<int32_t>(s_next[i]);
        if (c) csum[r] += c[i];
      }
    }
    o.c.row_ptr = static_cast<int64_t*>(o.get(static_cast<size_t>(rows + 1) * sizeof(int64_t)));
    o.c.cost = static_cast<double*>(o.get(static_cast<size_t>(rows) * sizeof(double)));
    if (!o.c.row_ptr || !o.c.cost) {
      o.release();
      return ifail(MDP_ERR_OOM, "host allocation of %lld rows failed",
                   static_cast<long long>(rows));
    }
    // per row: sort the successors, count the distinct ones
    const int T = thread_count(threads, rows);
    parallel_blocks(T, rows, [&](int, int64_t r0, int64_t r1) {
      for (int64_t r = r0; r < r1; ++r) {
        int32_t* b = next.data() + start[r];
        int32_t* e = next.data() + start[r + 1];
        std::sort(b, e);
        int64_t k = b == e ? 1 : 0;  // an unseen pair becomes a self-loop
        for (int32_t* p = b; p < e; ++p) k += (p == b || p[0] != p[-1]) ? 1 : 0;
        o.c.row_ptr[r + 1] = k;
      }
    });
    const int64_t nnz = prefix_sum(o.c.row_ptr, rows);
    o.c.nnz = nnz;
    o.c.col = static_cast<int32_t*>(o.get(static_cast<size_t>(nnz) * sizeof(int32_t)));
    o.c.val = static_cast<double*>(o.get(static_cast<size_t>(nnz) * sizeof(double)));
    if (!o.c.col || !o.c.val) {
      o.release();
      return ifail(MDP_ERR_OOM, "host allocation of %lld entries failed",
                   static_cast<long long>(nnz));
    }
    parallel_blocks(T, rows, [&](int, int64_t r0, int64_t r1) {
      for (int64_t r = r0; r < r1; ++r) {
        const int64_t N = start[r + 1] - start[r];
        int64_t w = o.c.row_ptr[r];
        if (N == 0) {
          o.c.col[w] = static_cast<int32_t>(r / m);
          o.c.val[w] = 1.0;
          o.c.cost[r] = unseen_cost;
          continue;
        }
        const int32_t* b = next.data() + start[r];
        for (int64_t i = 0; i < N;) {
          int64_t j = i + 1;
          while (j < N && b[j] == b[i]) ++j;
          o.c.col[w] = b[i];
          o.c.val[w] = static_cast<double>(j - i) / static_cast<double>(N);
          ++w;
          i = j;
        }
        o.c.cost[r] = c ? csum[r] / static_cast<double>(N) : 0.0;
      }
    });
  } catch (const std::bad_alloc&) {
    o.release();
    return ifail(MDP_ERR_OOM, "host allocation failed");
  } catch (const std::system_error& e) {
    o.release();
    return ifail(MDP_ERR_ARG, "could not start host threads: %s", e.what());
  }
  *out = o.c;
  return MDP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// PETSc binary matrix files (big-endian): header {class id, rows, columns,
// nonzeros or -1 for dense}; sparse: row lengths, column indices, values;
// dense: the values by rows.  Integers 32-bit, or 64-bit from PETSc builds
// with 64-bit indices; values IEEE doubles.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kMatClassId = 1211216;
constexpr int64_t kDenseFormat = -1;
constexpr int64_t kChunkBytes = int64_t(64) << 20;

uint32_t be32(const unsigned char* p) {
  return (uint32_t(p[0]) << 24) | (uint32_t(p[1]) << 16) | (uint32_t(p[2]) << 8) | uint32_t(p[3]);
}
uint64_t be64(const unsigned char* p) {
  return (uint64_t(be32(p)) << 32) | uint64_t(be32(p + 4));
}
void put_be32(unsigned char* p, uint32_t v) {
  p[0] = static_cast<unsigned char>(v >> 24);
  p[1] = static_cast<unsigned char>(v >> 16);
  p[2] = static_cast<unsigned char>(v >> 8);
  p[3] = static_cast<unsigned char>(v);
}
void put_be64(unsigned char* p, uint64_t v) {
  put_be32(p, static_cast<uint32_t>(v >> 32));
  put_be32(p + 4, static_cast<uint32_t>(v));
}
double as_double(uint64_t bits) {
  double d;
  memcpy(&d, &bits, sizeof(d));
  return d;
}
uint64_t bits_of(double d) {
  uint64_t b;
  memcpy(&b, &d, sizeof(b));
  return b;
}

// Positional reads (pread) so that several threads fill disjoint slices of an
// array at once; `pos` is the offset of the next sequential read.
struct Reader {
  int fd = -1;
  const char* path = "";
  int64_t size = 0;
  int64_t pos = 0;
  ~Reader() {
    if (fd >= 0) close(fd);
  }
  mdp_status open(const char* p) {
    path = p;
    fd = ::open(p, O_RDONLY);
    if (fd < 0) return ifail(MDP_ERR_ARG, "cannot open %s", p);
    struct stat sb;
    if (fstat(fd, &sb) != 0) return ifail(MDP_ERR_ARG, "cannot stat %s", p);
    size = static_cast<int64_t>(sb.st_size);
    return MDP_OK;
  }
  // Read bytes at an absolute offset; false on a short read or an error.
  bool read_at(void* dst, int64_t bytes, int64_t off) const {
    unsigned char* d = static_cast<unsigned char*>(dst);
    while (bytes > 0) {
      const ssize_t got = pread(fd, d, static_cast<size_t>(std::min<int64_t>(bytes, 1 << 30)),
                                static_cast<off_t>(off));
      if (got < 0 && errno == EINTR) continue;
      if (got <= 0) return false;
      d += got;
      off += got;
      bytes -= got;
    }
    return true;
  }
  bool read(void* dst, int64_t bytes) {
    if (!read_at(dst, bytes, pos)) return false;
    pos += bytes;
    return true;
  }
  mdp_status truncated() { return ifail(MDP_ERR_ARG, "%s is truncated", path); }
};

struct MatHeader {
  int w = 4;  // integer width in bytes
  int64_t rows = 0, cols = 0, nz = 0;
};

mdp_status read_header(Reader& rd, MatHeader* h) {
  unsigned char b[32];
  if (!rd.read(b, 4)) return rd.truncated();
  if (be32(b) == static_cast<uint32_t>(kMatClassId)) {
    h->w = 4;
    if (!rd.read(b + 4, 12)) return rd.truncated();
    h->rows = static_cast<int32_t>(be32(b + 4));
    h->cols = static_cast<int32_t>(be32(b + 8));
    h->nz = static_cast<int32_t>(be32(b + 12));
  } else {
    if (!rd.read(b + 4, 4)) return rd.truncated();
    if (be64(b) != static_cast<uint64_t>(kMatClassId))
      return ifail(MDP_ERR_ARG, "%s is not a PETSc binary matrix (class id %u)", rd.path,
                   be32(b));
    h->w = 8;
    if (!rd.read(b + 8, 24)) return rd.truncated();
    h->rows = static_cast<int64_t>(be64(b + 8));
    h->cols = static_cast<int64_t>(be64(b + 16));
    h->nz = static_cast<int64_t>(be64(b + 24));
  }
  if (h->rows < 0 || h->cols < 0 || h->nz < kDenseFormat)
    return ifail(MDP_ERR_ARG, "%s: bad matrix header (%lld x %lld, nz %lld)", rd.path,
                 static_cast<long long>(h->rows), static_cast<long long>(h->cols),
                 static_cast<long long>(h->nz));
  return MDP_OK;
}

// Read `count` big-endian integers of width w from the current position;
// sink(i, value) sees each one.  T threads each read and decode a contiguous
// slice (disjoint i).  Returns false on a short read.
template <class Sink>
bool read_ints(Reader& rd, int w, int64_t count, int T, Sink&& sink) {
  const int64_t base_off = rd.pos;
  std::atomic<int> short_read{0};
  parallel_blocks(thread_count(T, count / 65536), count, [&](int, int64_t i0, int64_t i1) {
    const int64_t chunk = kChunkBytes / 8 / w;  // entries per read
    std::vector<unsigned char> buf(static_cast<size_t>(std::min(chunk, i1 - i0) * w));
    for (int64_t b = i0; b < i1; b += chunk) {
      const int64_t k = std::min(chunk, i1 - b);
      if (!rd.read_at(buf.data(), k * w, base_off + b * w)) {
        short_read.store(1);
        return;
      }
      for (int64_t i = 0; i < k; ++i) {
        const unsigned char* p = buf.data() + i * w;
        const int64_t v = w == 4 ? static_cast<int64_t>(static_cast<int32_t>(be32(p)))
                                 : static_cast<int64_t>(be64(p));
        sink(b + i, v);
      }
    }
  });
  rd.pos = base_off + count * w;
  return short_read.load() == 0;
}

// Read `count` big-endian doubles into dst (each thread reads its slice in
// place and converts it); returns false on a short read.  *bad receives the
// lowest index of a NaN/Inf (or -1).
bool read_doubles(Reader& rd, int64_t count, int T, double* dst, int64_t* bad) {
  const int64_t base_off = rd.pos;
  std::atomic<int64_t> first{INT64_MAX};
  std::atomic<int> short_read{0};
  parallel_blocks(thread_count(T, count / 65536), count, [&](int, int64_t i0, int64_t i1) {
    unsigned char* raw = reinterpret_cast<unsigned char*>(dst + i0);
    if (!rd.read_at(raw, (i1 - i0) * 8, base_off + i0 * 8)) {
      short_read.store(1);
      return;
    }
    for (int64_t i = i0; i < i1; ++i) {
      const double v = as_double(be64(reinterpret_cast<unsigned char*>(dst + i)));
      dst[i] = v;
      if (!std::isfinite(v)) lower_limit(first, i);
    }
  });
  rd.pos = base_off + count * 8;
  *bad = first.load() == INT64_MAX ? -1 : first.load();
  return short_read.load() == 0;
}

// Positional writes: every array of the file is encoded by T threads, each
// turning a contiguous slice into big-endian bytes and writing it at its own
// offset, so the file is the same whatever the thread count.
struct Writer {
  int fd = -1;
  const char* path = "";
  std::atomic<bool> ok{true};  // cleared by any thread whose write fails
  int64_t pos = 0;
  ~Writer() {
    if (fd >= 0) close(fd);
  }
  mdp_status open(const char* p) {
    path = p;
    fd = ::open(p, O_WRONLY | O_CREAT | O_TRUNC, 0644);
    if (fd < 0) return ifail(MDP_ERR_ARG, "cannot create %s", p);
    return MDP_OK;
  }
  void write_at(const unsigned char* src, int64_t bytes, int64_t off) {
    while (bytes > 0) {
      const ssize_t put = pwrite(fd, src, static_cast<size_t>(std::min<int64_t>(bytes, 1 << 30)),
                                 static_cast<off_t>(off));
      if (put < 0 && errno == EINTR) continue;
      if (put <= 0) {
        ok.store(false);
        return;
      }
      src += put;
      off += put;
      bytes -= put;
    }
  }
  // Append `count` items, item i encoded by enc(i, p) into `width` bytes at p.
  template <class Enc>
  void put_array(int64_t count, int width, Enc&& enc) {
    const int64_t base = pos;
    parallel_blocks(thread_count(0, count / 65536), count, [&](int, int64_t i0, int64_t i1) {
      const int64_t chunk = (int64_t(8) << 20) / width;
      std::vector<unsigned char> buf(static_cast<size_t>(std::min(chunk, i1 - i0) * width));
      for (int64_t b = i0; b < i1; b += chunk) {
        const int64_t k = std::min(chunk, i1 - b);
        for (int64_t i = 0; i < k; ++i) enc(b + i, buf.data() + i * width);
        write_at(buf.data(), k * width, base + b * width);
      }
    });
    pos = base + count * width;
  }
  void put_ints(int w, const int64_t* v, int count) {
    unsigned char b[32];
    for (int i = 0; i < count; ++i) {
      if (w == 4) put_be32(b + 4 * i, static_cast<uint32_t>(static_cast<int32_t>(v[i])));
      else put_be64(b + 8 * i, static_cast<uint64_t>(v[i]));
    }
    write_at(b, static_cast<int64_t>(count) * w, pos);
    pos += static_cast<int64_t>(count) * w;
  }
  mdp_status finish() {
    const int rc = close(fd);
    fd = -1;
    return ok.load() && rc == 0 ? MDP_OK : ifail(MDP_ERR_ARG, "write to %s failed", path);
  }
};

}  // namespace

extern "C" {

mdp_status mdp_csr_read_petsc(const char* p_path, const char* g_path, int32_t threads,
                              mdp_alloc_fn alloc, void* alloc_user, mdp_host_csr* out) {
  if (!out) return ifail(MDP_ERR_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  if (!p_path) return ifail(MDP_ERR_ARG, "p_path is NULL");
  Outputs o{alloc, alloc_user};
  o.c.owned = alloc ? 0 : 1;
  auto bail = [&](mdp_status st) {
    o.release();
    return st;
  };
  try {
    Reader rp;
    mdp_status st = rp.open(p_path);
    if (st != MDP_OK) return st;
    MatHeader hp;
    if ((st = read_header(rp, &hp)) != MDP_OK) return st;
    if (hp.nz == kDenseFormat) return ifail(MDP_ERR_ARG, "%s: P must be a sparse matrix", p_path);
    const int64_t n = hp.cols, rows = hp.rows, nz = hp.nz;
    if (n < 1 || n > kMaxStates || rows < n || rows % n != 0 || rows / n > 0x7fffffff)
      return ifail(MDP_ERR_ARG,
                   "%s: P is %lld x %lld; it must have n*m rows for its n columns (states)",
                   p_path, static_cast<long long>(rows), static_cast<long long>(n));
    const int64_t m = rows / n;
    const int w = hp.w;
    if (rows > rp.size / w || nz > (rp.size - 4 * w - rows * w) / (w + 8))
      return rp.truncated();
    const int T = thread_count(threads, rows);
    o.c.n_states = n;
    o.c.n_actions = static_cast<int32_t>(m);
    o.c.row_ptr = static_cast<int64_t*>(o.get(static_cast<size_t>(rows + 1) * sizeof(int64_t)));
    o.c.col = static_cast<int32_t*>(o.get(static_cast<size_t>(nz) * sizeof(int32_t)));
    o.c.val = static_cast<double*>(o.get(static_cast<size_t>(nz) * sizeof(double)));
    o.c.cost = static_cast<double*>(o.get(static_cast<size_t>(rows) * sizeof(double)));
    if (!o.c.row_ptr || !o.c.col || !o.c.val || !o.c.cost)
      return bail(ifail(MDP_ERR_OOM, "host allocation for %lld entries failed",
                        static_cast<long long>(nz)));
    std::atomic<int64_t> bad{INT64_MAX};
    if (!read_ints(rp, w, rows, T, [&](int64_t i, int64_t v) {
          if (v < 0 || v > nz) lower_limit(bad, i);
          o.c.row_ptr[i + 1] = v;
        }))
      return bail(rp.truncated());
    if (bad.load() != INT64_MAX)
      return bail(ifail(MDP_ERR_ARG, "%s: row %lld has a bad length", p_path,
                        static_cast<long long>(bad.load())));
    if (prefix_sum(o.c.row_ptr, rows) != nz)
      return bail(ifail(MDP_ERR_ARG, "%s: the row lengths do not add up to %lld", p_path,
                        static_cast<long long>(nz)));
    if (!read_ints(rp, w, nz, T, [&](int64_t i, int64_t v) {
          if (v < 0 || v >= n) lower_limit(bad, i);
          o.c.col[i] = static_cast<int32_t>(v);
        }))
      return bail(rp.truncated());
    if (bad.load() != INT64_MAX)
      return bail(ifail(MDP_ERR_BAD_CSR, "%s: column index %lld is outside [0, %lld)", p_path,
                        static_cast<long long>(bad.load()), static_cast<long long>(n)));
    int64_t bad_val = -1;
    if (!read_doubles(rp, nz, T, o.c.val, &bad_val)) return bail(rp.truncated());
    if (bad_val >= 0)
      return bail(ifail(MDP_ERR_NONFINITE, "%s: value %lld is not finite", p_path,
                        static_cast<long long>(bad_val)));
    // columns ascending and unique within each row; compact if a row shrank
    std::vector<int64_t> len(static_cast<size_t>(rows));
    std::atomic<int> shrank{0};
    parallel_blocks(T, rows, [&](int, int64_t r0, int64_t r1) {
      std::vector<std::pair<int32_t, double>> tmp;
      for (int64_t r = r0; r < r1; ++r) {
        const int64_t b = o.c.row_ptr[r], k = o.c.row_ptr[r + 1] - b;
        len[r] = canon_row(o.c.col + b, o.c.val + b, k, tmp);
        if (len[r] != k) shrank.store(1);
      }
    });
    o.c.nnz = nz;
    if (shrank.load()) {
      int64_t wpos = 0;
      for (int64_t r = 0; r < rows; ++r) {
        const int64_t b = o.c.row_ptr[r];
        memmove(o.c.col + wpos, o.c.col + b, static_cast<size_t>(len[r]) * sizeof(int32_t));
        memmove(o.c.val + wpos, o.c.val + b, static_cast<size_t>(len[r]) * sizeof(double));
        o.c.row_ptr[r] = wpos;
        wpos += len[r];
      }
      o.c.row_ptr[rows] = wpos;
      o.c.nnz = wpos;
    }
    // costs: n x m, dense or sparse; zero without a file
    std::fill(o.c.cost, o.c.cost + rows, 0.0);
    if (g_path) {
      Reader rg;
      if ((st = rg.open(g_path)) != MDP_OK) return bail(st);
      MatHeader hg;
      if ((st = read_header(rg, &hg)) != MDP_OK) return bail(st);
      if (hg.rows != n || hg.cols != m)
        return bail(ifail(MDP_ERR_ARG, "%s: the costs are %lld x %lld, P needs %lld x %lld",
                          g_path, static_cast<long long>(hg.rows),
                          static_cast<long long>(hg.cols), static_cast<long long>(n),
                          static_cast<long long>(m)));
      if (hg.nz == kDenseFormat) {
        if (rows > (rg.size - 4 * hg.w) / 8) return bail(rg.truncated());
        if (!read_doubles(rg, rows, T, o.c.cost, &bad_val)) return bail(rg.truncated());
      } else {
        const int64_t gz = hg.nz;
        if (gz > (rg.size - 4 * hg.w - n * hg.w) / (hg.w + 8)) return bail(rg.truncated());
        std::vector<int64_t> grp(static_cast<size_t>(n + 1), 0);
        std::vector<int64_t> gcol(static_cast<size_t>(gz));
        std::vector<double> gval(static_cast<size_t>(gz));
        if (!read_ints(rg, hg.w, n, T, [&](int64_t i, int64_t v) {
              if (v < 0 || v > m) lower_limit(bad, i);
              grp[i + 1] = v;
            }))
          return bail(rg.truncated());
        if (bad.load() != INT64_MAX || prefix_sum(grp.data(), n) != gz)
          return bail(ifail(MDP_ERR_ARG, "%s: bad row lengths", g_path));
        if (!read_ints(rg, hg.w, gz, T, [&](int64_t i, int64_t v) {
              if (v < 0 || v >= m) lower_limit(bad, i);
              gcol[i] = v;
            }))
          return bail(rg.truncated());
        if (bad.load() != INT64_MAX)
          return bail(ifail(MDP_ERR_ARG, "%s: an action index is outside [0, %lld)", g_path,
                            static_cast<long long>(m)));
        if (!read_doubles(rg, gz, T, gval.data(), &bad_val)) return bail(rg.truncated());
        if (bad_val < 0)
          for (int64_t s = 0; s < n; ++s)
            for (int64_t e = grp[s]; e < grp[s + 1]; ++e) o.c.cost[s * m + gcol[e]] += gval[e];
      }
      if (bad_val >= 0)
        return bail(ifail(MDP_ERR_NONFINITE, "%s: value %lld is not finite", g_path,
                          static_cast<long long>(bad_val)));
    }
  } catch (const std::bad_alloc&) {
    return bail(ifail(MDP_ERR_OOM, "host allocation failed"));
  } catch (const std::system_error& e) {
    return bail(ifail(MDP_ERR_ARG, "could not start host threads: %s", e.what()));
  }
  *out = o.c;
  return MDP_OK;
}

mdp_status mdp_csr_write_petsc(const mdp_host_csr* c, const char* p_path, const char* g_path) {
  if (!c || !c->row_ptr || (p_path && (!c->col || !c->val)) || (g_path && !c->cost))
    return ifail(MDP_ERR_ARG, "NULL csr or array");
  if (c->n_states < 1 || c->n_actions < 1) return ifail(MDP_ERR_ARG, "empty csr");
  const int64_t n = c->n_states, m = c->n_actions, rows = n * m, nnz = c->row_ptr[rows];
  try {
    if (p_path) {
      const int w = (rows <= 0x7fffffff && nnz <= 0x7fffffff) ? 4 : 8;
      Writer wr;
      mdp_status st = wr.open(p_path);
      if (st != MDP_OK) return st;
      const int64_t head[4] = {kMatClassId, rows, n, nnz};
      wr.put_ints(w, head, 4);
      auto put_int = [w](int64_t v, unsigned char* p) {
        if (w == 4) put_be32(p, static_cast<uint32_t>(static_cast<int32_t>(v)));
        else put_be64(p, static_cast<uint64_t>(v));
      };
      wr.put_array(rows, w, [&](int64_t r, unsigned char* p) {
        put_int(c->row_ptr[r + 1] - c->row_ptr[r], p);
      });
      wr.put_array(nnz, w, [&](int64_t e, unsigned char* p) { put_int(c->col[e], p); });
      wr.put_array(nnz, 8, [&](int64_t e, unsigned char* p) { put_be64(p, bits_of(c->val[e])); });
      if ((st = wr.finish()) != MDP_OK) return st;
    }
    if (g_path) {
      Writer wr;
      mdp_status st = wr.open(g_path);
      if (st != MDP_OK) return st;
      const int64_t head[4] = {kMatClassId, n, m, kDenseFormat};
      wr.put_ints(4, head, 4);
      wr.put_array(rows, 8, [&](int64_t r, unsigned char* p) { put_be64(p, bits_of(c->cost[r])); });
      if ((st = wr.finish()) != MDP_OK) return st;
    }
  } catch (const std::bad_alloc&) {
    return ifail(MDP_ERR_OOM, "host allocation failed");
  } catch (const std::system_error& e) {
    return ifail(MDP_ERR_ARG, "could not start host threads: %s", e.what());
  }
  return MDP_OK;
}

}  // extern "C"
