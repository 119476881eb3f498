/*
 * Seeded synthetic MDP generators (host C, OpenMP over rows).
 *
 * These produce the CSR transition matrices and stage costs that both the
 * FP64 CPU oracle and the GPU solver consume.  They hold none of the solver's
 * arithmetic: only random draws, sorting, normalisation of the drawn weights
 * and the CSR layout.
 *
 * Layout (shared by every generator):
 *   state s in [0, n), action a in [0, m), row r = s*m + a  (state-major),
 *   row_ptr[n*m+1] int64, col[nnz] int32 ascending within a row, no
 *   duplicates, val[nnz] the transition probabilities P(col | s, a),
 *   g[n*m] the stage cost g(s, a).
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), keyed by the seed, with the counter
 * (row low, row high, stream, draw index).  Every row draws from its own
 * counter space, so the output is independent of the thread count and any
 * state sub-range can be regenerated on its own.
 *
 * Probabilities: Dirichlet(alpha) = normalised Gamma(alpha, 1) draws
 * (Marsaglia & Tsang, "A simple method for generating gamma variables",
 * ACM TOMS 2000, with the alpha < 1 boost G(a) = G(a+1) U^(1/a)), normalised
 * in FP64 and stored as FP64 or FP32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- Philox4x32-10 ---------------- */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A stream of 32-bit words for one (seed, row, stream id). */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t buf[4];
  int left;
} rng_t;

static void rng_init(rng_t* g, uint64_t seed, uint64_t row, uint32_t stream) {
  g->key[0] = (uint32_t)seed;
  g->key[1] = (uint32_t)(seed >> 32);
  g->ctr[0] = (uint32_t)row;
  g->ctr[1] = (uint32_t)(row >> 32);
  g->ctr[2] = stream;
  g->ctr[3] = 0;
  g->left = 0;
}

static uint32_t rng_u32(rng_t* g) {
  if (g->left == 0) {
    synth_philox4x32_10(g->ctr, g->key, g->buf);
    g->ctr[3] += 1;
    g->left = 4;
  }
  return g->buf[4 - (g->left--)];
}

/* Uniform double in the open interval (0, 1) with 53 random bits. */
static double rng_open01(rng_t* g) {
  uint64_t a = rng_u32(g) >> 5; /* 27 bits */
  uint64_t b = rng_u32(g) >> 6; /* 26 bits */
  uint64_t x = (a << 26) | b;   /* 53 bits */
  return ((double)x + 0.5) * (1.0 / 9007199254740992.0);
}

/* Uniform integer in [0, range) without modulo bias (Lemire-style rejection). */
static uint32_t rng_below(rng_t* g, uint32_t range) {
  uint64_t m = (uint64_t)rng_u32(g) * (uint64_t)range;
  uint32_t lo = (uint32_t)m;
  if (lo < range) {
    uint32_t t = (uint32_t)(-range) % range;
    while (lo < t) {
      m = (uint64_t)rng_u32(g) * (uint64_t)range;
      lo = (uint32_t)m;
    }
  }
  return (uint32_t)(m >> 32);
}

static double rng_normal(rng_t* g) {
  /* Box-Muller, one of the pair. */
  double u1 = rng_open01(g), u2 = rng_open01(g);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

static double rng_gamma(rng_t* g, double alpha) {
  if (alpha < 1.0) {
    double x = rng_gamma(g, alpha + 1.0);
    double u = rng_open01(g);
    return x * pow(u, 1.0 / alpha);
  }
  double d = alpha - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  for (;;) {
    double x, v;
    do {
      x = rng_normal(g);
      v = 1.0 + c * x;
    } while (v <= 0.0);
    v = v * v * v;
    double u = rng_open01(g);
    if (u < 1.0 - 0.0331 * x * x * x * x) return d * v;
    if (log(u) < 0.5 * x * x + d * (1.0 - v + log(v))) return d * v;
  }
}

/* Stream ids. */
enum { ST_SUCC = 1, ST_PROB = 2, ST_COST = 3, ST_LEN = 4, ST_GOAL = 5 };

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Draw k distinct states uniformly from [lo, lo+width), sorted ascending. */
static void draw_distinct(rng_t* g, int64_t lo, int64_t width, int k, int32_t* out) {
  for (int i = 0; i < k; ++i) {
    for (;;) {
      int32_t c = (int32_t)(lo + (int64_t)rng_below(g, (uint32_t)width));
      int dup = 0;
      for (int j = 0; j < i; ++j)
        if (out[j] == c) { dup = 1; break; }
      if (!dup) { out[i] = c; break; }
    }
  }
  qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
}

static void draw_dirichlet(rng_t* g, double alpha, int k, double* w) {
  double s = 0.0;
  for (int i = 0; i < k; ++i) {
    w[i] = rng_gamma(g, alpha);
    s += w[i];
  }
  for (int i = 0; i < k; ++i) w[i] /= s;
}

static void put_val(void* val, int val_f64, int64_t e, double p) {
  if (val_f64) ((double*)val)[e] = p;
  else ((float*)val)[e] = (float)p;
}

/*
 * Per-row successor count for the random/banded generators: k_min..k_max
 * uniform (k_min == k_max gives a fixed count).
 */
static int row_len(uint64_t seed, int64_t r, int k_min, int k_max) {
  if (k_min == k_max) return k_min;
  rng_t g;
  rng_init(&g, seed, (uint64_t)r, ST_LEN);
  return k_min + (int)rng_below(&g, (uint32_t)(k_max - k_min + 1));
}

/*
 * Row pointers of a random or banded MDP for the states [s0, s1).
 * row_ptr has (s1-s0)*m + 1 entries and starts at 0.
 */
int64_t synth_random_row_ptr(int64_t s0, int64_t s1, int32_t m, int32_t k_min, int32_t k_max,
                             uint64_t seed, int64_t* row_ptr) {
  int64_t rows = (s1 - s0) * (int64_t)m;
  row_ptr[0] = 0;
  if (k_min == k_max) {
    for (int64_t i = 0; i < rows; ++i) row_ptr[i + 1] = (i + 1) * (int64_t)k_min;
    return rows * (int64_t)k_min;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i) row_ptr[i + 1] = row_len(seed, s0 * m + i, k_min, k_max);
  for (int64_t i = 0; i < rows; ++i) row_ptr[i + 1] += row_ptr[i];
  return row_ptr[rows];
}

/*
 * Random (band < 0) or banded (band >= 0) MDP over the states [s0, s1) of an
 * n-state MDP.  Row r = s*m + a draws its successor count, then that many
 * distinct successors uniformly from all n states (band < 0) or from the
 * clipped window [max(0, s-band), min(n-1, s+band)] (band >= 0), then
 * Dirichlet(alpha) probabilities over them, and a cost g ~ U[0, 1].
 * row_ptr must already hold synth_random_row_ptr's output for the same range.
 * Exactly one of val_f64 / val_f32 selects the stored precision (likewise g).
 * Returns 0, or -1 when a row asks for more successors than its window has.
 */
int synth_random_fill(int64_t n, int64_t s0, int64_t s1, int32_t m, int64_t band, double alpha,
                      uint64_t seed, const int64_t* row_ptr, int32_t* col, void* val,
                      int32_t val_is_f64, void* g, int32_t g_is_f64) {
  int64_t rows = (s1 - s0) * (int64_t)m;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : bad)
  for (int64_t i = 0; i < rows; ++i) {
    int64_t r = s0 * m + i;
    int64_t s = r / m;
    int64_t b = row_ptr[i], e = row_ptr[i + 1];
    int k = (int)(e - b);
    int64_t lo = 0, width = n;
    if (band >= 0) {
      lo = s - band < 0 ? 0 : s - band;
      int64_t hi = s + band > n - 1 ? n - 1 : s + band;
      width = hi - lo + 1;
    }
    if (k > width || k > 4096) { bad |= 1; continue; }
    rng_t gs, gp, gc;
    rng_init(&gs, seed, (uint64_t)r, ST_SUCC);
    rng_init(&gp, seed, (uint64_t)r, ST_PROB);
    rng_init(&gc, seed, (uint64_t)r, ST_COST);
    double w[4096];
    draw_distinct(&gs, lo, width, k, col + b);
    draw_dirichlet(&gp, alpha, k, w);
    for (int j = 0; j < k; ++j) put_val(val, val_is_f64, b + j, w[j]);
    double c = rng_open01(&gc);
    if (g_is_f64) ((double*)g)[i] = c;
    else ((float*)g)[i] = (float)c;
  }
  return bad ? -1 : 0;
}

/*
 * 2-D grid world.  States s = y*W + x on a W x H grid; actions in the order
 * N (y-1), E (x+1), S (y+1), W (x-1), stay.  Action a moves to its intended
 * cell with probability p_int and to each of the other four cells of the
 * 5-point stencil {self, N, E, S, W} with probability p_oth.  A move off the
 * grid stays in place (reflecting wall) and its mass is merged into the self
 * entry, so border rows have fewer than five entries.  Cost 1 for every (s, a)
 * except the goal cells, where it is 0 for every action.  With absorbing != 0,
 * goal rows are self-loops with probability 1.
 *
 * goals[n_goals] (int64, output) receives the goal cells, drawn distinct with
 * stream ST_GOAL of row 0.  The function fills rows of the states [s0, s1);
 * row_ptr is local to the range (starts at 0) and must hold (s1-s0)*5+1
 * entries; pass col == NULL to compute only row_ptr.
 */
static const int GRID_DX[5] = {0, 1, 0, -1, 0};
static const int GRID_DY[5] = {-1, 0, 1, 0, 0};

static int is_goal(int64_t s, const int64_t* goals, int n_goals) {
  for (int i = 0; i < n_goals; ++i)
    if (goals[i] == s) return 1;
  return 0;
}

void synth_grid_goals(int64_t W, int64_t H, int32_t n_goals, uint64_t seed, int64_t* goals) {
  rng_t gg;
  rng_init(&gg, seed, 0, ST_GOAL);
  int64_t n = W * H;
  for (int i = 0; i < n_goals; ++i) {
    for (;;) {
      uint64_t hi = rng_u32(&gg), lo = rng_u32(&gg);
      int64_t c = (int64_t)(((hi << 32) | lo) % (uint64_t)n);
      int dup = 0;
      for (int j = 0; j < i; ++j)
        if (goals[j] == c) dup = 1;
      if (!dup) { goals[i] = c; break; }
    }
  }
}

/* Row entries of grid row (s, a): sorted distinct columns with merged mass. */
static int grid_row(int64_t W, int64_t H, int64_t s, int a, double p_int, double p_oth,
                    int absorbing, int goal, int64_t* cols, double* probs) {
  if (absorbing && goal) {
    cols[0] = s;
    probs[0] = 1.0;
    return 1;
  }
  int64_t x = s % W, y = s / W;
  /* mass per stencil cell: index 0..3 = N,E,S,W neighbour, 4 = self */
  double mass[5];
  for (int d = 0; d < 5; ++d) mass[d] = (d == a) ? p_int : p_oth;
  /* target of each stencil cell, reflecting off-grid moves onto self */
  int64_t tgt[5];
  for (int d = 0; d < 5; ++d) {
    int64_t xx = x + GRID_DX[d], yy = y + GRID_DY[d];
    if (xx < 0 || xx >= W || yy < 0 || yy >= H) tgt[d] = s;
    else tgt[d] = yy * W + xx;
  }
  /* merge duplicates (off-grid moves land on s), then sort by column */
  int cnt = 0;
  for (int d = 0; d < 5; ++d) {
    int found = -1;
    for (int j = 0; j < cnt; ++j)
      if (cols[j] == tgt[d]) found = j;
    if (found >= 0) probs[found] += mass[d];
    else { cols[cnt] = tgt[d]; probs[cnt] = mass[d]; ++cnt; }
  }
  for (int i = 1; i < cnt; ++i) /* insertion sort, at most 5 entries */
    for (int j = i; j > 0 && cols[j - 1] > cols[j]; --j) {
      int64_t tc = cols[j]; cols[j] = cols[j - 1]; cols[j - 1] = tc;
      double tp = probs[j]; probs[j] = probs[j - 1]; probs[j - 1] = tp;
    }
  return cnt;
}

int64_t synth_grid_fill(int64_t W, int64_t H, int64_t s0, int64_t s1, double p_int, double p_oth,
                        const int64_t* goals, int32_t n_goals, int32_t absorbing,
                        int64_t* row_ptr, int32_t* col, void* val, int32_t val_is_f64, void* g,
                        int32_t g_is_f64) {
  const int m = 5;
  int64_t rows = (s1 - s0) * m;
  if (col == NULL) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i) {
      int64_t s = s0 + i / m;
      int a = (int)(i % m);
      int64_t c[5];
      double p[5];
      row_ptr[i + 1] = grid_row(W, H, s, a, p_int, p_oth, absorbing, is_goal(s, goals, n_goals), c, p);
    }
    row_ptr[0] = 0;
    for (int64_t i = 0; i < rows; ++i) row_ptr[i + 1] += row_ptr[i];
    return row_ptr[rows];
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i) {
    int64_t s = s0 + i / m;
    int a = (int)(i % m);
    int64_t c[5];
    double p[5];
    int goal = is_goal(s, goals, n_goals);
    int cnt = grid_row(W, H, s, a, p_int, p_oth, absorbing, goal, c, p);
    int64_t b = row_ptr[i];
    for (int j = 0; j < cnt; ++j) {
      col[b + j] = (int32_t)c[j];
      put_val(val, val_is_f64, b + j, p[j]);
    }
    double cost = goal ? 0.0 : 1.0;
    if (g_is_f64) ((double*)g)[i] = cost;
    else ((float*)g)[i] = (float)cost;
  }
  return row_ptr[rows];
}
