/*
 * Oracle (test infrastructure only; the product path never loads this file).
 *
 * K-means++ on the feature columns of X (Section 3.4, "K-means++"): seeding
 * by squared-distance weighting, then Lloyd assignment/update steps until no
 * assignment changes.  Euclidean distance between features, as in Section 4
 * (all experiments use the Euclidean distance).
 *
 * Binary X: every quantity is an integer, so the whole clustering is computed
 * exactly:
 *   D2(i, c)      = n_i + n_c - 2 |x_i AND x_c|          (seeding distances)
 *   score(i, S)   = ||x_i - c_S/n_S||^2 - ||x_i||^2
 *                 = (Q_S - 2 n_S D_iS) / n_S^2,
 *   with c_S the integer sum of the columns in S, Q_S = ||c_S||^2 and
 *   D_iS = x_i . c_S.  Scores are compared by exact 128-bit cross
 *   multiplication; ties go to the smallest cluster index; empty clusters are
 *   skipped.
 * Dense X: the same steps in FP64, no fused multiply-add (compiled with
 *   -ffp-contract=off). The paper fixes no summation order; every sum over
 *   the N rows is taken in blocks of ORACLE_ROW_BLOCK consecutive rows: each
 *   block summed in ascending row order, then the block sums in ascending
 *   block order. Centroids sum their member columns in ascending feature
 *   order.
 *
 * Random draws: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) seeded with
 * `seed`; draw t is output t (counting from 0), u_t = (x_t >> 11) * 2^-53.
 *   first centre:  floor(u_0 * F)
 *   centre t >= 1: first i with cumsum(D2)_i > floor(u_t * sum(D2)); if every
 *                  D2 is zero, the lowest index not yet chosen.
 * Plain loops: slow and obviously correct on purpose. The Lloyd assignment
 * step, where each feature's argmin is independent of the others and computed
 * in exact integers, may run its features on several OpenMP threads (one
 * feature per thread at a time, each with its own accumulator), which cannot
 * change any result; oracle_set_threads(n) sets the count (1 = one thread).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* Threads of the Lloyd assignment step (1 when built without OpenMP). */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n < 1) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return n;
#else
  (void)n;
  return 1;
#endif
}

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t seed, int64_t t) {
  return mix64(seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ULL);
}

double oracle_u53(uint64_t seed, int64_t t) {
  return (double)(oracle_splitmix64(seed, t) >> 11) * 0x1.0p-53;
}

/* ov[j] = |x_j AND x_c| for every feature j, computed through the rows of x_c. */
static void overlaps(const int64_t *row_ptr, const int32_t *col_idx,
                     const int64_t *col_ptr, const int32_t *row_idx,
                     int64_t c, int64_t *ov) {
  for (int64_t p = col_ptr[c]; p < col_ptr[c + 1]; ++p) {
    int64_t r = row_idx[p];
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) ov[col_idx[e]] += 1;
  }
}

static int64_t pick(const uint64_t seed, int64_t t, int64_t F, const int64_t *d2,
                    const unsigned char *chosen) {
  int64_t total = 0;
  for (int64_t i = 0; i < F; ++i) total += d2[i];
  if (total == 0) {
    for (int64_t i = 0; i < F; ++i)
      if (!chosen[i]) return i;
    return -1;
  }
  int64_t thr = (int64_t)floor(oracle_u53(seed, t) * (double)total);
  if (thr >= total) thr = total - 1;
  int64_t cum = 0;
  for (int64_t i = 0; i < F; ++i) {
    cum += d2[i];
    if (cum > thr) return i;
  }
  return -1;
}

/* K-means++ seeding on binary X. centers[k] receives feature ids. Returns 0 or -1. */
int oracle_kmeanspp_binary(int64_t N, int64_t F, const int64_t *row_ptr,
                           const int32_t *col_idx, const int64_t *col_ptr,
                           const int32_t *row_idx, int32_t k, uint64_t seed,
                           int32_t *centers) {
  (void)N;
  if (k < 1 || k > F) return -1;
  int64_t *d2 = (int64_t *)malloc(sizeof(int64_t) * F);
  int64_t *ov = (int64_t *)calloc(F, sizeof(int64_t));
  unsigned char *chosen = (unsigned char *)calloc(F, 1);
  int64_t c = (int64_t)floor(oracle_u53(seed, 0) * (double)F);
  if (c >= F) c = F - 1;
  for (int32_t t = 0; t < k; ++t) {
    if (t > 0) c = pick(seed, t, F, d2, chosen);
    if (c < 0) { free(d2); free(ov); free(chosen); return -1; }
    centers[t] = (int32_t)c;
    chosen[c] = 1;
    memset(ov, 0, sizeof(int64_t) * F);
    overlaps(row_ptr, col_idx, col_ptr, row_idx, c, ov);
    int64_t nc = col_ptr[c + 1] - col_ptr[c];
    for (int64_t i = 0; i < F; ++i) {
      int64_t ni = col_ptr[i + 1] - col_ptr[i];
      int64_t dist = ni + nc - 2 * ov[i];
      if (t == 0 || dist < d2[i]) d2[i] = dist;
    }
  }
  free(d2); free(ov); free(chosen);
  return 0;
}

/* Lloyd iterations on binary X from the given centres (feature ids, distinct).
 * labels[F] receives cluster indices in [0, k); *iters the number of
 * assignment steps taken (the last one changed nothing unless max_iter hit).
 * Returns 0, or -1 on invalid centres. */
int oracle_lloyd_binary(int64_t N, int64_t F, const int64_t *row_ptr,
                        const int32_t *col_idx, const int64_t *col_ptr,
                        const int32_t *row_idx, int32_t k, const int32_t *centers,
                        int32_t max_iter, int32_t *labels, int32_t *iters) {
  if (k < 1 || k > F) return -1;
  for (int64_t i = 0; i < F; ++i) labels[i] = -1;
  for (int32_t s = 0; s < k; ++s) {
    if (centers[s] < 0 || centers[s] >= F || labels[centers[s]] >= 0) return -1;
    labels[centers[s]] = s;
  }
  int64_t *n = (int64_t *)malloc(sizeof(int64_t) * k);
  int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * k);
  int64_t *acc = (int64_t *)malloc(sizeof(int64_t) * k);
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * F);
  int32_t it = 0;
  while (it < max_iter) {
    ++it;
    /* cluster sizes n_S and Q_S = ||c_S||^2 = sum_r C[r,S]^2 */
    memset(n, 0, sizeof(int64_t) * k);
    memset(Q, 0, sizeof(int64_t) * k);
    for (int64_t i = 0; i < F; ++i)
      if (labels[i] >= 0) n[labels[i]] += 1;
    memset(acc, 0, sizeof(int64_t) * k);
    for (int64_t r = 0; r < N; ++r) {
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        int32_t l = labels[col_idx[e]];
        if (l >= 0) acc[l] += 1;
      }
      for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        int32_t l = labels[col_idx[e]];
        if (l >= 0 && acc[l] != 0) { Q[l] += acc[l] * acc[l]; acc[l] = 0; }
      }
    }
    /* assignment: argmin_S (Q_S - 2 n_S D_iS) / n_S^2, feature by feature */
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
      int64_t *dacc = (int64_t *)malloc(sizeof(int64_t) * k);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t i = 0; i < F; ++i) {
        memset(dacc, 0, sizeof(int64_t) * k);
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) {
          int64_t r = row_idx[p];
          for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            int32_t l = labels[col_idx[e]];
            if (l >= 0) dacc[l] += 1;
          }
        }
        int32_t best = -1;
        int64_t best_a = 0, best_n = 0;
        for (int32_t s = 0; s < k; ++s) {
          if (n[s] == 0) continue;
          int64_t a = Q[s] - 2 * n[s] * dacc[s];
          if (best < 0 ||
              (i128)a * (i128)(best_n * best_n) < (i128)best_a * (i128)(n[s] * n[s])) {
            best = s; best_a = a; best_n = n[s];
          }
        }
        next[i] = best;
      }
      free(dacc);
    }
    int64_t changes = 0;
    for (int64_t i = 0; i < F; ++i) {
      if (next[i] != labels[i]) ++changes;
      labels[i] = next[i];
    }
    if (changes == 0) break;
  }
  *iters = it;
  free(n); free(Q); free(acc); free(next);
  return 0;
}

/* ---------------- dense X (N x F, row-major float32 values) -------------- */

#define ORACLE_ROW_BLOCK 64

/* Squared Euclidean distance between features i and j (blocked row order). */
static double dense_d2(int64_t N, int64_t F, const float *X, int64_t i, int64_t j) {
  double total = 0.0;
  for (int64_t b0 = 0; b0 < N; b0 += ORACLE_ROW_BLOCK) {
    const int64_t b1 = b0 + ORACLE_ROW_BLOCK < N ? b0 + ORACLE_ROW_BLOCK : N;
    double s = 0.0;
    for (int64_t r = b0; r < b1; ++r) {
      double t = (double)X[r * F + i] - (double)X[r * F + j];
      s = s + t * t;
    }
    total = total + s;
  }
  return total;
}

int oracle_kmeanspp_dense(int64_t N, int64_t F, const float *X, int32_t k,
                          uint64_t seed, int32_t *centers) {
  if (k < 1 || k > F) return -1;
  double *d2 = (double *)malloc(sizeof(double) * F);
  unsigned char *chosen = (unsigned char *)calloc(F, 1);
  int64_t c = (int64_t)floor(oracle_u53(seed, 0) * (double)F);
  if (c >= F) c = F - 1;
  for (int32_t t = 0; t < k; ++t) {
    if (t > 0) {
      double total = 0.0;
      for (int64_t i = 0; i < F; ++i) total = total + d2[i];
      c = -1;
      if (total == 0.0) {
        for (int64_t i = 0; i < F; ++i) if (!chosen[i]) { c = i; break; }
      } else {
        double thr = oracle_u53(seed, t) * total;
        double cum = 0.0;
        for (int64_t i = 0; i < F; ++i) {
          cum = cum + d2[i];
          if (cum > thr && !chosen[i]) { c = i; break; }
        }
        if (c < 0) for (int64_t i = F - 1; i >= 0; --i) if (!chosen[i] && d2[i] > 0.0) { c = i; break; }
      }
      if (c < 0) { free(d2); free(chosen); return -1; }
    }
    centers[t] = (int32_t)c;
    chosen[c] = 1;
    for (int64_t i = 0; i < F; ++i) {
      double dist = (i == c) ? 0.0 : dense_d2(N, F, X, i, c);
      if (t == 0 || dist < d2[i]) d2[i] = dist;
    }
  }
  free(d2); free(chosen);
  return 0;
}

/* Dense Lloyd: centroid mu_S = (sum over members, ascending feature index) / n_S,
 * score(i, S) = ||mu_S||^2 - 2 x_i . mu_S (the common ||x_i||^2 dropped),
 * each sum over rows in the blocked order above. */
int oracle_lloyd_dense(int64_t N, int64_t F, const float *X, int32_t k,
                       const int32_t *centers, int32_t max_iter, int32_t *labels,
                       int32_t *iters) {
  if (k < 1 || k > F) return -1;
  for (int64_t i = 0; i < F; ++i) labels[i] = -1;
  for (int32_t s = 0; s < k; ++s) {
    if (centers[s] < 0 || centers[s] >= F || labels[centers[s]] >= 0) return -1;
    labels[centers[s]] = s;
  }
  int64_t *n = (int64_t *)malloc(sizeof(int64_t) * k);
  double *mu = (double *)malloc(sizeof(double) * k * N); /* k x N */
  double *mm = (double *)malloc(sizeof(double) * k);
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * F);
  int32_t it = 0;
  while (it < max_iter) {
    ++it;
    memset(n, 0, sizeof(int64_t) * k);
    memset(mu, 0, sizeof(double) * k * N);
    for (int64_t i = 0; i < F; ++i) {
      int32_t l = labels[i];
      if (l < 0) continue;
      n[l] += 1;
      for (int64_t r = 0; r < N; ++r) mu[l * N + r] = mu[l * N + r] + (double)X[r * F + i];
    }
    for (int32_t s = 0; s < k; ++s) {
      double q = 0.0;
      if (n[s] > 0)
        for (int64_t b0 = 0; b0 < N; b0 += ORACLE_ROW_BLOCK) {
          const int64_t b1 = b0 + ORACLE_ROW_BLOCK < N ? b0 + ORACLE_ROW_BLOCK : N;
          double part = 0.0;
          for (int64_t r = b0; r < b1; ++r) {
            mu[s * N + r] = mu[s * N + r] / (double)n[s];
            part = part + mu[s * N + r] * mu[s * N + r];
          }
          q = q + part;
        }
      mm[s] = q;
    }
    for (int64_t i = 0; i < F; ++i) {
      int32_t best = -1;
      double best_v = 0.0;
      for (int32_t s = 0; s < k; ++s) {
        if (n[s] == 0) continue;
        double dot = 0.0;
        for (int64_t b0 = 0; b0 < N; b0 += ORACLE_ROW_BLOCK) {
          const int64_t b1 = b0 + ORACLE_ROW_BLOCK < N ? b0 + ORACLE_ROW_BLOCK : N;
          double part = 0.0;
          for (int64_t r = b0; r < b1; ++r) part = part + (double)X[r * F + i] * mu[s * N + r];
          dot = dot + part;
        }
        double v = mm[s] - 2.0 * dot;
        if (best < 0 || v < best_v) { best = s; best_v = v; }
      }
      next[i] = best;
    }
    int64_t changes = 0;
    for (int64_t i = 0; i < F; ++i) {
      if (next[i] != labels[i]) ++changes;
      labels[i] = next[i];
    }
    if (changes == 0) break;
  }
  *iters = it;
  free(n); free(mu); free(mm); free(next);
  return 0;
}
