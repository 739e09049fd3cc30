/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU reference for sparse
 * MTTKRP along every mode of an N-mode COO tensor and for CPD-ALS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or helper with the CUDA library; the library never calls it.
 *
 * Every routine is written from the definition it follows, with no blocking,
 * fusion or reordering beyond that definition:
 *
 *   oracle_mttkrp        Sec. II-A6 elementwise computation, generalised to N
 *                        modes as in Algorithm 2 (value times the input-mode
 *                        factor rows, added into row c_d of the output); the
 *                        output is a fresh matrix (Eq. 1 is a product).
 *   oracle_mttkrp_rows   the same definition restricted to chosen output rows.
 *   oracle_mttkrp_omp    the same definition on T threads with thread-private
 *                        outputs added in thread order (only in the OpenMP
 *                        build; a CPU baseline, not a parity reference).
 *   oracle_mode_permutation
 *                        Sec. III-B2: nonzeros ordered by the output-mode
 *                        index; ties broken by the other modes in ascending
 *                        mode order, then by input position (stable).
 *   oracle_partition_equal
 *                        Sec. III-B2: kappa equal-size partitions of the
 *                        ordered nonzeros, offsets floor(z*nnz/kappa).
 *   oracle_partition_balanced
 *                        a design choice of this library (not a rule of the
 *                        paper): Sec. III-B2's ordered nonzeros cut into
 *                        equal-cost pieces, a nonzero costing 1 plus a fixed
 *                        extra for the first nonzero of each output row.
 *   oracle_partition_scheme1
 *                        Sec. III-B1: rows ordered by degree (descending,
 *                        ties by index), dealt cyclically to kappa partitions,
 *                        nonzeros ordered by partition id (then mode order).
 *   oracle_cpd_als       Sec. II-A5 CP-ALS (one MTTKRP per mode, then the
 *                        factor update and column normalisation), with the
 *                        standard normal-equation update of Kolda & Bader:
 *                        Y_d = M_d V^{-1}, V = Hadamard of the other Grams,
 *                        solved through a Cholesky factorisation, lambda = the
 *                        column 2-norms, and the fit 1 - |X - Xhat| / |X|.
 *
 * Build: gcc -O2 -shared -fPIC -o liboracle.so oracle.c -lm
 *        (and with -fopenmp into liboracle_omp.so for the all-core baseline)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_INDEX 2
#define ORACLE_ERR_NOMEM 3
#define ORACLE_ERR_NUMERIC 5

/* ------------------------------------------------------------------------ */
/* MTTKRP by the elementwise definition                                      */
/* ------------------------------------------------------------------------ */

/* out[i*R + r] = sum over nonzeros k with idx[mode][k] == i of
 *                vals[k] * prod_{w != mode} factors[w][idx[w][k]*R + r].
 * factors[w] is I_w x R row-major (factors[mode] is not read).
 * out is I_mode x R row-major and is overwritten. */
int oracle_mttkrp(int nmodes, const int64_t *dims, int64_t nnz,
                  const int32_t *const *idx, const double *vals, int rank,
                  const double *const *factors, int mode, double *out) {
  if (nmodes < 1 || mode < 0 || mode >= nmodes || rank < 1 || nnz < 0)
    return ORACLE_ERR_ARG;
  memset(out, 0, sizeof(double) * (size_t)dims[mode] * (size_t)rank);
  for (int64_t k = 0; k < nnz; ++k) {
    for (int w = 0; w < nmodes; ++w)
      if (idx[w][k] < 0 || idx[w][k] >= dims[w]) return ORACLE_ERR_INDEX;
    int64_t i = idx[mode][k];
    for (int r = 0; r < rank; ++r) {
      double t = vals[k];
      for (int w = 0; w < nmodes; ++w) {
        if (w == mode) continue;
        t *= factors[w][(int64_t)idx[w][k] * rank + r];
      }
      out[i * rank + r] += t;
    }
  }
  return ORACLE_OK;
}

#ifdef _OPENMP
#include <omp.h>

/* The same definition evaluated by T threads, for the all-core CPU baseline
 * (built only into the OpenMP copy of this file, liboracle_omp.so): thread t
 * takes the nonzeros [t*nnz/T, (t+1)*nnz/T) in input order and adds their
 * terms into its own zeroed I_mode x R output; the T outputs are then added
 * element by element in thread order.  Only the grouping of the FP64 sum
 * differs from oracle_mttkrp.  nthreads <= 0 uses the OpenMP default;
 * *threads_used receives the number of threads that ran. */
int oracle_mttkrp_omp(int nmodes, const int64_t *dims, int64_t nnz,
                      const int32_t *const *idx, const double *vals, int rank,
                      const double *const *factors, int mode, int nthreads,
                      double *out, int *threads_used) {
  if (nmodes < 1 || mode < 0 || mode >= nmodes || rank < 1 || nnz < 0)
    return ORACLE_ERR_ARG;
  const size_t cells = (size_t)dims[mode] * (size_t)rank;
  int T = nthreads > 0 ? nthreads : omp_get_max_threads();
  double *priv = (double *)calloc((size_t)T * cells, sizeof(double));
  if (!priv) return ORACLE_ERR_NOMEM;
  int bad = 0, ran = 1;
#pragma omp parallel num_threads(T) reduction(| : bad)
  {
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
    if (t == 0) ran = nt;
    double *o = priv + (size_t)t * cells;
    for (int64_t k = nnz * t / nt; k < nnz * (t + 1) / nt; ++k) {
      int ok = 1;
      for (int w = 0; w < nmodes; ++w)
        if (idx[w][k] < 0 || idx[w][k] >= dims[w]) ok = 0;
      if (!ok) {
        bad = 1;
        continue;
      }
      int64_t i = idx[mode][k];
      for (int r = 0; r < rank; ++r) {
        double v = vals[k];
        for (int w = 0; w < nmodes; ++w) {
          if (w == mode) continue;
          v *= factors[w][(int64_t)idx[w][k] * rank + r];
        }
        o[i * rank + r] += v;
      }
    }
  }
  if (bad) {
    free(priv);
    return ORACLE_ERR_INDEX;
  }
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t e = 0; e < (int64_t)cells; ++e) {
    double acc = 0.0;
    for (int t = 0; t < ran; ++t) acc += priv[(size_t)t * cells + (size_t)e];
    out[e] = acc;
  }
  free(priv);
  if (threads_used) *threads_used = ran;
  return ORACLE_OK;
}
#endif

/* The same definition for a chosen set of output rows only.
 * rows[j] (distinct, in [0, I_mode)) -> out[j*R + r]. */
int oracle_mttkrp_rows(int nmodes, const int64_t *dims, int64_t nnz,
                       const int32_t *const *idx, const double *vals, int rank,
                       const double *const *factors, int mode, int64_t nrows,
                       const int32_t *rows, double *out) {
  if (nmodes < 1 || mode < 0 || mode >= nmodes || rank < 1 || nnz < 0 ||
      nrows < 0)
    return ORACLE_ERR_ARG;
  int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)dims[mode]);
  if (!slot) return ORACLE_ERR_NOMEM;
  for (int64_t i = 0; i < dims[mode]; ++i) slot[i] = -1;
  for (int64_t j = 0; j < nrows; ++j) {
    if (rows[j] < 0 || rows[j] >= dims[mode]) {
      free(slot);
      return ORACLE_ERR_ARG;
    }
    slot[rows[j]] = j;
  }
  memset(out, 0, sizeof(double) * (size_t)nrows * (size_t)rank);
  for (int64_t k = 0; k < nnz; ++k) {
    int64_t i = idx[mode][k];
    if (i < 0 || i >= dims[mode]) {
      free(slot);
      return ORACLE_ERR_INDEX;
    }
    int64_t j = slot[i];
    if (j < 0) continue;
    for (int r = 0; r < rank; ++r) {
      double t = vals[k];
      for (int w = 0; w < nmodes; ++w) {
        if (w == mode) continue;
        t *= factors[w][(int64_t)idx[w][k] * rank + r];
      }
      out[j * rank + r] += t;
    }
  }
  free(slot);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Mode-specific ordering (the permutation of one tensor copy)               */
/* ------------------------------------------------------------------------ */

/* Key comparison for the mode-`mode` copy: first c_mode, then every other
 * mode in ascending mode order, then the input position (so the order is a
 * total order and the sort is stable). Returns <0, 0, >0. */
static int key_cmp(int nmodes, const int32_t *const *idx, int mode, int64_t a,
                   int64_t b) {
  if (idx[mode][a] != idx[mode][b]) return idx[mode][a] < idx[mode][b] ? -1 : 1;
  for (int w = 0; w < nmodes; ++w) {
    if (w == mode) continue;
    if (idx[w][a] != idx[w][b]) return idx[w][a] < idx[w][b] ? -1 : 1;
  }
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* Plain top-down merge sort of positions by key_cmp. */
static void merge_sort(int nmodes, const int32_t *const *idx, int mode,
                       int64_t *p, int64_t *tmp, int64_t n) {
  if (n < 2) return;
  int64_t h = n / 2;
  merge_sort(nmodes, idx, mode, p, tmp, h);
  merge_sort(nmodes, idx, mode, p + h, tmp, n - h);
  int64_t i = 0, j = h, o = 0;
  while (i < h && j < n) {
    if (key_cmp(nmodes, idx, mode, p[i], p[j]) <= 0)
      tmp[o++] = p[i++];
    else
      tmp[o++] = p[j++];
  }
  while (i < h) tmp[o++] = p[i++];
  while (j < n) tmp[o++] = p[j++];
  memcpy(p, tmp, sizeof(int64_t) * (size_t)n);
}

/* perm[k] = input position of the k-th nonzero of the mode-`mode` copy. */
int oracle_mode_permutation(int nmodes, int64_t nnz, const int32_t *const *idx,
                            int mode, int64_t *perm) {
  if (nmodes < 1 || mode < 0 || mode >= nmodes || nnz < 0) return ORACLE_ERR_ARG;
  for (int64_t k = 0; k < nnz; ++k) perm[k] = k;
  int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  if (!tmp) return ORACLE_ERR_NOMEM;
  merge_sort(nmodes, idx, mode, perm, tmp, nnz);
  free(tmp);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Partitioning                                                              */
/* ------------------------------------------------------------------------ */

/* Scheme 2 (equal distribution of nonzeros): off[z] = floor(z*nnz/kappa),
 * z = 0..kappa, so partition sizes differ by at most one. */
int oracle_partition_equal(int64_t nnz, int kappa, int64_t *off) {
  if (kappa < 1 || nnz < 0) return ORACLE_ERR_ARG;
  for (int z = 0; z <= kappa; ++z) {
    /* exact floor(z*nnz/kappa) without overflow for nnz < 2^62/kappa */
    off[z] = (int64_t)(((__int128)z * nnz) / kappa);
  }
  return ORACLE_OK;
}

/* Cost-balanced work units over a copy: rows[k] is the output index of the
 * k-th nonzero in copy order.  A nonzero costs 1, plus row_cost if it starts
 * its row (k == 0 or rows[k] != rows[k-1]).  With C(k) the cost of positions
 * before k and P units, unit j starts at the smallest k with
 * C(k) * P >= j * C(nnz).  off has P + 1 entries. */
int oracle_partition_balanced(int64_t nnz, const int32_t *rows, int64_t parts,
                              int64_t row_cost, int64_t *off) {
  if (parts < 1 || nnz < 0 || row_cost < 0) return ORACLE_ERR_ARG;
  int64_t *C = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz + 1));
  if (!C) return ORACLE_ERR_NOMEM;
  C[0] = 0;
  for (int64_t k = 0; k < nnz; ++k) {
    int start = (k == 0) || rows[k] != rows[k - 1];
    C[k + 1] = C[k] + 1 + (start ? row_cost : 0);
  }
  int64_t k = 0;
  for (int64_t j = 0; j <= parts; ++j) {
    while (C[k] * parts < j * C[nnz]) ++k;
    off[j] = k;
  }
  free(C);
  return ORACLE_OK;
}

static const int64_t *g_deg; /* qsort context for the degree ordering */

static int row_order_cmp(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  if (g_deg[a] != g_deg[b]) return g_deg[a] > g_deg[b] ? -1 : 1; /* degree desc */
  return a < b ? -1 : (a > b ? 1 : 0);                             /* index asc */
}

/* Scheme 1 (equal distribution of output indices):
 *   degree(i) = number of nonzeros with c_mode == i;
 *   rows with degree >= 1 ordered by (degree descending, index ascending);
 *   the t-th row in that order goes to partition t mod kappa;
 *   nonzeros ordered by (partition id, then the mode-`mode` copy order).
 * Outputs perm[nnz] (input positions in that order), off[kappa+1] and
 * row_part[I_mode] (partition of each row, -1 for empty rows). */
int oracle_partition_scheme1(int nmodes, const int64_t *dims, int64_t nnz,
                             const int32_t *const *idx, int mode, int kappa,
                             int64_t *perm, int64_t *off, int32_t *row_part) {
  if (nmodes < 1 || mode < 0 || mode >= nmodes || kappa < 1 || nnz < 0)
    return ORACLE_ERR_ARG;
  int64_t I = dims[mode];
  int64_t *deg = (int64_t *)calloc((size_t)(I > 0 ? I : 1), sizeof(int64_t));
  int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)(I > 0 ? I : 1));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t *cnt = (int64_t *)calloc((size_t)kappa + 1, sizeof(int64_t));
  if (!deg || !rows || !order || !cnt) {
    free(deg); free(rows); free(order); free(cnt);
    return ORACLE_ERR_NOMEM;
  }
  for (int64_t k = 0; k < nnz; ++k) deg[idx[mode][k]]++;
  int64_t nr = 0;
  for (int64_t i = 0; i < I; ++i) {
    row_part[i] = -1;
    if (deg[i] > 0) rows[nr++] = i;
  }
  g_deg = deg;
  qsort(rows, (size_t)nr, sizeof(int64_t), row_order_cmp);
  for (int64_t t = 0; t < nr; ++t) row_part[rows[t]] = (int32_t)(t % kappa);
  /* nonzeros in mode order, then a stable counting distribution by partition */
  int rc = oracle_mode_permutation(nmodes, nnz, idx, mode, order);
  if (rc == ORACLE_OK) {
    for (int64_t k = 0; k < nnz; ++k) cnt[row_part[idx[mode][order[k]]] + 1]++;
    for (int z = 0; z < kappa; ++z) cnt[z + 1] += cnt[z];
    for (int z = 0; z <= kappa; ++z) off[z] = cnt[z];
    for (int64_t k = 0; k < nnz; ++k) {
      int32_t z = row_part[idx[mode][order[k]]];
      perm[cnt[z]++] = order[k];
    }
  }
  free(deg); free(rows); free(order); free(cnt);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* CPD-ALS                                                                   */
/* ------------------------------------------------------------------------ */

/* Round an FP64 value to the storage format of the factor matrices:
 * prec 0 = keep FP64, 1 = FP32 (round to nearest even), 2 = FP32 then
 * bfloat16 (round to nearest even on the FP32 bit pattern). */
static double store_round(double x, int prec) {
  if (prec == 0) return x;
  float f = (float)x;
  if (prec == 1) return (double)f;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) { /* inf / nan: truncate, keep nan */
    if (u & 0x007fffffu) u |= 0x00400000u;
    u &= 0xffff0000u;
  } else {
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
  }
  memcpy(&f, &u, 4);
  return (double)f;
}

double oracle_store_round(double x, int prec) { return store_round(x, prec); }

void oracle_store_round_array(double *x, int64_t n, int prec) {
  for (int64_t i = 0; i < n; ++i) x[i] = store_round(x[i], prec);
}

/* G = Y^T Y for Y (I x R) row-major. */
static void gram(const double *Y, int64_t I, int R, double *G) {
  for (int r = 0; r < R; ++r)
    for (int s = 0; s < R; ++s) {
      double acc = 0.0;
      for (int64_t i = 0; i < I; ++i) acc += Y[i * R + r] * Y[i * R + s];
      G[r * R + s] = acc;
    }
}

/* In-place Cholesky V = L L^T (lower triangle of V overwritten by L).
 * Returns ORACLE_ERR_NUMERIC if V is not numerically positive definite. */
static int cholesky(double *V, int R) {
  for (int j = 0; j < R; ++j) {
    double d = V[j * R + j];
    for (int k = 0; k < j; ++k) d -= V[j * R + k] * V[j * R + k];
    if (!(d > 0.0) || !isfinite(d)) return ORACLE_ERR_NUMERIC;
    double ljj = sqrt(d);
    V[j * R + j] = ljj;
    for (int i = j + 1; i < R; ++i) {
      double s = V[i * R + j];
      for (int k = 0; k < j; ++k) s -= V[i * R + k] * V[j * R + k];
      V[i * R + j] = s / ljj;
    }
  }
  return ORACLE_OK;
}

/* Solve (L L^T) z = m for one vector (forward then back substitution). */
static void chol_solve(const double *L, int R, const double *m, double *z) {
  for (int i = 0; i < R; ++i) {
    double s = m[i];
    for (int k = 0; k < i; ++k) s -= L[i * R + k] * z[k];
    z[i] = s / L[i * R + i];
  }
  for (int i = R - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < R; ++k) s -= L[k * R + i] * z[k];
    z[i] = s / L[i * R + i];
  }
}

/* One CP-ALS update of factor `mode` given the MTTKRP result M (I x R):
 *   V = Hadamard product of the Grams of every other factor,
 *   Z = M V^{-1} (row by row, through the Cholesky factor of V),
 *   lambda_r = |Z(:, r)|_2, Y_mode(:, r) = Z(:, r) / lambda_r (lambda_r > 0),
 *   Y_mode rounded to the storage format.
 * grams[w] holds Y_w^T Y_w of the stored factors and is refreshed for `mode`. */
static int als_update_mode(int nmodes, const int64_t *dims, int R,
                           double *const *factors, double *const *grams,
                           int mode, const double *M, int prec,
                           double *lambda) {
  int64_t I = dims[mode];
  double *V = (double *)malloc(sizeof(double) * (size_t)R * R);
  double *z = (double *)malloc(sizeof(double) * (size_t)R);
  double *Z = (double *)malloc(sizeof(double) * (size_t)(I > 0 ? I : 1) * R);
  if (!V || !z || !Z) {
    free(V); free(z); free(Z);
    return ORACLE_ERR_NOMEM;
  }
  for (int e = 0; e < R * R; ++e) V[e] = 1.0;
  for (int w = 0; w < nmodes; ++w) {
    if (w == mode) continue;
    for (int e = 0; e < R * R; ++e) V[e] *= grams[w][e];
  }
  int rc = cholesky(V, R);
  if (rc != ORACLE_OK) {
    free(V); free(z); free(Z);
    return rc;
  }
  for (int64_t i = 0; i < I; ++i) chol_solve(V, R, M + i * R, Z + i * R);
  for (int r = 0; r < R; ++r) {
    double s = 0.0;
    for (int64_t i = 0; i < I; ++i) s += Z[i * R + r] * Z[i * R + r];
    lambda[r] = sqrt(s);
  }
  double *Y = factors[mode];
  for (int64_t i = 0; i < I; ++i)
    for (int r = 0; r < R; ++r) {
      double y = lambda[r] > 0.0 ? Z[i * R + r] / lambda[r] : Z[i * R + r];
      Y[i * R + r] = store_round(y, prec);
    }
  gram(Y, I, R, grams[mode]);
  free(V); free(z); free(Z);
  return ORACLE_OK;
}

/* fit = 1 - sqrt(max(0, |X|^2 + |Xhat|^2 - 2 <X, Xhat>)) / |X| with
 *   |Xhat|^2   = lambda^T (Hadamard of all Grams) lambda,
 *   <X, Xhat>  = sum_r lambda_r sum_i M(i, r) Y_last(i, r)
 * where M is the MTTKRP of the last mode (computed with the other factors
 * already updated) and Y_last the stored, normalised last factor. */
static double fit_value(int nmodes, const int64_t *dims, int R,
                        double *const *factors, double *const *grams,
                        const double *M, const double *lambda, double normX2) {
  int last = nmodes - 1;
  double xhat2 = 0.0;
  for (int r = 0; r < R; ++r)
    for (int s = 0; s < R; ++s) {
      double h = 1.0;
      for (int w = 0; w < nmodes; ++w) h *= grams[w][r * R + s];
      xhat2 += lambda[r] * lambda[s] * h;
    }
  double inner = 0.0;
  for (int r = 0; r < R; ++r) {
    double s = 0.0;
    for (int64_t i = 0; i < dims[last]; ++i)
      s += M[i * R + r] * factors[last][i * R + r];
    inner += lambda[r] * s;
  }
  double res2 = normX2 + xhat2 - 2.0 * inner;
  if (res2 < 0.0) res2 = 0.0;
  return 1.0 - sqrt(res2) / sqrt(normX2);
}

/* |X|^2 = sum of squared values (duplicates at one coordinate are summed
 * first, since the tensor holds their sum). Positions with equal coordinates
 * are found through the mode-0 ordering. */
int oracle_norm2(int nmodes, int64_t nnz, const int32_t *const *idx,
                 const double *vals, double *out) {
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  if (!perm) return ORACLE_ERR_NOMEM;
  int rc = oracle_mode_permutation(nmodes, nnz, idx, 0, perm);
  if (rc != ORACLE_OK) {
    free(perm);
    return rc;
  }
  double total = 0.0, cell = 0.0;
  for (int64_t k = 0; k < nnz; ++k) {
    int same = 0;
    if (k > 0) {
      same = 1;
      for (int w = 0; w < nmodes; ++w)
        if (idx[w][perm[k]] != idx[w][perm[k - 1]]) { same = 0; break; }
    }
    if (same) {
      cell += vals[perm[k]];
    } else {
      total += cell * cell;
      cell = vals[perm[k]];
    }
  }
  total += cell * cell;
  free(perm);
  *out = total;
  return ORACLE_OK;
}

/* One factor update on its own (the step CP-ALS repeats per mode): Grams of
 * the current factors, then als_update_mode with the given MTTKRP M. */
int oracle_als_update(int nmodes, const int64_t *dims, int R,
                      double *const *factors, int mode, const double *M,
                      int prec, double *lambda) {
  if (nmodes < 2 || R < 1 || mode < 0 || mode >= nmodes) return ORACLE_ERR_ARG;
  double **grams = (double **)calloc((size_t)nmodes, sizeof(double *));
  if (!grams) return ORACLE_ERR_NOMEM;
  int rc = ORACLE_OK;
  for (int w = 0; w < nmodes && rc == ORACLE_OK; ++w) {
    grams[w] = (double *)malloc(sizeof(double) * (size_t)R * R);
    if (!grams[w]) rc = ORACLE_ERR_NOMEM;
    else gram(factors[w], dims[w], R, grams[w]);
  }
  if (rc == ORACLE_OK)
    rc = als_update_mode(nmodes, dims, R, factors, grams, mode, M, prec, lambda);
  for (int w = 0; w < nmodes; ++w) free(grams[w]);
  free(grams);
  return rc;
}

/* CP-ALS: `sweeps` sweeps over the modes 0..N-1 in order (Gauss-Seidel: each
 * MTTKRP uses the factors already updated in this sweep). factors[w] (I_w x R,
 * FP64, already in storage precision) are updated in place; lambda[R] receives
 * the weights of the last updated mode; fit[s] the fit after sweep s.
 * prec: storage rounding of the factors after each update (0 FP64, 1 FP32,
 * 2 BF16). */
int oracle_cpd_als(int nmodes, const int64_t *dims, int64_t nnz,
                   const int32_t *const *idx, const double *vals, int R,
                   double *const *factors, int sweeps, int prec, double *lambda,
                   double *fit) {
  if (nmodes < 2 || R < 1 || sweeps < 0) return ORACLE_ERR_ARG;
  int64_t Imax = 1;
  for (int w = 0; w < nmodes; ++w) Imax = dims[w] > Imax ? dims[w] : Imax;
  double *M = (double *)malloc(sizeof(double) * (size_t)Imax * R);
  double **grams = (double **)calloc((size_t)nmodes, sizeof(double *));
  if (!M || !grams) {
    free(M); free(grams);
    return ORACLE_ERR_NOMEM;
  }
  int rc = ORACLE_OK;
  for (int w = 0; w < nmodes && rc == ORACLE_OK; ++w) {
    grams[w] = (double *)malloc(sizeof(double) * (size_t)R * R);
    if (!grams[w]) rc = ORACLE_ERR_NOMEM;
    else gram(factors[w], dims[w], R, grams[w]);
  }
  double normX2 = 0.0;
  if (rc == ORACLE_OK) rc = oracle_norm2(nmodes, nnz, idx, vals, &normX2);
  for (int s = 0; s < sweeps && rc == ORACLE_OK; ++s) {
    for (int d = 0; d < nmodes && rc == ORACLE_OK; ++d) {
      rc = oracle_mttkrp(nmodes, dims, nnz, idx, vals, R,
                         (const double *const *)factors, d, M);
      if (rc == ORACLE_OK)
        rc = als_update_mode(nmodes, dims, R, factors, grams, d, M, prec, lambda);
    }
    if (rc == ORACLE_OK)
      fit[s] = normX2 > 0.0
                   ? fit_value(nmodes, dims, R, factors, grams, M, lambda, normX2)
                   : 1.0;
  }
  for (int w = 0; w < nmodes; ++w) free(grams[w]);
  free(grams);
  free(M);
  return rc;
}
