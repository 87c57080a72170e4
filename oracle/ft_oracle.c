/*
 * Plain FP64 CPU oracle of the FastTuckerPlus stochastic epoch
 * (arXiv 2404.10087, "cuFastTuckerPlus").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library and never calls it.
 *
 * Everything is written to be checked against the paper by eye: FP64
 * throughout, one nonzero at a time, every product taken exactly as the
 * equations define it (no blocking, fusion or reordering beyond them).
 *
 * Model (Sec. 2.3, Eq. "fasttucker"):
 *     c^(n)_r  = sum_j a^(n)_{i_n, j} B^(n)_{j, r}          (c^(n) = a^(n) B^(n))
 *     xhat     = sum_r prod_n c^(n)_r
 * Leave-one-out product (definition after Eq. "Gradient_core_tensor_cp"):
 *     d^(n)_r  = prod_{k != n} c^(k)_r
 * Factor gradient of one nonzero (Eq. "Gradient_low_rank_cp"):
 *     g^(n)    = -(x - xhat) d^(n) B^(n)^T + lambda_A a^(n)
 * FastTuckerPlus factor update, all N rows from one snapshot
 * (Eq. "Update_FastTuckerPlus_factor", Algorithm 3 / Algorithm 4):
 *     a^(n) <- a^(n) - gamma_A * g^(n)        for every n simultaneously
 * Core gradient of one nonzero (Eq. "Gradient_core_tensor_cp"):
 *     G^(n)    = -(x - xhat) a^(n)^T d^(n)      (J_n x R)
 * Core step, accumulated over the whole training set (Algorithm 5):
 *     B^(n) <- B^(n) - gamma_B (sum_Omega G^(n) / |Omega| + lambda_B B^(n))
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - the gradient carries no factor 2 (it is the gradient of
 *     1/2 (x - xhat)^2 + 1/2 lambda ||a||^2), as the printed update rules do;
 *   - factor updates carry no 1/M; the core step divides by |Omega|;
 *   - batch-synchronous epoch: nonzeros are taken in the stored order in
 *     consecutive batches of S; every nonzero of a batch reads the factors as
 *     they were at the batch start; the per-nonzero gradients of a row are
 *     summed in increasing nonzero order and applied once at the batch end
 *     (S = 1 is plain sequential SGD);
 *   - an optional per-row step multiplier s scales gamma_A for that row.
 *
 * Parity pins: the tests check this file against a brute-force dense Tucker
 * reconstruction, central finite differences, textbook CP and matrix-
 * factorisation SGD, exact invariants and planted-model recovery.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EARG (-1)
#define ORC_ENOMEM (-2)

#define ORC_MAX_ORDER 16
#define ORC_MAX_RANK 256

/* c^(n) = a^(n)_{i_n,:} B^(n) for every mode n (Eq. "fasttucker"). */
static void orc_c_rows(int N, const int *J, int R, double *const *A,
                       double *const *B, const int32_t *const *idx, int64_t m,
                       double *c /* N*R */) {
  for (int n = 0; n < N; ++n) {
    const double *a = A[n] + (int64_t)idx[n][m] * J[n];
    for (int r = 0; r < R; ++r) {
      double s = 0.0;
      for (int j = 0; j < J[n]; ++j) s += a[j] * B[n][(int64_t)j * R + r];
      c[n * R + r] = s;
    }
  }
}

/* d^(n)_r = prod_{k != n} c^(k)_r (definition of d^(n) in Sec. 2.4). */
static void orc_d_rows(int N, int R, const double *c, double *d /* N*R */) {
  for (int n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r) {
      double p = 1.0;
      for (int k = 0; k < N; ++k)
        if (k != n) p *= c[k * R + r];
      d[n * R + r] = p;
    }
}

/* xhat = sum_r prod_n c^(n)_r (Eq. "fasttucker"). */
static double orc_xhat(int N, int R, const double *c) {
  double x = 0.0;
  for (int r = 0; r < R; ++r) {
    double p = 1.0;
    for (int n = 0; n < N; ++n) p *= c[n * R + r];
    x += p;
  }
  return x;
}

static int orc_check_shape(int N, const int *J, int R) {
  if (N < 1 || N > ORC_MAX_ORDER || R < 1 || R > ORC_MAX_RANK) return ORC_EARG;
  for (int n = 0; n < N; ++n)
    if (J[n] < 1) return ORC_EARG;
  return ORC_OK;
}

/* Predictions xhat for nnz coordinates. */
int orc_predict(int N, const int *J, int R, double *const *A, double *const *B,
                int64_t nnz, const int32_t *const *idx, double *out, int nthreads) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int64_t m = 0; m < nnz; ++m) {
    double c[ORC_MAX_ORDER * ORC_MAX_RANK];
    orc_c_rows(N, J, R, A, B, idx, m, c);
    out[m] = orc_xhat(N, R, c);
  }
  (void)nthreads;
  return ORC_OK;
}

/*
 * Every intermediate of one nonzero m, for the tests:
 *   c[N*R], d[N*R], p[sum_n J_n] with p^(n) = d^(n) B^(n)^T, xhat.
 * p^(n) is the back-projection that appears in the factor update
 * (Eq. "Update_FastTuckerPlus_factor": d^(n) B^(n)^T).
 */
int orc_nonzero_terms(int N, const int *J, int R, double *const *A,
                      double *const *B, const int32_t *const *idx, int64_t m,
                      double *c, double *d, double *p, double *xhat) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  orc_c_rows(N, J, R, A, B, idx, m, c);
  orc_d_rows(N, R, c, d);
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    for (int j = 0; j < J[n]; ++j) {
      double s = 0.0;
      for (int r = 0; r < R; ++r) s += d[n * R + r] * B[n][(int64_t)j * R + r];
      p[off + j] = s;
    }
    off += J[n];
  }
  *xhat = orc_xhat(N, R, c);
  return ORC_OK;
}

/*
 * Factor gradients of one nonzero for every mode (Eq. "Gradient_low_rank_cp"):
 *   g^(n) = -(x - xhat) d^(n) B^(n)^T + lambda a^(n)       -> g[sum_n J_n]
 */
int orc_factor_grads(int N, const int *J, int R, double *const *A,
                     double *const *B, const int32_t *const *idx, int64_t m,
                     double x, double lambda, double *g) {
  double c[ORC_MAX_ORDER * ORC_MAX_RANK], d[ORC_MAX_ORDER * ORC_MAX_RANK];
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  orc_c_rows(N, J, R, A, B, idx, m, c);
  orc_d_rows(N, R, c, d);
  double e = x - orc_xhat(N, R, c);
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    const double *a = A[n] + (int64_t)idx[n][m] * J[n];
    for (int j = 0; j < J[n]; ++j) {
      double dbt = 0.0;
      for (int r = 0; r < R; ++r) dbt += d[n * R + r] * B[n][(int64_t)j * R + r];
      g[off + j] = -e * dbt + lambda * a[j];
    }
    off += J[n];
  }
  return ORC_OK;
}

/*
 * One epoch of the FastTuckerPlus factor phase (Algorithm 3, factor loop;
 * Eq. "Update_FastTuckerPlus_factor"), batch-synchronous with batch size S.
 *
 * For each batch of S consecutive nonzeros (stored order), every nonzero's
 * gradients g^(n) are taken from the factors as they were at the batch
 * start; the gradients that land on the same row are summed in increasing
 * nonzero order; then every touched row takes
 *     a <- a - gamma * s_row * sum g.
 * row_scale: NULL, or N pointers (each NULL or I_n multipliers s_row).
 */
int orc_factor_epoch(int N, const int64_t *I, const int *J, int R,
                     double *const *A, double *const *B, int64_t nnz,
                     const int32_t *const *idx, const double *x, int64_t S,
                     double gamma, double lambda, const double *const *row_scale) {
  if (orc_check_shape(N, J, R) || S < 1) return ORC_EARG;
  double *acc[ORC_MAX_ORDER] = {0};
  unsigned char *touched[ORC_MAX_ORDER] = {0};
  int64_t *rows[ORC_MAX_ORDER] = {0};
  int64_t nrows[ORC_MAX_ORDER];
  int64_t Sb = S < nnz ? S : (nnz > 0 ? nnz : 1);
  int rc = ORC_OK;
  for (int n = 0; n < N; ++n) {
    acc[n] = (double *)calloc((size_t)I[n] * (size_t)J[n], sizeof(double));
    touched[n] = (unsigned char *)calloc((size_t)I[n], 1);
    rows[n] = (int64_t *)malloc((size_t)Sb * sizeof(int64_t));
    if (!acc[n] || !touched[n] || !rows[n]) { rc = ORC_ENOMEM; goto done; }
  }
  for (int64_t b0 = 0; b0 < nnz; b0 += S) {
    int64_t b1 = b0 + S < nnz ? b0 + S : nnz;
    for (int n = 0; n < N; ++n) nrows[n] = 0;
    /* gradients of every nonzero of the batch, from the batch-start factors */
    for (int64_t m = b0; m < b1; ++m) {
      double c[ORC_MAX_ORDER * ORC_MAX_RANK], d[ORC_MAX_ORDER * ORC_MAX_RANK];
      orc_c_rows(N, J, R, A, B, idx, m, c);
      orc_d_rows(N, R, c, d);
      double e = x[m] - orc_xhat(N, R, c);
      for (int n = 0; n < N; ++n) {
        int64_t row = idx[n][m];
        const double *a = A[n] + row * J[n];
        double *g = acc[n] + row * J[n];
        if (!touched[n][row]) { touched[n][row] = 1; rows[n][nrows[n]++] = row; }
        for (int j = 0; j < J[n]; ++j) {
          double dbt = 0.0;
          for (int r = 0; r < R; ++r) dbt += d[n * R + r] * B[n][(int64_t)j * R + r];
          g[j] += -e * dbt + lambda * a[j];
        }
      }
    }
    /* apply the summed gradients once per touched row */
    for (int n = 0; n < N; ++n)
      for (int64_t q = 0; q < nrows[n]; ++q) {
        int64_t row = rows[n][q];
        double s = (row_scale && row_scale[n]) ? row_scale[n][row] : 1.0;
        double *a = A[n] + row * J[n];
        double *g = acc[n] + row * J[n];
        for (int j = 0; j < J[n]; ++j) { a[j] -= gamma * s * g[j]; g[j] = 0.0; }
        touched[n][row] = 0;
      }
  }
done:
  for (int n = 0; n < N; ++n) { free(acc[n]); free(touched[n]); free(rows[n]); }
  return rc;
}

/*
 * Hogwild form of the factor epoch on nthreads host threads, for TIMING the
 * CPU baseline only (it is not a parity reference: its result depends on
 * the thread schedule).  Thread t takes the contiguous range
 * [nnz t / T, nnz (t + 1) / T) of the stored order and applies the rule of
 * Eq. "Update_FastTuckerPlus_factor" one nonzero at a time (S = 1), all N
 * rows from the values it has just read, directly to the shared factor
 * matrices, as the paper's kernel does on the GPU: concurrent updates of a
 * row may be lost.  The shared entries are read and written with relaxed
 * atomic loads and stores (plain loads and stores on x86-64 and aarch64), so
 * the races are well defined.
 */
static double orc_ld(const double *p) {
  double v;
  __atomic_load(p, &v, __ATOMIC_RELAXED);
  return v;
}

static void orc_st(double *p, double v) { __atomic_store(p, &v, __ATOMIC_RELAXED); }

int orc_factor_epoch_hogwild(int N, const int *J, int R, double *const *A,
                             double *const *B, int64_t nnz, const int32_t *const *idx,
                             const double *x, double gamma, double lambda, int nthreads) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  for (int n = 0; n < N; ++n)
    if (J[n] > ORC_MAX_RANK) return ORC_EARG;
  if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
  {
    int tid = 0, nt = 1;
#ifdef _OPENMP
    tid = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    int64_t lo = nnz * tid / nt, hi = nnz * (tid + 1) / nt;
    double a[ORC_MAX_ORDER * ORC_MAX_RANK];   /* the N rows as read */
    double c[ORC_MAX_ORDER * ORC_MAX_RANK], d[ORC_MAX_ORDER * ORC_MAX_RANK];
    for (int64_t m = lo; m < hi; ++m) {
      for (int n = 0; n < N; ++n) {
        const double *row = A[n] + (int64_t)idx[n][m] * J[n];
        for (int j = 0; j < J[n]; ++j) a[n * ORC_MAX_RANK + j] = orc_ld(row + j);
        for (int r = 0; r < R; ++r) {
          double sum = 0.0;
          for (int j = 0; j < J[n]; ++j) sum += a[n * ORC_MAX_RANK + j] * B[n][(int64_t)j * R + r];
          c[n * R + r] = sum;
        }
      }
      orc_d_rows(N, R, c, d);
      double e = x[m] - orc_xhat(N, R, c);
      for (int n = 0; n < N; ++n) {
        double *row = A[n] + (int64_t)idx[n][m] * J[n];
        for (int j = 0; j < J[n]; ++j) {
          double dbt = 0.0;
          for (int r = 0; r < R; ++r) dbt += d[n * R + r] * B[n][(int64_t)j * R + r];
          const double av = a[n * ORC_MAX_RANK + j];
          orc_st(row + j, av - gamma * (-e * dbt + lambda * av));
        }
      }
    }
  }
  return ORC_OK;
}

/*
 * Core gradient summed over the training set (Algorithm 5 accumulation of
 * Eq. "Gradient_core_tensor_cp" without the regulariser):
 *     G^(n) = sum_m (xhat_m - x_m) a^(n)_{i_n}^T d^(n)        (J_n x R)
 * With nthreads > 1 the nonzeros are cut into nthreads contiguous ranges,
 * each summed in order, and the range sums are added in range order.
 */
int orc_core_grad(int N, const int *J, int R, double *const *A, double *const *B,
                  int64_t nnz, const int32_t *const *idx, const double *x,
                  double *const *G, int nthreads) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  if (nthreads < 1) nthreads = 1;
  int64_t sumJR = 0;
  for (int n = 0; n < N; ++n) sumJR += (int64_t)J[n] * R;
  double *part = (double *)calloc((size_t)nthreads * (size_t)sumJR, sizeof(double));
  if (!part) return ORC_ENOMEM;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
  {
    int tid = 0, nt = 1;
#ifdef _OPENMP
    tid = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    int64_t lo = nnz * tid / nt, hi = nnz * (tid + 1) / nt;
    double *gp = part + (int64_t)tid * sumJR;
    for (int64_t m = lo; m < hi; ++m) {
      double c[ORC_MAX_ORDER * ORC_MAX_RANK], d[ORC_MAX_ORDER * ORC_MAX_RANK];
      orc_c_rows(N, J, R, A, B, idx, m, c);
      orc_d_rows(N, R, c, d);
      double ne = orc_xhat(N, R, c) - x[m];
      int64_t off = 0;
      for (int n = 0; n < N; ++n) {
        const double *a = A[n] + (int64_t)idx[n][m] * J[n];
        for (int j = 0; j < J[n]; ++j)
          for (int r = 0; r < R; ++r) gp[off + (int64_t)j * R + r] += ne * a[j] * d[n * R + r];
        off += (int64_t)J[n] * R;
      }
    }
  }
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    for (int64_t q = 0; q < (int64_t)J[n] * R; ++q) {
      double s = 0.0;
      for (int t = 0; t < nthreads; ++t) s += part[(int64_t)t * sumJR + off + q];
      G[n][q] = s;
    }
    off += (int64_t)J[n] * R;
  }
  free(part);
  return ORC_OK;
}

/*
 * One core phase (Algorithm 5): gradient over all nnz training nonzeros,
 * then B^(n) <- B^(n) - gamma (G^(n) / nnz + lambda B^(n)) for every n.
 */
int orc_core_epoch(int N, const int *J, int R, double *const *A, double *const *B,
                   int64_t nnz, const int32_t *const *idx, const double *x,
                   double gamma, double lambda, int nthreads) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  double *G[ORC_MAX_ORDER] = {0};
  int rc = ORC_OK;
  for (int n = 0; n < N; ++n) {
    G[n] = (double *)malloc((size_t)J[n] * (size_t)R * sizeof(double));
    if (!G[n]) { rc = ORC_ENOMEM; goto done; }
  }
  rc = orc_core_grad(N, J, R, A, B, nnz, idx, x, G, nthreads);
  if (rc) goto done;
  for (int n = 0; n < N; ++n)
    for (int64_t q = 0; q < (int64_t)J[n] * R; ++q) {
      double gq = nnz > 0 ? G[n][q] / (double)nnz : 0.0;
      B[n][q] -= gamma * (gq + lambda * B[n][q]);
    }
done:
  for (int n = 0; n < N; ++n) free(G[n]);
  return rc;
}

/*
 * Core phase in the per-sample-set reading of Algorithm 3, whose core loop
 * applies rule "Update_FastTuckerPlus_core" for every sampled set Psi: the
 * nonzeros are taken in stored order in consecutive sets of S, and each set
 * makes one step of Algorithm 5 restricted to it, from the core matrices as
 * they were at the set's start:
 *     B^(n) <- B^(n) - gamma (sum_Psi G^(n) / |Psi| + lambda B^(n))
 * S >= nnz is one step of Algorithm 5 (orc_core_epoch).
 */
int orc_core_epoch_sgd(int N, const int *J, int R, double *const *A, double *const *B,
                       int64_t nnz, const int32_t *const *idx, const double *x, int64_t S,
                       double gamma, double lambda, int nthreads) {
  if (orc_check_shape(N, J, R) || S < 1) return ORC_EARG;
  for (int64_t lo = 0; lo < nnz; lo += S) {
    const int64_t cnt = (nnz - lo < S) ? nnz - lo : S;
    const int32_t *set_idx[ORC_MAX_ORDER];
    for (int n = 0; n < N; ++n) set_idx[n] = idx[n] + lo;
    const int rc = orc_core_epoch(N, J, R, A, B, cnt, set_idx, x + lo, gamma, lambda, nthreads);
    if (rc) return rc;
  }
  return ORC_OK;
}

/*
 * Test-set errors (Sec. 5.2): out[0] = RMSE = sqrt(sum e^2 / n),
 * out[1] = MAE = sum |e| / n, out[2] = sum e^2, with e = x - xhat.
 */
int orc_errors(int N, const int *J, int R, double *const *A, double *const *B,
               int64_t nnz, const int32_t *const *idx, const double *x, double *out,
               int nthreads) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  if (nthreads < 1) nthreads = 1;
  double *part = (double *)calloc((size_t)nthreads * 2, sizeof(double));
  if (!part) return ORC_ENOMEM;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
  {
    int tid = 0, nt = 1;
#ifdef _OPENMP
    tid = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    int64_t lo = nnz * tid / nt, hi = nnz * (tid + 1) / nt;
    double se = 0.0, ae = 0.0;
    for (int64_t m = lo; m < hi; ++m) {
      double c[ORC_MAX_ORDER * ORC_MAX_RANK];
      orc_c_rows(N, J, R, A, B, idx, m, c);
      double e = x[m] - orc_xhat(N, R, c);
      se += e * e;
      ae += fabs(e);
    }
    part[2 * tid] = se;
    part[2 * tid + 1] = ae;
  }
  double se = 0.0, ae = 0.0;
  for (int t = 0; t < nthreads; ++t) { se += part[2 * t]; ae += part[2 * t + 1]; }
  free(part);
  out[0] = nnz > 0 ? sqrt(se / (double)nnz) : 0.0;
  out[1] = nnz > 0 ? ae / (double)nnz : 0.0;
  out[2] = se;
  return ORC_OK;
}

/*
 * Objective of Eq. "low_rank_optimization_all" with the regulariser summed
 * over every mode:  sum_Omega (x - xhat)^2 + lambda_A sum_n ||A^(n)||^2
 *                    + lambda_B sum_n ||B^(n)||^2.
 */
int orc_objective(int N, const int64_t *I, const int *J, int R, double *const *A,
                  double *const *B, int64_t nnz, const int32_t *const *idx,
                  const double *x, double lambda_a, double lambda_b, double *out,
                  int nthreads) {
  double err[3];
  int rc = orc_errors(N, J, R, A, B, nnz, idx, x, err, nthreads);
  if (rc) return rc;
  double na = 0.0, nb = 0.0;
  for (int n = 0; n < N; ++n) {
    for (int64_t q = 0; q < I[n] * J[n]; ++q) na += A[n][q] * A[n][q];
    for (int64_t q = 0; q < (int64_t)J[n] * R; ++q) nb += B[n][q] * B[n][q];
  }
  *out = err[2] + lambda_a * na + lambda_b * nb;
  return ORC_OK;
}

/* ======================================================================
 * Learned per-row step sizes (not in the paper; an optional extension of the
 * factor step of Eq. "Update_FastTuckerPlus_factor" with a per-row
 * multiplier s: a <- a - gamma * s * g).
 *
 * Row statistics of mode n, row r, from the current A and B:
 *   count_r  number of nonzeros whose mode-n index is r
 *   g_r      sum over those nonzeros of the factor gradient
 *            -e_m p_m + lambda a_r,  p_m = d_m B^(n)T   (Eq. "Gradient_low_rank_cp")
 *   ebar_r   mean residual  sum e_m / count_r
 *   gnorm_r  |g_r| / max(count_r, 1);  ema_r = beta ema_in_r + (1 - beta) gnorm_r
 * Features: f0 = log(1 + count_r), f1 = log(1 + ema_r), f2 = ebar_r.
 * Label: the exact line-search step of the row's convex subproblem
 *   F_r(a) = sum_m [1/2 (x_m - a.p_m)^2 + 1/2 lambda |a|^2]
 * along -g_r:  t* = |g|^2 / (sum_m (p_m.g)^2 + lambda count |g|^2).  Every
 * nonzero moves its N rows at once, and each row's exact step alone would
 * remove the nonzero's residual, so together they would remove it N times
 * over; the row's share is t* / N.  Expressed as a multiplier of the epoch's
 * SGD step gamma * g:  s* = t* / (N gamma), clipped to [1/16, 16]; the label
 * is log s* (rows without nonzeros, or with g = 0, get log 1 = 0).
 * Rows of all modes are concatenated (mode 0 first).
 * ====================================================================== */
#define ORC_SMIN (1.0 / 16.0)
#define ORC_SMAX 16.0

int orc_row_stats(int N, const int64_t *I, const int *J, int R, double *const *A,
                  double *const *B, int64_t nnz, const int32_t *const *idx, const double *x,
                  double lambda, double gamma, double beta, const double *ema_in,
                  double *feat /* rows x 3 */, double *label /* rows, nullable */) {
  if (orc_check_shape(N, J, R)) return ORC_EARG;
  int64_t rows = 0, off[ORC_MAX_ORDER + 1];
  int64_t goff[ORC_MAX_ORDER + 1];
  off[0] = 0;
  goff[0] = 0;
  for (int n = 0; n < N; ++n) {
    off[n + 1] = off[n] + I[n];
    goff[n + 1] = goff[n] + I[n] * J[n];
  }
  rows = off[N];
  double *cnt = (double *)calloc((size_t)rows, sizeof(double));
  double *esum = (double *)calloc((size_t)rows, sizeof(double));
  double *hsum = (double *)calloc((size_t)rows, sizeof(double));
  double *g = (double *)calloc((size_t)goff[N], sizeof(double));
  double *p = (double *)malloc(sizeof(double) * ORC_MAX_RANK);
  int rc = ORC_OK;
  if (!cnt || !esum || !hsum || !g || !p) { rc = ORC_ENOMEM; goto done; }
  /* pass 1: counts, residual sums, row gradients */
  for (int64_t m = 0; m < nnz; ++m) {
    double c[ORC_MAX_ORDER * ORC_MAX_RANK], d[ORC_MAX_ORDER * ORC_MAX_RANK];
    orc_c_rows(N, J, R, A, B, idx, m, c);
    orc_d_rows(N, R, c, d);
    double e = x[m] - orc_xhat(N, R, c);
    for (int n = 0; n < N; ++n) {
      int64_t row = idx[n][m];
      const double *a = A[n] + row * J[n];
      cnt[off[n] + row] += 1.0;
      esum[off[n] + row] += e;
      for (int j = 0; j < J[n]; ++j) {
        double pj = 0.0;
        for (int r = 0; r < R; ++r) pj += d[n * R + r] * B[n][(int64_t)j * R + r];
        g[goff[n] + row * J[n] + j] += -e * pj + lambda * a[j];
      }
    }
  }
  /* pass 2: curvature along g, sum_m (p_m . g_r)^2 */
  if (label) {
    for (int64_t m = 0; m < nnz; ++m) {
      double c[ORC_MAX_ORDER * ORC_MAX_RANK], d[ORC_MAX_ORDER * ORC_MAX_RANK];
      orc_c_rows(N, J, R, A, B, idx, m, c);
      orc_d_rows(N, R, c, d);
      for (int n = 0; n < N; ++n) {
        int64_t row = idx[n][m];
        double q = 0.0;
        for (int j = 0; j < J[n]; ++j) {
          double pj = 0.0;
          for (int r = 0; r < R; ++r) pj += d[n * R + r] * B[n][(int64_t)j * R + r];
          q += pj * g[goff[n] + row * J[n] + j];
        }
        hsum[off[n] + row] += q * q;
      }
    }
  }
  for (int n = 0; n < N; ++n)
    for (int64_t row = 0; row < I[n]; ++row) {
      int64_t q = off[n] + row;
      double gg = 0.0;
      for (int j = 0; j < J[n]; ++j) {
        double v = g[goff[n] + row * J[n] + j];
        gg += v * v;
      }
      double k = cnt[q];
      double gnorm = sqrt(gg) / (k > 1.0 ? k : 1.0);
      double ema = ema_in ? beta * ema_in[q] + (1.0 - beta) * gnorm : gnorm;
      feat[3 * q + 0] = log(1.0 + k);
      feat[3 * q + 1] = log(1.0 + ema);
      feat[3 * q + 2] = k > 0.0 ? esum[q] / k : 0.0;
      if (label) {
        double s = 1.0;
        double den = hsum[q] + lambda * k * gg;
        if (k > 0.0 && gg > 0.0 && den > 0.0) {
          s = gg / den / ((double)N * gamma);
          if (s < ORC_SMIN) s = ORC_SMIN;
          if (s > ORC_SMAX) s = ORC_SMAX;
        }
        label[q] = log(s);
      }
    }
done:
  free(cnt); free(esum); free(hsum); free(g); free(p);
  return rc;
}

/*
 * Step-size network: features (3) -> 64 -> 64 -> 1 with ReLU and a linear
 * output u, the predicted log-multiplier; the multiplier is
 * s = exp(min(max(u, log 1/16), log 16)).  Parameters, in this order:
 * W1 [64][3], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1]  (4481 values).
 */
#define ORC_H 64
#define ORC_NPARAM (ORC_H * 3 + ORC_H + ORC_H * ORC_H + ORC_H + ORC_H + 1)

int orc_mlp_nparams(void) { return ORC_NPARAM; }

/* The network's output u (the log-multiplier) for one row of features. */
static double orc_mlp_row(const double *P, const double *x, double *h1, double *h2) {
  const double *W1 = P, *b1 = W1 + ORC_H * 3, *W2 = b1 + ORC_H, *b2 = W2 + ORC_H * ORC_H;
  const double *w3 = b2 + ORC_H, *b3 = w3 + ORC_H;
  for (int i = 0; i < ORC_H; ++i) {
    double s = b1[i];
    for (int k = 0; k < 3; ++k) s += W1[i * 3 + k] * x[k];
    h1[i] = s > 0.0 ? s : 0.0;
  }
  double u = b3[0];
  for (int i = 0; i < ORC_H; ++i) {
    double s = b2[i];
    for (int j = 0; j < ORC_H; ++j) s += W2[i * ORC_H + j] * h1[j];
    h2[i] = s > 0.0 ? s : 0.0;
    u += w3[i] * h2[i];
  }
  return u;
}

/* Multipliers s = exp(clamp(u, log 1/16, log 16)) of n rows. */
int orc_mlp_forward(const double *P, int64_t n, const double *X, double *s) {
  double h1[ORC_H], h2[ORC_H];
  for (int64_t m = 0; m < n; ++m) {
    double u = orc_mlp_row(P, X + 3 * m, h1, h2);
    if (u < log(ORC_SMIN)) u = log(ORC_SMIN);
    if (u > log(ORC_SMAX)) u = log(ORC_SMAX);
    s[m] = exp(u);
  }
  return ORC_OK;
}

/* Gradient of L = (1/n) sum_m 1/2 (u_m - y_m)^2, u the linear output and y
 * the log-multiplier labels, with respect to every parameter (same layout);
 * *loss receives L.  The output is not clamped in the loss, so its gradient
 * never vanishes. */
int orc_mlp_grad(const double *P, int64_t n, const double *X, const double *y, double *G,
                 double *loss) {
  const double *W2 = P + ORC_H * 3 + ORC_H, *w3 = W2 + ORC_H * ORC_H + ORC_H;
  double *gW1 = G, *gb1 = gW1 + ORC_H * 3, *gW2 = gb1 + ORC_H, *gb2 = gW2 + ORC_H * ORC_H;
  double *gw3 = gb2 + ORC_H, *gb3 = gw3 + ORC_H;
  double h1[ORC_H], h2[ORC_H], dh1[ORC_H], L = 0.0;
  for (int q = 0; q < ORC_NPARAM; ++q) G[q] = 0.0;
  for (int64_t m = 0; m < n; ++m) {
    const double *x = X + 3 * m;
    double u = orc_mlp_row(P, x, h1, h2);
    double r = u - y[m];
    L += 0.5 * r * r;
    double dz = r / (double)n;
    gb3[0] += dz;
    for (int j = 0; j < ORC_H; ++j) dh1[j] = 0.0;
    for (int i = 0; i < ORC_H; ++i) {
      gw3[i] += dz * h2[i];
      double dh2 = h2[i] > 0.0 ? dz * w3[i] : 0.0;
      gb2[i] += dh2;
      for (int j = 0; j < ORC_H; ++j) {
        gW2[i * ORC_H + j] += dh2 * h1[j];
        dh1[j] += dh2 * W2[i * ORC_H + j];
      }
    }
    for (int j = 0; j < ORC_H; ++j) {
      double d = h1[j] > 0.0 ? dh1[j] : 0.0;
      gb1[j] += d;
      for (int k = 0; k < 3; ++k) gW1[j * 3 + k] += d * x[k];
    }
  }
  *loss = n > 0 ? L / (double)n : 0.0;
  return ORC_OK;
}
