/*
 * Multi-threaded timing copy of the oracle's pipelined CG (Algorithm 2, beta from Eq. (3)),
 * for the CPU baseline of the benchmark only.
 *
 * TEST INFRASTRUCTURE ONLY.  The parity oracle is the sequential orc_cg_pipelined in
 * pk_oracle.c; this file exists so that the CPU baseline can be reported the way the paper's
 * Sec. 4 reports its CPU comparison (the best of several process counts): the same steps of
 * Algorithm 2, in the same order and with the same per-row arithmetic, with every loop over
 * rows split into equal contiguous ranges, one per OpenMP thread (static schedule).  Inner
 * products are summed per thread with Neumaier's compensated summation, as in the
 * sequential oracle, and the per-thread sums are added in thread order, so the result
 * depends on the thread count only through that final order.
 * It shares no code with the CUDA library and none with pk_oracle.c (it is compiled into a
 * library of its own, with -fopenmp).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OMP_OK = 0, OMP_ERR_OOM = 3, OMP_NOT_CONVERGED = 4, OMP_NOT_SPD = 6, OMP_NAN = 7 };

/* threads the parallel regions will use; set them (t > 0) before a solve */
int32_t orc_omp_threads(void) { return (int32_t)omp_get_max_threads(); }
void orc_omp_set_threads(int32_t t) { if (t > 0) omp_set_num_threads(t); }

static void spmv_par(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                     const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j) s += va[j] * x[ci[j]];
    y[i] = s;
  }
}

/* Neumaier-compensated sum of x_i y_i over this thread's static range; sums added in
 * thread order. */
static double dot_par(int32_t n, const double* x, const double* y) {
  const int nt = omp_get_max_threads();
  double* part = calloc((size_t)nt, sizeof(double));
  if (!part) return NAN;
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num(), T = omp_get_num_threads();
    const int64_t lo = (int64_t)n * t / T, hi = (int64_t)n * (t + 1) / T;
    double s = 0.0, c = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
      const double p = x[i] * y[i];
      const double u = s + p;
      if (fabs(s) >= fabs(p)) c += (s - u) + p;
      else c += (p - u) + s;
      s = u;
    }
    part[t] = s + c;
  }
  double tot = 0.0;
  for (int t = 0; t < nt; ++t) tot += part[t];
  free(part);
  return tot;
}

int orc_cg_pipelined_omp(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                         const double* b, double* x, double tol, int32_t maxit,
                         int32_t* iters_out) {
  *iters_out = 0;
  if (n <= 0) return OMP_OK;
  const double bb = dot_par(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return OMP_OK; }
  const double thr2 = tol * tol * bb;
  double *r = malloc(sizeof(double) * (size_t)n), *p = malloc(sizeof(double) * (size_t)n),
         *ap = malloc(sizeof(double) * (size_t)n);
  if (!r || !p || !ap) { free(r); free(p); free(ap); return OMP_ERR_OOM; }
  int status = OMP_NOT_CONVERGED;
  spmv_par(n, rp, ci, va, x, ap);
#pragma omp parallel for schedule(static)
  for (int32_t k = 0; k < n; ++k) { r[k] = b[k] - ap[k]; p[k] = r[k]; }
  double rr = dot_par(n, r, r);
  if (!isfinite(rr)) { status = OMP_NAN; goto done; }
  if (rr <= thr2) { status = OMP_OK; goto done; }
  spmv_par(n, rp, ci, va, p, ap);
  double apap = dot_par(n, ap, ap), pap = dot_par(n, p, ap);
  if (!isfinite(apap) || !isfinite(pap)) { status = OMP_NAN; goto done; }
  if (pap <= 0.0) { status = OMP_NOT_SPD; goto done; }
  double alpha = rr / pap;
  double beta = alpha * alpha * apap / rr - 1.0;
  for (int32_t i = 1; i <= maxit; ++i) {
#pragma omp parallel for schedule(static)
    for (int32_t k = 0; k < n; ++k) {
      x[k] += alpha * p[k];
      r[k] -= alpha * ap[k];
      p[k] = r[k] + beta * p[k];
    }
    rr = dot_par(n, r, r);
    *iters_out = i;
    if (!isfinite(rr)) { status = OMP_NAN; break; }
    if (rr <= thr2) { status = OMP_OK; break; }
    if (i == maxit) break;
    spmv_par(n, rp, ci, va, p, ap);
    apap = dot_par(n, ap, ap);
    pap = dot_par(n, p, ap);
    if (!isfinite(apap) || !isfinite(pap)) { status = OMP_NAN; break; }
    if (pap <= 0.0) { status = OMP_NOT_SPD; break; }
    alpha = rr / pap;
    beta = alpha * alpha * apap / rr - 1.0;
  }
done:
  free(r); free(p); free(ap);
  return status;
}
