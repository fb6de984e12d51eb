/*
 * Plain FP64 CPU oracle for the pipelined Krylov solvers of Rupp, Weinbub, Juengel and
 * Grasser, "Pipelined Iterative Solvers with Kernel Fusion for Graphics Processing Units"
 * (ACM TOMS 2015, arXiv:1410.4054).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls this file:
 * only the test suite, the smoke check and the CPU-baseline leg of the benchmark do.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Everything is sequential FP64 in natural row order (matrix rows summed left to right, inner
 * products with compensated summation), following the algorithms step by step:
 *   orc_cg_classical        Algorithm 1 (classical CG)
 *   orc_cg_pipelined        Algorithm 2 (pipelined CG, beta from Eq. (3))
 *   orc_bicgstab_classical  Algorithm 3 (classical BiCGStab)
 *   orc_bicgstab_pipelined  Algorithm 4 (pipelined BiCGStab, beta = -<As,r0*>/<Ap,r0*>,
 *                           residual-norm expansion of Sec. 3.2)
 *   orc_gmres               Algorithms 5 and 6 (restarted simpler GMRES with classical
 *                           Gram-Schmidt; classical form updates the residual, pipelined
 *                           form uses xi_i = <v_0, v_i>)
 *   orc_gmres_cgs2          the same with Gram-Schmidt applied twice per step (CGS2)
 *   orc_gmres_shift3        the shift-invariant three-kernel form of Sec. 3.3 (||v_i||
 *                           from the Gram-Schmidt inner products of the shifted vector)
 *   orc_jacobi_right_begin  right preconditioning with M = diag(A) for BiCGStab and GMRES:
 *   orc_jacobi_right_end    the solver runs on A M^-1 y = b, and x = M^-1 y
 *   orc_pcg_jacobi          CG with the Jacobi preconditioner M = diag(A) (Sec. 5 names
 *                           preconditioner fusion as the natural extension): the standard
 *                           preconditioned CG, and the pipelined form of Algorithm 2 with
 *                           the preconditioned inner products, beta from the analogue of
 *                           Eq. (3): beta = alpha^2 <Ap, M^-1 Ap> / <r, M^-1 r> - 1.
 *
 * Readings of points the paper leaves open (they are listed with reasons in the design
 * notes of the repository):
 *   - r0* = r0 (Alg. 3/4 "choose r0* arbitrary").
 *   - Stop when ||r||_2 <= tol * ||b||_2; b = 0 gives x = 0 after zero iterations.
 *   - CG: the squared residual <r_i, r_i> that the update step produces is tested before
 *     A p_i is formed; "iterations" counts updates of x.  <p, Ap> <= 0 -> NOT_SPD.
 *   - BiCGStab: ||s|| <= tol ||b|| ends the iteration after x += alpha p (standard early
 *     exit); otherwise the iteration completes and the directly computed <r_{i+1}, r_{i+1}>
 *     is tested.  The pipelined form also records the Sec. 3.2 expansion
 *     <s,s> - 2 omega <s,As> + omega^2 <As,As>.  A zero or non-finite denominator is a
 *     BREAKDOWN.
 *   - GMRES: R_{i,i} = ||v_i|| before normalisation; the update is
 *     x <- x0 + rho0 (eta_1 v_0 + sum_{i=2..k} eta_i v_{i-1}) with R eta = xi.
 *     Within a cycle the residual estimate rho0 sqrt(max(0, 1 - sum xi_j^2)) (pipelined)
 *     or rho0 ||r|| (classical) ends the cycle when <= tol ||b||, when the squared relative
 *     estimate is <= 1e-12, at k = m, or when the iteration budget is spent.  Convergence is
 *     declared only from the true residual b - A x at a cycle boundary.  maxit counts
 *     Arnoldi steps over all cycles.  R_{i,i} <= 1e-14 ||A v_{i-1}|| ends the cycle before
 *     step i (lucky breakdown).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* status codes of the oracle */
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 4, ORC_BREAKDOWN = 5, ORC_NOT_SPD = 6, ORC_NAN = 7,
       ORC_ERR_ARG = 1, ORC_ERR_OOM = 3 };

/* ---------------------------------------------------------------- basic operations */

/* y = A x, row by row, each row summed left to right (Sec. 2.2 CSR product). */
void orc_spmv(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
              const double* x, double* y) {
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j) s += va[j] * x[ci[j]];
    y[i] = s;
  }
}

/* <x, y>: the products x_i y_i summed left to right with Neumaier's compensated summation
 * (A. Neumaier, ZAMM 54, 1974), so that the inner products <.,.> of Algorithms 1-6 are
 * evaluated to about one rounding error independently of n.  A plain running sum carries an
 * O(n eps) error that, at n = 10^6 and after the cancellation in Eq. (3)
 * (beta = alpha^2 <Ap,Ap>/<r,r> - 1), is larger than the 1e-12 parity bar itself. */
double orc_dot(int32_t n, const double* x, const double* y) {
  double s = 0.0, c = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double t = x[i] * y[i];
    const double u = s + t;
    if (fabs(s) >= fabs(t)) c += (s - u) + t;
    else c += (t - u) + s;
    s = u;
  }
  return s + c;
}

static void record(double* tr, int32_t cap, int32_t k, double v) {
  if (tr && k >= 0 && k < cap) tr[k] = v;
}

static int finite3(double a, double b, double c) { return isfinite(a) && isfinite(b) && isfinite(c); }

/* ---------------------------------------------------------------- CG, Algorithm 1 */

int orc_cg_classical(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                     const double* b, double* x, double tol, int32_t maxit, int32_t cap,
                     double* tr_alpha, double* tr_beta, double* tr_res2, int32_t* iters_out) {
  *iters_out = 0;
  if (n <= 0) return ORC_OK;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double thr2 = tol * tol * bb;
  double *r = malloc(sizeof(double) * (size_t)n), *p = malloc(sizeof(double) * (size_t)n),
         *ap = malloc(sizeof(double) * (size_t)n);
  if (!r || !p || !ap) { free(r); free(p); free(ap); return ORC_ERR_OOM; }
  int status = ORC_NOT_CONVERGED;
  /* p0 = r0 = b - A x0 */
  orc_spmv(n, rp, ci, va, x, ap);
  for (int32_t k = 0; k < n; ++k) { r[k] = b[k] - ap[k]; p[k] = r[k]; }
  double rr = orc_dot(n, r, r);
  if (!isfinite(rr)) { status = ORC_NAN; goto done; }
  if (rr <= thr2) { status = ORC_OK; goto done; }
  for (int32_t i = 0; i < maxit; ++i) {
    orc_spmv(n, rp, ci, va, p, ap);              /* A p_i */
    double pap = orc_dot(n, p, ap);              /* <p_i, A p_i> */
    if (!isfinite(pap)) { status = ORC_NAN; break; }
    if (pap <= 0.0) { status = ORC_NOT_SPD; break; }
    double alpha = rr / pap;
    for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k];
    for (int32_t k = 0; k < n; ++k) r[k] -= alpha * ap[k];
    double rr_new = orc_dot(n, r, r);            /* <r_{i+1}, r_{i+1}> */
    record(tr_alpha, cap, i, alpha);
    record(tr_res2, cap, i, rr_new);
    *iters_out = i + 1;
    if (!isfinite(rr_new)) { status = ORC_NAN; break; }
    if (rr_new <= thr2) { status = ORC_OK; break; }
    double beta = rr_new / rr;
    record(tr_beta, cap, i, beta);
    for (int32_t k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
    rr = rr_new;
  }
done:
  free(r); free(p); free(ap);
  return status;
}

/* ---------------------------------------------------------------- CG, Algorithm 2 */

int orc_cg_pipelined(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                     const double* b, double* x, double tol, int32_t maxit, int32_t cap,
                     double* tr_alpha, double* tr_beta, double* tr_res2, int32_t* iters_out) {
  *iters_out = 0;
  if (n <= 0) return ORC_OK;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double thr2 = tol * tol * bb;
  double *r = malloc(sizeof(double) * (size_t)n), *p = malloc(sizeof(double) * (size_t)n),
         *ap = malloc(sizeof(double) * (size_t)n);
  if (!r || !p || !ap) { free(r); free(p); free(ap); return ORC_ERR_OOM; }
  int status = ORC_NOT_CONVERGED;
  /* p0 = r0 = b - A x0 */
  orc_spmv(n, rp, ci, va, x, ap);
  for (int32_t k = 0; k < n; ++k) { r[k] = b[k] - ap[k]; p[k] = r[k]; }
  double rr = orc_dot(n, r, r);
  if (!isfinite(rr)) { status = ORC_NAN; goto done; }
  if (rr <= thr2) { status = ORC_OK; goto done; }
  /* A p0, alpha_0 = <r0,r0>/<p0,Ap0>, beta_0 = alpha_0^2 <Ap0,Ap0>/<r0,r0> - 1 */
  orc_spmv(n, rp, ci, va, p, ap);
  double apap = orc_dot(n, ap, ap);
  double pap = orc_dot(n, p, ap);
  if (!finite3(apap, pap, rr)) { status = ORC_NAN; goto done; }
  if (pap <= 0.0) { status = ORC_NOT_SPD; goto done; }
  double alpha = rr / pap;
  double beta = alpha * alpha * apap / rr - 1.0;
  record(tr_alpha, cap, 0, alpha);
  record(tr_beta, cap, 0, beta);
  for (int32_t i = 1; i <= maxit; ++i) {
    /* x_i, r_i, p_i from alpha_{i-1}, beta_{i-1} */
    for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k];
    for (int32_t k = 0; k < n; ++k) r[k] -= alpha * ap[k];
    for (int32_t k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
    rr = orc_dot(n, r, r);                        /* <r_i, r_i> */
    record(tr_res2, cap, i - 1, rr);
    *iters_out = i;
    if (!isfinite(rr)) { status = ORC_NAN; break; }
    if (rr <= thr2) { status = ORC_OK; break; }
    if (i == maxit) break;
    orc_spmv(n, rp, ci, va, p, ap);               /* A p_i */
    apap = orc_dot(n, ap, ap);                    /* <Ap_i, Ap_i> */
    pap = orc_dot(n, p, ap);                      /* <p_i, Ap_i> */
    if (!finite3(apap, pap, rr)) { status = ORC_NAN; break; }
    if (pap <= 0.0) { status = ORC_NOT_SPD; break; }
    alpha = rr / pap;
    beta = alpha * alpha * apap / rr - 1.0;       /* Eq. (3) */
    record(tr_alpha, cap, i, alpha);
    record(tr_beta, cap, i, beta);
  }
done:
  free(r); free(p); free(ap);
  return status;
}

/* ---------------------------------------------------------------- Jacobi-preconditioned CG */

/* M^-1 = diag(A)^-1, applied as a product with the reciprocal of every diagonal entry
 * (entries of a row in column i summed).  A zero or negative diagonal entry cannot belong to
 * an SPD matrix: NOT_SPD. */
static int jacobi_inverse(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                          double* dinv) {
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j)
      if (ci[j] == i) d += va[j];
    if (!(d > 0.0)) return ORC_NOT_SPD;
    dinv[i] = 1.0 / d;
  }
  return ORC_OK;
}

/* Preconditioned CG with M = diag(A).  Classical (pipelined = 0): z = M^-1 r, gamma = <r, z>,
 * alpha = gamma / <p, Ap>, beta = gamma_{i+1} / gamma_i, p = z + beta p.  Pipelined
 * (pipelined = 1): the structure of Algorithm 2 -- the update step forms x, r and
 * p = M^-1 r + beta p with <r, M^-1 r> and <r, r>; the SpMV step forms Ap with <p, Ap> and
 * <Ap, M^-1 Ap>, and alpha = <r, M^-1 r>/<p, Ap>, beta = alpha^2 <Ap, M^-1 Ap>/<r, M^-1 r> - 1.
 * The stopping test is on the unpreconditioned ||r||.  The traces record alpha_i, beta_i and
 * <r_i, r_i>. */
int orc_pcg_jacobi(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                   const double* b, double* x, double tol, int32_t maxit, int32_t pipelined,
                   int32_t cap, double* tr_alpha, double* tr_beta, double* tr_res2,
                   int32_t* iters_out) {
  *iters_out = 0;
  if (n <= 0) return ORC_OK;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double thr2 = tol * tol * bb;
  size_t sz = sizeof(double) * (size_t)n;
  double *r = malloc(sz), *p = malloc(sz), *ap = malloc(sz), *z = malloc(sz), *dinv = malloc(sz);
  if (!r || !p || !ap || !z || !dinv) { free(r); free(p); free(ap); free(z); free(dinv); return ORC_ERR_OOM; }
  int status = jacobi_inverse(n, rp, ci, va, dinv);
  if (status != ORC_OK) goto done;
  status = ORC_NOT_CONVERGED;
  /* r0 = b - A x0, z0 = M^-1 r0, p0 = z0 */
  orc_spmv(n, rp, ci, va, x, ap);
  for (int32_t k = 0; k < n; ++k) { r[k] = b[k] - ap[k]; z[k] = r[k] * dinv[k]; p[k] = z[k]; }
  double rr = orc_dot(n, r, r);
  double gamma = orc_dot(n, r, z);
  if (!isfinite(rr) || !isfinite(gamma)) { status = ORC_NAN; goto done; }
  if (rr <= thr2) { status = ORC_OK; goto done; }
  if (!pipelined) {
    for (int32_t i = 0; i < maxit; ++i) {
      orc_spmv(n, rp, ci, va, p, ap);
      const double pap = orc_dot(n, p, ap);
      if (!finite3(pap, gamma, rr)) { status = ORC_NAN; break; }
      if (pap <= 0.0) { status = ORC_NOT_SPD; break; }
      const double alpha = gamma / pap;
      record(tr_alpha, cap, i, alpha);
      for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k];
      for (int32_t k = 0; k < n; ++k) r[k] -= alpha * ap[k];
      rr = orc_dot(n, r, r);
      record(tr_res2, cap, i, rr);
      *iters_out = i + 1;
      if (!isfinite(rr)) { status = ORC_NAN; break; }
      if (rr <= thr2) { status = ORC_OK; break; }
      for (int32_t k = 0; k < n; ++k) z[k] = r[k] * dinv[k];
      const double gnew = orc_dot(n, r, z);
      const double beta = gnew / gamma;
      record(tr_beta, cap, i, beta);
      gamma = gnew;
      for (int32_t k = 0; k < n; ++k) p[k] = z[k] + beta * p[k];
    }
    goto done;
  }
  /* pipelined: A p0, alpha_0, beta_0 */
  orc_spmv(n, rp, ci, va, p, ap);
  for (int32_t k = 0; k < n; ++k) z[k] = ap[k] * dinv[k];
  double qdq = orc_dot(n, ap, z);                 /* <Ap, M^-1 Ap> */
  double pap = orc_dot(n, p, ap);
  if (!finite3(qdq, pap, gamma)) { status = ORC_NAN; goto done; }
  if (pap <= 0.0) { status = ORC_NOT_SPD; goto done; }
  double alpha = gamma / pap;
  double beta = alpha * alpha * qdq / gamma - 1.0;
  record(tr_alpha, cap, 0, alpha);
  record(tr_beta, cap, 0, beta);
  for (int32_t i = 1; i <= maxit; ++i) {
    for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k];
    for (int32_t k = 0; k < n; ++k) r[k] -= alpha * ap[k];
    for (int32_t k = 0; k < n; ++k) p[k] = r[k] * dinv[k] + beta * p[k];
    for (int32_t k = 0; k < n; ++k) z[k] = r[k] * dinv[k];
    gamma = orc_dot(n, r, z);                     /* <r_i, M^-1 r_i> */
    rr = orc_dot(n, r, r);                        /* <r_i, r_i> */
    record(tr_res2, cap, i - 1, rr);
    *iters_out = i;
    if (!isfinite(rr) || !isfinite(gamma)) { status = ORC_NAN; break; }
    if (rr <= thr2) { status = ORC_OK; break; }
    if (i == maxit) break;
    orc_spmv(n, rp, ci, va, p, ap);
    for (int32_t k = 0; k < n; ++k) z[k] = ap[k] * dinv[k];
    qdq = orc_dot(n, ap, z);
    pap = orc_dot(n, p, ap);
    if (!finite3(qdq, pap, gamma)) { status = ORC_NAN; break; }
    if (pap <= 0.0) { status = ORC_NOT_SPD; break; }
    alpha = gamma / pap;
    beta = alpha * alpha * qdq / gamma - 1.0;
    record(tr_alpha, cap, i, alpha);
    record(tr_beta, cap, i, beta);
  }
done:
  free(r); free(p); free(ap); free(z); free(dinv);
  return status;
}

/* ---------------------------------------------------------------- right Jacobi preconditioning */

/* Right preconditioning with M = diag(A) (entries of row i in column i summed): a Krylov
 * solver applied to A M^-1 y = b has the residual b - A M^-1 y = b - A x of x = M^-1 y, so
 * its iterates, stopping test and iteration count are those of the preconditioned solve.
 * begin: va_out = the values of A M^-1 (every entry times the reciprocal diagonal entry of
 * its column), dinv_out = M^-1, x <- M x (y0 from x0).  A zero or non-finite diagonal entry
 * leaves everything untouched and returns ERR_ARG. */
int orc_jacobi_right_begin(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                           double* x, double* va_out, double* dinv_out) {
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j)
      if (ci[j] == i) d += va[j];
    if (d == 0.0 || !isfinite(d)) return ORC_ERR_ARG;
    dinv_out[i] = 1.0 / d;
  }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j) va_out[j] = va[j] * dinv_out[ci[j]];
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j)
      if (ci[j] == i) d += va[j];
    x[i] = x[i] * d;
  }
  return ORC_OK;
}

/* end: x = M^-1 y. */
void orc_jacobi_right_end(int32_t n, const double* dinv, double* x) {
  for (int32_t i = 0; i < n; ++i) x[i] = dinv[i] * x[i];
}

/* ---------------------------------------------------------------- BiCGStab, Algorithm 3 */

int orc_bicgstab_classical(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                           const double* b, double* x, double tol, int32_t maxit, int32_t cap,
                           double* tr_alpha, double* tr_beta, double* tr_omega, double* tr_res2,
                           int32_t* iters_out) {
  *iters_out = 0;
  if (n <= 0) return ORC_OK;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double thr2 = tol * tol * bb;
  size_t sz = sizeof(double) * (size_t)n;
  double *r = malloc(sz), *p = malloc(sz), *ap = malloc(sz), *s = malloc(sz), *as = malloc(sz),
         *r0s = malloc(sz);
  if (!r || !p || !ap || !s || !as || !r0s) {
    free(r); free(p); free(ap); free(s); free(as); free(r0s); return ORC_ERR_OOM;
  }
  int status = ORC_NOT_CONVERGED;
  orc_spmv(n, rp, ci, va, x, ap);
  for (int32_t k = 0; k < n; ++k) { r[k] = b[k] - ap[k]; p[k] = r[k]; r0s[k] = r[k]; }
  double rr = orc_dot(n, r, r);
  double rr0s = orc_dot(n, r, r0s);                    /* <r0, r0*> */
  if (!isfinite(rr)) { status = ORC_NAN; goto done; }
  if (rr <= thr2) { status = ORC_OK; goto done; }
  for (int32_t i = 0; i < maxit; ++i) {
    orc_spmv(n, rp, ci, va, p, ap);                    /* A p_i */
    double apr0s = orc_dot(n, ap, r0s);                /* <Ap_i, r0*> */
    if (!isfinite(apr0s)) { status = ORC_NAN; break; }
    if (apr0s == 0.0 || rr0s == 0.0) { status = ORC_BREAKDOWN; break; }
    double alpha = rr0s / apr0s;
    for (int32_t k = 0; k < n; ++k) s[k] = r[k] - alpha * ap[k];
    record(tr_alpha, cap, i, alpha);
    double ss = orc_dot(n, s, s);
    if (!isfinite(ss)) { status = ORC_NAN; break; }
    if (ss <= thr2) {                                  /* early exit on a small s */
      for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k];
      record(tr_res2, cap, i, ss);
      *iters_out = i + 1; status = ORC_OK; break;
    }
    orc_spmv(n, rp, ci, va, s, as);                    /* A s_i */
    double ass = orc_dot(n, as, s);
    double asas = orc_dot(n, as, as);
    if (!finite3(ass, asas, 0.0)) { status = ORC_NAN; break; }
    if (asas == 0.0) { status = ORC_BREAKDOWN; break; }
    double omega = ass / asas;
    record(tr_omega, cap, i, omega);
    for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k] + omega * s[k];
    for (int32_t k = 0; k < n; ++k) r[k] = s[k] - omega * as[k];
    double rr0s_new = orc_dot(n, r, r0s);              /* <r_{i+1}, r0*> */
    if (omega == 0.0) { status = ORC_BREAKDOWN; *iters_out = i + 1; break; }
    double beta = (rr0s_new / rr0s) * (alpha / omega);
    record(tr_beta, cap, i, beta);
    for (int32_t k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * ap[k]);
    rr0s = rr0s_new;
    rr = orc_dot(n, r, r);                             /* explicit residual norm */
    record(tr_res2, cap, i, rr);
    *iters_out = i + 1;
    if (!finite3(rr, beta, rr0s)) { status = ORC_NAN; break; }
    if (rr <= thr2) { status = ORC_OK; break; }
  }
done:
  free(r); free(p); free(ap); free(s); free(as); free(r0s);
  return status;
}

/* ---------------------------------------------------------------- BiCGStab, Algorithm 4 */

int orc_bicgstab_pipelined(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                           const double* b, double* x, double tol, int32_t maxit, int32_t cap,
                           double* tr_alpha, double* tr_beta, double* tr_omega, double* tr_res2,
                           double* tr_res2_est, int32_t* iters_out) {
  *iters_out = 0;
  if (n <= 0) return ORC_OK;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double thr2 = tol * tol * bb;
  size_t sz = sizeof(double) * (size_t)n;
  double *r = malloc(sz), *p = malloc(sz), *ap = malloc(sz), *s = malloc(sz), *as = malloc(sz),
         *r0s = malloc(sz);
  if (!r || !p || !ap || !s || !as || !r0s) {
    free(r); free(p); free(ap); free(s); free(as); free(r0s); return ORC_ERR_OOM;
  }
  int status = ORC_NOT_CONVERGED;
  orc_spmv(n, rp, ci, va, x, ap);
  for (int32_t k = 0; k < n; ++k) { r[k] = b[k] - ap[k]; p[k] = r[k]; r0s[k] = r[k]; }
  double rr = orc_dot(n, r, r);
  double rr0s = orc_dot(n, r, r0s);
  if (!isfinite(rr)) { status = ORC_NAN; goto done; }
  if (rr <= thr2) { status = ORC_OK; goto done; }
  for (int32_t i = 0; i < maxit; ++i) {
    /* A p_i and <Ap_i, r0*> -> alpha_i */
    orc_spmv(n, rp, ci, va, p, ap);
    double apr0s = orc_dot(n, ap, r0s);
    if (!isfinite(apr0s)) { status = ORC_NAN; break; }
    if (apr0s == 0.0 || rr0s == 0.0) { status = ORC_BREAKDOWN; break; }
    double alpha = rr0s / apr0s;
    record(tr_alpha, cap, i, alpha);
    /* s_i = r_i - alpha_i A p_i and <s_i, s_i> */
    for (int32_t k = 0; k < n; ++k) s[k] = r[k] - alpha * ap[k];
    double ss = orc_dot(n, s, s);
    if (!isfinite(ss)) { status = ORC_NAN; break; }
    if (ss <= thr2) {
      for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k];
      record(tr_res2, cap, i, ss);
      *iters_out = i + 1; status = ORC_OK; break;
    }
    /* A s_i and <As_i, s_i>, <As_i, As_i>, <As_i, r0*> -> omega_i, beta_i */
    orc_spmv(n, rp, ci, va, s, as);
    double ass = orc_dot(n, as, s);
    double asas = orc_dot(n, as, as);
    double asr0s = orc_dot(n, as, r0s);
    if (!finite3(ass, asas, asr0s)) { status = ORC_NAN; break; }
    if (asas == 0.0) { status = ORC_BREAKDOWN; break; }
    double beta = -asr0s / apr0s;
    double omega = ass / asas;
    double est = ss - 2.0 * omega * ass + omega * omega * asas;   /* Sec. 3.2 expansion */
    if (est < 0.0) est = 0.0;
    record(tr_beta, cap, i, beta);
    record(tr_omega, cap, i, omega);
    record(tr_res2_est, cap, i, est);
    /* x_{i+1}, r_{i+1}, p_{i+1} and <r_{i+1}, r0*> (plus <r_{i+1}, r_{i+1}> for the test) */
    for (int32_t k = 0; k < n; ++k) x[k] += alpha * p[k] + omega * s[k];
    for (int32_t k = 0; k < n; ++k) r[k] = s[k] - omega * as[k];
    for (int32_t k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * ap[k]);
    rr0s = orc_dot(n, r, r0s);
    rr = orc_dot(n, r, r);
    record(tr_res2, cap, i, rr);
    *iters_out = i + 1;
    if (!finite3(rr, rr0s, omega)) { status = ORC_NAN; break; }
    if (rr <= thr2) { status = ORC_OK; break; }
  }
done:
  free(r); free(p); free(ap); free(s); free(as); free(r0s);
  return status;
}

/* ---------------------------------------------------------------- GMRES(m), Alg. 5 / 6 */

/*
 * pipelined = 1: Algorithm 6 (xi_i = <v_0, v_i>, no residual update);
 * pipelined = 0: Algorithm 5 (xi_i = <r, v_i>, r <- r - xi_i v_i, monitor rho0 ||r||).
 * tr_R (m*m, row-major R[j-1][i-1]) and tr_xi (m) receive the first cycle's values;
 * tr_est (cap) the per-step residual estimate; tr_res (cap) the true residual norm at
 * every cycle boundary (index = cycle).
 */
static int gmres_run(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                     const double* b, double* x, double tol, int32_t maxit, int32_t m, int32_t pipelined,
                     int32_t cgs2, int32_t cap, double* tr_R, double* tr_xi, double* tr_est,
                     double* tr_res, double* tr_V, int32_t* iters_out, int32_t* cycles_out);

int orc_gmres(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
              const double* b, double* x, double tol, int32_t maxit, int32_t m, int32_t pipelined,
              int32_t cap, double* tr_R, double* tr_xi, double* tr_est, double* tr_res,
              int32_t* iters_out, int32_t* cycles_out) {
  return gmres_run(n, rp, ci, va, b, x, tol, maxit, m, pipelined, 0, cap, tr_R, tr_xi, tr_est, tr_res,
                   NULL, iters_out, cycles_out);
}

/* The same GMRES with classical Gram-Schmidt applied twice per step (CGS2, "twice is
 * enough": Giraud, Langou, Rozloznik, Comput. Math. Appl. 50, 2005): after v_i -= sum_j
 * R_{j,i} v_j, the coefficients c_j = <v_j, v_i> (j = 1 .. i-1) are computed again, v_i -=
 * sum_j c_j v_j, and R_{j,i} += c_j; the norm, R_{i,i} and the breakdown test follow the
 * second pass.  tr_V (optional, n x (m+1), vector after vector) receives the first cycle's
 * basis v_0 .. v_m. */
int orc_gmres_cgs2(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                   const double* b, double* x, double tol, int32_t maxit, int32_t m, int32_t pipelined,
                   int32_t cap, double* tr_R, double* tr_xi, double* tr_est, double* tr_res,
                   int32_t* iters_out, int32_t* cycles_out, double* tr_V) {
  return gmres_run(n, rp, ci, va, b, x, tol, maxit, m, pipelined, 1, cap, tr_R, tr_xi, tr_est, tr_res,
                   tr_V, iters_out, cycles_out);
}

static int gmres_run(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                     const double* b, double* x, double tol, int32_t maxit, int32_t m, int32_t pipelined,
                     int32_t cgs2, int32_t cap, double* tr_R, double* tr_xi, double* tr_est,
                     double* tr_res, double* tr_V, int32_t* iters_out, int32_t* cycles_out) {
  *iters_out = 0;
  if (cycles_out) *cycles_out = 0;
  if (n <= 0) return ORC_OK;
  if (m < 1) return ORC_ERR_ARG;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double bnorm = sqrt(bb);
  size_t sz = sizeof(double) * (size_t)n;
  double* V = malloc(sz * (size_t)(m + 1));          /* v_0 .. v_m, each length n */
  double* r = malloc(sz);
  double* acc = malloc(sz);
  double* R = calloc((size_t)(m + 1) * (size_t)(m + 1), sizeof(double)); /* R[j][i], 1-based */
  double* xi = calloc((size_t)(m + 1), sizeof(double));
  double* eta = calloc((size_t)(m + 1), sizeof(double));
  double* c2 = calloc((size_t)(m + 1), sizeof(double));
  if (!V || !r || !acc || !R || !xi || !eta || !c2) {
    free(V); free(r); free(acc); free(R); free(xi); free(eta); free(c2); return ORC_ERR_OOM;
  }
#define VEC(i) (V + (size_t)(i) * (size_t)n)
#define RR(j, i) R[(size_t)(j) * (size_t)(m + 1) + (size_t)(i)]
  int status = ORC_NOT_CONVERGED;
  int32_t total = 0, cycle = 0, est_k = 0;
  for (;;) {
    /* r0 = b - A x0, rho0 = ||r0|| (true residual at the cycle boundary) */
    orc_spmv(n, rp, ci, va, x, r);
    for (int32_t k = 0; k < n; ++k) r[k] = b[k] - r[k];
    double rho0 = sqrt(orc_dot(n, r, r));
    record(tr_res, cap, cycle, rho0);
    if (!isfinite(rho0)) { status = ORC_NAN; break; }
    if (rho0 <= tol * bnorm) { status = ORC_OK; break; }
    if (total >= maxit) { status = ORC_NOT_CONVERGED; break; }
    /* v_0 = r = r0 / rho0 */
    for (int32_t k = 0; k < n; ++k) { VEC(0)[k] = r[k] / rho0; r[k] = VEC(0)[k]; }
    memset(R, 0, sizeof(double) * (size_t)(m + 1) * (size_t)(m + 1));
    double sumxi2 = 0.0;
    int32_t kdone = 0;
    int broke = 0;
    for (int32_t i = 1; i <= m; ++i) {
      if (total >= maxit) break;
      double* vi = VEC(i);
      orc_spmv(n, rp, ci, va, VEC(i - 1), vi);         /* v_i = A v_{i-1} */
      for (int32_t j = 1; j <= i - 1; ++j) RR(j, i) = orc_dot(n, VEC(j), vi); /* CGS */
      for (int32_t j = 1; j <= i - 1; ++j) {
        double rji = RR(j, i);
        const double* vj = VEC(j);
        for (int32_t k = 0; k < n; ++k) vi[k] -= rji * vj[k];
      }
      if (cgs2) {                                       /* second pass (CGS2) */
        for (int32_t j = 1; j <= i - 1; ++j) c2[j] = orc_dot(n, VEC(j), vi);
        for (int32_t j = 1; j <= i - 1; ++j) {
          const double* vj = VEC(j);
          for (int32_t k = 0; k < n; ++k) vi[k] -= c2[j] * vj[k];
        }
        for (int32_t j = 1; j <= i - 1; ++j) RR(j, i) += c2[j];
      }
      double nrm2 = orc_dot(n, vi, vi);
      double rii = sqrt(nrm2);
      double col2 = nrm2;                               /* ||A v_{i-1}||^2 = sum R_{j,i}^2 */
      for (int32_t j = 1; j <= i - 1; ++j) col2 += RR(j, i) * RR(j, i);
      if (!isfinite(rii)) { status = ORC_NAN; broke = 2; break; }
      if (rii == 0.0 || rii <= 1e-14 * sqrt(col2)) { broke = 1; break; }  /* lucky breakdown */
      RR(i, i) = rii;
      for (int32_t k = 0; k < n; ++k) vi[k] /= rii;
      double xii;
      if (pipelined) {
        xii = orc_dot(n, VEC(0), vi);                   /* xi_i = <v_0, v_i> */
      } else {
        xii = orc_dot(n, r, vi);                        /* xi_i = <r, v_i> */
        for (int32_t k = 0; k < n; ++k) r[k] -= xii * vi[k];
      }
      xi[i] = xii;
      total++;
      kdone = i;
      double rel2;
      if (pipelined) {
        sumxi2 += xii * xii;
        rel2 = 1.0 - sumxi2;
      } else {
        rel2 = orc_dot(n, r, r);
      }
      if (rel2 < 0.0) rel2 = 0.0;
      double est = rho0 * sqrt(rel2);
      record(tr_est, cap, est_k++, est);
      if (est <= tol * bnorm || rel2 <= 1e-12) break;
    }
    if (cycle == 0) {
      if (tr_R)
        for (int32_t j = 1; j <= m; ++j)
          for (int32_t i = 1; i <= m; ++i) tr_R[(size_t)(j - 1) * m + (i - 1)] = RR(j, i);
      if (tr_xi)
        for (int32_t i = 1; i <= m; ++i) tr_xi[i - 1] = xi[i];
      if (tr_V) memcpy(tr_V, V, sz * (size_t)(kdone + 1));
    }
    if (broke == 2) break;
    if (kdone == 0) { status = ORC_BREAKDOWN; break; }
    /* solve R eta = xi (upper triangular, k x k) by back-substitution */
    for (int32_t i = kdone; i >= 1; --i) {
      double s = xi[i];
      for (int32_t j = i + 1; j <= kdone; ++j) s -= RR(i, j) * eta[j];
      eta[i] = s / RR(i, i);
    }
    /* x <- x0 + rho0 (eta_1 v_0 + sum_{i=2..k} eta_i v_{i-1}) */
    for (int32_t k = 0; k < n; ++k) {
      double a = 0.0;
      for (int32_t i = 1; i <= kdone; ++i) a += eta[i] * VEC(i - 1)[k];
      x[k] += rho0 * a;
    }
    cycle++;
    (void)broke;
  }
#undef VEC
#undef RR
  *iters_out = total;
  if (cycles_out) *cycles_out = cycle;
  free(V); free(r); free(acc); free(R); free(xi); free(eta); free(c2);
  return status;
}

/* ---------------------------------------------------------------- GMRES(m), three-kernel form */

/*
 * The shift-invariant variant of the pipelined GMRES(m) that Sec. 3.3 names as the way to
 * drop the normalisation kernel.  For i >= 2, v_{i-1} is in span{v_1 .. v_{i-1}}, so
 * A v_{i-1} and w = (A - sigma I) v_{i-1} have the same part orthogonal to that span for every
 * shift sigma (the Krylov space does not change under a shift), and the norm of that part,
 * R_{i,i}, follows from inner products the step already forms (v_1 .. v_{i-1} orthonormal,
 * Pythagoras applied to w):
 *     y = A v_{i-1},  R_{j,i} = <v_j, y> (j = 1 .. i-1),  nu = <w, w> = ||y - sigma v_{i-1}||^2,
 *     R_{i,i}^2 = nu - sum_{j < i-1} R_{j,i}^2 - (R_{i-1,i} - sigma)^2,
 *     v_i = (y - sum_j R_{j,i} v_j) / R_{i,i}.
 * R, xi, eta and x are those of Algorithm 6; only R_{i,i} comes from the identity instead of
 * a separate norm.  The shift reduces the cancellation in the difference: the paper gives
 * none, and the reading here needs no extra inner product: sigma_1 = 0 (v_0 is not in the
 * span) and sigma_{i+1} = <v_{i-1}, A v_{i-1}>, the Rayleigh quotient of the previous basis
 * vector, which step i forms anyway (it is R_{i-1,i} for i >= 2, and <v_0, A v_0> for i = 1).  The difference is only trusted while R_{i,i}^2 > 1e-8 nu
 * (below, its rounding error is a visible fraction of it): otherwise the cycle ends before
 * step i, as in a lucky breakdown.  Everything else (xi_i = <v_0, v_i>, the estimate, the end
 * of a cycle, the update, the restart from the true residual) is Algorithm 6 as in orc_gmres.
 */
int orc_gmres_shift3(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                     const double* b, double* x, double tol, int32_t maxit, int32_t m, int32_t cap,
                     double* tr_R, double* tr_xi, double* tr_est, double* tr_res, double* tr_sigma,
                     int32_t* iters_out, int32_t* cycles_out) {
  *iters_out = 0;
  if (cycles_out) *cycles_out = 0;
  if (n <= 0) return ORC_OK;
  if (m < 1) return ORC_ERR_ARG;
  double bb = orc_dot(n, b, b);
  if (bb == 0.0) { memset(x, 0, sizeof(double) * (size_t)n); return ORC_OK; }
  double bnorm = sqrt(bb);
  size_t sz = sizeof(double) * (size_t)n;
  double* V = malloc(sz * (size_t)(m + 1));          /* v_0 .. v_m */
  double* r = malloc(sz);
  double* acc = malloc(sz);                           /* w = (A - sigma I) v_{i-1} */
  double* R = calloc((size_t)(m + 1) * (size_t)(m + 1), sizeof(double)); /* R[j][i] */
  double* xi = calloc((size_t)(m + 1), sizeof(double));
  double* eta = calloc((size_t)(m + 1), sizeof(double));
  if (!V || !r || !acc || !R || !xi || !eta) {
    free(V); free(r); free(acc); free(R); free(xi); free(eta); return ORC_ERR_OOM;
  }
#define VEC(i) (V + (size_t)(i) * (size_t)n)
#define RR(j, i) R[(size_t)(j) * (size_t)(m + 1) + (size_t)(i)]
  int status = ORC_NOT_CONVERGED;
  int32_t total = 0, cycle = 0, est_k = 0;
  for (;;) {
    orc_spmv(n, rp, ci, va, x, r);                    /* r0 = b - A x0 */
    for (int32_t k = 0; k < n; ++k) r[k] = b[k] - r[k];
    double rho0 = sqrt(orc_dot(n, r, r));
    record(tr_res, cap, cycle, rho0);
    if (!isfinite(rho0)) { status = ORC_NAN; break; }
    if (rho0 <= tol * bnorm) { status = ORC_OK; break; }
    if (total >= maxit) { status = ORC_NOT_CONVERGED; break; }
    for (int32_t k = 0; k < n; ++k) VEC(0)[k] = r[k] / rho0;
    memset(R, 0, sizeof(double) * (size_t)(m + 1) * (size_t)(m + 1));
    double sumxi2 = 0.0, sigma = 0.0;
    int32_t kdone = 0;
    int broke = 0;
    for (int32_t i = 1; i <= m; ++i) {
      if (total >= maxit) break;
      double* vi = VEC(i);
      const double* vp = VEC(i - 1);
      orc_spmv(n, rp, ci, va, vp, vi);                 /* y = A v_{i-1} */
      for (int32_t k = 0; k < n; ++k) acc[k] = vi[k] - sigma * vp[k];  /* w = y - sigma v_{i-1} */
      double nu = orc_dot(n, acc, acc);                /* <w, w> */
      double rq = orc_dot(n, vp, vi);                  /* <v_{i-1}, A v_{i-1}> */
      double sum2 = 0.0;
      for (int32_t j = 1; j <= i - 1; ++j) {           /* R_{j,i} = <v_j, y> (CGS) */
        RR(j, i) = orc_dot(n, VEC(j), vi);
        double c = j == i - 1 ? RR(j, i) - sigma : RR(j, i);  /* <v_j, w> */
        sum2 += c * c;
      }
      double rii2 = nu - sum2;
      if (!isfinite(rii2)) { status = ORC_NAN; broke = 2; break; }
      if (!(rii2 > 1e-8 * nu)) { broke = 1; break; }  /* the identity is not trusted: end */
      double rii = sqrt(rii2);
      for (int32_t j = 1; j <= i - 1; ++j) {
        double rji = RR(j, i);
        const double* vj = VEC(j);
        for (int32_t k = 0; k < n; ++k) vi[k] -= rji * vj[k];
      }
      for (int32_t k = 0; k < n; ++k) vi[k] /= rii;
      RR(i, i) = rii;
      record(tr_sigma, cap, total, sigma);
      sigma = rq;                                      /* sigma_{i+1} */
      double xii = orc_dot(n, VEC(0), vi);             /* xi_i = <v_0, v_i> */
      xi[i] = xii;
      total++;
      kdone = i;
      sumxi2 += xii * xii;
      double rel2 = 1.0 - sumxi2;
      if (rel2 < 0.0) rel2 = 0.0;
      double est = rho0 * sqrt(rel2);
      record(tr_est, cap, est_k++, est);
      if (est <= tol * bnorm || rel2 <= 1e-12) break;
    }
    if (cycle == 0) {
      if (tr_R)
        for (int32_t j = 1; j <= m; ++j)
          for (int32_t i = 1; i <= m; ++i) tr_R[(size_t)(j - 1) * m + (i - 1)] = RR(j, i);
      if (tr_xi)
        for (int32_t i = 1; i <= m; ++i) tr_xi[i - 1] = xi[i];
    }
    if (broke == 2) break;
    if (kdone == 0) { status = ORC_BREAKDOWN; break; }
    for (int32_t i = kdone; i >= 1; --i) {             /* R eta = xi */
      double s = xi[i];
      for (int32_t j = i + 1; j <= kdone; ++j) s -= RR(i, j) * eta[j];
      eta[i] = s / RR(i, i);
    }
    for (int32_t k = 0; k < n; ++k) {                  /* x += rho0 (eta_1 v_0 + ...) */
      double a = 0.0;
      for (int32_t i = 1; i <= kdone; ++i) a += eta[i] * VEC(i - 1)[k];
      x[k] += rho0 * a;
    }
    cycle++;
  }
#undef VEC
#undef RR
  *iters_out = total;
  if (cycles_out) *cycles_out = cycle;
  free(V); free(r); free(acc); free(R); free(xi); free(eta);
  return status;
}
