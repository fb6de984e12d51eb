// Conjugate gradients: pipelined (Alg. 2) with two fused kernels per iteration, the split
// variant (three kernels), and classical CG (Alg. 1) as six kernels per iteration.
//
// Pipelined iteration i (Sec. 3.1):
//   K-CG-U  x_i = x_{i-1} + alpha p_{i-1};  r_i = r_{i-1} - alpha A p_{i-1};
//           p_i = r_i + beta p_{i-1};  first stage of <r_i, r_i>.
//           Last block: <r_i, r_i>, convergence test (||r_i|| <= tol ||b||), maxit.
//   K-CG-S  A p_i fused with the first stage of <Ap_i, Ap_i> and <p_i, Ap_i>.
//           Last block: alpha_i = <r_i,r_i>/<p_i,Ap_i>,
//                       beta_i  = alpha_i^2 <Ap_i,Ap_i>/<r_i,r_i> - 1   (Eq. (3)).
// Every vector is read once and written once per kernel: K-CG-U moves 56 bytes per row,
// K-CG-S 12 bytes per nonzero + 20 bytes per row.
#include <algorithm>
#include <cmath>

#include "pk_tile.cuh"

namespace pk {

// r = b - A x, p = r; first stage of <r, r> and <b, b>.  Last block: rr, bb, thr2, and the
// zero-iteration exits (b = 0 -> x = 0; ||r0|| <= tol ||b||).
__global__ void __launch_bounds__(kBlock) k_residual_init(RowArgs a, const double* __restrict__ b,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ r,
                                                          double* __restrict__ p,
                                                          double* __restrict__ r0s) {
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[2] = {0.0, 0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double bi = b[row];
    const double ri = bi - csr_row(a, x, row);
    r[row] = ri;
    if (p) p[row] = ri;
    if (r0s) r0s[row] = ri;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(bi, bi, v[1]);
  }
  block_partials<2>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      DevState* st = a.st;
      const double tol = st->thr2;
      st->rr = t[0];
      st->bb = t[1];
      st->thr2 = tol * tol * t[1];
      st->iter = 0;
      if (r0s) st->s[0] = t[0];  // BiCGStab: <r0, r0*> with r0* = r0
      if (!isfinite(t[0]) || !isfinite(t[1])) {
        finish(st, PK_ERR_NAN);
      } else if (t[1] == 0.0) {
        st->zero_x = 1;
        st->rr = 0.0;
        finish(st, PK_OK);
      } else if (t[0] <= st->thr2) {
        finish(st, PK_OK);
      } else if (st->maxit <= 0) {
        finish(st, PK_NOT_CONVERGED);
      }
      st->counter = 0;
    }
  }
}

// x = 0 when b = 0 (flag set by k_residual_init).
__global__ void __launch_bounds__(kBlock) k_zero_x(RowArgs a, double* __restrict__ x) {
  if (!__ldcg(&a.st->zero_x)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) x[row] = 0.0;
}

// Second stage shared by K-CG-S and the split dots kernel: alpha_i and beta_i (Eq. (3)).
__device__ __forceinline__ void cg_alpha_beta(DevState* st, double apap, double pap) {
  const double rr = st->rr;
  const int i = st->iter;
  if (!isfinite(apap) || !isfinite(pap)) {
    finish(st, PK_ERR_NAN);
  } else if (pap <= 0.0) {
    finish(st, PK_NOT_SPD);
  } else {
    const double alpha = rr / pap;
    const double beta = alpha * alpha * apap / rr - 1.0;
    st->alpha = alpha;
    st->beta = beta;
    trace_put(st, i, 0, alpha);
    trace_put(st, i, 1, beta);
  }
}

// K-CG-S: Ap = A p with the first stage of <Ap, Ap> and <p, Ap> (Sec. 3.1, Alg. 2).
__global__ void __launch_bounds__(kBlock, 8) k_cg_spmv_dots(RowArgs a, const double* __restrict__ p,
                                                         double* __restrict__ ap) {
  if (state_done(a.st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[2] = {0.0, 0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double s = csr_row(a, p, row);
    ap[row] = s;
    v[0] = fma(s, s, v[0]);
    v[1] = fma(__ldg(p + row), s, v[1]);
  }
  block_partials<2>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      cg_alpha_beta(a.st, t[0], t[1]);
      a.st->counter = 0;
    }
  }
}

// Split variant: <Ap, Ap> and <p, Ap> in their own kernel after a plain SpMV.
__global__ void __launch_bounds__(kBlock) k_cg_dots(RowArgs a, const double* __restrict__ p,
                                                    const double* __restrict__ ap) {
  if (state_done(a.st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[2] = {0.0, 0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double s = ap[row];
    v[0] = fma(s, s, v[0]);
    v[1] = fma(p[row], s, v[1]);
  }
  block_partials<2>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      cg_alpha_beta(a.st, t[0], t[1]);
      a.st->counter = 0;
    }
  }
}

// Plain SpMV that honours the done flag (split and classical loops).
__global__ void __launch_bounds__(kBlock) k_spmv_live(RowArgs a, const double* __restrict__ x,
                                                      double* __restrict__ y, int first) {
  if (first) count_pass(a.st);
  if (state_done(a.st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) y[row] = csr_row(a, x, row);
}

// K-CG-U: x, r, p updates with the first stage of <r_i, r_i> (Sec. 3.1).
__global__ void __launch_bounds__(kBlock) k_cg_update(RowArgs a, double* __restrict__ x,
                                                      double* __restrict__ r,
                                                      double* __restrict__ p,
                                                      const double* __restrict__ ap) {
  DevState* st = a.st;
  count_pass(st);
  if (state_done(st)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(st->cond, 0u);
    return;
  }
  const double alpha = __ldcg(&st->alpha), beta = __ldcg(&st->beta);
  int r0, r1;
  ew_range(a.n, r0, r1);
  double v[1] = {0.0};
  // two rows per thread with 16-byte accesses (block ranges start on a multiple of 32 rows)
  const int pairs = (r1 - r0) >> 1;
  for (int k = threadIdx.x; k < pairs; k += blockDim.x) {
    const int row = r0 + 2 * k;
    const double2 pk = ld2(p + row), xk = ld2(x + row), ak = ld2(ap + row), rk0 = ld2(r + row);
    double2 rk, xn, pn;
    xn.x = fma(alpha, pk.x, xk.x);
    xn.y = fma(alpha, pk.y, xk.y);
    rk.x = fma(-alpha, ak.x, rk0.x);
    rk.y = fma(-alpha, ak.y, rk0.y);
    pn.x = fma(beta, pk.x, rk.x);
    pn.y = fma(beta, pk.y, rk.y);
    st2(x + row, xn);
    st2(r + row, rk);
    st2(p + row, pn);
    v[0] = fma(rk.x, rk.x, v[0]);
    v[0] = fma(rk.y, rk.y, v[0]);
  }
  if (((r1 - r0) & 1) && threadIdx.x == 0) {
    const int row = r1 - 1;
    const double pk = p[row];
    x[row] = fma(alpha, pk, x[row]);
    const double rk = fma(-alpha, ap[row], r[row]);
    r[row] = rk;
    p[row] = fma(beta, pk, rk);
    v[0] = fma(rk, rk, v[0]);
  }
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter + 1;
      st->iter = i;
      st->rr = t[0];
      trace_put(st, i - 1, 3, t[0]);
      if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] <= st->thr2) finish(st, PK_OK);
      else if (i >= st->maxit) finish(st, PK_NOT_CONVERGED);
      st->counter = 0;
    }
  }
}

// ---------------------------------------------------------------- warp-specialised forms

// K-CG-U on the streaming tile engine: inputs p, x, Ap, r arrive in shared memory through
// bulk copies; results are stored straight to global memory.
__global__ void __launch_bounds__(kTileThreads, 2) k_cg_update_tma(int n, double* __restrict__ x,
                                                                   double* __restrict__ r,
                                                                   double* __restrict__ p,
                                                                   const double* __restrict__ ap,
                                                                   double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  count_pass(st);
  int r0, r1;
  ew_range(n, r0, r1);
  double v[1] = {0.0};
  double alpha = 0.0, beta = 0.0;
  // x and r do not depend on the preceding K-CG-S: prefetched before the dependency wait
  StreamIn<4> in{{x, r, p, ap}};
  const bool live = stream_tiles<4, 2, double, 2>(in, r0, r1, smem, st, [&]() {
    alpha = __ldcg(&st->alpha);
    beta = __ldcg(&st->beta);
    return !state_done(st);
  }, [&](int row, const double2* val, int nv) {
    const double2 xk = val[0], rq = val[1], pk = val[2], ak = val[3];
    double2 xn, rn, pn;
    xn.x = fma(alpha, pk.x, xk.x);
    xn.y = fma(alpha, pk.y, xk.y);
    rn.x = fma(-alpha, ak.x, rq.x);
    rn.y = fma(-alpha, ak.y, rq.y);
    pn.x = fma(beta, pk.x, rn.x);
    pn.y = fma(beta, pk.y, rn.y);
    if (nv == 2) {
      st2(x + row, xn);
      st2(r + row, rn);
      st2(p + row, pn);
      v[0] = fma(rn.x, rn.x, v[0]);
      v[0] = fma(rn.y, rn.y, v[0]);
    } else {
      x[row] = xn.x;
      r[row] = rn.x;
      p[row] = pn.x;
      v[0] = fma(rn.x, rn.x, v[0]);
    }
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) {
    // the solve had finished before this launch: only clear the loop condition
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(st->cond, 0u);
    return;
  }
  tile_block_partials<1>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter + 1;
      st->iter = i;
      st->rr = t[0];
      trace_put(st, i - 1, 3, t[0]);
      if (__ldcg(&st->timeout)) finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] <= st->thr2) finish(st, PK_OK);
      else if (i >= st->maxit) finish(st, PK_NOT_CONVERGED);
      st->counter = 0;
    }
  }
}

// K-CG-S on the CSR tile engine.
template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_cg_spmv_dots_tma(CsrTiles T,
                                                                      const double* __restrict__ p,
                                                                      double* __restrict__ ap,
                                                                      double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  double v[2] = {0.0, 0.0};
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return !state_done(st); }, p,
                              [&](int row, double y) {
    ap[row] = y;
    v[0] = fma(y, y, v[0]);
    v[1] = fma(__ldg(p + row), y, v[1]);
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<2>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(partials, t);
    if (threadIdx.x == 0) {
      if (__ldcg(&st->timeout)) finish(st, PK_TIMEOUT);
      else cg_alpha_beta(st, t[0], t[1]);
      st->counter = 0;
    }
  }
}

// K-CG-S on the SELL-C-sigma copy (PK_FLAG_SELL): warp per slice, lane per row, Ap with the
// first stage of <Ap, Ap> and <p, Ap>; alpha, beta in the last block.  Launched with
// programmatic dependent launch after K-CG-U: nothing is read before the dependency wait.
__global__ void __launch_bounds__(kBlock) k_cg_sell_spmv_dots(SellArgs s, const double* __restrict__ p,
                                                              double* __restrict__ ap, double* partials,
                                                              DevState* st) {
  griddep_wait();
  if (state_done(st)) return;  // uniform in the grid
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[2] = {0.0, 0.0};
  for (int sl = blockIdx.x * kSellWarps + warp; sl < s.nslices; sl += gridDim.x * kSellWarps) {
    const int64_t base = s.ptr[sl];
    const int w = (int)((s.ptr[sl + 1] - base) / kSellC);
    const int row = s.perm[(size_t)sl * kSellC + lane];
    const double y = sell_row(s, base + lane, w, p);
    if (row >= 0) {
      ap[row] = y;
      v[0] = fma(y, y, v[0]);
      v[1] = fma(__ldg(p + row), y, v[1]);
    }
  }
  griddep_trigger();
  block_partials<2>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(partials, t);
    if (threadIdx.x == 0) {
      cg_alpha_beta(st, t[0], t[1]);
      st->counter = 0;
    }
  }
}

// Plain y = A x on the CSR tile engine, no inner products: the SpMV of the unfused forms
// (classical and split CG, classical BiCGStab), so that fused and unfused solvers differ only
// in the fusion.  `first` counts a loop pass; `skip_early`: BiCGStab's early-exit flag also
// ends the solve.
template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_spmv_tma(CsrTiles T, const double* __restrict__ x,
                                                              double* __restrict__ y, DevState* st,
                                                              int first, int skip_early) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (first) count_pass(st);
  csr_tiles<IRR>(T, smem, st, [&]() { return !state_done(st) && !(skip_early && __ldcg(&st->early)); }, x,
            [&](int row, double v) { y[row] = v; });
}

static pk_status tma_setup() {
  static bool done = false;
  if (!done) {
    PK_CUDA(cudaFuncSetAttribute(k_cg_update_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 stream_smem_bytes<4, double, 2>()));
    for (auto k : {k_cg_spmv_dots_tma<false>, k_cg_spmv_dots_tma<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem_bytes()));
    for (auto k : {k_spmv_tma<false>, k_spmv_tma<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem_bytes()));
    done = true;
  }
  return PK_OK;
}

// ---------------------------------------------------------------- classical CG, Alg. 1

// <p, Ap> -> alpha_i = <r_i,r_i>/<p_i,Ap_i>.
__global__ void __launch_bounds__(kBlock) k_cls_alpha(RowArgs a, const double* __restrict__ p,
                                                      const double* __restrict__ ap) {
  DevState* st = a.st;
  if (state_done(st)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(st->cond, 0u);
    return;
  }
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(p[row], ap[row], v[0]);
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] <= 0.0) finish(st, PK_NOT_SPD);
      else {
        st->alpha = st->rr / t[0];
        trace_put(st, st->iter, 0, st->alpha);
      }
      st->counter = 0;
    }
  }
}

// y += sign * alpha x  (x_{i+1} = x_i + alpha p_i  or  r_{i+1} = r_i - alpha A p_i).
__global__ void __launch_bounds__(kBlock) k_axpy_alpha(RowArgs a, double* __restrict__ y,
                                                       const double* __restrict__ x, double sign) {
  if (state_done(a.st)) return;
  const double alpha = sign * __ldcg(&a.st->alpha);
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) y[row] = fma(alpha, x[row], y[row]);
}

// <r_{i+1}, r_{i+1}> -> convergence test, beta_i = <r_{i+1},r_{i+1}>/<r_i,r_i>.
__global__ void __launch_bounds__(kBlock) k_cls_beta(RowArgs a, const double* __restrict__ r) {
  DevState* st = a.st;
  if (state_done(st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double rk = r[row];
    v[0] = fma(rk, rk, v[0]);
  }
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter;
      st->iter = i + 1;
      trace_put(st, i, 3, t[0]);
      if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] <= st->thr2) finish(st, PK_OK);
      else if (i + 1 >= st->maxit) finish(st, PK_NOT_CONVERGED);
      else {
        st->beta = t[0] / st->rr;
        trace_put(st, i, 1, st->beta);
      }
      st->rr = t[0];
      st->counter = 0;
    }
  }
}

// p_{i+1} = r_{i+1} + beta_i p_i.
__global__ void __launch_bounds__(kBlock) k_xpay_beta(RowArgs a, const double* __restrict__ r,
                                                      double* __restrict__ p) {
  if (state_done(a.st)) return;
  const double beta = __ldcg(&a.st->beta);
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) p[row] = fma(beta, p[row], r[row]);
}

pk_status cg_mixed(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                   cudaStream_t s);
bool persistent_usable(const pk_csr* A, const pk_opts* o);
pk_status pcg_jacobi_solve(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                           cudaStream_t s);
pk_status launch_cg_persistent(pk_csr* A, double* x, double* r, double* p, double* ap,
                               cudaStream_t s);
pk_status resident_prepare(pk_csr* A, cudaStream_t s, bool* usable);
pk_status launch_cg_resident(pk_csr* A, double* x, double* r, double* p, double* ap, cudaStream_t s);

pk_status cg_solve(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                   cudaStream_t s) {
  pk_status e = check_opts(A, b, x, o, info);
  if (e) return e;
  *info = pk_info{};
  info->rel_res_true = -1.0;
  if (A->n == 0) return PK_OK;
  if (o->flags & PK_FLAG_CGS2) { set_error("PK_FLAG_CGS2 applies to GMRES"); return PK_ERR_ARG; }
  const bool sell = (o->flags & PK_FLAG_SELL) != 0;
  if (sell && (o->precond != PK_PRECOND_NONE || o->precision != PK_PREC_FP64 ||
               o->variant != PK_VARIANT_PIPELINED || o->loop == PK_LOOP_PERSISTENT)) {
    set_error("PK_FLAG_SELL runs pipelined FP64 CG without preconditioner on the graph or host loop");
    return PK_ERR_ARG;
  }
  if (o->precond == PK_PRECOND_JACOBI) return pcg_jacobi_solve(A, b, x, o, info, s);
  if (o->precond != PK_PRECOND_NONE) { set_error("bad precond"); return PK_ERR_ARG; }
  if (o->precision == PK_PREC_MIXED) return cg_mixed(A, b, x, o, info, s);
  if (o->precision != PK_PREC_FP64) { set_error("precision must be PK_PREC_FP64 or PK_PREC_MIXED"); return PK_ERR_ARG; }
  if (o->variant < 0 || o->variant > 2) { set_error("bad variant"); return PK_ERR_ARG; }
  bool persistent = false;
  if (o->loop == PK_LOOP_PERSISTENT) {
    if (o->variant != PK_VARIANT_PIPELINED) {
      set_error("PK_LOOP_PERSISTENT runs pipelined CG only");
      return PK_ERR_ARG;
    }
    if (!persistent_usable(A, o)) {
      set_error("PK_LOOP_PERSISTENT: persistent loop needs n <= 16 x 4096 rows (one thread-block cluster) and cluster launch");
      return PK_ERR_ARG;
    }
    persistent = true;
  } else if (o->loop == PK_LOOP_AUTO && !sell) {
    persistent = o->variant == PK_VARIANT_PIPELINED && A->n <= PK_PERSISTENT_AUTO_N &&
                 A->nnz <= PK_PERSISTENT_AUTO_NNZ &&
                 !(o->flags & PK_FLAG_TIMING) && persistent_usable(A, o);
  }
  bool resident = false;
  if (o->loop == PK_LOOP_RESIDENT) {
    if (o->variant != PK_VARIANT_PIPELINED || sell || (o->flags & PK_FLAG_NO_TMA)) {
      set_error("PK_LOOP_RESIDENT runs pipelined CG on the CSR tiles (no PK_FLAG_SELL, PK_FLAG_NO_TMA)");
      return PK_ERR_ARG;
    }
    if ((e = resident_prepare(A, s, &resident))) return e;
    if (!resident) {
      set_error("PK_LOOP_RESIDENT: the resident loop needs a tile grid of two blocks per SM "
                "(n >= 512 x 2 x SMs rows or nnz >= 4096 x 2 x SMs) and cooperative launch");
      return PK_ERR_ARG;
    }
  }
  cudaEvent_t e0, e1;
  PK_CUDA(cudaEventCreate(&e0));
  PK_CUDA(cudaEventCreate(&e1));
  PK_CUDA(cudaEventRecord(e0, s));
  if ((e = state_init(A, o, s))) return e;
  VecStage v;
  if ((e = stage_in(A, b, x, 14, 15, s, &v))) return e;
  double *r, *p, *ap;
  if ((e = work_vec(A, 0, &r)) || (e = work_vec(A, 1, &p)) || (e = work_vec(A, 2, &ap))) return e;
  const RowArgs ra = row_args(A);
  double* xd = v.x_dev;
  // The bulk-copy kernels read x in 16-byte units: a caller's x that is not 16-byte aligned or
  // has odd length is iterated in a padded library copy.
  const bool tma_engine = A->tma_ok && !(o->flags & PK_FLAG_NO_TMA) && !persistent;
  double* x_copy_back = nullptr;
  if (tma_engine && (((uintptr_t)xd & 15) || (A->n & 1))) {
    double* xi;
    if ((e = work_vec(A, 13, &xi))) return e;
    PK_CUDA(cudaMemcpyAsync(xi, xd, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, s));
    x_copy_back = xd;
    xd = xi;
  }
  const double* bd = v.b_dev;
  Timer T;
  T.A = A;
  T.on = (o->flags & PK_FLAG_TIMING) != 0;
  T.s = s;
  int launches = 0;
  if (resident) {
    // r0, p0, <r0,r0>, <b,b>; then the whole iteration loop in one cooperative launch
    if ((e = T.begin(PK_SLOT_OTHER))) return e;
    k_residual_init<<<A->grid, kBlock, 0, s>>>(row_args(A), bd, xd, r, p, nullptr);
    if ((e = T.end())) return e;
    k_zero_x<<<A->grid, kBlock, 0, s>>>(row_args(A), xd);
    PK_CUDA(cudaGetLastError());
    if ((e = T.begin(PK_SLOT_RESIDENT))) return e;
    if ((e = launch_cg_resident(A, xd, r, p, ap, s))) return e;
    if ((e = T.end())) return e;
    launches += 3;
    if ((e = T.flush())) return e;
    if (x_copy_back)
      PK_CUDA(cudaMemcpyAsync(x_copy_back, xd, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, s));
    if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
    for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
      info->kernel_count[k] = T.count[k];
      info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (pk_status)info->status;
  }
  const int G = A->grid;
  if (!A->grid_ew) {
    // elementwise kernels run as many resident blocks as their register use allows
    int nb = 1, sms = 1;
    PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_update, kBlock, 0));
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
    const int64_t need = ((int64_t)A->n + 2 * kBlock - 1) / (2 * kBlock);
    A->grid_ew = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(nb, 1) * sms, need));
  }
  const int Gu = A->grid_ew;

  // setup: r0 = b - A x0, p0 = r0, <r0,r0>, <b,b>
  if ((e = T.begin(PK_SLOT_OTHER))) return e;
  k_residual_init<<<G, kBlock, 0, s>>>(ra, bd, xd, r, p, nullptr);
  if ((e = T.end())) return e;
  k_zero_x<<<G, kBlock, 0, s>>>(ra, xd);
  launches += 2;
  PK_CUDA(cudaGetLastError());
  if (persistent) {
    // the whole iteration loop in one cooperative launch
    if ((e = T.begin(PK_SLOT_OTHER))) return e;
    if ((e = launch_cg_persistent(A, xd, r, p, ap, s))) return e;
    if ((e = T.end())) return e;
    launches += 1;
    if ((e = T.flush())) return e;
    if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
    for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
      info->kernel_count[k] = T.count[k];
      info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (pk_status)info->status;
  }
  const int variant = o->variant;
  const bool tma = tma_engine;
  if (tma && (e = tma_setup())) return e;
  const CsrTiles ct = csr_tiles_of(A);
  const bool irr = csr_irregular(A);  // some tile needs the grouped or whole-warp rows
  const int Gt = A->grid_tma, Gs = A->grid_stream;
  double* part = A->partials;
  DevState* dst = A->st;
  const int n = A->n;
  if (sell && (e = sell_build(A, s))) return e;
  const SellArgs sa = sell ? sell_args(A) : SellArgs{};
  const int Gsell = A->sell_grid;
  if (variant == PK_VARIANT_PIPELINED || variant == PK_VARIANT_SPLIT) {
    // A p0, alpha_0, beta_0
    if ((e = T.begin(PK_SLOT_SPMV_DOTS))) return e;
    if (sell) k_cg_sell_spmv_dots<<<Gsell, kBlock, 0, s>>>(sa, p, ap, part, dst);
    else if (tma) (irr ? k_cg_spmv_dots_tma<true> : k_cg_spmv_dots_tma<false>)<<<Gt, kTileThreads, csr_smem_bytes(), s>>>(ct, p, ap, part, dst);
    else k_cg_spmv_dots<<<G, kBlock, 0, s>>>(ra, p, ap);
    if ((e = T.end())) return e;
    launches += 1;
  }
  PK_CUDA(cudaGetLastError());

  LoopSpec L;
  L.keys[0] = xd;
  L.keys[1] = bd;
  L.ikeys[0] = variant;
  if (variant == PK_VARIANT_PIPELINED) {
    L.kind = 1;
    L.body_kernels = 2;
    L.unroll = tma ? 4 : 1;  // more back-to-back programmatic launches per graph body pass
    L.ikeys[1] = tma;
    L.ikeys[2] = sell;  // the SpMV kernel in the graph body
    L.body = [=](cudaStream_t cs, Timer* t) {
      if (t) t->begin(PK_SLOT_UPDATE);
      if (tma) launch_pdl(k_cg_update_tma, Gs, kTileThreads, stream_smem_bytes<4, double, 2>(), cs, n, xd, r, p, ap, part, dst);
      else k_cg_update<<<Gu, kBlock, 0, cs>>>(ra, xd, r, p, ap);
      if (t) { t->end(); t->begin(PK_SLOT_SPMV_DOTS); }
      if (sell) launch_pdl(k_cg_sell_spmv_dots, Gsell, kBlock, 0, cs, sa, (const double*)p, ap, part, dst);
      else if (tma) launch_pdl(irr ? k_cg_spmv_dots_tma<true> : k_cg_spmv_dots_tma<false>, Gt, kTileThreads, csr_smem_bytes(), cs, ct, (const double*)p, ap, part, dst);
      else k_cg_spmv_dots<<<G, kBlock, 0, cs>>>(ra, p, ap);
      if (t) t->end();
    };
  } else if (variant == PK_VARIANT_SPLIT) {
    L.kind = 2;
    L.body_kernels = 3;
    L.body = [=](cudaStream_t cs, Timer* t) {
      if (t) t->begin(PK_SLOT_UPDATE);
      k_cg_update<<<Gu, kBlock, 0, cs>>>(ra, xd, r, p, ap);
      if (t) { t->end(); t->begin(PK_SLOT_SPMV); }
      if (tma) (irr ? k_spmv_tma<true> : k_spmv_tma<false>)<<<Gt, kTileThreads, csr_smem_bytes(), cs>>>(ct, p, ap, dst, 0, 0);
      else k_spmv_live<<<G, kBlock, 0, cs>>>(ra, p, ap, 0);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_cg_dots<<<G, kBlock, 0, cs>>>(ra, p, ap);
      if (t) t->end();
    };
  } else {
    L.kind = 3;
    L.body_kernels = 6;
    L.body = [=](cudaStream_t cs, Timer* t) {
      if (t) t->begin(PK_SLOT_SPMV);
      if (tma) (irr ? k_spmv_tma<true> : k_spmv_tma<false>)<<<Gt, kTileThreads, csr_smem_bytes(), cs>>>(ct, p, ap, dst, 1, 0);
      else k_spmv_live<<<G, kBlock, 0, cs>>>(ra, p, ap, 1);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_cls_alpha<<<G, kBlock, 0, cs>>>(ra, p, ap);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_axpy_alpha<<<G, kBlock, 0, cs>>>(ra, xd, p, 1.0);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_axpy_alpha<<<G, kBlock, 0, cs>>>(ra, r, ap, -1.0);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_cls_beta<<<G, kBlock, 0, cs>>>(ra, r);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_xpay_beta<<<G, kBlock, 0, cs>>>(ra, r, p);
      if (t) t->end();
    };
  }
  if ((e = run_loop(A, o, s, L, &T, &launches))) return e;
  if ((e = T.flush())) return e;
  if (x_copy_back)
    PK_CUDA(cudaMemcpyAsync(x_copy_back, xd, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, s));
  const bool graph = o->loop != PK_LOOP_HOST && !T.on;
  if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
  if (graph) info->launches += (int)(passes_of(A->st_host) * L.body_kernels);
  for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
    info->kernel_count[k] = T.count[k];
    info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (pk_status)info->status;
}

pk_status launch_spmv_tma(pk_csr* A, const double* x, double* y, int first, int skip_early, cudaStream_t s) {
  pk_status e = tma_setup();
  if (e) return e;
  (csr_irregular(A) ? k_spmv_tma<true> : k_spmv_tma<false>)<<<A->grid_tma, kTileThreads, csr_smem_bytes(), s>>>(
      csr_tiles_of(A), x, y, A->st, first, skip_early);
  return PK_OK;
}

void launch_residual_init(const pk_csr* A, const double* b, const double* x, double* r,
                          double* p, double* r0s, cudaStream_t s) {
  k_residual_init<<<A->grid, kBlock, 0, s>>>(row_args(A), b, x, r, p, r0s);
}

void launch_zero_x(const pk_csr* A, double* x, cudaStream_t s) {
  k_zero_x<<<A->grid, kBlock, 0, s>>>(row_args(A), x);
}

}  // namespace pk

extern "C" pk_status pk_cg_solve(pk_csr* A, const double* b, double* x, const pk_opts* opts,
                                 pk_info* info, void* stream) {
  return pk::cg_solve(A, b, x, opts, info, (cudaStream_t)stream);
}
