// BiCGStab: pipelined (Alg. 4) with four fused kernels per iteration, and classical
// (Alg. 3) with one kernel per operation.  r0* = r0.
//
// Pipelined iteration i (Sec. 3.2):
//   K-BI-1  A p_i with the first stage of <Ap_i, r0*>.  Last block: alpha_i = <r_i,r0*>/<Ap_i,r0*>.
//   K-BI-2  s_i = r_i - alpha_i A p_i with the first stage of <s_i, s_i>.  Last block: ||s_i||;
//           if ||s_i|| <= tol ||b|| the iteration ends with x += alpha p (early exit).
//   K-BI-3  A s_i with the first stages of <As_i, s_i>, <As_i, As_i>, <As_i, r0*>.  Last block:
//           omega_i = <As,s>/<As,As>, beta_i = -<As,r0*>/<Ap,r0*> and the residual expansion
//           <s,s> - 2 omega <s,As> + omega^2 <As,As>.
//   K-BI-4  x += alpha p + omega s; r = s - omega As; p = r + beta (p - omega Ap) with the first
//           stages of <r_{i+1}, r0*> and <r_{i+1}, r_{i+1}>.  Last block: convergence test.
// Scalars in DevState::s: [0] <r_i, r0*>, [1] <Ap_i, r0*>, [2] <s_i, s_i>.
#include <algorithm>
#include <cmath>

#include "pk_guard.cuh"
#include "pk_tile.cuh"

namespace pk {

// ---------------------------------------------------------------- pipelined, tile engine

template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_bi1_tma(CsrTiles T, const double* __restrict__ p,
                                                             double* __restrict__ ap,
                                                             const double* __restrict__ r0s,
                                                             double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  count_pass(st);
  double v[1] = {0.0};
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return !state_done(st); }, p,
                              [&](int row, double y) {
    ap[row] = y;
    v[0] = fma(y, __ldg(r0s + row), v[0]);
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(st->cond, 0u);
    return;
  }
  tile_block_partials<1>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(partials, t);
    if (threadIdx.x == 0) {
      const double rr0s = st->s[0];
      if (__ldcg(&st->timeout)) finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] == 0.0 || rr0s == 0.0) finish(st, PK_BREAKDOWN);
      else {
        st->s[1] = t[0];
        st->alpha = rr0s / t[0];
        trace_put(st, st->iter, 0, st->alpha);
      }
      st->counter = 0;
    }
  }
}

__global__ void __launch_bounds__(kTileThreads, 2) k_bi2_tma(int n, const double* __restrict__ r,
                                                             const double* __restrict__ ap,
                                                             double* __restrict__ s_out,
                                                             double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  int r0, r1;
  ew_range(n, r0, r1);
  double v[1] = {0.0};
  double alpha = 0.0;
  StreamIn<2> in{{r, ap}};
  const bool live = stream_tiles<2, 1, double, 4>(in, r0, r1, smem, st, [&]() {
    alpha = __ldcg(&st->alpha);
    return !state_done(st);
  }, [&](int row, const double2* val, int nv) {
    double2 sn;
    sn.x = fma(-alpha, val[1].x, val[0].x);
    sn.y = fma(-alpha, val[1].y, val[0].y);
    if (nv == 2) {
      st2(s_out + row, sn);
      v[0] = fma(sn.x, sn.x, v[0]);
      v[0] = fma(sn.y, sn.y, v[0]);
    } else {
      s_out[row] = sn.x;
      v[0] = fma(sn.x, sn.x, v[0]);
    }
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<1>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(partials, t);
    if (threadIdx.x == 0) {
      st->s[2] = t[0];
      if (__ldcg(&st->timeout)) finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] <= st->thr2) st->early = 1;
      st->counter = 0;
    }
  }
}

template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_bi3_tma(CsrTiles T, const double* __restrict__ s,
                                                             double* __restrict__ as,
                                                             const double* __restrict__ r0s,
                                                             double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  double v[3] = {0.0, 0.0, 0.0};
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return !state_done(st) && !__ldcg(&st->early); }, s,
                              [&](int row, double y) {
    as[row] = y;
    v[0] = fma(y, __ldg(s + row), v[0]);
    v[1] = fma(y, y, v[1]);
    v[2] = fma(y, __ldg(r0s + row), v[2]);
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<3>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[3];
    final_sums<3>(partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter;
      if (__ldcg(&st->timeout)) finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0]) || !isfinite(t[1]) || !isfinite(t[2])) finish(st, PK_ERR_NAN);
      else if (t[1] == 0.0) finish(st, PK_BREAKDOWN);
      else {
        const double omega = t[0] / t[1];
        const double beta = -t[2] / st->s[1];
        st->omega = omega;
        st->beta = beta;
        trace_put(st, i, 1, beta);
        trace_put(st, i, 2, omega);
      }
      st->counter = 0;
    }
  }
}

__global__ void __launch_bounds__(kTileThreads, 2) k_bi4_tma(int n, double* __restrict__ x,
                                                             double* __restrict__ p,
                                                             const double* __restrict__ s,
                                                             const double* __restrict__ ap,
                                                             const double* __restrict__ r0s,
                                                             const double* __restrict__ as,
                                                             double* __restrict__ r,
                                                             double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  int r0, r1;
  ew_range(n, r0, r1);
  double v[2] = {0.0, 0.0};
  double alpha = 0.0, omega = 0.0, beta = 0.0;
  bool early = false;
  // everything but As (written by K-BI-3) is prefetched before the dependency wait
  StreamIn<6> in{{x, p, s, ap, r0s, as}};
  const bool live = stream_tiles<6, 5, double, 2>(in, r0, r1, smem, st, [&]() {
    alpha = __ldcg(&st->alpha);
    omega = __ldcg(&st->omega);
    beta = __ldcg(&st->beta);
    early = __ldcg(&st->early) != 0;
    return !state_done(st);
  }, [&](int row, const double2* val, int nv) {
    const double2 xk = val[0], pk = val[1], sk = val[2], ak = val[3], zk = val[4], bk = val[5];
    double2 xn, rn, pn;
    if (early) {  // ||s|| small: x += alpha p only
      xn.x = fma(alpha, pk.x, xk.x);
      xn.y = fma(alpha, pk.y, xk.y);
      if (nv == 2) st2(x + row, xn);
      else x[row] = xn.x;
      return;
    }
    // x + alpha p + omega s, r = s - omega As, p = r + beta (p - omega Ap): 6 FMA per row
    xn.x = fma(omega, sk.x, fma(alpha, pk.x, xk.x));
    xn.y = fma(omega, sk.y, fma(alpha, pk.y, xk.y));
    rn.x = fma(-omega, bk.x, sk.x);
    rn.y = fma(-omega, bk.y, sk.y);
    pn.x = fma(beta, fma(-omega, ak.x, pk.x), rn.x);
    pn.y = fma(beta, fma(-omega, ak.y, pk.y), rn.y);
    if (nv == 2) {
      st2(x + row, xn);
      st2(r + row, rn);
      st2(p + row, pn);
      v[0] = fma(rn.x, zk.x, v[0]);
      v[1] = fma(rn.x, rn.x, v[1]);
      v[0] = fma(rn.y, zk.y, v[0]);
      v[1] = fma(rn.y, rn.y, v[1]);
    } else {
      x[row] = xn.x;
      r[row] = rn.x;
      p[row] = pn.x;
      v[0] = fma(rn.x, zk.x, v[0]);
      v[1] = fma(rn.x, rn.x, v[1]);
    }
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<2>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter;
      st->iter = i + 1;
      if (__ldcg(&st->timeout)) {
        finish(st, PK_TIMEOUT);
      } else if (st->early) {
        st->rr = st->s[2];
        trace_put(st, i, 3, st->s[2]);
        finish(st, PK_OK);
      } else {
        st->rr = t[1];
        st->s[0] = t[0];
        trace_put(st, i, 3, t[1]);
        if (!isfinite(t[0]) || !isfinite(t[1])) finish(st, PK_ERR_NAN);
        else if (t[1] <= st->thr2) finish(st, PK_OK);
        else if (i + 1 >= st->maxit) finish(st, PK_NOT_CONVERGED);
      }
      st->counter = 0;
    }
  }
}

// ---------------------------------------------------------------- classical, Alg. 3

__device__ __forceinline__ bool cls_skip(DevState* st) {
  return state_done(st) || __ldcg(&st->early);
}

__global__ void __launch_bounds__(kBlock) k_bc_spmv(RowArgs a, const double* __restrict__ xin,
                                                    double* __restrict__ y, int first) {
  if (first) count_pass(a.st);
  if (cls_skip(a.st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) y[row] = csr_row(a, xin, row);
}

// <Ap, r0*> -> alpha
__global__ void __launch_bounds__(kBlock) k_bc_alpha(RowArgs a, const double* __restrict__ ap,
                                                     const double* __restrict__ r0s) {
  DevState* st = a.st;
  if (state_done(st)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(st->cond, 0u);
    return;
  }
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(ap[row], r0s[row], v[0]);
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      const double rr0s = st->s[0];
      if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] == 0.0 || rr0s == 0.0) finish(st, PK_BREAKDOWN);
      else {
        st->s[1] = t[0];
        st->alpha = rr0s / t[0];
        trace_put(st, st->iter, 0, st->alpha);
      }
      st->counter = 0;
    }
  }
}

// s = r - alpha Ap
__global__ void __launch_bounds__(kBlock) k_bc_s(RowArgs a, const double* __restrict__ r,
                                                 const double* __restrict__ ap, double* __restrict__ s) {
  if (cls_skip(a.st)) return;
  const double alpha = __ldcg(&a.st->alpha);
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) s[row] = fma(-alpha, ap[row], r[row]);
}

// <s, s> -> early exit flag
__global__ void __launch_bounds__(kBlock) k_bc_ss(RowArgs a, const double* __restrict__ s) {
  DevState* st = a.st;
  if (cls_skip(st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(s[row], s[row], v[0]);
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      st->s[2] = t[0];
      if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (t[0] <= st->thr2) st->early = 1;
      st->counter = 0;
    }
  }
}

// <As, s>, <As, As> -> omega
__global__ void __launch_bounds__(kBlock) k_bc_omega(RowArgs a, const double* __restrict__ as,
                                                     const double* __restrict__ s) {
  DevState* st = a.st;
  if (cls_skip(st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[2] = {0.0, 0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    v[0] = fma(as[row], s[row], v[0]);
    v[1] = fma(as[row], as[row], v[1]);
  }
  block_partials<2>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      if (!isfinite(t[0]) || !isfinite(t[1])) finish(st, PK_ERR_NAN);
      else if (t[1] == 0.0) finish(st, PK_BREAKDOWN);
      else {
        st->omega = t[0] / t[1];
        trace_put(st, st->iter, 2, st->omega);
      }
      st->counter = 0;
    }
  }
}

// x += alpha p + omega s  (early exit: x += alpha p)
__global__ void __launch_bounds__(kBlock) k_bc_x(RowArgs a, double* __restrict__ x,
                                                 const double* __restrict__ p,
                                                 const double* __restrict__ s) {
  if (state_done(a.st)) return;
  const bool early = __ldcg(&a.st->early) != 0;
  const double alpha = __ldcg(&a.st->alpha), omega = early ? 0.0 : __ldcg(&a.st->omega);
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x)
    x[row] = early ? fma(alpha, p[row], x[row]) : x[row] + fma(alpha, p[row], omega * s[row]);
}

// r = s - omega As
__global__ void __launch_bounds__(kBlock) k_bc_r(RowArgs a, double* __restrict__ r,
                                                 const double* __restrict__ s,
                                                 const double* __restrict__ as) {
  if (cls_skip(a.st)) return;
  const double omega = __ldcg(&a.st->omega);
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) r[row] = fma(-omega, as[row], s[row]);
}

// <r_{i+1}, r0*> -> beta = (<r_{i+1},r0*>/<r_i,r0*>) (alpha/omega)
__global__ void __launch_bounds__(kBlock) k_bc_beta(RowArgs a, const double* __restrict__ r,
                                                    const double* __restrict__ r0s) {
  DevState* st = a.st;
  if (cls_skip(st)) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(r[row], r0s[row], v[0]);
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
      else if (st->omega == 0.0) { st->iter += 1; finish(st, PK_BREAKDOWN); }
      else {
        st->beta = (t[0] / st->s[0]) * (st->alpha / st->omega);
        trace_put(st, st->iter, 1, st->beta);
        st->s[0] = t[0];
      }
      st->counter = 0;
    }
  }
}

// p = r + beta (p - omega Ap)
__global__ void __launch_bounds__(kBlock) k_bc_p(RowArgs a, double* __restrict__ p,
                                                 const double* __restrict__ r,
                                                 const double* __restrict__ ap) {
  if (cls_skip(a.st)) return;
  const double beta = __ldcg(&a.st->beta), omega = __ldcg(&a.st->omega);
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x)
    p[row] = fma(beta, fma(-omega, ap[row], p[row]), r[row]);
}

// <r, r> -> convergence (early exit: finish after x += alpha p)
__global__ void __launch_bounds__(kBlock) k_bc_rr(RowArgs a, const double* __restrict__ r) {
  DevState* st = a.st;
  if (state_done(st)) return;
  const bool early = __ldcg(&st->early) != 0;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  if (!early)
    for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(r[row], r[row], v[0]);
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter;
      st->iter = i + 1;
      if (early) {
        st->rr = st->s[2];
        trace_put(st, i, 3, st->s[2]);
        finish(st, PK_OK);
      } else {
        st->rr = t[0];
        trace_put(st, i, 3, t[0]);
        if (!isfinite(t[0])) finish(st, PK_ERR_NAN);
        else if (t[0] <= st->thr2) finish(st, PK_OK);
        else if (i + 1 >= st->maxit) finish(st, PK_NOT_CONVERGED);
      }
      st->counter = 0;
    }
  }
}

// ---------------------------------------------------------------- driver

static pk_status bi_tma_setup() {
  static bool done = false;
  if (!done) {
    for (auto k : {k_bi1_tma<false>, k_bi1_tma<true>, k_bi3_tma<false>, k_bi3_tma<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem_bytes()));
    PK_CUDA(cudaFuncSetAttribute(k_bi2_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, stream_smem_bytes<2, double, 4>()));
    PK_CUDA(cudaFuncSetAttribute(k_bi4_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, stream_smem_bytes<6, double, 2>()));
    done = true;
  }
  return PK_OK;
}

// pk_bicgstab_cluster.cu: the whole pipelined loop on one thread-block cluster
bool bicgstab_persistent_usable(const pk_csr* A);
pk_status launch_bicgstab_persistent(pk_csr* A, double* x, const double* r, const double* r0s, cudaStream_t s);

pk_status bicgstab_solve(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                         cudaStream_t s) {
  pk_status e = check_opts(A, b, x, o, info);
  if (e) return e;
  if (o->loop == PK_LOOP_RESIDENT) { set_error("PK_LOOP_RESIDENT runs pipelined CG only"); return PK_ERR_ARG; }
  *info = pk_info{};
  info->rel_res_true = -1.0;
  if (A->n == 0) return PK_OK;
  if (o->precision != PK_PREC_FP64) { set_error("BiCGStab runs in FP64 only"); return PK_ERR_ARG; }
  if (o->variant != PK_VARIANT_PIPELINED && o->variant != PK_VARIANT_CLASSICAL) {
    set_error("BiCGStab variants: pipelined or classical");
    return PK_ERR_ARG;
  }
  if (o->precond != PK_PRECOND_NONE && o->precond != PK_PRECOND_JACOBI) { set_error("bad precond"); return PK_ERR_ARG; }
  if (o->flags & PK_FLAG_SELL) { set_error("PK_FLAG_SELL applies to pipelined FP64 CG"); return PK_ERR_ARG; }
  if (o->flags & PK_FLAG_CGS2) { set_error("PK_FLAG_CGS2 applies to GMRES"); return PK_ERR_ARG; }
  // the whole loop on one thread-block cluster (small systems): asked for, or chosen by AUTO
  bool persistent = false;
  if (o->loop == PK_LOOP_PERSISTENT) {
    if (o->variant != PK_VARIANT_PIPELINED) {
      set_error("PK_LOOP_PERSISTENT runs the pipelined forms of CG and BiCGStab only");
      return PK_ERR_ARG;
    }
    if (!bicgstab_persistent_usable(A)) {
      set_error("PK_LOOP_PERSISTENT: the persistent BiCGStab loop needs n <= 16 x 4096 rows (one thread-block cluster) and cluster launch");
      return PK_ERR_ARG;
    }
    persistent = true;
  } else if (o->loop == PK_LOOP_AUTO) {
    // (rows of very different lengths stay on the tile engine: one thread per row leaves the
    // cluster waiting for the longest)
    persistent = o->variant == PK_VARIANT_PIPELINED && A->n <= PK_PERSISTENT_BICGSTAB_AUTO_N &&
                 A->nnz <= PK_PERSISTENT_BICGSTAB_AUTO_NNZ && A->stats.tiles_long == 0 &&
                 !(o->flags & PK_FLAG_TIMING) && bicgstab_persistent_usable(A);
  }
  cudaEvent_t e0, e1;
  PK_CUDA(cudaEventCreate(&e0));
  PK_CUDA(cudaEventCreate(&e1));
  PK_CUDA(cudaEventRecord(e0, s));
  if ((e = state_init(A, o, s))) return e;
  VecStage v;
  if ((e = stage_in(A, b, x, 14, 15, s, &v))) return e;
  double *r, *p, *ap, *sv, *as, *r0s;
  if ((e = work_vec(A, 0, &r)) || (e = work_vec(A, 1, &p)) || (e = work_vec(A, 2, &ap)) ||
      (e = work_vec(A, 3, &sv)) || (e = work_vec(A, 4, &as)) || (e = work_vec(A, 5, &r0s)))
    return e;
  const bool tma = A->tma_ok && !(o->flags & PK_FLAG_NO_TMA) && o->variant == PK_VARIANT_PIPELINED && !persistent;
  // the classical form's SpMV runs on the same tile engine (only the fusion differs)
  const bool tma_spmv = A->tma_ok && !(o->flags & PK_FLAG_NO_TMA);
  double* xd = v.x_dev;
  double* x_copy_back = nullptr;
  if (tma && (((uintptr_t)xd & 15) || (A->n & 1))) {
    double* xi;
    if ((e = work_vec(A, 13, &xi))) return e;
    PK_CUDA(cudaMemcpyAsync(xi, xd, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, s));
    x_copy_back = xd;
    xd = xi;
  }
  if (tma && (e = bi_tma_setup())) return e;
  // right Jacobi preconditioning: iterate on A M^-1 with y = M x (values swapped until leave)
  JacobiRight jac;
  if (o->precond == PK_PRECOND_JACOBI && (e = jacobi_right_enter(A, xd, s, &jac))) return e;
  Timer T;
  T.A = A;
  T.on = (o->flags & PK_FLAG_TIMING) != 0;
  T.s = s;
  int launches = 0;
  const RowArgs ra = row_args(A);
  const CsrTiles ct = csr_tiles_of(A);
  const bool irr = csr_irregular(A);  // some tile needs the grouped or whole-warp rows
  const int G = A->grid, Gt = A->grid_tma, Gs = A->grid_stream, n = A->n;
  double* part = A->partials;
  DevState* dst = A->st;

  // setup: r0 = b - A x0, p0 = r0, r0* = r0, <r0, r0*>
  if ((e = T.begin(PK_SLOT_OTHER))) return e;
  launch_residual_init(A, v.b_dev, xd, r, p, r0s, s);
  if ((e = T.end())) return e;
  launch_zero_x(A, xd, s);
  launches += 2;
  PK_CUDA(cudaGetLastError());
  if (persistent) {
    if ((e = T.begin(PK_SLOT_OTHER))) return e;
    if ((e = launch_bicgstab_persistent(A, xd, r, r0s, s))) return e;
    if ((e = T.end())) return e;
    launches += 1;
    if ((e = T.flush())) return e;
    if (jac.A) {
      if ((e = jacobi_right_leave(&jac, xd, s))) return e;
      launches += 2;
    }
    if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
    for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
      info->kernel_count[k] = T.count[k];
      info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (pk_status)info->status;
  }

  LoopSpec L;
  L.keys[0] = xd;
  L.ikeys[0] = o->variant;
  L.ikeys[1] = tma;
  L.ikeys[2] = o->precond;  // the graph holds the value pointer of A or of A M^-1
  if (o->variant == PK_VARIANT_PIPELINED) {
    L.kind = 4;
    L.body_kernels = 4;
    L.unroll = tma ? 2 : 1;
    L.body = [=](cudaStream_t cs, Timer* t) {
      if (tma) {
        if (t) t->begin(PK_SLOT_SPMV_DOTS);
        launch_pdl(irr ? k_bi1_tma<true> : k_bi1_tma<false>, Gt, kTileThreads, csr_smem_bytes(), cs, ct, (const double*)p, ap, (const double*)r0s, part, dst);
        if (t) { t->end(); t->begin(PK_SLOT_UPDATE); }
        launch_pdl(k_bi2_tma, Gs, kTileThreads, stream_smem_bytes<2, double, 4>(), cs, n, (const double*)r, (const double*)ap, sv, part, dst);
        if (t) { t->end(); t->begin(PK_SLOT_SPMV_DOTS); }
        launch_pdl(irr ? k_bi3_tma<true> : k_bi3_tma<false>, Gt, kTileThreads, csr_smem_bytes(), cs, ct, (const double*)sv, as, (const double*)r0s, part, dst);
        if (t) { t->end(); t->begin(PK_SLOT_UPDATE); }
        launch_pdl(k_bi4_tma, Gs, kTileThreads, stream_smem_bytes<6, double, 2>(), cs, n, xd, p, (const double*)sv,
                   (const double*)ap, (const double*)r0s, (const double*)as, r, part, dst);
        if (t) t->end();
      }
    };
    if (!tma) {
      set_error("pipelined BiCGStab needs the tile engine (PK_FLAG_NO_TMA: only the classical form has thread-per-row kernels)");
      return PK_ERR_ARG;
    }
  } else {
    L.kind = 5;
    L.body_kernels = 11;
    L.body = [=](cudaStream_t cs, Timer* t) {
      auto k = [&](int slot) { if (t) t->begin(slot); };
      auto kend = [&]() { if (t) t->end(); };
      k(PK_SLOT_SPMV);
      if (tma_spmv) launch_spmv_tma(A, p, ap, 1, 1, cs);
      else k_bc_spmv<<<G, kBlock, 0, cs>>>(ra, p, ap, 1);
      kend();
      k(PK_SLOT_BLAS1); k_bc_alpha<<<G, kBlock, 0, cs>>>(ra, ap, r0s); kend();
      k(PK_SLOT_BLAS1); k_bc_s<<<G, kBlock, 0, cs>>>(ra, r, ap, sv); kend();
      k(PK_SLOT_BLAS1); k_bc_ss<<<G, kBlock, 0, cs>>>(ra, sv); kend();
      k(PK_SLOT_SPMV);
      if (tma_spmv) launch_spmv_tma(A, sv, as, 0, 1, cs);
      else k_bc_spmv<<<G, kBlock, 0, cs>>>(ra, sv, as, 0);
      kend();
      k(PK_SLOT_BLAS1); k_bc_omega<<<G, kBlock, 0, cs>>>(ra, as, sv); kend();
      k(PK_SLOT_BLAS1); k_bc_x<<<G, kBlock, 0, cs>>>(ra, xd, p, sv); kend();
      k(PK_SLOT_BLAS1); k_bc_r<<<G, kBlock, 0, cs>>>(ra, r, sv, as); kend();
      k(PK_SLOT_BLAS1); k_bc_beta<<<G, kBlock, 0, cs>>>(ra, r, r0s); kend();
      k(PK_SLOT_BLAS1); k_bc_p<<<G, kBlock, 0, cs>>>(ra, p, r, ap); kend();
      k(PK_SLOT_BLAS1); k_bc_rr<<<G, kBlock, 0, cs>>>(ra, r); kend();
    };
  }
  if ((e = run_loop(A, o, s, L, &T, &launches))) return e;
  if ((e = T.flush())) return e;
  if (jac.A) {
    if ((e = jacobi_right_leave(&jac, xd, s))) return e;
    launches += 2;  // y0 = M x0 and x = M^-1 y
  }
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

}  // namespace pk

extern "C" pk_status pk_bicgstab_solve(pk_csr* A, const double* b, double* x, const pk_opts* opts,
                                       pk_info* info, void* stream) {
  return pk::guarded([&] { return pk::bicgstab_solve(A, b, x, opts, info, (cudaStream_t)stream); });
}
