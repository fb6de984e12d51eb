// CG with the Jacobi preconditioner M = diag(A) in the pipelined structure of Alg. 2 (the
// preconditioner fusion Sec. 5 names as the natural extension).  M^-1 is a product with the
// reciprocal diagonal, so it fuses into the existing two kernels of an iteration:
//   K-PCG-U  x += alpha p;  r -= alpha Ap;  p = M^-1 r + beta p;  first stages of
//            <r, M^-1 r> and <r, r>.  Last block: convergence test on ||r||.
//   K-PCG-S  Ap fused with the first stages of <p, Ap> and <Ap, M^-1 Ap>.  Last block:
//            alpha = <r, M^-1 r>/<p, Ap>, beta = alpha^2 <Ap, M^-1 Ap>/<r, M^-1 r> - 1 (the
//            preconditioned analogue of Eq. (3)).
// Bytes per iteration: 12 nnz + 92 n (the reciprocal diagonal is read by both kernels).
#include <algorithm>
#include <cmath>

#include "pk_tile.cuh"

namespace pk {

namespace {

constexpr int kPcgRowPairs = 1;  // row pairs per consumer thread per stage of K-PCG-U

// dinv = 1 / diag(A); a diagonal entry that is not > 0 ends the solve with PK_NOT_SPD.
__global__ void __launch_bounds__(kBlock) k_jacobi_inverse(RowArgs a, double* __restrict__ dinv) {
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    double d = 0.0;
    for (int j = __ldg(a.rp + row); j < __ldg(a.rp + row + 1); ++j)
      if (__ldg(a.ci + j) == row) d += __ldg(a.va + j);
    if (!(d > 0.0)) {
      a.st->status = PK_NOT_SPD;  // every writer stores the same values
      a.st->done = 1;
      d = 1.0;
    }
    dinv[row] = 1.0 / d;
  }
}

// r0 = b - A x0, p0 = M^-1 r0, first stages of <r0, r0>, <b, b>, <r0, M^-1 r0>.  Last block:
// rr, bb, thr2, gamma (DevState::s[0]) and the zero-iteration exits.
__global__ void __launch_bounds__(kBlock) k_pcg_init(RowArgs a, const double* __restrict__ b,
                                                     const double* __restrict__ x,
                                                     const double* __restrict__ dinv,
                                                     double* __restrict__ r, double* __restrict__ p) {
  if (state_done(a.st)) return;  // a non-positive diagonal entry (uniform in the grid)
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[3] = {0.0, 0.0, 0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double bi = b[row];
    const double ri = bi - csr_row(a, x, row);
    const double zi = ri * dinv[row];
    r[row] = ri;
    p[row] = zi;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(bi, bi, v[1]);
    v[2] = fma(ri, zi, v[2]);
  }
  block_partials<3>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[3];
    final_sums<3>(a.partials, t);
    if (threadIdx.x == 0) {
      DevState* st = a.st;
      const double tol = st->thr2;
      st->rr = t[0];
      st->bb = t[1];
      st->s[0] = t[2];
      st->thr2 = tol * tol * t[1];
      st->iter = 0;
      if (!isfinite(t[0]) || !isfinite(t[1]) || !isfinite(t[2])) finish(st, PK_ERR_NAN);
      else if (t[1] == 0.0) { st->zero_x = 1; st->rr = 0.0; finish(st, PK_OK); }
      else if (t[0] <= st->thr2) finish(st, PK_OK);
      else if (st->maxit <= 0) finish(st, PK_NOT_CONVERGED);
      st->counter = 0;
    }
  }
}

// K-PCG-S on the CSR tile engine.
template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_pcg_spmv_dots_tma(CsrTiles T, const double* __restrict__ p,
                                                                       double* __restrict__ ap,
                                                                       const double* __restrict__ dinv,
                                                                       double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  double v[2] = {0.0, 0.0};
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return !state_done(st); }, p,
                                   [&](int row, double y) {
    ap[row] = y;
    v[0] = fma(__ldg(p + row), y, v[0]);
    v[1] = fma(y * __ldg(dinv + row), y, v[1]);
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<2>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(partials, t);
    if (threadIdx.x == 0) {
      const double gamma = st->s[0];
      if (__ldcg(&st->timeout)) {
        finish(st, PK_TIMEOUT);
      } else if (!isfinite(t[0]) || !isfinite(t[1])) {
        finish(st, PK_ERR_NAN);
      } else if (t[0] <= 0.0) {
        finish(st, PK_NOT_SPD);
      } else {
        const double alpha = gamma / t[0];
        const double beta = alpha * alpha * t[1] / gamma - 1.0;
        st->alpha = alpha;
        st->beta = beta;
        trace_put(st, st->iter, 0, alpha);
        trace_put(st, st->iter, 1, beta);
      }
      st->counter = 0;
    }
  }
}

// K-PCG-U on the streaming engine: x, r and the reciprocal diagonal do not depend on the
// preceding K-PCG-S and are prefetched before the dependency wait.
__global__ void __launch_bounds__(kTileThreads, 2) k_pcg_update_tma(int n, double* __restrict__ x,
                                                                    double* __restrict__ r,
                                                                    double* __restrict__ p,
                                                                    const double* __restrict__ ap,
                                                                    const double* __restrict__ dinv,
                                                                    double* partials, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  count_pass(st);
  int r0, r1;
  ew_range(n, r0, r1);
  double v[2] = {0.0, 0.0};
  double alpha = 0.0, beta = 0.0;
  StreamIn<5> in{{x, r, dinv, p, ap}};
  const bool live = stream_tiles<5, 3, double, kPcgRowPairs>(in, r0, r1, smem, st, [&]() {
    alpha = __ldcg(&st->alpha);
    beta = __ldcg(&st->beta);
    return !state_done(st);
  }, [&](int row, const double2* val, int nv) {
    const double2 xk = val[0], rq = val[1], dk = val[2], pk = val[3], ak = val[4];
    double2 xn, rn, zn, pn;
    xn.x = fma(alpha, pk.x, xk.x);
    xn.y = fma(alpha, pk.y, xk.y);
    rn.x = fma(-alpha, ak.x, rq.x);
    rn.y = fma(-alpha, ak.y, rq.y);
    zn.x = rn.x * dk.x;
    zn.y = rn.y * dk.y;
    pn.x = fma(beta, pk.x, zn.x);
    pn.y = fma(beta, pk.y, zn.y);
    if (nv == 2) {
      st2(x + row, xn);
      st2(r + row, rn);
      st2(p + row, pn);
      v[0] = fma(rn.x, zn.x, v[0]);
      v[1] = fma(rn.x, rn.x, v[1]);
      v[0] = fma(rn.y, zn.y, v[0]);
      v[1] = fma(rn.y, rn.y, v[1]);
    } else {
      x[row] = xn.x;
      r[row] = rn.x;
      p[row] = pn.x;
      v[0] = fma(rn.x, zn.x, v[0]);
      v[1] = fma(rn.x, rn.x, v[1]);
    }
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) cudaGraphSetConditional(st->cond, 0u);
    return;
  }
  tile_block_partials<2>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(partials, t);
    if (threadIdx.x == 0) {
      const int i = st->iter + 1;
      st->iter = i;
      st->s[0] = t[0];  // <r_i, M^-1 r_i>
      st->rr = t[1];
      trace_put(st, i - 1, 3, t[1]);
      if (__ldcg(&st->timeout)) finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0]) || !isfinite(t[1])) finish(st, PK_ERR_NAN);
      else if (t[1] <= st->thr2) finish(st, PK_OK);
      else if (i >= st->maxit) finish(st, PK_NOT_CONVERGED);
      st->counter = 0;
    }
  }
}

pk_status pcg_setup() {
  static bool done = false;
  if (!done) {
    for (auto k : {k_pcg_spmv_dots_tma<false>, k_pcg_spmv_dots_tma<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem_bytes()));
    PK_CUDA(cudaFuncSetAttribute(k_pcg_update_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 stream_smem_bytes<5, double, kPcgRowPairs>()));
    // two blocks of up to 113 KB each need the largest shared-memory carveout
    PK_CUDA(cudaFuncSetAttribute(k_pcg_update_tma, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    done = true;
  }
  return PK_OK;
}

}  // namespace

pk_status pcg_jacobi_solve(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                           cudaStream_t s) {
  if (o->variant != PK_VARIANT_PIPELINED || o->precision != PK_PREC_FP64 || o->loop == PK_LOOP_PERSISTENT || o->loop == PK_LOOP_RESIDENT) {
    set_error("PK_PRECOND_JACOBI runs pipelined FP64 CG on the graph or host loop");
    return PK_ERR_ARG;
  }
  if (!A->tma_ok || (o->flags & PK_FLAG_NO_TMA)) {
    set_error("PK_PRECOND_JACOBI needs the tile engine (PK_FLAG_NO_TMA is not supported)");
    return PK_ERR_ARG;
  }
  pk_status e;
  if ((e = pcg_setup())) return e;
  cudaEvent_t e0, e1;
  PK_CUDA(cudaEventCreate(&e0));
  PK_CUDA(cudaEventCreate(&e1));
  PK_CUDA(cudaEventRecord(e0, s));
  if ((e = state_init(A, o, s))) return e;
  VecStage v;
  if ((e = stage_in(A, b, x, 14, 15, s, &v))) return e;
  double *r, *p, *ap, *dinv;
  if ((e = work_vec(A, 0, &r)) || (e = work_vec(A, 1, &p)) || (e = work_vec(A, 2, &ap)) ||
      (e = work_vec(A, 6, &dinv)))
    return e;
  double* xd = v.x_dev;
  double* x_copy_back = nullptr;  // the bulk-copy kernels read x in 16-byte units
  if (((uintptr_t)xd & 15) || (A->n & 1)) {
    double* xi;
    if ((e = work_vec(A, 13, &xi))) return e;
    PK_CUDA(cudaMemcpyAsync(xi, xd, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, s));
    x_copy_back = xd;
    xd = xi;
  }
  const double* bd = v.b_dev;
  const RowArgs ra = row_args(A);
  Timer T;
  T.A = A;
  T.on = (o->flags & PK_FLAG_TIMING) != 0;
  T.s = s;
  int launches = 0;
  const int G = A->grid, Gt = A->grid_tma, Gs = A->grid_stream, n = A->n;
  const CsrTiles ct = csr_tiles_of(A);
  const bool irr = csr_irregular(A);
  double* part = A->partials;
  DevState* dst = A->st;
  if ((e = T.begin(PK_SLOT_OTHER))) return e;
  k_jacobi_inverse<<<G, kBlock, 0, s>>>(ra, dinv);
  k_pcg_init<<<G, kBlock, 0, s>>>(ra, bd, xd, dinv, r, p);
  if ((e = T.end())) return e;
  launch_zero_x(A, xd, s);
  launches += 3;
  // A p0, alpha_0, beta_0
  if ((e = T.begin(PK_SLOT_SPMV_DOTS))) return e;
  (irr ? k_pcg_spmv_dots_tma<true> : k_pcg_spmv_dots_tma<false>)<<<Gt, kTileThreads, csr_smem_bytes(), s>>>(
      ct, p, ap, dinv, part, dst);
  if ((e = T.end())) return e;
  launches += 1;
  PK_CUDA(cudaGetLastError());
  LoopSpec L;
  L.kind = 6;
  L.keys[0] = xd;
  L.keys[1] = bd;
  L.ikeys[0] = PK_PRECOND_JACOBI;
  L.ikeys[1] = irr;
  L.body_kernels = 2;
  L.unroll = 4;
  L.body = [=](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_UPDATE);
    launch_pdl(k_pcg_update_tma, Gs, kTileThreads, stream_smem_bytes<5, double, kPcgRowPairs>(), cs, n, xd, r, p, (const double*)ap,
               (const double*)dinv, part, dst);
    if (t) { t->end(); t->begin(PK_SLOT_SPMV_DOTS); }
    launch_pdl(irr ? k_pcg_spmv_dots_tma<true> : k_pcg_spmv_dots_tma<false>, Gt, kTileThreads, csr_smem_bytes(),
               cs, ct, (const double*)p, ap, (const double*)dinv, part, dst);
    if (t) t->end();
  };
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

}  // namespace pk
