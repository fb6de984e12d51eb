// Mixed-precision pipelined CG for one system: FP32 SpMV and vector updates with FP32
// accumulation inside an FP64 iterative-refinement loop.
//
// Outer step (FP64): r = b - A x with ||r|| and the convergence test; the inner right-hand
// side is r / ||r|| rounded to FP32; after the inner solve x += ||r|| d.  Inner loop: Alg. 2
// in FP32 (values rounded to FP32, FP32 vectors), stopped when the inner residual has dropped
// by tol_in = 1e-4.  The inner products that set alpha and beta are accumulated per thread as
// float-float pairs (error-free products with fmaf, TwoSum) and summed across threads and
// blocks in FP64, so the step lengths carry FP64-level accuracy while the slow FP64 pipe of
// GB300 is left out of the inner loop.  Inner bytes per iteration: 8 nnz + 40 n.
// The loops run as two nested CUDA-graph WHILE nodes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pk_guard.cuh"
#include "pk_tile.cuh"

namespace pk {

constexpr double kTolInner = 1e-4;
constexpr int kMaxOuter = 20;

struct MxArgs {
  int n;
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const float* va32;
  const int32_t* rowblk;
  const double* b;
  double* x;
  double* r64;
  float *r, *p, *ap, *d;
  double* partials;
  DevState* st;
};

__device__ __forceinline__ float row32(const MxArgs& a, const float* __restrict__ x, int row) {
  int j = __ldg(a.rp + row);
  const int j1 = __ldg(a.rp + row + 1);
  float s = 0.0f;
  for (; j + 4 <= j1; j += 4) {
    int c[4];
    float v[4], xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { c[k] = __ldg(a.ci + j + k); v[k] = __ldg(a.va32 + j + k); }
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = __ldg(x + c[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fmaf(v[k], xv[k], s);
  }
  for (; j < j1; ++j) s = fmaf(__ldg(a.va32 + j), __ldg(x + __ldg(a.ci + j)), s);
  return s;
}

__device__ __forceinline__ double row64(const MxArgs& a, const double* __restrict__ x, int row) {
  int j = __ldg(a.rp + row);
  const int j1 = __ldg(a.rp + row + 1);
  double s = 0.0;
  for (; j + 4 <= j1; j += 4) {
    int c[4];
    double v[4], xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { c[k] = __ldg(a.ci + j + k); v[k] = __ldg(a.va + j + k); }
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = __ldg(x + c[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fma(v[k], xv[k], s);
  }
  for (; j < j1; ++j) s = fma(__ldg(a.va + j), __ldg(x + __ldg(a.ci + j)), s);
  return s;
}

__device__ __forceinline__ void mx_stop_inner(DevState* st) {
  st->gm_phase = 0;
  if (st->use_cond) cudaGraphSetConditional(st->cond2, 0u);
}

__device__ __forceinline__ void mx_finish(DevState* st, int status) {
  finish(st, status);
  if (st->use_cond) cudaGraphSetConditional(st->cond2, 0u);
}

// Outer: r = b - A x in FP64, ||r||, convergence test.
__global__ void __launch_bounds__(kBlock) k_mx_residual(MxArgs a) {
  DevState* st = a.st;
  if (state_done(st)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) {
      cudaGraphSetConditional(st->cond, 0u);
      cudaGraphSetConditional(st->cond2, 0u);
    }
    return;
  }
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[2] = {0.0, 0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double bi = a.b[row];
    const double ri = bi - row64(a, a.x, row);
    a.r64[row] = ri;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(bi, bi, v[1]);
  }
  block_partials<2>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      if (st->gm_cycle == 0) {
        const double tol = st->thr2;
        st->bb = t[1];
        st->thr2 = tol * tol * t[1];
      }
      st->rr = t[0];
      if (!isfinite(t[0]) || !isfinite(t[1])) mx_finish(st, PK_ERR_NAN);
      else if (st->bb == 0.0) { st->zero_x = 1; st->rr = 0.0; mx_finish(st, PK_OK); }
      else if (t[0] <= st->thr2) mx_finish(st, PK_OK);
      else if (st->gm_cycle >= kMaxOuter || st->iter >= st->maxit) mx_finish(st, PK_NOT_CONVERGED);
      else {
        st->s[0] = sqrt(t[0]);  // ||r||: the inner right-hand side is r / ||r||
        st->s[5] = 1.0 / st->s[0];
        st->gm_cycle += 1;
        st->gm_phase = 1;
        if (st->use_cond) cudaGraphSetConditional(st->cond2, 1u);
      }
      st->counter = 0;
    }
  }
}

// Inner start: r32 = p32 = fl(r / ||r||), d = 0, <r32, r32>.
__global__ void __launch_bounds__(kBlock) k_mx_prep(MxArgs a) {
  DevState* st = a.st;
  if (state_done(st)) return;
  const double inv = __ldcg(&st->s[5]);
  int r0, r1;
  ew_range(a.n, r0, r1);
  FF acc{0.0f, 0.0f};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const float ri = (float)(a.r64[row] * inv);
    a.r[row] = ri;
    a.p[row] = ri;
    a.d[row] = 0.0f;
    ff_add_prod(acc, ri, ri);
  }
  double v[1] = {ff_value(acc)};
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      st->s[2] = t[0];                          // inner <r, r>
      st->s[3] = kTolInner * kTolInner * t[0];  // inner stopping threshold
      st->counter = 0;
    }
  }
}

// Inner K-CG-S in FP32: Ap = A p, <Ap,Ap>, <p,Ap> -> alpha, beta (Eq. (3)) in FP64.
__global__ void __launch_bounds__(kBlock) k_mx_spmv(MxArgs a) {
  DevState* st = a.st;
  if (state_done(st) || __ldcg(&st->gm_phase) != 1) return;
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  FF aa{0.0f, 0.0f}, pa{0.0f, 0.0f};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const float s = row32(a, a.p, row);
    a.ap[row] = s;
    ff_add_prod(aa, s, s);
    ff_add_prod(pa, __ldg(a.p + row), s);
  }
  double v[2] = {ff_value(aa), ff_value(pa)};
  block_partials<2>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      const double rr = st->s[2];
      if (!isfinite(t[0]) || !isfinite(t[1])) mx_finish(st, PK_ERR_NAN);
      else if (t[1] <= 0.0) mx_finish(st, PK_NOT_SPD);
      else {
        st->alpha = rr / t[1];
        st->beta = st->alpha * st->alpha * t[0] / rr - 1.0;
      }
      st->counter = 0;
    }
  }
}

// Inner K-CG-U in FP32: d += alpha p, r -= alpha Ap, p = r + beta p, <r, r>.
__global__ void __launch_bounds__(kBlock) k_mx_update(MxArgs a) {
  DevState* st = a.st;
  count_pass(st);
  if (state_done(st) || __ldcg(&st->gm_phase) != 1) return;
  const float af = (float)__ldcg(&st->alpha), bf = (float)__ldcg(&st->beta);
  int r0, r1;
  ew_range(a.n, r0, r1);
  FF acc{0.0f, 0.0f};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const float pk = a.p[row];
    a.d[row] = fmaf(af, pk, a.d[row]);
    const float rk = fmaf(-af, a.ap[row], a.r[row]);
    a.r[row] = rk;
    a.p[row] = fmaf(bf, pk, rk);
    ff_add_prod(acc, rk, rk);
  }
  double v[1] = {ff_value(acc)};
  block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      st->s[2] = t[0];
      st->iter += 1;
      trace_put(st, st->iter - 1, 0, st->alpha);
      trace_put(st, st->iter - 1, 1, st->beta);
      trace_put(st, st->iter - 1, 3, t[0]);
      if (!isfinite(t[0])) mx_finish(st, PK_ERR_NAN);
      else if (t[0] <= st->s[3] || st->iter >= st->maxit) mx_stop_inner(st);
      st->counter = 0;
    }
  }
}

// ---------------------------------------------------------------- tile-engine forms
// The inner loop on the warp-specialised engines: the FP32 CSR copy streamed in bulk-copied
// tiles (producer warp) for K-CG-S, the four FP32 vectors streamed for K-CG-U, both launched
// with programmatic dependent launch.  Same per-element arithmetic as the row kernels above.

__device__ __forceinline__ bool mx_inner_live(DevState* st) {
  return !state_done(st) && __ldcg(&st->gm_phase) == 1;
}

template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_mx_spmv_tma(CsrTilesT<float> T, MxArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = a.st;
  FF aa{0.0f, 0.0f}, pa{0.0f, 0.0f};
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return mx_inner_live(st); }, (const float*)a.p,
                              [&](int row, float y) {
    a.ap[row] = y;
    ff_add_prod(aa, y, y);
    ff_add_prod(pa, __ldg(a.p + row), y);
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  double v[2] = {ff_value(aa), ff_value(pa)};
  tile_block_partials<2>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(a.partials, t);
    if (threadIdx.x == 0) {
      const double rr = st->s[2];
      if (__ldcg(&st->timeout)) mx_finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0]) || !isfinite(t[1])) mx_finish(st, PK_ERR_NAN);
      else if (t[1] <= 0.0) mx_finish(st, PK_NOT_SPD);
      else {
        st->alpha = rr / t[1];
        st->beta = st->alpha * st->alpha * t[0] / rr - 1.0;
      }
      st->counter = 0;
    }
  }
}

__global__ void __launch_bounds__(kTileThreads, 2) k_mx_update_tma(MxArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = a.st;
  count_pass(st);
  int r0, r1;
  ew_range(a.n, r0, r1);
  float af = 0.0f, bf = 0.0f;
  FF acc{0.0f, 0.0f};
  // d and r do not depend on the preceding K-CG-S: prefetched before the dependency wait
  StreamIn<4, float> in{{a.d, a.r, a.p, a.ap}};
  const bool live = stream_tiles<4, 2, float, 2>(in, r0, r1, smem, st, [&]() {
    af = (float)__ldcg(&st->alpha);
    bf = (float)__ldcg(&st->beta);
    return mx_inner_live(st);
  }, [&](int row, const float2* val, int nv) {
    const float2 dk = val[0], rq = val[1], pk = val[2], ak = val[3];
    float2 dn, rn, pn;
    dn.x = fmaf(af, pk.x, dk.x);
    dn.y = fmaf(af, pk.y, dk.y);
    rn.x = fmaf(-af, ak.x, rq.x);
    rn.y = fmaf(-af, ak.y, rq.y);
    pn.x = fmaf(bf, pk.x, rn.x);
    pn.y = fmaf(bf, pk.y, rn.y);
    if (nv == 2) {
      *reinterpret_cast<float2*>(a.d + row) = dn;
      *reinterpret_cast<float2*>(a.r + row) = rn;
      *reinterpret_cast<float2*>(a.p + row) = pn;
      ff_add_prod(acc, rn.x, rn.x);
      ff_add_prod(acc, rn.y, rn.y);
    } else {
      a.d[row] = dn.x;
      a.r[row] = rn.x;
      a.p[row] = pn.x;
      ff_add_prod(acc, rn.x, rn.x);
    }
  });
  griddep_trigger();
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  double v[1] = {ff_value(acc)};
  tile_block_partials<1>(v, a.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      st->s[2] = t[0];
      st->iter += 1;
      trace_put(st, st->iter - 1, 0, st->alpha);
      trace_put(st, st->iter - 1, 1, st->beta);
      trace_put(st, st->iter - 1, 3, t[0]);
      if (__ldcg(&st->timeout)) mx_finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0])) mx_finish(st, PK_ERR_NAN);
      else if (t[0] <= st->s[3] || st->iter >= st->maxit) mx_stop_inner(st);
      st->counter = 0;
    }
  }
}

static pk_status mx_tma_setup() {
  static bool done = false;
  if (!done) {
    for (auto k : {k_mx_spmv_tma<false>, k_mx_spmv_tma<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem_bytes()));
    PK_CUDA(cudaFuncSetAttribute(k_mx_update_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 stream_smem_bytes<4, float, 2>()));
    // two blocks of up to 113 KB each need the largest shared-memory carveout
    PK_CUDA(cudaFuncSetAttribute(k_mx_update_tma, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    done = true;
  }
  return PK_OK;
}

// Outer correction: x += ||r|| d in FP64.
__global__ void __launch_bounds__(kBlock) k_mx_correct(MxArgs a) {
  DevState* st = a.st;
  if (state_done(st)) return;
  const double scale = __ldcg(&st->s[0]);
  int r0, r1;
  ew_range(a.n, r0, r1);
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x)
    a.x[row] = fma(scale, (double)a.d[row], a.x[row]);
}

__global__ void k_mx_init(DevState* st) {
  st->gm_cycle = 0;
  st->gm_phase = 0;
}

// FP32 copy of A's values for the mixed-precision kernels (single and batched), made once per
// handle.  A->va32 is set only once the copy is complete: a failed attempt leaves nothing
// half-made for the next solve to pick up.
pk_status ensure_fp32_values(pk_csr* A, cudaStream_t s) {
  if (A->va32 || A->nnz == 0) return PK_OK;
  float* d = nullptr;
  const pk_status e = guarded([&]() -> pk_status {
    std::vector<double> hv(A->nnz);
    std::vector<float> hf(A->nnz);
    PK_CUDA(cudaMalloc(&d, sizeof(float) * ((size_t)A->nnz + 64)));
    PK_CUDA(cudaMemsetAsync(d + A->nnz, 0, sizeof(float) * 64, s));
    PK_CUDA(cudaMemcpyAsync(hv.data(), A->va, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < A->nnz; ++j) hf[j] = (float)hv[j];
    PK_CUDA(cudaMemcpyAsync(d, hf.data(), sizeof(float) * A->nnz, cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaStreamSynchronize(s));
    return PK_OK;
  });
  if (e) {
    if (d) cudaFree(d);
    return e;
  }
  A->va32 = d;
  return PK_OK;
}

pk_status cg_mixed(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                   cudaStream_t s) {
  pk_status e;
  if (o->loop == PK_LOOP_PERSISTENT || o->loop == PK_LOOP_RESIDENT) { set_error("PK_LOOP_PERSISTENT / PK_LOOP_RESIDENT run pipelined FP64 CG only"); return PK_ERR_ARG; }
  if ((e = ensure_fp32_values(A, s))) return e;
  cudaEvent_t e0, e1;
  PK_CUDA(cudaEventCreate(&e0));
  PK_CUDA(cudaEventCreate(&e1));
  PK_CUDA(cudaEventRecord(e0, s));
  if ((e = state_init(A, o, s))) return e;
  k_mx_init<<<1, 1, 0, s>>>(A->st);
  VecStage v;
  if ((e = stage_in(A, b, x, 14, 15, s, &v))) return e;
  double *r64, *w1, *w2, *w3, *w4;
  if ((e = work_vec(A, 0, &r64)) || (e = work_vec(A, 1, &w1)) || (e = work_vec(A, 2, &w2)) ||
      (e = work_vec(A, 3, &w3)) || (e = work_vec(A, 4, &w4)))
    return e;
  MxArgs a;
  a.n = A->n;
  a.rp = A->rp;
  a.ci = A->ci;
  a.va = A->va;
  a.va32 = A->va32;
  a.rowblk = A->rowblk;
  a.b = v.b_dev;
  a.x = v.x_dev;
  a.r64 = r64;
  a.r = reinterpret_cast<float*>(w1);
  a.p = reinterpret_cast<float*>(w2);
  a.ap = reinterpret_cast<float*>(w3);
  a.d = reinterpret_cast<float*>(w4);
  a.partials = A->partials;
  a.st = A->st;
  const int G = A->grid;
  int Ge = A->grid_ew;
  if (!Ge) {
    int sms = 1;
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
    Ge = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, ((int64_t)A->n + 2 * kBlock - 1) / (2 * kBlock)));
  }
  Timer T;
  T.A = A;
  T.on = (o->flags & PK_FLAG_TIMING) != 0;
  T.s = s;
  int launches = 1;
  auto pre = [&](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_OTHER);
    k_mx_residual<<<G, kBlock, 0, cs>>>(a);
    if (t) { t->end(); t->begin(PK_SLOT_OTHER); }
    k_mx_prep<<<Ge, kBlock, 0, cs>>>(a);
    if (t) t->end();
  };
  // the tile engines need FP32 vectors on 16-byte boundaries (the work vectors are);
  // PK_FLAG_NO_TMA selects the thread-per-row kernels
  const bool tma = A->tma_ok && !(o->flags & PK_FLAG_NO_TMA);
  if (tma && (e = mx_tma_setup())) return e;
  const CsrTilesT<float> ct = csr_tiles32_of(A);
  const bool irr = csr_irregular(A);  // some tile needs the grouped or whole-warp rows
  const int Gt = A->grid_tma, Gs = A->grid_stream;
  auto step = [&](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_SPMV_DOTS);
    if (tma) launch_pdl(irr ? k_mx_spmv_tma<true> : k_mx_spmv_tma<false>, Gt, kTileThreads, csr_smem_bytes(), cs, ct, a);
    else k_mx_spmv<<<G, kBlock, 0, cs>>>(a);
    if (t) { t->end(); t->begin(PK_SLOT_UPDATE); }
    if (tma) launch_pdl(k_mx_update_tma, Gs, kTileThreads, stream_smem_bytes<4, float, 2>(), cs, a);
    else k_mx_update<<<Ge, kBlock, 0, cs>>>(a);
    if (t) t->end();
  };
  auto post = [&](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_OTHER);
    k_mx_correct<<<Ge, kBlock, 0, cs>>>(a);
    if (t) t->end();
  };
  const bool graph = o->loop != PK_LOOP_HOST && !T.on;
  if (graph) {
    const void* keys[4] = {v.x_dev, v.b_dev, nullptr, nullptr};
    const int64_t ikeys[4] = {PK_PREC_MIXED, tma ? 1 : 0, 0, 0};
    pk_graph_entry* ge = nullptr;
    if ((e = build_nested_graph(A, 8, keys, ikeys, [&](cudaStream_t cs) { pre(cs, nullptr); },
                                [&](cudaStream_t cs) {
                                  // four inner iterations per graph pass; kernels after the
                                  // inner stop return at once
                                  for (int u = 0; u < (tma ? 4 : 1); ++u) step(cs, nullptr);
                                },
                                [&](cudaStream_t cs) { post(cs, nullptr); }, &ge)))
      return e;
    launch_enable_cond2(A, ge, s);
    PK_CUDA(cudaGetLastError());
    PK_CUDA(cudaGraphLaunch(ge->exec, s));
    launches += 1;
  } else {
    const int every = T.on ? 1 : (o->check_every > 0 ? o->check_every : 16);
    for (;;) {
      pre(s, T.on ? &T : nullptr);
      launches += 2;
      for (;;) {
        for (int k = 0; k < every; ++k) {
          step(s, T.on ? &T : nullptr);
          launches += 2;
        }
        if ((e = T.flush())) return e;
        PK_CUDA(cudaMemcpyAsync(&A->st_host->gm_phase, &A->st->gm_phase, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaMemcpyAsync(&A->st_host->done, &A->st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (A->st_host->gm_phase != 1 || A->st_host->done) break;
      }
      post(s, T.on ? &T : nullptr);
      launches += 1;
      PK_CUDA(cudaGetLastError());
      if ((e = T.flush())) return e;
      PK_CUDA(cudaMemcpyAsync(&A->st_host->done, &A->st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
      PK_CUDA(cudaStreamSynchronize(s));
      if (A->st_host->done) break;
    }
  }
  launch_zero_x(A, v.x_dev, s);
  launches += 1;
  if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
  const DevState* h = A->st_host;
  info->cycles = h->gm_cycle;
  if (graph) info->launches += (int)(passes_of(h) * 2 + (long long)(h->gm_cycle + 1) * 3);
  for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
    info->kernel_count[k] = T.count[k];
    info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (pk_status)info->status;
}

}  // namespace pk
