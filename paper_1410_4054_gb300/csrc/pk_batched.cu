// Batched solves: many independent SPD systems of uneven size in one persistent launch.
//
// The paper's motivation for pipelining is that small and medium systems are bound by launch
// and transfer latency (Sec. 2.1, 4.1), and that transient problems solve many such systems
// (Sec. 1).  Here a persistent grid of thread blocks takes systems from a device work queue
// (largest first); one block runs pipelined CG (Alg. 2) on its system to completion, with the
// two global synchronisations of an iteration done as block-wide reductions, then takes the
// next system.  A system that converges simply leaves the queue, which is the per-system
// convergence mask.  No block ever waits for another block (the queue is one atomic counter).
//
// Two arithmetics: FP64 throughout, and mixed precision -- FP32 SpMV and vector updates with
// FP32 accumulation inside an FP64 iterative-refinement loop whose true residual b - A x, the
// correction x += d and the inner products that set alpha and beta are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "pk_guard.cuh"
#include "pk_tile.cuh"

namespace pk {

struct BatchSys {
  int32_t n, nnz;
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const float* va32;
  const double* b;
  double* x;
  double *r, *p, *ap;           // FP64 work vectors
  float *r32, *p32, *ap32, *d32;  // mixed-precision work vectors
  // the system's bulk-copy tiles (the tile engine path): tiles [0, ntiles) of its handle
  const int32_t* tile_row;
  const int8_t* tile_grp;
  const int16_t* tile_perm;
  const int32_t* tile_z0;
  int32_t ntiles, x_streamed;   // x_streamed: x is 16-byte aligned (bulk copies of x)
  // results
  int32_t iters, status, outer, inner_total;
  double rel_res;
};

// Block-wide sums of NV values, broadcast to every thread.  GB300 issues about two FP64
// operations per clock per SM with a 64-cycle latency, so the sum is done by one warp: every
// thread stages its values in shared memory, each lane of warp 0 adds blockDim/32 of them
// with four interleaved accumulators (fixed order), and a butterfly finishes (both partners
// of a pair add the same two values, so every lane ends with the same bits).
template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV]) {
  __shared__ double buf[NV][1024];
  __shared__ double bc[NV];
  const int lane = threadIdx.x & 31, per = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int m = 0;
      for (; m + 4 <= per; m += 4) {
        a0 += buf[k][(m + 0) * 32 + lane];
        a1 += buf[k][(m + 1) * 32 + lane];
        a2 += buf[k][(m + 2) * 32 + lane];
        a3 += buf[k][(m + 3) * 32 + lane];
      }
      for (; m < per; ++m) a0 += buf[k][m * 32 + lane];
      double t = (a0 + a1) + (a2 + a3);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) bc[k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = bc[k];
}

// Scalars of an iteration decided by thread 0 and broadcast (every FP64 instruction issued
// by all warps of a block, like a division, costs the SM's narrow FP64 pipe).
struct CtaScalars {
  double a, b;
  int status;
};

__device__ __forceinline__ double row_f64(const BatchSys& S, const double* __restrict__ x, int row) {
  const int j0 = __ldg(S.rp + row), j1 = __ldg(S.rp + row + 1);
  double s = 0.0;
  int j = j0;
  for (; j + 4 <= j1; j += 4) {
    int c[4];
    double v[4], xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { c[k] = __ldg(S.ci + j + k); v[k] = __ldg(S.va + j + k); }
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = x[c[k]];
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fma(v[k], xv[k], s);
  }
  for (; j < j1; ++j) s = fma(__ldg(S.va + j), x[__ldg(S.ci + j)], s);
  return s;
}

__device__ __forceinline__ float row_f32(const BatchSys& S, const float* __restrict__ x, int row) {
  const int j0 = __ldg(S.rp + row), j1 = __ldg(S.rp + row + 1);
  float s = 0.0f;
  int j = j0;
  for (; j + 4 <= j1; j += 4) {
    int c[4];
    float v[4], xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { c[k] = __ldg(S.ci + j + k); v[k] = __ldg(S.va32 + j + k); }
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = x[c[k]];
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fmaf(v[k], xv[k], s);
  }
  for (; j < j1; ++j) s = fmaf(__ldg(S.va32 + j), x[__ldg(S.ci + j)], s);
  return s;
}

// Rows computed by groups of G lanes (G = 2, 4 or 8, aligned in the warp; the autotuned
// lanes per row): lane q sums entries j0 + q, j0 + q + G, ... left to right, then the group
// adds by a butterfly over its own lanes.  Every lane of a group walks the same rows, so the
// group is converged at the shuffles.
struct RowGroup {
  int G, q, g0, gs;
  unsigned mask;
};

__device__ __forceinline__ RowGroup row_group(int G) {
  RowGroup g;
  g.G = G;
  g.q = (int)threadIdx.x & (G - 1);
  g.g0 = (int)threadIdx.x / G;
  g.gs = (int)blockDim.x / G;
  g.mask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (((int)threadIdx.x & 31) & ~(G - 1)));
  return g;
}

__device__ __forceinline__ double fma_b(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_b(float a, float b, float c) { return fmaf(a, b, c); }

template <class T>
__device__ __forceinline__ T row_grouped(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                         const T* __restrict__ va, const T* __restrict__ x, int row,
                                         const RowGroup& g) {
  const int j1 = __ldg(rp + row + 1);
  T s = (T)0;
  int j = __ldg(rp + row) + g.q;
  for (; j + 3 * g.G < j1; j += 4 * g.G) {
    int c[4];
    T v[4], xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { c[k] = __ldg(ci + j + k * g.G); v[k] = __ldg(va + j + k * g.G); }
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = x[c[k]];
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fma_b(v[k], xv[k], s);
  }
  for (; j < j1; j += g.G) s = fma_b(__ldg(va + j), x[__ldg(ci + j)], s);
  for (int o = g.G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(g.mask, s, o);
  return s;
}

// Row products of the block's system: one thread per row (G = 1, the plain loop) or a group
// of G lanes per row; f(row, y) runs in the row's first lane.
template <class F>
__device__ __forceinline__ void rows_f64(const BatchSys& S, const double* __restrict__ x, int G, F&& f) {
  if (G == 1) {
    for (int row = threadIdx.x; row < S.n; row += blockDim.x) f(row, row_f64(S, x, row));
  } else {
    const RowGroup g = row_group(G);
    for (int row = g.g0; row < S.n; row += g.gs) {
      const double y = row_grouped(S.rp, S.ci, S.va, x, row, g);
      if (g.q == 0) f(row, y);
    }
  }
}

template <class F>
__device__ __forceinline__ void rows_f32(const BatchSys& S, const float* __restrict__ x, int G, F&& f) {
  if (G == 1) {
    for (int row = threadIdx.x; row < S.n; row += blockDim.x) f(row, row_f32(S, x, row));
  } else {
    const RowGroup g = row_group(G);
    for (int row = g.g0; row < S.n; row += g.gs) {
      const float y = row_grouped(S.rp, S.ci, S.va32, x, row, g);
      if (g.q == 0) f(row, y);
    }
  }
}

// Pipelined CG (Alg. 2) on one system by one block, FP64, G lanes per row.  Returns the status.
__device__ int cta_cg64(BatchSys& S, double tol, int maxit, int G) {
  const int n = S.n, t0 = threadIdx.x, bs = blockDim.x;
  __shared__ CtaScalars sc;
  double v[2] = {0.0, 0.0};
  rows_f64(S, S.x, G, [&](int row, double y) {
    const double bi = S.b[row];
    const double ri = bi - y;
    S.r[row] = ri;
    S.p[row] = ri;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(bi, bi, v[1]);
  });
  cta_sum<2>(v);
  double rr = v[0];
  const double bb = v[1], thr2 = tol * tol * bb;
  S.iters = 0;
  if (t0 == 0) S.rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
  if (!isfinite(rr) || !isfinite(bb)) return PK_ERR_NAN;
  if (bb == 0.0) {
    for (int row = t0; row < n; row += bs) S.x[row] = 0.0;
    S.rel_res = 0.0;
    return PK_OK;
  }
  if (rr <= thr2) return PK_OK;
  if (maxit <= 0) return PK_NOT_CONVERGED;
  for (int it = 0;; ++it) {
    // A p_it with <Ap,Ap>, <p,Ap> -> alpha, beta (Eq. (3))
    v[0] = v[1] = 0.0;
    rows_f64(S, S.p, G, [&](int row, double s) {
      S.ap[row] = s;
      v[0] = fma(s, s, v[0]);
      v[1] = fma(S.p[row], s, v[1]);
    });
    cta_sum<2>(v);
    if (t0 == 0) {
      sc.status = kRunning;
      if (!isfinite(v[0]) || !isfinite(v[1])) sc.status = PK_ERR_NAN;
      else if (v[1] <= 0.0) sc.status = PK_NOT_SPD;
      else {
        sc.a = rr / v[1];
        sc.b = sc.a * sc.a * v[0] / rr - 1.0;
      }
    }
    __syncthreads();
    if (sc.status != kRunning) return sc.status;
    const double alpha = sc.a, beta = sc.b;
    // x, r, p updates with <r,r>
    double w[1] = {0.0};
    for (int row = t0; row < n; row += bs) {
      const double pk = S.p[row];
      S.x[row] = fma(alpha, pk, S.x[row]);
      const double rk = fma(-alpha, S.ap[row], S.r[row]);
      S.r[row] = rk;
      S.p[row] = fma(beta, pk, rk);
      w[0] = fma(rk, rk, w[0]);
    }
    cta_sum<1>(w);
    rr = w[0];
    if (t0 == 0) {
      S.iters = it + 1;
      S.rel_res = sqrt(rr / bb);
      sc.status = kRunning;
      if (!isfinite(rr)) sc.status = PK_ERR_NAN;
      else if (rr <= thr2) sc.status = PK_OK;
      else if (it + 1 >= maxit) sc.status = PK_NOT_CONVERGED;
    }
    __syncthreads();
    if (sc.status != kRunning) return sc.status;
  }
}

// Mixed precision: FP64 refinement around an FP32 pipelined CG whose inner products (and so
// alpha, beta) are accumulated in FP64.  Inner stop: ||r_in|| <= tol_in ||r_outer||.
__device__ int cta_cg_mixed(BatchSys& S, double tol, int maxit, double tol_in, int max_outer, int G) {
  const int n = S.n, t0 = threadIdx.x, bs = blockDim.x;
  __shared__ CtaScalars sc;
  S.iters = 0;
  S.outer = 0;
  S.inner_total = 0;
  double bb = -1.0;
  for (int outer = 0;; ++outer) {
    // FP64 true residual r = b - A x
    double v[2] = {0.0, 0.0};
    rows_f64(S, S.x, G, [&](int row, double y) {
      const double bi = S.b[row];
      const double ri = bi - y;
      S.r[row] = ri;
      v[0] = fma(ri, ri, v[0]);
      v[1] = fma(bi, bi, v[1]);
    });
    cta_sum<2>(v);
    if (bb < 0) bb = v[1];
    const double rr_out = v[0];
    if (t0 == 0) S.rel_res = bb > 0 ? sqrt(rr_out / bb) : 0.0;
    if (!isfinite(rr_out) || !isfinite(bb)) return PK_ERR_NAN;
    if (bb == 0.0) {
      for (int row = t0; row < n; row += bs) S.x[row] = 0.0;
      S.rel_res = 0.0;
      return PK_OK;
    }
    if (rr_out <= tol * tol * bb) return PK_OK;
    if (outer >= max_outer || S.iters >= maxit) return PK_NOT_CONVERGED;
    S.outer = outer + 1;
    // inner FP32 system A d = r / ||r|| (unit right-hand side keeps FP32 in range)
    if (t0 == 0) {
      sc.a = sqrt(rr_out);
      sc.b = 1.0 / sc.a;
    }
    __syncthreads();
    const double scale = sc.a, inv = sc.b;
    FF acc{0.0f, 0.0f};
    for (int row = t0; row < n; row += bs) {
      const float ri = (float)(S.r[row] * inv);
      S.r32[row] = ri;
      S.p32[row] = ri;
      S.d32[row] = 0.0f;
      ff_add_prod(acc, ri, ri);
    }
    double w[1] = {ff_value(acc)};
    cta_sum<1>(w);
    double rr = w[0];
    const double thr_in = tol_in * tol_in * rr;
    const int budget = maxit - S.iters;
    for (int it = 0; it < budget; ++it) {
      FF aa{0.0f, 0.0f}, pa{0.0f, 0.0f};
      rows_f32(S, S.p32, G, [&](int row, float s) {
        S.ap32[row] = s;
        ff_add_prod(aa, s, s);
        ff_add_prod(pa, S.p32[row], s);
      });
      double u[2] = {ff_value(aa), ff_value(pa)};
      cta_sum<2>(u);
      if (t0 == 0) {
        sc.status = kRunning;
        if (!isfinite(u[0]) || !isfinite(u[1])) sc.status = PK_ERR_NAN;
        else if (u[1] <= 0.0) sc.status = PK_NOT_SPD;
        else {
          sc.a = rr / u[1];
          sc.b = sc.a * sc.a * u[0] / rr - 1.0;
        }
      }
      __syncthreads();
      if (sc.status != kRunning) return sc.status;
      const float af = (float)sc.a, bf = (float)sc.b;
      FF racc{0.0f, 0.0f};
      for (int row = t0; row < n; row += bs) {
        const float pk = S.p32[row];
        S.d32[row] = fmaf(af, pk, S.d32[row]);
        const float rk = fmaf(-af, S.ap32[row], S.r32[row]);
        S.r32[row] = rk;
        S.p32[row] = fmaf(bf, pk, rk);
        ff_add_prod(racc, rk, rk);
      }
      double q[1] = {ff_value(racc)};
      cta_sum<1>(q);
      rr = q[0];
      S.iters += 1;
      S.inner_total += 1;
      if (!isfinite(rr)) return PK_ERR_NAN;
      if (rr <= thr_in) break;
    }
    // FP64 correction x += ||r|| d
    for (int row = t0; row < n; row += bs) S.x[row] = fma(scale, (double)S.d32[row], S.x[row]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024, 1) k_batched(BatchSys* sys, int nsys, int* queue, double tol, int maxit, int mixed,
                          double tol_in, int max_outer, int lanes) {
  __shared__ int cur;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) cur = atomicAdd(queue, 1);
    __syncthreads();
    const int k = cur;
    if (k >= nsys) return;
    BatchSys S = sys[k];
    const int st = mixed ? cta_cg_mixed(S, tol, maxit, tol_in, max_outer, lanes) : cta_cg64(S, tol, maxit, lanes);
    if (threadIdx.x == 0) {
      sys[k].iters = S.iters;
      sys[k].status = st;
      sys[k].outer = S.outer;
      sys[k].inner_total = S.inner_total;
      sys[k].rel_res = S.rel_res;
    }
  }
}

// ------------------------------------------------------------------ tile-engine form (FP64)
//
// The same pipelined CG per block, with the block's memory traffic on the warp-specialised
// bulk-copy engines of the single-system kernels: in the SpMV phase the producer warp
// streams the system's CSR tiles (row pointers, values, columns) into shared memory and the
// eight consumer warps compute from there, so no consumer waits on a chain of dependent
// loads per row; in the update phase x, r, p, Ap stream through the same region.  One block
// runs 288 threads and two blocks share an SM.  Every reduction is a fixed-order block sum.

// Fixed-order sum of NV values over all threads of a tile block, broadcast to every thread.
template <int NV>
__device__ __forceinline__ void tile_block_sum(double (&v)[NV]) {
  __shared__ double sm[NV][kTileThreads / 32];
  __shared__ double bc[NV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k][warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < kTileThreads / 32 ? sm[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) bc[k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = bc[k];
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_invalidate(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

constexpr int kBtStream = stream_smem_bytes<4, double, 1>();
constexpr int kBtSmem = kBtStream > csr_smem_bytes() ? kBtStream : csr_smem_bytes();

// Pipelined CG (Alg. 2) on system S by one tile block.  The CSR ring and the vector ring
// overlay one shared-memory region, used by one phase at a time; after each phase thread 0
// invalidates that ring's barriers (their memory then holds the other ring's data).
template <bool IRR>
__device__ int tile_cg64(BatchSys& S, double tol, int maxit, DevState* st, unsigned char* smem) {
  const int n = S.n;
  const bool consumer = threadIdx.x < kConsumers;
  uint64_t* bars_s = reinterpret_cast<uint64_t*>(smem + (size_t)kCsrStages * kStageBytes);
  uint64_t* bars_u = reinterpret_cast<uint64_t*>(smem + (size_t)stream_stages<4, double, 1>() * 4 *
                                                             kStreamRows * sizeof(double));
  auto inval = [&](uint64_t* bars, int count) {
    __syncthreads();
    if (threadIdx.x == 0)
      for (int k = 0; k < count; ++k) mbar_invalidate(bars + k);
  };
  CsrTiles T;
  T.rp = S.rp;
  T.ci = S.ci;
  T.va = S.va;
  T.tile_row = S.tile_row;
  T.blk_tile = nullptr;
  T.tile_grp = S.tile_grp;
  T.tile_perm = S.tile_perm;
  T.tile_z0 = S.tile_z0;
  auto live = []() { return true; };
  // r0 = b - A x0, p0 = r0, <r0,r0>, <b,b>
  double v[2] = {0.0, 0.0};
  csr_tiles_range<IRR>(T, 0, S.ntiles, smem, st, live, BlockVec<double>{S.x}, [&](int row, double y) {
    const double bi = __ldg(S.b + row);
    const double ri = bi - y;
    S.r[row] = ri;
    S.p[row] = ri;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(bi, bi, v[1]);
  });
  if (consumer) fence_proxy_async_global();
  inval(bars_s, 2 * kCsrStages);
  tile_block_sum<2>(v);
  if (__ldcg(&st->timeout)) return PK_TIMEOUT;  // a wait gave up: the sums are incomplete
  double rr = v[0];
  const double bb = v[1], thr2 = tol * tol * bb;
  S.iters = 0;
  S.rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
  if (!isfinite(rr) || !isfinite(bb)) return PK_ERR_NAN;
  if (bb == 0.0) {
    for (int row = threadIdx.x; row < n; row += blockDim.x) S.x[row] = 0.0;
    S.rel_res = 0.0;
    return PK_OK;
  }
  if (rr <= thr2) return PK_OK;
  if (maxit <= 0) return PK_NOT_CONVERGED;
  // update rows [0, ne) through the vector ring: an even count of 16-byte-aligned doubles
  // (every bulk copy a whole number of 16-byte units); an odd last row directly
  const int ne = S.x_streamed ? (n & ~1) : 0;
  __shared__ double s_ab[2];
  __shared__ int s_status;
  for (int it = 0;; ++it) {
    // A p_it with <Ap,Ap>, <p,Ap> -> alpha, beta (Eq. (3))
    v[0] = v[1] = 0.0;
    csr_tiles_range<IRR>(T, 0, S.ntiles, smem, st, live, BlockVec<double>{S.p}, [&](int row, double y) {
      S.ap[row] = y;
      v[0] = fma(y, y, v[0]);
      v[1] = fma(__ldca(S.p + row), y, v[1]);
    });
    if (consumer) fence_proxy_async_global();  // Ap is read back by bulk copies
    inval(bars_s, 2 * kCsrStages);
    tile_block_sum<2>(v);
    if (threadIdx.x == 0) {
      s_status = kRunning;
      if (__ldcg(&st->timeout)) s_status = PK_TIMEOUT;
      else if (!isfinite(v[0]) || !isfinite(v[1])) s_status = PK_ERR_NAN;
      else if (v[1] <= 0.0) s_status = PK_NOT_SPD;
      else {
        s_ab[0] = rr / v[1];
        s_ab[1] = s_ab[0] * s_ab[0] * v[0] / rr - 1.0;
      }
    }
    __syncthreads();
    if (s_status != kRunning) return s_status;
    const double alpha = s_ab[0], beta = s_ab[1];
    // x, r, p updates with <r,r>
    double w[1] = {0.0};
    auto upd = [&](int row, double xk, double rq, double pk, double ak) {
      S.x[row] = fma(alpha, pk, xk);
      const double rk = fma(-alpha, ak, rq);
      S.r[row] = rk;
      S.p[row] = fma(beta, pk, rk);
      w[0] = fma(rk, rk, w[0]);
    };
    if (ne > 0) {
      StreamIn<4> in{{S.x, S.r, S.p, S.ap}};
      stream_tiles<4, 4, double, 1>(in, 0, ne, smem, st, live, [&](int row, const double2* val, int nv) {
        upd(row, val[0].x, val[1].x, val[2].x, val[3].x);
        if (nv == 2) upd(row + 1, val[0].y, val[1].y, val[2].y, val[3].y);
      });
      inval(bars_u, 2 * stream_stages<4, double, 1>());
    }
    for (int row = ne + (int)threadIdx.x; row < n; row += blockDim.x)
      upd(row, __ldca(S.x + row), __ldca(S.r + row), __ldca(S.p + row), __ldca(S.ap + row));
    if (consumer) fence_proxy_async_global();  // x, r, p are read back by bulk copies
    tile_block_sum<1>(w);
    rr = w[0];
    S.iters = it + 1;
    S.rel_res = sqrt(rr / bb);
    if (__ldcg(&st->timeout)) return PK_TIMEOUT;
    if (!isfinite(rr)) return PK_ERR_NAN;
    if (rr <= thr2) return PK_OK;
    if (it + 1 >= maxit) return PK_NOT_CONVERGED;
  }
}

template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_batched_tiles(BatchSys* sys, int nsys, int* queue,
                                                                   double tol, int maxit, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int cur;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) cur = atomicAdd(queue, 1);
    __syncthreads();
    const int k = cur;
    if (k >= nsys) return;
    BatchSys S = sys[k];
    const int status = S.n > 0 ? tile_cg64<IRR>(S, tol, maxit, st, smem) : PK_OK;
    __syncthreads();
    if (threadIdx.x == 0) {
      sys[k].iters = S.iters;
      sys[k].status = status;
      sys[k].outer = 0;
      sys[k].inner_total = 0;
      sys[k].rel_res = S.rel_res;
    }
  }
}

// ------------------------------------------------------------------ host side

struct TuneKey {
  int nsys;
  long long rows, nnz;
  int mixed;
  bool operator<(const TuneKey& o) const {
    return std::tie(nsys, rows, nnz, mixed) < std::tie(o.nsys, o.rows, o.nnz, o.mixed);
  }
};
struct TuneVal {
  int block, per_sm, lanes;  // lanes -1: the tile engine (block 288, 2 per SM); -2: clusters
  int rows_cta;              // cluster engine: rows per CTA it aims for (a power of 2)
};
static std::mutex g_tune_mutex;
static std::map<TuneKey, TuneVal> g_tune;
static TuneVal g_last{512, 2, 1, 0};

// The cluster engine (pk_batched_cluster.cu): classes are (CTA shape, cluster size) pairs.
constexpr int kClSizes = 5;  // clusters of 1, 2, 4, 8, 16 CTAs
constexpr int kClClasses = kBcShapeCount * kClSizes;
constexpr int kClRowsDefault = 2048;

// Class of a system of n rows when the batch aims at rows_cta rows per CTA: the CTA shape
// whose row limit is rows_cta, else the next larger one that holds n on 16 CTAs, with the
// smallest power-of-2 cluster that holds n.  shape * kClSizes + log2(C), or -1.
static int cluster_class(int n, int rows_cta) {
  int s0 = -1;
  for (int sh = 0; sh < kBcShapeCount; ++sh)
    if (batched_cluster_max_rows(sh) == rows_cta) s0 = sh;
  for (int sh = s0; sh >= 0; --sh) {  // shape 0 has the largest row limit
    const long long mx = batched_cluster_max_rows(sh);
    for (int c = 0; c < kClSizes; ++c)
      if (mx << c >= n) return sh * kClSizes + c;
  }
  return -1;
}

// The batch as the cluster engine runs it: systems grouped by class, the classes that hold the
// most rows per cluster first (within a class, largest systems first); one persistent launch
// per class, each class on a stream of its own, so that the classes fill the SMs that the
// others leave free.
struct ClusterPlan {
  std::vector<BatchClSys> sys;  // in launch order
  std::vector<int> order;       // sys[i] is the caller's system order[i]
  int cls[kClClasses];          // class of launch slot j
  int first[kClClasses + 1];    // slot j's systems: [first[j], first[j + 1])
};

static bool plan_clusters(const std::vector<BatchSys>& h, int rows_cta, ClusterPlan& P) {
  const int nsys = (int)h.size();
  // launch slots: classes by rows per cluster (descending), then by shape
  std::vector<int> slots(kClClasses);
  for (int c = 0; c < kClClasses; ++c) slots[c] = c;
  auto held = [](int c) { return (long long)batched_cluster_max_rows(c / kClSizes) << (c % kClSizes); };
  std::stable_sort(slots.begin(), slots.end(), [&](int a, int b) { return held(a) > held(b); });
  int slot_of[kClClasses];
  for (int j = 0; j < kClClasses; ++j) {
    P.cls[j] = slots[j];
    slot_of[slots[j]] = j;
  }
  std::vector<int> sl(nsys);
  for (int k = 0; k < nsys; ++k) {
    const int c = cluster_class(std::max(h[k].n, 1), rows_cta);
    if (c < 0 || batched_cluster_capacity(c / kClSizes, 1 << (c % kClSizes)) <= 0) return false;
    sl[k] = slot_of[c];
  }
  P.order.resize(nsys);
  for (int k = 0; k < nsys; ++k) P.order[k] = k;
  std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int c) {
    return sl[a] != sl[c] ? sl[a] < sl[c] : h[a].nnz + 2LL * h[a].n > h[c].nnz + 2LL * h[c].n;
  });
  P.sys.resize(nsys);
  int count[kClClasses] = {};
  for (int i = 0; i < nsys; ++i) {
    const BatchSys& S = h[P.order[i]];
    P.sys[i] = BatchClSys{S.n, S.rp, S.ci, S.va, S.b, S.x, 0, 0, 0.0};
    ++count[sl[P.order[i]]];
  }
  P.first[0] = 0;
  for (int j = 0; j < kClClasses; ++j) P.first[j + 1] = P.first[j] + count[j];
  return true;
}

static cudaStream_t g_cl_stream[kClClasses];
static cudaEvent_t g_cl_fork, g_cl_join[kClClasses];

static pk_status run_clusters(BatchClSys* dsys, const ClusterPlan& P, int* queues, double tol, int maxit,
                              cudaStream_t s) {
  static bool init = false;
  if (!init) {
    for (int j = 0; j < kClClasses; ++j) {
      PK_CUDA(cudaStreamCreateWithFlags(&g_cl_stream[j], cudaStreamNonBlocking));
      PK_CUDA(cudaEventCreateWithFlags(&g_cl_join[j], cudaEventDisableTiming));
    }
    PK_CUDA(cudaEventCreateWithFlags(&g_cl_fork, cudaEventDisableTiming));
    init = true;
  }
  int hq[kClClasses];
  for (int j = 0; j < kClClasses; ++j) hq[j] = P.first[j];
  PK_CUDA(cudaMemcpyAsync(queues, hq, sizeof(hq), cudaMemcpyHostToDevice, s));
  PK_CUDA(cudaEventRecord(g_cl_fork, s));
  pk_status e = PK_OK;
  for (int j = 0; j < kClClasses; ++j) {
    if (P.first[j] == P.first[j + 1]) continue;
    const int c = P.cls[j];
    PK_CUDA(cudaStreamWaitEvent(g_cl_stream[j], g_cl_fork, 0));
    if (!e)
      e = launch_batched_cluster(c / kClSizes, dsys, P.first[j], P.first[j + 1], queues + j, 1 << (c % kClSizes), tol,
                                 maxit, g_cl_stream[j]);
    PK_CUDA(cudaEventRecord(g_cl_join[j], g_cl_stream[j]));
    PK_CUDA(cudaStreamWaitEvent(s, g_cl_join[j], 0));
  }
  return e;
}

static pk_status run_tiles(BatchSys* dsys, int* dqueue, int nsys, bool irr, double tol, int maxit,
                           DevState* st, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    for (auto k : {k_batched_tiles<false>, k_batched_tiles<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kBtSmem));
    attr = true;
  }
  int sms = 1, dev = 0, occ = 1;
  PK_CUDA(cudaGetDevice(&dev));
  PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, irr ? k_batched_tiles<true> : k_batched_tiles<false>,
                                                        kTileThreads, kBtSmem));
  const int grid = std::max(1, std::min(nsys, sms * std::max(1, std::min(2, occ))));
  PK_CUDA(cudaMemsetAsync(dqueue, 0, sizeof(int), s));
  (irr ? k_batched_tiles<true> : k_batched_tiles<false>)<<<grid, kTileThreads, kBtSmem, s>>>(dsys, nsys, dqueue, tol,
                                                                                              maxit, st);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

static pk_status run_batch(BatchSys* dsys, int* dqueue, int nsys, int block, int per_sm, int lanes,
                           double tol, int maxit, int mixed, cudaStream_t s) {
  int sms = 1, dev = 0;
  PK_CUDA(cudaGetDevice(&dev));
  PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int occ = 1;
  PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched, block, 0));
  const int grid = std::max(1, std::min(nsys, sms * std::max(1, std::min(per_sm, occ))));
  PK_CUDA(cudaMemsetAsync(dqueue, 0, sizeof(int), s));
  k_batched<<<grid, block, 0, s>>>(dsys, nsys, dqueue, tol, maxit, mixed, 1e-4, 20, lanes);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status ensure_fp32_values(pk_csr* A, cudaStream_t s);  // pk_mixed.cu

pk_status batched_solve(int32_t nsys, pk_csr* const* A, const double* const* b, double* const* x,
                        const pk_opts* o, pk_info* infos, cudaStream_t s) {
  if (nsys < 0 || (nsys > 0 && (!A || !b || !x)) || !o) { set_error("bad batched arguments"); return PK_ERR_ARG; }
  if (!(o->tol >= 0.0) || o->maxit < 0) { set_error("tol must be >= 0 and maxit >= 0"); return PK_ERR_ARG; }
  if (o->precond != PK_PRECOND_NONE) { set_error("the batched solver has no preconditioner"); return PK_ERR_ARG; }
  if (o->flags & PK_FLAG_SELL) { set_error("PK_FLAG_SELL applies to pipelined FP64 CG"); return PK_ERR_ARG; }
  if (o->flags & PK_FLAG_CGS2) { set_error("PK_FLAG_CGS2 applies to GMRES"); return PK_ERR_ARG; }
  if (nsys == 0) return PK_OK;
  const int mixed = o->precision == PK_PREC_MIXED;
  pk_status e;
  std::vector<BatchSys> h(nsys);
  long long rows = 0, nnz = 0;
  bool tiles_ok = !mixed, irr = false;  // every system on the tile engine (FP64 only)
  for (int k = 0; k < nsys; ++k) {
    pk_csr* M = A[k];
    if (!M || (M->n > 0 && (!b[k] || !x[k]))) { set_error("NULL system in batch"); return PK_ERR_ARG; }
    BatchSys& S = h[k];
    memset(&S, 0, sizeof(S));
    S.n = M->n;
    S.nnz = M->nnz;
    S.rp = M->rp;
    S.ci = M->ci;
    S.va = M->va;
    S.b = b[k];
    S.x = x[k];
    S.tile_row = M->tile_row;
    S.tile_grp = M->tile_grp;
    S.tile_perm = M->tile_perm;
    S.tile_z0 = M->tile_z0;
    S.ntiles = M->ntiles;
    S.x_streamed = ((uintptr_t)x[k] & 15) == 0;
    if (M->n > 0 && !M->tma_ok) tiles_ok = false;
    if (M->n > 0 && csr_irregular(M)) irr = true;
    if (M->n > 0) {
      if ((e = work_vec(M, 0, &S.r)) || (e = work_vec(M, 1, &S.p)) || (e = work_vec(M, 2, &S.ap))) return e;
      if (mixed) {
        if ((e = ensure_fp32_values(M, s))) return e;
        S.va32 = M->va32;
        // FP32 vectors live in the FP64 work slots 3..6 (each holds 2n floats)
        double *w3, *w4, *w5, *w6;
        if ((e = work_vec(M, 3, &w3)) || (e = work_vec(M, 4, &w4)) || (e = work_vec(M, 5, &w5)) ||
            (e = work_vec(M, 6, &w6)))
          return e;
        S.r32 = reinterpret_cast<float*>(w3);
        S.p32 = reinterpret_cast<float*>(w4);
        S.ap32 = reinterpret_cast<float*>(w5);
        S.d32 = reinterpret_cast<float*>(w6);
      }
    }
    rows += M->n;
    nnz += M->nnz;
  }
  // largest systems first: the queue then ends with short jobs (better load balance)
  std::vector<int> order(nsys);
  for (int k = 0; k < nsys; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return h[a].nnz + 2LL * h[a].n > h[c].nnz + 2LL * h[c].n; });
  std::vector<BatchSys> hs(nsys);
  for (int k = 0; k < nsys; ++k) hs[k] = h[order[k]];
  BatchSys* dsys = nullptr;
  const size_t sys_bytes = (sizeof(BatchSys) * nsys + 255) & ~size_t(255);
  const size_t cl_bytes = (sizeof(BatchClSys) * nsys + 255) & ~size_t(255);
  const size_t bytes = sys_bytes + 256 + sizeof(DevState) + 256 + cl_bytes;
  PK_CUDA(cudaMallocAsync((void**)&dsys, bytes, s));
  // work queues: [0] the row and tile engines, [1 ..] the cluster engine's classes
  int* dqueue = reinterpret_cast<int*>(reinterpret_cast<char*>(dsys) + sys_bytes);
  // the tile engine's bounded waits read their limit and record a timeout here
  DevState* dst = reinterpret_cast<DevState*>(reinterpret_cast<char*>(dsys) + sys_bytes + 256);
  BatchClSys* dcl = reinterpret_cast<BatchClSys*>(reinterpret_cast<char*>(dsys) + bytes - cl_bytes);
  DevState hst;
  memset(&hst, 0, sizeof(hst));
  hst.wait_ns = o->wait_ns > 0 ? (unsigned long long)o->wait_ns : 2000000000ull;
  hst.stall_test = (o->flags & PK_FLAG_TEST_STALL) ? 1 : 0;
  PK_CUDA(cudaMemcpyAsync(dsys, hs.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, s));
  PK_CUDA(cudaMemcpyAsync(dst, &hst, sizeof(DevState), cudaMemcpyHostToDevice, s));

  // lanes per row: given, else from the batch's mean row length (one thread up to 12
  // nonzeros per row, then 2, 4, 8 lanes), else tuned
  if (o->lanes < -2 || (o->lanes > 2 && o->lanes != 4 && o->lanes != 8)) {
    set_error("lanes per row must be 0 (automatic), 1, 2, 4 or 8, -1 (the tile engine) or -2 (the cluster engine)");
    return PK_ERR_ARG;
  }
  if (o->lanes == -1 && !tiles_ok) {
    set_error("lanes = -1: the tile engine runs FP64 batches whose systems all have CSR tiles");
    return PK_ERR_ARG;
  }
  ClusterPlan plan;
  const int max_cl_rows = 16 * batched_cluster_max_rows(0);
  bool clusters_ok = !mixed;
  for (int k = 0; k < nsys && clusters_ok; ++k) clusters_ok = h[k].n <= max_cl_rows;
  if (clusters_ok) clusters_ok = plan_clusters(h, kClRowsDefault, plan);
  if (o->lanes == -2 && !clusters_ok) {
    set_error("lanes = -2: the cluster engine runs FP64 batches of systems of at most 65536 rows");
    return PK_ERR_ARG;
  }
  const double mean_len = rows > 0 ? (double)nnz / (double)rows : 0.0;
  const int lanes_auto = mean_len <= 12 ? 1 : mean_len <= 24 ? 2 : mean_len <= 48 ? 4 : 8;
  // lanes -1: the tile engine; -2: the cluster engine; otherwise the row kernel with the
  // given (or automatic) lanes
  TuneVal cfg = o->lanes == -1   ? TuneVal{kTileThreads, 2, -1, 0}
                : o->lanes == -2 ? TuneVal{kClRowsDefault / 8, 4096 / kClRowsDefault, -2, kClRowsDefault}
                                 : TuneVal{512, 2, o->lanes ? o->lanes : lanes_auto, 0};
  const TuneKey key{nsys, rows, nnz, mixed};
  bool have = false;
  if (o->lanes == 0) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { cfg = it->second; have = true; }
  }
  if (have && ((cfg.lanes == -1 && !tiles_ok) || (cfg.lanes == -2 && !clusters_ok))) {
    cfg = TuneVal{512, 2, lanes_auto, 0};  // tuned on handles that allowed that engine
    have = false;
  }
  if (!have && o->lanes >= 0 && (o->flags & PK_FLAG_AUTOTUNE)) {
    // autotuner: time every candidate engine and shape on the whole batch solved to the
    // caller's tol and maxit, from x as given (restored afterwards), so that the spread of
    // the systems' iteration counts (which decides how the engines balance their load) is
    // part of the measurement; lanes per row beyond one only for rows of more than 8 nonzeros
    // on average, and only the given number when the caller fixes it
    std::vector<double*> xsave(nsys, nullptr);
    for (int k = 0; k < nsys; ++k) {
      if (!h[k].n) continue;
      PK_CUDA(cudaMallocAsync((void**)&xsave[k], sizeof(double) * h[k].n, s));
      PK_CUDA(cudaMemcpyAsync(xsave[k], h[k].x, sizeof(double) * h[k].n, cudaMemcpyDeviceToDevice, s));
    }
    cudaEvent_t a0, a1;
    PK_CUDA(cudaEventCreate(&a0));
    PK_CUDA(cudaEventCreate(&a1));
    // every timed run starts from x as given (a run to tolerance changes it)
    auto restore = [&]() -> pk_status {
      for (int k = 0; k < nsys; ++k)
        if (xsave[k]) PK_CUDA(cudaMemcpyAsync(h[k].x, xsave[k], sizeof(double) * h[k].n, cudaMemcpyDeviceToDevice, s));
      return PK_OK;
    };
    float best = 1e30f;
    const int blocks[] = {128, 256, 512, 1024};
    const int per[] = {1, 2, 4, 8};
    std::vector<int> lane_set;
    if (o->lanes) lane_set.push_back(o->lanes);
    else if (mean_len > 8) lane_set = {1, 2, 4, 8};
    else lane_set.push_back(1);
    if (tiles_ok && o->lanes == 0) {  // the tile engine is one more candidate
      for (int rep = 0; rep < 2; ++rep) {
        if ((e = restore())) return e;
        PK_CUDA(cudaEventRecord(a0, s));
        if ((e = run_tiles(dsys, dqueue, nsys, irr, o->tol, o->maxit, dst, s))) return e;
        PK_CUDA(cudaEventRecord(a1, s));
        PK_CUDA(cudaEventSynchronize(a1));
        float ms = 0;
        PK_CUDA(cudaEventElapsedTime(&ms, a0, a1));
        if (rep == 1 && ms < best) { best = ms; cfg = TuneVal{kTileThreads, 2, -1, 0}; }
      }
    }
    if (clusters_ok && o->lanes == 0) {  // the cluster engine at 1024, 2048, 4096 rows per CTA
      for (int rc = 1024; rc <= 4096; rc *= 2) {
        ClusterPlan P;
        if (!plan_clusters(h, rc, P)) continue;
        PK_CUDA(cudaMemcpyAsync(dcl, P.sys.data(), sizeof(BatchClSys) * nsys, cudaMemcpyHostToDevice, s));
        for (int rep = 0; rep < 2; ++rep) {
          if ((e = restore())) return e;
          PK_CUDA(cudaEventRecord(a0, s));
          if ((e = run_clusters(dcl, P, dqueue + 1, o->tol, o->maxit, s))) return e;
          PK_CUDA(cudaEventRecord(a1, s));
          PK_CUDA(cudaEventSynchronize(a1));
          float ms = 0;
          PK_CUDA(cudaEventElapsedTime(&ms, a0, a1));
          if (rep == 1 && ms < best) { best = ms; cfg = TuneVal{rc / 8, 4096 / rc, -2, rc}; }
        }
      }
    }
    for (int ln : lane_set) {
      for (int bsz : blocks) {
        for (int ps : per) {
          if (bsz * ps > 2048) continue;
          for (int rep = 0; rep < 2; ++rep) {
            if ((e = restore())) return e;
            PK_CUDA(cudaEventRecord(a0, s));
            if ((e = run_batch(dsys, dqueue, nsys, bsz, ps, ln, o->tol, o->maxit, mixed, s))) return e;
            PK_CUDA(cudaEventRecord(a1, s));
            PK_CUDA(cudaEventSynchronize(a1));
            float ms = 0;
            PK_CUDA(cudaEventElapsedTime(&ms, a0, a1));
            if (rep == 1 && ms < best) { best = ms; cfg = TuneVal{bsz, ps, ln, 0}; }
          }
        }
      }
    }
    if ((e = restore())) return e;  // the solve itself starts from x as given
    for (int k = 0; k < nsys; ++k) if (xsave[k]) PK_CUDA(cudaFreeAsync(xsave[k], s));
    cudaEventDestroy(a0);
    cudaEventDestroy(a1);
    if (o->lanes == 0) {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune[key] = cfg;
    }
  }
  g_last = cfg;
  cudaEvent_t e0, e1;
  PK_CUDA(cudaEventCreate(&e0));
  PK_CUDA(cudaEventCreate(&e1));
  if (cfg.lanes == -2) {
    if (cfg.rows_cta != kClRowsDefault && !plan_clusters(h, cfg.rows_cta, plan)) {
      set_error("cluster engine: no plan for the tuned rows per CTA");
      return PK_ERR_ARG;
    }
    PK_CUDA(cudaMemcpyAsync(dcl, plan.sys.data(), sizeof(BatchClSys) * nsys, cudaMemcpyHostToDevice, s));
  }
  PK_CUDA(cudaEventRecord(e0, s));
  if (cfg.lanes == -2) {
    if ((e = run_clusters(dcl, plan, dqueue + 1, o->tol, o->maxit, s))) return e;
  } else if (cfg.lanes == -1) {
    if ((e = run_tiles(dsys, dqueue, nsys, irr, o->tol, o->maxit, dst, s))) return e;
  } else if ((e = run_batch(dsys, dqueue, nsys, cfg.block, cfg.per_sm, cfg.lanes, o->tol, o->maxit, mixed, s))) {
    return e;
  }
  PK_CUDA(cudaEventRecord(e1, s));
  PK_CUDA(cudaMemcpyAsync(hs.data(), dsys, sizeof(BatchSys) * nsys, cudaMemcpyDeviceToHost, s));
  if (cfg.lanes == -2)
    PK_CUDA(cudaMemcpyAsync(plan.sys.data(), dcl, sizeof(BatchClSys) * nsys, cudaMemcpyDeviceToHost, s));
  PK_CUDA(cudaFreeAsync(dsys, s));
  PK_CUDA(cudaStreamSynchronize(s));
  float ms = 0;
  PK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cfg.lanes == -2) {  // the cluster engine's results, back in the row engine's order
    std::vector<int> pos(nsys);
    for (int k = 0; k < nsys; ++k) pos[order[k]] = k;
    for (int i = 0; i < nsys; ++i) {
      BatchSys& S = hs[pos[plan.order[i]]];
      S.iters = plan.sys[i].iters;
      S.status = plan.sys[i].status;
      S.outer = 0;
      S.rel_res = plan.sys[i].rel_res;
    }
  }
  pk_status worst = PK_OK;
  for (int k = 0; k < nsys; ++k) {
    const BatchSys& S = hs[k];
    const int orig = order[k];
    if (infos) {
      pk_info& I = infos[orig];
      I = pk_info{};
      I.iters = S.iters;
      I.status = S.n ? S.status : PK_OK;
      I.cycles = S.outer;
      I.launches = 1;
      I.rel_res_est = S.rel_res;
      I.rel_res_true = mixed ? S.rel_res : -1.0;
      I.solve_ms = ms;
    }
    if (S.n && S.status != PK_OK && worst == PK_OK) worst = (pk_status)S.status;
  }
  return worst;
}

}  // namespace pk

extern "C" pk_status pk_batched_solve(int32_t nsys, pk_csr* const* A, const double* const* b,
                                      double* const* x, const pk_opts* opts, pk_info* infos,
                                      void* stream) {
  return pk::guarded([&] { return pk::batched_solve(nsys, A, b, x, opts, infos, (cudaStream_t)stream); });
}

extern "C" pk_status pk_batched_last_config(int32_t* block, int32_t* blocks_per_sm) {
  if (!block || !blocks_per_sm) return PK_ERR_ARG;
  *block = pk::g_last.block;
  *blocks_per_sm = pk::g_last.per_sm;
  return PK_OK;
}

extern "C" pk_status pk_batched_last_lanes(int32_t* lanes) {
  if (!lanes) return PK_ERR_ARG;
  *lanes = pk::g_last.lanes;
  return PK_OK;
}
