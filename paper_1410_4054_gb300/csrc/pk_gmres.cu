// Restarted simpler GMRES(m) with classical Gram-Schmidt (Walker-Zhou), pipelined form
// (Alg. 6) and classical form (Alg. 5), fully device resident.
//
// One cycle (Sec. 3.3):
//   START  r = b - A x (true residual) with the first stages of <r,r> and <b,b>; last block:
//          rho0 = ||r||, convergence test at the cycle boundary, v_0 <- r.
//   SCALE  v_0 = r / rho0.
//   step i = 1..k (k <= m):
//     K-GM-1  v_i = A v_{i-1} with the first stage of <v_{i-1}, v_i>      -> R_{i-1,i}
//     K-GM-2  first stages of <v_j, v_i>, j = 1..i-2 (one pass over the basis) -> R_{j,i}
//     K-GM-3  v_i -= sum_{j<i} R_{j,i} v_j with the first stage of ||v_i||^2 -> R_{i,i}
//     K-GM-4  v_i /= R_{i,i} with the first stage of xi_i = <v_0, v_i>; last block: residual
//             estimate rho0 sqrt(1 - sum xi^2) and the end-of-cycle decision.
//   END    R eta = xi by back-substitution (every block, redundantly) and
//          x += rho0 (eta_1 v_0 + sum_{i>=2} eta_i v_{i-1}).
// The classical form replaces K-GM-4 by a normalisation kernel, xi_i = <r, v_i>, the residual
// update r -= xi_i v_i and ||r|| as separate kernels (r is only monitored, R12).
// PK_FLAG_CGS2 applies Gram-Schmidt twice per step: K-GM-3 without the norm, then K-GM-2
// for c_j = <v_j, v_i>, j = 1 .. i-1, and K-GM-3 again with v_i -= sum c_j v_j,
// R_{j,i} += c_j and ||v_i|| (two more launches per step).
// PK_FLAG_GM_SHIFT, the shift-invariant three-kernel form (Sec. 3.3): A v_{i-1} and
// w = (A - sigma_i I) v_{i-1} have the same part orthogonal to v_1 .. v_{i-1}, so its norm is
// R_{i,i}^2 = <w,w> - sum_{j<i-1} R_{j,i}^2 - (R_{i-1,i} - sigma_i)^2.  K-GM-1 adds the first
// stage of <w, w> to its product; K-GM-2 as above; K-GM-3 takes R_{i,i} from the identity
// (every block, from the same values in the same order), writes
// v_i = (A v_{i-1} - sum_j R_{j,i} v_j) / R_{i,i} and forms the first stage of
// xi_i = <v_0, v_i>, so K-GM-4 is not needed.  sigma_1 = 0, sigma_{i+1} = <v_{i-1}, A v_{i-1}>
// (the Rayleigh quotient that K-GM-1 forms anyway).  The identity is trusted while
// R_{i,i}^2 > 1e-8 <w,w>; otherwise the cycle ends before step i.
// The graph is an outer WHILE loop over cycles around an inner WHILE loop over steps.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pk_guard.cuh"
#include "pk_tile.cuh"

namespace pk {

enum { GM_START = 0, GM_STEP = 1, GM_END = 2 };
constexpr int kGmMax = 64;           // largest restart length
constexpr int kRld = kGmMax + 1;     // leading dimension of R in device scratch
constexpr int kXiOff = kRld * kRld;  // xi after R
// A cycle ends once the squared relative residual estimate 1 - sum xi^2 (pipelined) or
// ||r~||^2 (classical) is <= this floor: below it the estimate is rounding (a difference of
// O(1) terms accumulated over up to 64 steps, with classical Gram-Schmidt's loss of
// orthogonality on top), and the true residual at the restart decides.
constexpr double kGmEstFloor = 1e-12;
// Three-kernel form: R_{i,i}^2 = <w,w> - sum R'^2 is used only above this fraction of <w,w>.
constexpr double kGmShiftFloor = 1e-8;

struct GmArgs {
  int n, ld;
  double* V;         // basis v_0..v_m, column j at V + j * ld
  double* R;         // R[j * kRld + i]
  double* xi;        // xi[i]
  double* C;         // CGS2: second-pass coefficients c_j, j = 1 .. i-1
  double* r;         // classical form: the monitored residual
  const double* b;
  double* x;
  double* partials;
  DevState* st;
};

__device__ __forceinline__ void cond2_set(DevState* st, unsigned v) {
  if (st->use_cond) cudaGraphSetConditional(st->cond2, v);
}

__device__ __forceinline__ void gm_finish(DevState* st, int status) {
  finish(st, status);
  cond2_set(st, 0u);
}

__device__ __forceinline__ bool gm_step_live(const DevState* st) {
  return !state_done(st) && __ldcg(&st->gm_phase) == GM_STEP;
}

// START: r = b - A x into v_0, <r,r>, <b,b>; cycle-boundary tests.
template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_gm_start(CsrTiles T, GmArgs g) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = g.st;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long* c = reinterpret_cast<long long*>(&st->s[6]);
    *c += 1;  // cycles started (launch accounting)
  }
  double* r = g.V;
  double v[2] = {0.0, 0.0};
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return !state_done(st); }, (const double*)g.x,
                              [&](int row, double y) {
    const double bi = __ldg(g.b + row), q = bi - y;
    r[row] = q;
    v[0] = fma(q, q, v[0]);
    v[1] = fma(bi, bi, v[1]);
  });
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && st->use_cond) {
      cudaGraphSetConditional(st->cond, 0u);
      cudaGraphSetConditional(st->cond2, 0u);
    }
    return;
  }
  tile_block_partials<2>(v, g.partials);
  if (arrive_last(&st->counter)) {
    double t[2];
    final_sums<2>(g.partials, t);
    if (threadIdx.x == 0) {
      if (st->gm_cycle == 0) {
        const double tol = st->thr2;
        st->bb = t[1];
        st->thr2 = tol * tol * t[1];
      }
      st->rr = t[0];
      if (__ldcg(&st->timeout)) gm_finish(st, PK_TIMEOUT);
      else if (!isfinite(t[0]) || !isfinite(t[1])) gm_finish(st, PK_ERR_NAN);
      else if (st->bb == 0.0) { st->zero_x = 1; st->rr = 0.0; gm_finish(st, PK_OK); }
      else if (t[0] <= st->thr2) gm_finish(st, PK_OK);
      else if (st->iter >= st->maxit) gm_finish(st, PK_NOT_CONVERGED);
      else if (st->gm_cycle > 0 && st->gm_k == 0) gm_finish(st, PK_BREAKDOWN);
      else {
        st->s[0] = sqrt(t[0]);  // rho0
        st->s[3] = 1.0 / st->s[0];  // once here, not in every thread of the scaling kernel
        st->s[1] = 0.0;         // sum of xi^2
        st->s[2] = 0.0;         // three-kernel form: sigma_1
        st->gm_i = 1;
        st->gm_k = 0;
        st->gm_phase = GM_STEP;
        cond2_set(st, 1u);
      }
      st->counter = 0;
    }
  }
}

// SCALE: v_0 = r / rho0 (also the classical form's monitored residual r = v_0).
__global__ void __launch_bounds__(kTileThreads, 2) k_gm_scale(GmArgs g) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = g.st;
  int r0, r1;
  ew_range(g.n, r0, r1);
  double inv = 0.0;
  double* v0 = g.V;
  double* rc = g.r;
  StreamIn<1> in{{v0}};
  stream_tiles<1, 1>(in, r0, r1, smem, st, [&]() {
    inv = __ldcg(&st->s[3]);
    return gm_step_live(st);
  }, [&](int row, const double2* val, int nv) {
    double2 w = val[0];
    w.x *= inv;
    w.y *= inv;
    if (nv == 2) {
      st2(v0 + row, w);
      if (rc) st2(rc + row, w);
    } else {
      v0[row] = w.x;
      if (rc) rc[row] = w.x;
    }
  });
}

// K-GM-1: v_i = A v_{i-1} and the first stage of <v_{i-1}, v_i> (i >= 2).
// SHIFT (three-kernel form): also the first stage of <w, w>, w = v_i - sigma_i v_{i-1}; the
// last block keeps <w, w> and sigma_{i+1} = <v_{i-1}, A v_{i-1}>.
template <bool IRR, bool SHIFT>
__global__ void __launch_bounds__(kTileThreads, 2) k_gm1(CsrTiles T, GmArgs g) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = g.st;
  count_pass(st);
  const int i = __ldcg(&st->gm_i);
  const double sigma = SHIFT ? __ldcg(&st->s[2]) : 0.0;
  const double* vp = g.V + (size_t)(i - 1) * g.ld;
  double* vi = g.V + (size_t)i * g.ld;
  constexpr int NV = SHIFT ? 2 : 1;
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  const bool live = csr_tiles<IRR>(T, smem, st, [&]() { return gm_step_live(st); }, vp,
                              [&](int row, double y) {
    const double p = __ldg(vp + row);
    vi[row] = y;
    v[0] = fma(p, y, v[0]);
    if (SHIFT) {
      const double w = fma(-sigma, p, y);
      v[NV - 1] = fma(w, w, v[NV - 1]);
    }
  });
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<NV>(v, g.partials);
  if (arrive_last(&st->counter)) {
    double t[NV];
    final_sums<NV>(g.partials, t);
    if (threadIdx.x == 0) {
      if (i >= 2) g.R[(i - 1) * kRld + i] = t[0];
      if (SHIFT) {
        st->s[5] = t[NV - 1];  // <w, w>
        st->s[4] = t[0];       // sigma_{i+1} = <v_{i-1}, A v_{i-1}> (s[4] is K-GM-4's otherwise)
      }
      st->counter = 0;
    }
  }
}

// ---------------------------------------------------------------- Gram-Schmidt streaming
// K-GM-2 and K-GM-3 read i+1 basis columns per step and do one FP64 FMA per element read.
// On GB300 a warp that waits for its own loads starves both HBM and the narrow FP64 pipe, so
// both kernels stream the basis through shared memory: one producer warp copies 256-row
// tiles of up to kBsVecs columns with cp.async.bulk into a kBsStages-deep ring (completion on
// mbarriers, every wait bounded by 2 s -> PK_TIMEOUT), and eight consumer warps, one row per
// thread, do the FMAs from shared memory with independent accumulators.

constexpr int kBsRows = kConsumers;  // rows per tile: one per consumer thread
constexpr int kBsCols = 16;          // basis columns per stage
constexpr int kBsVecs = kBsCols + 1; // + v_i
constexpr int kBsStages = 3;
constexpr int kBsSmem = kBsStages * kBsVecs * kBsRows * 8 + 2 * kBsStages * 8;

struct BasisRing {
  double* buf;      // [kBsStages][kBsVecs][kBsRows]
  uint64_t* full;   // [kBsStages]
  uint64_t* empty;  // [kBsStages]
  __device__ double* slot(int s, int k) const { return buf + ((size_t)s * kBsVecs + k) * kBsRows; }
};

__device__ __forceinline__ BasisRing basis_ring(unsigned char* smem) {
  BasisRing R;
  R.buf = reinterpret_cast<double*>(smem);
  R.full = reinterpret_cast<uint64_t*>(smem + (size_t)kBsStages * kBsVecs * kBsRows * 8);
  R.empty = R.full + kBsStages;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kBsStages; ++s) {
      mbar_init(&R.full[s], 1);
      mbar_init(&R.empty[s], kConsumerWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  return R;
}

// Producer loop (one lane): stage q = 0 .. nq-1 copies the vectors that cols(q, ptrs) lists,
// rows [row0(q), row0(q) + rows(q)) rounded up to whole 16-byte units (the basis columns are
// padded, so the rounding stays inside them).  Returns false after a timed-out wait.
template <class Plan>
__device__ __forceinline__ bool basis_produce(const BasisRing& R, int nq, DevState* st, Plan&& plan) {
  int issued = 0;
  bool ok = true;
  for (int q = 0; q < nq; ++q) {
    const int s = q % kBsStages;
    if (q >= kBsStages && !mbar_wait_st(&R.empty[s], ((q / kBsStages) - 1) & 1, st)) { ok = false; break; }
    const double* src[kBsVecs];
    int row0, rows, nv;
    plan(q, src, row0, rows, nv);
    const uint32_t bytes = (uint32_t)(((rows + 1) & ~1) * 8);
    int cnt = 0;
    for (int k = 0; k < kBsVecs; ++k) cnt += src[k] != nullptr;
    mbar_expect_tx(&R.full[s], bytes * cnt);
    for (int k = 0; k < kBsVecs; ++k)
      if (src[k]) bulk_load(R.slot(s, k), src[k] + row0, bytes, &R.full[s]);
    issued = q + 1;
    (void)nv;
  }
  for (int q = max(0, issued - kBsStages); q < issued; ++q)
    if (!mbar_wait(&R.full[q % kBsStages], (q / kBsStages) & 1)) { ok = false; break; }
  if (!ok) report_timeout(st);
  return ok;
}

// Named barrier over the consumer warps only (the producer warp does not take part).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kConsumers) : "memory");
}

// Per-row work of one stage with the column count a compile-time constant: a predicated-off
// FP64 instruction still occupies GB300's narrow FP64 pipe, so the loops below must not run
// over the full kBsCols with a guard.
template <int NC>
__device__ __forceinline__ void gm2_row(const BasisRing& R, int s, int row, double w,
                                        double (&acc)[kBsCols]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = fma(R.slot(s, 1 + c)[row], w, acc[c]);
}

template <int NC>
__device__ __forceinline__ double gm3_row(const BasisRing& R, int s, int row, const double* cf,
                                          double w) {
#pragma unroll
  for (int c = 0; c < NC; ++c) w = fma(-cf[c], R.slot(s, 1 + c)[row], w);
  return w;
}

#define PK_GM_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) \
  X(14) X(15) X(16)

// K-GM-2: partial <v_j, v_i> for j = 1 .. i-2 (Sec. 3.3, Alg. 6), column groups of kBsCols
// streamed one after the other (v_i with every group).  Each consumer thread keeps one
// accumulator per column of the group; the warp's accumulators are reduced across the lanes
// by recursive halving (16 shuffle-adds per lane), then over the warps in a fixed order.
// pass = 1 (CGS2): j = 1 .. i-1 into C.
__global__ void __launch_bounds__(kTileThreads, 2) k_gm2(GmArgs g, int pass) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = g.st;
  if (!gm_step_live(st)) return;
  const int i = __ldcg(&st->gm_i);
  const int nj = pass ? i - 1 : i - 2;
  if (nj <= 0) return;
  int r0, r1;
  ew_range(g.n, r0, r1);
  const int ntiles = r1 > r0 ? (r1 - r0 + kBsRows - 1) / kBsRows : 0;
  const int ngroups = (nj + kBsCols - 1) / kBsCols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* vi = g.V + (size_t)i * g.ld;
  const BasisRing R = basis_ring(smem);
  __shared__ double red[kConsumerWarps][kBsCols];
  if (warp == kConsumerWarps) {
    if (lane == 0)
      basis_produce(R, ntiles * ngroups, st, [&](int q, const double** src, int& row0, int& rows, int& nv) {
        const int grp = q / ntiles, t = q % ntiles;
        const int j0 = 1 + grp * kBsCols, nc = min(kBsCols, nj - j0 + 1);
        row0 = r0 + t * kBsRows;
        rows = min(kBsRows, r1 - row0);
        nv = nc + 1;
        src[0] = vi;
        for (int c = 0; c < kBsCols; ++c) src[1 + c] = c < nc ? g.V + (size_t)(j0 + c) * g.ld : nullptr;
      });
  } else {
    bool ok = true;
    for (int grp = 0; grp < ngroups; ++grp) {
      const int j0 = 1 + grp * kBsCols, nc = min(kBsCols, nj - j0 + 1);
      double acc[kBsCols];
#pragma unroll
      for (int c = 0; c < kBsCols; ++c) acc[c] = 0.0;
      for (int t = 0; t < ntiles && ok; ++t) {
        const int q = grp * ntiles + t, s = q % kBsStages;
        if (!mbar_wait_st(&R.full[s], (q / kBsStages) & 1, st)) { report_timeout(st); ok = false; break; }
        const int rows = min(kBsRows, r1 - (r0 + t * kBsRows));
        if ((int)threadIdx.x < rows) {
          const double w = R.slot(s, 0)[threadIdx.x];
          switch (nc) {
#define PK_GM2_CASE(N) \
  case N: gm2_row<N>(R, s, threadIdx.x, w, acc); break;
            PK_GM_CASES(PK_GM2_CASE)
#undef PK_GM2_CASE
            default: break;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[s]);
      }
      // recursive halving over the lanes: after offsets 16, 8, 4, 2 lane l holds column
      // (l >> 1) & 15 summed over 16 lanes; offset 1 adds the last pair (a + b == b + a)
      double h8[8], h4[4], h2[2], h1;
      {
        const bool up = lane & 16;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const double keep = up ? acc[c + 8] : acc[c], send = up ? acc[c] : acc[c + 8];
          h8[c] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
      }
      {
        const bool up = lane & 8;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double keep = up ? h8[c + 4] : h8[c], send = up ? h8[c] : h8[c + 4];
          h4[c] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
      }
      {
        const bool up = lane & 4;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const double keep = up ? h4[c + 2] : h4[c], send = up ? h4[c] : h4[c + 2];
          h2[c] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
      }
      {
        const bool up = lane & 2;
        const double keep = up ? h2[1] : h2[0], send = up ? h2[0] : h2[1];
        h1 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
      }
      h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
      if ((lane & 1) == 0) red[warp][(lane >> 1) & 15] = h1;
      consumers_sync();
      if ((int)threadIdx.x < nc) {
        double tsum = 0.0;
#pragma unroll
        for (int w = 0; w < kConsumerWarps; ++w) tsum += red[w][threadIdx.x];
        g.partials[(size_t)(j0 + threadIdx.x - 1) * gridDim.x + blockIdx.x] = tsum;
      }
      consumers_sync();
    }
  }
  if (arrive_last(&st->counter)) {
    const int G = gridDim.x;
    for (int j = 1 + warp; j <= nj; j += kTileThreads / 32) {  // one warp per column
      // the slots lane, lane + 32, ... added in order; loads issued 8 at a time (one L2 round
      // trip per batch instead of one per slot)
      const double* pj = g.partials + (size_t)(j - 1) * G;
      double t = 0.0;
      for (int base = lane; base < G; base += 32 * 8) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = base + 32 * q < G ? ld_cg(pj + base + 32 * q) : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (base + 32 * q < G) t += v[q];
      }
      t = warp_sum(t);
      if (lane == 0) {
        if (pass) g.C[j] = t;
        else g.R[j * kRld + i] = t;
      }
    }
    if (threadIdx.x == 0) st->counter = 0;
  }
}

// End-of-step bookkeeping shared by the pipelined and classical forms.
__device__ __forceinline__ void gm_step_done(DevState* st, GmArgs& g, int i, double xi_i, double rel2) {
  g.xi[i] = xi_i;
  st->iter += 1;
  st->gm_k = i;
  if (rel2 < 0.0) rel2 = 0.0;
  const double est = st->s[0] * sqrt(rel2);
  const int step = st->iter - 1;
  trace_put(st, step, 0, i >= 2 ? g.R[(i - 1) * kRld + i] : 0.0);
  trace_put(st, step, 1, g.R[i * kRld + i]);
  trace_put(st, step, 2, xi_i);
  trace_put(st, step, 3, est);
  if (!isfinite(xi_i)) {
    gm_finish(st, PK_ERR_NAN);
  } else if (est * est <= st->thr2 || rel2 <= kGmEstFloor || i >= st->gm_m || st->iter >= st->maxit) {
    st->gm_phase = GM_END;
    cond2_set(st, 0u);
  } else {
    st->gm_i = i + 1;
  }
}

// K-GM-3: v_i -= sum_{j=1}^{i-1} R_{j,i} v_j (in order j = 1, 2, ...) with the first stage of
// ||v_i||^2.  Tiles outer, column groups inner: each consumer thread keeps its row of v_i in
// a register across the groups of the tile, then stores it.  Last block: R_{i,i} and the
// lucky-breakdown test (R13).  mode 1 (CGS2, first pass): no norm, no epilogue; mode 2 (CGS2,
// second pass): coefficients c_j from C, then R_{j,i} += c_j before R_{i,i} and the test.
// mode 3 (three-kernel form): v_i = (v_i - sum_j R_{j,i} v_j) / R_{i,i} with R_{i,i} from the
// norm identity (computed by every block before the pass) and the first stage of
// xi_i = <v_0, v_i> (v_0 streamed with the first column group, which then holds 15 columns);
// last block: R's diagonal, the next shift and the end of the step.
__global__ void __launch_bounds__(kTileThreads, 2) k_gm3(GmArgs g, int mode) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = g.st;
  if (!gm_step_live(st)) return;
  const int i = __ldcg(&st->gm_i);
  __shared__ double coef[kGmMax];
  for (int j = threadIdx.x; j < i - 1; j += blockDim.x)
    coef[j] = mode == 2 ? ld_cg(g.C + j + 1) : ld_cg(g.R + (j + 1) * kRld + i);
  int r0, r1;
  ew_range(g.n, r0, r1);
  const int ntiles = r1 > r0 ? (r1 - r0 + kBsRows - 1) / kBsRows : 0;
  const int ncols = i - 1;                                     // v_1 .. v_{i-1}
  const bool shift = mode == 3;
  const int cpg = shift ? kBsCols - 1 : kBsCols;               // columns per group
  const int ngroups = max(1, (ncols + cpg - 1) / cpg);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* vi = g.V + (size_t)i * g.ld;
  const BasisRing R = basis_ring(smem);  // (its __syncthreads also publishes coef)
  // three-kernel form: R_{i,i}^2 = <w,w> - sum_{j<i-1} R_{j,i}^2 - (R_{i-1,i} - sigma_i)^2,
  // the same bits in every block
  double rii2 = 0.0, inv = 0.0;
  bool go = true;
  if (shift) {
    const double sigma = __ldcg(&st->s[2]);
    double sum2 = 0.0;
    for (int j = 0; j < ncols; ++j) {
      const double c = j == ncols - 1 ? coef[j] - sigma : coef[j];
      sum2 = fma(c, c, sum2);
    }
    const double nu = __ldcg(&st->s[5]);
    rii2 = nu - sum2;
    go = isfinite(rii2) && rii2 > kGmShiftFloor * nu;
    inv = go ? 1.0 / sqrt(rii2) : 0.0;
  }
  const int ntl = go ? ntiles : 0;  // (a step that the identity cannot take streams nothing)
  double v[1] = {0.0};
  if (warp == kConsumerWarps) {
    if (lane == 0)
      basis_produce(R, ntl * ngroups, st, [&](int q, const double** src, int& row0, int& rows, int& nv) {
        const int t = q / ngroups, grp = q % ngroups;
        const int j0 = 1 + grp * cpg, nc = max(0, min(cpg, ncols - j0 + 1));
        row0 = r0 + t * kBsRows;
        rows = min(kBsRows, r1 - row0);
        nv = nc + (grp == 0);
        src[0] = grp == 0 ? vi : nullptr;
        for (int c = 0; c < kBsCols; ++c) src[1 + c] = c < nc ? g.V + (size_t)(j0 + c) * g.ld : nullptr;
        if (shift && grp == 0) src[kBsVecs - 1] = g.V;  // v_0
      });
  } else {
    for (int t = 0; t < ntl; ++t) {
      const int row0 = r0 + t * kBsRows, rows = min(kBsRows, r1 - row0);
      const bool mine = (int)threadIdx.x < rows;
      double w = 0.0, v0r = 0.0;
      bool ok = true;
      for (int grp = 0; grp < ngroups; ++grp) {
        const int q = t * ngroups + grp, s = q % kBsStages;
        if (!mbar_wait_st(&R.full[s], (q / kBsStages) & 1, st)) { report_timeout(st); ok = false; break; }
        const int j0 = 1 + grp * cpg, nc = max(0, min(cpg, ncols - j0 + 1));
        if (mine) {
          if (grp == 0) {
            w = R.slot(s, 0)[threadIdx.x];
            if (shift) v0r = R.slot(s, kBsVecs - 1)[threadIdx.x];
          }
          const double* cf = coef + (j0 - 1);
          switch (nc) {
#define PK_GM3_CASE(N) \
  case N: w = gm3_row<N>(R, s, threadIdx.x, cf, w); break;
            PK_GM_CASES(PK_GM3_CASE)
#undef PK_GM3_CASE
            default: break;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[s]);
      }
      if (!ok) break;
      if (mine) {
        if (shift) {
          w *= inv;
          vi[row0 + threadIdx.x] = w;
          v[0] = fma(v0r, w, v[0]);
        } else {
          vi[row0 + threadIdx.x] = w;
          if (mode != 1) v[0] = fma(w, w, v[0]);
        }
      }
    }
  }
  if (mode == 1) return;
  tile_block_partials<1>(v, g.partials);
  if (shift) {
    if (arrive_last(&st->counter)) {
      double t[1];
      final_sums<1>(g.partials, t);
      if (threadIdx.x == 0) {
        if (__ldcg(&st->timeout)) {
          gm_finish(st, PK_TIMEOUT);
        } else if (!isfinite(rii2)) {
          gm_finish(st, PK_ERR_NAN);
        } else if (!go) {
          st->gm_k = i - 1;  // the cycle ends before step i
          st->gm_phase = GM_END;
          cond2_set(st, 0u);
        } else {
          g.R[i * kRld + i] = sqrt(rii2);
          st->s[2] = st->s[4];  // sigma_{i+1}
          const double xi_i = t[0];
          st->s[1] += xi_i * xi_i;
          gm_step_done(st, g, i, xi_i, 1.0 - st->s[1]);
        }
        st->counter = 0;
      }
    }
    return;
  }
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(g.partials, t);
    if (threadIdx.x == 0) {
      const double nrm2 = t[0];
      double col2 = nrm2;
      if (mode == 2)
        for (int j = 1; j < i; ++j) g.R[j * kRld + i] += coef[j - 1];
      for (int j = 1; j < i; ++j) {
        const double rji = mode == 2 ? g.R[j * kRld + i] : coef[j - 1];
        col2 += rji * rji;
      }
      const double rii = sqrt(nrm2);
      if (!isfinite(rii)) {
        gm_finish(st, PK_ERR_NAN);
      } else if (rii == 0.0 || rii <= 1e-14 * sqrt(col2)) {
        st->gm_k = i - 1;  // the cycle ends before step i
        st->gm_phase = GM_END;
        cond2_set(st, 0u);
      } else {
        g.R[i * kRld + i] = rii;
        st->s[4] = 1.0 / rii;  // once here, not in every thread of the normalising kernel
      }
      st->counter = 0;
    }
  }
}

// K-GM-4 (pipelined): v_i /= R_{i,i} with the first stage of xi_i = <v_0, v_i>.
__global__ void __launch_bounds__(kTileThreads, 2) k_gm4(GmArgs g) {
  extern __shared__ __align__(128) unsigned char smem[];
  DevState* st = g.st;
  const int i = __ldcg(&st->gm_i);
  double* vi = g.V + (size_t)i * g.ld;
  int r0, r1;
  ew_range(g.n, r0, r1);
  double inv = 0.0;
  double v[1] = {0.0};
  StreamIn<2> in{{g.V, vi}};
  const bool live = stream_tiles<2, 2, double, 4>(in, r0, r1, smem, st, [&]() {
    inv = __ldcg(&st->s[4]);
    return gm_step_live(st);
  }, [&](int row, const double2* val, int nv) {
    double2 w = val[1];
    w.x *= inv;
    w.y *= inv;
    if (nv == 2) {
      st2(vi + row, w);
      v[0] = fma(val[0].x, w.x, v[0]);
      v[0] = fma(val[0].y, w.y, v[0]);
    } else {
      vi[row] = w.x;
      v[0] = fma(val[0].x, w.x, v[0]);
    }
  });
  if (!__syncthreads_or(threadIdx.x < kConsumers && live)) return;
  tile_block_partials<1>(v, g.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(g.partials, t);
    if (threadIdx.x == 0) {
      const double xi_i = t[0];
      st->s[1] += xi_i * xi_i;
      if (__ldcg(&st->timeout)) gm_finish(st, PK_TIMEOUT);
      else gm_step_done(st, g, i, xi_i, 1.0 - st->s[1]);
      st->counter = 0;
    }
  }
}

// Classical form (Alg. 5): v_i /= R_{i,i} (plain kernel).
__global__ void __launch_bounds__(kBlock) k_gmc_norm(GmArgs g) {
  DevState* st = g.st;
  if (!gm_step_live(st)) return;
  const int i = __ldcg(&st->gm_i);
  double* vi = g.V + (size_t)i * g.ld;
  const double inv = __ldcg(&st->s[4]);
  int r0, r1;
  ew_range(g.n, r0, r1);
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) vi[row] *= inv;
}

// Classical form: xi_i = <r, v_i>.
__global__ void __launch_bounds__(kBlock) k_gmc_xi(GmArgs g) {
  DevState* st = g.st;
  if (!gm_step_live(st)) return;
  const int i = __ldcg(&st->gm_i);
  const double* vi = g.V + (size_t)i * g.ld;
  int r0, r1;
  ew_range(g.n, r0, r1);
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(g.r[row], vi[row], v[0]);
  block_partials<1>(v, g.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(g.partials, t);
    if (threadIdx.x == 0) {
      g.xi[i] = t[0];
      st->counter = 0;
    }
  }
}

// Classical form: r -= xi_i v_i.
__global__ void __launch_bounds__(kBlock) k_gmc_rupd(GmArgs g) {
  DevState* st = g.st;
  if (!gm_step_live(st)) return;
  const int i = __ldcg(&st->gm_i);
  const double* vi = g.V + (size_t)i * g.ld;
  const double xi_i = ld_cg(g.xi + i);
  int r0, r1;
  ew_range(g.n, r0, r1);
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) g.r[row] = fma(-xi_i, vi[row], g.r[row]);
}

// Classical form: ||r||^2 monitors the residual; end-of-step decision.
__global__ void __launch_bounds__(kBlock) k_gmc_rnorm(GmArgs g) {
  DevState* st = g.st;
  if (!gm_step_live(st)) return;
  const int i = __ldcg(&st->gm_i);
  int r0, r1;
  ew_range(g.n, r0, r1);
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(g.r[row], g.r[row], v[0]);
  block_partials<1>(v, g.partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(g.partials, t);
    if (threadIdx.x == 0) {
      gm_step_done(st, g, i, g.xi[i], t[0]);
      st->counter = 0;
    }
  }
}

// END: eta from R eta = xi (warp 0 of every block), x += rho0 sum_i eta_i z_i.
__global__ void __launch_bounds__(kBlock) k_gm_end(GmArgs g) {
  DevState* st = g.st;
  if (state_done(st) || __ldcg(&st->gm_phase) != GM_END) return;
  const int k = __ldcg(&st->gm_k);
  const double rho0 = __ldcg(&st->s[0]);
  __shared__ double eta[kGmMax + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    for (int ii = k; ii >= 1; --ii) {
      double s = 0.0;
      for (int j = ii + 1 + lane; j <= k; j += 32) s = fma(ld_cg(g.R + ii * kRld + j), eta[j], s);
      s = warp_sum(s);
      if (lane == 0) eta[ii] = (ld_cg(g.xi + ii) - s) / ld_cg(g.R + ii * kRld + ii);
      __syncwarp();
    }
  }
  __syncthreads();
  int r0, r1;
  ew_range(g.n, r0, r1);
  if (k > 0) {
    for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
      double a = 0.0;
      for (int ii = 1; ii <= k; ++ii) a = fma(eta[ii], g.V[(size_t)(ii - 1) * g.ld + row], a);
      g.x[row] = fma(rho0, a, g.x[row]);
    }
  }
  if (arrive_last(&st->counter)) {
    if (threadIdx.x == 0) {
      st->gm_phase = GM_START;
      st->gm_cycle += 1;
      st->counter = 0;
    }
  }
}

__global__ void k_gm_init(DevState* st, int m) {
  st->gm_m = m;
  st->gm_i = 0;
  st->gm_k = 0;
  st->gm_cycle = 0;
  st->gm_phase = GM_START;
}

static pk_status gm_setup() {
  static bool done = false;
  if (!done) {
    for (auto k : {k_gm_start<false>, k_gm_start<true>, k_gm1<false, false>, k_gm1<true, false>, k_gm1<false, true>,
                   k_gm1<true, true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, csr_smem_bytes()));
    PK_CUDA(cudaFuncSetAttribute(k_gm_scale, cudaFuncAttributeMaxDynamicSharedMemorySize, stream_smem_bytes<1>()));
    PK_CUDA(cudaFuncSetAttribute(k_gm4, cudaFuncAttributeMaxDynamicSharedMemorySize, stream_smem_bytes<2, double, 4>()));
    PK_CUDA(cudaFuncSetAttribute(k_gm2, cudaFuncAttributeMaxDynamicSharedMemorySize, kBsSmem));
    PK_CUDA(cudaFuncSetAttribute(k_gm3, cudaFuncAttributeMaxDynamicSharedMemorySize, kBsSmem));
    done = true;
  }
  return PK_OK;
}

// pk_gmres_cluster.cu: the whole restarted pipelined loop on one thread-block cluster
bool gmres_persistent_usable(const pk_csr* A, int m);
pk_status launch_gmres_persistent(pk_csr* A, const double* b, double* x, int m, double* V, int64_t ld,
                                  double* Rout, double* xiout, cudaStream_t s);

pk_status gmres_solve(pk_csr* A, const double* b, double* x, const pk_opts* o, pk_info* info,
                      cudaStream_t s) {
  pk_status e = check_opts(A, b, x, o, info);
  if (e) return e;
  if (o->loop == PK_LOOP_RESIDENT) { set_error("PK_LOOP_RESIDENT runs pipelined CG only"); return PK_ERR_ARG; }
  *info = pk_info{};
  info->rel_res_true = -1.0;
  if (A->n == 0) return PK_OK;
  const int m = o->restart;
  if (m < 1 || m > kGmMax) { set_error("GMRES restart must be in 1..64"); return PK_ERR_ARG; }
  if (o->precision != PK_PREC_FP64) { set_error("GMRES runs in FP64 only"); return PK_ERR_ARG; }
  if (o->variant != PK_VARIANT_PIPELINED && o->variant != PK_VARIANT_CLASSICAL) {
    set_error("GMRES variants: pipelined or classical");
    return PK_ERR_ARG;
  }
  if (o->precond != PK_PRECOND_NONE && o->precond != PK_PRECOND_JACOBI) { set_error("bad precond"); return PK_ERR_ARG; }
  if (o->flags & PK_FLAG_SELL) { set_error("PK_FLAG_SELL applies to pipelined FP64 CG"); return PK_ERR_ARG; }
  const bool cgs2 = (o->flags & PK_FLAG_CGS2) != 0;
  const bool shift = (o->flags & PK_FLAG_GM_SHIFT) != 0;
  if (shift && (cgs2 || o->variant != PK_VARIANT_PIPELINED)) {
    set_error("PK_FLAG_GM_SHIFT is a form of pipelined GMRES with one Gram-Schmidt pass (not with PK_FLAG_CGS2)");
    return PK_ERR_ARG;
  }
  // the whole loop on one thread-block cluster (small systems): asked for, or chosen by AUTO
  bool persistent = false;
  const bool plain = o->variant == PK_VARIANT_PIPELINED && !cgs2 && !shift;
  if (o->loop == PK_LOOP_PERSISTENT) {
    if (!plain) {
      set_error("PK_LOOP_PERSISTENT runs pipelined GMRES with one Gram-Schmidt pass (no PK_FLAG_CGS2, PK_FLAG_GM_SHIFT)");
      return PK_ERR_ARG;
    }
    if (!gmres_persistent_usable(A, m)) {
      set_error("PK_LOOP_PERSISTENT: the persistent GMRES loop needs n <= 16 x 4096 rows (one thread-block cluster) and cluster launch");
      return PK_ERR_ARG;
    }
    persistent = true;
  } else if (o->loop == PK_LOOP_AUTO) {
    // (rows of very different lengths stay on the tile engine: one thread per row leaves the
    // cluster waiting for the longest)
    persistent = plain && A->n <= PK_PERSISTENT_GMRES_AUTO_N && A->nnz <= PK_PERSISTENT_GMRES_AUTO_NNZ &&
                 A->stats.tiles_long == 0 && !(o->flags & PK_FLAG_TIMING) && gmres_persistent_usable(A, m);
  }
  if (!A->tma_ok && !persistent) { set_error("GMRES needs the tile engine"); return PK_ERR_ARG; }
  if ((e = gm_setup())) return e;
  const int n = A->n;
  const int ld = ((n + 31) & ~31) + 32;
  if (A->basis_m < m) {
    if (A->basis) cudaFree(A->basis);
    A->basis = nullptr;
    A->basis_m = 0;
    PK_CUDA(cudaMalloc(&A->basis, sizeof(double) * (size_t)(m + 1) * ld));
    PK_CUDA(cudaMemset(A->basis, 0, sizeof(double) * (size_t)(m + 1) * ld));
    A->basis_m = m;
  }
  cudaEvent_t e0, e1;
  PK_CUDA(cudaEventCreate(&e0));
  PK_CUDA(cudaEventCreate(&e1));
  PK_CUDA(cudaEventRecord(e0, s));
  if ((e = state_init(A, o, s))) return e;
  k_gm_init<<<1, 1, 0, s>>>(A->st, m);
  VecStage v;
  if ((e = stage_in(A, b, x, 14, 15, s, &v))) return e;
  // right Jacobi preconditioning: iterate on A M^-1 with y = M x (values swapped until leave)
  JacobiRight jac;
  if (o->precond == PK_PRECOND_JACOBI && (e = jacobi_right_enter(A, v.x_dev, s, &jac))) return e;
  if (persistent) {
    Timer T;
    T.A = A;
    T.on = (o->flags & PK_FLAG_TIMING) != 0;
    T.s = s;
    if ((e = T.begin(PK_SLOT_OTHER))) return e;
    if ((e = launch_gmres_persistent(A, v.b_dev, v.x_dev, m, A->basis, ld, A->small, A->small + kXiOff, s))) return e;
    if ((e = T.end())) return e;
    launch_zero_x(A, v.x_dev, s);
    int launches = 3;  // state, the loop, the b = 0 case
    if ((e = T.flush())) return e;
    if (jac.A) {
      if ((e = jacobi_right_leave(&jac, v.x_dev, s))) return e;
      launches += 2;
    }
    if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
    info->cycles = A->st_host->gm_cycle;
    for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
      info->kernel_count[k] = T.count[k];
      info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (pk_status)info->status;
  }
  const bool classical = o->variant == PK_VARIANT_CLASSICAL;
  double* rc = nullptr;
  if (classical && (e = work_vec(A, 6, &rc))) return e;
  GmArgs g;
  g.n = n;
  g.ld = ld;
  g.V = A->basis;
  g.R = A->small;
  g.xi = A->small + kXiOff;
  g.C = A->small + kXiOff + kRld;
  g.r = rc;
  g.b = v.b_dev;
  g.x = v.x_dev;
  g.partials = A->partials;
  g.st = A->st;
  const CsrTiles ct = csr_tiles_of(A);
  const bool irr = csr_irregular(A);  // some tile needs the grouped or whole-warp rows
  const int Gt = A->grid_tma, Gs = A->grid_stream;
  int Ge = A->grid_ew;
  if (!Ge) {
    int sms = 1;
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
    Ge = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, ((int64_t)n + 2 * kBlock - 1) / (2 * kBlock)));
  }
  Timer T;
  T.A = A;
  T.on = (o->flags & PK_FLAG_TIMING) != 0;
  T.s = s;
  int launches = 1;  // k_gm_init
  auto pre = [&](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_OTHER);
    (irr ? k_gm_start<true> : k_gm_start<false>)<<<Gt, kTileThreads, csr_smem_bytes(), cs>>>(ct, g);
    if (t) { t->end(); t->begin(PK_SLOT_OTHER); }
    k_gm_scale<<<Gs, kTileThreads, stream_smem_bytes<1>(), cs>>>(g);
    if (t) t->end();
  };
  auto step = [&](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_SPMV_DOTS);
    auto k1 = shift ? (irr ? k_gm1<true, true> : k_gm1<false, true>) : (irr ? k_gm1<true, false> : k_gm1<false, false>);
    k1<<<Gt, kTileThreads, csr_smem_bytes(), cs>>>(ct, g);
    if (t) { t->end(); t->begin(PK_SLOT_MULTIDOT); }
    k_gm2<<<Gs, kTileThreads, kBsSmem, cs>>>(g, 0);
    if (t) { t->end(); t->begin(PK_SLOT_ORTHO); }
    k_gm3<<<Gs, kTileThreads, kBsSmem, cs>>>(g, shift ? 3 : cgs2 ? 1 : 0);
    if (t) t->end();
    if (shift) return;  // (K-GM-3 normalised v_i and formed xi_i)
    if (cgs2) {  // second Gram-Schmidt pass
      if (t) t->begin(PK_SLOT_MULTIDOT);
      k_gm2<<<Gs, kTileThreads, kBsSmem, cs>>>(g, 1);
      if (t) { t->end(); t->begin(PK_SLOT_ORTHO); }
      k_gm3<<<Gs, kTileThreads, kBsSmem, cs>>>(g, 2);
      if (t) t->end();
    }
    if (!classical) {
      if (t) t->begin(PK_SLOT_UPDATE);
      k_gm4<<<Gs, kTileThreads, stream_smem_bytes<2, double, 4>(), cs>>>(g);
      if (t) t->end();
    } else {
      if (t) t->begin(PK_SLOT_BLAS1);
      k_gmc_norm<<<Ge, kBlock, 0, cs>>>(g);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_gmc_xi<<<Ge, kBlock, 0, cs>>>(g);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_gmc_rupd<<<Ge, kBlock, 0, cs>>>(g);
      if (t) { t->end(); t->begin(PK_SLOT_BLAS1); }
      k_gmc_rnorm<<<Ge, kBlock, 0, cs>>>(g);
      if (t) t->end();
    }
  };
  auto post = [&](cudaStream_t cs, Timer* t) {
    if (t) t->begin(PK_SLOT_OTHER);
    k_gm_end<<<Ge, kBlock, 0, cs>>>(g);
    if (t) t->end();
  };
  const int step_kernels = shift ? 3 : (classical ? 7 : 4) + (cgs2 ? 2 : 0);
  const bool graph = o->loop != PK_LOOP_HOST && !T.on;
  if (graph) {
    const void* keys[4] = {v.x_dev, v.b_dev, nullptr, nullptr};
    const int64_t ikeys[4] = {o->variant, m, o->precond, (int64_t)cgs2 | (int64_t)shift << 1};  // precond: values of A or of A M^-1
    pk_graph_entry* ge = nullptr;
    if ((e = build_nested_graph(A, 6 + (classical ? 1 : 0), keys, ikeys,
                                [&](cudaStream_t cs) { pre(cs, nullptr); },
                                [&](cudaStream_t cs) { step(cs, nullptr); },
                                [&](cudaStream_t cs) { post(cs, nullptr); }, &ge)))
      return e;
    launch_enable_cond2(A, ge, s);
    PK_CUDA(cudaGetLastError());
    PK_CUDA(cudaGraphLaunch(ge->exec, s));
    launches += 1;
  } else {
    for (;;) {
      pre(s, T.on ? &T : nullptr);
      launches += 2;
      for (int i = 0; i < m; ++i) {
        step(s, T.on ? &T : nullptr);
        launches += step_kernels;
        if (T.on) {
          if ((e = T.flush())) return e;
          PK_CUDA(cudaMemcpyAsync(&A->st_host->gm_phase, &A->st->gm_phase, sizeof(int), cudaMemcpyDeviceToHost, s));
          PK_CUDA(cudaStreamSynchronize(s));
          if (A->st_host->gm_phase != GM_STEP) break;
        }
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
  if (jac.A) {
    if ((e = jacobi_right_leave(&jac, v.x_dev, s))) return e;
    launches += 2;  // y0 = M x0 and x = M^-1 y
  }
  if ((e = finish_info(A, o, info, s, v, e0, e1, launches))) return e;
  const DevState* h = A->st_host;
  info->cycles = h->gm_cycle;
  if (graph) {
    const long long steps = passes_of(h);
    const long long cycles = *reinterpret_cast<const long long*>(&h->s[6]);
    info->launches += (int)(steps * step_kernels + cycles * 3);
  }
  for (int k = 0; k < PK_MAX_KERNEL_SLOTS; ++k) {
    info->kernel_count[k] = T.count[k];
    info->kernel_ms[k] = T.count[k] ? T.ms[k] / T.count[k] : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (pk_status)info->status;
}

}  // namespace pk

extern "C" pk_status pk_gmres_solve(pk_csr* A, const double* b, double* x, const pk_opts* opts,
                                    pk_info* info, void* stream) {
  return pk::guarded([&] { return pk::gmres_solve(A, b, x, opts, info, (cudaStream_t)stream); });
}

// The R factor and xi of the most recent GMRES cycle on the handle (device scratch -> host).
extern "C" pk_status pk_gmres_cycle_factors(const pk_csr* A, int32_t m, double* R, double* xi,
                                            void* stream) {
  return pk::guarded([&]() -> pk_status {
    using namespace pk;
    if (!A || !R || !xi) { set_error("pk_gmres_cycle_factors: NULL argument"); return PK_ERR_ARG; }
    if (m < 1 || m > kGmMax) { set_error("pk_gmres_cycle_factors: m must be in 1..64"); return PK_ERR_ARG; }
    if (!A->small) { set_error("pk_gmres_cycle_factors: no GMRES solve has run on this handle"); return PK_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> h((size_t)kXiOff + kRld);
    PK_CUDA(cudaMemcpyAsync(h.data(), A->small, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    for (int j = 1; j <= m; ++j)
      for (int i = 1; i <= m; ++i) R[(size_t)(j - 1) * m + (i - 1)] = j <= i ? h[(size_t)j * kRld + i] : 0.0;
    for (int i = 1; i <= m; ++i) xi[i - 1] = h[(size_t)kXiOff + i];
    return PK_OK;
  });
}
