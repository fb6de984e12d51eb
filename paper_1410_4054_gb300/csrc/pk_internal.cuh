// Internal declarations shared by the translation units of the pk library.
//
// Device-side building blocks of the fused kernels (Sec. 2.2 of Rupp et al.,
// arXiv:1410.4054): the first reduction stage of inner products is a per-block sum written
// to a fixed slot; the second stage is done by the last block to finish (arrival counter),
// which sums the slots in a fixed order -- so every reduction is deterministic -- and then
// computes the solver's scalars and convergence test on the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/pk.h"

namespace pk {

constexpr int kBlock = 256;        // threads per block of the fused kernels
constexpr int kMaxGridPerSm = 8;   // resident blocks per SM used for the persistent grid
constexpr int kMaxDots = 64;       // partial-sum slots per block (GMRES needs up to m+1)
constexpr int kRunning = -1;       // DevState::status while iterating

// Scalars of one solve, in device memory.  One arrival counter suffices: kernels of a solve
// run one after another on one stream, and each last block resets it.
struct DevState {
  double rr;      // <r_i, r_i> (CG, BiCGStab), squared true residual (GMRES)
  double alpha, beta, omega;
  double bb;      // <b, b>
  double thr2;    // tol^2 <b, b>
  double s[8];    // solver-specific scalars
  int32_t iter, maxit, status, done;
  int32_t zero_x;         // b = 0: the solution is x = 0
  int32_t trace_cap;
  double* trace;          // [trace_cap][4] or nullptr
  unsigned int counter;   // last-block arrival counter
  int32_t use_cond;       // kernels run inside a conditional WHILE graph node
  cudaGraphConditionalHandle cond;
  int32_t timeout;        // a bounded device-side wait ran out
  int32_t early;          // BiCGStab: ||s|| <= tol ||b||, finish with x += alpha p
  // GMRES(m): step i of the cycle, steps k done in it, restart count, phase, inner loop
  int32_t gm_i, gm_k, gm_cycle, gm_phase;
  int32_t gm_m, gm_pad;
  cudaGraphConditionalHandle cond2;
  unsigned int gbar;      // grid-barrier arrivals of the persistent (cooperative) solve
  unsigned long long wait_ns;  // bound on a pipeline wait that should make progress
  int32_t stall_test;          // PK_FLAG_TEST_STALL: the CSR tile producer issues no copies
  int32_t stall_pad;
  // grid-resident CG loop: the last block of iteration i's reduction publishes epoch = i + 1
  // once alpha_i, beta_i and the exit decision are in place
  int32_t epoch;
  int32_t epoch_pad;
};

// Loads that bypass L1 (the value was written by another block or an earlier kernel).
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ld_cg(const int* p) { return __ldcg(p); }

// Warp sum with a fixed xor tree: every lane ends with the same, order-fixed sum.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// First reduction stage: block sum of NV per-thread values into partials[k * G + block].
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* partials) {
  __shared__ double sm[NV][kBlock / 32];
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
      double t = lane < (int)(blockDim.x >> 5) ? sm[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) partials[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Float-float accumulator for FP32 inner products: s.hi + s.lo holds the running sum of the
// exact float products (error-free product with fmaf, TwoSum), all in the FP32 pipe.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ void ff_add_prod(FF& s, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);  // p + e == a * b exactly
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);  // s.hi + p == t + err exactly
  s.hi = t;
  s.lo += err + e;
}

__device__ __forceinline__ double ff_value(const FF& s) { return (double)s.hi + (double)s.lo; }

// Arrival on the grid-wide counter; true in every thread of the last block to arrive.
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ unsigned int ticket;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    ticket = atomicAdd(counter, 1u);
  }
  __syncthreads();
  const bool last = ticket == gridDim.x - 1;
  if (last) __threadfence();
  return last;
}

// A lane's share of a fixed-order second stage over G block slots: for every k < NV, the
// slots c = lane, lane + 32, lane + 64, ... of partials[k * G + c], added in that order
// alternately into two accumulators (even steps a0, odd steps a1), t[k] = a0 + a1.  The loads
// of B steps of all NV sums are issued before their adds: a warp issues in order, so a loop
// that adds each load before issuing the next waits one L2 round trip per step (measured on
// GB300 with 304 slots: about 10 us for two sums, on the critical path of every iteration).
// The adds are the same, in the same order, as in that loop.
template <int NV, int B>
__device__ __forceinline__ void lane_slot_sums(const double* partials, int G, int lane, double (&t)[NV]) {
  static_assert(B % 2 == 0, "batches keep the even / odd step parity");
  double a0[NV], a1[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) a0[k] = a1[k] = 0.0;
  for (int base = lane; base < G; base += 32 * B) {
    double v[NV][B];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int c = base + 32 * q;
        v[k][q] = c < G ? ld_cg(partials + (size_t)k * G + c) : 0.0;
      }
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int q = 0; q < B; ++q)
        if (base + 32 * q < G) {
          if (q & 1) a1[k] += v[k][q];
          else a0[k] += v[k][q];
        }
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) t[k] = a0[k] + a1[k];
}

// Second reduction stage in the last block: out[k] = sum over blocks of partials[k][.], in a
// fixed order, broadcast to every thread.  One warp does it (two interleaved accumulators
// per lane, loads issued in batches, then a butterfly): on GB300 every FP64 instruction that
// all warps of the block would issue costs the SM's narrow FP64 pipe, and this runs on the
// critical path.
template <int NV>
__device__ __forceinline__ void final_sums(const double* partials, double (&out)[NV]) {
  __shared__ double sm[NV];
  const int G = gridDim.x;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double t[NV];
    lane_slot_sums<NV, (NV <= 2 ? 6 : 4)>(partials, G, lane, t);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double u = t[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
      if (lane == 0) sm[k] = u;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = sm[k];
}

__device__ __forceinline__ void trace_put(DevState* st, int i, int slot, double v) {
  if (st->trace && i >= 0 && i < st->trace_cap) st->trace[(size_t)i * 4 + slot] = v;
}

// Ends the solve: status, done flag, and (inside a graph WHILE node) the loop condition.
__device__ __forceinline__ void finish(DevState* st, int status) {
  st->status = status;
  st->done = 1;
  if (st->use_cond) cudaGraphSetConditional(st->cond, 0u);
}

// Host-side maxima of the tile engine (defined in pk_tile.cuh).
// Common kernel arguments of the row-parallel kernels.
// One system of a batch as the cluster engine of the batched solver sees it: the CSR copy of
// its handle, b, x, and the results written back by the cluster that solved it.
struct BatchClSys {
  int32_t n;
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const double* b;
  double* x;
  int32_t iters, status;
  double rel_res;
};

// The batched solver's cluster engine (pk_batched_cluster.cu): shapes 0, 1, 2 are CTAs of
// 512 threads and up to 4096 rows, 256 and 2048, 128 and 1024.
constexpr int kBcShapeCount = 3;
int batched_cluster_max_rows(int shape);
int batched_cluster_capacity(int shape, int C);
pk_status launch_batched_cluster(int shape, BatchClSys* sys, int first, int end, int* queue, int C, double tol,
                                 int maxit, cudaStream_t s);

struct RowArgs {
  int32_t n;
  const int32_t* rp;      // row pointers
  const int32_t* ci;      // column indices
  const double* va;       // values
  const int32_t* rowblk;  // rows of block b: [rowblk[b], rowblk[b+1])
  double* partials;       // [kMaxDots][grid]
  DevState* st;
};

}  // namespace pk

// ------------------------------------------------------------------ host side

struct pk_graph_entry {
  int kind = -1;              // solver kind (0 = none)
  const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t ikey[4] = {0, 0, 0, 0};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond_handle = 0;
  cudaGraphConditionalHandle cond2_handle = 0;  // inner loop of a nested graph
  int body_kernels = 0;
};

struct pk_csr {
  int32_t n = 0, nnz = 0;
  int device = 0;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* va = nullptr;
  float* va32 = nullptr;
  int32_t* rowblk = nullptr;  // grid + 1
  int grid = 1;
  int grid_ew = 0;             // grid of the elementwise update kernels (0 = not chosen yet)
  // warp-specialised CSR tiles (cp.async.bulk pipeline); tma_ok = 0 if a row is too long
  int tma_ok = 0;
  int grid_tma = 0;
  int32_t* tile_row = nullptr;  // ntiles + 1
  int32_t* blk_tile = nullptr;  // grid_tma + 1
  int8_t* tile_grp = nullptr;   // ntiles: 1 if the tile has no row longer than 32 nonzeros
  int16_t* tile_perm = nullptr; // ntiles x 512: row order of the irregular tiles (or null)
  int32_t* tile_z0 = nullptr;   // ntiles: first nonzero of a chunk tile, -1 otherwise (or null)
  int ntiles = 0;
  int grid_stream = 0;          // grid of the streaming (vector-only) tile kernels
  int partial_cap = 0;         // blocks the partials buffer can hold
  pk_csr_stats stats{};
  cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
  // cached work memory
  double* vec[16] = {nullptr};        // n-length work vectors, allocated on demand
  int32_t vec_len[16] = {0};
  double* partials = nullptr;         // [kMaxDots][grid]
  pk::DevState* st = nullptr;         // device scalars
  pk::DevState* st_host = nullptr;    // pinned host mirror
  double* basis = nullptr;            // GMRES Krylov basis, (m+1) x n column-contiguous
  int basis_m = 0;
  double* small = nullptr;            // small device scratch (R, xi, eta ...): 8192 doubles
  // right Jacobi preconditioning (built on first use): values of A diag(A)^-1, diag(A) and its
  // reciprocal; jac_state 0 = not built, 1 = built, -1 = a zero or non-finite diagonal entry
  // SELL-C-sigma copy (built on first use; sell_nslices -1 = not built)
  int32_t sell_nslices = -1;
  int64_t sell_padded = 0;
  int sell_grid = 1;
  int64_t* sell_ptr = nullptr;
  int32_t* sell_perm = nullptr;
  int32_t* sell_col = nullptr;
  double* sell_val = nullptr;
  double* jac_va = nullptr;
  double* jac_d = nullptr;
  double* jac_dinv = nullptr;
  int jac_state = 0;
  // grid-resident CG loop (built on first use): blocks, their rows, the range of
  // blocks whose p each block's SpMV reads, the per-block "p written" flags
  int res_grid = 0;                 // 0 = not built, -1 = not usable on this matrix / device
  int32_t* res_rows = nullptr;      // res_grid + 1
  int32_t* res_nbr = nullptr;       // 2 per block: first and last neighbour block
  int32_t* res_flag = nullptr;      // res_grid
  pk_graph_entry graphs[4];
  cudaEvent_t ev_pool[64] = {nullptr};
  int ev_count = 0;
};

namespace pk {

// thread-local last error message
void set_error(const std::string& msg);
pk_status cuda_fail(cudaError_t e, const char* what);

#define PK_CUDA(call)                                                     \
  do {                                                                    \
    cudaError_t e__ = (call);                                             \
    if (e__ != cudaSuccess) return ::pk::cuda_fail(e__, #call);           \
  } while (0)

// Work vector slot `id` of length n (allocated on first use).
pk_status work_vec(pk_csr* A, int id, double** out);
pk_status ensure_state(pk_csr* A);

// Host/device pointer staging for b and x (host pointers are copied in and out).
struct VecStage {
  const double* b_dev = nullptr;
  double* x_dev = nullptr;
  double* x_user = nullptr;
  bool x_host = false;
};
pk_status stage_in(pk_csr* A, const double* b, double* x, int slot_b, int slot_x,
                   cudaStream_t s, VecStage* out);
pk_status stage_out(pk_csr* A, const VecStage& v, cudaStream_t s);

// Initialise DevState for a solve and read it back afterwards.
pk_status state_init(pk_csr* A, const pk_opts* o, cudaStream_t s);
pk_status state_read(pk_csr* A, cudaStream_t s);

// Kernel timing helper (PK_FLAG_TIMING).
struct Timer {
  pk_csr* A = nullptr;
  bool on = false;
  cudaStream_t s = nullptr;
  int used = 0;
  int slot[32] = {0};
  double ms[PK_MAX_KERNEL_SLOTS] = {0};
  int count[PK_MAX_KERNEL_SLOTS] = {0};
  pk_status begin(int slot_id);
  pk_status end();
  pk_status flush();  // synchronise and accumulate
};

// Plain kernels shared by several solvers (pk_blas.cu).
void launch_spmv(const pk_csr* A, const double* x, double* y, cudaStream_t s);
void launch_dot_store(const pk_csr* A, const double* x, const double* y, double* out,
                      cudaStream_t s);
void launch_true_residual(pk_csr* A, const double* b, const double* x, double* tmp,
                          double* out2, cudaStream_t s);
RowArgs row_args(const pk_csr* A);

void launch_residual_init(const pk_csr* A, const double* b, const double* x, double* r,
                          double* p, double* r0s, cudaStream_t s);
void launch_zero_x(const pk_csr* A, double* x, cudaStream_t s);
pk_status check_opts(const pk_csr* A, const double* b, double* x, const pk_opts* o,
                     pk_info* info);

// Right preconditioning with M = diag(A) for BiCGStab and GMRES: while a JacobiRight is
// entered, A's values are those of A M^-1 and x holds y = M x; leave() restores both.
struct JacobiRight {
  pk_csr* A = nullptr;
  double* saved_va = nullptr;
  ~JacobiRight() {
    if (A) A->va = saved_va;  // error paths: values restored, x left in y form
  }
};
pk_status jacobi_right_enter(pk_csr* A, double* x, cudaStream_t s, JacobiRight* g);
pk_status jacobi_right_leave(JacobiRight* g, double* x, cudaStream_t s);

// SELL-C-sigma copy of a matrix (pk_sell.cu): slices of kSellC sorted rows, column-major.
constexpr int kSellC = 32;
constexpr int kSellWarps = kBlock / 32;
struct SellArgs {
  int32_t nslices;
  const int64_t* ptr;    // slice starts (entries), nslices + 1
  const int32_t* perm;   // row of every slice lane, -1 for padding lanes
  const int32_t* col;    // -1 for padding entries
  const double* val;
};
pk_status sell_build(pk_csr* A, cudaStream_t s);
SellArgs sell_args(const pk_csr* A);
pk_status launch_sell_spmv_dot(pk_csr* A, const double* p, double* q, double* out, cudaStream_t s);

// Row product of lane `lane` of a slice: entries k < w at stride 32, four loads in flight
// before their gathers and FMAs.
__device__ __forceinline__ double sell_row(const SellArgs& s, int64_t base, int w,
                                         const double* __restrict__ x) {
  const int32_t* __restrict__ cc = s.col + base;
  const double* __restrict__ vv = s.val + base;
  double acc = 0.0;
  int k = 0;
  for (; k + 4 <= w; k += 4) {
    int c[4];
    double v[4], xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = __ldg(cc + (size_t)(k + u) * kSellC);
      v[u] = __ldg(vv + (size_t)(k + u) * kSellC);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
  }
  for (; k < w; ++k) {
    const int c = __ldg(cc + (size_t)k * kSellC);
    if (c >= 0) acc = fma(__ldg(vv + (size_t)k * kSellC), __ldg(x + c), acc);
  }
  return acc;
}

// Kernels on the CSR tile engine take the instantiation with the grouped and whole-warp row
// paths when some tile needs one of them.
inline bool csr_irregular(const pk_csr* A) { return A->stats.tiles_long > 0 || A->stats.tiles_group > 0; }

inline long long passes_of(const DevState* h) {
  return *reinterpret_cast<const long long*>(&h->s[7]);
}

pk_status finish_info(pk_csr* A, const pk_opts* o, pk_info* info, cudaStream_t s,
                      const VecStage& v, cudaEvent_t e0, cudaEvent_t e1, int launches);

}  // namespace pk

namespace pk {

// y_row = sum_j A[row, j] x[j], left to right over the row (Sec. 2.2 CSR product).
// The row is walked in chunks of 4: all value / column loads of a chunk are issued before
// the dependent gathers of x, so a thread keeps several independent loads in flight instead
// of one load -> gather -> FMA round trip per nonzero.  The summation order is unchanged.
__device__ __forceinline__ double csr_row(const RowArgs& a, const double* __restrict__ x, int row) {
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
  if (j < j1) {
    int c[3];
    double v[3], xv[3];
    const int m = j1 - j;  // 1..3
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      c[k] = k < m ? __ldg(a.ci + j + k) : 0;
      v[k] = k < m ? __ldg(a.va + j + k) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) xv[k] = k < m ? __ldg(x + c[k]) : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < m) s = fma(v[k], xv[k], s);
  }
  return s;
}

// Rows of this block for elementwise kernels: equal chunks (multiples of 32 rows) over the
// launch grid, independent of the SpMV schedule.
__device__ __forceinline__ void ew_range(int n, int& r0, int& r1) {
  const int G = gridDim.x;
  const int chunk = (int)((((long long)n + G - 1) / G + 31) & ~31LL);
  const long long lo = (long long)blockIdx.x * chunk;
  r0 = (int)(lo < n ? lo : n);
  r1 = (int)(lo + chunk < n ? lo + chunk : n);
}

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

__device__ __forceinline__ bool state_done(const DevState* st) { return __ldcg(&st->done) != 0; }

}  // namespace pk

#include <functional>

namespace pk {

// One iteration's launches, replayed by the loop driver either inside a CUDA graph WHILE
// node (condition cleared on the device by the kernel that finishes the solve) or from a
// host loop that checks the device "done" flag.
struct LoopSpec {
  int kind = 0;                         // graph cache key: solver kind
  const void* keys[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t ikeys[4] = {0, 0, 0, 0};
  int body_kernels = 0;                 // kernels per body() call
  int unroll = 1;                       // body() calls per graph body pass
  std::function<void(cudaStream_t, Timer*)> body;
};

// Runs the loop until the device sets `done`; adds the launched kernels to *launches.
pk_status run_loop(pk_csr* A, const pk_opts* o, cudaStream_t s, const LoopSpec& L, Timer* T,
                   int* launches);

// Graph of two nested WHILE loops: outer { pre(); inner { body() }; post(); }.  The kernels
// clear DevState::cond (outer) and DevState::cond2 (inner); `g` caches the executable.
pk_status build_nested_graph(pk_csr* A, int kind, const void* const keys[4], const int64_t ikeys[4],
                             const std::function<void(cudaStream_t)>& pre,
                             const std::function<void(cudaStream_t)>& body,
                             const std::function<void(cudaStream_t)>& post, pk_graph_entry** out);
void launch_enable_cond2(pk_csr* A, const pk_graph_entry* g, cudaStream_t s);
// y = A x on the CSR tile engine (the unfused forms' SpMV); needs A->tma_ok.
pk_status launch_spmv_tma(pk_csr* A, const double* x, double* y, int first, int skip_early, cudaStream_t s);

// Counts body passes (first kernel of every body increments st->s[7] as an integer count).
__device__ __forceinline__ void count_pass(DevState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long* c = reinterpret_cast<long long*>(&st->s[7]);
    *c += 1;
  }
}

}  // namespace pk
