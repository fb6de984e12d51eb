// Grid-resident pipelined CG (Alg. 2, Sec. 3.1): the whole iteration loop in one cooperative
// launch of two blocks per SM, for systems too large for one thread-block cluster.
//
// In the launched form every iteration pays two grid-wide dependencies, each as the end of a
// kernel (grid completion, memory flush, release of the next kernel).  That fixed cost does
// not shrink with n, and at about 10^6 rows it is as long as the iteration's HBM traffic.
// Here the two fused phases of an iteration run back to back inside one launch, and only one
// dependency per iteration is grid-wide:
//   U_i  x_i = x_{i-1} + alpha p, r_i = r_{i-1} - alpha Ap, p_i = r_i + beta p, and the block's
//        part of <r_i, r_i>, over the block's own rows.  It needs alpha_{i-1}, beta_{i-1}: the
//        one grid-wide dependency (the reduction at the end of S_{i-1}).
//   S_i  Ap_i over the same rows, with the block's parts of <Ap_i, Ap_i> and <p_i, Ap_i>.  It
//        gathers p_i at the columns of its rows, so it only waits until the blocks that own
//        those rows have finished U_i (a flag per block, polled by one warp's lanes at once)
//        -- for a banded or stencil matrix a few neighbouring blocks, not the grid.
// Each block writes its three block sums to its own slot and releases an arrival flag; then
// warp 0 of EVERY block waits for all flags (all lanes polling at once), adds the slots in
// block order -- the same fixed order everywhere, so every block holds bit-identical sums, as
// deterministic as the launched kernels' last-block stage -- tests <r_i, r_i> against
// tol^2 <b, b> and maxit, and forms alpha_i and beta_i by Eq. (3).  No single block has to
// finish the reduction and publish it (measured on GB300: a last-block counter with 304
// blocks took 12 us from the last arrival to the published result).  The convergence test
// therefore comes one SpMV later than in the launched form; the iterates, alpha, beta and
// the iteration count are the same.
//
// Both phases run on the warp-specialised tile engines of the launched kernels, on the same
// blocks and tiles: the producer warp streams the block's vector rows (U) and CSR tiles (S)
// with bulk copies into one shared-memory region that the two phases take in turn (two blocks
// per SM, as in the launched kernels, keep enough warps in flight to hide the gathers and the
// FP64 latency; one block per SM with both rings measured 1.4x slower per iteration at 160^3).
// The data that does not depend on the awaited result is already in flight while the block
// waits (all four vectors of U are the block's own rows, written by its own threads; the
// matrix never changes).  The gathers of p read through L2 (other
// blocks rewrite p inside the launch).  Every wait is bounded (pk_opts.wait_ns): a block
// that gives up records PK_TIMEOUT, drains its copies and leaves, and the others then give
// up too, so the launch always ends.
#include <algorithm>
#include <vector>

#include "pk_tile.cuh"

namespace pk {

namespace {

constexpr int kResU = stream_smem_bytes<4, double, 1>();  // U ring: x, r, p, Ap
constexpr int kResSmem = kResU > csr_smem_bytes() ? kResU : csr_smem_bytes();  // the larger ring
constexpr int kResPerSm = 2;                                // resident blocks per SM
constexpr int kResSlotsPerLane = 10;                        // grid <= 320 blocks: one batch

struct ResArgs {
  CsrTiles T;              // the tiles of block b: [T.blk_tile[b], T.blk_tile[b+1])
  const int32_t* rows;     // block b owns rows [rows[b], rows[b+1])
  const int32_t* nbr;      // blocks [nbr[2b], nbr[2b+1]] own the columns block b gathers
  int32_t* flag;           // flag[b] = i once block b has written p_i (U_i done)
  int32_t* arrive;         // arrive[b] = i + 1 once block b's partials of iteration i are out
  double* x;
  double* r;
  double* p;
  double* ap;
  double* partials;        // [2][3][grid]: iteration parity, <r,r> <Ap,Ap> <p,Ap>, block
  DevState* st;
};

__device__ __forceinline__ void st_release(int32_t* a, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Generic-proxy writes of this thread made visible to later bulk copies (async proxy).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// After a phase, thread 0 invalidates the ring's barriers: the other phase's ring overlays the
// same shared memory (an mbarrier's memory may serve another purpose only once invalidated).
// Every copy has landed and every thread has left the phase (a block-wide barrier precedes).
__device__ __forceinline__ void inval_ring(unsigned char* bars, int count) {
  if (threadIdx.x == 0)
    for (int k = 0; k < count; ++k) mbar_inval(reinterpret_cast<uint64_t*>(bars) + k);
}

// Named barrier of the consumer warps (the producer warp runs its own path).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kConsumers) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int32_t* a) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Warp-wide bounded wait until flags[c] >= target for every c in [c0, c1] except `skip`:
// lane l polls blocks c0 + l, c0 + l + 32, ... with relaxed loads, all of them in flight at
// once (acquire loads would serialise: one round trip each), and once every flag has been
// seen the fence turns the observed releases into an acquire for the whole warp.  False once
// the solve's wait bound runs out or another block has given up (PK_TIMEOUT recorded).
// Called by all 32 lanes of one warp.
__device__ __forceinline__ bool warp_wait_flags(const int32_t* flags, int c0, int c1, int skip, int target,
                                                DevState* st) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  for (;;) {
    bool mine = true;
    for (int c = c0 + lane; c <= c1; c += 32)
      if (c != skip && ld_relaxed(flags + c) < target) mine = false;
    if (__all_sync(0xffffffffu, mine)) break;
    int give_up = 0;
    if (lane == 0) {
      if (!t0) t0 = global_ns();
      give_up = __ldcg(&st->timeout) || global_ns() - t0 > st->wait_ns;
    }
    if (__shfl_sync(0xffffffffu, give_up, 0)) {
      if (lane == 0) report_timeout(st);
      return false;
    }
    __nanosleep(32);
  }
  fence_acq_rel();
  __syncwarp();
  return true;
}

// Bounded spin of the producer lane on its own block's decision (shared memory).
__device__ __forceinline__ bool wait_block_decision(const volatile int* dec, int target, DevState* st) {
  if (*dec >= target) return true;
  const uint64_t t0 = global_ns();
  while (*dec < target) {
    if (global_ns() - t0 > st->wait_ns) {
      report_timeout(st);
      return false;
    }
    __nanosleep(32);
  }
  __threadfence_block();  // the decision's other fields were written before *dec
  return true;
}

template <bool IRR>
__global__ void __launch_bounds__(kTileThreads, 2) k_cg_resident(ResArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* smem_u = smem;  // U ring and CSR ring overlay one region
  unsigned char* smem_s = smem;
  __shared__ int s_go;          // consumers: the awaited data arrived and the solve is live
  __shared__ int s_stop;        // this block leaves the loop (a wait gave up)
  __shared__ volatile int s_dec;   // iteration whose reduction this block has completed
  __shared__ volatile int s_live;  // ... and whether the solve goes on after it
  __shared__ double s_ab[2];    // alpha, beta for U
  // barriers of the two rings (full + empty per stage), as the engines lay them out
  unsigned char* bars_u = smem_u + (size_t)stream_stages<4, double, 1>() * 4 * kStreamRows * sizeof(double);
  unsigned char* bars_s = smem_s + (size_t)kCsrStages * kStageBytes;
  DevState* st = a.st;
  if (state_done(st)) return;   // decided by the setup kernel, the same for every block
  const int b = blockIdx.x, G = gridDim.x;
  const int rb0 = a.rows[b], rb1 = a.rows[b + 1];
  const bool consumer = threadIdx.x < kConsumers;
  const int nb0 = a.nbr[2 * b], nb1 = a.nbr[2 * b + 1];
  const int maxit = st->maxit;
  const double thr2 = st->thr2;
  double rr = st->rr;           // <r_{i-1}, r_{i-1}>; <r_0, r_0> from the setup kernel
  CsrTiles T = a.T;
  if (threadIdx.x == 0) s_dec = -1;
  __syncthreads();

  // Second stage of iteration j's reductions, in warp 0 of every block: wait for every block's
  // slot (released after its partials), add the partials in block order -- the same order in
  // every block, so every block holds bit-identical sums -- test <r_j, r_j>, and form alpha_j,
  // beta_j (Eq. (3)).  Block 0 records the solver state for the host.  Result in s_ab / s_live.
  auto reduce = [&](int j) {
    const int lane = threadIdx.x & 31;
    bool ok = warp_wait_flags(a.arrive, 0, G - 1, -1, j + 1, st);
    double t[3] = {0.0, 0.0, 0.0};
    if (ok) {
      // all 3 x G slots in one batch of loads (G <= 32 * kResSlotsPerLane), then fixed-order adds
      lane_slot_sums<3, kResSlotsPerLane>(a.partials + (size_t)(j & 1) * 3 * G, G, lane, t);
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = warp_sum(t[k]);
    }
    if (lane == 0) {
      int status = kRunning;
      double alpha = 0.0, beta = 0.0;
      if (!ok) {
        status = PK_TIMEOUT;
      } else {
        if (j >= 1) rr = t[0];
        if (j >= 1 && !isfinite(t[0])) status = PK_ERR_NAN;
        else if (j >= 1 && t[0] <= thr2) status = PK_OK;
        else if (j >= 1 && j >= maxit) status = PK_NOT_CONVERGED;
        else if (!isfinite(t[1]) || !isfinite(t[2])) status = PK_ERR_NAN;
        else if (t[2] <= 0.0) status = PK_NOT_SPD;
        else {
          alpha = rr / t[2];
          beta = alpha * alpha * t[1] / rr - 1.0;
        }
      }
      if (b == 0 && ok) {
        if (j >= 1) {
          st->iter = j;
          st->rr = t[0];
          trace_put(st, j - 1, 3, t[0]);
        }
        if (status == kRunning) {
          st->alpha = alpha;
          st->beta = beta;
          trace_put(st, j, 0, alpha);
          trace_put(st, j, 1, beta);
        } else {
          finish(st, status);
        }
      }
      s_ab[0] = alpha;
      s_ab[1] = beta;
      s_live = status == kRunning;
      __threadfence_block();
      s_dec = j;
    }
    __syncwarp();
  };

  for (int i = 0;; ++i) {
    double vr = 0.0;  // this thread's part of <r_i, r_i>
    if (i >= 1) {
      // ---- U_i: needs alpha_{i-1}, beta_{i-1} (the reduction of iteration i - 1); the ring
      // is filling with this block's x, r, p, Ap meanwhile
      StreamIn<4> in{{a.x, a.r, a.p, a.ap}};
      stream_tiles<4, 4, double, 1>(in, rb0, rb1, smem_u, st, [&]() {
        if (consumer) {
          if (threadIdx.x < 32) reduce(i - 1);
          consumers_sync();
          if (threadIdx.x == 0) s_go = s_live;
          consumers_sync();
          return s_go != 0;
        }
        return wait_block_decision(&s_dec, i - 1, st) && s_live;
      }, [&](int row, const double2* val, int nv) {
        const double alpha = s_ab[0], beta = s_ab[1];
        const double2 xk = val[0], rq = val[1], pk = val[2], ak = val[3];
        double2 xn, rn, pn;
        xn.x = fma(alpha, pk.x, xk.x);
        xn.y = fma(alpha, pk.y, xk.y);
        rn.x = fma(-alpha, ak.x, rq.x);
        rn.y = fma(-alpha, ak.y, rq.y);
        pn.x = fma(beta, pk.x, rn.x);
        pn.y = fma(beta, pk.y, rn.y);
        if (nv == 2) {
          st2(a.x + row, xn);
          st2(a.r + row, rn);
          st2(a.p + row, pn);
          vr = fma(rn.x, rn.x, vr);
          vr = fma(rn.y, rn.y, vr);
        } else {
          a.x[row] = xn.x;
          a.r[row] = rn.x;
          a.p[row] = pn.x;
          vr = fma(rn.x, rn.x, vr);
        }
      });
      __syncthreads();  // s_go is final in every thread (producer included); the ring is idle
      inval_ring(bars_u, 2 * stream_stages<4, double, 1>());
      if (!s_go) break;
      // p_i of this block's rows is written: publish it to the blocks that gather it
      if (consumer) {
        fence_proxy_async();  // x, r, p are read back by this block's bulk copies next time
        consumers_sync();     // every consumer's p stores precede thread 0's release
        if (threadIdx.x == 0) {
          __threadfence();
          st_release(&a.flag[b], i);
        }
      }
    }
    // ---- S_i: wait until the blocks owning this block's columns have written p_i
    double v[3] = {vr, 0.0, 0.0};
    const CohVec<double> pv{a.p};
    csr_tiles<IRR>(T, smem_s, st, [&]() {
      if (!consumer) return true;  // the matrix tiles do not depend on p
      if (threadIdx.x < 32) {
        const bool ok = i == 0 || warp_wait_flags(a.flag, nb0, nb1, b, i, st);
        if (threadIdx.x == 0) s_go = ok;
      }
      consumers_sync();
      return s_go != 0;
    }, pv, [&](int row, double y) {
      a.ap[row] = y;
      v[1] = fma(y, y, v[1]);
      v[2] = fma(__ldcg(a.p + row), y, v[2]);
    });
    if (consumer) fence_proxy_async();  // Ap is read back by this block's bulk copies in U_{i+1}
    // ---- this block's part of iteration i's reductions: slot (i & 1), then its arrival
    tile_block_partials<3>(v, a.partials + (size_t)(i & 1) * 3 * G);  // written by thread 0
    inval_ring(bars_s, 2 * kCsrStages);  // (after the barrier inside: the CSR ring is idle)
    if (threadIdx.x == 0) {
      st_release(&a.arrive[b], i + 1);
      s_stop = __ldcg(&st->timeout);
    }
    __syncthreads();
    if (s_stop) break;
  }
}

// Rows and neighbour blocks of the resident grid: resident block b is tile block b of the
// launched kernels (contiguous rows starting on a multiple of 32); its SpMV reads p at the
// columns [cmin, cmax] of its rows, owned by blocks [lo, hi].
__global__ void k_res_plan_rows(const int32_t* tile_row, const int32_t* blk_tile, int G, int32_t* rows) {
  for (int b = threadIdx.x; b <= G; b += blockDim.x) rows[b] = tile_row[blk_tile[b]];
}

__global__ void k_res_plan_nbr(const int32_t* rp, const int32_t* ci, const int32_t* rows, int G,
                               int32_t* nbr) {
  __shared__ int smin[32], smax[32];
  const int b = blockIdx.x;
  const int z0 = rp[rows[b]], z1 = rp[rows[b + 1]];
  int mn = INT32_MAX, mx = -1;
  for (int z = z0 + threadIdx.x; z < z1; z += blockDim.x) {
    const int c = ci[z];
    mn = min(mn, c);
    mx = max(mx, c);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    smin[threadIdx.x >> 5] = mn;
    smax[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)blockDim.x / 32; ++w) {
      mn = min(mn, smin[w]);
      mx = max(mx, smax[w]);
    }
    mn = min(mn, smin[0]);
    mx = max(mx, smax[0]);
    int lo = b, hi = b;  // no nonzeros: only its own rows
    if (mx >= 0) {
      // owner of column c: the last block with rows[blk] <= c
      auto owner = [&](int c) {
        int l = 0, h = G - 1;
        while (l < h) {
          const int m = (l + h + 1) / 2;
          if (rows[m] <= c) l = m; else h = m - 1;
        }
        return l;
      };
      lo = owner(mn);
      hi = owner(mx);
    }
    nbr[2 * b] = lo;
    nbr[2 * b + 1] = hi;
  }
}

pk_status res_setup_attrs() {
  static bool done = false;
  if (!done) {
    for (auto k : {k_cg_resident<false>, k_cg_resident<true>})
      PK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmem));
    done = true;
  }
  return PK_OK;
}

}  // namespace

// Whether the grid-resident loop can run A on this device: the tile engine is in use, the
// tile grid has two blocks per SM, and two blocks with the larger ring fit on every SM.
pk_status resident_prepare(pk_csr* A, cudaStream_t s, bool* usable) {
  *usable = false;
  if (A->res_grid < 0) return PK_OK;
  if (A->res_grid > 0) { *usable = true; return PK_OK; }
  A->res_grid = -1;
  if (!A->tma_ok) return PK_OK;
  int sms = 1, coop = 0;
  PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
  PK_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, A->device));
  if (!coop || A->grid_tma != kResPerSm * sms || A->grid_tma > 32 * kResSlotsPerLane) return PK_OK;
  pk_status e = res_setup_attrs();
  if (e) return e;
  int per_sm = 0;
  PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_resident<true>, kTileThreads, kResSmem));
  int per_sm0 = 0;
  PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm0, k_cg_resident<false>, kTileThreads, kResSmem));
  if (std::min(per_sm, per_sm0) < kResPerSm) return PK_OK;
  const int G = A->grid_tma;
  PK_CUDA(cudaMalloc(&A->res_rows, sizeof(int32_t) * (G + 1)));
  PK_CUDA(cudaMalloc(&A->res_nbr, sizeof(int32_t) * 2 * G));
  PK_CUDA(cudaMalloc(&A->res_flag, sizeof(int32_t) * 2 * G));  // p-written flags, arrivals
  k_res_plan_rows<<<1, 256, 0, s>>>(A->tile_row, A->blk_tile, G, A->res_rows);
  k_res_plan_nbr<<<G, 256, 0, s>>>(A->rp, A->ci, A->res_rows, G, A->res_nbr);
  PK_CUDA(cudaGetLastError());
  A->res_grid = G;
  *usable = true;
  return PK_OK;
}

// Launches the resident loop after the setup kernel (r0, p0, <r0,r0>, <b,b>): the phases
// S_0, U_1, S_1, ... until the last block of a reduction ends the solve.
pk_status launch_cg_resident(pk_csr* A, double* x, double* r, double* p, double* ap, cudaStream_t s) {
  const int G = A->res_grid;
  PK_CUDA(cudaMemsetAsync(A->res_flag, 0, sizeof(int32_t) * 2 * G, s));
  ResArgs ra;
  ra.T = csr_tiles_of(A);
  ra.rows = A->res_rows;
  ra.nbr = A->res_nbr;
  ra.flag = A->res_flag;
  ra.arrive = A->res_flag + G;
  ra.x = x;
  ra.r = r;
  ra.p = p;
  ra.ap = ap;
  ra.partials = A->partials;
  ra.st = A->st;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kTileThreads);
  cfg.dynamicSmemBytes = kResSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // every block resident at once (they wait on each other)
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PK_CUDA(cudaLaunchKernelEx(&cfg, csr_irregular(A) ? k_cg_resident<true> : k_cg_resident<false>, ra));
  return PK_OK;
}

}  // namespace pk
