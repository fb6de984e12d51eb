// Warp-specialised tile engine for the bandwidth-bound fused kernels (sm_100+ / sm_103a).
//
// On GB300 the FP64 pipe (about 2 FMA per clock per SM) is as much of a bound as HBM for the
// fused Krylov kernels, and a warp that waits for its own loads cannot feed the FP64 pipe.
// Here one producer warp per block streams the block's data into a ring of shared-memory
// stages with bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier)
// while eight consumer warps do the floating-point work on stages that have already arrived,
// so memory traffic and FP64 work overlap.  Every wait on an mbarrier is bounded: after
// 2 s the kernel records PK_TIMEOUT and returns.
#pragma once

#include "pk_internal.cuh"

namespace pk {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;        // 256 consumer threads
constexpr int kTileThreads = kConsumers + 32;          // + one producer warp
constexpr uint64_t kWaitNs = 2000000000ull;            // 2 s bound on every mbarrier wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on phase `parity`: false once about `budget_ns` nanoseconds have passed.
// Pipeline waits that should make progress take the solve's budget (pk_opts.wait_ns, 2 s by
// default); the drain of a block's own copies before it exits always takes kWaitNs.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, uint64_t budget_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > budget_ns) return false;
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitNs);
}

// A progress wait bounded by the solve's budget, read only once the first try has failed.
__device__ __forceinline__ bool mbar_wait_st(uint64_t* bar, uint32_t parity, const DevState* st) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_for(bar, parity, st->wait_ns);
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completion
// signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// L2 policy that evicts the streamed data first (the matrix is read once per pass and does not
// fit in L2; the gathered vector should stay there).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes,
                                               uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
      "%2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

// Adds expected transaction bytes to the current phase without arriving.
__device__ __forceinline__ void mbar_add_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Programmatic dependent launch: wait until the preceding kernel of the stream has completed
// and its memory is visible (a no-op when launched without the programmatic attribute) ...
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// ... and allow the next kernel to be scheduled once every block of this one got here.
__device__ __forceinline__ void griddep_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Record a timed-out wait (first writer wins) so the host sees PK_TIMEOUT.
__device__ __forceinline__ void report_timeout(DevState* st) {
  atomicExch(&st->timeout, 1);
}

// Reduction of NV values over the consumer threads of a tile block (the producer warp
// contributes zeros), written to partials[k * gridDim.x + blockIdx.x].
template <int NV>
__device__ __forceinline__ void tile_block_partials(double (&v)[NV], double* partials) {
  __shared__ double sm[NV][kTileThreads / 32];
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
      if (lane == 0) partials[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
  }
}

// ----------------------------------------------------------------------------------------
// Streaming tiles: NIN length-n float64 vectors, TROWS rows per tile, NST stages.
// Rows of block b: equal chunks of the grid (multiples of 32 rows).

// Element pair read by a consumer thread (two consecutive rows of one input).
template <class ET>
struct Pair;
template <>
struct Pair<double> { using type = double2; };
template <>
struct Pair<float> { using type = float2; };

template <int NIN, class ET = double>
struct StreamIn {
  const ET* v[NIN];
};

constexpr int kStreamRows = 512;  // rows per streaming tile: 2 per consumer thread

// Stages of the streaming ring: as many as fit in kStreamBudget bytes, 2..8.  U row pairs
// per consumer thread per stage (kStreamRows * U rows): light kernels take several so that the
// per-stage barrier traffic is amortised over more work.  96 KB keeps two blocks per SM; a
// 112 KB ring measured no faster on GB300 (the 5-input update kernel is bound by FP64 issue
// as much as by HBM).
constexpr int kStreamBudget = 98304;

template <int NIN, class ET = double, int U = 1>
__host__ __device__ constexpr int stream_stages() {
  return (kStreamBudget / (NIN * kStreamRows * U * (int)sizeof(ET))) > 8 ? 8
         : (kStreamBudget / (NIN * kStreamRows * U * (int)sizeof(ET))) < 2
             ? 2
             : (kStreamBudget / (NIN * kStreamRows * U * (int)sizeof(ET)));
}

template <int NIN, class ET = double, int U = 1>
__host__ __device__ constexpr int stream_smem_bytes() {
  return stream_stages<NIN, ET, U>() * NIN * kStreamRows * U * (int)sizeof(ET) + 2 * stream_stages<NIN, ET, U>() * 8;
}

// Runs the streaming pipeline.  The first NPRE inputs do not depend on the preceding
// kernel: the producer copies them for the first stages before the grid-dependency wait
// (programmatic dependent launch), the remaining inputs after it.  After the wait the
// producer and every consumer call `setup()`, which reads the solver state and returns false
// if this kernel has nothing to do (the block then only drains what was prefetched); it must
// give the same answer in every thread.  `body(row, vals, nvalid)` is called for row pairs
// (vals[k] = the pair of input k at rows row, row+1; nvalid = 1 or 2).  Returns, in consumer
// threads, whether the solve was live (a timed-out wait is recorded in the state and ends the
// loop early).  ET is the element type (double, or float for the mixed-precision inner loop).
template <int NIN, int NPRE, class ET = double, int U = 1, class Setup, class Body>
__device__ __forceinline__ bool stream_tiles(const StreamIn<NIN, ET>& in, int r0, int r1,
                                             unsigned char* smem, DevState* st, Setup&& setup,
                                             Body&& body) {
  using P2 = typename Pair<ET>::type;
  constexpr int kStreamStages = stream_stages<NIN, ET, U>();
  constexpr int kRows = kStreamRows * U;  // rows per stage
  constexpr int kPerUnit = 16 / (int)sizeof(ET);  // elements per 16-byte copy unit
  ET* buf = reinterpret_cast<ET*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kStreamStages * NIN * kRows * sizeof(ET));
  uint64_t* empty = full + kStreamStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStreamStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int ntiles = r1 > r0 ? (r1 - r0 + kRows - 1) / kRows : 0;
  const int npro = min(kStreamStages, ntiles);
  auto tile_bytes = [&](int t) {
    const int rows = min(kRows, r1 - (r0 + t * kRows));
    return (uint32_t)(((rows + kPerUnit - 1) / kPerUnit) * 16);  // whole 16-byte units
  };
  auto issue = [&](int t, int k0, int k1) {
    const int s = t % kStreamStages;
    const int row0 = r0 + t * kRows;
    const uint32_t bytes = tile_bytes(t);
#pragma unroll
    for (int k = 0; k < NIN; ++k)
      if (k >= k0 && k < k1)
        bulk_load(buf + ((size_t)s * NIN + k) * kRows, in.v[k] + row0, bytes, &full[s]);
  };
  bool ok = true;
  if (warp == kConsumerWarps) {
    if (lane == 0) {
      // prologue: inputs independent of the preceding kernel, first stages
      for (int t = 0; t < npro; ++t) {
        mbar_add_tx(&full[t], tile_bytes(t) * NPRE);
        issue(t, 0, NPRE);
      }
      griddep_wait();
      const bool live = setup();  // the same predicate the consumers evaluate
      for (int t = 0; t < npro; ++t) {
        if (live) {
          mbar_expect_tx(&full[t], tile_bytes(t) * (NIN - NPRE));
          issue(t, NPRE, NIN);
        } else {
          mbar_arrive(&full[t]);
        }
      }
      int issued = npro;
      if (live) {
        for (int t = npro; t < ntiles; ++t) {
          const int s = t % kStreamStages;
          if (!mbar_wait_st(&empty[s], ((t / kStreamStages) - 1) & 1, st)) { ok = false; report_timeout(st); break; }
          mbar_expect_tx(&full[s], tile_bytes(t) * NIN);
          issue(t, 0, NIN);
          issued = t + 1;
        }
      }
      // drain: wait (bounded) until the copies this block issued have landed
      for (int t = max(0, issued - kStreamStages); t < issued; ++t)
        if (!mbar_wait(&full[t % kStreamStages], (t / kStreamStages) & 1)) { ok = false; report_timeout(st); break; }
    }
    return ok;
  }
  griddep_wait();
  const bool live = setup();
  const int nproc = live ? ntiles : npro;
  for (int t = 0; t < nproc; ++t) {
    const int s = t % kStreamStages;
    if (!mbar_wait_st(&full[s], (t / kStreamStages) & 1, st)) { report_timeout(st); break; }
    if (live) {
      const int row0 = r0 + t * kRows;
      const int rows = min(kRows, r1 - row0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = 2 * ((int)threadIdx.x + u * kConsumers);  // consumer thread -> row pairs
        if (i < rows) {
          P2 vals[NIN];
#pragma unroll
          for (int k = 0; k < NIN; ++k)
            vals[k] = *reinterpret_cast<const P2*>(buf + ((size_t)s * NIN + k) * kRows + i);
          body(row0 + i, vals, min(2, rows - i));
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  return live;
}

// ----------------------------------------------------------------------------------------
// CSR tiles: each tile holds <= kTileRows rows and <= kTileNnz nonzeros; the producer copies
// the tile's row pointers, values and column indices (16-byte aligned windows).

constexpr int kTileRows = 512;       // two rows per consumer thread
constexpr int kTileNnz = 4096;
constexpr int kCsrStages = 2;
constexpr int kRpWords = kTileRows + 8;       // ints, incl. alignment slack
constexpr int kVaWords = kTileNnz + 2;        // doubles
constexpr int kCiWords = kTileNnz + 8;        // ints (window rounded out to 16 bytes on both ends)
constexpr int kCiBytes = (kCiWords * 4 + 15) & ~15;
constexpr int kStageBytes = ((kRpWords * 4 + 15) & ~15) + kVaWords * 8 + kCiBytes + kTileRows * 2;  // + row order

constexpr int csr_smem_bytes() { return kCsrStages * kStageBytes + 2 * kCsrStages * 8 + kCsrStages * 16; }

// Gathers of the SpMV's input vector.  A plain pointer reads through the non-coherent path
// (the vector is read-only while the kernel runs); CohVec reads through L2 only, for the
// grid-resident CG loop, in which other blocks rewrite the vector between the phases of one
// launch and a non-coherent copy could be stale.
template <class VT>
struct CohVec {
  const VT* p;
};
__device__ __forceinline__ double gather(const double* __restrict__ x, int c) { return __ldg(x + c); }
__device__ __forceinline__ float gather(const float* __restrict__ x, int c) { return __ldg(x + c); }
template <class VT>
__device__ __forceinline__ VT gather(CohVec<VT> x, int c) { return __ldcg(x.p + c); }
// BlockVec: a vector that only the reading block writes (the batched solver: one block owns a
// system's vectors).  Plain L1-cached loads see the block's own earlier stores after a block
// barrier; the non-coherent path might not.
template <class VT>
struct BlockVec {
  const VT* p;
};
template <class VT>
__device__ __forceinline__ VT gather(BlockVec<VT> x, int c) { return __ldca(x.p + c); }

template <class VT>
struct CsrTilesT {
  const int32_t* rp;
  const int32_t* ci;
  const VT* va;             // values: FP64, or the FP32 copy for the mixed-precision inner loop
  const int32_t* tile_row;  // row start of every tile (global tile list), plus n at the end
  const int32_t* blk_tile;  // tiles of block b: [blk_tile[b], blk_tile[b+1])
  const int8_t* tile_grp;   // 1: every row of the tile has at most kLongRow nonzeros
  const int16_t* tile_perm; // [tile][512]: row (offset in the tile) of every consumer slot, or -1
  const int32_t* tile_z0;   // chunk tiles (tile_grp 64): first nonzero of the chunk, else -1
};
using CsrTiles = CsrTilesT<double>;

// FMAs k < M of one gathered batch of any element type, lane-predicated on k < m.
template <int M, class VT>
__device__ __forceinline__ void fma_batch_g(const VT (&v)[8], const VT (&xv)[8], int m, VT& s) {
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k < m) s = fma_t(v[k], xv[k], s);
}

template <class VT>
__device__ __forceinline__ void fma_batch_gn(int mx, const VT (&v)[8], const VT (&xv)[8], int m, VT& s) {
  switch (mx) {
    case 1: fma_batch_g<1>(v, xv, m, s); break;
    case 2: fma_batch_g<2>(v, xv, m, s); break;
    case 3: fma_batch_g<3>(v, xv, m, s); break;
    case 4: fma_batch_g<4>(v, xv, m, s); break;
    case 5: fma_batch_g<5>(v, xv, m, s); break;
    case 6: fma_batch_g<6>(v, xv, m, s); break;
    case 7: fma_batch_g<7>(v, xv, m, s); break;
    case 8: fma_batch_g<8>(v, xv, m, s); break;
    default: break;
  }
}

// One row product by a group of G lanes (G a power of two <= 16, the group aligned in the
// warp): lane q sums entries j0 + q, j0 + q + G, ... left to right, up to 8 gathers in flight
// before their FMAs, then the group adds its partial sums by a butterfly.  Warp-uniform:
// every lane of the warp calls it together (lanes without a row pass j = j1), and the batch
// loop runs to the warp's longest share, issuing only that many FMAs (predicated-off FP64
// instructions still take issue slots).
template <int G, class VT, class XP>
__device__ __forceinline__ VT group_row(const VT* sva, const int32_t* sci, int j, int j1, XP x) {
  VT s = (VT)0;
  for (;;) {
    const int m = j < j1 ? min(8, (j1 - j + G - 1) / G) : 0;
    const int mx = __reduce_max_sync(0xffffffffu, m);
    if (mx == 0) break;
    int c[8];
    VT v[8], xv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c[k] = k < m ? sci[j + k * G] : 0;
      v[k] = k < m ? sva[j + k * G] : (VT)0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] = k < m ? gather(x, c[k]) : (VT)0;
    fma_batch_gn(mx, v, xv, m, s);
    j += 8 * G;
  }
#pragma unroll
  for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// The rows of a grouped tile: kConsumers / G rows per round, rows in order.  Rounds are the
// same for the whole block, so every lane reaches the group's shuffles.
template <int G, class VT, class XP, class RowDone>
__device__ __forceinline__ void group_rows(const int32_t* srp, const VT* sva, const int32_t* sci, int R0,
                                           int R1, XP x, RowDone& row_done) {
  constexpr int ng = kConsumers / G;
  const int gid = (int)threadIdx.x / G, q = (int)threadIdx.x & (G - 1);
  const int rounds = (R1 - R0 + ng - 1) / ng;
  for (int k = 0; k < rounds; ++k) {
    const int r = R0 + gid + k * ng;
    const int j0 = r < R1 ? srp[r] + q : 0, j1 = r < R1 ? srp[r + 1] : 0;
    const VT acc = group_row<G>(sva, sci, j0, j1, x);
    if (r < R1 && q == 0) row_done(r, acc);
  }
}

// Two row products from a shared-memory window (defined below): FP64 and FP32.
template <class XP>
__device__ __forceinline__ void row_pair(const double* sva, const int32_t* sci, int ja, int ja1, int jb,
                                         int jb1, XP x, double& sa, double& sb);
template <class XP>
__device__ __forceinline__ void row_pair(const float* sva, const int32_t* sci, int ja, int ja1, int jb,
                                         int jb1, XP x, float& sa, float& sb);

// Runs the CSR pipeline and the row products y_row = sum_j A[row][j] x[col j]; every finished
// row goes to `row_done(row, y_row)`, called by the one consumer thread that owns the row.
// Consumer thread t computes rows R0 + t and R0 + t + 256 of every tile itself (summed left
// to right, the order of a plain CSR loop).  In tiles that hold rows longer than kLongRow
// nonzeros (T.tile_grp != 1, set at pk_csr_create) a thread skips its long rows, and each
// warp then takes its lanes' long rows one at a time with all 32 lanes (lane l sums entries
// l, l + 32, ... left to right, then a butterfly), so that no thread walks a long row alone;
// no synchronisation beyond the warp is involved.  Tiles of rows of similar length that are
// too long for one thread (T.tile_grp = G in 2..16) give each row a group of G lanes instead.
// A row longer than a tile is cut into chunk tiles of kTileNnz nonzeros (T.tile_grp = 64,
// consecutive tiles of one block) and summed by the whole block: see block_row_chunk.
constexpr int kLongRow = 32;
constexpr int kChunkTile = 64;

// One chunk tile of a row longer than a tile (block per row).  The chunk's nonzeros
// [zc0, min(zr1, zc0 + kTileNnz)) sit in the stage's value and column windows.  Thread t
// takes the entries whose offset in the row is t modulo kConsumers (chunks hold whole
// multiples of kConsumers, so that share is the same in every chunk) and sums its share left to
// right across all the row's chunks in `acc`.  After the row's last chunk each warp adds its
// lanes by a butterfly and posts the sum; the warp that posts last adds the kConsumerWarps
// sums in warp order and hands the row to row_done.  No warp waits for another (a warp that
// timed out elsewhere cannot stall this one).  The warp that posts last resets the counter
// before it releases the stage; with two stages no warp can reach the next long row's last
// chunk (at least two tiles on) before that.
static_assert(kCsrStages <= 2, "the chunk-row counter is reused two tiles after its last use");
static_assert(kTileNnz % kConsumers == 0, "chunks must hold whole multiples of the consumer count");

template <class VT, class XP, class RowDone>
__device__ __forceinline__ void block_row_chunk(int row, int zc0, int zr1, VT* stage_va, int32_t* stage_ci,
                                                XP x, VT& acc, VT* red, int* cnt,
                                                int warp, int lane, RowDone& row_done) {
  constexpr int kVaUnit = 16 / (int)sizeof(VT);
  const int zc1 = min(zr1, zc0 + kTileNnz);
  const VT* sva = stage_va - (zc0 & ~(kVaUnit - 1));
  const int32_t* sci = stage_ci - (zc0 & ~3);
  for (int j = zc0 + (int)threadIdx.x; j < zc1; j += kConsumers) acc = fma_t(sva[j], gather(x, sci[j]), acc);
  if (zc1 != zr1) return;  // more chunks of this row follow
  VT w = acc;
  acc = (VT)0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  int last = 0;
  if (lane == 0) {
    red[warp] = w;
    __threadfence_block();
    last = atomicAdd(cnt, 1) == kConsumerWarps - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last && lane == 0) {
    __threadfence_block();
    VT tot = (VT)0;
    const volatile VT* vr = red;
    for (int k = 0; k < kConsumerWarps; ++k) tot += vr[k];
    *cnt = 0;
    row_done(row, tot);
  }
}

// IRR = false compiles the thread-per-row path only (matrices without long rows).
// csr_tiles_range runs the tiles [t0, t1) of T in this block; csr_tiles runs the block's own
// range [T.blk_tile[blockIdx.x], T.blk_tile[blockIdx.x + 1]).
template <bool IRR, class VT, class XP, class Setup, class RowDone>
__device__ __forceinline__ bool csr_tiles_range(const CsrTilesT<VT>& T, int t0, int t1, unsigned char* smem,
                                                DevState* st, Setup&& setup, XP x, RowDone&& row_done) {
  constexpr int kVaUnit = 16 / (int)sizeof(VT);  // values per 16-byte copy unit
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kCsrStages * kStageBytes);
  uint64_t* empty = full + kCsrStages;
  int4* meta = reinterpret_cast<int4*>(empty + kCsrStages);  // tile rows [R0, R1), lanes per row
  __shared__ VT chunk_red[kConsumerWarps];  // warp sums of a long row (chunk tiles)
  __shared__ int chunk_cnt;                 // warps that have added their sum
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kCsrStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    mbar_fence_init();
    chunk_cnt = 0;
  }
  __syncthreads();
  const int ntiles = t1 - t0;
  auto stage_rp = [&](int s) { return reinterpret_cast<int32_t*>(smem + (size_t)s * kStageBytes); };
  auto stage_va = [&](int s) {
    return reinterpret_cast<VT*>(smem + (size_t)s * kStageBytes + ((kRpWords * 4 + 15) & ~15));
  };
  auto stage_ci = [&](int s) {
    return reinterpret_cast<int32_t*>(smem + (size_t)s * kStageBytes + ((kRpWords * 4 + 15) & ~15) +
                                      kVaWords * 8);
  };
  auto stage_perm = [&](int s) {
    return reinterpret_cast<int16_t*>(smem + (size_t)s * kStageBytes + ((kRpWords * 4 + 15) & ~15) +
                                      kVaWords * 8 + kCiBytes);
  };
  const int npro = min(kCsrStages, ntiles);
  bool ok = true;
  if (warp == kConsumerWarps) {
    // PK_FLAG_TEST_STALL: no copy is issued, so every consumer's first wait runs out after the
    // solve's wait bound (the timeout path, tested without a fault: nothing is in flight)
    if (st->stall_test) {
      griddep_wait();
      return false;
    }
    // producer warp: lanes prefetch tile bounds 32 tiles at a time, lane 0 issues copies.
    // The matrix does not depend on the preceding kernel: the first stages are issued before
    // the grid-dependency wait; after it the producer stops if the solve has finished.
    int issued = 0;
    bool live = true;
    const uint64_t pol = l2_evict_first();
    for (int base = 0; base < ntiles && ok && live; base += 32) {
      const int tt = t0 + base + lane;
      int R0 = 0, R1 = 0, z0 = 0, z1 = 0, gr = 1;
      if (tt < t1) {
        R0 = __ldg(T.tile_row + tt);
        gr = T.tile_grp ? (int)__ldg(T.tile_grp + tt) : 1;
        if (gr == kChunkTile) {  // one chunk of row R0: nonzeros [z0, z1)
          R1 = R0 + 1;
          z0 = __ldg(T.tile_z0 + tt);
          z1 = min(__ldg(T.rp + R0 + 1), z0 + kTileNnz);
        } else {
          R1 = __ldg(T.tile_row + tt + 1);
          z0 = __ldg(T.rp + R0);
          z1 = __ldg(T.rp + R1);
        }
      }
      const int cnt = min(32, ntiles - base);
      for (int q = 0; q < cnt; ++q) {
        const int a0 = __shfl_sync(0xffffffffu, R0, q), a1 = __shfl_sync(0xffffffffu, R1, q);
        const int b0 = __shfl_sync(0xffffffffu, z0, q), b1 = __shfl_sync(0xffffffffu, z1, q);
        const int g0 = __shfl_sync(0xffffffffu, gr, q);
        if (lane == 0) {
          const int t = base + q;
          const int s = t % kCsrStages;
          const int use = t / kCsrStages;
          if (use > 0 && !mbar_wait_st(&empty[s], (use - 1) & 1, st)) { ok = false; report_timeout(st); }
          if (ok) {
            const int rs = a0 & ~3, re = (a1 + 1 + 3) & ~3;    // row pointers a0..a1
            const int vs = b0 & ~(kVaUnit - 1), ve = (b1 + kVaUnit - 1) & ~(kVaUnit - 1);  // values
            const int cs = b0 & ~3, ce = (b1 + 3) & ~3;        // columns b0..b1-1
            const uint32_t nrp = (uint32_t)(re - rs) * 4, nva = (uint32_t)(ve - vs) * (uint32_t)sizeof(VT),
                           nci = (uint32_t)(ce - cs) * 4;
            const bool perm = g0 == 32 && T.tile_perm;  // irregular tile: its row order too
            // published by the arrive below (release); w: the row order flag, or a chunk's start
            meta[s] = make_int4(a0, a1, g0, g0 == kChunkTile ? b0 : (perm ? 1 : 0));
            mbar_expect_tx(&full[s], nrp + nva + nci + (perm ? kTileRows * 2 : 0));
            bulk_load_hint(stage_rp(s), T.rp + rs, nrp, &full[s], pol);
            if (nva) bulk_load_hint(stage_va(s), T.va + vs, nva, &full[s], pol);
            if (nci) bulk_load_hint(stage_ci(s), T.ci + cs, nci, &full[s], pol);
            if (perm) bulk_load_hint(stage_perm(s), T.tile_perm + (size_t)(t0 + t) * kTileRows, kTileRows * 2, &full[s], pol);
            issued = t + 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        if (base + q + 1 == npro) {
          griddep_wait();
          live = setup();  // the same predicate the consumers evaluate
          if (!live) break;
        }
      }
    }
    if (npro == 0) griddep_wait();
    if (lane == 0) {
      for (int t = max(0, issued - kCsrStages); t < issued; ++t)
        if (!mbar_wait(&full[t % kCsrStages], (t / kCsrStages) & 1)) { report_timeout(st); break; }
    }
    return ok;
  }
  griddep_wait();
  const bool live = setup();
  const int nproc = live ? ntiles : npro;
  VT chunk_acc = (VT)0;  // this thread's share of the current long row (chunk tiles)
  for (int t = 0; t < nproc; ++t) {
    const int s = t % kCsrStages;
    if (!mbar_wait_st(&full[s], (t / kCsrStages) & 1, st)) { report_timeout(st); break; }
    if (!live) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      continue;
    }
    const int4 m = meta[s];
    const int R0 = m.x, R1 = m.y, G = m.z;
    const int32_t* srp = stage_rp(s) - (R0 & ~3);
    const int z0 = srp[R0];
    const VT* sva = stage_va(s) - (z0 & ~(kVaUnit - 1));  // windows start at the first row's nonzeros
    const int32_t* sci = stage_ci(s) - (z0 & ~3);
    if (IRR && G == kChunkTile) {
      block_row_chunk(R0, m.w, srp[R0 + 1], stage_va(s), stage_ci(s), x, chunk_acc, chunk_red, &chunk_cnt,
                      warp, lane, row_done);
    } else if (!IRR || G == 1) {
      const int ra = R0 + (int)threadIdx.x;
      if (ra < R1) {
        const int rb = ra + kConsumers < R1 ? ra + kConsumers : -1;
        VT sa, sb;
        row_pair(sva, sci, srp[ra], srp[ra + 1], rb >= 0 ? srp[rb] : 0, rb >= 0 ? srp[rb + 1] : 0, x, sa, sb);
        row_done(ra, sa);
        if (rb >= 0) row_done(rb, sb);
      }
    } else if (G < 32) {
      // rows of similar length, too long for one thread: G lanes per row (G = 2..16)
      switch (G) {
        case 2: group_rows<2>(srp, sva, sci, R0, R1, x, row_done); break;
        case 4: group_rows<4>(srp, sva, sci, R0, R1, x, row_done); break;
        case 8: group_rows<8>(srp, sva, sci, R0, R1, x, row_done); break;
        default: group_rows<16>(srp, sva, sci, R0, R1, x, row_done); break;
      }
    } else {
      // every lane takes part (the ballots below need the whole warp).  With a row order
      // (sorted by length, dealt round-robin over the warps) each warp holds rows of similar
      // length, so its FMA batches carry few idle lanes.
      const int16_t* sperm = m.w ? stage_perm(s) : nullptr;
      const int ka = sperm ? sperm[threadIdx.x] : (int)threadIdx.x;
      const int kb = sperm ? sperm[threadIdx.x + kConsumers] : (int)threadIdx.x + kConsumers;
      const int ra = ka >= 0 && R0 + ka < R1 ? R0 + ka : -1;
      const int rb = kb >= 0 && R0 + kb < R1 ? R0 + kb : -1;
      int ja0 = ra >= 0 ? srp[ra] : 0, ja1 = ra >= 0 ? srp[ra + 1] : 0;
      int jb0 = rb >= 0 ? srp[rb] : 0, jb1 = rb >= 0 ? srp[rb + 1] : 0;
      const bool la = ja1 - ja0 > kLongRow, lb = jb1 - jb0 > kLongRow;
      if (ra >= 0 || rb >= 0) {
        VT sa, sb;
        row_pair(sva, sci, ja0, la ? ja0 : ja1, jb0, lb ? jb0 : jb1, x, sa, sb);
        if (ra >= 0 && !la) row_done(ra, sa);
        if (rb >= 0 && !lb) row_done(rb, sb);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        unsigned pending = __ballot_sync(0xffffffffu, h == 0 ? la : lb);
        while (pending) {
          const int src = __ffs(pending) - 1;
          pending &= pending - 1;
          const int r = __shfl_sync(0xffffffffu, h == 0 ? ra : rb, src);
          const int j0 = srp[r], j1 = srp[r + 1];
          VT acc = (VT)0;
          for (int j = j0 + lane; j < j1; j += 32) acc = fma_t(sva[j], gather(x, sci[j]), acc);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == src) row_done(r, acc);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  return live;
}

template <bool IRR, class VT, class XP, class Setup, class RowDone>
__device__ __forceinline__ bool csr_tiles(const CsrTilesT<VT>& T, unsigned char* smem, DevState* st,
                                          Setup&& setup, XP x, RowDone&& row_done) {
  return csr_tiles_range<IRR>(T, T.blk_tile[blockIdx.x], T.blk_tile[blockIdx.x + 1], smem, st,
                              static_cast<Setup&&>(setup), x, static_cast<RowDone&&>(row_done));
}

// Two row products from a shared-memory window.  Each pass loads up to 8 entries of both
// rows and issues all their gathers before the FMAs, so a thread keeps up to 16 gathers in
// flight; each row is still summed left to right.
// FMAs k < M of one gathered batch, lane-predicated on k < m.  M is the largest batch length
// among the warp's converged lanes: on GB300 a warp instruction that is predicated off in
// every lane still takes a slot of the narrow FP64 pipe, so the count issued must not be a
// fixed 8 (a 7-point stencil row would pay for 8).
template <int M>
__device__ __forceinline__ void fma_batch(const double (&v)[8], const double (&xv)[8], int m,
                                          double& s) {
#pragma unroll
  for (int k = 0; k < M; ++k)
    if (k < m) s = fma(v[k], xv[k], s);
}

__device__ __forceinline__ void fma_batch_n(int mx, const double (&v)[8], const double (&xv)[8],
                                            int m, double& s) {
  switch (mx) {
    case 1: fma_batch<1>(v, xv, m, s); break;
    case 2: fma_batch<2>(v, xv, m, s); break;
    case 3: fma_batch<3>(v, xv, m, s); break;
    case 4: fma_batch<4>(v, xv, m, s); break;
    case 5: fma_batch<5>(v, xv, m, s); break;
    case 6: fma_batch<6>(v, xv, m, s); break;
    case 7: fma_batch<7>(v, xv, m, s); break;
    case 8: fma_batch<8>(v, xv, m, s); break;
    default: break;
  }
}

template <class XP>
__device__ __forceinline__ void smem_row2(const double* sva, const int32_t* sci, int ja, int ja1,
                                          int jb, int jb1, XP x, double& sa, double& sb) {
  sa = 0.0;
  sb = 0.0;
  for (;;) {
    const int ma = min(8, ja1 - ja), mb = min(8, jb1 - jb);
    if (ma <= 0 && mb <= 0) break;
    int ca[8], cb[8];
    double va[8], vb[8], xa[8], xb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      ca[k] = k < ma ? sci[ja + k] : 0;
      va[k] = k < ma ? sva[ja + k] : 0.0;
      cb[k] = k < mb ? sci[jb + k] : 0;
      vb[k] = k < mb ? sva[jb + k] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      xa[k] = k < ma ? gather(x, ca[k]) : 0.0;
      xb[k] = k < mb ? gather(x, cb[k]) : 0.0;
    }
    // the same FMAs in the same order as a fixed 8-wide loop, without the dead issue slots
    const unsigned conv = __activemask();
    fma_batch_n(__reduce_max_sync(conv, max(ma, 0)), va, xa, ma, sa);
    fma_batch_n(__reduce_max_sync(conv, max(mb, 0)), vb, xb, mb, sb);
    ja += ma > 0 ? ma : 0;
    jb += mb > 0 ? mb : 0;
  }
}

// Row product from a shared-memory window, chunked like csr_row (same summation order).
__device__ __forceinline__ double smem_row(const double* sva, const int32_t* sci, int j, int j1,
                                           const double* __restrict__ x) {
  double s = 0.0;
  for (; j + 4 <= j1; j += 4) {
    int c[4];
    double v[4], xv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { c[k] = sci[j + k]; v[k] = sva[j + k]; }
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] = __ldg(x + c[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fma(v[k], xv[k], s);
  }
  if (j < j1) {
    const int m = j1 - j;
    int c[3];
    double v[3], xv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      c[k] = k < m ? sci[j + k] : 0;
      v[k] = k < m ? sva[j + k] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) xv[k] = k < m ? __ldg(x + c[k]) : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < m) s = fma(v[k], xv[k], s);
  }
  return s;
}

// Launch with the programmatic-stream-serialization attribute: the kernel may start while
// the preceding kernel of the stream finishes; it orders itself with griddep_wait().
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// FP32 row product from a shared-memory window: the row's products summed left to right
// (the order of a plain CSR row loop), gathers of a batch of 8 issued before the FMAs.
template <class XP>
__device__ __forceinline__ float smem_row_f32(const float* sva, const int32_t* sci, int j, int j1, XP x) {
  float s = 0.0f;
  for (; j < j1; j += 8) {
    const int m = min(8, j1 - j);
    int c[8];
    float v[8], xv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c[k] = k < m ? sci[j + k] : 0;
      v[k] = k < m ? sva[j + k] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] = k < m ? gather(x, c[k]) : 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < m) s = fmaf(v[k], xv[k], s);
  }
  return s;
}

template <class XP>
__device__ __forceinline__ void row_pair(const double* sva, const int32_t* sci, int ja, int ja1, int jb,
                                         int jb1, XP x, double& sa, double& sb) {
  smem_row2(sva, sci, ja, ja1, jb, jb1, x, sa, sb);
}

template <class XP>
__device__ __forceinline__ void row_pair(const float* sva, const int32_t* sci, int ja, int ja1, int jb,
                                         int jb1, XP x, float& sa, float& sb) {
  sa = smem_row_f32(sva, sci, ja, ja1, x);
  sb = jb1 > jb ? smem_row_f32(sva, sci, jb, jb1, x) : 0.0f;
}

inline CsrTilesT<float> csr_tiles32_of(const pk_csr* A) {
  CsrTilesT<float> t;
  t.rp = A->rp;
  t.ci = A->ci;
  t.va = A->va32;
  t.tile_row = A->tile_row;
  t.blk_tile = A->blk_tile;
  t.tile_grp = A->tile_grp;
  t.tile_perm = A->tile_perm;
  t.tile_z0 = A->tile_z0;
  return t;
}

inline CsrTiles csr_tiles_of(const pk_csr* A) {
  CsrTiles t;
  t.rp = A->rp;
  t.ci = A->ci;
  t.va = A->va;
  t.tile_row = A->tile_row;
  t.blk_tile = A->blk_tile;
  t.tile_grp = A->tile_grp;
  t.tile_perm = A->tile_perm;
  t.tile_z0 = A->tile_z0;
  return t;
}

}  // namespace pk
