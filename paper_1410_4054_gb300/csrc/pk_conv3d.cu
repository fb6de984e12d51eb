// BF16 implicit-GEMM 3D convolutions (FP32 accumulation) for the learned initial guess, plus
// the small kernels of its training step (input packing, loss gradient, Adam, prediction).
//
// Layout: activations channels-last BF16 [D][H][W][16] (channel counts padded to 16, padded
// channels are zero); weights BF16 [tap][co][ci] = [27][16][16], tap = 9(dz+1)+3(dy+1)+(dx+1);
// zero padding of 1 at the grid boundary.
//
// Forward / backward-data (conv3d_fwd): the tcgen05 tensor-core kernel below (TMA-staged
// input blocks, one M128 N16 K16 MMA per tap, FP32 accumulators in tensor memory).  The
// backward-data pass is the same kernel on flipped, transposed weights with the ReLU mask of
// the layer input applied in the epilogue.
// Weight gradient (conv3d_wgrad): tcgen05 as well, the taps stacked into M (8 taps x 16 input
// channels per M128 tile), N = 16 output channels, K = voxels; the K-major operands are
// written per 64-voxel segment with ldmatrix.trans / stmatrix (see k_conv3d_wgrad_tc), then a
// fixed-order reduction over blocks (deterministic).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "pk_tile.cuh"

namespace pk {

constexpr int kCh = 16;         // channels (padded)


struct ConvArgs {
  const __nv_bfloat16* X;     // input activations [D][H][W][16]
  const __nv_bfloat16* Wt;    // weights [27][16 co][16 ci]
  const float* bias;          // [16] or null
  __nv_bfloat16* Y;           // output BF16 [D][H][W][16] (unless out_f32)
  float* Yf;                  // output FP32 channel 0 [D][H][W] (out_f32)
  const __nv_bfloat16* mask;  // ReLU mask source [D][H][W][16] or null
  int D, H, W;
  int relu;
  int out_f32;
};

// ---------------------------------------------------------------- tcgen05 forward kernel
// Implicit GEMM on the 5th-generation tensor cores: an M = 128 tile of output voxels (8 along
// x by 16 along y at one z) times N = 16 output channels, K = 27 taps x 16 input channels,
// one tcgen05.mma (M128 N16 K16, BF16 operands, FP32 accumulator in tensor memory) per tap.
// The input block around a tile -- 3 planes x 18 rows x 10 voxels, each voxel's 16 channels
// as two 8-channel halves -- arrives by TMA: six cp.async.bulk.tensor copies of an
// [18][10][8] box per tile, the halo outside the grid filled with zeros by the copy engine.
// Each box lands in the no-swizzle K-major layout of the MMA's A operand: a core matrix is 8
// voxels consecutive in x (8 x 16 bytes), the two K halves are kTcHalf bytes apart (leading
// byte offset) and consecutive y rows kTcRow bytes apart (stride byte offset); a tap
// (dz, dy, dx) is the same descriptor with its start moved by (dz, dy, dx) voxels; the taps
// of each dz accumulate in their own tensor-memory accumulator (three independent MMA chains
// per tile, summed in the epilogue).  Weights
// [tap][half][co][8 ci] stay in shared memory for the whole launch.  A ring of kTcStages
// staging buffers and two accumulators pipeline a persistent block's tiles: thread 0 issues
// the copies and the MMAs of the next tile while all four warps run the epilogue of the
// current one (tcgen05.ld, bias, ReLU or mask, BF16 store).  Every mbarrier wait is bounded
// (2 s): a wait that runs out sets a device flag (pk_conv3d_check reports PK_TIMEOUT), the
// block waits (bounded) for what it issued, frees its tensor memory and returns.

constexpr int kTcX = 8, kTcY = 16;                  // tile: 8 x 16 voxels = M 128
constexpr int kTcBx = kTcX + 2, kTcBy = kTcY + 2;   // staged block with the halo
constexpr int kTcRow = kTcBx * 16;                  // bytes between staged y rows (SBO)
constexpr int kTcBox = kTcBy * kTcRow;              // bytes of one [18][10][8] box (2880)
constexpr int kTcHalf = (kTcBox + 127) & ~127;      // box pitch, 128-byte aligned (LBO)
constexpr int kTcPlane = 2 * kTcHalf;
constexpr int kTcStage = 3 * kTcPlane;              // 17,664 bytes
constexpr int kTcStages = 2;
constexpr int kTcW = 27 * 512;                      // weights, 13,824 bytes
constexpr int kTcSmem = kTcStages * kTcStage + kTcW;
constexpr int kTcChains = 3;                        // independent accumulators per tile (9 taps each)
constexpr uint32_t kTcCols = 128;                   // tensor memory: 2 tiles x 3 accumulators x 16 columns

__device__ int g_conv_timeout = 0;

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4
  // (32-45), fixed 0b001 (46-48), base offset 0, relative LBO, no swizzle (61-63 = 0)
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 =
// 1), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28)
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// One [18][10][8] box of the channels-last input at (c, x, y, z) (x, y, z may lie outside
// the grid: zero fill) into shared memory, completion on `bar`.
__device__ __forceinline__ void tc_tma_box(uint32_t dst, const CUtensorMap* map, int c, int x, int y,
                                           int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

__global__ void __launch_bounds__(128) k_conv3d_tc(const __grid_constant__ CUtensorMap xmap, ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* stg0 = smem_tc;                          // kTcStages staging buffers
  unsigned char* wsm = smem_tc + kTcStages * kTcStage;    // weights
  __shared__ __align__(8) uint64_t full_bar[kTcStages];   // staging buffer loaded
  __shared__ __align__(8) uint64_t mma_bar[2];            // accumulator complete
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tx = (a.W + kTcX - 1) / kTcX, ty = (a.H + kTcY - 1) / kTcY;
  const int ntiles = tx * ty * a.D;
  const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // my tiles
  for (int e = threadIdx.x; e < 27 * kCh * 2; e += blockDim.x) {
    const int half = e & 1, row = e >> 1, t = row / kCh, co = row % kCh;
    *reinterpret_cast<uint4*>(wsm + t * 512 + half * 256 + co * 16) =
        __ldg(reinterpret_cast<const uint4*>(a.Wt + row * kCh + 8 * half));
  }
  proxy_fence();  // the weights are read by the tensor core (async proxy)
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) mbar_init(&full_bar[s], 1);
    mbar_init(&mma_bar[0], 1);
    mbar_init(&mma_bar[1], 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t w_addr = smem_addr(wsm), s_base = smem_addr(stg0);
  auto tile_of = [&](int k, int& z, int& y0, int& x0) {  // the block's k-th tile
    const int t = blockIdx.x + k * gridDim.x;
    x0 = (t % tx) * kTcX;
    y0 = ((t / tx) % ty) * kTcY;
    z = t / (tx * ty);
  };
  auto load = [&](int k) {  // thread 0: the six boxes of tile k into stage k % kTcStages
    int z, y0, x0;
    tile_of(k, z, y0, x0);
    const int s = k % kTcStages;
    mbar_expect_tx(&full_bar[s], 6 * kTcBox);
    for (int pl = 0; pl < 3; ++pl)
      for (int h = 0; h < 2; ++h)
        tc_tma_box(s_base + s * kTcStage + pl * kTcPlane + h * kTcHalf, &xmap, 8 * h, x0 - 1, y0 - 1,
                   z + pl - 1, &full_bar[s]);
  };
  bool ok = true;
  auto issue = [&](int k) {  // thread 0: wait for tile k's data, 27 MMAs into accumulator k & 1
    const int s = k % kTcStages;
    if (!mbar_wait(&full_bar[s], (k / kTcStages) & 1)) return false;
    tc_fence_after();
    const uint32_t sa0 = s_base + s * kTcStage;
    const uint32_t acc = tmem + (k & 1) * (kTcChains * 16);
    // three chains of nine taps (dz = -1, 0, +1), issued interleaved: consecutive MMAs write
    // different accumulators and overlap in the tensor pipe
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
      const int dy = i / 3, dx = i % 3;
#pragma unroll
      for (int c = 0; c < kTcChains; ++c) {
        const int tap = 9 * c + i;  // dz = c - 1
        tc_mma(acc + c * 16, tc_desc(sa0 + c * kTcPlane + dy * kTcRow + dx * 16, kTcHalf, kTcRow),
               tc_desc(w_addr + tap * 512, 256, 128), i > 0 ? 1u : 0u);
      }
    }
    tc_commit(&mma_bar[k & 1]);
    return true;
  };
  float bias[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) bias[c] = a.bias ? a.bias[c] : 0.f;
  if (threadIdx.x == 0 && mine > 0) {
    for (int k = 0; k < min(kTcStages, mine); ++k) load(k);
    ok = issue(0);
  }
  int issued_mma = threadIdx.x == 0 && mine > 0 && ok ? 1 : 0;
  for (int k = 0; k < mine; ++k) {
    // thread 0: the next tile's MMAs go out before this tile's epilogue (other accumulator)
    if (threadIdx.x == 0 && ok && k + 1 < mine) {
      ok = issue(k + 1);
      issued_mma += ok;
    }
    if (!ok) abort_flag = 1;
    if (!mbar_wait(&mma_bar[k & 1], (k >> 1) & 1)) abort_flag = 1;
    tc_fence_after();
    __syncthreads();
    if (abort_flag) break;
    // the stage of tile k is free: thread 0 refills it with tile k + kTcStages
    if (threadIdx.x == 0 && k + kTcStages < mine) load(k + kTcStages);
    int z, y0, x0;
    tile_of(k, z, y0, x0);
    float o[16];
    {
      // the three partial sums (taps with dz = -1, 0, +1), added in that order
      const uint32_t row = tmem + ((uint32_t)(32 * warp) << 16) + (k & 1) * (kTcChains * 16);
      float p1[16], p2[16];
      tc_ld16(row, o);
      tc_ld16(row + 16, p1);
      tc_ld16(row + 32, p2);
#pragma unroll
      for (int c = 0; c < 16; ++c) o[c] = (o[c] + p1[c]) + p2[c];
    }
    const int m = 32 * warp + lane;
    const int y = y0 + m / kTcX, x = x0 + m % kTcX;
    if (y < a.H && x < a.W) {
      const size_t v = ((size_t)z * a.H + y) * a.W + x;
      if (a.out_f32) {
        a.Yf[v] = o[0] + bias[0];
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          o[c] += bias[c];
          if (a.relu) o[c] = fmaxf(o[c], 0.f);
        }
        if (a.mask) {
          const uint4 m0 = *reinterpret_cast<const uint4*>(a.mask + v * kCh);
          const uint4 m1 = *reinterpret_cast<const uint4*>(a.mask + v * kCh + 8);
          const __nv_bfloat16* mb0 = reinterpret_cast<const __nv_bfloat16*>(&m0);
          const __nv_bfloat16* mb1 = reinterpret_cast<const __nv_bfloat16*>(&m1);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (!(__bfloat162float(mb0[c]) > 0.f)) o[c] = 0.f;
            if (!(__bfloat162float(mb1[c]) > 0.f)) o[8 + c] = 0.f;
          }
        }
        uint4 p0, p1;
        __nv_bfloat162* q0 = reinterpret_cast<__nv_bfloat162*>(&p0);
        __nv_bfloat162* q1 = reinterpret_cast<__nv_bfloat162*>(&p1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          q0[c] = __floats2bfloat162_rn(o[2 * c], o[2 * c + 1]);
          q1[c] = __floats2bfloat162_rn(o[8 + 2 * c], o[8 + 2 * c + 1]);
        }
        *reinterpret_cast<uint4*>(a.Y + v * kCh) = p0;
        *reinterpret_cast<uint4*>(a.Y + v * kCh + 8) = p1;
      }
    }
    tc_fence_before();
    __syncthreads();  // accumulator k & 1 is free again
  }
  if (abort_flag && threadIdx.x == 0) {
    atomicExch(&g_conv_timeout, 1);
    // bounded waits for what this block still has in flight before its tensor memory goes
    for (int s = 0; s < kTcStages; ++s) mbar_wait(&full_bar[s], 0);
    mbar_wait(&mma_bar[0], 0);
    mbar_wait(&mma_bar[1], 0);
  }
  (void)issued_mma;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

// ---------------------------------------------------------------- tcgen05 weight gradient
// dW[tap][co][ci] = sum_v G[v][co] A[v + s][ci] (s the tap's shift) as one implicit GEMM per
// 16 voxels on the tensor cores.  The shift is split between the operands: with
// s = s_a + s_b, sum_v G[v] A[v + s] = sum_k A[k + s_a] G[k - s_b], so a product of
//   M = 128 rows (s_a, ci): the 8 shifts s_a = (dz, dy, 0) other than (1, 1, 0), x 16 ci,
//   N = 96 rows (s_b, co): the 6 shifts s_b = (0, 0, dx) and (1, 1, dx), x 16 co,
// over K = voxels k holds every tap once: s_a + (0, 0, dx) for the 24 taps with (dz, dy) !=
// (1, 1), and (0, 0, 0) + (1, 1, dx) for the other 3 (the remaining (s_a, s_b) pairs are not
// taps and are not read).  One M128 N96 K16 MMA per 16 voxels covers all 27 taps.
// A block takes 64-voxel x segments of (z, y) rows in turn.  For a segment, bulk copies bring
// the 3 x 3 rows of A around it and the rows (z, y), (z-1, y-1) of G, 66 voxels each with the
// x halo (one contiguous run of 32-byte voxels per row; the parts outside the grid are not
// copied, and the operand writers read zeros for them), into one of five staging buffers,
// four segments ahead.  Eight warps write the K-major operands -- the
// shifted copies of A and of G, transposed -- with ldmatrix.trans / stmatrix: each 8 x 8
// block of [voxel][channel] becomes the [channel][voxel] core matrix of the no-swizzle
// K-major layout (8 rows of 16 bytes; K-adjacent core matrices kWgLboA / kWgLboB bytes apart,
// M- or N-adjacent 128).  A loader warp issues the copies (one lane per row), and one thread
// of another warp issues, per segment, 4 MMAs into one
// FP32 accumulator of 96 columns in tensor memory that persists over all of the block's
// segments; three operand buffers rotate, so the writers run up to two segments ahead of
// the tensor core's completions (mbarriers: operands written by the 8 warps, operands read by
// the MMAs).  Every wait is bounded (a wait that runs out sets the device
// flag that pk_conv3d_check reports, and the block waits, bounded, for what it issued before
// it frees its tensor memory).  At the end each thread reads its accumulator lane (one
// (s_a, ci) row) into the block's partial; a fixed-order reduction over blocks follows.
constexpr int kWgSeg = 64;                       // voxels (K) per segment
constexpr int kWgKg = kWgSeg / 8;                // K core matrices per segment
constexpr int kWgSa = 8, kWgSb = 6;              // shifts on the A side and on the G side
constexpr int kWgN = kWgSb * 16;                 // 96
constexpr int kWgLboA = kWgSa * 2 * 128;         // bytes between K-adjacent core matrices of A (2 KB)
constexpr int kWgLboB = kWgSb * 2 * 128;         // ... of G^T (1.5 KB)
constexpr int kWgA = kWgKg * kWgLboA;            // 16 KB: A operand of one segment
constexpr int kWgB = kWgKg * kWgLboB;            // 12 KB: G operand of one segment
constexpr int kWgHx = kWgSeg + 2;                // staged x extent (halo of one)
constexpr int kWgRow = kWgHx * 32;               // one staged row: 66 voxels x 16 channels BF16
constexpr int kWgStageA = 9 * kWgRow;            // A rows (z + dz, y + dy), (dz + 1) 3 + (dy + 1)
constexpr int kWgStage = (kWgStageA + 2 * kWgRow + 127) & ~127;  // + G rows (z-1, y-1), (z, y)
constexpr int kWgOp = kWgA + kWgB;               // one operand buffer (28 KB)
constexpr int kWgStages = 5;                     // staging buffers (copies four segments ahead)
constexpr int kWgOps = 3;                        // operand buffers (the writers run 2 segments ahead)
constexpr int kWgSmem = kWgOps * kWgOp + kWgStages * kWgStage;
constexpr int kWgMaxBlocks = 256;
constexpr uint32_t kWgCols = 128;                // tensor memory: one accumulator of 96 columns
constexpr int kWgThreads = 256;                  // 8 warps write the operands
// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N = 96, M = 128
constexpr uint32_t kWgIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kWgN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void wg_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kWgIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void stsm4(uint32_t addr, const uint32_t (&r)[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3])
               : "memory");
}

__global__ void __launch_bounds__(kWgThreads + 64) k_conv3d_wgrad_tc(const __nv_bfloat16* __restrict__ A,
                                                                   const __nv_bfloat16* __restrict__ G,
                                                                   float* partial, float* partial_db, int D,
                                                                   int H, int W) {
  extern __shared__ __align__(1024) unsigned char smem_wg[];
  unsigned char* obuf = smem_wg;                                // kWgOps operand buffers
  unsigned char* stage = smem_wg + kWgOps * kWgOp;              // kWgStages staging buffers
  __shared__ __align__(8) uint64_t full_bar[kWgStages];         // staging buffer loaded
  __shared__ __align__(8) uint64_t empty_bar[kWgStages];        // staging buffer read (8 warps)
  __shared__ __align__(8) uint64_t ready_bar[kWgOps];           // operands written (8 warps)
  __shared__ __align__(8) uint64_t free_bar[kWgOps];            // operands read (MMA commit)
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, consumed;
  __shared__ __align__(16) uint4 zero16;  // what the operand writers read outside the grid
  __shared__ float dbs[kWgThreads / kCh][kCh];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nseg = (W + kWgSeg - 1) / kWgSeg;
  const int nchunks = D * H * nseg;  // (< 2^31: checked by the host)
  const int mine = (int)blockIdx.x < nchunks ? (nchunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  proxy_fence();
  if (threadIdx.x == 0) {
    for (int k = 0; k < kWgStages; ++k) {
      mbar_init(&full_bar[k], 1);
      mbar_init(&empty_bar[k], kWgThreads / 32);
    }
    for (int k = 0; k < kWgOps; ++k) {
      mbar_init(&ready_bar[k], kWgThreads / 32);
      mbar_init(&free_bar[k], 1);
    }
    mbar_fence_init();
    abort_flag = 0;
    consumed = 0;
    zero16 = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kWgCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t o_base = smem_addr(obuf), s_base = smem_addr(stage);
  float db = 0.f;  // builders: output channel t % 16 over voxels (t / 16) + 16 k of every segment
  if (warp == kWgThreads / 32) {
    // MMA warp, lane 0: per segment, once its operands are written, 4 MMAs and a commit
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < mine; ++j) {
        const int b = j % kWgOps;
        if (!mbar_wait(&ready_bar[b], (j / kWgOps) & 1) || *(volatile int*)&abort_flag) {
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t ob = o_base + b * kWgOp;
#pragma unroll
        for (int ks = 0; ks < kWgKg / 2; ++ks)
          wg_mma(tmem, tc_desc(ob + 2 * ks * kWgLboA, kWgLboA, 128), tc_desc(ob + kWgA + 2 * ks * kWgLboB, kWgLboB, 128),
                 (j > 0 || ks > 0) ? 1u : 0u);
        tc_commit(&free_bar[b]);
        issued = j + 1;
      }
      // the last commit covers every MMA the block issued
      if (issued > 0 && !mbar_wait(&free_bar[(issued - 1) % kWgOps], ((issued - 1) / kWgOps) & 1)) abort_flag = 1;
    }
  } else if (warp == kWgThreads / 32 + 1) {
    // loader warp: the bulk copies of segment j into staging buffer j % kWgStages, once the
    // writers are done with segment j - kWgStages there (its empty barrier: one phase per use
    // of the buffer, so the wait cannot mistake a later phase for it); lane r < 11 copies row
    // r (9 rows of A, then G at (z-1, y-1), (z, y)): the in-grid part [xa, xb) of an in-grid
    // row, x0 - 1 at staged voxel 0
    int loaded = 0;
    for (int j = 0; j < mine; ++j) {
      if (j >= kWgStages) {
        const int jr = j - kWgStages;
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&empty_bar[j % kWgStages], (jr / kWgStages) & 1) && !*(volatile int*)&abort_flag;
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
      }
      const int c = (int)blockIdx.x + j * (int)gridDim.x;
      const int seg = c % nseg, zy = c / nseg;
      const int z = zy / H, y = zy % H, x0 = seg * kWgSeg;
      const int xa = max(0, x0 - 1), xb = min(W, x0 + kWgSeg + 1);
      const uint32_t bytes = (uint32_t)(xb - xa) * 32;
      const int sb = j % kWgStages;
      const int row = lane;
      const int zz = row < 9 ? z + row / 3 - 1 : z + row - 10, yy = row < 9 ? y + row % 3 - 1 : y + row - 10;
      const bool in = row < 11 && zz >= 0 && zz < D && yy >= 0 && yy < H;
      const uint32_t total = bytes * (uint32_t)__popc(__ballot_sync(0xffffffffu, in));
      if (lane == 0) mbar_expect_tx(&full_bar[sb], total);
      __syncwarp();
      if (in)
        bulk_load(stage + sb * kWgStage + (xa - x0 + 1) * 32 + row * kWgRow,
                  (row < 9 ? A : G) + (((size_t)zz * H + yy) * W + xa) * kCh, bytes, &full_bar[sb]);
      loaded = j + 1;
    }
    if (lane == 0 && *(volatile int*)&abort_flag) {
      // bounded waits for the copies the writers did not consume before the memory goes
      for (int k = *(volatile int*)&consumed; k < loaded; ++k)
        mbar_wait(&full_bar[k % kWgStages], (k / kWgStages) & 1);
    }
  } else {
    // builders: the operand-writing jobs of this thread, 7 blocks of 8 x 8, their source
    // offsets in a staging buffer and destinations in an operand buffer, the same for every
    // segment: 8 shifts s_a x 2 channel halves x 8 K groups of A (128 blocks), then 6 shifts
    // s_b x 2 x 8 of G (96); lanes 8i .. 8i+7 address the rows of block i of a four-block
    // instruction
    constexpr int kGroups = (kWgSa + kWgSb) * 2 * kWgKg / 4;  // 56 instructions per segment
    constexpr int kWarps = kWgThreads / 32;
    constexpr int kJobs = kGroups / kWarps;                     // 7 per warp
    static_assert(kGroups % kWarps == 0, "whole instructions per warp");
    // where each lane's row comes from: staged row 0 .. 10 and voxel x0 + xoff, read as zeros
    // outside the grid (coded as row << 8 | (xoff + 1))
    uint32_t src_off[kJobs], dst_off[kJobs], where[kJobs];
    {
      const int r = lane & 7, i = lane >> 3;
#pragma unroll
      for (int k = 0; k < kJobs; ++k) {
        const int grp = warp + kWarps * k;
        const int q = 4 * grp + i;
        if (q < kWgSa * 2 * kWgKg) {
          // A[k + s_a][ci], s_a = combo sa of (dz, dy) without (1, 1): staged row sa
          const int sa = q >> 4, h = (q >> 3) & 1, kg = q & 7;
          src_off[k] = (sa * kWgHx + kg * 8 + r + 1) * 32 + h * 16;
          dst_off[k] = kg * kWgLboA + (sa * 2 + h) * 128 + r * 16;
          where[k] = ((uint32_t)sa << 8) | (uint32_t)(kg * 8 + r + 1);
        } else {
          // G[k - s_b][co]: s_b = (0, 0, dx) reads G row (z, y), (1, 1, dx) row (z-1, y-1)
          const int qb = q - kWgSa * 2 * kWgKg, sb = qb >> 4, h = (qb >> 3) & 1, kg = qb & 7;
          const int dx = sb % 3 - 1, grow = sb < 3 ? 10 : 9;
          src_off[k] = (grow * kWgHx + kg * 8 + r - dx + 1) * 32 + h * 16;
          dst_off[k] = kWgA + kg * kWgLboB + (sb * 2 + h) * 128 + r * 16;
          where[k] = ((uint32_t)grow << 8) | (uint32_t)(kg * 8 + r - dx + 1);
        }
      }
    }
    const uint32_t zero_addr = smem_addr(&zero16);
    const int c = threadIdx.x & (kCh - 1);
    for (int j = 0; j < mine; ++j) {
      const int b = j % kWgOps, sb = j % kWgStages;
      // segment j's data, and operand buffer b free (read by the MMAs of segment j - kWgOps)
      if (lane == 0) {
        if (!mbar_wait(&full_bar[sb], (j / kWgStages) & 1) ||
            (j >= kWgOps && !mbar_wait(&free_bar[b], ((j - kWgOps) / kWgOps) & 1)))
          abort_flag = 1;
        else if (warp == 0)
          consumed = j + 1;
      }
      __syncwarp();
      if (*(volatile int*)&abort_flag) break;
      const uint32_t st = s_base + sb * kWgStage;
      const int cc = (int)blockIdx.x + j * (int)gridDim.x;
      const int zy = cc / nseg, z = zy / H, y = zy % H, x0 = (cc % nseg) * kWgSeg;
      uint32_t rows_in = 0;  // staged rows inside the grid (bit = row, as the loader numbers them)
#pragma unroll
      for (int row = 0; row < 11; ++row) {
        const int zz = row < 9 ? z + row / 3 - 1 : z + row - 10, yy = row < 9 ? y + row % 3 - 1 : y + row - 10;
        if (zz >= 0 && zz < D && yy >= 0 && yy < H) rows_in |= 1u << row;
      }
      {
        // G at (z, y), x0 + xx: staged row 10, voxel xx + 1 (inside the grid only)
        const __nv_bfloat16* g16 = reinterpret_cast<const __nv_bfloat16*>(stage + sb * kWgStage +
                                                                            (10 * kWgHx + 1) * 32);
#pragma unroll
        for (int xx = threadIdx.x / kCh; xx < kWgSeg; xx += kWgThreads / kCh)
          if (x0 + xx < W) db += __bfloat162float(g16[xx * kCh + c]);
      }
      const uint32_t ob = o_base + b * kWgOp;
      uint32_t f[kJobs][4];  // all loads in flight before the stores
#pragma unroll
      for (int k = 0; k < kJobs; ++k) {
        const bool in = ((rows_in >> (where[k] >> 8)) & 1u) && (unsigned)(x0 + (int)(where[k] & 255) - 1) < (unsigned)W;
        ldsm4t(f[k], in ? st + src_off[k] : zero_addr);
      }
#pragma unroll
      for (int k = 0; k < kJobs; ++k) stsm4(ob + dst_off[k], f[k]);
      proxy_fence();  // the operands are read by the tensor core (async proxy)
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ready_bar[b]);
        mbar_arrive(&empty_bar[sb]);
      }
    }
    dbs[threadIdx.x / kCh][c] = db;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  float* P = partial + (size_t)blockIdx.x * 27 * kCh * kCh;
  if (!abort_flag && warp < kWgThreads / 32) {
    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31, column blocks s_b = 3 (w / 4) ..
    // + 2; row m = (s_a, ci): s_a = m / 16 is (dz, dy) = combo s_a of the 3 x 3 without (1, 1)
    const int q4 = warp & 3, m = 32 * q4 + lane;
    const int sa = m >> 4, ci = m & 15, dzdy = sa;  // combos 0 .. 7 are (dz + 1) 3 + (dy + 1)
#pragma unroll 1
    for (int sb = 3 * (warp >> 2); sb < 3 * (warp >> 2) + 3; ++sb) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(32 * q4) << 16) + sb * 16, v);
      const int dx = sb % 3 - 1;
      int tap = -1;
      if (sb < 3) tap = 3 * dzdy + (dx + 1);             // (dz, dy, dx)
      else if (dzdy == 4) tap = 3 * 8 + (dx + 1);        // (0, 0, 0) + (1, 1, dx)
      if (tap >= 0) {
#pragma unroll
        for (int co = 0; co < 16; ++co) P[(tap * kCh + co) * kCh + ci] = mine > 0 ? v[co] : 0.f;
      }
    }
    if (threadIdx.x < kCh) {
      float t = 0.f;
      for (int g = 0; g < kWgThreads / kCh; ++g) t += dbs[g][threadIdx.x];
      partial_db[blockIdx.x * kCh + threadIdx.x] = t;
    }
  } else if (abort_flag && threadIdx.x == 0) {
    atomicExch(&g_conv_timeout, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgCols) : "memory");
  }
}

// dW = sum over blocks of the partials (deterministic): a block of 8 warps per 32 outputs;
// warp w adds blocks w, w + 8, ... in order (their loads in flight together), then the 8 sums
// are added in warp order.
__global__ void __launch_bounds__(256) k_conv3d_wgrad_reduce(const float* partial, const float* partial_db,
                                                             int nblk, float* dW, float* db) {
  __shared__ float part[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * 32 + lane;
  constexpr int nw = 27 * kCh * kCh;
  float s = 0.f;
  if (e < nw + kCh) {
    const float* src = e < nw ? partial + e : partial_db + (e - nw);
    const size_t stride = e < nw ? (size_t)nw : (size_t)kCh;
    constexpr int kPer = (kWgMaxBlocks + 7) / 8;  // every load of the thread in flight at once
    float v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) v[q] = warp + 8 * q < nblk ? src[(size_t)(warp + 8 * q) * stride] : 0.f;
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (warp + 8 * q < nblk) s += v[q];
  }
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && e < nw + kCh) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w][lane];
    if (e < nw) dW[e] = t;
    else db[e - nw] = t;
  }
}

// Wf[26 - t][ci][co] = W[t][co][ci]: the weights of the backward-data convolution.
__global__ void k_conv3d_flip(const __nv_bfloat16* W, __nv_bfloat16* Wf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 27 * kCh * kCh) return;
  const int t = e / (kCh * kCh), co = (e / kCh) % kCh, ci = e % kCh;
  Wf[((26 - t) * kCh + ci) * kCh + co] = W[e];
}

// ------------------------------------------------------------------ training-step helpers

// Deterministic two-stage sums of up to 3 FP64 values over n (scratch: 3 x gridDim doubles,
// then the arrival counter as an unsigned at scratch[3 * gridDim]).
template <int NV, class F>
__device__ __forceinline__ void grid_sums(int n, double* scratch, F&& f, double (&out)[NV], bool& last) {
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) f(i, v);
  block_partials<NV>(v, scratch);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + 3 * gridDim.x);
  last = arrive_last(counter);
  if (last) {
    final_sums<NV>(scratch, out);
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0;
  }
}

constexpr int kWsGrid = 152;

// Residual of the linear extrapolation e = 2 x_{t-1} - x_{t-2} in row i:
// r = b_i - sum_j a_ij e_j; d = a_ii (1 where the row has no nonzero diagonal entry).
__device__ __forceinline__ void ws_row(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const double* __restrict__ va, const double* xm1,
                                       const double* xm2, const double* b, int i, double& r,
                                       double& d) {
  double s = 0.0;
  d = 0.0;
  for (int j = rp[i]; j < rp[i + 1]; ++j) {
    const int c = ci[j];
    const double e = 2.0 * xm1[c] - xm2[c];
    s = fma(va[j], e, s);
    if (c == i) d = va[j];
  }
  r = b[i] - s;
  if (d == 0.0) d = 1.0;
}

// scales = rms of (r / d, r, d) (1 where zero).
__global__ void __launch_bounds__(kBlock) k_ws_rms(int n, const int32_t* rp, const int32_t* ci,
                                                   const double* va, const double* xm1,
                                                   const double* xm2, const double* b,
                                                   double* scales, double* scratch) {
  double out[3];
  bool last;
  grid_sums<3>(n, scratch, [&](int i, double (&v)[3]) {
    double r, d;
    ws_row(rp, ci, va, xm1, xm2, b, i, r, d);
    const double z = r / d;
    v[0] = fma(z, z, v[0]);
    v[1] = fma(r, r, v[1]);
    v[2] = fma(d, d, v[2]);
  }, out, last);
  if (last && threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      const double s = sqrt(out[k] / n);
      scales[k] = s > 0 ? s : 1.0;
    }
  }
}

// X16[v] = bf16((r/d)/s0, r/s1, d/s2, 0, ..., 0): the Jacobi-scaled residual of the
// extrapolation, the residual itself and the diagonal, each channel of order one.
__global__ void k_ws_pack(int n, const int32_t* rp, const int32_t* ci, const double* va,
                          const double* xm1, const double* xm2, const double* b,
                          const double* scales, __nv_bfloat16* X16) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double r, d;
  ws_row(rp, ci, va, xm1, xm2, b, v, r, d);
  __nv_bfloat16* o = X16 + (size_t)v * kCh;
  o[0] = __float2bfloat16_rn((float)(r / d / scales[0]));
  o[1] = __float2bfloat16_rn((float)(r / scales[1]));
  o[2] = __float2bfloat16_rn((float)(d / scales[2]));
  for (int c = 3; c < kCh; ++c) o[c] = __float2bfloat16_rn(0.f);
}

// target y = (x_t - 2 x_{t-1} + x_{t-2}) / s0 (what linear extrapolation misses, in units of
// the Jacobi-scaled residual); G[v][0] = bf16(2 (out - y) / n); loss = mean((out - y)^2).
__global__ void __launch_bounds__(kBlock) k_ws_loss(int n, const float* out, const double* xt,
                                                    const double* xm1, const double* xm2,
                                                    const double* scales, __nv_bfloat16* G,
                                                    double* loss, double* scratch) {
  const double is = 1.0 / scales[0];
  double sum[1];
  bool last;
  grid_sums<1>(n, scratch, [&](int i, double (&v)[1]) {
    const double d = (double)out[i] - (xt[i] - 2.0 * xm1[i] + xm2[i]) * is;
    v[0] = fma(d, d, v[0]);
    __nv_bfloat16* gi = G + (size_t)i * kCh;
    gi[0] = __float2bfloat16_rn((float)(2.0 * d / n));
    for (int c = 1; c < kCh; ++c) gi[c] = __float2bfloat16_rn(0.f);
  }, sum, last);
  if (last && threadIdx.x == 0) *loss = sum[0] / n;
}

// x_hat = 2 x_{t-1} - x_{t-2} + s0 out (out == nullptr: the extrapolation alone).
__global__ void k_ws_apply(int n, const float* out, const double* xm1, const double* xm2,
                           const double* scales, double* xhat) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double e = 2.0 * xm1[v] - xm2[v];
  xhat[v] = out ? fma(scales[0], (double)out[v], e) : e;
}

// The energy step along the network's correction: d = s0 out, r = b - A e,
// gamma = <r, d> / <d, A d> -- the step from e along d that minimises the A-norm of the error
// (<x_t - e - gamma d, A (x_t - e - gamma d)> is a parabola in gamma with its minimum there,
// because A (x_t - e) = r).  Row i adds r_i d_i and d_i (A d)_i; d is formed at every gathered
// column from out.  gamma = 0 when <d, A d> <= 0 or is not finite (the extrapolation alone).
__global__ void __launch_bounds__(kBlock) k_ws_energy(int n, const int32_t* rp, const int32_t* ci,
                                                      const double* va, const float* out,
                                                      const double* xm1, const double* xm2,
                                                      const double* b, const double* scales,
                                                      double* gamma, double* scratch) {
  const double s0 = scales[0];
  double sums[2];
  bool last;
  grid_sums<2>(n, scratch, [&](int i, double (&v)[2]) {
    double se = 0.0, sd = 0.0;
    for (int j = rp[i]; j < rp[i + 1]; ++j) {
      const int c = ci[j];
      se = fma(va[j], 2.0 * xm1[c] - xm2[c], se);
      sd = fma(va[j], s0 * (double)out[c], sd);
    }
    const double r = b[i] - se, d = s0 * (double)out[i];
    v[0] = fma(r, d, v[0]);
    v[1] = fma(d, sd, v[1]);
  }, sums, last);
  if (last && threadIdx.x == 0) {
    const double g = sums[0] / sums[1];
    gamma[0] = sums[1] > 0.0 && isfinite(g) ? g : 0.0;
  }
}

// x_hat = 2 x_{t-1} - x_{t-2} + gamma s0 out.
__global__ void k_ws_apply_gamma(int n, const float* out, const double* xm1, const double* xm2,
                                 const double* scales, const double* gamma, double* xhat) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double e = 2.0 * xm1[v] - xm2[v];
  xhat[v] = fma(gamma[0], scales[0] * (double)out[v], e);
}

// One damped Jacobi sweep from a starting guess: xout_i = x_i + omega (b_i - sum_j a_ij x_j) / d_i,
// d_i = a_ii (1 where the row has no nonzero diagonal entry); the row's products are summed
// left to right.  Applied to the learned guess it damps the rough part of the guess's error,
// the part CG removes slowest on this operator.
__global__ void k_ws_relax(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ va, const double* __restrict__ b,
                           const double* __restrict__ x, double omega, double* __restrict__ xout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0, d = 0.0;
  for (int j = rp[i]; j < rp[i + 1]; ++j) {
    const int c = ci[j];
    s = fma(va[j], x[c], s);
    if (c == i) d = va[j];
  }
  if (d == 0.0) d = 1.0;
  xout[i] = fma(omega, (b[i] - s) / d, x[i]);
}

// Loss of the learned guess after damped Jacobi sweeps (training through the sweeps).  The
// guess's error in units of s0 is delta = out - (x_t - 2 x_{t-1} + x_{t-2}) / s0; a sweep maps
// an error e to P e = e - omega D^-1 A e; the loss is mean((P^s delta)^2) and its gradient
// (2/n) (P^T)^s P^s delta, P^T g = g - omega A (D^-1 g) for a symmetric A.
// d_i = a_ii (1 where the row has no nonzero diagonal entry).
__global__ void k_ws_diag(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ va, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double di = 1.0;
  for (int j = rp[i]; j < rp[i + 1]; ++j)
    if (ci[j] == i && va[j] != 0.0) di = va[j];
  d[i] = di;
}

__global__ void k_ws_delta(int n, const float* __restrict__ out, const double* __restrict__ xt,
                           const double* __restrict__ xm1, const double* __restrict__ xm2,
                           const double* __restrict__ scales, double* __restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  e[i] = (double)out[i] - (xt[i] - 2.0 * xm1[i] + xm2[i]) / scales[0];
}

// eout = e - omega D^-1 A e (one sweep's error propagator)
__global__ void k_ws_prop(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ va, const double* __restrict__ d, double omega,
                          const double* __restrict__ e, double* __restrict__ eout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = rp[i]; j < rp[i + 1]; ++j) s = fma(va[j], e[ci[j]], s);
  eout[i] = fma(omega, (0.0 - s) / d[i], e[i]);
}

// gout = g - omega A (D^-1 g) (its transpose, A symmetric)
__global__ void k_ws_prop_t(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ va, const double* __restrict__ d, double omega,
                            const double* __restrict__ g, double* __restrict__ gout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = rp[i]; j < rp[i + 1]; ++j) {
    const int c = ci[j];
    s = fma(va[j], g[c] / d[c], s);
  }
  gout[i] = fma(-omega, s, g[i]);
}

// *loss = mean(e^2)
__global__ void __launch_bounds__(kBlock) k_ws_sq_mean(int n, const double* e, double* loss, double* scratch) {
  double sum[1];
  bool last;
  grid_sums<1>(n, scratch, [&](int i, double (&v)[1]) { v[0] = fma(e[i], e[i], v[0]); }, sum, last);
  if (last && threadIdx.x == 0) *loss = sum[0] / n;
}

// G[v][0] = bf16(2 g_v / n), other channels 0
__global__ void k_ws_grad_pack(int n, const double* __restrict__ g, __nv_bfloat16* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  __nv_bfloat16* gi = G + (size_t)i * kCh;
  gi[0] = __float2bfloat16_rn((float)(2.0 * g[i] / n));
  for (int c = 1; c < kCh; ++c) gi[c] = __float2bfloat16_rn(0.f);
}

// Adam on FP32 master parameters, optional BF16 copy.
__global__ void k_adam(int count, float* p, const float* grad, float* m, float* v, float lr,
                       float b1, float b2, float eps, float c1, float c2, __nv_bfloat16* p16) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gr = grad[e];
  const float mm = b1 * m[e] + (1.f - b1) * gr;
  const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
  m[e] = mm;
  v[e] = vv;
  const float mh = mm / c1, vh = vv / c2;
  const float np = p[e] - lr * mh / (sqrtf(vh) + eps);
  p[e] = np;
  if (p16) p16[e] = __float2bfloat16_rn(np);
}

// Tensor map of a channels-last BF16 activation [D][H][W][16] for the TMA boxes of
// k_conv3d_tc: dimensions (channel, x, y, z), box (8, 10, 18, 1), zero fill outside.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

static pk_status input_map(CUtensorMap* map, const __nv_bfloat16* X, int D, int H, int W, int bx = kTcBx,
                           int by = kTcBy, int bz = 1) {
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      set_error("cuTensorMapEncodeTiled is not available");
      return PK_ERR_CUDA;
    }
    encode = reinterpret_cast<EncodeTiled>(fn);
  }
  if (reinterpret_cast<uintptr_t>(X) & 15) {
    set_error("pk_conv3d: activations and gradients must be 16-byte aligned");
    return PK_ERR_ARG;
  }
  const cuuint64_t dims[4] = {(cuuint64_t)kCh, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
  const cuuint64_t strides[3] = {(cuuint64_t)kCh * 2, (cuuint64_t)W * kCh * 2, (cuuint64_t)H * W * kCh * 2};
  const cuuint32_t box[4] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(X), dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("pk_conv3d_fwd: cuTensorMapEncodeTiled failed");
    return PK_ERR_CUDA;
  }
  return PK_OK;
}

static pk_status conv_setup() {
  static bool done = false;
  if (!done) {
    PK_CUDA(cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    // several blocks per SM (each with its own chain of accumulating MMAs): the largest
    // shared-memory carveout
    PK_CUDA(cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    PK_CUDA(cudaFuncSetAttribute(k_conv3d_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem));
    done = true;
  }
  return PK_OK;
}

}  // namespace pk

using namespace pk;

extern "C" {

pk_status pk_conv3d_fwd(const void* X, const void* Wt, const float* bias, void* Y, int32_t D,
                        int32_t H, int32_t W, int32_t relu, int32_t out_f32, const void* mask,
                        void* stream) {
  if (!X || !Wt || !Y || D <= 0 || H <= 0 || W <= 0 ||
      (int64_t)D * ((H + kTcY - 1) / kTcY) * ((W + kTcX - 1) / kTcX) >= (int64_t(1) << 31)) {
    set_error("pk_conv3d_fwd: bad arguments");
    return PK_ERR_ARG;
  }
  pk_status e = conv_setup();
  if (e) return e;
  ConvArgs a;
  a.X = static_cast<const __nv_bfloat16*>(X);
  a.Wt = static_cast<const __nv_bfloat16*>(Wt);
  a.bias = bias;
  a.Y = out_f32 ? nullptr : static_cast<__nv_bfloat16*>(Y);
  a.Yf = out_f32 ? static_cast<float*>(Y) : nullptr;
  a.mask = static_cast<const __nv_bfloat16*>(mask);
  a.D = D;
  a.H = H;
  a.W = W;
  a.relu = relu;
  a.out_f32 = out_f32;
  static int grid_max = 0;
  if (!grid_max) {
    // resident blocks per SM from the kernel's own footprint (shared memory incl. the
    // per-block reservation, registers, threads)
    int dev = 0, sms = 1, smem_sm = 0, resv = 0, regs_sm = 0;
    PK_CUDA(cudaGetDevice(&dev));
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PK_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    PK_CUDA(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    PK_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    PK_CUDA(cudaFuncGetAttributes(&fa, k_conv3d_tc));
    const int per_block = kTcSmem + (int)fa.sharedSizeBytes + resv;
    const int by_smem = smem_sm / per_block;
    const int by_regs = regs_sm / (128 * ((fa.numRegs + 7) & ~7));
    grid_max = sms * std::max(1, std::min(std::min(by_smem, by_regs), 16));
  }
  CUtensorMap map;
  if ((e = input_map(&map, a.X, D, H, W))) return e;
  const int64_t ntiles = (int64_t)D * ((H + kTcY - 1) / kTcY) * ((W + kTcX - 1) / kTcX);
  const int grid = (int)std::min<int64_t>(ntiles, grid_max);
  k_conv3d_tc<<<grid, 128, kTcSmem, (cudaStream_t)stream>>>(map, a);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_conv3d_check(void* stream) {
  int flag = 0, zero = 0;
  cudaStream_t s = (cudaStream_t)stream;
  PK_CUDA(cudaMemcpyFromSymbolAsync(&flag, g_conv_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  PK_CUDA(cudaMemcpyToSymbolAsync(g_conv_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  PK_CUDA(cudaStreamSynchronize(s));
  if (flag) {
    set_error("a tensor-core convolution timed out waiting for its MMAs");
    return PK_TIMEOUT;
  }
  return PK_OK;
}

// Blocks of the weight-gradient launch: one per SM (its shared memory allows one), at most
// one per segment and at most kWgMaxBlocks (the scratch size).
static int wgrad_blocks(int32_t D, int32_t H, int32_t W, int sms) {
  const int64_t chunks = (int64_t)D * H * ((W + kWgSeg - 1) / kWgSeg);
  return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, std::min(sms, kWgMaxBlocks)));
}

int64_t pk_conv3d_wgrad_scratch_floats(int32_t D, int32_t H, int32_t W) {
  return (int64_t)wgrad_blocks(D, H, W, kWgMaxBlocks) * (27 * kCh * kCh + kCh);
}

pk_status pk_conv3d_wgrad(const void* A, const void* G, float* scratch, float* dW, float* db,
                          int32_t D, int32_t H, int32_t W, void* stream) {
  if (!A || !G || !scratch || !dW || !db || D <= 0 || H <= 0 || W <= 0 ||
      (int64_t)D * H * ((W + kWgSeg - 1) / kWgSeg) >= (int64_t(1) << 31)) {
    set_error("pk_conv3d_wgrad: bad arguments");
    return PK_ERR_ARG;
  }
  pk_status e = conv_setup();
  if (e) return e;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    PK_CUDA(cudaGetDevice(&dev));
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int nblk = wgrad_blocks(D, H, W, sms);
  // partials laid out for the scratch size's block count (the launch may use fewer blocks)
  const int nmax = wgrad_blocks(D, H, W, kWgMaxBlocks);
  float* partial = scratch;
  float* partial_db = scratch + (size_t)nmax * 27 * kCh * kCh;
  cudaStream_t s = (cudaStream_t)stream;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(G)) & 15) {
    set_error("pk_conv3d_wgrad: activations and gradients must be 16-byte aligned");
    return PK_ERR_ARG;
  }
  k_conv3d_wgrad_tc<<<nblk, kWgThreads + 64, kWgSmem, s>>>(static_cast<const __nv_bfloat16*>(A),
                                                         static_cast<const __nv_bfloat16*>(G), partial,
                                                         partial_db, D, H, W);
  k_conv3d_wgrad_reduce<<<(27 * kCh * kCh + kCh + 31) / 32, 256, 0, s>>>(partial, partial_db, nblk, dW, db);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_conv3d_flip(const void* W, void* Wf, void* stream) {
  if (!W || !Wf) { set_error("pk_conv3d_flip: NULL"); return PK_ERR_ARG; }
  k_conv3d_flip<<<(27 * kCh * kCh + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(W), static_cast<__nv_bfloat16*>(Wf));
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

int64_t pk_warmstart_scratch_doubles(void) { return 3 * kWsGrid + 8; }

pk_status pk_warmstart_input(pk_csr* A, const double* xm1, const double* xm2, const double* b,
                             void* X16, double* scales, double* scratch, void* stream) {
  if (!A || !xm1 || !xm2 || !b || !X16 || !scales || !scratch) {
    set_error("pk_warmstart_input: bad arguments");
    return PK_ERR_ARG;
  }
  const int n = A->n;
  cudaStream_t s = (cudaStream_t)stream;
  PK_CUDA(cudaMemsetAsync(scratch + 3 * kWsGrid, 0, sizeof(double), s));
  k_ws_rms<<<kWsGrid, kBlock, 0, s>>>(n, A->rp, A->ci, A->va, xm1, xm2, b, scales, scratch);
  k_ws_pack<<<(n + 255) / 256, 256, 0, s>>>(n, A->rp, A->ci, A->va, xm1, xm2, b, scales,
                                             static_cast<__nv_bfloat16*>(X16));
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_warmstart_loss(int64_t n, const float* out, const double* xt, const double* xm1,
                            const double* xm2, const double* scales, void* G, double* loss,
                            double* scratch, void* stream) {
  if (n <= 0 || n >= (int64_t(1) << 31) || !out || !xt || !xm1 || !xm2 || !scales || !G || !loss ||
      !scratch) {
    set_error("pk_warmstart_loss: bad arguments");
    return PK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  PK_CUDA(cudaMemsetAsync(scratch + 3 * kWsGrid, 0, sizeof(double), s));
  k_ws_loss<<<kWsGrid, kBlock, 0, s>>>((int)n, out, xt, xm1, xm2, scales,
                                       static_cast<__nv_bfloat16*>(G), loss, scratch);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_warmstart_apply(int64_t n, const float* out, const double* xm1, const double* xm2,
                             const double* scales, double* xhat, void* stream) {
  if (n <= 0 || n >= (int64_t(1) << 31) || !xm1 || !xm2 || !scales || !xhat) {
    set_error("pk_warmstart_apply: bad arguments");
    return PK_ERR_ARG;
  }
  k_ws_apply<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((int)n, out, xm1, xm2,
                                                                       scales, xhat);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_warmstart_apply_energy(pk_csr* A, const float* out, const double* xm1, const double* xm2,
                                    const double* b, const double* scales, double* xhat, double* gamma,
                                    double* scratch, void* stream) {
  if (!A || !out || !xm1 || !xm2 || !b || !scales || !xhat || !gamma || !scratch) {
    set_error("pk_warmstart_apply_energy: bad arguments");
    return PK_ERR_ARG;
  }
  const int n = A->n;
  if (n == 0) return PK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  PK_CUDA(cudaMemsetAsync(scratch + 3 * kWsGrid, 0, sizeof(double), s));
  k_ws_energy<<<kWsGrid, kBlock, 0, s>>>(n, A->rp, A->ci, A->va, out, xm1, xm2, b, scales, gamma, scratch);
  k_ws_apply_gamma<<<(n + 255) / 256, 256, 0, s>>>(n, out, xm1, xm2, scales, gamma, xhat);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_warmstart_relax(pk_csr* A, const double* b, const double* x, double omega, double* xout,
                             void* stream) {
  if (!A || !b || !x || !xout || !(omega > 0.0 && omega < 2.0)) {
    set_error("pk_warmstart_relax: bad arguments (omega must lie in (0, 2))");
    return PK_ERR_ARG;
  }
  if (x == xout) {
    set_error("pk_warmstart_relax: xout must not be x (rows read x at other rows' columns)");
    return PK_ERR_ARG;
  }
  const int n = A->n;
  if (n == 0) return PK_OK;
  k_ws_relax<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, A->rp, A->ci, A->va, b, x, omega, xout);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_warmstart_loss_swept(pk_csr* A, const float* out, const double* xt, const double* xm1,
                                  const double* xm2, const double* scales, double omega, int32_t sweeps,
                                  void* G, double* loss, double* work, double* scratch, void* stream) {
  if (!A || !out || !xt || !xm1 || !xm2 || !scales || !G || !loss || !work || !scratch ||
      !(omega > 0.0 && omega < 2.0) || sweeps < 0 || sweeps > PK_WS_MAX_SWEEPS || A->n == 0) {
    set_error("pk_warmstart_loss_swept: bad arguments (omega in (0, 2), sweeps in [0, 8], n > 0)");
    return PK_ERR_ARG;
  }
  const int n = A->n;
  const int nb = (n + 255) / 256;
  cudaStream_t s = (cudaStream_t)stream;
  double* d = work;
  double* buf[2] = {work + n, work + 2 * (size_t)n};
  k_ws_diag<<<nb, 256, 0, s>>>(n, A->rp, A->ci, A->va, d);
  k_ws_delta<<<nb, 256, 0, s>>>(n, out, xt, xm1, xm2, scales, buf[0]);
  int cur = 0;
  for (int k = 0; k < sweeps; ++k, cur ^= 1)
    k_ws_prop<<<nb, 256, 0, s>>>(n, A->rp, A->ci, A->va, d, omega, buf[cur], buf[cur ^ 1]);
  PK_CUDA(cudaMemsetAsync(scratch + 3 * kWsGrid, 0, sizeof(double), s));
  k_ws_sq_mean<<<kWsGrid, kBlock, 0, s>>>(n, buf[cur], loss, scratch);
  for (int k = 0; k < sweeps; ++k, cur ^= 1)
    k_ws_prop_t<<<nb, 256, 0, s>>>(n, A->rp, A->ci, A->va, d, omega, buf[cur], buf[cur ^ 1]);
  k_ws_grad_pack<<<nb, 256, 0, s>>>(n, buf[cur], static_cast<__nv_bfloat16*>(G));
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_adam_step(int64_t count, float* p, const float* grad, float* m, float* v, float lr,
                       float beta1, float beta2, float eps, int32_t step, void* p_bf16, void* stream) {
  if (count <= 0 || !p || !grad || !m || !v || step < 1) {
    set_error("pk_adam_step: bad arguments");
    return PK_ERR_ARG;
  }
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<(int)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (int)count, p, grad, m, v, lr, beta1, beta2, eps, c1, c2, static_cast<__nv_bfloat16*>(p_bf16));
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

}  // extern "C"
