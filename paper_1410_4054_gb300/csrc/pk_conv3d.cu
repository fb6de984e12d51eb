// BF16 implicit-GEMM 3D convolutions (FP32 accumulation) for the learned initial guess, plus
// the small kernels of its training step (input packing, loss gradient, Adam, prediction).
//
// Layout: activations channels-last BF16 [D][H][W][16] (channel counts padded to 16, padded
// channels are zero); weights BF16 [tap][co][ci] = [27][16][16], tap = 9(dz+1)+3(dy+1)+(dx+1);
// zero padding of 1 at the grid boundary.
//
// Forward / backward-data (conv3d_fwd): one block per (z, y) row and 64-voxel x segment, four
// warps of 16 voxels.  The block stages the 9 neighbouring rows (+-1 voxel halo in x) and all
// weights in shared memory; for every tap a warp multiplies its 16 x 16 activation tile by
// the tap's 16 x 16 weight tile with two m16n8k16 BF16 tensor-core MMAs (operands through
// ldmatrix), i.e. an implicit GEMM with M = voxels, N = 16 output channels, K = 27 x 16.
// The backward-data pass is the same kernel on flipped, transposed weights with the ReLU mask
// of the layer input applied in the epilogue.
// Weight gradient (conv3d_wgrad): dW[tap] = G^T A_shift(tap), M = 16 output channels,
// N = 16 input channels, K = voxels: each block accumulates a band of rows in registers
// (warp w owns taps w, w+4, ...), operands transposed on the fly with ldmatrix.trans, then a
// fixed-order reduction over blocks (deterministic).
#include <cuda_bf16.h>

#include <algorithm>

#include "pk_internal.cuh"

namespace pk {

constexpr int kCh = 16;         // channels (padded)
constexpr int kSeg = 64;        // voxels per x segment = 4 warps x 16
constexpr int kHx = kSeg + 2;   // with the +-1 halo
constexpr int kVs = 24;         // shared-memory stride of one voxel in BF16 (48 bytes)
constexpr int kWgradRows = 16;  // (z, y) rows per weight-gradient block

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(sa(p)));
}

__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(sa(p)));
}

// D = A B + D, A 16x16 BF16 (row), B 16x8 BF16 (col), D 16x8 FP32.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage the 9 rows (z+dz, y+dy), x in [x0-1, x0+64], into halo[9][66][kVs] (zeros outside).
__device__ __forceinline__ void load_halo(__nv_bfloat16* halo, const __nv_bfloat16* __restrict__ X,
                                          int D, int H, int W, int z, int y, int x0) {
  for (int e = threadIdx.x; e < 9 * kHx * 2; e += blockDim.x) {
    const int half = e & 1, xx = (e >> 1) % kHx, zy = (e >> 1) / kHx;
    const int zz = z + zy / 3 - 1, yy = y + zy % 3 - 1, x = x0 + xx - 1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (zz >= 0 && zz < D && yy >= 0 && yy < H && x >= 0 && x < W)
      v = *reinterpret_cast<const uint4*>(X + (((size_t)zz * H + yy) * W + x) * kCh + 8 * half);
    *reinterpret_cast<uint4*>(halo + (zy * kHx + xx) * kVs + 8 * half) = v;
  }
}

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

__global__ void __launch_bounds__(128) k_conv3d(ConvArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* wsm = halo + 9 * kHx * kVs;
  const int y = blockIdx.x, z = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < 27 * kCh * 2; e += blockDim.x) {
    const int half = e & 1, row = e >> 1;  // row = tap * 16 + co
    *reinterpret_cast<uint4*>(wsm + row * kVs + 8 * half) =
        *reinterpret_cast<const uint4*>(a.Wt + row * kCh + 8 * half);
  }
  const int j = lane >> 3, r = lane & 7;
  const int g = lane >> 2, tq = lane & 3;
  float bias0[2], bias1[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    bias0[k] = a.bias ? a.bias[2 * tq + k] : 0.f;
    bias1[k] = a.bias ? a.bias[8 + 2 * tq + k] : 0.f;
  }
  for (int x0 = 0; x0 < a.W; x0 += kSeg) {
    __syncthreads();
    load_halo(halo, a.X, a.D, a.H, a.W, z, y, x0);
    __syncthreads();
    float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
    const int ai = r + 8 * (j & 1), ach = 8 * (j >> 1);  // A: voxel row, channel block
    const int bco = r + 8 * (j >> 1), bci = 8 * (j & 1);  // B: output channel, input block
#pragma unroll 3
    for (int t = 0; t < 27; ++t) {
      const int dzdy = t / 3, dx = t % 3 - 1;
      uint32_t af[4], bf[4];
      ldsm4(af, halo + (dzdy * kHx + 16 * warp + ai + dx + 1) * kVs + ach);
      ldsm4(bf, wsm + (t * kCh + bco) * kVs + bci);
      mma16816(acc0, af, bf[0], bf[1]);
      mma16816(acc1, af, bf[2], bf[3]);
    }
    // epilogue: rows g and g + 8 of the warp's 16 voxels
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = x0 + 16 * warp + g + 8 * h;
      if (x >= a.W) continue;
      const size_t v = ((size_t)z * a.H + y) * a.W + x;
      float o[4] = {acc0[2 * h] + bias0[0], acc0[2 * h + 1] + bias0[1], acc1[2 * h] + bias1[0],
                    acc1[2 * h + 1] + bias1[1]};
      if (a.out_f32) {
        if (tq == 0) a.Yf[v] = o[0];
        continue;
      }
      if (a.relu) {
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = fmaxf(o[k], 0.f);
      }
      if (a.mask) {
        const __nv_bfloat162 m0 = *reinterpret_cast<const __nv_bfloat162*>(a.mask + v * kCh + 2 * tq);
        const __nv_bfloat162 m1 = *reinterpret_cast<const __nv_bfloat162*>(a.mask + v * kCh + 8 + 2 * tq);
        if (!(__bfloat162float(m0.x) > 0.f)) o[0] = 0.f;
        if (!(__bfloat162float(m0.y) > 0.f)) o[1] = 0.f;
        if (!(__bfloat162float(m1.x) > 0.f)) o[2] = 0.f;
        if (!(__bfloat162float(m1.y) > 0.f)) o[3] = 0.f;
      }
      *reinterpret_cast<__nv_bfloat162*>(a.Y + v * kCh + 2 * tq) = __floats2bfloat162_rn(o[0], o[1]);
      *reinterpret_cast<__nv_bfloat162*>(a.Y + v * kCh + 8 + 2 * tq) = __floats2bfloat162_rn(o[2], o[3]);
    }
  }
}

// Weight and bias gradients of one band of rows: partial[block][tap][co][ci], partial_db[block][co].
__global__ void __launch_bounds__(128) k_conv3d_wgrad(const __nv_bfloat16* __restrict__ A,
                                                      const __nv_bfloat16* __restrict__ G,
                                                      float* partial, float* partial_db, int D,
                                                      int H, int W) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* gsm = halo + 9 * kHx * kVs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = lane >> 3, r = lane & 7;
  float acc[7][2][4];
#pragma unroll
  for (int q = 0; q < 7; ++q)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[q][nt][k] = 0.f;
  float db = 0.f;  // thread c < 16: bias gradient of output channel c
  const int row_lo = blockIdx.x * kWgradRows, row_hi = min(D * H, row_lo + kWgradRows);
  for (int zy = row_lo; zy < row_hi; ++zy) {
    const int z = zy / H, y = zy % H;
    for (int x0 = 0; x0 < W; x0 += kSeg) {
      __syncthreads();
      load_halo(halo, A, D, H, W, z, y, x0);
      for (int e = threadIdx.x; e < kSeg * 2; e += blockDim.x) {
        const int half = e & 1, xx = e >> 1, x = x0 + xx;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (x < W) v = *reinterpret_cast<const uint4*>(G + (((size_t)z * H + y) * W + x) * kCh + 8 * half);
        *reinterpret_cast<uint4*>(gsm + xx * kVs + 8 * half) = v;
      }
      __syncthreads();
      if (threadIdx.x < kCh) {
        for (int xx = 0; xx < kSeg; ++xx) db += __bfloat162float(gsm[xx * kVs + threadIdx.x]);
      }
#pragma unroll
      for (int kk = 0; kk < kSeg / 16; ++kk) {
        uint32_t af[4];
        // A = G^T (m = co, k = voxel) from storage rows = voxel, cols = co
        ldsm4t(af, gsm + (16 * kk + r + 8 * (j >> 1)) * kVs + 8 * (j & 1));
#pragma unroll
        for (int q = 0; q < 7; ++q) {
          const int t = warp + 4 * q;
          if (t < 27) {
            const int dzdy = t / 3, dx = t % 3 - 1;
            uint32_t bf[4];
            // B = A_shift (k = voxel, n = ci) from storage rows = voxel, cols = ci
            ldsm4t(bf, halo + (dzdy * kHx + 16 * kk + r + 8 * (j & 1) + dx + 1) * kVs + 8 * (j >> 1));
            mma16816(acc[q][0], af, bf[0], bf[1]);
            mma16816(acc[q][1], af, bf[2], bf[3]);
          }
        }
      }
    }
  }
  const int g = lane >> 2, tq = lane & 3;
  float* P = partial + (size_t)blockIdx.x * 27 * kCh * kCh;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const int t = warp + 4 * q;
    if (t >= 27) continue;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int ci = 8 * nt + 2 * tq;
      P[(t * kCh + g) * kCh + ci] = acc[q][nt][0];
      P[(t * kCh + g) * kCh + ci + 1] = acc[q][nt][1];
      P[(t * kCh + g + 8) * kCh + ci] = acc[q][nt][2];
      P[(t * kCh + g + 8) * kCh + ci + 1] = acc[q][nt][3];
    }
  }
  if (threadIdx.x < kCh) partial_db[blockIdx.x * kCh + threadIdx.x] = db;
}

// dW = sum over blocks of the partials, in block order (deterministic).
__global__ void k_conv3d_wgrad_reduce(const float* partial, const float* partial_db, int nblk,
                                      float* dW, float* db) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 27 * kCh * kCh) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * 27 * kCh * kCh + e];
    dW[e] = s;
  } else if (e < 27 * kCh * kCh + kCh) {
    const int c = e - 27 * kCh * kCh;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial_db[b * kCh + c];
    db[c] = s;
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

static pk_status conv_setup() {
  static bool done = false;
  if (!done) {
    const int fwd_smem = (9 * kHx * kVs + 27 * kCh * kVs) * 2;
    const int wg_smem = (9 * kHx * kVs + kSeg * kVs) * 2;
    PK_CUDA(cudaFuncSetAttribute(k_conv3d, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd_smem));
    PK_CUDA(cudaFuncSetAttribute(k_conv3d_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem));
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
  if (!X || !Wt || !Y || D <= 0 || H <= 0 || W <= 0 || H > 65535 || D > 65535) {
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
  const int smem = (9 * kHx * kVs + 27 * kCh * kVs) * 2;
  k_conv3d<<<dim3(H, D), 128, smem, (cudaStream_t)stream>>>(a);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

int64_t pk_conv3d_wgrad_scratch_floats(int32_t D, int32_t H, int32_t W) {
  (void)W;
  const int64_t nblk = ((int64_t)D * H + kWgradRows - 1) / kWgradRows;
  return nblk * (27 * kCh * kCh + kCh);
}

pk_status pk_conv3d_wgrad(const void* A, const void* G, float* scratch, float* dW, float* db,
                          int32_t D, int32_t H, int32_t W, void* stream) {
  if (!A || !G || !scratch || !dW || !db || D <= 0 || H <= 0 || W <= 0) {
    set_error("pk_conv3d_wgrad: bad arguments");
    return PK_ERR_ARG;
  }
  pk_status e = conv_setup();
  if (e) return e;
  const int nblk = (int)(((int64_t)D * H + kWgradRows - 1) / kWgradRows);
  float* partial = scratch;
  float* partial_db = scratch + (size_t)nblk * 27 * kCh * kCh;
  const int smem = (9 * kHx * kVs + kSeg * kVs) * 2;
  cudaStream_t s = (cudaStream_t)stream;
  k_conv3d_wgrad<<<nblk, 128, smem, s>>>(static_cast<const __nv_bfloat16*>(A),
                                         static_cast<const __nv_bfloat16*>(G), partial, partial_db,
                                         D, H, W);
  k_conv3d_wgrad_reduce<<<(27 * kCh * kCh + kCh + 255) / 256, 256, 0, s>>>(partial, partial_db, nblk, dW, db);
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
