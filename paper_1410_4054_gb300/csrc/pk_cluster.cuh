// Reductions shared by the solvers that run a whole iteration loop on one thread-block
// cluster with their vectors in the CTAs' shared memory (pipelined CG and BiCGStab on one
// system, and the batched solver's cluster engine).
//
// A fused phase ends with a block sum of its partial inner products into the CTA's slots, a
// hardware cluster barrier, and the cluster total: every CTA reads all C CTAs' slots in rank
// order through distributed shared memory and adds them with the same butterfly, so every CTA
// holds bit-identical scalars and takes the same decisions (control flow stays uniform across
// the cluster; there is no spin-wait).
#pragma once

#include <cooperative_groups.h>

#include "pk_internal.cuh"

namespace pk {

namespace cg = cooperative_groups;

// Fixed-order block sum of NV values over NT threads, broadcast to every thread.  GB300
// issues about two FP64 operations per clock per SM and an FP64 add has a long latency, so the
// sum is done by one warp with short dependency chains: every thread stages its values in buf
// (NV * NT doubles), each lane of warp 0 adds NT/32 of them as a pairwise tree (the NV sums
// interleaved), and a butterfly finishes (both partners of a pair add the same two values, so
// every lane ends with the same bits).
template <int NT, int NV>
__device__ __forceinline__ void cluster_block_sum(const double (&v)[NV], double* buf, double (&out)[NV]) {
  constexpr int PER = NT / 32;
  static_assert(PER == 4 || PER == 8 || PER == 16, "4, 8 or 16 values per lane");
  __shared__ double bc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) buf[k * NT + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    double t[NV][PER];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int m = 0; m < PER; ++m) t[k][m] = buf[k * NT + m * 32 + threadIdx.x];
#pragma unroll
    for (int h = PER / 2; h >= 1; h >>= 1)
#pragma unroll
      for (int m = 0; m < h; ++m)
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k][m] = t[k][m] + t[k][m + h];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k) t[k][0] += __shfl_xor_sync(0xffffffffu, t[k][0], o);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) bc[k] = t[k][0];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = bc[k];
}

// Cluster total of slots [s0, s0 + NV) of every CTA (after a cluster barrier): lane c of warp
// 0 reads CTA c's values from distributed shared memory, then a butterfly over the lanes (the
// NV sums interleaved); every CTA runs the same additions on the same values.
template <int NV>
__device__ __forceinline__ void cluster_total(cg::cluster_group& cl, double* slots, int s0, double (&out)[NV]) {
  __shared__ double bc[NV];
  if (threadIdx.x < 32) {
    const int C = (int)cl.num_blocks();
    double t[NV];
    const double* rem = threadIdx.x < C ? cl.map_shared_rank(slots, (int)threadIdx.x) : nullptr;
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = rem ? rem[s0 + k] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) bc[k] = t[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = bc[k];
}

// Element `c` of a vector distributed over the cluster, R = 2^lg rows per CTA, each CTA's part
// at `local` in its shared memory.
__device__ __forceinline__ double cluster_elem(cg::cluster_group& cl, double* local, int lg, int c) {
  return *cl.map_shared_rank(local + (c & ((1 << lg) - 1)), c >> lg);
}

// Row `row` of A times a distributed vector: four entries per step with their loads
// independent, products added left to right.  j, j1: the row's entries.
__device__ __forceinline__ double cluster_row(cg::cluster_group& cl, const int32_t* __restrict__ ci,
                                              const double* __restrict__ va, double* local, int lg, int j,
                                              const int j1) {
  double s = 0.0;
  for (; j + 4 <= j1; j += 4) {
    int c[4];
    double w[4], pv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c[k] = __ldg(ci + j + k);
      w[k] = __ldg(va + j + k);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) pv[k] = cluster_elem(cl, local, lg, c[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) s = fma(w[k], pv[k], s);
  }
  for (; j < j1; ++j) s = fma(__ldg(va + j), cluster_elem(cl, local, lg, __ldg(ci + j)), s);
  return s;
}

}  // namespace pk
