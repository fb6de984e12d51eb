// SELL-C-sigma storage and the fused SpMV + inner-product kernels on it (the sliced ELLPACK
// format of Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J. Sci. Comput. 36(5), 2014; the
// paper runs its finite-element benchmarks in ELLPACK, Sec. 4.1).
//
// Rows are sorted by length (longest first) inside windows of kSellSigma rows, cut into
// slices of kSellC = 32 consecutive sorted rows, and each slice is padded to its longest row
// and stored column-major: entry k of the slice's lane l sits at ptr[slice] + 32 k + l.  A
// warp takes a slice, lane l its row: every load of values and column indices is one
// coalesced 256- or 128-byte line, no row pointer is read, and a padding entry (column -1)
// issues no gather.  Each row is summed left to right like the CSR loop.
#include <algorithm>
#include <vector>

#include "pk_guard.cuh"
#include "pk_internal.cuh"
#include "pk_tile.cuh"

namespace pk {

namespace {

constexpr int kSellSigma = 1024;

// q = A p with the first reduction stage of <p, q>; the last block writes *out.
__global__ void __launch_bounds__(kBlock) k_sell_spmv_dot(SellArgs s, const double* __restrict__ p,
                                                          double* __restrict__ q, double* partials,
                                                          DevState* st, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[1] = {0.0};
  for (int sl = blockIdx.x * kSellWarps + warp; sl < s.nslices; sl += gridDim.x * kSellWarps) {
    const int64_t base = s.ptr[sl];
    const int w = (int)((s.ptr[sl + 1] - base) / kSellC);
    const int row = s.perm[(size_t)sl * kSellC + lane];
    const double y = sell_row(s, base + lane, w, p);
    if (row >= 0) {
      q[row] = y;
      v[0] = fma(__ldg(p + row), y, v[0]);
    }
  }
  block_partials<1>(v, partials);
  if (arrive_last(&st->counter)) {
    double t[1];
    final_sums<1>(partials, t);
    if (threadIdx.x == 0) {
      *out = t[0];
      st->counter = 0;
    }
  }
}

}  // namespace

// Builds A's SELL-C-sigma copy on first use (synchronous on stream s: the CSR arrays are read
// back to the host once).  The handle's SELL fields are set only once every copy is complete;
// a failed attempt frees what it allocated and leaves the handle as it was.
pk_status sell_build(pk_csr* A, cudaStream_t s) {
  if (A->sell_nslices >= 0) return PK_OK;
  int64_t* d_ptr = nullptr;
  int32_t *d_perm = nullptr, *d_col = nullptr;
  double* d_val = nullptr;
  int64_t ns = 0, total = 0;
  int grid = 1;
  const pk_status e = guarded([&]() -> pk_status {
    const int64_t n = A->n, nnz = A->nnz;
    std::vector<int32_t> rp(n + 1), ci(nnz);
    std::vector<double> va(nnz);
    PK_CUDA(cudaStreamSynchronize(s));
    PK_CUDA(cudaMemcpy(rp.data(), A->rp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
    if (nnz) {
      PK_CUDA(cudaMemcpy(ci.data(), A->ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
      PK_CUDA(cudaMemcpy(va.data(), A->va, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
    }
    // rows sorted by length inside each window of kSellSigma rows (stable: ties keep row order)
    std::vector<int32_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    for (int64_t w0 = 0; w0 < n; w0 += kSellSigma) {
      const int64_t w1 = std::min<int64_t>(n, w0 + kSellSigma);
      std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int32_t a, int32_t b) {
        return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
      });
    }
    ns = (n + kSellC - 1) / kSellC;
    std::vector<int64_t> ptr(ns + 1, 0);
    for (int64_t sl = 0; sl < ns; ++sl) {
      int64_t w = 0;
      for (int l = 0; l < kSellC; ++l) {
        const int64_t i = sl * kSellC + l;
        if (i < n) w = std::max<int64_t>(w, rp[order[i] + 1] - rp[order[i]]);
      }
      ptr[sl + 1] = ptr[sl] + w * kSellC;
    }
    total = ptr[ns];
    if (total >= (int64_t(1) << 31)) { set_error("SELL-C-sigma copy: padded size >= 2^31"); return PK_ERR_ARG; }
    std::vector<int32_t> col(total, -1), perm(ns * kSellC, -1);
    std::vector<double> val(total, 0.0);
    for (int64_t sl = 0; sl < ns; ++sl)
      for (int l = 0; l < kSellC; ++l) {
        const int64_t i = sl * kSellC + l;
        if (i >= n) continue;
        const int32_t r = order[i];
        perm[i] = r;
        for (int64_t k = 0; k < rp[r + 1] - rp[r]; ++k) {
          col[ptr[sl] + k * kSellC + l] = ci[rp[r] + k];
          val[ptr[sl] + k * kSellC + l] = va[rp[r] + k];
        }
      }
    PK_CUDA(cudaMalloc(&d_ptr, sizeof(int64_t) * (ns + 1)));
    PK_CUDA(cudaMalloc(&d_perm, sizeof(int32_t) * std::max<int64_t>(1, ns * kSellC)));
    PK_CUDA(cudaMalloc(&d_col, sizeof(int32_t) * std::max<int64_t>(1, total)));
    PK_CUDA(cudaMalloc(&d_val, sizeof(double) * std::max<int64_t>(1, total)));
    PK_CUDA(cudaMemcpy(d_ptr, ptr.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice));
    if (ns) PK_CUDA(cudaMemcpy(d_perm, perm.data(), sizeof(int32_t) * ns * kSellC, cudaMemcpyHostToDevice));
    if (total) {
      PK_CUDA(cudaMemcpy(d_col, col.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice));
      PK_CUDA(cudaMemcpy(d_val, val.data(), sizeof(double) * total, cudaMemcpyHostToDevice));
    }
    int sms = 1;
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
    grid = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)A->partial_cap, (int64_t)sms * kMaxGridPerSm, (ns + kSellWarps - 1) / kSellWarps}));
    return PK_OK;
  });
  if (e) {
    if (d_ptr) cudaFree(d_ptr);
    if (d_perm) cudaFree(d_perm);
    if (d_col) cudaFree(d_col);
    if (d_val) cudaFree(d_val);
    return e;
  }
  A->sell_ptr = d_ptr;
  A->sell_perm = d_perm;
  A->sell_col = d_col;
  A->sell_val = d_val;
  A->sell_padded = total;
  A->sell_grid = grid;
  A->sell_nslices = (int32_t)ns;
  return PK_OK;
}

SellArgs sell_args(const pk_csr* A) {
  SellArgs s;
  s.nslices = A->sell_nslices;
  s.ptr = A->sell_ptr;
  s.perm = A->sell_perm;
  s.col = A->sell_col;
  s.val = A->sell_val;
  return s;
}

pk_status launch_sell_spmv_dot(pk_csr* A, const double* p, double* q, double* out, cudaStream_t s) {
  pk_status e = sell_build(A, s);
  if (e) return e;
  k_sell_spmv_dot<<<A->sell_grid, kBlock, 0, s>>>(sell_args(A), p, q, A->partials, A->st, out);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

}  // namespace pk
