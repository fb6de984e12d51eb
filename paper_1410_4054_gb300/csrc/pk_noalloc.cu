// Allocation-free variant of the fused SpMV + inner product (q = A p, <p, q>).
//
// Some callers cannot allocate device memory at the point where they need this product:
// real-time or embedded loops whose memory budget is fixed up front (an allocation could fail
// or stall mid-loop), and host code that must not touch a caching allocator it does not own
// (a second allocator in the process fragments or double-books device memory).  pk_spmv_dot needs a pk_csr handle, whose
// creation allocates; this entry point takes the caller's own device CSR arrays and keeps its
// scratch -- one partial sum per thread block plus the arrival counter of the last-block
// reduction -- in a fixed, file-scope device array instead.
//
// The array is part of the library's device image, so every GPU that loads the library holds
// it (PK_NOALLOC_SCRATCH_BYTES) until the process exits, and every call on a device shares
// it: calls that overlap on the GPU (for example on two streams at once) race with each
// other.  Each call clears the counter before its kernel, so no state carries over from the
// previous call beyond the array's stale contents, which the kernel overwrites.
#include <algorithm>
#include <mutex>

#include "pk_internal.cuh"

namespace pk {

constexpr int kNaBlocks = PK_NOALLOC_MAX_BLOCKS;          // partial-sum slots
constexpr int kNaScratchBytes = PK_NOALLOC_SCRATCH_BYTES;  // counter line + partials

static_assert(256 + 8 * kNaBlocks <= kNaScratchBytes, "scratch layout");

// Device scratch: bytes [0, 4) the arrival counter, bytes [256, 256 + 8 * kNaBlocks) the
// per-block partial sums.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Host-side addresses of g_noalloc_scratch, one per device (the symbol itself is only a
// host stand-in and must never be passed to a kernel).  Looked up once per device for the
// life of the process: after a cudaDeviceReset the library's module, and with it the array,
// may be loaded at another address, so calls after a reset are not supported.
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64] = {nullptr};

static pk_status noalloc_scratch(void** out) {
  int dev = 0;
  PK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("pk_spmv_dot_noalloc: device index above 63");
    return PK_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    PK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return PK_OK;
}

// Thread-per-row fused product over equal row chunks; block partials in the scratch array,
// second reduction stage (fixed order) in the last block to arrive.
__global__ void __launch_bounds__(kBlock) k_spmv_dot_noalloc(RowArgs a, int chunk,
                                                             const double* __restrict__ p,
                                                             double* __restrict__ q,
                                                             unsigned char* scratch,
                                                             double* result) {
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + 256);
  const long long lo = (long long)blockIdx.x * chunk;
  const int r0 = (int)(lo < a.n ? lo : a.n);
  const int r1 = (int)(lo + chunk < a.n ? lo + chunk : a.n);
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double s = csr_row(a, p, row);
    q[row] = s;
    v[0] = fma(__ldg(p + row), s, v[0]);
  }
  block_partials<1>(v, partials);
  if (arrive_last(counter)) {
    double t[1];
    final_sums<1>(partials, t);
    if (threadIdx.x == 0) {
      *result = t[0];
      *counter = 0;
    }
  }
}

}  // namespace pk

using namespace pk;

extern "C" pk_status pk_spmv_dot_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                         const double* vals, const double* p, double* q,
                                         double* result, void* stream) {
  if (n < 0 || n > PK_NOALLOC_MAX_N) {
    set_error("pk_spmv_dot_noalloc: n must be in [0, PK_NOALLOC_MAX_N = 16777216]");
    return PK_ERR_ARG;
  }
  if (!result || (n > 0 && (!row_ptr || !col_idx || !vals || !p || !q))) {
    set_error("pk_spmv_dot_noalloc: NULL argument");
    return PK_ERR_ARG;
  }
  if (n > 0 && (const void*)q == (const void*)p) {  // rows read p[col] while others write q
    set_error("pk_spmv_dot_noalloc: q must not be p");
    return PK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    PK_CUDA(cudaMemsetAsync(result, 0, sizeof(double), s));
    return PK_OK;
  }
  void* scratch = nullptr;
  pk_status e = noalloc_scratch(&scratch);
  if (e) return e;
  // equal chunks of at least kBlock rows (multiples of 32), at most kNaBlocks blocks
  const int64_t need = (n + kNaBlocks - 1) / kNaBlocks;
  const int chunk = (int)std::max<int64_t>(kBlock, (need + 31) & ~int64_t(31));
  const int grid = (int)((n + chunk - 1) / chunk);
  RowArgs a{};
  a.n = (int32_t)n;
  a.rp = row_ptr;
  a.ci = col_idx;
  a.va = vals;
  PK_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s));  // the counter starts at 0
  k_spmv_dot_noalloc<<<grid, kBlock, 0, s>>>(a, chunk, p, q, static_cast<unsigned char*>(scratch),
                                             result);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}
