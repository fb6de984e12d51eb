// Right preconditioning with M = diag(A) for BiCGStab and GMRES (the preconditioner fusion that
// Sec. 5 names as the extension of the method, taken to its limit for a diagonal M).
//
// A Krylov solver applied to A M^-1 y = b has the residual b - A M^-1 y = b - A x of x = M^-1 y:
// its stopping test is the unpreconditioned one and its iterates are those of the right-
// preconditioned solver.  A M^-1 is A with every column scaled by the reciprocal diagonal
// entry, so the solver's fused kernels run unchanged on a scaled copy of the values, built
// once per matrix: no byte and no flop is added to an iteration.  y0 = M x0 before the solve,
// x = M^-1 y after it.
#include "pk_internal.cuh"

#include <cmath>

namespace pk {

namespace {

// d = diag(A) (entries of row i in column i summed), dinv = 1/d; *bad = 1 if some d_i is zero
// or not finite.
__global__ void __launch_bounds__(kBlock) k_jacobi_diag(int n, const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci,
                                                        const double* __restrict__ va,
                                                        double* __restrict__ d, double* __restrict__ dinv,
                                                        int* bad) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = rp[row]; j < rp[row + 1]; ++j)
      if (ci[j] == row) s += va[j];
    if (s == 0.0 || !isfinite(s)) {
      *bad = 1;
      s = 1.0;
    }
    d[row] = s;
    dinv[row] = 1.0 / s;
  }
}

// Values of A M^-1: every entry times the reciprocal diagonal entry of its column.
__global__ void __launch_bounds__(kBlock) k_scale_columns(int nnz, const int32_t* __restrict__ ci,
                                                          const double* __restrict__ va,
                                                          const double* __restrict__ dinv,
                                                          double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += gridDim.x * blockDim.x)
    out[j] = va[j] * dinv[ci[j]];
}

// x <- s .* x (s = d for y0 = M x0, s = dinv for x = M^-1 y).
__global__ void __launch_bounds__(kBlock) k_scale_vec(int n, double* __restrict__ x,
                                                      const double* __restrict__ s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = x[i] * s[i];
}

int grid_for(int64_t items) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (items + kBlock - 1) / kBlock));
}

pk_status build_cache(pk_csr* A, cudaStream_t s) {
  const size_t nv = (size_t)A->n + 64, nz = (size_t)A->nnz + 64;
  // a retry after a failed allocation reuses what the earlier attempt got
  if (!A->jac_va) PK_CUDA(cudaMalloc(&A->jac_va, sizeof(double) * nz));
  if (!A->jac_d) PK_CUDA(cudaMalloc(&A->jac_d, sizeof(double) * nv));
  if (!A->jac_dinv) PK_CUDA(cudaMalloc(&A->jac_dinv, sizeof(double) * nv));
  PK_CUDA(cudaMemsetAsync(A->jac_va, 0, sizeof(double) * nz, s));
  int* bad = reinterpret_cast<int*>(A->small + 8100);
  PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_jacobi_diag<<<grid_for(A->n), kBlock, 0, s>>>(A->n, A->rp, A->ci, A->va, A->jac_d, A->jac_dinv, bad);
  k_scale_columns<<<grid_for(A->nnz), kBlock, 0, s>>>(A->nnz, A->ci, A->va, A->jac_dinv, A->jac_va);
  PK_CUDA(cudaGetLastError());
  int h = 0;
  PK_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  PK_CUDA(cudaStreamSynchronize(s));
  A->jac_state = h ? -1 : 1;
  return PK_OK;
}

}  // namespace

pk_status jacobi_right_enter(pk_csr* A, double* x, cudaStream_t s, JacobiRight* g) {
  if (A->jac_state == 0) {
    pk_status e = build_cache(A, s);
    if (e) return e;
  }
  if (A->jac_state < 0) {
    set_error("PK_PRECOND_JACOBI needs a nonzero finite diagonal");
    return PK_ERR_ARG;
  }
  k_scale_vec<<<grid_for(A->n), kBlock, 0, s>>>(A->n, x, A->jac_d);
  PK_CUDA(cudaGetLastError());
  g->A = A;
  g->saved_va = A->va;
  A->va = A->jac_va;
  return PK_OK;
}

pk_status jacobi_right_leave(JacobiRight* g, double* x, cudaStream_t s) {
  pk_csr* A = g->A;
  if (!A) return PK_OK;
  A->va = g->saved_va;
  g->A = nullptr;
  k_scale_vec<<<grid_for(A->n), kBlock, 0, s>>>(A->n, x, A->jac_dinv);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

}  // namespace pk
