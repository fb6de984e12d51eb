// The cluster engine of the batched solver: pipelined CG (Alg. 2, Sec. 3.1) on many
// independent systems, each solved to completion by one thread-block cluster whose CTAs hold
// the system's p, x, r and Ap in shared memory.
//
// A system of n rows goes to a cluster of C CTAs (C = 1, 2, 4, 8 or 16) of R rows each
// (R = 2^k, R C >= n); CTA k owns rows [k R, (k+1) R).  Per iteration only the matrix is read
// from global memory (12 bytes per nonzero, 4 per row pointer, and the matrices of the systems
// in flight fit in L2), against 76 bytes per row of vector traffic in the launched form.  An
// iteration is the launched form's two fused phases:
//   Ap = A p, gathering p from the owning CTA's shared memory through the cluster's
//   distributed shared memory, with the block sums of <Ap,Ap>, <p,Ap>;
//   the x, r, p updates with the block sum of <r,r>;
// each ending in a cluster barrier after which every CTA adds the C block sums in rank order,
// so all CTAs hold bit-identical alpha, beta and <r,r> and take the same decisions: control
// flow is uniform across the cluster and there is no spin-wait.
//
// Three shapes, so that more than one CTA can share an SM and one CTA's reductions and
// barriers overlap another's row products: 512 threads and up to 4096 rows (1 CTA per SM),
// 256 threads and 2048 rows (2 per SM), 128 threads and 1024 rows (4 per SM).  Each (shape,
// C) class of the batch is one persistent launch that takes systems from the class's queue;
// the host puts the classes on streams of their own so that they share the GPU.
#include <algorithm>

#include "pk_cluster.cuh"

namespace pk {

namespace {

struct BatchClArgs {
  BatchClSys* sys;
  int end;     // the class's systems: from the queue's start value to end
  int* queue;  // next system of the class (atomic)
  double tol;
  int maxit;
};

constexpr int kBcSlots = 4;  // block sums per CTA: <Ap,Ap>, <p,Ap> | <r,r>

// Shared memory of a CTA of NT threads and up to MAXR rows: p, x, r, Ap, the slots, the
// reduction buffer (2 NT) and MAXR + 1 row pointers (padded).
template <int NT, int MAXR>
constexpr size_t bc_smem() {
  return sizeof(double) * (4 * (size_t)MAXR + kBcSlots + 2 * NT) + sizeof(int) * (MAXR + 4);
}

// Row l of this CTA (row pointers staged in srp) times p.
__device__ __forceinline__ double bc_row(const BatchClSys& S, cg::cluster_group& cl, double* sp, const int* srp,
                                         int lg, int l) {
  return cluster_row(cl, S.ci, S.va, sp, lg, srp[l], srp[l + 1]);
}

}  // namespace

template <int NT, int MAXR>
__global__ void __launch_bounds__(NT, 512 / NT) k_batched_cluster(BatchClArgs a) {
  extern __shared__ __align__(16) double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  __shared__ int s_sys;
  __shared__ double sc[2];
  __shared__ int scs;
  double* slots = sm + 4 * MAXR;
  double* buf = slots + kBcSlots;
  int* srp = reinterpret_cast<int*>(buf + 2 * NT);  // this CTA's row pointers
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_sys = atomicAdd(a.queue, 1);
    cl.sync();
    const int k = *cl.map_shared_rank(&s_sys, 0);
    cl.sync();  // every CTA has read rank 0's choice before rank 0 takes the next one
    if (k >= a.end) break;  // the same k in every CTA: the cluster leaves together
    const BatchClSys S = a.sys[k];
    const int n = S.n;
    int lg = 5;
    while ((1 << lg) * C < n) ++lg;
    const int R = 1 << lg;
    if (R > MAXR) {  // the host plans classes so that this does not happen
      if (rank == 0 && threadIdx.x == 0) a.sys[k].status = PK_ERR_ARG;
      cl.sync();
      continue;
    }
    double* sp = sm;  // p (read remotely by the SpMV); x during the setup product
    double* sx = sm + R;
    double* sr = sm + 2 * R;
    double* sa = sm + 3 * R;
    const int row0 = rank * R;
    const int nown = max(0, min(n - row0, R));
    for (int l = threadIdx.x; l < nown; l += NT) {
      const double xv = S.x[row0 + l];
      sx[l] = xv;
      sp[l] = xv;
    }
    if (nown > 0)  // (a CTA past the last row reads no row pointer: rp has n + 1 entries)
      for (int l = threadIdx.x; l <= nown; l += NT) srp[l] = __ldg(S.rp + row0 + l);
    cl.sync();
    // r0 = b - A x0 (the product gathers x from sp), <r0,r0>, <b,b>
    double v[2] = {0.0, 0.0};
    for (int l = threadIdx.x; l < nown; l += NT) {
      const double bi = __ldg(S.b + row0 + l);
      const double ri = bi - bc_row(S, cl, sp, srp, lg, l);
      sr[l] = ri;
      v[0] = fma(ri, ri, v[0]);
      v[1] = fma(bi, bi, v[1]);
    }
    double t[2];
    cluster_block_sum<NT, 2>(v, buf, t);
    if (threadIdx.x == 0) {
      slots[0] = t[0];
      slots[1] = t[1];
    }
    cl.sync();  // (also: no CTA reads sp any more)
    cluster_total<2>(cl, slots, 0, t);
    double rr = t[0];
    const double bb = t[1], thr2 = a.tol * a.tol * bb;
    for (int l = threadIdx.x; l < nown; l += NT) sp[l] = sr[l];  // p0 = r0
    int status = kRunning, iters = 0;
    if (!isfinite(rr) || !isfinite(bb)) status = PK_ERR_NAN;
    else if (bb == 0.0) {
      for (int l = threadIdx.x; l < nown; l += NT) sx[l] = 0.0;
      status = PK_OK;
    } else if (rr <= thr2) status = PK_OK;
    else if (a.maxit <= 0) status = PK_NOT_CONVERGED;
    cl.sync();  // p0 in place before the first remote gather
    for (int i = 0; status == kRunning; ++i) {
      // A p_i and <Ap_i, Ap_i>, <p_i, Ap_i> -> alpha, beta (Eq. (3))
      v[0] = v[1] = 0.0;
      for (int l = threadIdx.x; l < nown; l += NT) {
        const double y = bc_row(S, cl, sp, srp, lg, l);
        sa[l] = y;
        v[0] = fma(y, y, v[0]);
        v[1] = fma(sp[l], y, v[1]);
      }
      cluster_block_sum<NT, 2>(v, buf, t);
      if (threadIdx.x == 0) {
        slots[0] = t[0];
        slots[1] = t[1];
      }
      cl.sync();
      cluster_total<2>(cl, slots, 0, t);
      if (threadIdx.x == 0) {
        int sts = kRunning;
        double al = 0.0, be = 0.0;
        if (!isfinite(t[0]) || !isfinite(t[1])) sts = PK_ERR_NAN;
        else if (t[1] <= 0.0) sts = PK_NOT_SPD;
        else {
          al = rr / t[1];
          be = al * al * t[0] / rr - 1.0;
        }
        sc[0] = al;
        sc[1] = be;
        scs = sts;
      }
      __syncthreads();
      if (scs != kRunning) {
        status = scs;
        break;
      }
      const double alpha = sc[0], beta = sc[1];
      // x, r, p updates (no CTA gathers p before the next cluster barrier) and <r, r>
      double w[1] = {0.0};
      for (int l = threadIdx.x; l < nown; l += NT) {
        const double pk = sp[l];
        sx[l] = fma(alpha, pk, sx[l]);
        const double rn = fma(-alpha, sa[l], sr[l]);
        sr[l] = rn;
        sp[l] = fma(beta, pk, rn);
        w[0] = fma(rn, rn, w[0]);
      }
      double u[1];
      cluster_block_sum<NT, 1>(w, buf, u);
      if (threadIdx.x == 0) slots[2] = u[0];
      cl.sync();
      cluster_total<1>(cl, slots, 2, u);
      rr = u[0];
      iters = i + 1;
      if (!isfinite(rr)) status = PK_ERR_NAN;
      else if (rr <= thr2) status = PK_OK;
      else if (i + 1 >= a.maxit) status = PK_NOT_CONVERGED;
    }
    for (int l = threadIdx.x; l < nown; l += NT) S.x[row0 + l] = sx[l];
    if (rank == 0 && threadIdx.x == 0) {
      a.sys[k].iters = iters;
      a.sys[k].status = status;
      a.sys[k].rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
    }
    cl.sync();  // no CTA reuses its shared memory while another may still read it
  }
}

namespace {

using BcKernel = void (*)(BatchClArgs);

struct BcShape {
  int threads, max_rows;
  BcKernel kernel;
  size_t smem;
};

const BcShape kBcShapes[kBcShapeCount] = {
    {512, 4096, k_batched_cluster<512, 4096>, bc_smem<512, 4096>()},
    {256, 2048, k_batched_cluster<256, 2048>, bc_smem<256, 2048>()},
    {128, 1024, k_batched_cluster<128, 1024>, bc_smem<128, 1024>()},
};

cudaLaunchConfig_t bc_config(const BcShape& sh, int C, int clusters, cudaLaunchAttribute* at, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * clusters);
  cfg.blockDim = dim3(sh.threads);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

int batched_cluster_max_rows(int shape) { return shape >= 0 && shape < kBcShapeCount ? kBcShapes[shape].max_rows : 0; }

// Clusters of C CTAs of the given shape that the device can run at once (0: not usable).
int batched_cluster_capacity(int shape, int C) {
  static int cap[kBcShapeCount][17];
  static bool init = false;
  if (!init) {
    for (auto& row : cap)
      for (int& c : row) c = -1;
    init = true;
  }
  if (shape < 0 || shape >= kBcShapeCount || C < 1 || C > 16) return 0;
  int& out = cap[shape][C];
  if (out >= 0) return out;
  out = 0;
  const BcShape& sh = kBcShapes[shape];
  if (cudaFuncSetAttribute(sh.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess ||
      cudaFuncSetAttribute(sh.kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = bc_config(sh, C, 1, at, 0);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, sh.kernel, &cfg) == cudaSuccess) out = nc;
  cudaGetLastError();
  return out;
}

// One persistent launch of clusters of C CTAs of the given shape over the systems
// [first, end) of sys (the queue starts at first; the caller sets it).
pk_status launch_batched_cluster(int shape, BatchClSys* sys, int first, int end, int* queue, int C, double tol,
                                 int maxit, cudaStream_t s) {
  const int cap = batched_cluster_capacity(shape, C);
  if (cap <= 0) {
    set_error("batched cluster engine: cluster shape not available on this device");
    return PK_ERR_ARG;
  }
  const int clusters = std::max(1, std::min(end - first, cap));
  BatchClArgs a{sys, end, queue, tol, maxit};
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = bc_config(kBcShapes[shape], C, clusters, at, s);
  PK_CUDA(cudaLaunchKernelEx(&cfg, kBcShapes[shape].kernel, a));
  return PK_OK;
}

}  // namespace pk
