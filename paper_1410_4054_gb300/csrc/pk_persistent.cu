// Persistent pipelined CG (Alg. 2, Sec. 3.1) on one thread-block cluster, for systems small
// enough that two kernel launches, or two grid-wide synchronisations through L2, per
// iteration would dominate the solve.
//
// One cluster of C CTAs (16 where the device allows it, else 8) runs every iteration of the
// solve.  CTA k owns rows [k*R, (k+1)*R) with R a power of two; their p, x, r and Ap live in
// the CTA's shared memory for the whole solve.  An iteration is the two fused phases of the
// launched form:
//   K-CG-S  Ap = A p (the gathers of p read the owning CTA's shared memory through the
//           cluster's distributed shared memory) with the block sums of <Ap,Ap>, <p,Ap>;
//   K-CG-U  x, r, p updates with the block sum of <r,r>;
// each ending in a hardware cluster barrier, after which every CTA reads the C block sums in
// rank order from distributed shared memory, so all CTAs hold bit-identical alpha, beta and
// <r,r> and take the same exit decision.  Control flow is uniform across the cluster (no CTA
// leaves a loop another one continues), there is no spin-wait, and a final cluster barrier
// keeps every CTA's shared memory alive until the last remote read.
#include <algorithm>

#include "pk_cluster.cuh"

namespace pk {

namespace {

constexpr int kCT = 512;          // threads per CTA
constexpr int kMaxRows = 4096;    // rows per CTA held in shared memory
constexpr int kSlots = 4;         // block sums per CTA: <Ap,Ap>, <p,Ap> | <r,r>

struct ClusterArgs {
  int32_t n;
  int32_t log_rows;  // rows per CTA = 1 << log_rows
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  double* x;
  double* r;
  double* p;
  DevState* st;
};

__global__ void __launch_bounds__(kCT, 1) k_cg_cluster(ClusterArgs a) {
  extern __shared__ __align__(16) double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int R = 1 << a.log_rows;
  const int rank = (int)cl.block_rank();
  double* sp = sm;            // p of the owned rows (read remotely by the SpMV)
  double* sx = sm + R;
  double* sr = sm + 2 * R;
  double* sa = sm + 3 * R;    // Ap
  double* slots = sm + 4 * R; // kSlots block sums
  double* buf = slots + kSlots; // 2 * kCT staging values of block_sum
  const int row0 = rank * R;
  const int nown = max(0, min(a.n - row0, R));
  DevState* st = a.st;
  // every CTA reads the same flag written by the setup kernel: a uniform decision
  const bool done0 = __ldcg(&st->done) != 0;
  for (int l = threadIdx.x; l < nown; l += kCT) {
    sp[l] = a.p[row0 + l];
    sx[l] = a.x[row0 + l];
    sr[l] = a.r[row0 + l];
  }
  const double thr2 = __ldcg(&st->thr2);
  const int maxit = __ldcg(&st->maxit);
  double rr = __ldcg(&st->rr);
  const bool lead = rank == 0 && threadIdx.x == 0;
  // the trace target is read once: a DevState line re-read after a store would cost an L2
  // round trip on the critical path of every iteration
  double* const trace = st->trace;
  const int trace_cap = st->trace_cap;
  double alpha_last = 0.0, beta_last = 0.0;
  int iters = 0;
  int status = kRunning;
  __shared__ double sc[2];  // alpha, beta
  __shared__ int scs;       // exit status decided by thread 0 (kRunning: continue)
  cl.sync();  // every CTA's p is in place before the first remote gather
  for (int i = 0; !done0; ++i) {
    // K-CG-S: Ap_i and <Ap_i, Ap_i>, <p_i, Ap_i>
    double v[2] = {0.0, 0.0};
    for (int l = threadIdx.x; l < nown; l += kCT) {
      const int row = row0 + l;
      const double s = cluster_row(cl, a.ci, a.va, sp, a.log_rows, __ldg(a.rp + row), __ldg(a.rp + row + 1));
      sa[l] = s;
      v[0] = fma(s, s, v[0]);
      v[1] = fma(sp[l], s, v[1]);
    }
    double t[2];
    cluster_block_sum<kCT, 2>(v, buf, t);
    if (threadIdx.x == 0) { slots[0] = t[0]; slots[1] = t[1]; }
    cl.sync();
    cluster_total<2>(cl, slots, 0, t);
    // the scalar work (two FP64 divisions) runs in one thread and is broadcast: on GB300 every
    // FP64 instruction issued by all warps of a CTA costs the SM's narrow FP64 pipe
    if (threadIdx.x == 0) {
      int sts = kRunning;
      double al = 0.0, be = 0.0;
      if (!isfinite(t[0]) || !isfinite(t[1])) sts = PK_ERR_NAN;
      else if (t[1] <= 0.0) sts = PK_NOT_SPD;
      else {
        // Eq. (3): alpha_i = <r_i,r_i>/<p_i,Ap_i>, beta_i = alpha_i^2 <Ap_i,Ap_i>/<r_i,r_i> - 1
        al = rr / t[1];
        be = al * al * t[0] / rr - 1.0;
        if (lead && trace && i < trace_cap) {
          trace[(size_t)i * 4 + 0] = al;
          trace[(size_t)i * 4 + 1] = be;
        }
      }
      sc[0] = al;
      sc[1] = be;
      scs = sts;
    }
    __syncthreads();
    if (scs != kRunning) { status = scs; break; }
    const double alpha = sc[0], beta = sc[1];
    alpha_last = alpha;
    beta_last = beta;
    // K-CG-U: x_{i+1}, r_{i+1}, p_{i+1} and <r_{i+1}, r_{i+1}>.  No CTA gathers p again
    // before the next barrier, so p is updated in place.
    double w[1] = {0.0};
    for (int l = threadIdx.x; l < nown; l += kCT) {
      const double pk = sp[l];
      sx[l] = fma(alpha, pk, sx[l]);
      const double rn = fma(-alpha, sa[l], sr[l]);
      sr[l] = rn;
      sp[l] = fma(beta, pk, rn);
      w[0] = fma(rn, rn, w[0]);
    }
    double u[1];
    cluster_block_sum<kCT, 1>(w, buf, u);
    if (threadIdx.x == 0) slots[2] = u[0];
    cl.sync();
    cluster_total<1>(cl, slots, 2, u);
    rr = u[0];
    iters = i + 1;
    if (threadIdx.x == 0) {
      int sts = kRunning;
      if (!isfinite(rr)) sts = PK_ERR_NAN;
      else if (rr <= thr2) sts = PK_OK;
      else if (i + 1 >= maxit) sts = PK_NOT_CONVERGED;
      if (lead && trace && i < trace_cap) trace[(size_t)i * 4 + 3] = rr;
      scs = sts;
    }
    __syncthreads();
    if (scs != kRunning) { status = scs; break; }
  }
  for (int l = threadIdx.x; l < nown; l += kCT) {
    a.x[row0 + l] = sx[l];
    a.r[row0 + l] = sr[l];
    a.p[row0 + l] = sp[l];
  }
  if (lead && !done0) {
    st->iter = iters;
    st->rr = rr;
    st->alpha = alpha_last;
    st->beta = beta_last;
    if (status != kRunning) {
      st->status = status;
      st->done = 1;
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

size_t cluster_smem(int rows) { return sizeof(double) * ((size_t)4 * rows + kSlots + 2 * kCT); }

// Cluster size the device runs with the largest shared-memory footprint (16, else 8); 0 if
// neither.
int cluster_size(int device) {
  static int cs = -1;
  if (cs >= 0) return cs;
  cs = 0;
  int ok = 0;
  if (cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, device) != cudaSuccess || !ok) return cs;
  const size_t smem = cluster_smem(kMaxRows);
  if (cudaFuncSetAttribute(k_cg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return cs;
  cudaFuncSetAttribute(k_cg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_cg_cluster, &cfg) == cudaSuccess && nc > 0) {
      cs = c;
      break;
    }
    cudaGetLastError();
  }
  return cs;
}

// Rows per CTA (a power of two, at least 32) for n rows on C CTAs; 0 if n does not fit.
int rows_per_cta(int64_t n, int C) {
  if (C <= 0) return 0;
  int R = 32;
  while ((int64_t)R * C < n) R *= 2;
  return R <= kMaxRows ? R : 0;
}

}  // namespace

bool persistent_usable(const pk_csr* A, const pk_opts* o) {
  (void)o;
  return rows_per_cta(A->n, cluster_size(A->device)) > 0;
}

pk_status launch_cg_persistent(pk_csr* A, double* x, double* r, double* p, double* ap,
                               cudaStream_t s) {
  (void)ap;
  const int C = cluster_size(A->device);
  const int R = rows_per_cta(A->n, C);
  if (R <= 0) {
    set_error("persistent loop: n too large for one cluster, or no cluster launch");
    return PK_ERR_ARG;
  }
  int lg = 0;
  while ((1 << lg) < R) ++lg;
  ClusterArgs a{A->n, lg, A->rp, A->ci, A->va, x, r, p, A->st};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = cluster_smem(R);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PK_CUDA(cudaLaunchKernelEx(&cfg, k_cg_cluster, a));
  return PK_OK;
}

}  // namespace pk
