// Persistent pipelined BiCGStab (Alg. 4, Sec. 3.2) on one thread-block cluster, for systems
// small enough that the launches and grid-wide reductions of the four fused kernels per
// iteration dominate the solve (the latency regime of Sec. 2.1).
//
// One cluster of C CTAs (16 where the device allows it, else 8) runs every iteration.  CTA k
// owns rows [k R, (k+1) R), R a power of two; p, s, r, Ap, As and r0* of its rows live in its
// shared memory for the whole solve (x stays in global memory: each element is read and
// written once per iteration by the thread that owns it).  An iteration is the launched
// form's four fused phases, each ending in a hardware cluster barrier and a cluster total
// added in rank order by every CTA (bit-identical scalars, uniform decisions):
//   1  Ap = A p (p gathered through distributed shared memory), <Ap, r0*>    -> alpha
//   2  s = r - alpha Ap, <s, s>                                              -> early exit
//   3  As = A s (s gathered likewise), <As, s>, <As, As>, <As, r0*>         -> omega, beta
//   4  x += alpha p + omega s, r = s - omega As, p = r + beta (p - omega Ap),
//      <r, r0*>, <r, r>                                                      -> convergence
// Phases alternate between two slot groups, so a phase never overwrites slots that another
// CTA may still be reading from the phase before (the barrier in between orders them).
// There is no spin-wait; a final cluster barrier keeps every CTA's shared memory alive until
// the last remote read.
#include <algorithm>

#include "pk_cluster.cuh"

namespace pk {

namespace {

constexpr int kBiCT = 512;        // threads per CTA
constexpr int kBiMaxRows = 4096;  // rows per CTA held in shared memory
constexpr int kBiSlots = 8;       // two groups of four block sums

struct BiClusterArgs {
  int32_t n;
  int32_t log_rows;  // rows per CTA = 1 << log_rows
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  double* x;
  const double* r;    // r0 (from the setup kernel)
  const double* r0s;  // r0*
  DevState* st;
};

// p, s, r, Ap, As, r0* (rows each), the slots and the block-sum buffer (4 values x kBiCT).
size_t bi_cluster_smem(int rows) { return sizeof(double) * ((size_t)6 * rows + kBiSlots + 4 * kBiCT); }

}  // namespace

__global__ void __launch_bounds__(kBiCT, 1) k_bi_cluster(BiClusterArgs a) {
  extern __shared__ __align__(16) double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int R = 1 << a.log_rows, lg = a.log_rows;
  const int rank = (int)cl.block_rank();
  double* sp = sm;           // p (gathered remotely in phase 1)
  double* ss = sm + R;       // s (gathered remotely in phase 3)
  double* sr = sm + 2 * R;
  double* sap = sm + 3 * R;  // Ap
  double* sas = sm + 4 * R;  // As
  double* sz = sm + 5 * R;   // r0*
  double* slots = sm + 6 * R;
  double* buf = slots + kBiSlots;
  const int row0 = rank * R;
  const int nown = max(0, min(a.n - row0, R));
  DevState* st = a.st;
  const bool done0 = __ldcg(&st->done) != 0;  // the same flag in every CTA
  for (int l = threadIdx.x; l < nown; l += kBiCT) {
    const double r0 = a.r[row0 + l];
    sr[l] = r0;
    sp[l] = r0;  // p0 = r0
    sz[l] = a.r0s[row0 + l];
  }
  const double thr2 = __ldcg(&st->thr2);
  const int maxit = __ldcg(&st->maxit);
  double rr = __ldcg(&st->rr), rr0s = __ldcg(&st->s[0]);
  const bool lead = rank == 0 && threadIdx.x == 0;
  double* const trace = st->trace;
  const int trace_cap = st->trace_cap;
  double alpha = 0.0, beta = 0.0, omega = 0.0;
  int iters = 0;
  int status = kRunning;
  __shared__ double sc[3];  // alpha | omega, beta
  __shared__ int scs;       // decision of thread 0 (kRunning: continue)
  cl.sync();  // every CTA's p is in place before the first remote gather
  for (int i = 0; !done0; ++i) {
    // phase 1: Ap_i and <Ap_i, r0*> -> alpha_i
    double w[1] = {0.0};
    for (int l = threadIdx.x; l < nown; l += kBiCT) {
      const int row = row0 + l;
      const double y = cluster_row(cl, a.ci, a.va, sp, lg, __ldg(a.rp + row), __ldg(a.rp + row + 1));
      sap[l] = y;
      w[0] = fma(y, sz[l], w[0]);
    }
    double t1[1];
    cluster_block_sum<kBiCT, 1>(w, buf, t1);
    if (threadIdx.x == 0) slots[0] = t1[0];
    cl.sync();
    cluster_total<1>(cl, slots, 0, t1);
    const double apr0s = t1[0];
    if (threadIdx.x == 0) {
      int sts = kRunning;
      double al = 0.0;
      if (!isfinite(apr0s)) sts = PK_ERR_NAN;
      else if (apr0s == 0.0 || rr0s == 0.0) sts = PK_BREAKDOWN;
      else {
        al = rr0s / apr0s;
        if (lead && trace && i < trace_cap) trace[(size_t)i * 4 + 0] = al;
      }
      sc[0] = al;
      scs = sts;
    }
    __syncthreads();
    if (scs != kRunning) { status = scs; break; }
    alpha = sc[0];
    // phase 2: s_i = r_i - alpha_i Ap_i and <s_i, s_i>
    w[0] = 0.0;
    for (int l = threadIdx.x; l < nown; l += kBiCT) {
      const double sv = fma(-alpha, sap[l], sr[l]);
      ss[l] = sv;
      w[0] = fma(sv, sv, w[0]);
    }
    cluster_block_sum<kBiCT, 1>(w, buf, t1);
    if (threadIdx.x == 0) slots[4] = t1[0];
    cl.sync();  // (also: every CTA's s is in place for phase 3)
    cluster_total<1>(cl, slots, 4, t1);
    const double sn = t1[0];
    if (!isfinite(sn)) { status = PK_ERR_NAN; break; }
    if (sn <= thr2) {  // ||s|| small: x += alpha p ends the solve (the early exit of Alg. 3)
      for (int l = threadIdx.x; l < nown; l += kBiCT) a.x[row0 + l] = fma(alpha, sp[l], a.x[row0 + l]);
      if (lead && trace && i < trace_cap) trace[(size_t)i * 4 + 3] = sn;
      rr = sn;
      iters = i + 1;
      status = PK_OK;
      break;
    }
    // phase 3: As_i and <As_i, s_i>, <As_i, As_i>, <As_i, r0*> -> omega_i, beta_i
    double v[3] = {0.0, 0.0, 0.0};
    for (int l = threadIdx.x; l < nown; l += kBiCT) {
      const int row = row0 + l;
      const double y = cluster_row(cl, a.ci, a.va, ss, lg, __ldg(a.rp + row), __ldg(a.rp + row + 1));
      sas[l] = y;
      v[0] = fma(y, ss[l], v[0]);
      v[1] = fma(y, y, v[1]);
      v[2] = fma(y, sz[l], v[2]);
    }
    double t3[3];
    cluster_block_sum<kBiCT, 3>(v, buf, t3);
    if (threadIdx.x == 0) {
      slots[0] = t3[0];
      slots[1] = t3[1];
      slots[2] = t3[2];
    }
    cl.sync();
    cluster_total<3>(cl, slots, 0, t3);
    if (threadIdx.x == 0) {
      int sts = kRunning;
      double om = 0.0, be = 0.0;
      if (!isfinite(t3[0]) || !isfinite(t3[1]) || !isfinite(t3[2])) sts = PK_ERR_NAN;
      else if (t3[1] == 0.0) sts = PK_BREAKDOWN;
      else {
        om = t3[0] / t3[1];
        be = -t3[2] / apr0s;
        if (lead && trace && i < trace_cap) {
          trace[(size_t)i * 4 + 1] = be;
          trace[(size_t)i * 4 + 2] = om;
        }
      }
      sc[1] = om;
      sc[2] = be;
      scs = sts;
    }
    __syncthreads();
    if (scs != kRunning) { status = scs; break; }
    omega = sc[1];
    beta = sc[2];
    // phase 4: x, r, p and <r_{i+1}, r0*>, <r_{i+1}, r_{i+1}>.  No CTA gathers p or s again
    // before the next barrier, so both are updated in place.
    double u[2] = {0.0, 0.0};
    for (int l = threadIdx.x; l < nown; l += kBiCT) {
      const int row = row0 + l;
      const double pk = sp[l], sk = ss[l];
      a.x[row] = fma(omega, sk, fma(alpha, pk, a.x[row]));
      const double rn = fma(-omega, sas[l], sk);
      sr[l] = rn;
      sp[l] = fma(beta, fma(-omega, sap[l], pk), rn);
      u[0] = fma(rn, sz[l], u[0]);
      u[1] = fma(rn, rn, u[1]);
    }
    double t2[2];
    cluster_block_sum<kBiCT, 2>(u, buf, t2);
    if (threadIdx.x == 0) {
      slots[4] = t2[0];
      slots[5] = t2[1];
    }
    cl.sync();
    cluster_total<2>(cl, slots, 4, t2);
    rr0s = t2[0];
    rr = t2[1];
    iters = i + 1;
    if (lead && trace && i < trace_cap) trace[(size_t)i * 4 + 3] = rr;
    if (!isfinite(rr) || !isfinite(rr0s)) { status = PK_ERR_NAN; break; }
    if (rr <= thr2) { status = PK_OK; break; }
    if (i + 1 >= maxit) { status = PK_NOT_CONVERGED; break; }
  }
  if (lead && !done0) {
    st->iter = iters;
    st->rr = rr;
    st->s[0] = rr0s;
    st->alpha = alpha;
    st->beta = beta;
    st->omega = omega;
    if (status != kRunning) {
      st->status = status;
      st->done = 1;
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

namespace {

// Cluster size the device runs with the largest shared-memory footprint (16, else 8); 0 if
// neither.
int bi_cluster_size() {
  static int cs = -1;
  if (cs >= 0) return cs;
  cs = 0;
  int dev = 0, ok = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !ok) {
    cudaGetLastError();
    return cs;
  }
  const size_t smem = bi_cluster_smem(kBiMaxRows);
  if (cudaFuncSetAttribute(k_bi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return cs;
  }
  cudaFuncSetAttribute(k_bi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kBiCT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_bi_cluster, &cfg) == cudaSuccess && nc > 0) {
      cs = c;
      break;
    }
    cudaGetLastError();
  }
  return cs;
}

// Rows per CTA (a power of two, at least 32) for n rows on C CTAs; 0 if n does not fit.
int bi_rows_per_cta(int64_t n, int C) {
  if (C <= 0) return 0;
  int R = 32;
  while ((int64_t)R * C < n) R *= 2;
  return R <= kBiMaxRows ? R : 0;
}

}  // namespace

bool bicgstab_persistent_usable(const pk_csr* A) { return bi_rows_per_cta(A->n, bi_cluster_size()) > 0; }

// The whole pipelined BiCGStab loop in one cluster launch, after the setup kernel has formed
// r0 (in r), r0* and the state's <r0,r0>, <r0,r0*>, thresholds and done flag.
pk_status launch_bicgstab_persistent(pk_csr* A, double* x, const double* r, const double* r0s, cudaStream_t s) {
  const int C = bi_cluster_size();
  const int R = bi_rows_per_cta(A->n, C);
  if (R <= 0) {
    set_error("persistent BiCGStab: n too large for one cluster, or no cluster launch");
    return PK_ERR_ARG;
  }
  int lg = 0;
  while ((1 << lg) < R) ++lg;
  BiClusterArgs a{A->n, lg, A->rp, A->ci, A->va, x, r, r0s, A->st};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kBiCT);
  cfg.dynamicSmemBytes = bi_cluster_smem(R);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PK_CUDA(cudaLaunchKernelEx(&cfg, k_bi_cluster, a));
  return PK_OK;
}

}  // namespace pk
