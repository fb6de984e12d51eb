// Persistent pipelined GMRES(m) (Alg. 6, Sec. 3.3) on one thread-block cluster, for systems
// small enough that the four launches and grid-wide reductions of a step dominate the solve
// (the latency regime of Sec. 2.1).
//
// One cluster of C CTAs (16 where the device allows it, else 8) runs every cycle and step.
// CTA k owns rows [k R, (k+1) R), R a power of two.  The basis v_0 .. v_m stays in global
// memory (each CTA reads and writes only its own rows, so no other CTA's writes are ever read
// from it); the vector that the SpMV gathers (x at a cycle start, v_{i-1} in step i) is in
// the CTAs' shared memory and read through distributed shared memory; every CTA keeps the
// same copy of R, xi and eta.  A step is the launched form's stages, each ending in a cluster
// barrier after which every CTA adds the C partial sums in rank order (bit-identical scalars,
// uniform decisions):
//   A+B  w = A v_{i-1}; partial <v_j, w>, j = 1 .. i-1 (classical Gram-Schmidt)  -> R_{j,i}
//   C    v_i = w - sum_j R_{j,i} v_j; partial ||v_i||^2            -> R_{i,i}, lucky breakdown
//   D    v_i /= R_{i,i}; partial xi_i = <v_0, v_i>        -> residual estimate, end of cycle
// A cycle starts with r = b - A x (the true residual, convergence test), v_0 = r / rho0, and
// ends with R eta = xi (back substitution, every CTA) and x += rho0 (eta_1 v_0 + sum_{i>=2}
// eta_i v_{i-1}).  Consecutive stages write alternate slot groups, so no CTA overwrites a
// partial that another may still read.  There is no spin-wait; a final cluster barrier keeps
// every CTA's shared memory alive until the last remote read.
#include <algorithm>

#include "pk_cluster.cuh"

namespace pk {

namespace {

constexpr int kGcCT = 512;        // threads per CTA
constexpr int kGcWarps = kGcCT / 32;
constexpr int kGcMaxRows = 4096;  // rows per CTA
constexpr int kGcMax = 64;        // largest restart length
constexpr int kGcLd = kGcMax + 1; // leading dimension of R (and of R in the handle's scratch)
constexpr int kGcSlots = 72;      // partial sums per slot group (up to m - 1 dots)
// A cycle ends once the squared relative residual estimate is at or below this floor (the
// same floor as the launched form and the oracle).
constexpr double kGcEstFloor = 1e-12;

struct GmClusterArgs {
  int32_t n, log_rows, m;
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const double* b;
  double* x;
  double* V;          // basis, column j at V + j * ld
  int64_t ld;
  double* Rout;       // the handle's scratch: R[j * kGcLd + i], then xi (for pk_gmres_cycle_factors)
  double* xiout;
  DevState* st;
};

// cur, w: R doubles each; R: kGcLd^2; xi, eta: kGcLd each; slots: 2 groups; warp partials.
size_t gc_smem(int rows) {
  return sizeof(double) * ((size_t)2 * rows + (size_t)kGcLd * kGcLd + 2 * kGcLd + 2 * kGcSlots + kGcWarps);
}

// Sum of one value over the CTA, valid in thread 0: a fixed xor butterfly per warp, then
// thread 0 adds the warp partials in warp order.  (On GB300 an FP64 operation repeated by
// every thread of the CTA costs the narrow FP64 pipe, so scalar work stays in thread 0.)
__device__ __forceinline__ double gc_block_sum(double v, double* wp) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kGcWarps; ++w) t += wp[w];
  }
  __syncthreads();  // (wp is reused by the next sum)
  return t;
}

// Cluster total of slot s of every CTA (after a cluster barrier), by one warp: lane c reads
// CTA c's value, then a fixed butterfly (every CTA runs the same additions).
__device__ __forceinline__ double gc_warp_total(cg::cluster_group& cl, double* slots, int s) {
  const int lane = threadIdx.x & 31;
  const double v = lane < (int)cl.num_blocks() ? *cl.map_shared_rank(slots + s, lane) : 0.0;
  return warp_sum(v);
}

}  // namespace

__global__ void __launch_bounds__(kGcCT, 1) k_gm_cluster(GmClusterArgs a) {
  extern __shared__ __align__(16) double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int R = 1 << a.log_rows, lg = a.log_rows;
  const int rank = (int)cl.block_rank();
  double* cur = sm;              // the gathered vector: x at a cycle start, then v_{i-1}
  double* sw = sm + R;           // own rows of r, then of w and v_i
  double* Rm = sm + 2 * R;       // R_{j,i} at j * kGcLd + i (the same in every CTA)
  double* xi = Rm + kGcLd * kGcLd;
  double* eta = xi + kGcLd;
  double* slots = eta + kGcLd;   // two groups of kGcSlots partial sums
  double* wp = slots + 2 * kGcSlots;
  __shared__ double tot[2];      // cluster totals
  __shared__ double bc[2];       // scalars broadcast by thread 0
  __shared__ int bdec;           // decision broadcast by thread 0
  const int row0 = rank * R, nown = max(0, min(a.n - row0, R));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DevState* st = a.st;
  const bool t0 = threadIdx.x == 0, lead = rank == 0 && t0;
  const int maxit = __ldcg(&st->maxit), m = a.m;
  const double tol = __ldcg(&st->thr2);  // (the state holds tol until the first residual)
  double* const trace = st->trace;
  const int trace_cap = st->trace_cap;
  // scalar state, meaningful in thread 0 (the same in every CTA); counters in every thread
  double bb = 0.0, thr2 = 0.0, rr = 0.0, sumxi2 = 0.0, rho0 = 0.0;
  int zero_x = 0, status = kRunning;
  int total = 0, cycle = 0, kprev = -1;
  int g = 0;  // slot group of the next stage
  auto vcol = [&](int j) { return a.V + (size_t)j * a.ld + row0; };
  for (;;) {
    // cycle start: r = b - A x (the true residual), <r, r> and <b, b>
    for (int l = threadIdx.x; l < nown; l += kGcCT) cur[l] = a.x[row0 + l];
    cl.sync();
    double p0 = 0.0, p1 = 0.0;
    for (int l = threadIdx.x; l < nown; l += kGcCT) {
      const int row = row0 + l;
      const double bi = __ldg(a.b + row);
      const double ri = bi - cluster_row(cl, a.ci, a.va, cur, lg, __ldg(a.rp + row), __ldg(a.rp + row + 1));
      sw[l] = ri;
      p0 = fma(ri, ri, p0);
      p1 = fma(bi, bi, p1);
    }
    p0 = gc_block_sum(p0, wp);
    p1 = gc_block_sum(p1, wp);
    double* sg = slots + g * kGcSlots;
    g ^= 1;
    if (t0) {
      sg[0] = p0;
      sg[1] = p1;
    }
    cl.sync();  // (also: every CTA has finished gathering x)
    if (warp < 2) {
      const double t = gc_warp_total(cl, sg, warp);
      if (lane == 0) tot[warp] = t;
    }
    __syncthreads();
    if (t0) {
      rr = tot[0];
      if (cycle == 0) {
        bb = tot[1];
        thr2 = tol * tol * bb;
      }
      int sts = kRunning;
      if (!isfinite(rr) || !isfinite(bb)) sts = PK_ERR_NAN;
      else if (bb == 0.0) {
        zero_x = 1;
        rr = 0.0;
        sts = PK_OK;
      } else if (rr <= thr2) sts = PK_OK;
      else if (total >= maxit) sts = PK_NOT_CONVERGED;
      else if (cycle > 0 && kprev == 0) sts = PK_BREAKDOWN;
      bdec = sts;
      if (sts == kRunning) {
        rho0 = sqrt(rr);
        bc[0] = rho0;
        bc[1] = 1.0 / rho0;
        sumxi2 = 0.0;
      }
    }
    __syncthreads();
    status = bdec;
    if (status != kRunning) break;
    const double rho = bc[0], inv0 = bc[1];
    for (int l = threadIdx.x; l < nown; l += kGcCT) {
      const double v0 = sw[l] * inv0;
      vcol(0)[l] = v0;
      cur[l] = v0;
    }
    int k = 0;
    cl.sync();  // v_0 in place before the first gather
    for (int i = 1; i <= m; ++i) {
      if (total >= maxit) break;
      // A: w = A v_{i-1}
      for (int l = threadIdx.x; l < nown; l += kGcCT) {
        const int row = row0 + l;
        sw[l] = cluster_row(cl, a.ci, a.va, cur, lg, __ldg(a.rp + row), __ldg(a.rp + row + 1));
      }
      __syncthreads();
      // B: partial <v_j, w>, j = 1 .. i-1, one warp per j (four interleaved row chains)
      sg = slots + g * kGcSlots;
      g ^= 1;
      for (int j = 1 + warp; j <= i - 1; j += kGcWarps) {
        const double* vj = vcol(j);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int l = lane;
        for (; l + 96 < nown; l += 128) {
          s0 = fma(vj[l], sw[l], s0);
          s1 = fma(vj[l + 32], sw[l + 32], s1);
          s2 = fma(vj[l + 64], sw[l + 64], s2);
          s3 = fma(vj[l + 96], sw[l + 96], s3);
        }
        for (; l < nown; l += 32) s0 = fma(vj[l], sw[l], s0);
        const double s = warp_sum((s0 + s1) + (s2 + s3));
        if (lane == 0) sg[j] = s;
      }
      cl.sync();  // (also: every CTA has finished gathering v_{i-1})
      for (int j = 1 + warp; j <= i - 1; j += kGcWarps) {
        const double t = gc_warp_total(cl, sg, j);
        if (lane == 0) Rm[j * kGcLd + i] = t;
      }
      __syncthreads();
      // C: v_i = w - sum_j R_{j,i} v_j (j = 1, 2, ... in order), partial ||v_i||^2; the basis
      // values of a row are loaded eight at a time (their loads in flight together)
      double p = 0.0;
      for (int l = threadIdx.x; l < nown; l += kGcCT) {
        double w = sw[l];
        int j = 1;
        for (; j + 8 <= i; j += 8) {
          double vv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) vv[q] = vcol(j + q)[l];
#pragma unroll
          for (int q = 0; q < 8; ++q) w = fma(-Rm[(j + q) * kGcLd + i], vv[q], w);
        }
        for (; j <= i - 1; ++j) w = fma(-Rm[j * kGcLd + i], vcol(j)[l], w);
        sw[l] = w;
        p = fma(w, w, p);
      }
      p = gc_block_sum(p, wp);
      sg = slots + g * kGcSlots;
      g ^= 1;
      if (t0) sg[0] = p;
      cl.sync();
      if (warp == 0) {
        const double t = gc_warp_total(cl, sg, 0);
        if (lane == 0) tot[0] = t;
      }
      __syncthreads();
      if (t0) {
        // R_{i,i} = ||v_i||, the lucky-breakdown test against ||A v_{i-1}||
        const double nrm2 = tot[0];
        double col2 = nrm2;
        for (int j = 1; j <= i - 1; ++j) col2 += Rm[j * kGcLd + i] * Rm[j * kGcLd + i];
        const double rii = sqrt(nrm2);
        int dec = 0;
        if (!isfinite(rii)) dec = 2;
        else if (rii == 0.0 || rii <= 1e-14 * sqrt(col2)) dec = 1;  // the cycle ends before step i
        else {
          Rm[i * kGcLd + i] = rii;
          bc[1] = 1.0 / rii;
        }
        bdec = dec;
      }
      __syncthreads();
      if (bdec == 2) {
        status = PK_ERR_NAN;
        break;
      }
      if (bdec == 1) break;
      const double inv = bc[1];
      // D: v_i /= R_{i,i}; partial xi_i = <v_0, v_i>
      p = 0.0;
      for (int l = threadIdx.x; l < nown; l += kGcCT) {
        const double v = sw[l] * inv;
        vcol(i)[l] = v;
        cur[l] = v;
        p = fma(vcol(0)[l], v, p);
      }
      p = gc_block_sum(p, wp);
      sg = slots + g * kGcSlots;
      g ^= 1;
      if (t0) sg[0] = p;
      cl.sync();  // (also: v_i is in place for the next gather)
      if (warp == 0) {
        const double t = gc_warp_total(cl, sg, 0);
        if (lane == 0) tot[0] = t;
      }
      __syncthreads();
      total += 1;
      k = i;
      if (t0) {
        // the residual estimate rho0 sqrt(1 - sum xi^2) and the end of the cycle
        const double xii = tot[0];
        xi[i] = xii;
        sumxi2 += xii * xii;
        double rel2 = 1.0 - sumxi2;
        if (rel2 < 0.0) rel2 = 0.0;
        const double est = rho0 * sqrt(rel2);
        if (lead) {
          const int step = total - 1;
          if (trace && step < trace_cap) {
            trace[(size_t)step * 4 + 0] = i >= 2 ? Rm[(i - 1) * kGcLd + i] : 0.0;
            trace[(size_t)step * 4 + 1] = Rm[i * kGcLd + i];
            trace[(size_t)step * 4 + 2] = xii;
            trace[(size_t)step * 4 + 3] = est;
          }
          for (int j = 1; j <= i; ++j) a.Rout[j * kGcLd + i] = Rm[j * kGcLd + i];
          a.xiout[i] = xii;
        }
        int dec = 0;
        if (!isfinite(xii)) dec = 2;
        else if (est * est <= thr2 || rel2 <= kGcEstFloor || i >= m || total >= maxit) dec = 1;
        bdec = dec;
      }
      __syncthreads();
      if (bdec == 2) {
        status = PK_ERR_NAN;
        break;
      }
      if (bdec == 1) break;
    }
    if (status != kRunning) break;
    // cycle end: R eta = xi (warp 0 of every CTA, the same additions everywhere), then
    // x += rho0 (eta_1 v_0 + sum_{i >= 2} eta_i v_{i-1})
    kprev = k;
    __syncthreads();
    if (k > 0) {
      if (warp == 0) {
        for (int ii = k; ii >= 1; --ii) {
          double s = 0.0;
          for (int j = ii + 1 + lane; j <= k; j += 32) s = fma(Rm[ii * kGcLd + j], eta[j], s);
          s = warp_sum(s);
          if (lane == 0) eta[ii] = (xi[ii] - s) / Rm[ii * kGcLd + ii];
          __syncwarp();
        }
      }
      __syncthreads();
      for (int l = threadIdx.x; l < nown; l += kGcCT) {
        double acc = 0.0;
        int ii = 1;
        for (; ii + 8 <= k + 1; ii += 8) {
          double vv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) vv[q] = vcol(ii + q - 1)[l];
#pragma unroll
          for (int q = 0; q < 8; ++q) acc = fma(eta[ii + q], vv[q], acc);
        }
        for (; ii <= k; ++ii) acc = fma(eta[ii], vcol(ii - 1)[l], acc);
        a.x[row0 + l] = fma(rho, acc, a.x[row0 + l]);
      }
    }
    cycle += 1;
  }
  if (lead) {
    st->iter = total;
    st->rr = rr;
    st->bb = bb;
    st->thr2 = thr2;
    st->gm_cycle = cycle;
    st->zero_x = zero_x;
    st->status = status;
    st->done = 1;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

namespace {

// Cluster size the device runs with the largest shared-memory footprint (16, else 8); 0 if
// neither.
int gc_cluster_size() {
  static int cs = -1;
  if (cs >= 0) return cs;
  cs = 0;
  int dev = 0, ok = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !ok) {
    cudaGetLastError();
    return cs;
  }
  const size_t smem = gc_smem(kGcMaxRows);
  if (cudaFuncSetAttribute(k_gm_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return cs;
  }
  cudaFuncSetAttribute(k_gm_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kGcCT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_gm_cluster, &cfg) == cudaSuccess && nc > 0) {
      cs = c;
      break;
    }
    cudaGetLastError();
  }
  return cs;
}

int gc_rows_per_cta(int64_t n, int C) {
  if (C <= 0) return 0;
  int R = 32;
  while ((int64_t)R * C < n) R *= 2;
  return R <= kGcMaxRows ? R : 0;
}

}  // namespace

bool gmres_persistent_usable(const pk_csr* A, int m) {
  return m >= 1 && m <= kGcMax && gc_rows_per_cta(A->n, gc_cluster_size()) > 0;
}

// The whole restarted pipelined GMRES(m) in one cluster launch.  x: the iterate (device, in
// place); V: the handle's basis (m + 1 columns of ld); Rout, xiout: where the latest cycle's
// R and xi go (the layout pk_gmres_cycle_factors reads).
pk_status launch_gmres_persistent(pk_csr* A, const double* b, double* x, int m, double* V, int64_t ld,
                                  double* Rout, double* xiout, cudaStream_t s) {
  const int C = gc_cluster_size();
  const int R = gc_rows_per_cta(A->n, C);
  if (R <= 0 || m < 1 || m > kGcMax) {
    set_error("persistent GMRES: n too large for one cluster, restart outside 1..64, or no cluster launch");
    return PK_ERR_ARG;
  }
  int lg = 0;
  while ((1 << lg) < R) ++lg;
  GmClusterArgs a{A->n, lg, m, A->rp, A->ci, A->va, b, x, V, ld, Rout, xiout, A->st};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kGcCT);
  cfg.dynamicSmemBytes = gc_smem(R);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PK_CUDA(cudaLaunchKernelEx(&cfg, k_gm_cluster, a));
  return PK_OK;
}

}  // namespace pk
