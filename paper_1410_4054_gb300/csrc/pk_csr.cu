// CSR handle, schedule, work memory, and the plain (unfused) kernels.
//
// pk_csr_create validates and copies the matrix and splits its rows into contiguous,
// nnz-balanced ranges, one per thread block of the persistent grid used by every fused
// kernel (the first reduction stage of Sec. 2.2 is one partial sum per block).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pk_guard.cuh"
#include "pk_tile.cuh"

namespace pk {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

pk_status host_failure(bool oom) noexcept {
  try {
    g_last_error = oom ? "host memory allocation failed" : "unexpected host-side exception";
  } catch (...) {  // no memory even for the message: keep the previous one
  }
  return oom ? PK_ERR_OOM : PK_ERR_ARG;
}

pk_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PK_ERR_OOM : PK_ERR_CUDA;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

pk_status work_vec(pk_csr* A, int id, double** out) {
  if (id < 0 || id >= 16) return PK_ERR_ARG;
  if (!A->vec[id]) {
    // 64 doubles of padding so vector loads of a ragged tail stay inside the allocation
    PK_CUDA(cudaMalloc(&A->vec[id], sizeof(double) * ((size_t)A->n + 64)));
    PK_CUDA(cudaMemset(A->vec[id], 0, sizeof(double) * ((size_t)A->n + 64)));
    A->vec_len[id] = A->n;
  }
  *out = A->vec[id];
  return PK_OK;
}

pk_status ensure_state(pk_csr* A) {
  if (!A->st) {
    PK_CUDA(cudaMalloc(&A->st, sizeof(DevState)));
    PK_CUDA(cudaMemset(A->st, 0, sizeof(DevState)));
    PK_CUDA(cudaMallocHost(&A->st_host, sizeof(DevState)));
    memset(A->st_host, 0, sizeof(DevState));
    int sms = 1;
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
    A->partial_cap = std::max(A->grid, sms * kMaxGridPerSm);
    PK_CUDA(cudaMalloc(&A->partials, sizeof(double) * (size_t)kMaxDots * A->partial_cap));
    PK_CUDA(cudaMalloc(&A->small, sizeof(double) * 8192));
    PK_CUDA(cudaMemset(A->small, 0, sizeof(double) * 8192));
  }
  return PK_OK;
}

pk_status stage_in(pk_csr* A, const double* b, double* x, int slot_b, int slot_x,
                   cudaStream_t s, VecStage* v) {
  v->x_user = x;
  if (is_device_ptr(b)) {
    v->b_dev = b;
  } else {
    double* d;
    pk_status st = work_vec(A, slot_b, &d);
    if (st) return st;
    PK_CUDA(cudaMemcpyAsync(d, b, sizeof(double) * A->n, cudaMemcpyHostToDevice, s));
    v->b_dev = d;
  }
  if (is_device_ptr(x)) {
    v->x_dev = x;
    v->x_host = false;
  } else {
    double* d;
    pk_status st = work_vec(A, slot_x, &d);
    if (st) return st;
    PK_CUDA(cudaMemcpyAsync(d, x, sizeof(double) * A->n, cudaMemcpyHostToDevice, s));
    v->x_dev = d;
    v->x_host = true;
  }
  return PK_OK;
}

pk_status stage_out(pk_csr* A, const VecStage& v, cudaStream_t s) {
  if (v.x_host)
    PK_CUDA(cudaMemcpyAsync(v.x_user, v.x_dev, sizeof(double) * A->n, cudaMemcpyDeviceToHost, s));
  return PK_OK;
}

pk_status state_init(pk_csr* A, const pk_opts* o, cudaStream_t s) {
  pk_status e = ensure_state(A);
  if (e) return e;
  DevState* h = A->st_host;
  memset(h, 0, sizeof(DevState));
  h->maxit = o->maxit;
  h->status = kRunning;
  h->trace = o->trace_cap > 0 ? o->trace : nullptr;
  h->trace_cap = o->trace_cap > 0 ? o->trace_cap : 0;
  h->thr2 = o->tol;  // the setup kernel turns tol into tol^2 <b,b>
  h->wait_ns = o->wait_ns > 0 ? (unsigned long long)o->wait_ns : 2000000000ull;
  h->stall_test = (o->flags & PK_FLAG_TEST_STALL) ? 1 : 0;
  PK_CUDA(cudaMemcpyAsync(A->st, h, sizeof(DevState), cudaMemcpyHostToDevice, s));
  return PK_OK;
}

pk_status state_read(pk_csr* A, cudaStream_t s) {
  PK_CUDA(cudaMemcpyAsync(A->st_host, A->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  PK_CUDA(cudaStreamSynchronize(s));
  return PK_OK;
}

pk_status Timer::begin(int slot_id) {
  if (!on) return PK_OK;
  if (used + 2 > 64) {
    pk_status e = flush();
    if (e) return e;
  }
  for (int k = A->ev_count; k < used + 2; ++k) {
    PK_CUDA(cudaEventCreate(&A->ev_pool[k]));
    A->ev_count = k + 1;
  }
  slot[used / 2] = slot_id;
  PK_CUDA(cudaEventRecord(A->ev_pool[used], s));
  return PK_OK;
}

pk_status Timer::end() {
  if (!on) return PK_OK;
  PK_CUDA(cudaEventRecord(A->ev_pool[used + 1], s));
  used += 2;
  return PK_OK;
}

pk_status Timer::flush() {
  if (!on || used == 0) return PK_OK;
  PK_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < used; k += 2) {
    float t = 0.f;
    PK_CUDA(cudaEventElapsedTime(&t, A->ev_pool[k], A->ev_pool[k + 1]));
    ms[slot[k / 2]] += t;
    count[slot[k / 2]] += 1;
  }
  used = 0;
  return PK_OK;
}

RowArgs row_args(const pk_csr* A) {
  RowArgs a;
  a.n = A->n;
  a.rp = A->rp;
  a.ci = A->ci;
  a.va = A->va;
  a.rowblk = A->rowblk;
  a.partials = A->partials;
  a.st = A->st;
  return a;
}

// ------------------------------------------------------------------ plain kernels

// y = A x (no reductions): the unfused SpMV of Sec. 2.2, step 1.
__global__ void __launch_bounds__(kBlock) k_spmv(RowArgs a, const double* __restrict__ x,
                                                 double* __restrict__ y) {
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) y[row] = csr_row(a, x, row);
}

// *out = <x, y> with the deterministic two-stage reduction (steps 2-3 of Sec. 2.2).
__global__ void __launch_bounds__(kBlock) k_dot_store(RowArgs a, const double* __restrict__ x,
                                                      const double* __restrict__ y, double* out) {
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) v[0] = fma(x[row], y[row], v[0]);
  block_partials<1>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      *out = t[0];
      a.st->counter = 0;
    }
  }
}

// Fused q = A p and <p, q> (Sec. 2.2 fused kernel): first stage in the SpMV loop, second
// stage in the last block.
__global__ void __launch_bounds__(kBlock) k_spmv_dot(RowArgs a, const double* __restrict__ p,
                                                     double* __restrict__ q, double* out) {
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double s = csr_row(a, p, row);
    q[row] = s;
    v[0] = fma(__ldg(p + row), s, v[0]);
  }
  block_partials<1>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      *out = t[0];
      a.st->counter = 0;
    }
  }
}

// tmp = b - A x and out2 = <tmp, tmp> (true residual at exit).
__global__ void __launch_bounds__(kBlock) k_true_residual(RowArgs a, const double* __restrict__ b,
                                                          const double* __restrict__ x,
                                                          double* out2) {
  const int r0 = a.rowblk[blockIdx.x], r1 = a.rowblk[blockIdx.x + 1];
  double v[1] = {0.0};
  for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const double r = b[row] - csr_row(a, x, row);
    v[0] = fma(r, r, v[0]);
  }
  block_partials<1>(v, a.partials);
  if (arrive_last(&a.st->counter)) {
    double t[1];
    final_sums<1>(a.partials, t);
    if (threadIdx.x == 0) {
      *out2 = t[0];
      a.st->counter = 0;
    }
  }
}

void launch_spmv(const pk_csr* A, const double* x, double* y, cudaStream_t s) {
  k_spmv<<<A->grid, kBlock, 0, s>>>(row_args(A), x, y);
}

void launch_dot_store(const pk_csr* A, const double* x, const double* y, double* out,
                      cudaStream_t s) {
  k_dot_store<<<A->grid, kBlock, 0, s>>>(row_args(A), x, y, out);
}

void launch_true_residual(pk_csr* A, const double* b, const double* x, double* tmp, double* out2,
                          cudaStream_t s) {
  (void)tmp;
  k_true_residual<<<A->grid, kBlock, 0, s>>>(row_args(A), b, x, out2);
}

pk_status check_opts(const pk_csr* A, const double* b, double* x, const pk_opts* o,
                            pk_info* info) {
  if (!A || !o || !info) { set_error("NULL handle, opts or info"); return PK_ERR_ARG; }
  if (A->n > 0 && (!b || !x)) { set_error("NULL b or x"); return PK_ERR_ARG; }
  if (!(o->tol >= 0.0) || o->maxit < 0) { set_error("tol must be >= 0 and maxit >= 0"); return PK_ERR_ARG; }
  if (o->trace_cap > 0 && !o->trace) { set_error("trace_cap > 0 needs a trace array"); return PK_ERR_ARG; }
  if (o->loop < PK_LOOP_GRAPH || o->loop > PK_LOOP_RESIDENT) { set_error("bad loop mode"); return PK_ERR_ARG; }
  if (o->wait_ns < 0) { set_error("wait_ns must be >= 0"); return PK_ERR_ARG; }
  return PK_OK;
}

pk_status finish_info(pk_csr* A, const pk_opts* o, pk_info* info, cudaStream_t s,
                      const VecStage& v, cudaEvent_t e0, cudaEvent_t e1, int launches) {
  pk_status e;
  double* res2 = A->small + 8000;
  if (o->flags & PK_FLAG_TRUE_RES) {
    launch_true_residual(A, v.b_dev, v.x_dev, nullptr, res2, s);
    PK_CUDA(cudaGetLastError());
    launches += 1;
  }
  PK_CUDA(cudaEventRecord(e1, s));
  if ((e = stage_out(A, v, s))) return e;
  if ((e = state_read(A, s))) return e;
  const DevState* h = A->st_host;
  info->iters = h->iter;
  info->status = h->status == kRunning ? PK_NOT_CONVERGED : h->status;
  info->launches = launches;
  if (h->timeout) info->status = PK_TIMEOUT;
  info->rel_res_est = h->bb > 0 ? std::sqrt(std::max(h->rr, 0.0) / h->bb) : 0.0;
  info->rel_res_true = -1.0;
  if (o->flags & PK_FLAG_TRUE_RES) {
    double r2 = 0;
    PK_CUDA(cudaMemcpy(&r2, res2, sizeof(double), cudaMemcpyDeviceToHost));
    info->rel_res_true = h->bb > 0 ? std::sqrt(r2 / h->bb) : 0.0;
  }
  float ms = 0.f;
  PK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  info->solve_ms = ms;
  return PK_OK;
}

}  // namespace pk

using namespace pk;

// The launch schedule of a CSR matrix, host only (pk_csr_create and pk_csr_plan): the row
// ranges of the persistent grid, the tile list of the bulk-copy engine with each tile's row
// schedule, and the tile counts by schedule.
struct CsrPlan {
  int grid = 1, grid_tma = 1, grid_stream = 1, ntiles = 0, tma_ok = 1;
  std::vector<int32_t> rb, tile_row, blk_tile, tile_z0;
  std::vector<int8_t> tile_grp;
  std::vector<int16_t> tile_perm;
  int32_t tiles_thread = 0, tiles_long = 0, tiles_group = 0;
};

static void build_plan(int64_t n, int64_t nnz, const std::vector<int32_t>& rp, int sms, CsrPlan& P) {
  // persistent grid: up to kMaxGridPerSm blocks per SM, at least kBlock rows per block
  const int64_t gmax = (int64_t)sms * kMaxGridPerSm;
  P.grid = (int)std::max<int64_t>(1, std::min<int64_t>(gmax, (n + kBlock - 1) / kBlock));
  // nnz-balanced contiguous row ranges: weight of a row = its nonzeros + 2
  P.rb.assign(P.grid + 1, 0);
  auto& rb = P.rb;
  const double wtot = (double)nnz + 2.0 * (double)n;
  rb[0] = 0;
  for (int b = 1; b < P.grid; ++b) {
    const double target = wtot * b / P.grid;
    int64_t lo = rb[b - 1], hi = n;  // first row with rp[row] + 2 row >= target
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if ((double)rp[mid] + 2.0 * (double)mid < target) lo = mid + 1; else hi = mid;
    }
    int64_t r = (lo / 32) * 32;  // warp-aligned boundaries
    rb[b] = (int32_t)std::max<int64_t>(r, rb[b - 1]);
  }
  rb[P.grid] = (int32_t)n;

  // warp-specialised CSR tiles: 2 blocks per SM, nnz-balanced block ranges, tiles of at most
  // kTileRows rows and kTileNnz nonzeros
  auto& tile_row = P.tile_row;
  auto& blk_tile = P.blk_tile;
  auto& tile_z0 = P.tile_z0;
  P.tma_ok = 1;
  // at least one tile per block where the matrix has that many: tiles end at kTileRows rows or
  // kTileNnz nonzeros, whichever comes first
  P.grid_tma = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sms * 2, std::max<int64_t>((n + kTileRows - 1) / kTileRows,
                                                               ((int64_t)nnz + kTileNnz - 1) / kTileNnz)));
  {
    const int Gt = P.grid_tma;
    std::vector<int32_t> tb(Gt + 1);
    tb[0] = 0;
    for (int b = 1; b < Gt; ++b) {
      const double target = wtot * b / Gt;
      int64_t lo = tb[b - 1], hi = n;
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if ((double)rp[mid] + 2.0 * (double)mid < target) lo = mid + 1; else hi = mid;
      }
      tb[b] = (int32_t)std::max<int64_t>((lo / 32) * 32, tb[b - 1]);
    }
    tb[Gt] = (int32_t)n;
    blk_tile.push_back(0);
    for (int b = 0; b < Gt && P.tma_ok; ++b) {
      int64_t R = tb[b];
      while (R < tb[b + 1]) {
        int64_t R1 = std::min<int64_t>(R + kTileRows, tb[b + 1]);
        if (rp[R1] - rp[R] > kTileNnz) {
          int64_t lo = R, hi = R1;  // largest R1 with rp[R1] - rp[R] <= kTileNnz
          while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (rp[mid] - rp[R] <= kTileNnz) lo = mid; else hi = mid - 1;
          }
          R1 = lo;
        }
        if (R1 == R) {
          // a row longer than a tile: one chunk tile per kTileNnz of its nonzeros, summed by
          // the whole block (csr_tiles, block per row)
          for (int64_t z = rp[R]; z < rp[R + 1]; z += kTileNnz) {
            tile_row.push_back((int32_t)R);
            tile_z0.resize(tile_row.size() - 1, -1);
            tile_z0.push_back((int32_t)z);
          }
          R = R + 1;
          continue;
        }
        tile_row.push_back((int32_t)R);
        R = R1;
      }
      blk_tile.push_back((int32_t)tile_row.size());
    }
    tile_row.push_back((int32_t)n);
    P.ntiles = (int)tile_row.size() - 1;
    if (!tile_z0.empty()) tile_z0.resize(P.ntiles, -1);
  }
  // per tile, the lanes that compute one row (see csr_tiles): 1 = one thread per row (two rows
  // per thread, in one pass), 2..16 = a group of lanes per row, 32 = short rows one thread and
  // rows longer than 32 nonzeros a whole warp each, in a length-sorted row order.  A tile
  // holds at most kTileNnz nonzeros, so long rows mean few rows per tile: with one thread per
  // row most consumer threads would idle.  The group size minimises the rounds of (at most 8)
  // dependent gathers a lane waits for: ceil(rows G / consumers) rows one after the other,
  // each ceil(lmax / 8 G) batches.  Tiles whose longest row is far above their mean (power-law
  // rows) take the sorted whole-warp schedule instead.
  auto tile_lanes = [&](int64_t rows, int64_t lmax, int64_t z) -> int {
    if (lmax <= 8) return 1;
    const double mean = (double)z / (double)rows;
    if (lmax > 32 && (double)lmax > 3.0 * mean + 8.0) return 32;
    int best = 1;
    double cost = std::ceil((double)lmax / 8.0);  // two rows per thread, interleaved
    for (int G = 2; G <= 16; G *= 2) {
      const double c = std::ceil((double)(rows * G) / kConsumers) * std::ceil((double)lmax / (8.0 * G));
      if (c <= cost) { best = G; cost = c; }  // ties: more lanes, fewer batches per row
    }
    return best == 1 && lmax > 32 ? 32 : best;
  };
  P.tile_grp.assign(P.tma_ok ? P.ntiles : 0, 1);
  auto& tile_grp = P.tile_grp;
  for (int t = 0; t < (int)tile_grp.size(); ++t) {
    if (!tile_z0.empty() && tile_z0[t] >= 0) {  // chunk of a row longer than a tile
      tile_grp[t] = 64;
      P.tiles_long += 1;
      continue;
    }
    int64_t lmax = 0;
    for (int64_t r = tile_row[t]; r < tile_row[t + 1]; ++r) lmax = std::max<int64_t>(lmax, rp[r + 1] - rp[r]);
    tile_grp[t] = (int8_t)tile_lanes(tile_row[t + 1] - tile_row[t], lmax, rp[tile_row[t + 1]] - rp[tile_row[t]]);
    (tile_grp[t] == 1 ? P.tiles_thread : tile_grp[t] == 32 ? P.tiles_long : P.tiles_group) += 1;
  }
  // row order of every irregular tile: rows sorted by length (longest first), dealt
  // round-robin over the 8 consumer warps -- slot (warp w, lane l) takes sorted rows
  // 8 l + w and 256 + 8 l + w -- so that each warp holds rows of similar length and the
  // long rows spread over all warps; -1 marks an empty slot
  auto& tile_perm = P.tile_perm;
  if (P.tiles_long > 0) {
    tile_perm.assign((size_t)P.ntiles * kTileRows, (int16_t)-1);
    std::vector<int32_t> order;
    for (int t = 0; t < P.ntiles; ++t) {
      if (tile_grp[t] != 32) continue;
      const int32_t R0 = tile_row[t], m = tile_row[t + 1] - R0;
      order.resize(m);
      for (int k = 0; k < m; ++k) order[k] = k;
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return rp[R0 + a + 1] - rp[R0 + a] > rp[R0 + b + 1] - rp[R0 + b];
      });
      int16_t* P = tile_perm.data() + (size_t)t * kTileRows;
      for (int tid = 0; tid < kTileRows / 2; ++tid) {
        const int w = tid / 32, l = tid % 32;
        const int k1 = 8 * l + w, k2 = kTileRows / 2 + 8 * l + w;
        P[tid] = k1 < m ? (int16_t)order[k1] : (int16_t)-1;
        P[kTileRows / 2 + tid] = k2 < m ? (int16_t)order[k2] : (int16_t)-1;
      }
    }
  }
  P.grid_stream = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 2, (n + 511) / 512));
}

// Row-length histogram: 0-8, 9-16, 17-32, 33-64, 65-256, 257-4096, > 4096 nonzeros.
static void row_histogram(int64_t n, const std::vector<int32_t>& rp, int64_t (&hist)[7]) {
  for (int k = 0; k < 7; ++k) hist[k] = 0;
  for (int64_t r = 0; r < n; ++r) {
    const int64_t L = rp[r + 1] - rp[r];
    hist[L <= 8 ? 0 : L <= 16 ? 1 : L <= 32 ? 2 : L <= 64 ? 3 : L <= 256 ? 4 : L <= 4096 ? 5 : 6] += 1;
  }
}

extern "C" {

const char* pk_status_string(pk_status s) {
  switch (s) {
    case PK_OK: return "PK_OK";
    case PK_ERR_ARG: return "PK_ERR_ARG";
    case PK_ERR_CUDA: return "PK_ERR_CUDA";
    case PK_ERR_OOM: return "PK_ERR_OOM";
    case PK_NOT_CONVERGED: return "PK_NOT_CONVERGED";
    case PK_BREAKDOWN: return "PK_BREAKDOWN";
    case PK_NOT_SPD: return "PK_NOT_SPD";
    case PK_ERR_NAN: return "PK_ERR_NAN";
    case PK_TIMEOUT: return "PK_TIMEOUT";
  }
  return "PK_UNKNOWN";
}

const char* pk_last_error(void) { return g_last_error.c_str(); }

int32_t pk_version(void) { return 100; }

static pk_status csr_create(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                            const double* vals, int32_t on_device, void* stream, pk_csr** out) {
  if (n < 0 || nnz < 0 || n >= (int64_t(1) << 31) - 64 || nnz >= (int64_t(1) << 31)) {
    set_error("n and nnz must be in [0, 2^31)");
    return PK_ERR_ARG;
  }
  if ((n > 0 && !row_ptr) || (nnz > 0 && (!col_idx || !vals))) {
    set_error("NULL CSR array");
    return PK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // host copies for validation and analysis
  std::vector<int32_t> rp(n + 1), ci(nnz);
  std::vector<double> va(nnz);
  if (n > 0) {
    if (on_device) {
      PK_CUDA(cudaMemcpy(rp.data(), row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
      if (nnz) {
        PK_CUDA(cudaMemcpy(ci.data(), col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
        PK_CUDA(cudaMemcpy(va.data(), vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
      }
    } else {
      memcpy(rp.data(), row_ptr, sizeof(int32_t) * (n + 1));
      if (nnz) {
        memcpy(ci.data(), col_idx, sizeof(int32_t) * nnz);
        memcpy(va.data(), vals, sizeof(double) * nnz);
      }
    }
  } else {
    rp[0] = 0;
  }
  if (rp[0] != 0 || rp[n] != nnz) {
    set_error("row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
    return PK_ERR_ARG;
  }
  int32_t rmin = n ? INT32_MAX : 0, rmax = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t len = rp[i + 1] - rp[i];
    if (len < 0) { set_error("row_ptr must be nondecreasing"); return PK_ERR_ARG; }
    rmin = std::min(rmin, len);
    rmax = std::max(rmax, len);
  }
  int fp32_exact = 1;
  for (int64_t j = 0; j < nnz; ++j) {
    if (ci[j] < 0 || ci[j] >= n) { set_error("column index out of range"); return PK_ERR_ARG; }
    if ((double)(float)va[j] != va[j]) fp32_exact = 0;
  }

  // every host allocation happens before the handle exists, so a failed one leaks nothing
  int device = 0, sms = 148;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  CsrPlan P;
  build_plan(n, nnz, rp, sms, P);
  pk_csr* A = new pk_csr();
  A->n = (int32_t)n;
  A->nnz = (int32_t)nnz;
  A->device = device;
  A->grid = P.grid;
  A->grid_tma = P.grid_tma;
  A->grid_stream = P.grid_stream;
  A->ntiles = P.ntiles;
  A->tma_ok = P.tma_ok;
  A->stats.tiles_thread = P.tiles_thread;
  A->stats.tiles_long = P.tiles_long;
  A->stats.tiles_group = P.tiles_group;
  auto& rb = P.rb;
  auto& tile_row = P.tile_row;
  auto& blk_tile = P.blk_tile;
  auto& tile_z0 = P.tile_z0;
  auto& tile_grp = P.tile_grp;
  auto& tile_perm = P.tile_perm;

  auto fail = [&](pk_status e) { pk_csr_destroy(A); return e; };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&A->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(cuda_fail(e, "cudaStreamCreate"));
  // pad every array by 64 elements so that vectorised loads of a ragged tail stay in bounds
  if ((e = cudaMalloc(&A->rp, sizeof(int32_t) * (n + 1 + 64))) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(row_ptr)"));
  if ((e = cudaMalloc(&A->ci, sizeof(int32_t) * (nnz + 64))) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(col)"));
  if ((e = cudaMalloc(&A->va, sizeof(double) * (nnz + 64))) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(val)"));
  if ((e = cudaMalloc(&A->rowblk, sizeof(int32_t) * (A->grid + 1))) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(rowblk)"));
  cudaMemsetAsync(A->rp, 0, sizeof(int32_t) * (n + 1 + 64), s);
  cudaMemsetAsync(A->ci, 0, sizeof(int32_t) * (nnz + 64), s);
  cudaMemsetAsync(A->va, 0, sizeof(double) * (nnz + 64), s);
  if ((e = cudaMemcpyAsync(A->rp, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(cuda_fail(e, "copy row_ptr"));
  if (nnz) {
    if ((e = cudaMemcpyAsync(A->ci, ci.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(cuda_fail(e, "copy col"));
    if ((e = cudaMemcpyAsync(A->va, va.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(cuda_fail(e, "copy val"));
  }
  if ((e = cudaMemcpyAsync(A->rowblk, rb.data(), sizeof(int32_t) * (A->grid + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(cuda_fail(e, "copy rowblk"));
  if (A->tma_ok) {
    if ((e = cudaMalloc(&A->tile_row, sizeof(int32_t) * tile_row.size())) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(tiles)"));
    if ((e = cudaMalloc(&A->blk_tile, sizeof(int32_t) * blk_tile.size())) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(tiles)"));
    if ((e = cudaMemcpyAsync(A->tile_row, tile_row.data(), sizeof(int32_t) * tile_row.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(cuda_fail(e, "copy tiles"));
    if ((e = cudaMemcpyAsync(A->blk_tile, blk_tile.data(), sizeof(int32_t) * blk_tile.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(cuda_fail(e, "copy tiles"));
    if ((e = cudaMalloc(&A->tile_grp, std::max<size_t>(1, tile_grp.size()))) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(tiles)"));
    if (!tile_perm.empty()) {
      if ((e = cudaMalloc(&A->tile_perm, sizeof(int16_t) * tile_perm.size())) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(tiles)"));
      if ((e = cudaMemcpyAsync(A->tile_perm, tile_perm.data(), sizeof(int16_t) * tile_perm.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(cuda_fail(e, "copy tiles"));
    }
    if (!tile_z0.empty()) {
      if ((e = cudaMalloc(&A->tile_z0, sizeof(int32_t) * tile_z0.size())) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(tiles)"));
      if ((e = cudaMemcpyAsync(A->tile_z0, tile_z0.data(), sizeof(int32_t) * tile_z0.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(cuda_fail(e, "copy tiles"));
    }
    if (!tile_grp.empty() &&
        (e = cudaMemcpyAsync(A->tile_grp, tile_grp.data(), tile_grp.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return fail(cuda_fail(e, "copy tiles"));
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_fail(e, "sync"));

  pk_csr_stats& st = A->stats;
  st.n = n;
  st.nnz = nnz;
  st.row_min = rmin;
  st.row_max = rmax;
  st.row_mean = n ? (double)nnz / (double)n : 0.0;
  st.grid = A->grid;
  st.block = kBlock;
  st.kernel = A->tma_ok ? 2 : 0;
  st.values_fp32_exact = fp32_exact;
  row_histogram(n, rp, st.row_hist);
  pk_status ps = ensure_state(A);
  if (ps) return fail(ps);
  *out = A;
  return PK_OK;
}

pk_status pk_csr_create(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* vals, int32_t on_device, void* stream, pk_csr** out) {
  if (!out) { set_error("out is NULL"); return PK_ERR_ARG; }
  *out = nullptr;
  return guarded([&] { return csr_create(n, nnz, row_ptr, col_idx, vals, on_device, stream, out); });
}

pk_status pk_csr_destroy(pk_csr* A) {
  if (!A) return PK_OK;
  cudaDeviceSynchronize();
  for (auto& g : A->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (int k = 0; k < A->ev_count; ++k) cudaEventDestroy(A->ev_pool[k]);
  for (auto* v : A->vec) if (v) cudaFree(v);
  if (A->basis) cudaFree(A->basis);
  if (A->jac_va) cudaFree(A->jac_va);
  if (A->sell_ptr) cudaFree(A->sell_ptr);
  if (A->sell_perm) cudaFree(A->sell_perm);
  if (A->sell_col) cudaFree(A->sell_col);
  if (A->sell_val) cudaFree(A->sell_val);
  if (A->jac_d) cudaFree(A->jac_d);
  if (A->jac_dinv) cudaFree(A->jac_dinv);
  if (A->res_rows) cudaFree(A->res_rows);
  if (A->res_nbr) cudaFree(A->res_nbr);
  if (A->res_flag) cudaFree(A->res_flag);
  if (A->small) cudaFree(A->small);
  if (A->partials) cudaFree(A->partials);
  if (A->st) cudaFree(A->st);
  if (A->st_host) cudaFreeHost(A->st_host);
  if (A->rp) cudaFree(A->rp);
  if (A->ci) cudaFree(A->ci);
  if (A->va) cudaFree(A->va);
  if (A->va32) cudaFree(A->va32);
  if (A->rowblk) cudaFree(A->rowblk);
  if (A->tile_row) cudaFree(A->tile_row);
  if (A->blk_tile) cudaFree(A->blk_tile);
  if (A->tile_grp) cudaFree(A->tile_grp);
  if (A->tile_perm) cudaFree(A->tile_perm);
  if (A->tile_z0) cudaFree(A->tile_z0);
  if (A->cap_stream) cudaStreamDestroy(A->cap_stream);
  delete A;
  return PK_OK;
}

static pk_status csr_plan(int64_t n, int64_t nnz, const int32_t* row_ptr, int32_t sms, pk_csr_stats* out) {
  std::vector<int32_t> rp(n + 1, 0);
  if (n > 0) memcpy(rp.data(), row_ptr, sizeof(int32_t) * (n + 1));
  if (rp[0] != 0 || rp[n] != nnz) {
    set_error("row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
    return PK_ERR_ARG;
  }
  pk_csr_stats st{};
  st.row_min = n ? INT32_MAX : 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t len = rp[i + 1] - rp[i];
    if (len < 0) { set_error("row_ptr must be nondecreasing"); return PK_ERR_ARG; }
    st.row_min = std::min(st.row_min, len);
    st.row_max = std::max(st.row_max, len);
  }
  CsrPlan P;
  build_plan(n, nnz, rp, sms, P);
  st.n = n;
  st.nnz = nnz;
  st.row_mean = n ? (double)nnz / (double)n : 0.0;
  st.grid = P.grid;
  st.block = kBlock;
  st.kernel = P.tma_ok ? 2 : 0;
  st.values_fp32_exact = -1;  // no values here
  st.tiles_thread = P.tiles_thread;
  st.tiles_long = P.tiles_long;
  st.tiles_group = P.tiles_group;
  row_histogram(n, rp, st.row_hist);
  *out = st;
  return PK_OK;
}

pk_status pk_csr_plan(int64_t n, int64_t nnz, const int32_t* row_ptr, int32_t sms, pk_csr_stats* out) {
  if (!out || n < 0 || nnz < 0 || n >= (int64_t(1) << 31) - 64 || nnz >= (int64_t(1) << 31) || sms < 1 ||
      (n > 0 && !row_ptr)) {
    set_error("pk_csr_plan: bad arguments");
    return PK_ERR_ARG;
  }
  return guarded([&] { return csr_plan(n, nnz, row_ptr, sms, out); });
}

pk_status pk_csr_stats_get(const pk_csr* A, pk_csr_stats* out) {
  if (!A || !out) { set_error("NULL argument"); return PK_ERR_ARG; }
  *out = A->stats;
  return PK_OK;
}

pk_status pk_residual_norm2(pk_csr* A, const double* b, const double* x, double* out2, void* stream) {
  if (!A || !out2 || (A->n && (!b || !x))) { set_error("NULL argument"); return PK_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n == 0) {
    PK_CUDA(cudaMemsetAsync(out2, 0, sizeof(double), s));
    return PK_OK;
  }
  launch_true_residual(A, b, x, nullptr, out2, s);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_spmv(pk_csr* A, const double* x, double* y, void* stream) {
  if (!A || (A->n && (!x || !y))) { set_error("NULL argument"); return PK_ERR_ARG; }
  if (A->n == 0) return PK_OK;
  launch_spmv(A, x, y, (cudaStream_t)stream);
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

pk_status pk_spmv_dot(pk_csr* A, const double* p, double* q, double* result, int32_t fused,
                      void* stream) {
  if (!A || !result || (A->n && (!p || !q))) { set_error("NULL argument"); return PK_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n == 0) {
    PK_CUDA(cudaMemsetAsync(result, 0, sizeof(double), s));
    return PK_OK;
  }
  if (fused == 2) {
    pk_status e = launch_sell_spmv_dot(A, p, q, result, s);
    if (e) return e;
  } else if (fused) {
    k_spmv_dot<<<A->grid, kBlock, 0, s>>>(row_args(A), p, q, result);
  } else {
    launch_spmv(A, p, q, s);
    launch_dot_store(A, p, q, result, s);
  }
  PK_CUDA(cudaGetLastError());
  return PK_OK;
}

}  // extern "C"
