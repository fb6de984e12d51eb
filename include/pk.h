/*
 * pk.h -- C ABI of the GB300 (sm_103a) pipelined Krylov solver library.
 *
 * Method: K. Rupp, J. Weinbub, A. Juengel, T. Grasser, "Pipelined Iterative Solvers with
 * Kernel Fusion for Graphics Processing Units", ACM TOMS 2015 (arXiv:1410.4054).
 * The problem statement (Sec. 1): solve A x = b for a sparse square matrix A and a right-hand
 * side b with CG (symmetric positive definite A), BiCGStab and restarted GMRES(m).
 *
 * Conventions shared by every entry point
 *   - Matrices are CSR with int32 row pointers / column indices and float64 values
 *     (Sec. 2.2).  pk_csr_create COPIES the matrix into library-owned device memory; the
 *     caller keeps ownership of its arrays.  Solver work vectors are allocated on first use
 *     (cudaMalloc) and cached in the pk_csr handle until pk_csr_destroy.
 *   - Vectors b (input) and x (in: initial guess x0, out: solution) are caller-owned,
 *     float64, length n.  They may be device pointers (no copies) or host pointers (the
 *     library copies them in and out inside the call; used for end-to-end timing).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *     stream-ordered and blocks only at its end, to read the final status into pk_info.
 *   - Stopping rule: ||r||_2 <= tol * ||b||_2.  b = 0 returns x = 0 after 0 iterations.
 *     tol = 0 runs exactly maxit iterations (fixed-iteration timing, Sec. 4).
 *   - Errors are returned as pk_status values, never by aborting.  Reaching maxit returns
 *     PK_NOT_CONVERGED with x valid.  A host allocation that fails inside the library (the
 *     CSR analysis, the SELL-C-sigma and FP32 copies, the batch tables) returns PK_ERR_OOM.
 *     pk_last_error() gives a message for the last failure on the calling thread.
 *   - The library uses one GPU: the device current on the calling thread.
 *   - A pk_csr handle carries its solves' work memory, cached graphs and state, and (during a
 *     right-Jacobi BiCGStab / GMRES solve) points its values at the scaled copy: calls on one
 *     handle must not overlap (one solve at a time per handle, from one host thread at a
 *     time, and in stream order when streams differ).  Different handles are independent.
 */
#ifndef PK_H_
#define PK_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PK_OK = 0,
  PK_ERR_ARG = 1,        /* invalid argument (bad CSR, NULL pointer, size limits) */
  PK_ERR_CUDA = 2,       /* a CUDA runtime call failed; see pk_last_error() */
  PK_ERR_OOM = 3,        /* a device or host allocation failed */
  PK_NOT_CONVERGED = 4,  /* maxit reached; x holds the last iterate */
  PK_BREAKDOWN = 5,      /* BiCGStab / GMRES breakdown (zero denominator, no progress) */
  PK_NOT_SPD = 6,        /* CG found <p, Ap> <= 0 */
  PK_ERR_NAN = 7,        /* a scalar became NaN / Inf */
  PK_TIMEOUT = 8         /* a bounded device-side wait ran out */
} pk_status;

/* Solver formulation. */
enum {
  PK_VARIANT_PIPELINED = 0, /* Alg. 2 / 4 / 6 with fused kernels (Sec. 3) */
  PK_VARIANT_CLASSICAL = 1, /* Alg. 1 / 3 / 5 as one kernel per BLAS-like operation */
  PK_VARIANT_SPLIT = 2      /* pipelined, SpMV not fused with the reductions (Sec. 3.1-3.3,
                               the "not possible or desired" fallbacks) */
};

/* Arithmetic of the iteration. */
enum {
  PK_PREC_FP64 = 0,  /* everything in float64 */
  PK_PREC_MIXED = 1  /* pk_cg_solve only: FP32 SpMV/vectors inside FP64 iterative refinement */
};

/* How the iteration loop is driven. */
enum {
  PK_LOOP_GRAPH = 0, /* CUDA graph with a device-controlled conditional WHILE node:
                        no host round-trip until the solve ends */
  PK_LOOP_HOST = 1,  /* plain launches; the host reads the device "done" flag every
                        `check_every` iterations (kernels after convergence return at once) */
  PK_LOOP_PERSISTENT = 2, /* pipelined FP64 CG, BiCGStab and GMRES(m): the whole iteration
                        loop in one launch on one thread-block cluster (16 CTAs where
                        available, else 8) with the gathered vectors in distributed shared
                        memory (CG: p, x, r, Ap; BiCGStab: p, s, r, Ap, As, r0*; GMRES: the
                        current basis vector, with the basis itself in global memory and R,
                        xi, eta in every CTA), hardware cluster barriers, every CTA summing
                        the block partials itself in a fixed order; for n <=
                        PK_PERSISTENT_MAX_N.  Larger n, other variants, precisions, GMRES
                        with PK_FLAG_CGS2 or PK_FLAG_GM_SHIFT return PK_ERR_ARG */
  PK_LOOP_AUTO = 3,  /* PK_LOOP_PERSISTENT for pipelined FP64 CG with n <= PK_PERSISTENT_AUTO_N
                        and nnz <= PK_PERSISTENT_AUTO_NNZ, pipelined BiCGStab with n <=
                        PK_PERSISTENT_BICGSTAB_AUTO_N and nnz <= PK_PERSISTENT_BICGSTAB_AUTO_NNZ,
                        and pipelined GMRES (one Gram-Schmidt pass) with n <=
                        PK_PERSISTENT_GMRES_AUTO_N and nnz <= PK_PERSISTENT_GMRES_AUTO_NNZ (and
                        no PK_FLAG_TIMING; for BiCGStab and GMRES also no rows of very
                        different lengths, stats.tiles_long == 0) when the device can run it,
                        PK_LOOP_GRAPH otherwise */
  PK_LOOP_RESIDENT = 4 /* pipelined FP64 CG only: the whole iteration loop in one cooperative
                        launch of one block per SM.  Each iteration's update (x, r, p) and fused
                        SpMV run back to back in the launch; the SpMV of a block waits only for
                        the blocks owning the columns it reads, and the one grid-wide step is
                        the deterministic reduction that forms alpha and beta (Eq. (3)).  Needs
                        the tile grid to cover two blocks per SM (n >= 1024 x SMs rows or
                        nnz >= 8192 x SMs) and cooperative launch; otherwise, or with
                        PK_FLAG_SELL or PK_FLAG_NO_TMA, PK_ERR_ARG.  PK_FLAG_TIMING times the
                        launch (PK_SLOT_RESIDENT).  Every wait is bounded by pk_opts.wait_ns
                        (PK_TIMEOUT) */
};
#define PK_PERSISTENT_MAX_N 65536  /* 16 CTAs x 4096 rows (8 x 4096 on devices without
                                      16-CTA clusters) */
#define PK_PERSISTENT_AUTO_N 65536
/* measured on GB300: the 16-SM cluster loop wins up to ~330k nonzeros (2D 5-point 256^2),
 * the full-GPU graph loop from ~450k (P1 triangles, 65,025 unknowns) */
#define PK_PERSISTENT_AUTO_NNZ 393216
/* BiCGStab (four cluster barriers and two products per iteration), measured on GB300 on 3D
 * convection-diffusion: the cluster loop takes 16 us per iteration against 33 for the graph
 * at 16^3, 29 against 35 at 32^3 (223k nonzeros), 48 against 36 at 40^3 (438k) */
#define PK_PERSISTENT_BICGSTAB_AUTO_N 32768
#define PK_PERSISTENT_BICGSTAB_AUTO_NNZ 262144
/* pipelined GMRES(m) (three cluster barriers per step, the basis in global memory) */
#define PK_PERSISTENT_GMRES_AUTO_N 32768
#define PK_PERSISTENT_GMRES_AUTO_NNZ 262144

/* pk_opts.flags */
#define PK_FLAG_TIMING 1u    /* time every kernel launch with CUDA events (host loop) and
                                report per-kernel averages in pk_info.kernel_ms */
#define PK_FLAG_TRUE_RES 2u  /* compute ||b - A x|| / ||b|| at exit into pk_info.rel_res_true */
#define PK_FLAG_NO_TMA 4u    /* use the thread-per-row kernels instead of the warp-specialised
                                bulk-copy tile kernels (for comparison) */
#define PK_FLAG_AUTOTUNE 8u  /* pk_batched_solve: time every engine and (block size, blocks
                                per SM, lanes per row) candidate on the batch first and keep
                                the fastest (cached per batch shape for the process) */
#define PK_FLAG_SELL 16u     /* pipelined FP64 CG: the fused SpMV kernel (Ap, <Ap,Ap>, <p,Ap>, alpha,
                                beta) reads a SELL-C-sigma copy of A (C = 32, sigma = 1024; built on
                                first use, kept with the handle) instead of the CSR tiles.  Other
                                solvers, variants, precisions, PK_LOOP_PERSISTENT and
                                preconditioners return PK_ERR_ARG */
#define PK_FLAG_CGS2 32u     /* GMRES: classical Gram-Schmidt applied twice per Arnoldi step
                                (c_j = <v_j, v_i> again after the first projection, v_i -=
                                sum c_j v_j, R_{j,i} += c_j; two more launches per step), which
                                keeps the basis orthonormal and the in-cycle residual estimate
                                exact on badly conditioned systems.  Other solvers return
                                PK_ERR_ARG */
#define PK_FLAG_TEST_STALL 64u  /* testing the failure path: the CSR tile engine's producer
                                   issues no copies, so the first wait of every consumer runs
                                   out after pk_opts.wait_ns and the solve returns PK_TIMEOUT
                                   (nothing is in flight; the context stays usable) */
#define PK_FLAG_GM_SHIFT 128u   /* pipelined GMRES: the shift-invariant three-kernel form that
                                   Sec. 3.3 names (after l1-GMRES).  A v_{i-1} and
                                   w = (A - sigma_i I) v_{i-1} have the same part orthogonal
                                   to v_1 .. v_{i-1}, so R_{i,i} = ||v_i|| before normalisation
                                   follows from <w,w> and the Gram-Schmidt coefficients:
                                   R_{i,i}^2 = <w,w> - sum_{j<i-1} R_{j,i}^2 - (R_{i-1,i} -
                                   sigma_i)^2.  <w,w> is formed with the product, so the
                                   normalisation and xi_i fuse into the update kernel: 3
                                   kernels per step instead of 4, R and xi those of the
                                   4-kernel form.  Shifts: sigma_1 = 0, sigma_{i+1} =
                                   <v_{i-1}, A v_{i-1}> (the previous basis vector's Rayleigh
                                   quotient).  While R_{i,i}^2 <= 1e-8 <w,w> the identity is
                                   not trusted and the cycle ends before step i (restart).
                                   Not with PK_FLAG_CGS2 or the classical variant (PK_ERR_ARG) */

typedef struct {
  double tol;          /* relative residual tolerance (>= 0) */
  int32_t maxit;       /* iteration limit: CG/BiCGStab loop iterations, GMRES Arnoldi steps */
  int32_t restart;     /* GMRES restart length m, 1..64 */
  int32_t variant;     /* PK_VARIANT_* */
  int32_t precision;   /* PK_PREC_* */
  int32_t loop;        /* PK_LOOP_* */
  int32_t check_every; /* PK_LOOP_HOST: iterations between host checks (0 -> 16) */
  uint32_t flags;      /* PK_FLAG_* */
  int32_t trace_cap;   /* capacity (iterations) of `trace`, 0 = no trace */
  double* trace;       /* optional DEVICE array [trace_cap][4]: per iteration i the solver
                          writes {alpha_i, beta_i, omega_i, res2_i} (unused slots untouched);
                          GMRES writes {R_{i-1,i}, R_{i,i}, xi_i, estimate_i} */
  int32_t precond;     /* PK_PRECOND_*: CG, BiCGStab, GMRES (0 = none; the batched solver
                          takes none) */
  int32_t lanes;       /* pk_batched_solve: lanes per matrix row in the row products (1, 2, 4
                          or 8; 0 = automatic: from the batch's mean row length, or tuned with
                          the block shape under PK_FLAG_AUTOTUNE; -1 = the tile engine, -2 = the
                          cluster engine).
                          Other solvers ignore it */
  int64_t wait_ns;     /* bound, in ns, on every device-side pipeline wait that should make
                          progress (0 = 2 s).  A wait that runs out ends the solve with
                          PK_TIMEOUT after the kernel has drained its own copies; the context
                          stays usable.  Small values exercise that path in tests */
} pk_opts;

/* pk_opts.precond.  JACOBI, M = diag(A) (entries of row i in column i summed; Sec. 5 names
 * preconditioner fusion as the method's extension).
 * CG: pipelined FP64 CG (Alg. 2 with the preconditioned
 * inner products <r, M^-1 r> and <Ap, M^-1 Ap>; beta = alpha^2 <Ap, M^-1 Ap>/<r, M^-1 r> - 1)
 * on the graph or host loop; the fused SpMV kernel forms Ap, <p, Ap>, <Ap, M^-1 Ap>, the
 * update kernel x, r, p = M^-1 r + beta p, <r, M^-1 r> and <r, r>.  The stopping test stays
 * ||r|| <= tol ||b||.  A diagonal entry <= 0 returns PK_NOT_SPD.  Other variants, precisions
 * and the persistent loop return PK_ERR_ARG (PK_LOOP_AUTO uses the graph loop).
 * BiCGStab and GMRES (both variants): right preconditioning.  The solver runs unchanged on
 * A M^-1 y = b, whose residual is b - A x for x = M^-1 y, so the stopping test and the trace
 * are those of the plain solver on A M^-1; the values of A M^-1 (columns scaled by the
 * reciprocal diagonal) are built on first use and kept with the handle (8 nnz + 16 n bytes),
 * x enters as y0 = M x0 and leaves as M^-1 y.  A zero or non-finite diagonal entry returns
 * PK_ERR_ARG before any iteration. */
enum { PK_PRECOND_NONE = 0, PK_PRECOND_JACOBI = 1 };

/* Per-kernel timing slots in pk_info (PK_FLAG_TIMING). */
#define PK_MAX_KERNEL_SLOTS 8

typedef struct {
  int32_t iters;         /* iterations performed (GMRES: Arnoldi steps over all cycles) */
  int32_t status;        /* pk_status of the solve */
  int32_t cycles;        /* GMRES restarts; mixed precision: outer refinement steps */
  int32_t launches;      /* kernels launched by the call (graph nodes counted per execution) */
  double rel_res_est;    /* last recursive residual estimate / ||b|| */
  double rel_res_true;   /* ||b - A x|| / ||b|| at exit (PK_FLAG_TRUE_RES), else -1 */
  double solve_ms;       /* device time of the call from its first to its last kernel */
  double kernel_ms[PK_MAX_KERNEL_SLOTS];      /* PK_FLAG_TIMING: mean ms per launch, by slot */
  int32_t kernel_count[PK_MAX_KERNEL_SLOTS];  /* PK_FLAG_TIMING: launches timed, by slot */
} pk_info;

/* Timing slots (index into kernel_ms / kernel_count). */
enum {
  PK_SLOT_SPMV_DOTS = 0, /* fused SpMV + first reduction stage (K-CG-S, K-BI-1/3, K-GM-1) */
  PK_SLOT_UPDATE = 1,    /* fused vector update + first reduction stage (K-CG-U, K-BI-2/4) */
  PK_SLOT_MULTIDOT = 2,  /* GMRES Gram-Schmidt inner products */
  PK_SLOT_ORTHO = 3,     /* GMRES update + norm, normalisation + xi */
  PK_SLOT_SPMV = 4,      /* plain SpMV (classical / split forms) */
  PK_SLOT_BLAS1 = 5,     /* plain BLAS-1 kernels (classical / split forms) */
  PK_SLOT_OTHER = 6,     /* setup, cycle end, refinement */
  PK_SLOT_RESIDENT = 7   /* the single launch of PK_LOOP_RESIDENT (the whole iteration loop) */
};

typedef struct pk_csr pk_csr;

/* Row statistics and schedule chosen by pk_csr_create (Sec. 2.2; rows are assigned to
 * thread blocks in nnz-balanced contiguous ranges). */
typedef struct {
  int64_t n, nnz;
  int32_t row_min, row_max;  /* shortest / longest row */
  double row_mean;
  int32_t grid;              /* thread blocks of the fused kernels */
  int32_t block;             /* threads per block */
  int32_t kernel;            /* SpMV engine: 0 thread-per-row loads, 2 warp-specialised bulk-copy tiles */
  int32_t values_fp32_exact; /* 1 if every value is exactly representable in float32 */
  /* bulk-copy tiles by row schedule: every row one thread (tiles_thread: rows short enough
   * for one thread to walk); short rows one thread and long rows a whole warp each
   * (tiles_long: rows of very different lengths); rows of similar length G = 2..16 lanes each
   * (tiles_group).  The chunk tiles of a row longer than a tile (4096 nonzeros), summed by
   * the whole block, count in tiles_long too: ceil(length / 4096) per such row */
  int32_t tiles_thread, tiles_long;
  int32_t tiles_group;
  /* row-length histogram: rows with 0-8, 9-16, 17-32, 33-64, 65-256, 257-4096 and more than
   * 4096 nonzeros (one thread, small groups, a warp, long warp rows, chunk tiles) */
  int64_t row_hist[7];
} pk_csr_stats;

/*
 * Create a CSR matrix handle (Sec. 2.2 "compressed sparse row representation").
 *   n, nnz      : rows (= columns) and nonzeros; 0 <= n, nnz < 2^31.
 *   row_ptr     : n+1 int32, row_ptr[0] = 0, nondecreasing, row_ptr[n] = nnz.
 *   col_idx     : nnz int32 in [0, n).
 *   vals        : nnz float64.
 *   on_device   : 1 if the three arrays are device pointers, 0 if host pointers.
 * The arrays are validated (PK_ERR_ARG on violation), copied and analysed (row-length
 * statistics -> schedule).  *out receives the handle; release it with pk_csr_destroy.
 */
pk_status pk_csr_create(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* vals, int32_t on_device, void* stream, pk_csr** out);

/* Release the handle, its matrix copy and all cached work memory. NULL is accepted. */
pk_status pk_csr_destroy(pk_csr* A);

/* Row statistics and the schedule chosen for A. */
pk_status pk_csr_stats_get(const pk_csr* A, pk_csr_stats* out);

/* The statistics and schedule pk_csr_create would choose for a matrix with these row pointers
 * on a device with `sms` multiprocessors, computed on the host alone (no GPU, nothing kept):
 * row_ptr is a HOST int32 array of n + 1 entries; values_fp32_exact is -1 (no values given).
 * An invalid row_ptr returns PK_ERR_ARG. */
pk_status pk_csr_plan(int64_t n, int64_t nnz, const int32_t* row_ptr, int32_t sms, pk_csr_stats* out);

/* y = A x (device pointers, length n) -- the plain CSR product of Sec. 2.2. */
pk_status pk_spmv(pk_csr* A, const double* x, double* y, void* stream);

/*
 * q = A p and *result = <p, q> (Sec. 2.2, Eq. (1)-(2)).  fused = 1 computes the first
 * reduction stage inside the SpMV kernel and the second in its last block (one launch);
 * fused = 0 runs the SpMV, then a separate inner-product kernel (two launches); fused = 2 is
 * the fused kernel on a SELL-C-sigma copy of A (sliced ELLPACK, 32 rows per slice sorted by
 * length within windows of 1024 rows; built on first use and kept with the handle, padded
 * entries skipped; every row summed left to right as in the CSR loop).
 * p, q: device, length n.  result: device pointer to one double.
 */
pk_status pk_spmv_dot(pk_csr* A, const double* p, double* q, double* result, int32_t fused,
                      void* stream);

/*
 * Conjugate gradients for SPD A.  variant PIPELINED = Alg. 2 with two fused kernels per
 * iteration (update x,r,p + <r,r>; SpMV + <Ap,Ap>, <p,Ap>, with alpha/beta from Eq. (3) in
 * the SpMV kernel's last block; Sec. 3.1); CLASSICAL = Alg. 1 as six kernels per iteration
 * (SpMV, dot, axpy, axpy, dot, xpay); SPLIT = Alg. 2 with SpMV and its dots in separate
 * kernels (three per iteration).  precision MIXED: Alg. 2 in FP32 (values rounded to FP32,
 * FP32 vectors and SpMV accumulation) on r / ||r||, stopped at a 1e-4 inner reduction, inside
 * an FP64 iterative-refinement loop (FP64 true residual b - A x, FP64 correction x += ||r|| d,
 * at most 20 refinement steps; maxit bounds the inner iterations in total; info.cycles =
 * refinement steps); the inner products that set alpha and beta are accumulated per thread
 * as float-float pairs and reduced in FP64.  opts / info may not be NULL.
 */
pk_status pk_cg_solve(pk_csr* A, const double* b, double* x, const pk_opts* opts, pk_info* info,
                      void* stream);

/*
 * BiCGStab (Alg. 3 / 4, Sec. 3.2), r0* = r0.  PIPELINED: four fused kernels per iteration
 * (SpMV Ap + <Ap,r0*> -> alpha; s = r - alpha Ap + <s,s>; SpMV As + <As,s>, <As,As>,
 * <As,r0*> -> omega, beta; x, r, p updates + <r,r0*>, <r,r>).  CLASSICAL: one kernel per
 * operation of Alg. 3.
 */
pk_status pk_bicgstab_solve(pk_csr* A, const double* b, double* x, const pk_opts* opts,
                            pk_info* info, void* stream);

/*
 * Restarted simpler GMRES(m) with classical Gram-Schmidt (Alg. 5 / 6, Sec. 3.3),
 * m = opts->restart (1..64).  PIPELINED: step 1 two kernels, later steps four (SpMV +
 * <v_{i-1}, v_i>; inner products with v_1..v_{i-2}; R column + update + ||v_i||^2;
 * normalisation + xi_i); the triangular solve R eta = xi and the x update run on the device
 * at the end of each cycle.  maxit counts Arnoldi steps over all cycles.
 */
pk_status pk_gmres_solve(pk_csr* A, const double* b, double* x, const pk_opts* opts,
                         pk_info* info, void* stream);

/*
 * The R factor and xi = (<v_0, v_1>, ..., <v_0, v_m>) of the most recent GMRES cycle run on A
 * (Alg. 5 / 6, Sec. 3.3: the upper-triangular R of the Arnoldi relation and the right-hand
 * side of R eta = xi), for inspection and testing.  R and xi are HOST arrays of m * m and m
 * doubles; R[(j-1) * m + (i-1)] receives R_{j,i} for 1 <= j <= i <= m (zero below the
 * diagonal), xi[i-1] receives xi_i.  Columns past the steps that cycle took hold values of an
 * earlier cycle (or zero).  m in 1..64; PK_ERR_ARG if no GMRES solve has run on A.
 * Synchronises `stream`.
 */
pk_status pk_gmres_cycle_factors(const pk_csr* A, int32_t m, double* R, double* xi, void* stream);

/*
 * Many independent SPD systems in one persistent launch (motivated by the paper's transient
 * and small-system regime, Sec. 1 and 4.1).  A persistent grid takes systems from a device
 * work queue, largest first; one thread block runs pipelined CG (Alg. 2) on a system to
 * completion with block-wide reductions, then takes the next, so a converged system simply
 * leaves the queue (per-system convergence mask).  A[k], b[k], x[k] for k < nsys; b and x
 * must be DEVICE pointers.  opts: tol, maxit (per system; MIXED: total inner iterations),
 * precision PK_PREC_FP64 or PK_PREC_MIXED (FP32 SpMV/vectors inside FP64 iterative
 * refinement, inner tolerance 1e-4, at most 20 refinement steps), lanes, wait_ns, flags
 * PK_FLAG_AUTOTUNE.  Two engines:
 *   - the row engine (default): plain row loops, lanes = 1, 2, 4 or 8 lanes per row (0 = from
 *     the batch's mean row length), FP64 or MIXED;
 *   - lanes = -1, FP64, every system with CSR tiles: the tile engine -- each block (288
 *     threads, 2 per SM) streams its system's CSR tiles and vectors through shared memory with
 *     bulk copies, as the single-system kernels do (bounded waits: PK_TIMEOUT).  Measured
 *     slower than the row engine on small systems (18 resident warps per SM against 64 hide
 *     less of the gather latency), so it is an option and a candidate of the tuner;
 *   - lanes = -2, FP64, every system of at most 65536 rows: the cluster engine -- a system of
 *     n rows is solved by a thread-block cluster of C = 1, 2, 4, 8 or 16 CTAs holding p, x, r
 *     and Ap in the CTAs' shared memory, the SpMV gathering p across the cluster (distributed
 *     shared memory), so that per iteration only the matrix is read from global memory.  CTA
 *     shapes: 256 threads and up to 2048 rows (2 per SM), the smallest C with C * 2048 >= n;
 *     systems of more than 32768 rows on CTAs of 512 threads and up to 4096 rows (1 per SM).
 *     One persistent cluster launch per (shape, C) class, the launches on streams of their
 *     own that join the caller's stream.
 * PK_FLAG_AUTOTUNE (lanes 0) times the tile engine and the cluster engine (FP64, the cluster
 * engine aiming at 1024, 2048 and 4096 rows per CTA: CTAs of 128, 256, 512 threads) and every
 * (block size, blocks per SM, lanes per row) of the row engine on the batch, each solving the
 * whole batch to tol / maxit from x as given (x is restored after each), and keeps the
 * fastest (cached per batch shape and precision for the process).  PK_FLAG_SELL, PK_FLAG_CGS2 and a
 * preconditioner return PK_ERR_ARG; variant, loop and the other flags are ignored (always
 * pipelined CG).  infos: nsys entries or NULL (iters, status, cycles = refinement steps,
 * rel_res_est).  Returns PK_OK if every system converged, else the first failing system's
 * status.
 */
pk_status pk_batched_solve(int32_t nsys, pk_csr* const* A, const double* const* b,
                           double* const* x, const pk_opts* opts, pk_info* infos, void* stream);

/* Block size and blocks per SM used by the last pk_batched_solve call in this process
 * (the cluster engine: the CTA shape of its default or tuned rows per CTA, e.g. 256 threads and
 * 2 blocks per SM for 2048 rows). */
pk_status pk_batched_last_config(int32_t* block, int32_t* blocks_per_sm);

/* Lanes per row (1, 2, 4 or 8) that the last pk_batched_solve call ran with; -1 = the tile
 * engine (pk_batched_last_config then gives 288 threads, 2 blocks per SM), -2 = the cluster
 * engine. */
pk_status pk_batched_last_lanes(int32_t* lanes);

/*
 * Allocation-free q = A p and *result = <p, q>.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory where they need the product --
 * loops with a memory budget fixed in advance (an allocation could fail or stall mid-loop),
 * or hosts that must not go through a caching allocator they do not own.
 * Unlike pk_spmv_dot it needs no pk_csr handle: the caller passes its own DEVICE CSR arrays
 * (same layout as pk_csr_create, not validated here), p, q (length n) and result (one
 * double), and the call allocates nothing.  Its scratch (per-block partial sums and the
 * last-block arrival counter) lives in a fixed device array of PK_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits.
 *   - n must be in [0, PK_NOALLOC_MAX_N]; larger n returns PK_ERR_ARG with a message.
 *   - q must not overlap p, row_ptr, col_idx, vals or result (q == p returns PK_ERR_ARG;
 *     other overlaps give wrong results).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current and keeps it for the process; make that first call before
 *     any stream capture.  Calls after a cudaDeviceReset of that device are not supported.
 *   - All calls on a device share the array (each call zeroes the counter first): calls that
 *     overlap on the GPU, e.g. on two streams at once, race and give wrong results.
 * Stream-ordered on `stream`; returns without synchronising.
 */
#define PK_NOALLOC_MAX_N 16777216
#define PK_NOALLOC_MAX_BLOCKS 2048
#define PK_NOALLOC_SCRATCH_BYTES (256 + 8 * PK_NOALLOC_MAX_BLOCKS)
pk_status pk_spmv_dot_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                              const double* vals, const double* p, double* q, double* result,
                              void* stream);

/* *out2 = ||b - A x||^2 (device pointers; deterministic reduction). */
pk_status pk_residual_norm2(pk_csr* A, const double* b, const double* x, double* out2, void* stream);

/*
 * Learned initial guess for transient problems (an extension; the paper has no counterpart): a 4-layer 3x3x3
 * convolutional network on a D x H x W grid, BF16 operands with FP32 accumulation on the
 * tensor cores as implicit GEMMs on tcgen05 (forward and backward-data: M = 128-voxel tiles;
 * weight gradient: M = 8 taps x 16 input channels, K = voxels).  Activations are channels-last BF16
 * [D][H][W][16] with channel counts padded to 16 (padded channels are zero); weights are BF16
 * [27][16 co][16 ci], tap = 9(dz+1) + 3(dy+1) + (dx+1); zero padding 1 at the boundary.
 * All pointers are device pointers; calls are stream-ordered and return at once.
 */
/* Y = conv(X, W) + bias, then ReLU if relu (tcgen05 tensor cores: M = 128-voxel tiles of
 * 8 x 16 voxels, one M128 N16 K16 MMA per tap, FP32 accumulator in tensor memory);
 * out_f32: Y is FP32 [D][H][W] holding channel 0
 * only; mask (nullable, BF16 [D][H][W][16]): Y[v][c] = 0 where mask[v][c] <= 0 (the ReLU
 * derivative, used by the backward-data pass with flipped weights). */
pk_status pk_conv3d_fwd(const void* X, const void* Wt, const float* bias, void* Y, int32_t D,
                        int32_t H, int32_t W, int32_t relu, int32_t out_f32, const void* mask,
                        void* stream);
/* Reads and clears the device flag a tensor-core convolution sets when its bounded wait for
 * its own MMAs runs out (PK_TIMEOUT; the output of that call is then incomplete); PK_OK
 * otherwise.  Synchronises the stream. */
pk_status pk_conv3d_check(void* stream);
/* dW[tap][co][ci] = sum_v G[v][co] A[v + tap][ci] (FP32), db[co] = sum_v G[v][co]; scratch:
 * pk_conv3d_wgrad_scratch_floats(D, H, W) floats (deterministic block partials).  A and G
 * 16-byte aligned (PK_ERR_ARG otherwise); a timed-out wait of the tensor-core kernel is
 * reported by pk_conv3d_check. */
int64_t pk_conv3d_wgrad_scratch_floats(int32_t D, int32_t H, int32_t W);
pk_status pk_conv3d_wgrad(const void* A, const void* G, float* scratch, float* dW, float* db,
                          int32_t D, int32_t H, int32_t W, void* stream);
/* Wf[26 - t][ci][co] = W[t][co][ci]: weights of the backward-data convolution. */
pk_status pk_conv3d_flip(const void* W, void* Wf, void* stream);
/* Network input from the residual of the linear extrapolation e = 2 x_{t-1} - x_{t-2} of the
 * system A x_t = b (A: the n x n matrix of the time step, n = D H W):
 * r = b - A e, d = diag(A) (1 where a row has no nonzero diagonal entry),
 * X16 = bf16((r/d)/s0, r/s1, d/s2, 0...) with s0, s1, s2 the rms of r/d, r, d written to
 * scales[0..2] (1 where zero; 3 doubles); scratch: pk_warmstart_scratch_doubles() doubles. */
pk_status pk_warmstart_input(pk_csr* A, const double* xm1, const double* xm2, const double* b,
                             void* X16, double* scales, double* scratch, void* stream);
/* Target y = (x_t - 2 x_{t-1} + x_{t-2}) / s0 (the part linear extrapolation misses):
 * *loss = mean((out - y)^2), G = bf16(2 (out - y) / n) in channel 0 (other channels 0). */
pk_status pk_warmstart_loss(int64_t n, const float* out, const double* xt, const double* xm1,
                            const double* xm2, const double* scales, void* G, double* loss,
                            double* scratch, void* stream);
/* x_hat = 2 x_{t-1} - x_{t-2} + s0 out; out = NULL gives the linear extrapolation alone. */
pk_status pk_warmstart_apply(int64_t n, const float* out, const double* xm1, const double* xm2,
                             const double* scales, double* xhat, void* stream);
/* The energy step along the network's correction d = s0 out from the extrapolation
 * e = 2 x_{t-1} - x_{t-2} (A SPD): gamma = <b - A e, d> / <d, A d>, the step length that
 * minimises the A-norm of the error of e + gamma d (A (x_t - e) = b - A e), written to
 * gamma[0] (device, one double; 0 if <d, A d> <= 0 or the quotient is not finite), and
 * x_hat = e + gamma d.  Unlike pk_warmstart_apply (gamma = 1), the start it gives is never
 * farther from the solution in the A-norm than e.  One pass over A plus one over the vectors;
 * scratch: pk_warmstart_scratch_doubles() doubles.  (An extension; the paper has no learned part.) */
pk_status pk_warmstart_apply_energy(pk_csr* A, const float* out, const double* xm1, const double* xm2,
                                    const double* b, const double* scales, double* xhat, double* gamma,
                                    double* scratch, void* stream);
/* One damped Jacobi sweep on A x = b from the starting guess x:
 * xout = x + omega (b - A x) / d, d = diag(A) (1 where a row has no nonzero diagonal entry),
 * each row's products summed left to right.  The learned warm start applies it to the network's
 * guess: the network's error is rough (rounding of its BF16 operands and approximation error
 * spread over every frequency), rough error lies at the large eigenvalues of D^-1 A, where a
 * sweep with omega near 0.8 damps it, and CG removes smooth error fastest.  A, b, x, xout on
 * the device (n doubles each); omega in (0, 2); xout must not overlap x, b or the matrix
 * (xout == x returns PK_ERR_ARG).  One pass over A; stream-ordered, no synchronisation.
 * (An extension; the paper has no learned part.) */
pk_status pk_warmstart_relax(pk_csr* A, const double* b, const double* x, double omega, double* xout,
                             void* stream);
/* Training loss of the learned guess in the form CG receives it: after `sweeps` damped Jacobi
 * sweeps (pk_warmstart_relax with the same omega).  With delta = out - (x_t - 2 x_{t-1} +
 * x_{t-2}) / s0 (the guess's error in units of s0 = scales[0]) and P = I - omega D^-1 A (one
 * sweep's error propagator), *loss = mean((P^s delta)^2) and G = bf16(gradient) in channel 0
 * (other channels 0), gradient = (2/n) (P^T)^s P^s delta with P^T g = g - omega A (D^-1 g),
 * which holds for a SYMMETRIC A (the implicit heat-equation operator).  sweeps = 0 gives the
 * loss of pk_warmstart_loss.  omega in (0, 2), sweeps in [0, PK_WS_MAX_SWEEPS], n > 0
 * (PK_ERR_ARG otherwise).  work: 3 n doubles of device memory owned by the caller; scratch:
 * pk_warmstart_scratch_doubles() doubles.  1 + 2 sweeps passes over A; stream-ordered.
 * (An extension; the paper has no learned part.) */
#define PK_WS_MAX_SWEEPS 8
pk_status pk_warmstart_loss_swept(pk_csr* A, const float* out, const double* xt, const double* xm1,
                                  const double* xm2, const double* scales, double omega, int32_t sweeps,
                                  void* G, double* loss, double* work, double* scratch, void* stream);
/* Adam (Kingma & Ba) on FP32 parameters, step >= 1; p_bf16 (nullable) receives a BF16 copy. */
pk_status pk_adam_step(int64_t count, float* p, const float* grad, float* m, float* v, float lr,
                       float beta1, float beta2, float eps, int32_t step, void* p_bf16,
                       void* stream);

/* Human-readable name of a status code (static string). */
const char* pk_status_string(pk_status s);

/* Message describing the last error on the calling thread ("" if none). */
const char* pk_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t pk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PK_H_ */
