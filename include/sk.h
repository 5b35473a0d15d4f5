/*
 * sk.h -- C ABI of the GB300 (sm_103a) sketched-Krylov library (libsk.so).
 *
 * Sketched GMRES and sketched Rayleigh-Ritz after Nakatsukasa & Tropp,
 * "Fast & Accurate Randomized Algorithms for Linear Systems and Eigenvalue
 * Problems".  Section/equation/algorithm references below are to that paper.
 *
 * Conventions for every call:
 *   - Vectors and matrices are DEVICE pointers (CUDA global memory) unless a
 *     parameter says "host".  The caller owns them; the library never frees
 *     or retains them past the call, except borrowed operator arrays (below).
 *   - Matrices are column-major with an explicit leading dimension.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous with respect to the host unless stated
 *     otherwise; calls that return scalar diagnostics (info structs, d_used,
 *     nconv) synchronise the stream before returning.
 *   - Every call returns an sk_status and never aborts or throws across the
 *     ABI.  Arguments are validated before any launch; on SK_EINVAL nothing
 *     was launched.  sk_last_error() gives a thread-local message.
 *   - Workspace is allocated internally with stream-ordered cudaMallocAsync
 *     and released before the call returns (SK_ENOMEM if that fails).
 */
#ifndef SK_H
#define SK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SK_OK = 0,
  SK_EINVAL = 1,     /* invalid argument (sizes, null pointers, unsupported combination) */
  SK_ENOMEM = 2,     /* device workspace allocation failed */
  SK_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  SK_ENAN = 4,       /* NaN/Inf met in an input or a reduction */
  SK_ENOCONV = 5,    /* maxit cycles without reaching tol; best x and info are still written */
  SK_EILLCOND = 6,   /* kappa(T) > stab_tol could not be cured by truncation */
  SK_ETIMEOUT = 7,   /* a bounded device-side wait gave up (persistent basis kernel's grid barrier) */
  SK_EHASH = 8       /* sketch hash found no distinct row in 16 attempts (s too small for zeta) */
} sk_status;

typedef enum { SK_F64 = 0, SK_F32 = 1, SK_BF16 = 2 } sk_dtype;
typedef enum { SK_SPARSE_SIGN = 0, SK_SRHT = 1 } sk_sketch_kind;

/* ------------------------------------------------------------------------
 * Operators.  "All algorithms in this paper access the matrix via products
 * x -> Ax" (§1.2).  Grid operators use nx x ny cells, unknown (ix, iy) at
 * index iy*nx + ix, neighbours E=(ix+1,iy) W=(ix-1,iy) N=(ix,iy+1)
 * S=(ix,iy-1), Dirichlet zero outside.  Arrays passed to constructors are
 * BORROWED: the caller keeps them alive and unchanged while the op exists.
 * ------------------------------------------------------------------------ */
typedef struct sk_op sk_op;

/* (Au)_P = c[0] u_P + c[1] u_E + c[2] u_W + c[3] u_N + c[4] u_S + shift_P u_P.
 * coef: host array of 5 doubles.  shift: device, nx*ny doubles, or NULL. */
sk_status sk_op_stencil5(sk_op** op, int nx, int ny, const double* coef, const double* shift);

/* -div(theta grad u), h^2-scaled: (Au)_P = sum_faces theta_f (u_P - u_Q),
 * theta_f = (theta_P + theta_Q)/2 inside, theta_P on boundary faces.
 * theta: device, nx*ny doubles (> 0). Symmetric positive definite. */
sk_status sk_op_diffusion_var(sk_op** op, int nx, int ny, const double* theta);

/* General sparse A in CSR (0-based, int32 indices), FP64 values, device
 * (borrowed).  The op also builds, on the device, a SELL-32 copy that the
 * kernels read (rows in slices of 32, each slice's entries stored
 * column-major and padded with zeros to its longest row, so that a warp of
 * consecutive rows reads consecutive words); it owns that copy.  Allocates
 * and synchronises the device. */
sk_status sk_op_csr(sk_op** op, int64_t n, int64_t nnz, const int32_t* rowptr,
                    const int32_t* colind, const double* val);

/* A^T as a new op (stencil: E<->W and N<->S swapped; diffusion: itself; both
 * borrow the same arrays).  CSR: the transpose is built on the device (rows
 * sorted by column; owned by the new op, with its own SELL-32 copy;
 * allocates and synchronises the device); the new op's parameter gradient
 * (sk_op_param_grad) is with respect to its own entries. */
sk_status sk_op_transpose(const sk_op* op, sk_op** opT);

/* y = A x in FP64 (x, y: device, n doubles; must not alias). */
sk_status sk_op_apply(const sk_op* op, const double* x, double* y, void* stream);

/* grad = alpha * (gradient of the bilinear form lam^T A x with respect to the
 * operator's parameters).  Not in the paper: the building block of the
 * adjoint of a solve x = A^{-1} b, whose parameter gradient is
 * dL/dparams = -grad(lam^T A x) with A^T lam = dL/dx, i.e. alpha = -1.
 * lam, x: device n doubles; alpha: finite scale.  grad: device doubles, layout by op kind:
 *   diffusion: n entries, d/dtheta_P (interior faces pass half of
 *              (lam_P - lam_Q)(x_P - x_Q) to each cell, boundary faces lam_P x_P);
 *   stencil5:  5 entries d/dc[0..4], then n entries d/dshift_P = lam_P x_P if
 *              the op has a shift;
 *   CSR:       nnz entries d/dval_e = lam_row(e) x_col(e).
 * Asynchronous; no allocation beyond a small reduction buffer. */
sk_status sk_op_param_grad(const sk_op* op, const double* lam, const double* x, double alpha, double* grad,
                           void* stream);

int64_t sk_op_n(const sk_op* op);
void sk_op_destroy(sk_op* op);

/* ------------------------------------------------------------------------
 * Sketches (§2.3).  Sparse sign map (§2.3.2, eq. (sparse-map)): column i of
 * S has zeta entries +-1/sqrt(zeta) in distinct rows chosen by the counter
 * hash H1(seed, i, slot, attempt) (SplitMix64 finalizer of
 * seed*0x9E3779B97F4A7C15 xor (i<<8|slot<<4|attempt); row = (lo32*s)>>32,
 * sign = bit 63).  SRHT (§2.3.1, eq. (SRFT) with Walsh-Hadamard for the DFT):
 * S = sqrt(n_p/s) D H E, n_p = 2^ceil(log2 n), E_i = sign of H1(seed,i,15,0),
 * D = s distinct rows from a partial Fisher-Yates shuffle driven by
 * H1(seed, q, 14, 0).  Output row q of an SRHT sketch is Hadamard row D[q].
 * ------------------------------------------------------------------------ */
typedef struct {
  sk_sketch_kind kind;
  int64_t n;      /* columns of S = rows of the data */
  int s;          /* embedding dimension (rows of S), >= 1 */
  int zeta;       /* nonzeros per column (sparse sign); 0 = ceil(2 ln(1+s/2)); 1..14 */
  uint64_t seed;
} sk_sketch;

/* SB = S * B.  B: device, n x ncols, column-major, leading dimension ldb >= n,
 * element type `dtype`.  SB: device, s x ncols FP64, leading dimension s.
 * FP64 input is accumulated in FP64; FP32/BF16 input in FP32 within a chunk
 * of rows, compensated (Kahan) FP32 across chunks, then FP64 across CTAs. */
sk_status sketch_apply(const sk_sketch* S, const void* B, int64_t ldb, int ncols,
                       sk_dtype dtype, double* SB, void* stream);

/* A reusable plan for one sketch (sparse sign: the row-sorted index tables;
 * SRHT: the signs and sampled rows), built once on the device by
 * sk_sketch_plan_create (allocates the tables; synchronises `stream`, and
 * returns SK_EHASH as sketch_apply does) and applied by sk_sketch_plan_apply
 * to any number of column blocks with the same n: SB = S * B with the
 * arguments, layout and accuracy of sketch_apply.  An apply allocates only
 * when it needs more partial-sum workspace than every earlier apply on the
 * plan (then it synchronises `stream` first).  Applies on one plan share
 * that workspace: issue them on one stream, or serialise them.
 * sk_sketch_plan_destroy frees the plan (synchronous; the plan's work must
 * be finished or ordered before it). */
typedef struct sk_sketch_plan sk_sketch_plan;
sk_status sk_sketch_plan_create(const sk_sketch* S, sk_sketch_plan** plan, void* stream);
sk_status sk_sketch_plan_apply(sk_sketch_plan* plan, const void* B, int64_t ldb, int ncols, sk_dtype dtype,
                               double* SB, void* stream);
void sk_sketch_plan_destroy(sk_sketch_plan* plan);

/* sketch_apply for the sparse sign sketch without any device allocation.
 * The paper has no counterpart: this is a deployment variant for callers
 * that cannot call cudaMalloc on their hot path (plugins inside another
 * framework's engine, which owns the memory budget and where cudaMalloc can
 * synchronise the device; latency-critical loops that must not risk an
 * allocation's cost or an out-of-memory failure mid-run).  Arguments,
 * layout and results are those of sketch_apply (SK_SPARSE_SIGN only).
 * Scratch: one file-scope device array of 32 MiB in libsk, held by every GPU
 * that loads the library until the process exits.  A sketch needing more
 * (about nchunks*(s+1)*4 + nchunks*1024*zeta*2 + partial sums, nchunks =
 * ceil(n/1024)) returns SK_EINVAL with the byte count; nothing is launched.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the previous call's contents: calls that overlap on the GPU (different
 * streams, or host threads) race and must be serialised by the caller.
 * Synchronises `stream` before returning (hash status check). */
sk_status sketch_apply_noalloc(const sk_sketch* S, const void* B, int64_t ldb, int ncols,
                               sk_dtype dtype, double* SB, void* stream);

/* ------------------------------------------------------------------------
 * Solver options and diagnostics.
 * ------------------------------------------------------------------------ */
typedef enum {
  SK_BASIS_ARNOLDI = 0,   /* k-truncated Arnoldi with classical Gram-Schmidt (§1.2.2, §4.2) */
  SK_BASIS_CHEBYSHEV = 1  /* shifted-and-scaled Chebyshev recurrence (§4.3, eq. (Chebrecurse)) */
} sk_basis_kind;

typedef struct {
  sk_sketch_kind sketch;   /* default SK_SPARSE_SIGN */
  int zeta;                /* 0 = ceil(2 ln(1+d)) (§2.3.2) */
  uint64_t seed;           /* sketch seed, default 7 */
  double stab_tol;         /* kappa(T) threshold (§3.4, §5.3); <= 0 = 1e14 (F64), 2e6 (F32), 1e2 (BF16) */
  int maxit;               /* restart cycles, default 10000 */
  sk_dtype basis;          /* basis storage and SpMV precision, default SK_F64 */
  int cgs_passes;          /* Gram-Schmidt passes, 1 or 2 (default 2: "double Gram-Schmidt");
                              1 needs an FP64 basis (SK_EINVAL otherwise: the one-pass norm
                              update ||m||^2 - ||h||^2 is unstable in FP32/BF16) */
  double tau;              /* sRR convergence tolerance for nconv (default 1e-8) */
  int symmetric;           /* sRR: keep real parts of lambda and x (§6.8) */
  double breakdown;        /* ||w_j|| <= breakdown*||A b_{j-1}|| ends the basis; <=0 = 1e-13 (F64) / 1e-6 */
  int use_graph;           /* capture each restart cycle in a CUDA graph (default 1) */
  int persistent;          /* grid operators: build the basis in one cooperative kernel
                              with bounded grid barriers (1), or 3 launches per step (0, default);
                              the persistent kernel covers k <= 4 with FP32/FP64 storage, other
                              cases take the 3-launch path */
  int batch_workers;       /* sgmres_solve_batched: concurrent jobs (threads x streams); 0 = 16 */
  sk_basis_kind basis_kind; /* default SK_BASIS_ARNOLDI.  SK_BASIS_CHEBYSHEV: no inner products;
                              needs the spectrum inside the rectangle [c - dx, c + dx] x [-dy, dy]
                              (max(dx, dy) > 0); k, cgs_passes, breakdown and persistent are
                              ignored; supported by trunc_arnoldi_basis, sgmres_solve and
                              sgmres_solve_batched (srr_eigs: SK_EINVAL) */
  double cheb_c, cheb_dx, cheb_dy;
  int barrier_spins;       /* persistent kernel: polls of a grid barrier before it gives up and
                              the call returns SK_ETIMEOUT; 0 = default (2^22, ~0.1 s), -1 = give
                              up at the first poll (exercises the timeout path) */
  int iter_chunk;          /* sgmres_solve / sgmres_solve_batched: 0 (default) = Algorithm 1 with
                              all d columns per cycle.  > 0 = iterative sGMRES (§5.2, §5.3): the
                              basis grows iter_chunk columns at a time, each chunk is sketched
                              and appended to the QR of S A B, and the cycle ends at the first
                              prefix j with ||(I - U_j U_j^T) g|| <= (tol ||b|| / ||r_0||) ||g||
                              (g = S r_0: the reduction that would meet tol), or when the kappa
                              estimate exceeds stab_tol, the basis breaks down, or j = d; the
                              solve uses exactly that prefix.  A positive multiple of 16, at most
                              1024; truncated-Arnoldi basis only (SK_EINVAL otherwise); no CUDA
                              graph and no persistent kernel; the host reads one flag per chunk */
  double srr_trunc_tol;    /* sRR (srr_eigs, srr_basis, srr_restarted): <= 0 (default) = Algorithm 2's
                              reduction (QR of S B, M-hat = T^{-1} U^T S A B); > 0 = the stabilized
                              form of §6.5 eq. (qz): thin SVD S B = U Sigma V^T (column-pivoted
                              Householder QR, then one-sided Jacobi on R^T), keeping the singular
                              values with sigma_1 / sigma_i <= srr_trunc_tol, and the eigenproblem
                              (U_r^T S A B V_r) z = theta Sigma_r z */
  int pipeline;            /* sgmres_solve with a captured cycle (use_graph), the truncated-Arnoldi
                              basis with 3 launches per step or the Chebyshev basis: 1 (default) =
                              sketch each finished block of 16 basis columns (Chebyshev: after its
                              column norms) and add the panels it completes to the QR of S A B on
                              a second, lower-priority stream while the basis passes continue (same
                              arithmetic, overlapped); 0 = one phase after another */
  int batch_mode;          /* sgmres_solve_batched: 0 (default) = grouped where supported, else
                              worker threads; 1 = grouped (SK_EINVAL where unsupported); 2 = worker
                              threads.  Grouped: every launch advances one phase of all resident
                              jobs (sparse sign sketch, truncated-Arnoldi basis, FP32 or FP64
                              storage, s <= 640, iter_chunk = 0) */
  long long batch_elems;   /* grouped batches: jobs are admitted, largest first, while the resident
                              systems' sizes n sum to at most this (at least one job is resident);
                              0 = 2^22 */
} sk_opts;

void sk_opts_default(sk_opts* o);

typedef struct {
  int cycles;          /* restart cycles run */
  int matvecs;         /* products with A (basis + residuals) */
  int d_used;          /* basis columns in the last cycle (iter_chunk > 0: the prefix its solve used) */
  int width;           /* columns kept by the kappa truncation in the last cycle */
  double relres;       /* final ||b - A x|| / ||b|| (FP64) */
  double rhat_est;     /* last sketched residual estimate (eq. (sgmres-rhat)) */
  double kappa_T_max;  /* largest kappa(T) estimate over cycles */
  float ms[6];         /* device ms summed over cycles (CUDA events on the call's stream):
                          [0] residual r = b - A x, [1] basis, [2] sketches (g = S r, S B),
                          [3] small dense solve, [4] solution update, [5] whole call.
                          pipelined cycles: [2] is the sketch and QR work left after the
                          basis passes end (the part not overlapped), [3] the LS solve.
                          iter_chunk > 0: [1] is the whole chunk loop (basis, S B, QR, the
                          per-chunk test), [2] is g = S r and [3] the final solve */
  long long launches;  /* CUDA kernels launched by the call */
} sk_info;

/* ------------------------------------------------------------------------
 * k-truncated Arnoldi basis (§1.2.2 eq. (partorth); Algorithm 1 loop with
 * double Gram-Schmidt).  b_1 = r0/||r0||; for j >= 2 w_j is A b_{j-1}
 * orthogonalised against b_{j-1..j-k} in `cgs_passes` classical passes.
 * With opts->basis_kind = SK_BASIS_CHEBYSHEV the columns are instead the
 * Chebyshev recurrence of §4.3 eq. (Chebrecurse), each rescaled to unit
 * norm, and Hbar is tridiagonal.
 *   A: op; r0: device n doubles; d >= 1; 1 <= k <= d.
 *   B: device, n x (d+1) of `basis_dtype`, ld = n (column d+1 = b_{d+1},
 *      needed for the Arnoldi relation AB = B_{d+1} Hbar).
 *   Hbar: device (d+1) x d FP64 col-major (ld d+1) or NULL: A b_j =
 *      sum_i Hbar[i,j] b_i (k+1 nonzeros per column).
 *   S, SB, SAB: optional (NULL) sketch and device outputs s x d FP64:
 *      SB = S [b_1..b_d], SAB = S [A b_1 .. A b_d].
 *   d_used: host int, columns actually built (< d on breakdown).
 * ------------------------------------------------------------------------ */
sk_status trunc_arnoldi_basis(const sk_op* A, const double* r0, int d, int k, sk_dtype basis_dtype,
                              void* B, double* Hbar, const sk_sketch* S, double* SB, double* SAB,
                              const sk_opts* opts, int* d_used, void* stream);

/* ------------------------------------------------------------------------
 * Restarted sGMRES (Algorithm 1, §3.3, §3.5): solve A x = b.
 *   b: device n doubles; x: device n doubles, in: initial guess, out: solution.
 *   d: basis size; k: truncation; s: sketch rows (>= d+1); tol: target
 *   ||b - A x||/||b|| (FP64, checked after every cycle).
 *   opts: NULL = defaults; info: host or NULL.
 * Returns SK_OK (converged), SK_ENOCONV (best x written), or an error.
 * ------------------------------------------------------------------------ */
sk_status sgmres_solve(const sk_op* A, const double* b, double* x, int d, int k, int s, double tol,
                       const sk_opts* opts, sk_info* info, void* stream);

/* Reusable solver for one operator and shape (not in the paper): the
 * buffers, the sketch plan, the side streams and the captured cycle graph of
 * sgmres_solve, built once by sgmres_plan_create and reused by every
 * sgmres_plan_solve (which copies b and the initial guess x into the plan's
 * own vectors, runs the cycles, and copies the iterate back into x whatever
 * the status).  Each solve computes exactly what sgmres_solve computes on the
 * same arguments; it skips the per-call setup (plan build, allocations, graph
 * capture).  A must outlive the plan; one solve at a time per plan; the
 * plan's device memory is released by sgmres_plan_destroy, which first waits
 * for its streams.  Errors: as sgmres_solve; the create call validates d, k,
 * s like sgmres_solve (SK_EINVAL) and returns SK_ENOMEM if the buffers do not
 * fit. */
typedef struct sk_solver sk_solver;
sk_status sgmres_plan_create(const sk_op* A, int d, int k, int s, const sk_opts* opts, sk_solver** plan,
                             void* stream);
sk_status sgmres_plan_solve(sk_solver* plan, const double* b, double* x, double tol, sk_info* info, void* stream);
void sgmres_plan_destroy(sk_solver* plan);

/* Device workspace in bytes that sgmres_solve(A, ., ., d, k, s, ., opts)
 * allocates (stream-ordered, released before it returns), for callers that
 * budget memory: the basis n x (d+1) in the basis precision, the Arnoldi
 * coefficients, the sketch's index tables and partial sums, the s x (d+1)
 * sketches and the n-vectors of the residual; each buffer rounded up to
 * 256 bytes (the allocator may reserve more).  Depends on the current
 * device's SM count.  0 for invalid arguments.  Not counted: the FP32 copies
 * of an operator's arrays that FP32/BF16 solves make once and the operator
 * keeps (4 bytes per shift/theta/value entry). */
size_t sk_workspace_bytes(const sk_op* A, int d, int k, int s, const sk_opts* opts);

/* ------------------------------------------------------------------------
 * Batched restarted sGMRES: nsys independent systems A[i] with nrhs
 * right-hand sides each (not in the paper: many small problems at once).
 *   A: host array of nsys ops; b, x: host arrays of nsys*nrhs device
 *   pointers (job i*nrhs + r = system i, right-hand side r); each x is the
 *   initial guess in, the solution out.  per_job: host array of nsys*nrhs
 *   statuses (or NULL).  job_info: host array of nsys*nrhs sk_info, each the
 *   job's own diagnostics as sgmres_solve reports them (or NULL).  info:
 *   aggregate (cycles and matvecs summed, relres the worst job, ms[5] =
 *   wall time).
 * Grouped batches (opts->batch_mode 0 where supported, or 1): jobs are
 *   admitted largest first while the resident systems' n sum to at most
 *   opts->batch_elems; every kernel launch runs one phase of the restart
 *   cycle for all resident jobs (a flat map of each job's blocks for the
 *   n-sized kernels, one grid row per job for the small dense problems),
 *   and the host reads one row of scalars per job and cycle, then retires
 *   and admits jobs.  Each job computes what sgmres_solve computes on its
 *   inputs, bit for bit.  info->ms[0..4] and launches: device time and
 *   kernel launches of the grouped phases; a job's ms[0..4] and launches
 *   are those of the grouped cycles it took part in (shared with the jobs
 *   resident beside it), its ms[5] the wall time from admission to exit.
 *   Workspace: one slab of the s x (d+1) problem per slot plus each
 *   resident job's n-sized buffers (the basis n x (d+1) dominates), so
 *   about batch_elems x (d+1) x (basis bytes + 1) bytes at the budget.
 *   `stream` carries all launches.  opts->persistent and opts->use_graph
 *   are ignored.
 * Worker threads (opts->batch_mode 2, or 0 where grouped is unsupported):
 *   jobs run on opts->batch_workers host threads with one stream each,
 *   largest systems first, each as sgmres_solve with eager launches
 *   (opts->use_graph ignored); `stream` is joined before and after; ms[0..4]
 *   summed over jobs.
 * Blocks until done.  Returns SK_OK if every job converged, else the first
 * failing job's status.
 * ------------------------------------------------------------------------ */
sk_status sgmres_solve_batched(int nsys, const sk_op* const* A, int nrhs, const double* const* b,
                               double* const* x, int d, int k, int s, double tol, const sk_opts* opts,
                               sk_status* per_job, sk_info* job_info, sk_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Sketched Rayleigh-Ritz (Algorithm 2, §6.3-§6.4): nev eigenpairs of A with
 * largest real part from a k-truncated Arnoldi basis of dimension d started
 * at w1 (device n doubles; Algorithm 2 draws it as randn).
 *   lam_re, lam_im, rhat: host arrays of nev doubles (rhat = eq.
 *   (srr-resid-est)).  X_re, X_im: device n x nev FP64 (ld n), unit-norm
 *   Ritz vectors B y_i (X_im may be NULL).  nconv: host, count with rhat <= tau.
 * ------------------------------------------------------------------------ */
sk_status srr_eigs(const sk_op* A, const double* w1, int nev, int d, int k, int s, const sk_opts* opts,
                   double* lam_re, double* lam_im, double* X_re, double* X_im, double* rhat,
                   int* nconv, sk_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Sketched Rayleigh-Ritz on a caller's basis (§6.3: sRR needs only a basis
 * B and the products A B; §6.5 for the stabilized form).
 *   B: device n x d, column-major, leading dimension ldb >= n, `dtype`; A B
 *   is formed column by column on the GPU (FP64).  s >= d sketch rows; opts:
 *   sketch kind/zeta/seed, tau, symmetric, srr_trunc_tol (> 0: stabilized).
 *   Outputs as srr_eigs; rank (host int or NULL): the singular values the
 *   stabilized form kept (d for Algorithm 2).  3 <= d <= 232, nev <= 32.
 *   SK_EILLCOND if the stabilized form keeps fewer than max(3, nev).
 * ------------------------------------------------------------------------ */
sk_status srr_basis(const sk_op* A, const void* B, int64_t ldb, int d, sk_dtype dtype, int nev, int s,
                    const sk_opts* opts, double* lam_re, double* lam_im, double* X_re, double* X_im,
                    double* rhat, int* nconv, int* rank, void* stream);

/* ------------------------------------------------------------------------
 * Restarted sRR (§7.2) on block Chebyshev bases (§7.5).  The paper leaves
 * the restart strategy open; this library restarts from the Krylov space of
 * the current Ritz vectors, built by the block Chebyshev recurrence for the
 * unwanted part of the real spectrum, as follows.  X_0 = Omega (device,
 * n x b FP64).  Restart t: Q = orth(X_t) (shifted CholeskyQR3); with
 * filter_degree = m > 0, Q = orth(T_m((A - c)/rho) Q), a degree-m
 * Chebyshev filter for the same interval (Q stays a block of the Krylov
 * space of X_t); B_0 = Q, B_1 = (A - c) B_0 / (2 rho),
 * B_j = ((A - c) B_{j-1} - (rho/4) B_{j-2}) / rho for the interval [lo, cut_t]
 * (c its centre, rho its half-width; cut_0 = hi, then the real part of the
 * b-th Ritz value of restart t-1); the d = b p columns of B_0..B_{p-1}
 * scaled to unit norm; the stabilized sRR of §6.5 (srr_trunc_tol, default
 * 1e13 here) with a fresh sparse sketch (seed opts->seed + t, s = 2d); X_{t+1}
 * = the real parts, then the imaginary parts, of the b leading Ritz vectors
 * (the first b with norm > 1e-10).  Stops when the nev leading residual
 * estimates are <= opts->tau, or after max_restarts.
 *   1 <= nev <= b <= 32, 3 <= b p <= 232, lo < hi (lo below the spectrum).
 *   Outputs: the nev leading pairs of the last restart (as srr_eigs);
 *   restarts (host int): restarts run; history (host, max_restarts doubles or
 *   NULL): each restart's largest estimate over the nev leading pairs.
 *   Returns SK_OK when all nev estimates are <= tau, else SK_ENOCONV.
 * ------------------------------------------------------------------------ */
sk_status srr_restarted(const sk_op* A, const double* Omega, int b, int p, int nev, double lo, double hi,
                        int max_restarts, int filter_degree, const sk_opts* opts, double* lam_re, double* lam_im,
                        double* X_re, double* X_im, double* rhat, int* nconv, int* restarts, double* history, void* stream);

const char* sk_last_error(void);
const char* sk_status_string(sk_status st);

#ifdef __cplusplus
}
#endif
#endif /* SK_H */
