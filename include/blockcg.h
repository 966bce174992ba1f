/*
 * blockcg.h -- C ABI of libblockcg.so: block-CGrQ on one GPU for the even-odd
 * improved-staggered (HISQ-type) normal operator.
 *
 * Method: Clark, Strelchenko, Vaquero, Wagner, Weinberg, "Pushing memory
 * bandwidth limitations through efficient implementations of Block-Krylov
 * space solvers on GPUs" (arXiv:1710.09745).  Operator: Eq. 2 and Sec. 3.2;
 * solver: Algorithm 1 (blockCGrQ), Algorithm 2 (thin QR), Algorithm 3 (block
 * reliable updates); kernels: Sec. 6.2 (block stencil), 5.3 (streaming
 * multi-BLAS), 5.4 (reduction multi-BLAS).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Lattice: dims = {Lx, Ly, Lz, Lt}, every extent even and >= 2.  V = Lx*Ly*Lz*Lt,
 *  Vh = V/2.  Lexicographic site index i = x + Lx*(y + Ly*(z + Lz*t)); parity
 *  (x+y+z+t) & 1; checkerboard index i >> 1.
 *
 *  Links: complex128 (interleaved re, im doubles) [4][V][3][3]: direction
 *  mu = x,y,z,t, lexicographic site, 3x3 matrix row-major with the row index
 *  the colour of the result.  F_mu(x) (fat) connects x to x+mu, G_mu(x) (long)
 *  connects x to x+3mu and includes its coefficient (e.g. -1/24).  Staggered
 *  phases eta_mu(x) = (-1)^(x_0+...+x_{mu-1}) are NOT in the links; the
 *  library applies them.
 *
 *  Operator: (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu)
 *      - F_mu(x-mu)^dag psi(x-mu) + G_mu(x) psi(x+3mu) - G_mu(x-3mu)^dag psi(x-3mu) ],
 *  periodic (optionally antiperiodic in t), and A = m^2 - D_eo D_oe on even
 *  sites, the Hermitian positive-definite Schur normal operator of
 *  M = m + D (Eq. 2 with the anti-Hermitian sign on backward hops).
 *
 *  Spinor blocks (user layout): complex128 [n_rhs][Vh][3], one parity,
 *  checkerboard-indexed; column j is right-hand side j.  1 <= n_rhs <= 64.
 *
 *  Memory: the library allocates no device memory.  All device buffers
 *  (internal gauge copy, workspace, inputs, outputs) are owned by the caller;
 *  pointers must stay valid while the handle uses them.  Every device pointer
 *  must be 16-byte aligned.
 *
 *  Streams: all work is enqueued on the stream given to blockcg_create.
 *  Calls return after enqueueing, except blockcg_solve / blockcg_solve_cg,
 *  which synchronise that stream to read the convergence status and fill the
 *  statistics.
 *
 *  Errors: every call returns a status; nothing is thrown across the ABI.
 *  blockcg_last_error() gives a one-line description of the latest failure
 *  on a handle.
 */
#ifndef BLOCKCG_H
#define BLOCKCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct blockcg_ctx* blockcg_t;

typedef enum {
  BLOCKCG_OK = 0,
  BLOCKCG_ERR_ARG = 1,           /* bad argument (null pointer, bad size, odd dims, ...) */
  BLOCKCG_ERR_CUDA = 2,          /* a CUDA call failed */
  BLOCKCG_ERR_NOMEM = 3,         /* workspace or gauge storage too small / missing */
  BLOCKCG_ERR_BREAKDOWN = 4,     /* Cholesky pivot <= 0 in a thin QR or in P^dag A P
                                    (e.g. linearly dependent right-hand sides) */
  BLOCKCG_ERR_NONFINITE = 5,     /* NaN or Inf met in a Gram matrix */
  BLOCKCG_ERR_NOT_CONVERGED = 6, /* max_iter reached; X holds the current iterate */
  BLOCKCG_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up */
} blockcg_status;

/* Precision of the solve (Sec. 5 storage formats, Algorithm 3).  In every
 * form the reliable updates of Algorithm 3 (solution accumulator Y, sources
 * B, true residual R = B - A Y with its own stencil, thin QR of R) and all
 * N x N algebra run in native FP64.
 *  F64         FP64-accurate iterations: P, Q, AP, T, the update X and the
 *              links stored as double-float pairs (two FP32 words per real,
 *              ~48 significant bits) with error-free-transformation
 *              double-float arithmetic on the FP32 pipes.
 *  F64_NATIVE  native FP64 storage and arithmetic in the iterations too (slow
 *              on GPUs with a reduced FP64 rate; for verification).
 *  MIXED_F32   sloppy P, Q, AP, T and links in FP32 with FP32 arithmetic; X
 *              in double-float.
 *  MIXED_F16   as MIXED_F32 with P, Q, AP, T and links stored as IEEE FP16
 *              (2^4 x value, see below) and FP32 arithmetic.
 *  MIXED_BF16  as MIXED_F16 with bfloat16 storage (no factor).
 *  With 16-bit storage the sloppy recursion can stagnate (bfloat16's 8-bit
 *  significand) or drift (FP16 on ill-conditioned problems) before the
 *  residual drops by ru_delta, so ru_every defaults to 10 for both 16-bit
 *  forms when the caller leaves it 0.  In every form a reliable update also
 *  happens when the iterated residual grows 100x above the true residual of
 *  the last update.
 *  FP16 storage keeps 2^4 times the value: the block vectors of the
 *  iteration are normalised (components ~ (3 V/2)^-1/2), so the fixed
 *  power-of-two factor keeps them clear of FP16's subnormal range while
 *  leaving ~10^5 of headroom for the growth of the search block P, without
 *  per-site scale arrays.  Data given to the operator entry points of a
 *  MIXED_F16 handle must fit |value| < 4000.  */
typedef enum {
  BLOCKCG_PREC_F64 = 0,
  BLOCKCG_PREC_F64_NATIVE = 1,
  BLOCKCG_PREC_MIXED_F32 = 2,
  BLOCKCG_PREC_MIXED_F16 = 3,
  BLOCKCG_PREC_MIXED_BF16 = 4
} blockcg_prec;

typedef struct {
  int max_iter;        /* iteration limit (default 100000) */
  double ru_delta;     /* reliable update when the max relative iterated residual
                          fell by this factor since the last one (default 0.1;
                          0 disables; Sec. 6 and 7.1) */
  int ru_every;        /* >0: also a reliable update every ru_every iterations */
  blockcg_prec prec;   /* default BLOCKCG_PREC_F64 */
  int antiperiodic_t;  /* 1: antiperiodic boundary in t (default 0) */
  int check_every;     /* host polls the device status every this many
                          iterations (0: chosen from the lattice size) */
  int profile;         /* 1: time every stencil launch of a solve with CUDA
                          events (fills the ms_stencil fields of the stats) */
  int dslash_variant;  /* stencil kernel: 0 = autotuned on first use (default);
                          else R in {1, 2, 4, 8} right-hand sides per thread,
                          plus one of: 256 for the bulk-copy (TMA) pipelined
                          kernel, 512 for the per-thread cp.async prefetch
                          kernel, 4096 for the plain kernel on a persistent
                          grid of contiguous site ranges, 8192 for the
                          tensor-core stencil (mma.sync): in the F64 form
                          double-float values split into bf16 slices with
                          exact products (N = 16 or 32 with a workspace set;
                          the cp.async kernel otherwise), in the FP16 and
                          bfloat16 forms the stored values themselves (N = 16
                          or 32 with full links; the plain kernel
                          otherwise).  Other values: BLOCKCG_ERR_ARG */
  int link_recon;      /* iteration links of the 32- and 16-bit forms: 0 = all 18
                          reals per link (default); 12 = the first two rows only,
                          the third rebuilt in the stencil as conj(row0 x row1)
                          divided by the link's scale.  Needs every fat link to
                          be c_f U and every long link c_l U with U in SU(3) and
                          c_f, c_l real constants (e.g. 1 and -1/24), which
                          blockcg_load_gauge checks (BLOCKCG_ERR_ARG otherwise);
                          only with MIXED_F32 / MIXED_F16 / MIXED_BF16 (the
                          FP64 links of the reliable updates stay complete) */
  long long wait_limit_ns; /* watchdog of bounded device-side waits (the
                          bulk-copy stencil's mbarrier waits): a thread block
                          gives up waiting once this many nanoseconds have
                          passed since it started, and the call reports
                          BLOCKCG_ERR_TIMEOUT; 0 = 4 s (default).  Copies
                          already issued are always waited for (up to 4 s)
                          before a kernel returns. */
} blockcg_params;

typedef struct {
  int iters;               /* iterations of Algorithm 1 (per RHS for solve_cg: the sum) */
  int reliable_updates;    /* Algorithm 3 updates, including convergence checks */
  double true_rel_res_max; /* max_i |b_i - A x_i| / |b_i| at exit (true residual) */
  double ms_total;         /* device time of the solve (CUDA events) */
  long long launches;      /* kernel launches the solve enqueued (gated ones included) */
  long long n_stencil;     /* launches of the iteration's stencil (params.profile) */
  double ms_stencil;       /* their summed device time (params.profile) */
  long long n_stencil_fine;  /* launches of the full-precision stencil (params.profile) */
  double ms_stencil_fine;    /* their summed device time (params.profile) */
  double ms_gram;          /* params.profile: Gram partials + reductions (Sec. 6.4) */
  double ms_stream;        /* params.profile: streaming block BLAS (Sec. 6.3) */
  double ms_dense;         /* params.profile: N x N algebra on the device */
  int stencil_variant;     /* the iteration stencil's kernel choice (the
                              params.dslash_variant encoding, plus 1024 for
                              two-row links) */
  double* true_rel_res;    /* set by the caller: a host array of n_rhs doubles
                              that receives |b_i - A x_i| / |b_i| per right-hand
                              side at exit (the true residual of each column,
                              computed in native FP64), or NULL to skip.  The
                              library writes through it and leaves the pointer
                              itself unchanged.  Entries are NaN if the solve
                              failed before its first true-residual check. */
} blockcg_stats;

/* Fill *p with the defaults listed above. */
void blockcg_default_params(blockcg_params* p);

/* Create a handle for an Lx x Ly x Lz x Lt lattice (Sec. 3.2), quark mass
 * `mass` (finite), parameters p (NULL: defaults) and stream (cudaStream_t,
 * NULL = legacy default stream).  Allocates host memory for the handle only.
 * Errors: BLOCKCG_ERR_ARG for odd or < 2 extents, V/2 >= 2^31, non-finite
 * mass, bad parameters. */
blockcg_status blockcg_create(blockcg_t* out, const int dims[4], double mass,
                              const blockcg_params* p, void* stream);

/* Bytes of device memory the caller must provide to blockcg_load_gauge. */
size_t blockcg_gauge_bytes(blockcg_t h);

/* Reorder the caller's links (device complex128 [4][V][3][3] each, layout
 * above) into `storage` (device, >= blockcg_gauge_bytes): per output parity
 * the 16 hop matrices of Eq. 2 with staggered phases, the factor 1/2, the
 * boundary sign and the backward-hop dagger and minus sign folded in, in
 * the storage formats the precision needs.  The caller may free fat/lng once
 * the stream has passed this call.  With params.link_recon = 12 it first
 * checks on the device that all fat links are c_f U and all long links c_l U
 * (U unitary with determinant 1, c real, taken from the first link of each
 * kind; tolerance 1e-10 relative) and synchronises the stream to read the
 * result.  Errors: ERR_ARG (null, or links not of that form with
 * link_recon = 12), ERR_NOMEM (storage too small), ERR_CUDA. */
blockcg_status blockcg_load_gauge(blockcg_t h, const void* fat, const void* lng, void* storage,
                                  size_t storage_bytes);

/* Bytes of device workspace needed by any call on this handle with up to
 * n_rhs right-hand sides. */
size_t blockcg_workspace_bytes(blockcg_t h, int n_rhs);

/* Hand the handle a caller-owned device workspace (>= the size above for the
 * largest n_rhs used).  Errors: ERR_ARG, ERR_NOMEM. */
blockcg_status blockcg_set_workspace(blockcg_t h, void* ws, size_t bytes);

/* out = D_{p,1-p} in: the block stencil of Sec. 6.2 (Eq. 2 hopping term),
 * in on parity 1-out_parity, out on parity out_parity, both user layout
 * [n_rhs][Vh][3] complex128 on the device, computed in the handle's
 * precision.  Errors: ERR_ARG, ERR_NOMEM (no workspace/gauge), ERR_CUDA. */
blockcg_status blockcg_dslash(blockcg_t h, const void* in, void* out, int n_rhs, int out_parity);

/* out = A in = m^2 in - D_eo D_oe in on even sites (Sec. 3.2), user layout.
 * in and out must not overlap.  Errors as blockcg_dslash. */
blockcg_status blockcg_apply_MdagM(blockcg_t h, const void* in, void* out, int n_rhs);

/* Gradient of a real loss L(x) of the solution x = A^-1 phi with respect to
 * the fat and long links, in the convention G = dL/dRe(u) + i dL/dIm(u) per
 * link entry u (so dL = Re sum conj(G) du; the convention of complex
 * automatic differentiation).  The paper only solves; this is the link part
 * of the adjoint of a differentiable solve (operator of Sec. 3.2, Eq. 2).
 *
 * X: the solution block x; Lam: the adjoint block lam = A^-1 g, g the
 * gradient of L with respect to x (a second solve with the same handle,
 * A being Hermitian).  Both device, user layout [n_rhs][Vh][3] on even sites.
 * With y = D_oe x and mu = D_oe lam (computed here in native FP64 on the
 * handle's FP64 links):
 *   dL = Re[lam^dag dD_eo y] + Re[x^dag dD_eo mu], so for the link U_mu(z)
 *   (fat: k = 1, long: k = 3; c = eta_mu(z) s / 2, s the hop's boundary sign)
 *   z even: G =  c sum_i [lam_i(z) y_i(z+k mu)^dag + x_i(z) mu_i(z+k mu)^dag]
 *   z odd:  G = -c sum_i [y_i(z) lam_i(z+k mu)^dag + mu_i(z) x_i(z+k mu)^dag].
 * grad_fat, grad_long: device complex128 [4][V][3][3] (the links' layout),
 * overwritten; either may be NULL to skip it.  Uses the workspace (n_rhs
 * within its size); enqueues and returns.  Errors: ERR_ARG, ERR_NOMEM,
 * ERR_CUDA. */
blockcg_status blockcg_link_grad(blockcg_t h, const void* X, const void* Lam, int n_rhs,
                                 void* grad_fat, void* grad_long);

/* K = X^dag Y (block cDotProduct, Sec. 6.4, Eq. 4): X, Y even-site blocks in user
 * layout; K device complex128 [n_rhs][n_rhs] row-major (K[i][j] = X_i^dag Y_j). */
blockcg_status blockcg_block_cdot(blockcg_t h, const void* X, const void* Y, int n_rhs, void* K);

/* Y = Y + X a (block caxpy, Sec. 6.3, Eq. 3): a device complex128 [n_rhs][n_rhs]
 * row-major (a[i][j] multiplies column i of X into column j of Y). */
blockcg_status blockcg_block_caxpy(blockcg_t h, const void* X, const void* a, void* Y, int n_rhs);

/* Thin QR of Algorithm 2: H = M^dag M, R^dag R = H (Cholesky), Q = M R^-1.
 * M, Q user layout (may alias); R device complex128 [n_rhs][n_rhs] row-major,
 * upper triangular with real positive diagonal.  ERR_BREAKDOWN if H is not
 * numerically positive definite. */
blockcg_status blockcg_thin_qr(blockcg_t h, const void* M, void* Q, void* R, int n_rhs);

/* Solve A X = B with blockCGrQ (Algorithm 1) and block reliable updates
 * (Algorithm 3) until max_i |b_i - A x_i| / |b_i| <= tol, verified on the true
 * residual.  B, X device, user layout; X holds the initial guess on entry and
 * the solution on exit.  st may be NULL.  Synchronises the stream.
 * Errors: ERR_ARG (tol <= 0, n_rhs out of range), ERR_NOMEM, ERR_BREAKDOWN,
 * ERR_NONFINITE, ERR_NOT_CONVERGED (X = current iterate), ERR_CUDA. */
blockcg_status blockcg_solve(blockcg_t h, const void* B, void* X, int n_rhs, double tol,
                             blockcg_stats* st);

/* Baseline of Sec. 7.1: n_rhs independent conjugate-gradient solves, one
 * right-hand side after the other, on the same operator kernels at N = 1 and
 * the same precision.  Arguments and errors as blockcg_solve; st->iters is
 * the sum over right-hand sides. */
blockcg_status blockcg_solve_cg(blockcg_t h, const void* B, void* X, int n_rhs, double tol,
                                blockcg_stats* st);

/* Time the block stencil of Sec. 6.2 alone (the measurement of Fig. 1):
 * `reps` back-to-back launches of out_parity = D in on n_rhs right-hand sides
 * in the iteration's precision (full precision if fine != 0), on internal
 * workspace buffers (whose contents are overwritten), bracketed by CUDA
 * events on the handle's stream.  *ms_per_launch receives the mean device
 * time per launch.  Synchronises the stream.  Errors: ERR_ARG, ERR_NOMEM,
 * ERR_CUDA. */
blockcg_status blockcg_bench_dslash(blockcg_t h, int n_rhs, int fine, int reps,
                                    double* ms_per_launch);

/* ---- Many right-hand sides: block width chosen by measurement ------------
 *
 * Sec. 7.1 solves 192 sources in blocks of N, and Sec. 7.2 finds that the
 * best N depends on the problem and the machine ("bigger is not necessarily
 * better": fewer iterations against costlier ones).  blockcg_solve_many
 * solves m_rhs right-hand sides (any count >= 1) in consecutive blocks of
 * `width` columns with blockcg_solve.  width = 0 picks the width itself:
 * unless the tuning cache (below) already holds a choice for this lattice,
 * precision form, mass, tolerance and device, it solves the first blocks at
 * the candidate widths 8, 16 and 32 in turn (each a real solve of distinct
 * right-hand sides, after tuning the stencil for that width, so no work is
 * thrown away), takes the width with the least device time per right-hand
 * side, solves the rest at that width and stores the choice in the cache.
 * Candidates must fit the workspace (blockcg_workspace_bytes); with fewer
 * than 8 right-hand sides all are solved in one block.
 * B, X: device, user layout [m_rhs][Vh][3]; X holds the initial guesses on
 * entry and the solutions on exit.  Synchronises the stream.
 * Errors: as blockcg_solve (the first failing block's status; later blocks
 * are not solved), ERR_ARG (width < 0 or > 64), ERR_NOMEM (width beyond the
 * workspace). */
typedef struct {
  int width;                 /* width of the blocks after the exploration */
  int from_cache;            /* 1: the width came from the tuning cache */
  int blocks;                /* blocks solved */
  long long iters_total;     /* Algorithm 1 iterations summed over blocks */
  double ms_total;           /* device time of all block solves */
  double true_rel_res_max;   /* max over all right-hand sides */
  int n_candidates;          /* widths timed in the exploration (<= 8) */
  int cand_width[8];
  double cand_ms_per_rhs[8]; /* device time per right-hand side of each */
  double* true_rel_res;      /* set by the caller: host array of m_rhs
                                doubles for the per-RHS true residuals, or NULL */
} blockcg_many_stats;

blockcg_status blockcg_solve_many(blockcg_t h, const void* B, void* X, int m_rhs, double tol,
                                  int width, blockcg_many_stats* st);

/* Persist this handle's tuning choices (stencil kernel per storage kind and
 * width, block width of blockcg_solve_many) in the text file `path` (a JSON
 * object of "key": integer lines; created if absent, shared by handles and
 * processes that name it; entries are keyed by lattice, kind, width and
 * device name).  NULL or "" turns persistence off.  Choices already in the
 * file are used instead of timing.  Errors: ERR_ARG (null handle). */
blockcg_status blockcg_set_tune_cache(blockcg_t h, const char* path);

/* Run the stencil autotuner for block width n_rhs now (the register-tile and
 * kernel choice of Sec. 6.2, each candidate timed on the normal operator's
 * pair of stencil launches), for the iteration's storage kind and for the
 * native-FP64 kind of the reliable updates, so that a following solve of
 * that width does not spend its first call tuning.  A no-op for a width
 * already tuned on this handle or when params.dslash_variant fixes the
 * kernel.  Zeroes and uses the workspace's block fields.  Synchronises the
 * stream.  Errors: ERR_ARG, ERR_NOMEM, ERR_CUDA. */
blockcg_status blockcg_tune(blockcg_t h, int n_rhs);

/* Measured arithmetic issue rates of the current device, the denominators of
 * the arithmetic roofline of the FP64-accurate form (whose double-float
 * stencil of Sec. 6.2 is bound by FP32 instruction issue on GPUs with a
 * reduced FP64 rate): long chains of independent fused multiply-adds on
 * 8 blocks of 256 threads per SM, timed with CUDA events on `stream`
 * (cudaStream_t, NULL = legacy default), in FP32 and in FP64.  Outputs
 * (host): *fp32_fma_per_s and *fp64_fma_per_s multiply-adds per second,
 * *sm_count the device's SM count.  Needs no handle; allocates nothing;
 * synchronises the stream.  Errors: ERR_ARG (null output), ERR_CUDA. */
blockcg_status blockcg_bench_alu(void* stream, double* fp32_fma_per_s, double* fp64_fma_per_s,
                                 int* sm_count);

/* Measured rate of the warp-level bf16 tensor-core product (mma.sync
 * m16n8k16 with FP32 accumulation) that the tensor-core double-float stencil
 * issues (its split-operand products, Sec. 6.2 stencil): 4 independent
 * accumulator chains per warp on register operands, 8 blocks of 256 threads
 * per SM, timed with CUDA events on `stream` (cudaStream_t, NULL = legacy
 * default).  Output (host): *bf16_flop_per_s = 4096 flops per instruction
 * times instructions per second.  Needs no handle; allocates nothing;
 * synchronises the stream.  Errors: ERR_ARG (null output), ERR_CUDA. */
blockcg_status blockcg_bench_mma(void* stream, double* bf16_flop_per_s);

/* K = X^dag Y, the same block inner product as blockcg_block_cdot, for
 * callers that cannot allocate device memory: code running inside a memory
 * pool it does not own, plug-ins that receive only the host application's
 * buffers, or programs that must avoid cudaMalloc because it may synchronise
 * the device.  The paper has no counterpart to this entry point.
 *
 * Needs no handle and no workspace.  X, Y: device complex128 [n_rhs][vh][3]
 * (user layout, vh = sites per parity); K: device complex128
 * [n_rhs][n_rhs] row-major; stream: cudaStream_t (NULL = legacy default).
 * Computed in native FP64.  Enqueues two kernels and returns.
 *
 * Scratch: the partial sums live in a fixed 4 MiB array inside the library's
 * device image, which every GPU that loads the library holds until the
 * process exits.  The entry point calls no cudaMalloc, cudaFree or any other
 * allocating routine.  On its first call on a device (with that device
 * current) it looks up the array's device address once, so make that first
 * call before any stream capture.  The looked-up address is kept for the life
 * of the process: after cudaDeviceReset on a device it no longer refers to
 * live memory, so do not call this entry point on a device that was reset.
 * Every call overwrites the whole region it
 * uses, so no state carries over from one call to the next, but all calls
 * share the one array: calls whose kernels overlap on the GPU (e.g. on two
 * streams at once) race and must be serialised by the caller.
 *
 * Errors: BLOCKCG_ERR_ARG for null pointers, vh < 1, or n_rhs outside
 * [1, 64] (the scratch holds 64 x 64 partial matrices per CTA at most);
 * BLOCKCG_ERR_CUDA if the symbol lookup or a launch fails. */
blockcg_status blockcg_block_cdot_noalloc(const void* X, const void* Y, int n_rhs, long long vh,
                                          void* K, void* stream);

/* ---- Batched solves ------------------------------------------------------
 *
 * Many independent problems (lattices, masses, block widths), each a handle
 * created, loaded and given a workspace as above, solved together: the
 * per-iteration kernel sequence of blockcg_solve (Algorithm 1 with the gated
 * reliable update of Algorithm 3) for every problem runs on a stream of its
 * own, so small lattices that cannot fill the GPU alone run side by side.
 * With BLOCKCG_BATCH_GRAPH, one chunk of iterations of every active problem
 * is captured once into a single CUDA graph and replayed until each problem
 * has converged, failed or reached its max_iter (the graph is captured again
 * when the set of active problems changes).  The stencil autotuner runs once
 * per (lattice, storage kind, N) and its choice is shared by the batch.
 * Results are the same as blockcg_solve on each handle.  The paper solves
 * one block at a time; batching many problems is this library's extension. */
typedef struct blockcg_batch* blockcg_batch_t;

#define BLOCKCG_BATCH_MAX 4096
#define BLOCKCG_BATCH_GRAPH 1 /* flags bit: replay a captured CUDA graph */
/* flags bits 8..15: iterations per device-loop trip with BLOCKCG_BATCH_GRAPH
 * (0: min(check_every, 4)) */
#define BLOCKCG_BATCH_TRIP_SHIFT 8

typedef struct {
  double ms_total;         /* device time of the whole batch (CUDA events) */
  int chunk;               /* iterations per replay (min of the problems' check_every) */
  long long graph_replays; /* graph launches (0 without BLOCKCG_BATCH_GRAPH) */
  long long graph_captures;
  long long graph_nodes;   /* nodes of the last captured graph */
  long long launches;      /* kernel launches executed (graph kernel nodes counted per replay) */
} blockcg_batch_stats;

/* problems: n distinct handles (1 <= n <= BLOCKCG_BATCH_MAX; the batch keeps
 * the pointers, the handles must outlive it and must not be used elsewhere
 * while a batch solve runs).  stream: cudaStream_t (NULL = legacy default);
 * batch solves start after the work enqueued on it before the call and the
 * stream waits for their end.  The batch owns one stream per problem plus
 * one of its own, a few events and n status words of pinned host memory.
 * Errors: BLOCKCG_ERR_ARG (null or repeated handles, n out of range),
 * BLOCKCG_ERR_CUDA. */
blockcg_status blockcg_batch_create(blockcg_batch_t* out, const blockcg_t* problems, int n,
                                    void* stream);

/* Solve problem p for B[p] (device, user layout, n_rhs[p] columns) with
 * initial guess / result X[p], to the true relative residual tol for every
 * column.  flags: BLOCKCG_BATCH_GRAPH or 0 (plain launches, same kernels),
 * plus (k << BLOCKCG_BATCH_TRIP_SHIFT) for k iterations per loop trip.
 * stats (optional, n entries): per-problem iterations, reliable updates and
 * true residual; ms_total is the batch's.  status (optional, n entries): the
 * per-problem outcome as blockcg_solve would return it.  bstats optional.
 * While it runs, each handle's kernels go to the batch's stream for it and
 * the handle's profile flag is off; both are restored on return.
 * Synchronises.  Returns BLOCKCG_OK if every problem converged, else the
 * first problem's failure (argument errors before any work: that problem's
 * check, e.g. BLOCKCG_ERR_ARG or BLOCKCG_ERR_NOMEM); blockcg_batch_last_error
 * names the problem. */
blockcg_status blockcg_batch_solve(blockcg_batch_t b, const void* const* B, void* const* X,
                                   const int* n_rhs, double tol, int flags, blockcg_stats* stats,
                                   int* status, blockcg_batch_stats* bstats);

/* Release the batch's streams, events, graph and pinned memory (not the
 * problems' handles). */
void blockcg_batch_destroy(blockcg_batch_t b);
const char* blockcg_batch_last_error(blockcg_batch_t b);

/* Release the handle (host memory only; caller-owned device buffers stay). */
void blockcg_destroy(blockcg_t h);

const char* blockcg_status_string(blockcg_status s);
const char* blockcg_last_error(blockcg_t h);

#ifdef __cplusplus
}
#endif

#endif /* BLOCKCG_H */
