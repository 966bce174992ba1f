// Small dense N x N algebra of blockCGrQ in native FP64, on the device, one
// CTA per call (N <= 64).  The paper does these on the host with Eigen
// (Sec. 6); keeping them on the device removes every host round trip from the
// iteration, so a whole iteration is a fixed sequence of launches gated by the
// status word.
//
//   dense_beta     beta = (P^dag A P)^-1 through a Cholesky factorisation,
//                  BC = beta C                                  (Algorithm 1)
//   dense_qr_step  thin QR of W = Q - AP beta from its Gram: W^dag W = S^dag S
//                  (Cholesky), S^-1, S^dag; C_prev = C; C = S C; iterated
//                  residuals |R_i| = |column i of C|; reliable-update trigger
//                                                   (Algorithms 1, 2 and 3)
//   dense_restart  thin QR of a true residual R = B - A Y: C = chol factor,
//                  C^-1, convergence on the true residual, and
//                  S = C C_old^-1 with C_old the C in force before the last
//                  C = S C                                      (Algorithm 3)
// Matrices are complex128 row-major [N][N] in global memory; the CTA works
// on copies in shared memory.
#include "internal.h"
#include "../../include/blockcg.h"

namespace bcg {

static constexpr int DENSE_THREADS = 256;
// reliable update when the iterated residual exceeds this factor times the
// true residual of the last update
static constexpr double RU_GROWTH = 100.0;

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// In-place lower Cholesky A = L L^dag of a Hermitian matrix in shared memory.
// A pivot that is not finite gives BLOCKCG_ERR_NONFINITE; a pivot d_k <= 0 or
// d_k <= CHOL_REL_TOL * A_kk (A_kk the diagonal before factorising) gives
// BLOCKCG_ERR_BREAKDOWN: d_k / A_kk is the squared sine of the angle between
// column k and the span of the columns before it, so a value at rounding
// level means the block is numerically rank deficient (e.g. linearly
// dependent right-hand sides, Sec. 4).  Returns 0 or the error (uniform over
// the CTA).
static constexpr double CHOL_REL_TOL = 1e-13;

__device__ int chol_lower(double2* A, int N, int* flag) {
  __shared__ double diag0[64];
  const int tid = threadIdx.x;
  for (int k = tid; k < N; k += blockDim.x) diag0[k] = A[k * N + k].x;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      double d = A[k * N + k].x;
      int f = 0;
      if (!isfinite(d) || !isfinite(diag0[k])) f = BLOCKCG_ERR_NONFINITE;
      else if (!(d > 0.0) || !(d > CHOL_REL_TOL * diag0[k])) f = BLOCKCG_ERR_BREAKDOWN;
      else A[k * N + k] = make_double2(sqrt(d), 0.0);
      *flag = f;
    }
    __syncthreads();
    int f = *flag;
    if (f) return f;
    double inv = 1.0 / A[k * N + k].x;
    for (int i = k + 1 + tid; i < N; i += blockDim.x) {
      double2 v = A[i * N + k];
      A[i * N + k] = make_double2(v.x * inv, v.y * inv);
    }
    __syncthreads();
    int m = N - k - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) A[i * N + j] = csub(A[i * N + j], cm(A[i * N + k], cconj(A[j * N + k])));
    }
    __syncthreads();
  }
  // zero the strict upper triangle
  for (int idx = tid; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    if (j > i) A[idx] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  return 0;
}

// Linv = L^-1 for lower-triangular L (shared memory), by forward
// substitution on the identity, right-looking: step k finishes row k
// (divide by L_kk) and removes its contribution from every later row, so each
// step is one parallel update of the whole block and the dependent chain is N
// steps long (a column-parallel substitution would leave N threads with
// O(N^2) dependent FP64 operations each).
__device__ void tri_inv_lower(const double2* L, double2* Linv, int N) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - (idx / N) * N;
    Linv[idx] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    const double inv = 1.0 / L[k * N + k].x;
    for (int j = tid; j <= k; j += blockDim.x) {
      const double2 v = Linv[k * N + j];
      Linv[k * N + j] = make_double2(v.x * inv, v.y * inv);
    }
    __syncthreads();
    // rows i > k, columns j <= k: Linv_ij -= L_ik Linv_kj
    const int m = N - k - 1;
    for (int idx = tid; idx < m * (k + 1); idx += blockDim.x) {
      const int i = k + 1 + idx / (k + 1), j = idx - (idx / (k + 1)) * (k + 1);
      Linv[i * N + j] = csub(Linv[i * N + j], cm(L[i * N + k], Linv[k * N + j]));
    }
    __syncthreads();
  }
}

__device__ void load_mat(double2* dst, const double2* __restrict__ src, int N) {
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) dst[idx] = src[idx];
  __syncthreads();
}


// ---------------------------------------------------------------- beta ----
__global__ void __launch_bounds__(DENSE_THREADS)
    k_dense_beta(const double2* __restrict__ H, const double2* __restrict__ Cm,
                 double2* __restrict__ beta, double2* __restrict__ BC, int N, SolverStatus* st,
                 Gate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int flag;
  if (gate_closed(gate)) return;
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* Li = A + N * N;
  double2* Bt = Li + N * N;
  load_mat(A, H, N);
  int f = chol_lower(A, N, &flag);
  if (f) {
    if (threadIdx.x == 0) st->error = f;
    return;
  }
  tri_inv_lower(A, Li, N);
  // beta = Li^dag Li
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    double2 s = make_double2(0.0, 0.0);
    for (int l = (i > j ? i : j); l < N; ++l) s = cadd(s, cm(cconj(Li[l * N + i]), Li[l * N + j]));
    Bt[idx] = s;
    beta[idx] = s;
  }
  __syncthreads();
  // BC = beta C
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    double2 s = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) s = cadd(s, cm(Bt[i * N + l], Cm[l * N + j]));
    BC[idx] = s;
  }
}

cudaError_t dense_beta(const double2* H, const double2* C, double2* beta, double2* BC, int N,
                       SolverStatus* st, Gate gate, cudaStream_t s) {
  size_t sm = 3ull * N * N * sizeof(double2);
  cudaFuncSetAttribute(k_dense_beta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dense_beta<<<1, DENSE_THREADS, sm, s>>>(H, C, beta, BC, N, st, gate);
  return cudaGetLastError();
}

// ------------------------------------------------------------- qr step ----
__global__ void __launch_bounds__(DENSE_THREADS)
    k_dense_qr_step(const double2* __restrict__ G, double2* __restrict__ C,
                    double2* __restrict__ C_prev, double2* __restrict__ Sinv,
                    double2* __restrict__ SH, const double* __restrict__ bnorm, QrStepParams p,
                    int N, SolverStatus* st, Gate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int flag;
  __shared__ double resv[64];
  if (gate_closed(gate)) return;
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* Li = A + N * N;
  double2* Cs = Li + N * N;
  load_mat(A, G, N);
  int f = chol_lower(A, N, &flag);
  if (f) {
    if (threadIdx.x == 0) st->error = f;
    return;
  }
  tri_inv_lower(A, Li, N);
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    Sinv[idx] = cconj(Li[j * N + i]);  // (L^-1)^dag, upper
    SH[idx] = A[idx];                  // S^dag = L, lower
    double2 c = C[idx];
    Cs[idx] = c;
    C_prev[idx] = c;
  }
  __syncthreads();
  // C = S C with S = L^dag: (S C)_ij = sum_{l >= i} conj(L_li) C_lj
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    double2 s = make_double2(0.0, 0.0);
    for (int l = i; l < N; ++l) s = cadd(s, cm(cconj(A[l * N + i]), Cs[l * N + j]));
    C[idx] = s;
  }
  __syncthreads();
  // iterated residual of column i: |R_i| = sqrt(sum_j |C_ji|^2)
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) {
      double2 c = C[j * N + i];
      s += c.x * c.x + c.y * c.y;
    }
    resv[i] = sqrt(s) / bnorm[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rmax = 0.0;
    for (int i = 0; i < N; ++i) rmax = fmax(rmax, resv[i]);
    int it = st->iters + 1;
    st->iters = it;
    st->res_max = rmax;
    int ru = 0;
    if (!(rmax <= p.tol) && !isfinite(rmax)) st->error = BLOCKCG_ERR_NONFINITE;
    if (rmax <= p.tol) ru = 1;
    else if (p.delta > 0.0 && rmax < p.delta * st->res_at_ru) ru = 1;
    else if (p.ru_every > 0 && (it % p.ru_every) == 0) ru = 1;
    // the iterated residual has grown far above the last true one: the
    // sloppy recursion is drifting, so recompute from the true residual
    else if (rmax > RU_GROWTH * st->res_at_ru) ru = 1;
    st->ru_pending = ru;
    // the iteration budget is spent: later chunks of gated launches do nothing
    if (p.max_iter > 0 && it >= p.max_iter) st->stopped = 1;
  }
}

cudaError_t dense_qr_step(const double2* G, double2* C, double2* C_prev, double2* Sinv,
                          double2* SH, const double* bnorm, QrStepParams p, int N,
                          SolverStatus* st, Gate gate, cudaStream_t s) {
  size_t sm = 3ull * N * N * sizeof(double2);
  cudaFuncSetAttribute(k_dense_qr_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dense_qr_step<<<1, DENSE_THREADS, sm, s>>>(G, C, C_prev, Sinv, SH, bnorm, p, N, st, gate);
  return cudaGetLastError();
}

// ------------------------------------------------------------- restart ----
__global__ void __launch_bounds__(DENSE_THREADS)
    k_dense_restart(const double2* __restrict__ G, double2* __restrict__ C,
                    double2* __restrict__ C_prev, double2* __restrict__ Cinv,
                    double2* __restrict__ SH, const double* __restrict__ bnorm,
                    double* __restrict__ tres_out, double tol, int init, int confirmed, int N,
                    SolverStatus* st, Gate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int flag;
  __shared__ double tres[64];
  if (gate_closed(gate)) return;
  double2* A = reinterpret_cast<double2*>(smem_raw);  // -> L of the true residual
  double2* Wk = A + N * N;                            // L^-1, then C_prev^dag (lower)
  double2* Pi = Wk + N * N;                           // (C_prev^dag)^-1
  load_mat(A, G, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tres[i] = sqrt(fmax(A[i * N + i].x, 0.0)) / bnorm[i];
    tres_out[i] = tres[i];
  }
  __syncthreads();
  int f = chol_lower(A, N, &flag);
  if (f) {
    if (threadIdx.x == 0) st->error = f;
    return;
  }
  tri_inv_lower(A, Wk, N);
  double tmax = 0.0;
  for (int i = 0; i < N; ++i) tmax = fmax(tmax, tres[i]);
  // C_new = L^dag (upper), Cinv = (L^-1)^dag
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    Cinv[idx] = cconj(Wk[j * N + i]);
  }
  __syncthreads();
  if (!init) {
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      int i = idx / N, j = idx % N;
      Wk[idx] = cconj(C_prev[j * N + i]);
    }
    __syncthreads();
    tri_inv_lower(Wk, Pi, N);  // Pi = (C_prev^dag)^-1 = (C_prev^-1)^dag
    // S = C_new C_prev^-1, so S^dag = (C_prev^-1)^dag C_new^dag = Pi L
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      int i = idx / N, j = idx % N;
      double2 s = make_double2(0.0, 0.0);
      for (int l = j; l <= i; ++l) s = cadd(s, cm(Pi[i * N + l], A[l * N + j]));
      SH[idx] = s;
    }
  }
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    C[idx] = cconj(A[j * N + i]);
  }
  if (threadIdx.x == 0) {
    st->true_res_max = tmax;
    st->res_max = tmax;
    st->res_at_ru = tmax;
    if (!isfinite(tmax)) st->error = BLOCKCG_ERR_NONFINITE;
    if (tmax <= tol) {
      st->done = 1;
      if (confirmed) st->verified = 1;
    }
    if (!init) st->reliable_updates += 1;
  }
}

// Native-FP64 confirmation of a convergence (see verify_fp64 in api.cu): G is
// the Gram of R = B - A Y computed in FP64; the per-column true residuals
// replace those of the double-float update.  All within tol: verified.
// Otherwise the solve goes on and all its later reliable updates are FP64.
__global__ void k_dense_verify(const double2* __restrict__ G, const double* __restrict__ bnorm,
                               double* __restrict__ tres, double tol, int N, SolverStatus* st) {
  __shared__ double r[64];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    r[i] = sqrt(fmax(G[i * N + i].x, 0.0)) / bnorm[i];
    tres[i] = r[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tmax = 0.0;
    bool finite = true;
    for (int i = 0; i < N; ++i) {
      tmax = fmax(tmax, r[i]);
      finite = finite && isfinite(r[i]);
    }
    st->true_res_max = tmax;
    if (!finite) {
      st->error = BLOCKCG_ERR_NONFINITE;
    } else if (tmax <= tol) {
      st->verified = 1;
    } else {
      st->done = 0;
      st->verified = 0;
      st->fp64_only = 1;
    }
  }
}

cudaError_t dense_verify(const double2* G, const double* bnorm, double* tres, double tol, int N,
                         SolverStatus* st, cudaStream_t s) {
  k_dense_verify<<<1, 64, 0, s>>>(G, bnorm, tres, tol, N, st);
  return cudaGetLastError();
}

cudaError_t dense_restart(const double2* G, double2* C, double2* C_prev, double2* Cinv,
                          double2* SH, const double* bnorm, double* tres, double tol, int init,
                          int confirmed, int N, SolverStatus* st, Gate gate, cudaStream_t s) {
  size_t sm = 3ull * N * N * sizeof(double2);
  cudaFuncSetAttribute(k_dense_restart, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dense_restart<<<1, DENSE_THREADS, sm, s>>>(G, C, C_prev, Cinv, SH, bnorm, tres, tol, init,
                                               confirmed, N, st, gate);
  return cudaGetLastError();
}

// --------------------------------------------------------------- misc ----
__global__ void k_dense_bnorm(const double2* __restrict__ Gb, double* __restrict__ bnorm, int N,
                              SolverStatus* st) {
  int i = threadIdx.x;
  if (i < N) {
    double v = Gb[i * N + i].x;
    bnorm[i] = sqrt(fmax(v, 0.0));
    if (!isfinite(v)) st->error = BLOCKCG_ERR_NONFINITE;
    else if (!(v > 0.0)) st->error = BLOCKCG_ERR_BREAKDOWN;
  }
}

cudaError_t dense_bnorm(const double2* Gb, double* bnorm, int N, SolverStatus* st,
                        cudaStream_t s) {
  k_dense_bnorm<<<1, 64, 0, s>>>(Gb, bnorm, N, st);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(DENSE_THREADS)
    k_dense_chol_upper(const double2* __restrict__ H, double2* __restrict__ R,
                       double2* __restrict__ Rinv, int N, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int flag;
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* Li = A + N * N;
  load_mat(A, H, N);
  int f = chol_lower(A, N, &flag);
  if (threadIdx.x == 0) *err = f;
  if (f) return;
  tri_inv_lower(A, Li, N);
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    int i = idx / N, j = idx % N;
    R[idx] = cconj(A[j * N + i]);
    Rinv[idx] = cconj(Li[j * N + i]);
  }
}

cudaError_t dense_chol_upper(const double2* H, double2* R, double2* Rinv, int N, int* err,
                             cudaStream_t s) {
  size_t sm = 2ull * N * N * sizeof(double2);
  cudaFuncSetAttribute(k_dense_chol_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dense_chol_upper<<<1, DENSE_THREADS, sm, s>>>(H, R, Rinv, N, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------ CG scalars ----
__global__ void k_cg_alpha(const double2* __restrict__ pAp, const double* __restrict__ rr,
                           const double* __restrict__ gam, double* __restrict__ alpha,
                           double* __restrict__ alpha_x, SolverStatus* st, Gate gate) {
  if (gate_closed(gate)) return;
  double d = pAp[0].x;
  if (!isfinite(d)) {
    st->error = BLOCKCG_ERR_NONFINITE;
    return;
  }
  if (!(d > 0.0)) {
    st->error = BLOCKCG_ERR_BREAKDOWN;
    return;
  }
  const double a = *rr / d;
  *alpha = a;
  *alpha_x = a / *gam;  // x is kept unscaled: x += (alpha / gamma) (gamma p)
}

__global__ void k_cg_beta(const double2* __restrict__ rr_new_sum, double* __restrict__ rr,
                          double* __restrict__ beta, const double* __restrict__ bnorm,
                          const double* __restrict__ gam, double tol, double delta,
                          SolverStatus* st, Gate gate) {
  if (gate_closed(gate)) return;
  double bnorm2 = bnorm[0] * bnorm[0];
  double rn = rr_new_sum[0].x;  // |gamma r|^2
  int it = st->iters + 1;
  st->iters = it;
  if (!isfinite(rn)) {
    st->error = BLOCKCG_ERR_NONFINITE;
    return;
  }
  double rel = sqrt(rn / bnorm2) / *gam;
  st->res_max = rel;
  // converged, or dropped by delta since the last reliable update: the host
  // runs a reliable update, which recomputes r and then forms beta from the
  // true residual (cg_restart_check); rr keeps the previous |r|^2 for that
  if (rel <= tol || (delta > 0.0 && rel < delta * st->res_at_ru)) {
    st->ru_pending = 1;
    return;
  }
  *beta = rn / *rr;
  *rr = rn;
}

cudaError_t cg_scalar_alpha(const double2* pAp, const double* rr, const double* gam, double* alpha,
                            double* alpha_x, SolverStatus* st, Gate gate, cudaStream_t s) {
  k_cg_alpha<<<1, 1, 0, s>>>(pAp, rr, gam, alpha, alpha_x, st, gate);
  return cudaGetLastError();
}

cudaError_t cg_scalar_beta(const double2* rr_new_sum, double* rr, double* beta,
                           const double* bnorm, const double* gam, double tol, double delta,
                           SolverStatus* st, Gate gate, cudaStream_t s) {
  k_cg_beta<<<1, 1, 0, s>>>(rr_new_sum, rr, beta, bnorm, gam, tol, delta, st, gate);
  return cudaGetLastError();
}

// The iteration works on gamma r and gamma p, gamma a power of two chosen at
// every reliable update so that the entries of gamma r have unit root mean
// square: CG's alpha and beta do not change under a common scaling of r and
// p, and 16-bit storage keeps the shrinking residual within its exponent
// range.  rr holds |gamma r|^2.
__global__ void k_cg_restart_check(const double2* __restrict__ rr_sum, double* __restrict__ rr,
                                   double* __restrict__ beta, double* __restrict__ gam,
                                   const double* __restrict__ bnorm, double n_elems, double tol,
                                   int init, SolverStatus* st) {
  if (st->error) return;
  double rn = rr_sum[0].x;  // true |r|^2
  double rel = sqrt(rn) / bnorm[0];
  st->true_res_max = rel;
  st->res_max = rel;
  st->res_at_ru = rel;
  if (!isfinite(rn)) {
    st->error = BLOCKCG_ERR_NONFINITE;
    return;
  }
  if (rel <= tol) {
    st->done = 1;
    return;
  }
  const double g_new = exp2(rint(log2(sqrt(n_elems / rn))));
  // p = r + beta p with beta from the true residual (p = r at the start);
  // in scaled form gamma' p' = gamma' r + beta (gamma' / gamma) (gamma p)
  const double g_old = *gam;
  *beta = init ? 0.0 : (rn * g_old * g_old / *rr) * (g_new / g_old);
  *rr = rn * g_new * g_new;
  *gam = g_new;
  st->ru_pending = 0;
}

cudaError_t cg_restart_check(const double2* rr_sum, double* rr, double* beta, double* gam,
                             const double* bnorm, double n_elems, double tol, int init,
                             SolverStatus* st, cudaStream_t s) {
  k_cg_restart_check<<<1, 1, 0, s>>>(rr_sum, rr, beta, gam, bnorm, n_elems, tol, init, st);
  return cudaGetLastError();
}

// Loop condition of a batched solve's device-side iteration loop (a CUDA
// graph WHILE node): continue while the problem has neither converged,
// failed nor used its iteration budget, and never beyond max_trips trips.
__global__ void k_loop_condition(cudaGraphConditionalHandle handle, SolverStatus* st,
                                 int max_trips) {
  const int trips = st->trips + 1;
  st->trips = trips;
  unsigned go = (st->done || st->error || st->stopped) ? 0u : 1u;
  if (trips >= max_trips) {
    if (go) st->stopped = 1;
    go = 0u;
  }
  cudaGraphSetConditional(handle, go);
}

cudaError_t loop_condition(cudaGraphConditionalHandle handle, SolverStatus* st, int max_trips,
                           cudaStream_t s) {
  k_loop_condition<<<1, 1, 0, s>>>(handle, st, max_trips);
  return cudaGetLastError();
}

}  // namespace bcg
