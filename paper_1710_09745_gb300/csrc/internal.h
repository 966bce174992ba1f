// Host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace bcg {

// Field storage kinds (element = one complex number).
enum FieldKind { FK_DF = 0, FK_F32 = 1, FK_F64 = 2, FK_H16 = 3, FK_BF16 = 4 };

inline size_t elem_bytes(FieldKind k) {
  return k == FK_F32 ? 8 : (k == FK_H16 || k == FK_BF16) ? 4 : 16;
}

// Kernel gating by the device status word, so that a host loop can enqueue
// whole iterations without reading back the convergence state.
// GATE_ACTIVE: run unless done or failed; GATE_RU: additionally only when a
// reliable update is pending; GATE_ITER: run unless done, failed or a
// convergence check is pending (CG baseline).  GATE_RU_CHEAP / GATE_RU_FINE
// split a pending reliable update by the iterated residual of this iteration:
// the cheap (double-float) residual while res_max > thr and no FP64
// confirmation has failed, the native-FP64 one otherwise.
enum GateMode {
  GATE_ALWAYS = 0,
  GATE_ACTIVE = 1,
  GATE_RU = 2,
  GATE_ITER = 3,
  GATE_RU_CHEAP = 4,
  GATE_RU_FINE = 5
};
struct Gate {
  const SolverStatus* st;
  int mode;
  double thr;  // res_max threshold of GATE_RU_CHEAP / GATE_RU_FINE
};

// launches gated on a pending reliable update are off in most iterations;
// their launchers use persistent grids (a few blocks per SM) so that a
// gated-off launch retires quickly
inline bool gate_mostly_off(const Gate& g) {
  return g.st && (g.mode == GATE_RU || g.mode == GATE_RU_CHEAP || g.mode == GATE_RU_FINE);
}

__device__ __forceinline__ bool gate_closed(const Gate& g) {
  if (g.mode == GATE_ALWAYS || g.st == nullptr) return false;
  const volatile SolverStatus* s = g.st;
  if (s->done || s->error || s->stopped) return true;
  if (g.mode == GATE_ITER) return s->ru_pending != 0;
  if (g.mode == GATE_ACTIVE) return false;
  if (!s->ru_pending) return true;  // the reliable-update modes
  if (g.mode == GATE_RU) return false;
  const bool cheap = !s->fp64_only && s->res_max > g.thr;
  return g.mode == GATE_RU_CHEAP ? !cheap : cheap;
}

// Stencil epilogues.
enum DslashEpi {
  EPI_NONE = 0,     // out = D in
  EPI_NORMAL = 1,   // out = m2 * c1 - D in         (A = m^2 - D_eo D_oe, second half)
  EPI_RESIDUAL = 2  // out = c2 - (m2 * c1 - D in)  (R = B - A Y)
};

// ---- stencil.cu
// recon: store the first two rows of every hop matrix only (6 elements)
cudaError_t pack_links(FieldKind k, const double2* fat, const double2* lng, void* out,
                       const Geom& g, int antiperiodic_t, int recon, cudaStream_t s);
size_t links_bytes(FieldKind k, const Geom& g, int recon = 0);  // both parities
// checks that every fat link is c_f U and every long link c_l U (U in SU(3),
// c real and the same for all links of a kind, from the first link); writes
// c_f, c_l to c[0], c[1] and a nonzero *bad otherwise
cudaError_t check_scaled_su3(const double2* fat, const double2* lng, long long V, double tol,
                             double* c, int* bad, cudaStream_t s);
// links points at the start of the packed array for both parities.
// R: right-hand sides per thread (1, 2, 4, 8); R | DSLASH_TMA selects the
// bulk-copy pipelined kernel (the plain kernel runs instead when the
// pipelined one cannot, e.g. FP32 rows that are not 16-byte multiples).
static constexpr int DSLASH_TMA = 0x100;
// R | DSLASH_ASYNC selects the per-thread cp.async prefetch kernel
static constexpr int DSLASH_ASYNC = 0x200;
// R | DSLASH_RECON: links packed as two rows (pack_links recon); plain kernel
// only, FP32 / FP16 / bfloat16 kinds
static constexpr int DSLASH_RECON = 0x400;
// R | DSLASH_BLOCKED: the plain kernel on a persistent grid whose blocks each
// walk one contiguous range of sites (cache reuse of neighbours in L1)
static constexpr int DSLASH_BLOCKED = 0x1000;
// R | DSLASH_TC: the tensor-core stencil: double-float as split products
// (stencil_tc.cu; N = 16 or 32 with a workspace set, the cp.async kernel
// otherwise), FP16 / bfloat16 on the stored values (stencil_tc16.cu; N = 16
// or 32 with full links, the plain kernel otherwise)
static constexpr int DSLASH_TC = 0x2000;
bool dslash_tc_supported(const Geom& g, int N);
bool dslash_tc16_supported(int N);
cudaError_t dslash_tc16(FieldKind k, int epi, const void* links, const void* in, void* out,
                        const void* c1, const void* c2, double m2, const Geom& g, int out_parity,
                        int N, Gate gate, cudaStream_t s);
cudaError_t dslash_df_tc(int epi, const void* links, const void* in, void* out, const void* c1,
                         const void* c2, double m2, const Geom& g, int out_parity, int N,
                         Gate gate, cudaStream_t s);
cudaError_t dslash(FieldKind k, int R, int epi, const void* links, const void* in, void* out,
                   const void* c1, const void* c2, double m2, const Geom& g, int out_parity,
                   int N, Gate gate, cudaStream_t s);

// per-kind stencil entry points (stencil_<kind>.cu)
#define BCG_DSLASH_KIND_DECL(name)                                                             \
  cudaError_t name(int R, int epi, const void* links, const void* in, void* out, const void* c1, \
                   const void* c2, double m2, const Geom& g, int out_parity, int N, Gate gate,  \
                   cudaStream_t s)
BCG_DSLASH_KIND_DECL(dslash_df);
BCG_DSLASH_KIND_DECL(dslash_f32);
BCG_DSLASH_KIND_DECL(dslash_f64);
BCG_DSLASH_KIND_DECL(dslash_h16);
BCG_DSLASH_KIND_DECL(dslash_bf16);

// ---- blas.cu
cudaError_t to_internal(FieldKind k, const double2* user, void* internal, int N, int Vh,
                        cudaStream_t s);
cudaError_t from_internal(FieldKind k, const void* internal, double2* user, int N, int Vh,
                          cudaStream_t s);
cudaError_t zero_field(FieldKind k, void* f, size_t n_elems, cudaStream_t s);
int gram_blocks(int N, int rows);
// tile (here and below): sites per shared-memory tile, 0 = the default;
// the solver's autotuner picks it per storage kind and N
cudaError_t gram_partials(FieldKind k, const void* X, const void* Y, int N, int Vh, int hermitian,
                          double2* partials, int nblocks, Gate gate, cudaStream_t s, int tile = 0);
cudaError_t gram_reduce(const double2* partials, int nblocks, int N, int hermitian, double2* out,
                        Gate gate, cudaStream_t s);
// Q <- W = Q - AP beta, and the per-CTA partials of the Hermitian Gram W^dag W
// (nblocks CTAs, reduced by gram_reduce)
cudaError_t w_update_gram(FieldKind k, void* Q, const void* AP, const double2* beta, int N, int Vh,
                          double2* partials, int nblocks, Gate gate, cudaStream_t s, int tile = 0);
// tile of bcg_update: sites per tile, plus UPD_TWO_ROWS for two rows per
// thread and UPD_X_GLOBAL for the old X read from global memory (not staged)
static constexpr int UPD_TWO_ROWS = 64;
static constexpr int UPD_X_GLOBAL = 128;
// tile | UPD_TC: the tensor-core form (16-bit kinds with N = 16 or 32, the
// double-float kind with N = 16; the CUDA-core kernel otherwise)
static constexpr int UPD_TC = 256;
// tile | WG_TC for w_update_gram: the tensor-core fused W + Gram (16-bit
// kinds, N = 16 or 32; the FP32-pipe kernel otherwise)
static constexpr int WG_TC = 256;
// tile | GR_TC for gram_partials: the tensor-core Gram (Hermitian Grams of
// the 16-bit kinds, N = 16 or 32; the FP32-pipe kernel otherwise)
static constexpr int GR_TC = 256;
// Q <- W Sinv ; X += P BC ; P <- Q + P SH unless st->ru_pending
cudaError_t bcg_update(FieldKind sk, FieldKind xk, void* Q, void* P, void* X, const double2* Sinv,
                       const double2* BC, const double2* SH, int N, int Vh, Gate gate,
                       cudaStream_t s, int tile = 0);
// the tensor-core fused update of the double-float kind (blas_tc_df.cu,
// exact split bf16 products), N = 16
bool bcg_update_tc_df_supported(int N);
cudaError_t bcg_update_tc_df(void* Q, void* P, void* X, const double2* Sinv, const double2* BC,
                             const double2* SH, int N, int Vh, Gate gate, cudaStream_t s);
// W = Q - AP beta over Q for the double-float kind on the tensor cores, N = 16
cudaError_t w_update_tc_df(void* Q, const void* AP, const double2* beta, int N, int Vh, Gate gate,
                           cudaStream_t s);
// the tensor-core fused update (blas_tc.cu): supported (kind, N) pairs
bool bcg_update_tc_supported(FieldKind sk, FieldKind xk, int N);
cudaError_t bcg_update_tc(FieldKind sk, void* Q, void* P, void* X, const double2* Sinv,
                          const double2* BC, const double2* SH, int N, int Vh, Gate gate,
                          cudaStream_t s);
bool w_gram_tc_supported(FieldKind k, int N);
// Hermitian K = X^dag Y on the tensor cores (the pairs of w_gram_tc_supported)
cudaError_t gram_partials_tc(FieldKind k, const void* X, const void* Y, int N, int Vh,
                             double2* partials, int nblocks, Gate gate, cudaStream_t s);
cudaError_t w_update_gram_tc(FieldKind k, void* Q, const void* AP, const double2* beta, int N,
                             int Vh, double2* partials, int nblocks, Gate gate, cudaStream_t s);
// Q <- R Cinv (converted to Q's kind) ; P <- Q + P SH (or P <- Q when init)
cudaError_t restart_update(FieldKind rk, FieldKind sk, const void* R, void* Q, void* P,
                           const double2* Cinv, const double2* SH, int init, int N, int Vh,
                           Gate gate, cudaStream_t s);
// Y (kind yk) += X (kind xk) ; X = 0
cudaError_t accumulate(FieldKind yk, FieldKind xk, void* Y, void* X, size_t n_elems, Gate gate,
                       cudaStream_t s);
// same-layout conversion between kinds (F64 -> any kind, or a copy), each
// value multiplied by *scale when scale is not null
cudaError_t convert_field(FieldKind from, FieldKind to, const void* in, void* out, size_t n_elems,
                          const double* scale, Gate gate, cudaStream_t s);
// Y += X a (generic block caxpy)
cudaError_t block_caxpy(FieldKind k, const void* X, const double2* a, void* Y, int N, int Vh,
                        cudaStream_t s);
// Q = M Rinv (generic right-multiplication by an upper-triangular matrix)
cudaError_t block_trmul(FieldKind k, const void* M, const double2* Rinv, void* Q, int N, int Vh,
                        cudaStream_t s);
// CG (N = 1) helpers
// x += alpha_x p ; r -= alpha Ap ; per-CTA partial sums of |r|^2
cudaError_t cg_axpy_norm(FieldKind k, FieldKind xk, void* x, void* r, const void* p, const void* Ap,
                         const double* alpha, const double* alpha_x, double2* partials,
                         int nblocks, int Vh, Gate gate, cudaStream_t s);
cudaError_t cg_xpay(FieldKind k, void* p, const void* r, const double* beta, int Vh, Gate gate,
                    cudaStream_t s);
cudaError_t copy_field(void* dst, const void* src, size_t bytes, cudaStream_t s);

// ---- dense.cu
// beta = H^-1 via Cholesky, BC = beta C
cudaError_t dense_beta(const double2* H, const double2* C, double2* beta, double2* BC, int N,
                       SolverStatus* st, Gate gate, cudaStream_t s);
// Cholesky of G = W^dag W -> S (upper), Sinv, SH = S^dag; C_prev = C; C = S C;
// residual norms and the reliable-update trigger.
struct QrStepParams {
  double tol, delta;
  int ru_every, max_iter;
};
cudaError_t dense_qr_step(const double2* G, double2* C, double2* C_prev, double2* Sinv,
                          double2* SH, const double* bnorm, QrStepParams p, int N,
                          SolverStatus* st, Gate gate, cudaStream_t s);
// Cholesky of the true-residual Gram -> C_new, Cinv; convergence on the true
// residual; S = C_new C_prev^-1 -> SH = S^dag (unless init).
// tres (N doubles) receives the per-column true relative residuals;
// confirmed: G is the Gram of a native-FP64 residual, so a convergence it
// shows is final (verified), else it awaits dense_verify.
cudaError_t dense_restart(const double2* G, double2* C, double2* C_prev, double2* Cinv,
                          double2* SH, const double* bnorm, double* tres, double tol, int init,
                          int confirmed, int N, SolverStatus* st, Gate gate, cudaStream_t s);
// native-FP64 confirmation of a convergence: true residuals from the FP64
// Gram G of R = B - A Y into tres; verified, or done cleared and fp64_only set
cudaError_t dense_verify(const double2* G, const double* bnorm, double* tres, double tol, int N,
                         SolverStatus* st, cudaStream_t s);
// bnorm_i = sqrt(Gb_ii); error if any is zero or not finite
cudaError_t dense_bnorm(const double2* Gb, double* bnorm, int N, SolverStatus* st,
                        cudaStream_t s);
// R upper with R^dag R = H, Rinv = R^-1; *err = blockcg_status
cudaError_t dense_chol_upper(const double2* H, double2* R, double2* Rinv, int N, int* err,
                             cudaStream_t s);
// CG scalars on the scaled iteration (gamma r, gamma p; rr = |gamma r|^2):
// alpha = rr / pAp and alpha_x = alpha / gamma; on the second call
// beta = rr_new / rr and the convergence / reliable-update test
cudaError_t cg_scalar_alpha(const double2* pAp, const double* rr, const double* gam, double* alpha,
                            double* alpha_x, SolverStatus* st, Gate gate, cudaStream_t s);
cudaError_t cg_scalar_beta(const double2* rr_new_sum, double* rr, double* beta,
                           const double* bnorm, const double* gam, double tol, double delta,
                           SolverStatus* st, Gate gate, cudaStream_t s);
// after a true-residual recomputation: done if it meets tol; else a new
// power-of-two gamma (unit RMS entries of gamma r for n_elems complex
// entries), beta for p = r + beta p from the true residual in scaled form
// (0 when init), rr = |gamma r|^2, and the pending check is cleared so that
// iterations resume
cudaError_t cg_restart_check(const double2* rr_sum, double* rr, double* beta, double* gam,
                             const double* bnorm, double n_elems, double tol, int init,
                             SolverStatus* st, cudaStream_t s);

// one-thread kernel ending a batched solve's device-side loop trip: sets the
// WHILE condition to "not done, no error, not stopped" (stops after max_trips)
cudaError_t loop_condition(cudaGraphConditionalHandle handle, SolverStatus* st, int max_trips,
                           cudaStream_t s);

// ---- grad.cu
// gradient of a real loss with respect to the links (user layout [4][V][3][3],
// either output may be null) from the internal native-FP64 blocks X, Lam (even)
// and Y = D_oe X, Mu = D_oe Lam (odd)
cudaError_t link_grad(const double2* X, const double2* Lam, const double2* Y, const double2* Mu,
                      double2* gfat, double2* glong, const Geom& g, int N, int antiperiodic_t,
                      cudaStream_t s);

}  // namespace bcg
