/*
 * Plain FP64 CPU oracle for the even-odd improved-staggered (HISQ-type) normal
 * operator and textbook CG.  TEST INFRASTRUCTURE ONLY: the product path never
 * links, loads or calls this file; only tests/, the smoke check and the CPU
 * baseline leg of the benchmark use it.
 *
 * Everything here is written for clarity, not speed: one output site at a
 * time, coordinates decoded from the lexicographic index on every access,
 * complex arithmetic through C99 `double complex`.
 *
 * Conventions (paper, Sec. 3.2, Eq. 2, with the readings stated below):
 *   - sites: lexicographic index i = x + Lx*(y + Ly*(z + Lz*t)), x fastest;
 *     parity p(x) = (x+y+z+t) & 1; checkerboard index cb = i >> 1 (Lx even).
 *   - links: fat F and long G, complex [4][V][3][3] (direction mu = x,y,z,t),
 *     row index = colour of the result; F_mu(x) connects x to x+mu,
 *     G_mu(x) connects x to x+3mu.  Long links carry their own coefficient
 *     (e.g. -1/24); staggered phases are NOT in the links.
 *   - staggered phases eta_mu(x) = (-1)^(sum_{nu<mu} x_nu).
 *   - hopping term (Eq. 2 with the anti-Hermitian sign reading on backward
 *     hops, so that M^dag M = m^2 - D_eo D_oe on even sites, Sec. 3.2):
 *       (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu)
 *                                          - F_mu(x-mu)^dag psi(x-mu)
 *                                          + G_mu(x) psi(x+3mu)
 *                                          - G_mu(x-3mu)^dag psi(x-3mu) ]
 *     periodic in all directions; with antiperiodic_t != 0 every hop that
 *     crosses the t boundary picks up a factor -1.  All sixteen terms are
 *     summed even when neighbours coincide on tiny lattices.
 *   - normal operator on even sites: A v = m^2 v - D_eo (D_oe v).
 *   - CG: Hestenes-Stiefel conjugate gradients on A for each column
 *     (the baseline solver of Sec. 7.1), x0 given, stop on the recursive
 *     residual, confirm with the true residual and restart if needed.
 *
 * Spinor blocks are complex [n_rhs][Vh][3] on one parity (cb-indexed).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* OpenMP threads of the parallel loops (timing the oracle on 1 core or all);
 * returns the previous setting (1 without OpenMP) */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  int old = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return old;
#else
  (void)n;
  return 1;
#endif
}

typedef struct {
  int L[4];
  long V, Vh;
} lattice;

static int make_lattice(lattice* g, const int dims[4]) {
  long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || (dims[mu] & 1)) return -1;
    g->L[mu] = dims[mu];
    V *= dims[mu];
  }
  g->V = V;
  g->Vh = V / 2;
  return 0;
}

static void coords_of(const lattice* g, long i, int c[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = (int)(i % g->L[mu]);
    i /= g->L[mu];
  }
}

static long lex_of(const lattice* g, const int c[4]) {
  return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* lexicographic index of the site with checkerboard index cb and parity p */
static long lex_of_cb(const lattice* g, long cb, int p) {
  int c[4];
  long i = 2 * cb;
  coords_of(g, i, c);
  if (parity_of(c) != p) i += 1;
  return i;
}

/* staggered phase eta_mu(x) */
static double eta(int mu, const int c[4]) {
  int s = 0;
  for (int nu = 0; nu < mu; ++nu) s += c[nu];
  return (s & 1) ? -1.0 : 1.0;
}

/* coordinates of x + k*mu (periodic wrap) and the boundary sign of that hop */
static double hop(const lattice* g, const int c[4], int mu, int k, int antiperiodic_t, int out[4]) {
  memcpy(out, c, 4 * sizeof(int));
  int L = g->L[mu];
  int y = c[mu] + k;
  double sign = 1.0;
  if (mu == 3 && antiperiodic_t && (y < 0 || y >= L)) sign = -1.0;
  out[mu] = ((y % L) + L) % L;
  return sign;
}

static const cplx* link_at(const cplx* U, const lattice* g, int mu, long x) {
  return U + ((long)mu * g->V + x) * 9;
}

/* r += s * U psi */
static void add_U_psi(cplx r[3], double s, const cplx* U, const cplx* psi) {
  for (int a = 0; a < 3; ++a) {
    cplx acc = 0;
    for (int b = 0; b < 3; ++b) acc += U[a * 3 + b] * psi[b];
    r[a] += s * acc;
  }
}

/* r += s * U^dag psi */
static void add_Udag_psi(cplx r[3], double s, const cplx* U, const cplx* psi) {
  for (int a = 0; a < 3; ++a) {
    cplx acc = 0;
    for (int b = 0; b < 3; ++b) acc += conj(U[b * 3 + a]) * psi[b];
    r[a] += s * acc;
  }
}

/* (D psi)(x) at one site x (lexicographic); psi is a cb-indexed colour field
 * of the opposite parity, psi[cb*3 + colour]. */
static void dslash_site(const lattice* g, const cplx* fat, const cplx* lng, int antiperiodic_t,
                        const cplx* psi, long x, cplx out[3]) {
  int c[4], y[4];
  coords_of(g, x, c);
  out[0] = out[1] = out[2] = 0;
  for (int mu = 0; mu < 4; ++mu) {
    double e = 0.5 * eta(mu, c);
    double s;
    long yl;
    /* + F_mu(x) psi(x+mu) */
    s = hop(g, c, mu, +1, antiperiodic_t, y);
    yl = lex_of(g, y);
    add_U_psi(out, e * s, link_at(fat, g, mu, x), psi + (yl >> 1) * 3);
    /* - F_mu(x-mu)^dag psi(x-mu) */
    s = hop(g, c, mu, -1, antiperiodic_t, y);
    yl = lex_of(g, y);
    add_Udag_psi(out, -e * s, link_at(fat, g, mu, yl), psi + (yl >> 1) * 3);
    /* + G_mu(x) psi(x+3mu) */
    s = hop(g, c, mu, +3, antiperiodic_t, y);
    yl = lex_of(g, y);
    add_U_psi(out, e * s, link_at(lng, g, mu, x), psi + (yl >> 1) * 3);
    /* - G_mu(x-3mu)^dag psi(x-3mu) */
    s = hop(g, c, mu, -3, antiperiodic_t, y);
    yl = lex_of(g, y);
    add_Udag_psi(out, -e * s, link_at(lng, g, mu, yl), psi + (yl >> 1) * 3);
  }
}

/* out (parity out_parity) = D in (parity 1-out_parity), n_rhs columns */
int oracle_dslash(const int dims[4], const cplx* fat, const cplx* lng, int antiperiodic_t,
                  const cplx* in, cplx* out, int out_parity, int n_rhs) {
  lattice g;
  if (make_lattice(&g, dims) || n_rhs < 0 || (out_parity & ~1)) return -1;
  for (int j = 0; j < n_rhs; ++j) {
    const cplx* src = in + (long)j * g.Vh * 3;
    cplx* dst = out + (long)j * g.Vh * 3;
#pragma omp parallel for schedule(static)
    for (long cb = 0; cb < g.Vh; ++cb) {
      long x = lex_of_cb(&g, cb, out_parity);
      dslash_site(&g, fat, lng, antiperiodic_t, src, x, dst + cb * 3);
    }
  }
  return 0;
}

/* out = m^2 in - D_eo D_oe in   (even-site blocks) */
int oracle_apply_A(const int dims[4], const cplx* fat, const cplx* lng, int antiperiodic_t,
                   double mass, const cplx* in, cplx* out, int n_rhs) {
  lattice g;
  if (make_lattice(&g, dims) || n_rhs < 0) return -1;
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * g.Vh * 3);
  cplx* dd = (cplx*)malloc(sizeof(cplx) * g.Vh * 3);
  if (!tmp || !dd) {
    free(tmp);
    free(dd);
    return -2;
  }
  for (int j = 0; j < n_rhs; ++j) {
    const cplx* v = in + (long)j * g.Vh * 3;
    cplx* w = out + (long)j * g.Vh * 3;
    oracle_dslash(dims, fat, lng, antiperiodic_t, v, tmp, 1, 1); /* odd  = D_oe v  */
    oracle_dslash(dims, fat, lng, antiperiodic_t, tmp, dd, 0, 1); /* even = D_eo tmp */
    for (long k = 0; k < g.Vh * 3; ++k) w[k] = mass * mass * v[k] - dd[k];
  }
  free(tmp);
  free(dd);
  return 0;
}

/* (A v)(x) only at the listed even sites (lexicographic indices), for
 * sampled checks on lattices too large for a full CPU application.
 * in: one even-site column [Vh][3]; out: [n_sites][3]. */
int oracle_apply_A_sites(const int dims[4], const cplx* fat, const cplx* lng, int antiperiodic_t,
                         double mass, const cplx* in, const long* sites, long n_sites, cplx* out) {
  lattice g;
  if (make_lattice(&g, dims)) return -1;
  cplx* tmp = (cplx*)calloc((size_t)g.Vh * 3, sizeof(cplx));
  if (!tmp) return -2;
  for (long s = 0; s < n_sites; ++s) {
    int c[4], y[4];
    long x = sites[s];
    if (x < 0 || x >= g.V) {
      free(tmp);
      return -1;
    }
    coords_of(&g, x, c);
    if (parity_of(c) != 0) {
      free(tmp);
      return -1;
    }
    /* T = D_oe v on the sixteen odd neighbours of x */
    static const int ks[4] = {+1, -1, +3, -3};
    for (int mu = 0; mu < 4; ++mu)
      for (int q = 0; q < 4; ++q) {
        hop(&g, c, mu, ks[q], 0, y);
        long yl = lex_of(&g, y);
        dslash_site(&g, fat, lng, antiperiodic_t, in, yl, tmp + (yl >> 1) * 3);
      }
    cplx dd[3];
    dslash_site(&g, fat, lng, antiperiodic_t, tmp, x, dd);
    for (int a = 0; a < 3; ++a) out[s * 3 + a] = mass * mass * in[(x >> 1) * 3 + a] - dd[a];
  }
  free(tmp);
  return 0;
}

static cplx cdot(const cplx* a, const cplx* b, long n) { /* sum conj(a) b */
  cplx s = 0;
  for (long k = 0; k < n; ++k) s += conj(a[k]) * b[k];
  return s;
}

static double norm2(const cplx* a, long n) {
  double s = 0;
  for (long k = 0; k < n; ++k) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
  return s;
}

/*
 * Textbook CG on A for each column j of b (even-site block [n_rhs][Vh][3]).
 * x holds the initial guess on entry and the solution on exit.
 * Stops when the recursive residual |r|/|b| <= tol; then recomputes the true
 * residual b - A x and restarts (r = p = true residual) while it exceeds tol.
 * With max_iter iterations done and no convergence the column stops there.
 * iters[j], true_rel_res[j] are filled.  Returns 0, or 1 if any column did
 * not converge.
 */
int oracle_cg(const int dims[4], const cplx* fat, const cplx* lng, int antiperiodic_t, double mass,
              const cplx* b, cplx* x, int n_rhs, double tol, int max_iter, int* iters,
              double* true_rel_res) {
  lattice g;
  if (make_lattice(&g, dims) || n_rhs < 0) return -1;
  long n = g.Vh * 3;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  cplx* p = (cplx*)malloc(sizeof(cplx) * n);
  cplx* Ap = (cplx*)malloc(sizeof(cplx) * n);
  int rc = 0;
  for (int j = 0; j < n_rhs; ++j) {
    const cplx* bj = b + (long)j * n;
    cplx* xj = x + (long)j * n;
    double bnorm = sqrt(norm2(bj, n));
    int k = 0;
    double rel = 0;
    for (;;) {
      /* r = b - A x, p = r */
      oracle_apply_A(dims, fat, lng, antiperiodic_t, mass, xj, Ap, 1);
      for (long q = 0; q < n; ++q) r[q] = bj[q] - Ap[q];
      rel = bnorm > 0 ? sqrt(norm2(r, n)) / bnorm : 0.0;
      if (rel <= tol || k >= max_iter) break;
      memcpy(p, r, sizeof(cplx) * n);
      double rr = norm2(r, n);
      while (k < max_iter) {
        oracle_apply_A(dims, fat, lng, antiperiodic_t, mass, p, Ap, 1);
        double pAp = creal(cdot(p, Ap, n));
        double alpha = rr / pAp;
        for (long q = 0; q < n; ++q) {
          xj[q] += alpha * p[q];
          r[q] -= alpha * Ap[q];
        }
        ++k;
        double rr_new = norm2(r, n);
        if (sqrt(rr_new) <= tol * bnorm) break;
        double beta = rr_new / rr;
        for (long q = 0; q < n; ++q) p[q] = r[q] + beta * p[q];
        rr = rr_new;
      }
    }
    if (iters) iters[j] = k;
    if (true_rel_res) true_rel_res[j] = rel;
    if (rel > tol) rc = 1;
  }
  free(r);
  free(p);
  free(Ap);
  return rc;
}

/*
 * Plain textbook CG without any restart, for exactly n_iter iterations on a
 * single column (x0 = 0).  Used to compare iterates with another solver.
 */
int oracle_cg_iterates(const int dims[4], const cplx* fat, const cplx* lng, int antiperiodic_t,
                       double mass, const cplx* b, cplx* x, int n_iter) {
  lattice g;
  if (make_lattice(&g, dims)) return -1;
  long n = g.Vh * 3;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  cplx* p = (cplx*)malloc(sizeof(cplx) * n);
  cplx* Ap = (cplx*)malloc(sizeof(cplx) * n);
  memset(x, 0, sizeof(cplx) * n);
  memcpy(r, b, sizeof(cplx) * n);
  memcpy(p, b, sizeof(cplx) * n);
  double rr = norm2(r, n);
  for (int k = 0; k < n_iter; ++k) {
    oracle_apply_A(dims, fat, lng, antiperiodic_t, mass, p, Ap, 1);
    double alpha = rr / creal(cdot(p, Ap, n));
    for (long q = 0; q < n; ++q) {
      x[q] += alpha * p[q];
      r[q] -= alpha * Ap[q];
    }
    double rr_new = norm2(r, n);
    double beta = rr_new / rr;
    for (long q = 0; q < n; ++q) p[q] = r[q] + beta * p[q];
    rr = rr_new;
  }
  free(r);
  free(p);
  free(Ap);
  return 0;
}

/*
 * Gradient of a real loss L with respect to the fat and long links (the
 * derivative convention of complex automatic differentiation: for each link
 * entry u, G = dL/dRe(u) + i dL/dIm(u), so that dL = Re sum conj(G) du).
 * Inputs: the even-site solution block x = A^-1 phi and the adjoint block
 * lam = A^-1 g, g being the gradient of L with respect to x.
 *
 * Derivation (Sec. 3.2 operator): dx = -A^-1 dA x, so dL = -Re lam^dag dA x,
 * and with dA = -(dD_eo D_oe + D_eo dD_oe), D anti-Hermitian (D_eo^dag =
 * -D_oe, and the same for dD), y = D_oe x and mu = D_oe lam:
 *     dL = Re[lam^dag dD_eo y] + Re[x^dag dD_eo mu].
 * A link U_mu(z) (fat: k = 1, long: k = 3) enters D_eo as the forward hop of
 * the even site z, or (z odd) as the backward hop of the even site z + k mu,
 * with weight c = 1/2 eta_mu(z) s (s the hop's boundary sign; eta_mu does not
 * depend on x_mu).  Hence
 *     z even: G_mu(z) =  c sum_i [lam_i(z) y_i(z+k mu)^dag + x_i(z) mu_i(z+k mu)^dag]
 *     z odd:  G_mu(z) = -c sum_i [y_i(z) lam_i(z+k mu)^dag + mu_i(z) x_i(z+k mu)^dag].
 * gfat, glong: complex [4][V][3][3] (the links' layout), either may be NULL.
 */
int oracle_link_grad(const int dims[4], const cplx* fat, const cplx* lng, int antiperiodic_t,
                     const cplx* x, const cplx* lam, int n_rhs, cplx* gfat, cplx* glong) {
  lattice g;
  if (make_lattice(&g, dims) || n_rhs < 0) return -1;
  long n = (long)n_rhs * g.Vh * 3;
  cplx* y = (cplx*)malloc(sizeof(cplx) * (n ? n : 1));
  cplx* mu_ = (cplx*)malloc(sizeof(cplx) * (n ? n : 1));
  if (!y || !mu_) {
    free(y);
    free(mu_);
    return -2;
  }
  oracle_dslash(dims, fat, lng, antiperiodic_t, x, y, 1, n_rhs);   /* y  = D_oe x   */
  oracle_dslash(dims, fat, lng, antiperiodic_t, lam, mu_, 1, n_rhs); /* mu = D_oe lam */
  for (int which = 0; which < 2; ++which) {
    cplx* G = which ? glong : gfat;
    int k = which ? 3 : 1;
    if (!G) continue;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < g.V; ++z) {
      int c[4], w[4];
      coords_of(&g, z, c);
      int even = parity_of(c) == 0;
      for (int m = 0; m < 4; ++m) {
        double s = hop(&g, c, m, k, antiperiodic_t, w);
        long wl = lex_of(&g, w);
        double cf = 0.5 * eta(m, c) * s;
        cplx* out = G + ((long)m * g.V + z) * 9;
        for (int a = 0; a < 9; ++a) out[a] = 0;
        for (int i = 0; i < n_rhs; ++i) {
          const long off = (long)i * g.Vh * 3;
          /* even z: (lam, x) at z with (y, mu) at z + k mu;
             odd z:  (y, mu) at z with (lam, x) at z + k mu */
          const cplx *a1, *b1, *a2, *b2;
          if (even) {
            a1 = lam + off + (z >> 1) * 3;
            b1 = y + off + (wl >> 1) * 3;
            a2 = x + off + (z >> 1) * 3;
            b2 = mu_ + off + (wl >> 1) * 3;
          } else {
            a1 = y + off + (z >> 1) * 3;
            b1 = lam + off + (wl >> 1) * 3;
            a2 = mu_ + off + (z >> 1) * 3;
            b2 = x + off + (wl >> 1) * 3;
          }
          for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q)
              out[r * 3 + q] += (even ? cf : -cf) * (a1[r] * conj(b1[q]) + a2[r] * conj(b2[q]));
        }
      }
    }
  }
  free(y);
  free(mu_);
  return 0;
}
