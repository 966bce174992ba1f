// Gradient of a real loss with respect to the fat and long links, for loss
// functions of the solution x = A^-1 phi of the Sec. 3.2 normal operator.
// (The paper solves and does not differentiate; this is the adjoint step of
// a differentiable solve.)
//
// With lam = A^-1 g the adjoint block (g the loss's gradient with respect to
// x), y = D_oe x and mu = D_oe lam, the loss changes by
//   dL = Re[lam^dag dD_eo y] + Re[x^dag dD_eo mu]
// (D and dD anti-Hermitian).  A link U_mu(z) (fat: hop k = 1, long: k = 3)
// enters D_eo as the forward hop of z when z is even, and as the backward hop
// of z + k mu when z is odd, with weight c = 1/2 eta_mu(z) s (s the hop's
// boundary sign), so per link, in the convention G = dL/dRe + i dL/dIm:
//   z even:  G =  c sum_i [lam_i(z) y_i(z+k mu)^dag + x_i(z) mu_i(z+k mu)^dag]
//   z odd:   G = -c sum_i [y_i(z) lam_i(z+k mu)^dag + mu_i(z) x_i(z+k mu)^dag]
// One thread per (direction, site) forms both links' 3x3 outer-product sums
// over the N right-hand sides in native FP64 and writes them in the links'
// user layout [4][V][3][3].
#include "internal.h"

namespace bcg {

__global__ void __launch_bounds__(256)
    k_link_grad(const double2* __restrict__ X, const double2* __restrict__ Lam,
                const double2* __restrict__ Y, const double2* __restrict__ Mu,
                double2* __restrict__ gfat, double2* __restrict__ glong, Geom g, int N,
                int antiperiodic_t) {
  const long long V = 2LL * g.Vh;
  for (long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x; tid < 4 * V;
       tid += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(tid / V);
    const long long z = tid - (long long)mu * V;
    int c[4];
    long long r = z;
    for (int d = 0; d < 4; ++d) {
      c[d] = (int)(r % g.L[d]);
      r /= g.L[d];
    }
    const bool even = ((c[0] + c[1] + c[2] + c[3]) & 1) == 0;
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += c[nu];
    const double eta = (s & 1) ? -1.0 : 1.0;
    for (int which = 0; which < 2; ++which) {
      double2* G = which ? glong : gfat;
      if (!G) continue;
      const int k = which ? 3 : 1;
      int w[4] = {c[0], c[1], c[2], c[3]};
      const int yv = c[mu] + k;
      double cf = 0.5 * eta;
      if (antiperiodic_t && mu == 3 && yv >= g.L[3]) cf = -cf;
      w[mu] = yv % g.L[mu];
      const long long wl =
          w[0] + (long long)g.L[0] * (w[1] + (long long)g.L[1] * (w[2] + (long long)g.L[2] * w[3]));
      const long long zc = z >> 1, wc = wl >> 1;
      // (a1 b1^dag + a2 b2^dag): a at z, b at z + k mu
      const double2* a1 = (even ? Lam : Y) + zc * 3 * N;
      const double2* b1 = (even ? Y : Lam) + wc * 3 * N;
      const double2* a2 = (even ? X : Mu) + zc * 3 * N;
      const double2* b2 = (even ? Mu : X) + wc * 3 * N;
      double2 acc[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) acc[e] = make_double2(0.0, 0.0);
      for (int i = 0; i < N; ++i) {
        double2 va1[3], vb1[3], va2[3], vb2[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          va1[q] = a1[q * N + i];
          vb1[q] = b1[q * N + i];
          va2[q] = a2[q * N + i];
          vb2[q] = b2[q * N + i];
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            // a b^dag = a * conj(b)
            double2& o = acc[p * 3 + q];
            o.x = fma(va1[p].x, vb1[q].x, o.x);
            o.x = fma(va1[p].y, vb1[q].y, o.x);
            o.y = fma(va1[p].y, vb1[q].x, o.y);
            o.y = fma(-va1[p].x, vb1[q].y, o.y);
            o.x = fma(va2[p].x, vb2[q].x, o.x);
            o.x = fma(va2[p].y, vb2[q].y, o.x);
            o.y = fma(va2[p].y, vb2[q].x, o.y);
            o.y = fma(-va2[p].x, vb2[q].y, o.y);
          }
      }
      const double f = even ? cf : -cf;
      double2* out = G + ((long long)mu * V + z) * 9;
#pragma unroll
      for (int e = 0; e < 9; ++e) out[e] = make_double2(f * acc[e].x, f * acc[e].y);
    }
  }
}

cudaError_t link_grad(const double2* X, const double2* Lam, const double2* Y, const double2* Mu,
                      double2* gfat, double2* glong, const Geom& g, int N, int antiperiodic_t,
                      cudaStream_t s) {
  const long long n = 8LL * g.Vh;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_link_grad<<<(unsigned)blocks, 256, 0, s>>>(X, Lam, Y, Mu, gfat, glong, g, N, antiperiodic_t);
  return cudaGetLastError();
}

}  // namespace bcg
