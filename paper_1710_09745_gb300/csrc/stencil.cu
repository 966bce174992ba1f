// Multi-RHS improved-staggered stencil (Sec. 5.2, Eq. 1).
//
// Links are repacked once per gauge field (pack_links) into, for each output
// parity p and each of the 16 hops d = 4*mu + q (q: +1, -1, +3, -3 along mu),
// the matrix that multiplies psi(x + k_q mu) in Eq. 1 with everything folded
// in: 1/2, the staggered phase eta_mu(x), the boundary sign, and for the
// backward hops the dagger and the minus sign of the anti-Hermitian reading.
// Layout [p][d][e][Vh] (e = 0..8 matrix element, site fastest), so that the
// loads of one matrix element by consecutive sites are contiguous.
//
// One thread owns one output site and a register tile of R right-hand sides
// (the register tiling of Sec. 5.2); the T = ceil(N/R) threads of a site sit
// next to each other in a warp, so each link element is fetched once per
// warp and broadcast (the cache tiling of Sec. 5.2 maps onto the broadcast of
// a warp-wide load).  Spinor blocks are site-major [site][rhs][colour], so the
// R x 3 neighbour values a thread needs are contiguous.
#include "internal.h"

namespace bcg {

template <class S>
__global__ void k_pack_links(const double2* __restrict__ fat, const double2* __restrict__ lng,
                             typename S::elem* __restrict__ out, Geom g, int antiperiodic_t) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = 2LL * 16 * g.Vh;
  if (tid >= total) return;
  int cb = (int)(tid % g.Vh);
  int d = (int)((tid / g.Vh) % 16);
  int p = (int)(tid / (16LL * g.Vh));
  int c[4];
  site_coords(g, cb, p, c);
  int mu = d >> 2, q = d & 3, k = hop_k(q);
  long long V = 2LL * g.Vh;
  // staggered phase
  int s = 0;
  for (int nu = 0; nu < mu; ++nu) s += c[nu];
  double factor = 0.5 * ((s & 1) ? -1.0 : 1.0);
  // boundary sign of the hop
  int y = c[mu] + k;
  if (antiperiodic_t && mu == 3 && (y < 0 || y >= g.L[3])) factor = -factor;
  // link site: x for forward hops, x + k*mu for backward hops
  int ls[4] = {c[0], c[1], c[2], c[3]};
  if (k < 0) {
    int v = y;
    while (v < 0) v += g.L[mu];
    ls[mu] = v;
  }
  long long lex = ls[0] + (long long)g.L[0] * (ls[1] + (long long)g.L[1] * (ls[2] + (long long)g.L[2] * ls[3]));
  const double2* U = ((q & 2) ? lng : fat) + ((long long)mu * V + lex) * 9;
  bool back = (k < 0);
  if (back) factor = -factor;
  typename S::elem* o = out + (((long long)p * 16 + d) * 9) * g.Vh + cb;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double2 u = back ? make_double2(U[b * 3 + a].x, -U[b * 3 + a].y) : U[a * 3 + b];
      u.x *= factor;
      u.y *= factor;
      o[(long long)(a * 3 + b) * g.Vh] = S::from_double2(u);
    }
}

template <class S, int R, int EPI>
__global__ void __launch_bounds__(128)
    k_dslash(const typename S::elem* __restrict__ links, const typename S::elem* __restrict__ in,
             typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
             const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity, int N,
             int T, Gate gate) {
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  if (gate_closed(gate)) return;
  long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int site = (int)(gid / T);
  int tile = (int)(gid - (long long)site * T);
  if (site >= g.Vh) return;
  int c[4];
  site_coords(g, site, parity, c);
  const int r0 = tile * R;
  const int nr = min(R, N - r0);

  cpx<acc> a[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i) a[r][i] = czero<C>();

  const typename S::elem* lp = links + (long long)parity * 16 * 9 * g.Vh + site;
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int d = mu * 4 + q;
      const int nb = neighbour_cb(g, c, mu, hop_k(q));
      cpx<real> U[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) U[e] = S::load(lp + (long long)(d * 9 + e) * g.Vh);
      const typename S::elem* ip = in + ((long long)nb * N + r0) * 3;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r < nr) {
          cpx<real> v0 = S::load(ip + r * 3 + 0);
          cpx<real> v1 = S::load(ip + r * 3 + 1);
          cpx<real> v2 = S::load(ip + r * 3 + 2);
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            cmac<C>(a[r][i], U[i * 3 + 0], v0);
            cmac<C>(a[r][i], U[i * 3 + 1], v1);
            cmac<C>(a[r][i], U[i * 3 + 2], v2);
          }
        }
      }
    }
  }
  const long long ob = ((long long)site * N + r0) * 3;
  const real m2 = C::from_double(m2d);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r < nr) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        cpx<acc> v = a[r][i];
        if (EPI != EPI_NONE) {
          // m2 * c1 - D in
          C::neg(v.re);
          C::neg(v.im);
          cpx<real> cc = S::load(c1 + ob + r * 3 + i);
          C::mac(v.re, m2, cc.re);
          C::mac(v.im, m2, cc.im);
          if (EPI == EPI_RESIDUAL) {  // c2 - (m2 c1 - D in)
            C::neg(v.re);
            C::neg(v.im);
            cpx<real> bb = S::load(c2 + ob + r * 3 + i);
            C::add(v.re, bb.re);
            C::add(v.im, bb.im);
          }
        }
        S::store(out + ob + r * 3 + i, cfin<C>(v));
      }
    }
  }
}

size_t links_bytes(FieldKind k, const Geom& g) { return 2ull * 16 * 9 * g.Vh * elem_bytes(k); }

cudaError_t pack_links(FieldKind k, const double2* fat, const double2* lng, void* out,
                       const Geom& g, int antiperiodic_t, cudaStream_t s) {
  long long total = 2LL * 16 * g.Vh;
  int threads = 256;
  unsigned blocks = (unsigned)((total + threads - 1) / threads);
  switch (k) {
    case FK_DF:
      k_pack_links<StoreDF><<<blocks, threads, 0, s>>>(fat, lng, (float4*)out, g, antiperiodic_t);
      break;
    case FK_F32:
      k_pack_links<StoreF32><<<blocks, threads, 0, s>>>(fat, lng, (float2*)out, g, antiperiodic_t);
      break;
    case FK_F64:
      k_pack_links<StoreF64><<<blocks, threads, 0, s>>>(fat, lng, (double2*)out, g, antiperiodic_t);
      break;
  }
  return cudaGetLastError();
}

template <class S, int R, int EPI>
static void launch_dslash_t(const void* links, const void* in, void* out, const void* c1,
                            const void* c2, double m2, const Geom& g, int parity, int N,
                            Gate gate, cudaStream_t s) {
  using E = typename S::elem;
  int T = (N + R - 1) / R;
  long long threads_total = (long long)g.Vh * T;
  int threads = 128;
  unsigned blocks = (unsigned)((threads_total + threads - 1) / threads);
  k_dslash<S, R, EPI><<<blocks, threads, 0, s>>>((const E*)links, (const E*)in, (E*)out,
                                                   (const E*)c1, (const E*)c2, m2, g, parity, N,
                                                   T, gate);
}

template <class S, int R>
static void launch_dslash_r(int epi, const void* links, const void* in, void* out, const void* c1,
                            const void* c2, double m2, const Geom& g, int parity, int N,
                            Gate gate, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE:
      launch_dslash_t<S, R, EPI_NONE>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    case EPI_NORMAL:
      launch_dslash_t<S, R, EPI_NORMAL>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    default:
      launch_dslash_t<S, R, EPI_RESIDUAL>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
  }
}

template <class S>
static void launch_dslash_s(int R, int epi, const void* links, const void* in, void* out,
                            const void* c1, const void* c2, double m2, const Geom& g, int parity,
                            int N, Gate gate, cudaStream_t s) {
  switch (R) {
    case 1:
      launch_dslash_r<S, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    case 2:
      launch_dslash_r<S, 2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    case 4:
      launch_dslash_r<S, 4>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    default:
      launch_dslash_r<S, 8>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
  }
}

cudaError_t dslash(FieldKind k, int R, int epi, const void* links, const void* in, void* out,
                   const void* c1, const void* c2, double m2, const Geom& g, int out_parity,
                   int N, Gate gate, cudaStream_t s) {
  switch (k) {
    case FK_DF:
      launch_dslash_s<StoreDF>(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
      break;
    case FK_F32:
      launch_dslash_s<StoreF32>(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
      break;
    case FK_F64:
      launch_dslash_s<StoreF64>(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
      break;
  }
  return cudaGetLastError();
}

}  // namespace bcg
