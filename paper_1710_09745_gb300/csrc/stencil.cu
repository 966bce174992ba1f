// Multi-RHS improved-staggered stencil (Sec. 6.2, Eq. 2).
//
// Links are repacked once per gauge field (pack_links) into, for each output
// parity p and each of the 16 hops d = 4*mu + q (q: +1, -1, +3, -3 along mu),
// the matrix that multiplies psi(x + k_q mu) in Eq. 2 with everything folded
// in: 1/2, the staggered phase eta_mu(x), the boundary sign, and for the
// backward hops the dagger and the minus sign of the anti-Hermitian reading.
// Layout [p][site / LW][d * 9 + e][site % LW] (e = 0..8 matrix element,
// LW = 32 sites per block): the loads of one matrix element by consecutive
// sites are contiguous, and all 144 link words a group of sites needs lie in
// one LW * 144-element block instead of 144 streams a parity apart.
//
// One thread owns one output site and a register tile of R right-hand sides
// (the register tiling of Sec. 6.2); the T = ceil(N/R) threads of a site sit
// next to each other in a warp, so each link element is fetched once per
// warp and broadcast (the cache tiling of Sec. 6.2 maps onto the broadcast of
// a warp-wide load).  Spinor blocks are site-major [site][colour][rhs] and
// thread k of a site owns the right-hand sides k, k + T, k + 2T, ...: for one
// (colour, r) the T threads of a site read T consecutive elements, so every
// warp-wide load uses whole 32-byte sectors.
#include "stencil_kernels.cuh"

namespace bcg {

template <class S>
__global__ void k_pack_links(const double2* __restrict__ fat, const double2* __restrict__ lng,
                             typename S::elem* __restrict__ out, Geom g, int antiperiodic_t,
                             int E) {
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
  // E = 9: the whole matrix; E = 6: its first two rows (the third is rebuilt)
  typename S::elem* o = out + link_offset(g, p, cb, E) + (long long)d * E * LINK_W;
  for (int a = 0; a < E / 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double2 u = back ? make_double2(U[b * 3 + a].x, -U[b * 3 + a].y) : U[a * 3 + b];
      u.x *= factor;
      u.y *= factor;
      o[(long long)(a * 3 + b) * LINK_W] = S::from_double2(u);
    }
}

size_t links_bytes(FieldKind k, const Geom& g, int recon) {
  return 2ull * link_blocks(g) * 16 * (recon ? 6 : 9) * LINK_W * elem_bytes(k);
}

cudaError_t pack_links(FieldKind k, const double2* fat, const double2* lng, void* out,
                       const Geom& g, int antiperiodic_t, int recon, cudaStream_t s) {
  long long total = 2LL * 16 * g.Vh;
  int threads = 256;
  unsigned blocks = (unsigned)((total + threads - 1) / threads);
  const int E = recon ? 6 : 9;
  switch (k) {
    case FK_DF:
      k_pack_links<StoreDF><<<blocks, threads, 0, s>>>(fat, lng, (float4*)out, g, antiperiodic_t, E);
      break;
    case FK_F32:
      k_pack_links<StoreF32><<<blocks, threads, 0, s>>>(fat, lng, (float2*)out, g, antiperiodic_t, E);
      break;
    case FK_F64:
      k_pack_links<StoreF64><<<blocks, threads, 0, s>>>(fat, lng, (double2*)out, g, antiperiodic_t, E);
      break;
    case FK_H16:
      k_pack_links<StoreH16><<<blocks, threads, 0, s>>>(fat, lng, (__half2*)out, g, antiperiodic_t, E);
      break;
    case FK_BF16:
      k_pack_links<StoreBF16><<<blocks, threads, 0, s>>>(fat, lng, (__nv_bfloat162*)out, g, antiperiodic_t, E);
      break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------- scaled SU(3) check ----
__device__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ double2 det3(const double2* U) {
  const double2 m0 = cmul2(U[4], U[8]), m1 = cmul2(U[5], U[7]);
  const double2 n0 = cmul2(U[3], U[8]), n1 = cmul2(U[5], U[6]);
  const double2 o0 = cmul2(U[3], U[7]), o1 = cmul2(U[4], U[6]);
  const double2 a = cmul2(U[0], make_double2(m0.x - m1.x, m0.y - m1.y));
  const double2 b = cmul2(U[1], make_double2(n0.x - n1.x, n0.y - n1.y));
  const double2 c = cmul2(U[2], make_double2(o0.x - o1.x, o0.y - o1.y));
  return make_double2(a.x - b.x + c.x, a.y - b.y + c.y);
}

// one thread per link: U U^dag = c^2 I and det U = c^3 with c = cbrt(Re det)
// of the first link of the same kind (fat: kind 0, long: kind 1)
__global__ void k_check_scaled_su3(const double2* __restrict__ fat, const double2* __restrict__ lng,
                                   long long V, double tol, double* c_out, int* bad) {
  const long long n = 4 * V;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kind = idx >= n;
    const double2* L = kind ? lng : fat;
    const double2 d0 = det3(L);
    const double c = cbrt(d0.x);
    if (idx == 0 || idx == n) c_out[kind] = c;
    const double2* U = L + (idx - (kind ? n : 0)) * 9;
    const double c2 = c * c, c3 = c2 * c;
    bool ok = isfinite(c) && c != 0.0 && fabs(d0.y) <= tol * fabs(c3);
    for (int i = 0; i < 3 && ok; ++i)
      for (int j = 0; j < 3; ++j) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < 3; ++k) {  // (U U^dag)_ij = sum_k U_ik conj(U_jk)
          const double2 a = U[i * 3 + k], b = U[j * 3 + k];
          re += a.x * b.x + a.y * b.y;
          im += a.y * b.x - a.x * b.y;
        }
        if (i == j) re -= c2;
        if (!(fabs(re) <= tol * c2 && fabs(im) <= tol * c2)) ok = false;
      }
    if (ok) {
      const double2 d = det3(U);
      if (!(fabs(d.x - c3) <= tol * fabs(c3) && fabs(d.y) <= tol * fabs(c3))) ok = false;
    }
    if (!ok) atomicOr(bad, 1);
  }
}

cudaError_t check_scaled_su3(const double2* fat, const double2* lng, long long V, double tol,
                             double* c, int* bad, cudaStream_t s) {
  const long long n = 8 * V;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_check_scaled_su3<<<(unsigned)blocks, 256, 0, s>>>(fat, lng, V, tol, c, bad);
  return cudaGetLastError();
}

cudaError_t dslash(FieldKind k, int R, int epi, const void* links, const void* in, void* out,
                   const void* c1, const void* c2, double m2, const Geom& g, int out_parity,
                   int N, Gate gate, cudaStream_t s) {
  switch (k) {
    case FK_DF: return dslash_df(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
    case FK_F32: return dslash_f32(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
    case FK_F64: return dslash_f64(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
    case FK_H16: return dslash_h16(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
    case FK_BF16: return dslash_bf16(R, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bcg
