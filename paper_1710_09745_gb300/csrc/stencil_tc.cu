// Tensor-core double-float stencil: the hopping term of Eq. 2 for a block of
// N = 16 or 32 right-hand sides (Sec. 6.2: every link loaded once per site and
// applied to all N spinors) with the products on the tensor cores.
//
// Why.  The FP64-accurate form keeps its iteration fields in double-float
// (hi + lo FP32 pairs); on the FP32 pipes each double-float multiply-add costs
// 12 instructions and the CUDA-core stencil is bound by instruction issue.
// Per output site the stencil is a small dense product: with the 16 hops and
// 3 colours as a K index of 48 complex (96 real) entries,
//     out^T (N x 3 complex) = Psi^T (N x 48) U^T (48 x 3),
// Psi the gathered neighbour spinors and U the site's 16 hop matrices, i.e.
// in real form D[n][o] = sum_k A[n][k] B[k][o] with n = right-hand side (the
// MMA's M), k = (hop, colour, re/im) (K = 96) and o = (colour, re/im) (6 of
// the MMA's N = 8).  One warp computes one site with mma.sync m16n8k16 (M = 16
// right-hand sides per M tile): the product has a different B (the site's
// links) for every site, which the 64-row minimum of a tcgen05 product cannot
// share, while the warp-level form fits it exactly.
//
// Exact split products (Ozaki's scheme).  Every double-float value is scaled
// by a power of two so that it lies in (-1, 1) and written as six bf16 slices
// x = sum_k x_k, x_k on the grid 2^(-7-8k) with |x_k| <= 1.5 * 2^(-8k) (at
// most 8 significant bits: exact in bf16); the first three come from hi, the
// last three from (hi's remainder + lo), so the slices represent x to
// 2^-47.  Scales: one per right-hand side for A (the column maximum of the
// input field, found by k_colmax before the stencil), one per site for B (the
// site's largest link entry).  The products A_s B_t with s + t = u <= 5 are
// accumulated into one FP32 accumulator D_u: all their terms are multiples
// of the same power of two 2^(-14-8u) and the sum of the 96 x (u + 1) terms
// stays below 2^24 of those units, so the tensor-core accumulation is exact.
// The epilogue adds D_0 .. D_5 in double-float and removes the scales (exact
// powers of two).  Error: about 2^-45 of (column max x link max) per term,
// the double-float level of the CUDA-core stencil.
#include "ozaki.cuh"
#include "stencil_kernels.cuh"

namespace bcg {

namespace {

constexpr int TC_SITES = 8;               // sites (one per warp) per CTA
constexpr int TC_LSTRIDE = 16 * 9 + 1;    // staged link elements per site (+1: banks)

}  // namespace

using namespace ozaki;

// Per-column maxima of |hi| (real and imaginary parts) of a double-float
// block field [site][colour][rhs], as float bit patterns (non-negative floats
// order like their bits).  colmax must hold N zeros (k_colmax_zero).
__global__ void k_colmax_zero(unsigned* colmax, int N, Gate gate) {
  if (gate_closed(gate)) return;
  if ((int)threadIdx.x < N) colmax[threadIdx.x] = 0u;
}

template <int N>
__global__ void __launch_bounds__(256) k_colmax(const float4* __restrict__ f, long long n_elems,
                                                unsigned* __restrict__ colmax, Gate gate) {
  __shared__ unsigned sm[N];
  if (gate_closed(gate)) return;
  if (threadIdx.x < N) sm[threadIdx.x] = 0u;
  __syncthreads();
  float m = 0.f;
  // the grid stride is a multiple of N (N divides 256), so a thread's elements
  // all belong to column threadIdx.x % N
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_elems; i += stride) {
    const float4 v = __ldg(f + i);
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  atomicMax(&sm[threadIdx.x % N], __float_as_uint(m));
  __syncthreads();
  if (threadIdx.x < N) atomicMax(colmax + threadIdx.x, sm[threadIdx.x]);
}

// One warp per output site (TC_SITES sites per CTA, the CTA's links staged
// in shared memory with coalesced loads, then each warp splits its site's
// 144 link entries once into bf16 slice words), MT M tiles of 16
// right-hand sides.  Lane = (gq, tig) = (lane / 4, lane % 4) in the MMA
// fragment layout: rows gq and gq + 8 of A (right-hand sides), K columns
// (complex entries) tig and tig + 4 of each 8-entry chunk, output column gq
// of B, outputs (colour tig, right-hand sides gq and gq + 8) of D.
// Each thread splits the double-float values it gathers; the values of
// chunk q + 1 are loaded while chunk q is split and multiplied.
template <int EPI, int MT>
__global__ void __launch_bounds__(TC_SITES * 32, 2)
    k_dslash_tc(const float4* __restrict__ links, const float4* __restrict__ in,
                float4* __restrict__ out,
                const float4* __restrict__ c1, const float4* __restrict__ c2, double m2d, Geom g,
                int parity, const unsigned* __restrict__ colmax, Gate gate) {
  using C = CompDF;
  constexpr int N = 16 * MT;
  __shared__ float4 sL[TC_SITES * TC_LSTRIDE];
  // per site: 144 entries x 6 slice words, words 0..3 in sB4, 4..5 in sB2
  __shared__ uint4 sB4[TC_SITES * 144];
  __shared__ uint2 sB2[TC_SITES * 144];
  if (gate_closed(gate)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tig = lane & 3;
  // A scales of this thread's rows n = gq + 8 r: 2^-e with max |hi| < 2^e
  int er[2 * MT];
  float ra[2 * MT];
#pragma unroll
  for (int r = 0; r < 2 * MT; ++r) {
    er[r] = pow2_above(__ldg(colmax + gq + 8 * r));
    ra[r] = exp2i(-er[r]);
  }
  const C::real m2 = C::from_double(m2d);
  const long long ngroups = ((long long)g.Vh + TC_SITES - 1) / TC_SITES;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int s0 = (int)(grp * TC_SITES);
    __syncthreads();  // the previous group's reads of sL and sB are done
    {
      // s0 % 32 is 0, 8, 16 or 24: the TC_SITES sites share one link block
      const float4* lb = links + link_offset(g, parity, s0);
      for (int i = threadIdx.x; i < 144 * TC_SITES; i += blockDim.x) {
        const int de = i / TC_SITES, k = i - de * TC_SITES;
        sL[k * TC_LSTRIDE + de] = __ldg(lb + (long long)de * LINK_W + k);
      }
    }
    __syncthreads();
    const int site = s0 + warp;
    if (site >= g.Vh) continue;  // warp-uniform
    const float4* Ls = sL + warp * TC_LSTRIDE;
    uint4* Bs4 = sB4 + warp * 144;
    uint2* Bs2 = sB2 + warp * 144;
    // B scale: the site's largest link entry
    float lm = 0.f;
    for (int i = lane; i < 144; i += 32) {
      const float4 v = Ls[i];
      lm = fmaxf(lm, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) lm = fmaxf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    const int eu = pow2_above(__float_as_uint(lm));
    const float us = exp2i(-eu);
    // the site's links as slice words (Re slice k, Im slice k), once per site
    for (int i = lane; i < 144; i += 32) {
      const float4 u = Ls[i];
      float sr[6], si[6];
      split6(__fmul_rn(u.x, us), __fmul_rn(u.z, us), sr);
      split6(__fmul_rn(u.y, us), __fmul_rn(u.w, us), si);
      Bs4[i] = make_uint4(pack_bf16(sr[0], si[0]), pack_bf16(sr[1], si[1]),
                          pack_bf16(sr[2], si[2]), pack_bf16(sr[3], si[3]));
      Bs2[i] = make_uint2(pack_bf16(sr[4], si[4]), pack_bf16(sr[5], si[5]));
    }
    __syncwarp();
    // neighbour of hop d = 4 mu + q computed by lane d (lanes 16..31 repeat them)
    int x, y, z, t;
    site_xyzt(g, site, parity, x, y, z, t);
    const int lex = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
    const int nbl = neighbour_cb_s(g, lex, x, y, z, t, (lane >> 2) & 3, hop_k(lane & 3));

    float acc[6][MT][4];
#pragma unroll
    for (int u = 0; u < 6; ++u)
#pragma unroll
      for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[u][m][i] = 0.f;

    const int bc = gq < 6 ? gq >> 1 : 0;  // colour of B column gq (6, 7: zero padding)
    const bool bim = gq & 1;              // column gq is the imaginary part
    // the double-float values of chunk q + 1 are loaded while chunk q is
    // split and multiplied (two chunks of loads in flight)
    float4 vn[MT][4];
    auto load_chunk = [&](int q, float4 (&dst)[MT][4]) {
      const int kc0 = 8 * q + tig, kc1 = kc0 + 4;
      const int d0 = kc0 / 3, j0 = kc0 - 3 * d0;
      const int d1 = kc1 / 3, j1 = kc1 - 3 * d1;
      const int nb0 = __shfl_sync(0xffffffffu, nbl, d0);
      const int nb1 = __shfl_sync(0xffffffffu, nbl, d1);
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        const long long e0 = ((long long)nb0 * 3 + j0) * N + 16 * m + gq;
        const long long e1 = ((long long)nb1 * 3 + j1) * N + 16 * m + gq;
        dst[m][0] = __ldg(in + e0);
        dst[m][1] = __ldg(in + e0 + 8);
        dst[m][2] = __ldg(in + e1);
        dst[m][3] = __ldg(in + e1 + 8);
      }
    };
    load_chunk(0, vn);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      // complex K entries kc0 = 8q + tig and kc1 = kc0 + 4 = (hop d, colour j)
      const int kc0 = 8 * q + tig, kc1 = kc0 + 4;
      const int d0 = kc0 / 3, j0 = kc0 - 3 * d0;
      const int d1 = kc1 / 3, j1 = kc1 - 3 * d1;
      // B fragments from the slice words w = (Re, Im): column (c, re) takes
      // (Re U_cj, -Im U_cj) = w with the high half negated, column (c, im)
      // takes (Im U_cj, Re U_cj) = w with its halves swapped
      uint32_t bf[6][2];
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int ent = (w ? d1 : d0) * 9 + bc * 3 + (w ? j1 : j0);
        const uint4 x0 = Bs4[ent];
        const uint2 x1 = Bs2[ent];
        const uint32_t ws[6] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y};
#pragma unroll
        for (int s = 0; s < 6; ++s)
          bf[s][w] = gq >= 6 ? 0u : bim ? __byte_perm(ws[s], 0u, 0x1032) : (ws[s] ^ 0x80000000u);
      }
        float4 v[MT][4];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
          for (int i = 0; i < 4; ++i) v[m][i] = vn[m][i];
        if (q < 5) load_chunk(q + 1, vn);
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          // raw hi and lo of the 8 reals (re, im of the 4 values) and their
          // scales (rows gq for i even, gq + 8 for i odd); the scaling is
          // folded into the first rounding and into the lo addition (fused
          // multiply-adds by a power of two: the same roundings as scaling
          // first)
          float x[8], l[8], sc[8], h[8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float c = ra[2 * m + (i & 1)];
            x[2 * i] = v[m][i].x;
            l[2 * i] = v[m][i].z;
            x[2 * i + 1] = v[m][i].y;
            l[2 * i + 1] = v[m][i].w;
            sc[2 * i] = sc[2 * i + 1] = c;
          }
          // slice s of every value (the steps of split6, one slice at a
          // time), multiplied at once into D_{s+t} for t = 0 .. 5 - s
#pragma unroll
          for (int s = 0; s < 6; ++s) {
            constexpr float CS[6] = {98304.f, 384.f, 1.5f, 0.005859375f, 2.288818359375e-05f,
                                     8.940696716308594e-08f};
            float sl[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (s == 0) {
                sl[k] = __fsub_rn(__fmaf_rn(x[k], sc[k], CS[0]), CS[0]);
                h[k] = __fmaf_rn(x[k], sc[k], -sl[k]);
              } else {
                sl[k] = rnd_grid(h[k], CS[s]);
                if (s == 2)
                  h[k] = __fmaf_rn(l[k], sc[k], __fsub_rn(h[k], sl[k]));
                else if (s < 5)
                  h[k] = __fsub_rn(h[k], sl[k]);
              }
            }
            uint32_t a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = pack_bf16(sl[2 * i], sl[2 * i + 1]);
#pragma unroll
            for (int t = 0; t + s < 6; ++t) mma_bf16(acc[s + t][m], a, bf[t][0], bf[t][1]);
          }
        }
    }
    // outputs: colour tig (tig < 3), right-hand sides 16 m + gq + 8 h
    if (tig < 3) {
#pragma unroll
      for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int n = 16 * m + gq + 8 * h;
          // remove the scales 2^-er and 2^-eu (two steps: each stays in range)
          const float fa = exp2i(er[2 * m + h]), fb = exp2i(eu);
          cpx<C::acc> vv;
          vv.re = combine6(acc[0][m][2 * h], acc[1][m][2 * h], acc[2][m][2 * h], acc[3][m][2 * h],
                           acc[4][m][2 * h], acc[5][m][2 * h]);
          vv.im = combine6(acc[0][m][2 * h + 1], acc[1][m][2 * h + 1], acc[2][m][2 * h + 1],
                           acc[3][m][2 * h + 1], acc[4][m][2 * h + 1], acc[5][m][2 * h + 1]);
          vv.re.s = __fmul_rn(__fmul_rn(vv.re.s, fa), fb);
          vv.re.e = __fmul_rn(__fmul_rn(vv.re.e, fa), fb);
          vv.im.s = __fmul_rn(__fmul_rn(vv.im.s, fa), fb);
          vv.im.e = __fmul_rn(__fmul_rn(vv.im.e, fa), fb);
          const long long oi = ((long long)site * 3 + tig) * N + n;
          if (EPI != EPI_NONE) {
            C::neg(vv.re);
            C::neg(vv.im);
            const cpx<C::real> cc = StoreDF::load(c1 + oi);
            C::mac(vv.re, m2, cc.re);
            C::mac(vv.im, m2, cc.im);
            if (EPI == EPI_RESIDUAL) {
              C::neg(vv.re);
              C::neg(vv.im);
              const cpx<C::real> bb = StoreDF::load(c2 + oi);
              C::add(vv.re, bb.re);
              C::add(vv.im, bb.im);
            }
          }
          StoreDF::store(out + oi, cfin<C>(vv));
        }
    }
  }
}

bool dslash_tc_supported(const Geom& g, int N) {
  return g.tc_colmax != nullptr && (N == 16 || N == 32);
}

template <int EPI, int MT>
static cudaError_t launch_tc(const float4* links, const float4* in, float4* out, const float4* c1,
                             const float4* c2, double m2, const Geom& g, int parity, Gate gate,
                             cudaStream_t s) {
  auto kern = k_dslash_tc<EPI, MT>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_SITES * 32, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long ngroups = ((long long)g.Vh + TC_SITES - 1) / TC_SITES;
  const long long want = (long long)stencil_sms() * per_sm;
  const unsigned blocks = (unsigned)(ngroups < want ? ngroups : want);
  kern<<<blocks, TC_SITES * 32, 0, s>>>(links, in, out, c1, c2, m2, g, parity, g.tc_colmax, gate);
  return cudaGetLastError();
}

template <int MT>
static cudaError_t launch_tc_epi(int epi, const float4* L, const float4* I, float4* O,
                                 const float4* A, const float4* B, double m2, const Geom& g,
                                 int p, Gate gate, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE: return launch_tc<EPI_NONE, MT>(L, I, O, A, B, m2, g, p, gate, s);
    case EPI_NORMAL: return launch_tc<EPI_NORMAL, MT>(L, I, O, A, B, m2, g, p, gate, s);
    default: return launch_tc<EPI_RESIDUAL, MT>(L, I, O, A, B, m2, g, p, gate, s);
  }
}

// column maxima of `in` into g.tc_colmax, then the tensor-core stencil
cudaError_t dslash_df_tc(int epi, const void* links, const void* in, void* out, const void* c1,
                         const void* c2, double m2, const Geom& g, int out_parity, int N,
                         Gate gate, cudaStream_t s) {
  if (!dslash_tc_supported(g, N)) return cudaErrorInvalidValue;
  k_colmax_zero<<<1, 64, 0, s>>>(g.tc_colmax, N, gate);
  const long long n_elems = (long long)g.Vh * 3 * N;
  const long long cb = (n_elems + 255) / 256;
  const long long cap = (long long)stencil_sms() * 4;
  const unsigned cblocks = (unsigned)(cb < cap ? cb : cap);
  const float4* I = (const float4*)in;
  if (N == 16)
    k_colmax<16><<<cblocks, 256, 0, s>>>(I, n_elems, g.tc_colmax, gate);
  else
    k_colmax<32><<<cblocks, 256, 0, s>>>(I, n_elems, g.tc_colmax, gate);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const float4 *L = (const float4*)links, *A = (const float4*)c1, *B = (const float4*)c2;
  float4* O = (float4*)out;
  if (N == 16) return launch_tc_epi<1>(epi, L, I, O, A, B, m2, g, out_parity, gate, s);
  return launch_tc_epi<2>(epi, L, I, O, A, B, m2, g, out_parity, gate, s);
}

}  // namespace bcg
