// Tensor-core stencil for the 16-bit storage kinds (FP16 with its 2^4 factor,
// bfloat16): the hopping term of Eq. 2 for N = 16 or 32 right-hand sides
// (Sec. 6.2) as per-site products on mma.sync with FP32 accumulation.
//
// The stored 16-bit spinors and links are exact MMA operands, so nothing is
// split (compare stencil_tc.cu): with the 16 hops and 3 colours as a K index
// of 96 reals, one warp computes one site's out^T = Psi^T U^T, A = the
// gathered neighbour spinors (M = 16 right-hand sides per tile; a stored
// (re, im) pair is one A register as it is), B = the site's hop matrices in
// real form (6 of the 8 columns), FP32 accumulation as in the CUDA-core
// kernel's FP32 arithmetic.  A thread's registers: 4 gathered words and 4
// accumulators per chunk and M tile, so many warps stay resident to hide the
// gather latency that bounds the CUDA-core 16-bit stencil.
#include "stencil_kernels.cuh"

namespace bcg {

namespace {

constexpr int T16_SITES = 8;             // sites (one per warp) per CTA
constexpr int T16_LSTRIDE = 16 * 9 + 1;  // staged link words per site (+1: banks)

template <class S>
struct Tc16Mma;
template <>
struct Tc16Mma<StoreH16> {
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                             uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};
template <>
struct Tc16Mma<StoreBF16> {
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                             uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};

}  // namespace

// Lane = (gq, tig) as in k_dslash_tc: rows gq, gq + 8 of A (right-hand
// sides), complex K entries tig and tig + 4 of each 8-entry chunk, B column
// gq, outputs (colour tig, right-hand sides gq and gq + 8).
template <class S, int EPI, int MT>
__global__ void __launch_bounds__(T16_SITES * 32, 4)
    k_dslash_tc16(const uint32_t* __restrict__ links, const uint32_t* __restrict__ in,
                  typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
                  const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity,
                  Gate gate) {
  constexpr int N = 16 * MT;
  constexpr float unraw = 1.f / (S::RAW_SCALE * S::RAW_SCALE);
  __shared__ uint32_t sL[T16_SITES * T16_LSTRIDE];
  if (gate_closed(gate)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tig = lane & 3;
  const float m2 = (float)m2d;
  const int bc = gq < 6 ? gq >> 1 : 0;  // colour of B column gq (6, 7: zero padding)
  const bool bim = gq & 1;              // column gq is the imaginary part
  const long long ngroups = ((long long)g.Vh + T16_SITES - 1) / T16_SITES;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int s0 = (int)(grp * T16_SITES);
    __syncthreads();  // the previous group's reads of sL are done
    {
      // s0 % 32 is 0, 8, 16 or 24: the sites share one link block
      const uint32_t* lb = links + link_offset(g, parity, s0);
      for (int i = threadIdx.x; i < 144 * T16_SITES; i += blockDim.x) {
        const int de = i / T16_SITES, k = i - de * T16_SITES;
        sL[k * T16_LSTRIDE + de] = __ldg(lb + (long long)de * LINK_W + k);
      }
    }
    __syncthreads();
    const int site = s0 + warp;
    if (site >= g.Vh) continue;  // warp-uniform
    const uint32_t* Ls = sL + warp * T16_LSTRIDE;
    int x, y, z, t;
    site_xyzt(g, site, parity, x, y, z, t);
    const int lex = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
    const int nbl = neighbour_cb_s(g, lex, x, y, z, t, (lane >> 2) & 3, hop_k(lane & 3));
    float acc[MT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[m][i] = 0.f;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int kc0 = 8 * q + tig, kc1 = kc0 + 4;
      const int d0 = kc0 / 3, j0 = kc0 - 3 * d0;
      const int d1 = kc1 / 3, j1 = kc1 - 3 * d1;
      const int nb0 = __shfl_sync(0xffffffffu, nbl, d0);
      const int nb1 = __shfl_sync(0xffffffffu, nbl, d1);
      // B from a stored link word w = (Re, Im): column (c, re) takes
      // (Re U_cj, -Im U_cj) = w with the high half negated, column (c, im)
      // takes (Im U_cj, Re U_cj) = w with its halves swapped
      const uint32_t w0 = Ls[d0 * 9 + bc * 3 + j0], w1 = Ls[d1 * 9 + bc * 3 + j1];
      const uint32_t b0 = gq >= 6 ? 0u : bim ? __byte_perm(w0, 0u, 0x1032) : (w0 ^ 0x80000000u);
      const uint32_t b1 = gq >= 6 ? 0u : bim ? __byte_perm(w1, 0u, 0x1032) : (w1 ^ 0x80000000u);
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        const long long e0 = ((long long)nb0 * 3 + j0) * N + 16 * m + gq;
        const long long e1 = ((long long)nb1 * 3 + j1) * N + 16 * m + gq;
        const uint32_t a[4] = {__ldg(in + e0), __ldg(in + e0 + 8), __ldg(in + e1),
                               __ldg(in + e1 + 8)};
        Tc16Mma<S>::mma(acc[m], a, b0, b1);
      }
    }
    if (tig < 3) {
#pragma unroll
      for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long oi = ((long long)site * 3 + tig) * N + 16 * m + gq + 8 * h;
          float re = acc[m][2 * h] * unraw, im = acc[m][2 * h + 1] * unraw;
          if (EPI != EPI_NONE) {
            const cpx<float> cc = S::load(c1 + oi);
            re = fmaf(m2, cc.re, -re);
            im = fmaf(m2, cc.im, -im);
            if (EPI == EPI_RESIDUAL) {
              const cpx<float> bb = S::load(c2 + oi);
              re = bb.re - re;
              im = bb.im - im;
            }
          }
          S::store(out + oi, cpx<float>{re, im});
        }
    }
  }
}

template <class S, int EPI, int MT>
static cudaError_t launch_tc16(const void* links, const void* in, void* out, const void* c1,
                               const void* c2, double m2, const Geom& g, int parity, Gate gate,
                               cudaStream_t s) {
  using E = typename S::elem;
  auto kern = k_dslash_tc16<S, EPI, MT>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T16_SITES * 32, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long ngroups = ((long long)g.Vh + T16_SITES - 1) / T16_SITES;
  const long long want = (long long)stencil_sms() * per_sm;
  const unsigned blocks = (unsigned)(ngroups < want ? ngroups : want);
  kern<<<blocks, T16_SITES * 32, 0, s>>>((const uint32_t*)links, (const uint32_t*)in, (E*)out,
                                         (const E*)c1, (const E*)c2, m2, g, parity, gate);
  return cudaGetLastError();
}

template <class S, int MT>
static cudaError_t launch_tc16_epi(int epi, const void* L, const void* I, void* O, const void* A,
                                   const void* B, double m2, const Geom& g, int p, Gate gate,
                                   cudaStream_t s) {
  switch (epi) {
    case EPI_NONE: return launch_tc16<S, EPI_NONE, MT>(L, I, O, A, B, m2, g, p, gate, s);
    case EPI_NORMAL: return launch_tc16<S, EPI_NORMAL, MT>(L, I, O, A, B, m2, g, p, gate, s);
    default: return launch_tc16<S, EPI_RESIDUAL, MT>(L, I, O, A, B, m2, g, p, gate, s);
  }
}

bool dslash_tc16_supported(int N) { return N == 16 || N == 32; }

cudaError_t dslash_tc16(FieldKind k, int epi, const void* links, const void* in, void* out,
                        const void* c1, const void* c2, double m2, const Geom& g, int out_parity,
                        int N, Gate gate, cudaStream_t s) {
  if (!dslash_tc16_supported(N) || (k != FK_H16 && k != FK_BF16)) return cudaErrorInvalidValue;
  const int p = out_parity;
  if (k == FK_H16)
    return N == 16 ? launch_tc16_epi<StoreH16, 1>(epi, links, in, out, c1, c2, m2, g, p, gate, s)
                   : launch_tc16_epi<StoreH16, 2>(epi, links, in, out, c1, c2, m2, g, p, gate, s);
  return N == 16 ? launch_tc16_epi<StoreBF16, 1>(epi, links, in, out, c1, c2, m2, g, p, gate, s)
                 : launch_tc16_epi<StoreBF16, 2>(epi, links, in, out, c1, c2, m2, g, p, gate, s);
}

}  // namespace bcg
