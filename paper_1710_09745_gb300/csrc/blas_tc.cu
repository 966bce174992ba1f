// Tensor-core form of the fused blockCGrQ update (Algorithm 1: Q = W S^-1,
// X += P (beta C), P = Q + P S^dag) for the 16-bit storage kinds, where the
// streaming multi-BLAS of Sec. 6.3 is a dense contraction once N >= 16:
// every row (site, colour) of W and P is multiplied by three N x N complex
// coefficient matrices.  On the FP32 pipes that costs 8 N^2 multiply-adds
// per row, read from shared memory; here each warp runs them as
// mma.sync m16n8k16 products with FP32 accumulation.
//
// Real form.  A complex row a (N entries, stored re/im-interleaved) times a
// complex N x N matrix M is the real row [re_0, im_0, re_1, ...] (2N) times
// the 2N x 2N real matrix M' with
//   M'[2i][2j] = Re M_ij,  M'[2i+1][2j] = -Im M_ij,
//   M'[2i][2j+1] = Im M_ij, M'[2i+1][2j+1] = Re M_ij,
// so the stored 16-bit rows are the MMA's A operand as they are (one 32-bit
// (re, im) pair per A register) and M' is the B operand.
//
// Exactness.  The stored W and P are 16-bit numbers, exact MMA inputs.  Each
// coefficient column j is scaled by a power of two s_j (its largest entry
// lands near 2^13, inside FP16's range) and split into NSL 16-bit slices
// (FP16: 2 slices, 22 significant bits; BF16: 3 slices, 24 bits); the slices
// are multiplied with the same A fragments and accumulated in FP32, and s_j is
// removed exactly in the epilogue.  The coefficient error is thus below
// 2^-22 of the column's largest entry, at or below the FP32 rounding of the
// FP32-pipe kernel, far below the 16-bit storage rounding of the results.
//
// Work split.  A warp owns 16 consecutive rows (a 16 x 2N A tile) and loops
// over output column tiles of 4 complex columns (an 8-wide MMA n tile): for
// each it forms Q (S^-1 is upper triangular: k blocks wholly below the
// diagonal are skipped), then P = Q + P S^dag (lower triangular) seeded with
// Q in the accumulator, then the increment P (beta C), which is added to
// the double-float X.  The k order inside each 16-column k block is permuted
// (consistently in A and B; a sum does not depend on its order) so that a
// thread's A registers for two k steps are 4 consecutive complex numbers of
// its row: one 128-bit load.  B fragments of all three matrices are built
// once per CTA in shared memory in fragment order (one 64-bit load per MMA,
// conflict-free).
#include <type_traits>

#include "internal.h"
#include "ozaki.cuh"

namespace bcg {

namespace {

template <class SS>
struct TcKind;
template <>
struct TcKind<StoreH16> {
  static constexpr int NSL = 2;
  static __device__ __forceinline__ uint32_t pack(double a, double b, double* ra, double* rb) {
    __half ha = __double2half(a), hb = __double2half(b);
    *ra = a - (double)__half2float(ha);
    *rb = b - (double)__half2float(hb);
    __half2 h = __halves2half2(ha, hb);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ uint32_t out(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 in(uint32_t u) {
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
  }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
  }
};
template <>
struct TcKind<StoreBF16> {
  static constexpr int NSL = 3;
  static __device__ __forceinline__ uint32_t pack(double a, double b, double* ra, double* rb) {
    __nv_bfloat16 ha = __double2bfloat16(a), hb = __double2bfloat16(b);
    *ra = a - (double)__bfloat162float(ha);
    *rb = b - (double)__bfloat162float(hb);
    __nv_bfloat162 h = __halves2bfloat162(ha, hb);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ uint32_t out(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 in(uint32_t u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
  }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
  }
};

constexpr int TC_WARPS = 8;  // warps per CTA

// coefficient entry (i, j) of matrix m in its triangular pattern: 0 = S^-1
// (upper), 1 = beta C (full), 2 = S^dag (lower)
__device__ __forceinline__ bool tc_in_pattern(int m, int i, int j) {
  return m == 1 || (m == 0 ? i <= j : i >= j);
}

}  // namespace

// Shared memory: B fragments [3][NSL][KS][NT][32] uint2, then the inverse
// column scales [3][N] float.  KS = N / 8 k steps of 16 reals, NT = N / 4
// n tiles of 8 reals.
template <class SS, int N>
__global__ void __launch_bounds__(TC_WARPS * 32, N >= 32 ? 3 : 4)
    k_bcg_update_tc(typename SS::elem* __restrict__ Q, typename SS::elem* __restrict__ P,
                    StoreDF::elem* __restrict__ X, const double2* __restrict__ Sinv,
                    const double2* __restrict__ BC, const double2* __restrict__ SH, int Vh,
                    Gate gate) {
  using K = TcKind<SS>;
  constexpr int NSL = K::NSL;
  constexpr int KS = N / 8, NT = N / 4, MB = N / 16;
  constexpr int FR = KS * NT * 32;  // fragments per slice of one matrix
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint2* sB = reinterpret_cast<uint2*>(smem_raw);
  float* sInv = reinterpret_cast<float*>(sB + 3 * NSL * FR);
  __shared__ double sScale[3 * N];
  if (gate_closed(gate)) return;
  const bool keepP = gate.st != nullptr && ((const volatile SolverStatus*)gate.st)->ru_pending;
  auto Ms = [&](int m) { return m == 0 ? Sinv : m == 1 ? BC : SH; };

  // column scales: a power of two that takes the column's largest entry to
  // [2^12, 2^13) (1 for an all-zero column)
  for (int c = threadIdx.x; c < 3 * N; c += blockDim.x) {
    const int m = c / N, j = c - m * N;
    double mx = 0.0;
    for (int i = 0; i < N; ++i) {
      if (!tc_in_pattern(m, i, j)) continue;
      const double2 v = Ms(m)[i * N + j];
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx in [2^(e-1), 2^e)
    const int sh = mx > 0.0 ? 13 - e : 0;
    sScale[c] = ldexp(1.0, sh);
    sInv[c] = (float)ldexp(1.0, -sh);
  }
  __syncthreads();
  // B fragments.  For k step ks (k block mb = ks / 2, half hh = ks % 2) and
  // lane (g = lane / 4, t = lane % 4): register b0 holds rows (re, im) of
  // input i0 = 16 mb + 4 t + 2 hh, b1 those of i0 + 1; the column is
  // n = 8 nt + g, i.e. complex column j = n / 2, real part when n is even.
  for (int idx = threadIdx.x; idx < 3 * FR; idx += blockDim.x) {
    const int m = idx / FR;
    int r = idx - m * FR;
    const int ks = r / (NT * 32);
    r -= ks * NT * 32;
    const int nt = r / 32, lane = r - nt * 32;
    const int g = lane >> 2, t = lane & 3;
    const int i0 = 16 * (ks >> 1) + 4 * t + 2 * (ks & 1);
    const int n = 8 * nt + g, j = n >> 1, part = n & 1;
    const double sc = sScale[m * N + j];
    double e[2][2];  // [input i0 / i0 + 1][re row, im row]
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + q;
      double re = 0.0, im = 0.0;
      if (tc_in_pattern(m, i, j)) {
        const double2 v = Ms(m)[i * N + j];
        re = v.x * sc;
        im = v.y * sc;
      }
      e[q][0] = part ? im : re;
      e[q][1] = part ? re : -im;
    }
    for (int sl = 0; sl < NSL; ++sl) {
      uint2 b;
      b.x = K::pack(e[0][0], e[0][1], &e[0][0], &e[0][1]);
      b.y = K::pack(e[1][0], e[1][1], &e[1][0], &e[1][1]);
      sB[((m * NSL + sl) * KS + ks) * NT * 32 + nt * 32 + lane] = b;
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long nrows = 3LL * Vh;
  const long long ntiles = (nrows + 15) / 16;
  constexpr float unraw = 1.f / SS::RAW_SCALE;
  const uint32_t* Qw = reinterpret_cast<const uint32_t*>(Q);
  const uint32_t* Pw = reinterpret_cast<const uint32_t*>(P);
  for (long long tile = (long long)blockIdx.x * TC_WARPS + (threadIdx.x >> 5); tile < ntiles;
       tile += (long long)gridDim.x * TC_WARPS) {
    const long long ra = tile * 16 + g, rb = ra + 8;
    const bool va = ra < nrows, vb = rb < nrows;
    // A fragments of W (held in the Q buffer) and P: per k block, the four
    // complex numbers 16 mb + 4t .. + 3 of rows ra and rb
    uint4 wa[MB], wb[MB], pa[MB], pb[MB];
#pragma unroll
    for (int mb = 0; mb < MB; ++mb) {
      const int c0 = 16 * mb + 4 * t;
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      wa[mb] = va ? *reinterpret_cast<const uint4*>(Qw + ra * N + c0) : z;
      wb[mb] = vb ? *reinterpret_cast<const uint4*>(Qw + rb * N + c0) : z;
      pa[mb] = va ? *reinterpret_cast<const uint4*>(Pw + ra * N + c0) : z;
      pb[mb] = vb ? *reinterpret_cast<const uint4*>(Pw + rb * N + c0) : z;
    }
    auto afrag = [&](const uint4* xa, const uint4* xb, int ks, uint32_t (&a)[4]) {
      const uint4 ua = xa[ks >> 1], ub = xb[ks >> 1];
      const bool hi = ks & 1;
      a[0] = hi ? ua.z : ua.x;
      a[1] = hi ? ub.z : ub.x;
      a[2] = hi ? ua.w : ua.y;
      a[3] = hi ? ub.w : ub.y;
    };
#pragma unroll 1
    for (int nt = 0; nt < NT; ++nt) {
      const int j = 4 * nt + t;  // this thread's complex output column
      float q[4] = {0.f, 0.f, 0.f, 0.f};
      // Q = W S^-1: k blocks with an entry i <= the tile's last column
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        if (16 * (ks >> 1) > 4 * nt + 3) continue;
        uint32_t a[4];
        afrag(wa, wb, ks, a);
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl) K::mma(q, a, sB[((0 * NSL + sl) * KS + ks) * NT * 32 + nt * 32 + lane]);
      }
      const float i0s = sInv[j];
#pragma unroll
      for (int e = 0; e < 4; ++e) q[e] *= i0s;  // Q in the stored (raw) scale
      const long long oa = ra * N + j, ob = rb * N + j;
      uint32_t* Qo = reinterpret_cast<uint32_t*>(Q);
      if (va) Qo[oa] = K::out(q[0], q[1]);
      if (vb) Qo[ob] = K::out(q[2], q[3]);
      if (!keepP) {
        // P = Q + P S^dag, with Q seeding the accumulator in S^dag's scale
        const float s2 = (float)sScale[2 * N + j];
        float p[4] = {q[0] * s2, q[1] * s2, q[2] * s2, q[3] * s2};
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          if (16 * (ks >> 1) + 15 < 4 * nt) continue;
          uint32_t a[4];
          afrag(pa, pb, ks, a);
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl) K::mma(p, a, sB[((2 * NSL + sl) * KS + ks) * NT * 32 + nt * 32 + lane]);
        }
        const float i2s = sInv[2 * N + j];
        uint32_t* Po = reinterpret_cast<uint32_t*>(P);
        if (va) Po[oa] = K::out(p[0] * i2s, p[1] * i2s);
        if (vb) Po[ob] = K::out(p[2] * i2s, p[3] * i2s);
      }
      // X += P (beta C), the increment from the old P (still in registers)
      float x[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        uint32_t a[4];
        afrag(pa, pb, ks, a);
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl) K::mma(x, a, sB[((1 * NSL + sl) * KS + ks) * NT * 32 + nt * 32 + lane]);
      }
      const float i1s = sInv[N + j] * unraw;
#pragma unroll
      for (int hrow = 0; hrow < 2; ++hrow) {
        if (!(hrow ? vb : va)) continue;
        StoreDF::elem* xp = X + (hrow ? ob : oa);
        cpx<dfacc> xa = cacc_from<CompDF>(StoreDF::load_nc(xp));
        CompDF::add(xa.re, df{x[2 * hrow] * i1s, 0.f});
        CompDF::add(xa.im, df{x[2 * hrow + 1] * i1s, 0.f});
        StoreDF::store(xp, cfin<CompDF>(xa));
      }
    }
  }
}

template <class SS, int N>
static cudaError_t launch_bcg_update_tc(void* Q, void* P, void* X, const double2* Sinv,
                                        const double2* BC, const double2* SH, int Vh, Gate gate,
                                        cudaStream_t s) {
  constexpr int NSL = TcKind<SS>::NSL;
  const size_t sm = (size_t)3 * NSL * (N / 8) * (N / 4) * 32 * sizeof(uint2) + 3 * N * sizeof(float);
  auto kern = k_bcg_update_tc<SS, N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_WARPS * 32, sm) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    cudaGetLastError();
  if (gate_mostly_off(gate) && per_sm > 2) per_sm = 2;
  const long long tiles = (3LL * Vh + 15) / 16;
  long long blocks = (tiles + TC_WARPS - 1) / TC_WARPS;
  if (blocks > (long long)sms * per_sm) blocks = (long long)sms * per_sm;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, TC_WARPS * 32, sm, s>>>((typename SS::elem*)Q, (typename SS::elem*)P,
                                                  (StoreDF::elem*)X, Sinv, BC, SH, Vh, gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// W = Q - AP beta and the Gram W^dag W of the thin QR (Algorithm 2) in one
// pass, on the tensor cores, for the 16-bit kinds.  A CTA tile is
// TC_WARPS x 16 rows.  Phase 1: each warp forms W for its 16 rows as the
// update kernel forms Q (A = AP, B = -beta split and column-scaled, the
// accumulator seeded with Q), stores W (in place of Q, rounded to the storage
// format) and copies the rounded rows into a padded shared-memory tile.
// Phase 2: the real Gram G = W_r^T W_r of the tile's real rows (2N columns)
// is taken with the rows as the MMA's k dimension: ldmatrix.trans turns the
// row-major tile into the transposed A and B fragments.  The complex Gram is
//   K_ij = G[2i][2j] + G[2i+1][2j+1] + i (G[2i][2j+1] - G[2i+1][2j]),
// Hermitian, so only 16 x 8 blocks of G that hold an entry i <= j are
// formed, spread over the CTA's warps.  Each block's sum over a tile (128
// rows) is exact up to FP32 rounding of its 128 products (16-bit inputs),
// then added to a double-float accumulator; the CTA writes its upper-triangle
// partial sums, which the fixed-order FP64 reduction of the FP32-pipe path
// combines.  The Gram is that of the stored (rounded) W, the block whose
// columns Q = W S^-1 orthonormalises.
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}

// Gram blocks (mt, nt) of G: rows 16 mt .. + 15 (complex i = 8 mt .. + 7),
// columns 8 nt .. + 7 (complex j = 4 nt .. + 3); HERM: only blocks holding an
// entry i <= j
template <int N, bool HERM>
struct GramBlocks {
  static constexpr int MT = N / 8, NT = N / 4;
  static constexpr __host__ __device__ bool used(int mt, int nt) {
    return !HERM || 8 * mt <= 4 * nt + 3;
  }
  static constexpr int count() {
    int c = 0;
    for (int mt = 0; mt < MT; ++mt)
      for (int nt = 0; nt < NT; ++nt)
        if (used(mt, nt)) ++c;
    return c;
  }
  static constexpr int COUNT = count();
  static constexpr int PER_WARP = (COUNT + TC_WARPS - 1) / TC_WARPS;
  // the b-th block in row-major order
  static __device__ __forceinline__ void at(int b, int& mt, int& nt) {
    int c = 0;
    for (int m = 0; m < MT; ++m)
      for (int n = 0; n < NT; ++n)
        if (used(m, n)) {
          if (c == b) {
            mt = m;
            nt = n;
            return;
          }
          ++c;
        }
    mt = nt = 0;
  }
};

// One CTA tile's contribution to this warp's Gram blocks: G += X_r^T Y_r
// over the TR rows of the shared tiles sX and sY (row stride RW words);
// X_r^T and Y_r fragments by ldmatrix.trans.  FP32 sums of 16 x TR products,
// added to the double-float accumulators.
template <class K, int N, bool HERM, int TR, int RW>
__device__ __forceinline__ void gram_tc_tile(const uint32_t* sX, const uint32_t* sY,
                                             dfacc (&gacc)[GramBlocks<N, HERM>::PER_WARP][4],
                                             int warp, int lane) {
  using GB = GramBlocks<N, HERM>;
#pragma unroll
  for (int bb = 0; bb < GB::PER_WARP; ++bb) {
    const int b = warp + bb * TC_WARPS;
    if (b >= GB::COUNT) break;
    int mt, nt;
    GB::at(b, mt, nt);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int q = lane >> 3, rr = lane & 7;
#pragma unroll 2
    for (int ks = 0; ks < TR / 16; ++ks) {
      // A = X^T: ldmatrix.x4 matrices (tile rows +0/+8) x (tile columns
      // +0/+8 halves) in the order (m +0, k +0), (m +8, k +0), (m +0, k +8),
      // (m +8, k +8) of the A fragment (m = G row = tile column, k = tile row)
      const int arow = 16 * ks + (q >> 1) * 8 + rr;
      const int acol = 8 * mt + (q & 1) * 4;  // 32-bit words: 16 mt halves
      uint32_t a[4];
      ldsm_x4_t(a, sX + arow * RW + acol);
      // B = Y (k = tile rows 16 ks .. + 15, n = tile columns 8 nt .. + 7)
      const int brow = 16 * ks + (q & 1) * 8 + rr;
      uint32_t bf[2];
      ldsm_x2_t(bf, sY + brow * RW + 4 * nt);
      K::mma(d, a, make_uint2(bf[0], bf[1]));
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) CompDF::add(gacc[bb][e], df{d[e], 0.f});
  }
}

// The CTA's partial sums of K = X^dag Y (HERM: the entries i <= j) from the
// warps' blocks of G: the lane pair (g even, g + 1) holds G rows (2i, 2i + 1)
template <int N, bool HERM>
__device__ __forceinline__ void gram_tc_write(double2* out,
                                              const dfacc (&gacc)[GramBlocks<N, HERM>::PER_WARP][4],
                                              double scale, int warp, int lane) {
  using GB = GramBlocks<N, HERM>;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int bb = 0; bb < GB::PER_WARP; ++bb) {
    const int b = warp + bb * TC_WARPS;
    if (b >= GB::COUNT) break;  // uniform per warp
    int mt, nt;
    GB::at(b, mt, nt);
    double v[4], p[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (double)gacc[bb][e].s + (double)gacc[bb][e].e;
#pragma unroll
    for (int e = 0; e < 4; ++e) p[e] = __shfl_xor_sync(0xffffffffu, v[e], 4);
    if ((g & 1) == 0) {
      const int j = 4 * nt + t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 8 * mt + (g >> 1) + 4 * h;
        if (!HERM || i <= j) {
          const double kre = v[2 * h] + p[2 * h + 1];
          const double kim = v[2 * h + 1] - p[2 * h];
          out[i * N + j] = make_double2(kre * scale, kim * scale);
        }
      }
    }
  }
}

template <class SS, int N>
__global__ void __launch_bounds__(TC_WARPS * 32, N >= 32 ? 3 : 4)
    k_w_gram_tc(typename SS::elem* __restrict__ Q, const typename SS::elem* __restrict__ AP,
                const double2* __restrict__ beta, int Vh, double2* __restrict__ partials,
                Gate gate) {
  using K = TcKind<SS>;
  using GB = GramBlocks<N, true>;
  constexpr int NSL = K::NSL;
  constexpr int KS = N / 8, NT = N / 4, MB = N / 16;
  constexpr int FR = KS * NT * 32;
  constexpr int TR = TC_WARPS * 16;  // rows per CTA tile
  constexpr int RW = N + 4;          // shared tile row stride in 32-bit words (16 B pad)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint2* sB = reinterpret_cast<uint2*>(smem_raw);
  float* sInv = reinterpret_cast<float*>(sB + NSL * FR);
  uint32_t* sW = reinterpret_cast<uint32_t*>(sInv + N);  // [TR][RW] (re, im) pairs
  __shared__ double sScale[N];
  if (gate_closed(gate)) return;

  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double mx = 0.0;
    for (int i = 0; i < N; ++i) {
      const double2 v = beta[i * N + j];
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    const int sh = mx > 0.0 ? 13 - e : 0;
    sScale[j] = ldexp(1.0, sh);
    sInv[j] = (float)ldexp(1.0, -sh);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < FR; idx += blockDim.x) {
    const int ks = idx / (NT * 32);
    const int r = idx - ks * NT * 32;
    const int nt = r / 32, lane = r - nt * 32;
    const int g = lane >> 2, t = lane & 3;
    const int i0 = 16 * (ks >> 1) + 4 * t + 2 * (ks & 1);
    const int n = 8 * nt + g, j = n >> 1, part = n & 1;
    const double sc = -sScale[j];  // B = -beta
    double e[2][2];
    for (int q = 0; q < 2; ++q) {
      const double2 v = beta[(i0 + q) * N + j];
      const double re = v.x * sc, im = v.y * sc;
      e[q][0] = part ? im : re;
      e[q][1] = part ? re : -im;
    }
    for (int sl = 0; sl < NSL; ++sl) {
      uint2 b;
      b.x = K::pack(e[0][0], e[0][1], &e[0][0], &e[0][1]);
      b.y = K::pack(e[1][0], e[1][1], &e[1][0], &e[1][1]);
      sB[(sl * KS + ks) * NT * 32 + nt * 32 + lane] = b;
    }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long nrows = 3LL * Vh;
  constexpr float unraw = 1.f / SS::RAW_SCALE;
  const uint32_t* APw = reinterpret_cast<const uint32_t*>(AP);
  uint32_t* Qw = reinterpret_cast<uint32_t*>(Q);
  dfacc gacc[GB::PER_WARP][4];
#pragma unroll
  for (int b = 0; b < GB::PER_WARP; ++b)
#pragma unroll
    for (int e = 0; e < 4; ++e) gacc[b][e] = CompDF::zero();

  for (long long tile = blockIdx.x; tile * TR < nrows; tile += gridDim.x) {
    // phase 1: W for rows tile * TR + 16 warp + (g, g + 8)
    const int la = 16 * warp + g, lb = la + 8;  // rows in the shared tile
    const long long ra = tile * TR + la, rb = tile * TR + lb;
    const bool va = ra < nrows, vb = rb < nrows;
    uint4 apa[MB], apb[MB];
#pragma unroll
    for (int mb = 0; mb < MB; ++mb) {
      const int c0 = 16 * mb + 4 * t;
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      apa[mb] = va ? *reinterpret_cast<const uint4*>(APw + ra * N + c0) : z;
      apb[mb] = vb ? *reinterpret_cast<const uint4*>(APw + rb * N + c0) : z;
    }
#pragma unroll 1
    for (int nt = 0; nt < NT; ++nt) {
      const int j = 4 * nt + t;
      const float sj = (float)sScale[j];
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      if (va) {
        const float2 qa = TcKind<SS>::in(Qw[ra * N + j]);
        acc[0] = qa.x * sj;
        acc[1] = qa.y * sj;
      }
      if (vb) {
        const float2 qb = TcKind<SS>::in(Qw[rb * N + j]);
        acc[2] = qb.x * sj;
        acc[3] = qb.y * sj;
      }
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const uint4 ua = apa[ks >> 1], ub = apb[ks >> 1];
        const bool hi = ks & 1;
        const uint32_t a[4] = {hi ? ua.z : ua.x, hi ? ub.z : ub.x, hi ? ua.w : ua.y,
                               hi ? ub.w : ub.y};
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl) K::mma(acc, a, sB[(sl * KS + ks) * NT * 32 + nt * 32 + lane]);
      }
      const float ij = sInv[j];
      const uint32_t wa = va ? K::out(acc[0] * ij, acc[1] * ij) : 0u;
      const uint32_t wb = vb ? K::out(acc[2] * ij, acc[3] * ij) : 0u;
      if (va) Qw[ra * N + j] = wa;
      if (vb) Qw[rb * N + j] = wb;
      sW[la * RW + j] = wa;  // rows past the end hold zeros
      sW[lb * RW + j] = wb;
    }
    __syncthreads();
    // phase 2: this warp's Gram blocks over the tile's TR rows
    gram_tc_tile<K, N, true, TR, RW>(sW, sW, gacc, warp, lane);
    __syncthreads();
  }

  gram_tc_write<N, true>(partials + (long long)blockIdx.x * N * N, gacc,
                        (double)unraw * (double)unraw, warp, lane);
}

template <class SS, int N>
static cudaError_t launch_w_gram_tc(void* Q, const void* AP, const double2* beta, int Vh,
                                    double2* partials, int nblocks, Gate gate, cudaStream_t s) {
  constexpr int NSL = TcKind<SS>::NSL;
  const size_t sm = (size_t)NSL * (N / 8) * (N / 4) * 32 * sizeof(uint2) + N * sizeof(float) +
                    (size_t)TC_WARPS * 16 * (N + 4) * sizeof(uint32_t);
  auto kern = k_w_gram_tc<SS, N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, TC_WARPS * 32, sm, s>>>((typename SS::elem*)Q, (const typename SS::elem*)AP,
                                          beta, Vh, partials, gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K = X^dag Y (the reduction multi-BLAS of Sec. 6.4; P^dag AP in Algorithm 1)
// on the tensor cores for the 16-bit kinds: each CTA tile of TR rows of X and
// Y is copied into padded shared-memory tiles with 128-bit loads, then the
// warps form their blocks of the real Gram as in the fused W + Gram kernel.
// HERM: only the entries i <= j (a Hermitian Gram; the reduction mirrors);
// the iteration's P^dag AP is the one user, so only HERM is instantiated.
template <class SS, int N, bool HERM>
__global__ void __launch_bounds__(TC_WARPS * 32, 4)
    k_gram_tc(const typename SS::elem* __restrict__ X, const typename SS::elem* __restrict__ Y,
              int Vh, double2* __restrict__ partials, Gate gate) {
  using K = TcKind<SS>;
  using GB = GramBlocks<N, HERM>;
  constexpr int TR = TC_WARPS * 16;
  constexpr int RW = N + 4;
  constexpr int CH = N / 4;  // 16-byte chunks per row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* sX = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* sY = sX + TR * RW;
  if (gate_closed(gate)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nrows = 3LL * Vh;
  const uint32_t* Xw = reinterpret_cast<const uint32_t*>(X);
  const uint32_t* Yw = reinterpret_cast<const uint32_t*>(Y);
  dfacc gacc[GB::PER_WARP][4];
#pragma unroll
  for (int b = 0; b < GB::PER_WARP; ++b)
#pragma unroll
    for (int e = 0; e < 4; ++e) gacc[b][e] = CompDF::zero();
  for (long long tile = blockIdx.x; tile * TR < nrows; tile += gridDim.x) {
    for (int idx = threadIdx.x; idx < TR * CH; idx += blockDim.x) {
      const int row = idx / CH, c = idx - row * CH;
      const long long r = tile * TR + row;
      uint4 x = make_uint4(0u, 0u, 0u, 0u), y = x;  // rows past the end: zeros
      if (r < nrows) {
        x = *reinterpret_cast<const uint4*>(Xw + r * N + 4 * c);
        y = *reinterpret_cast<const uint4*>(Yw + r * N + 4 * c);
      }
      *reinterpret_cast<uint4*>(sX + row * RW + 4 * c) = x;
      *reinterpret_cast<uint4*>(sY + row * RW + 4 * c) = y;
    }
    __syncthreads();
    gram_tc_tile<K, N, HERM, TR, RW>(sX, sY, gacc, warp, lane);
    __syncthreads();
  }
  constexpr double unraw = 1.0 / SS::RAW_SCALE;
  gram_tc_write<N, HERM>(partials + (long long)blockIdx.x * N * N, gacc, unraw * unraw, warp, lane);
}

template <class SS, int N>
static cudaError_t launch_gram_tc(const void* X, const void* Y, int Vh, double2* partials,
                                  int nblocks, Gate gate, cudaStream_t s) {
  const size_t sm = 2 * (size_t)TC_WARPS * 16 * (N + 4) * sizeof(uint32_t);
  using E = typename SS::elem;
  auto kern = k_gram_tc<SS, N, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, TC_WARPS * 32, sm, s>>>((const E*)X, (const E*)Y, Vh, partials, gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K = X^dag Y for the double-float kind (N = 16) on the tensor cores, as exact
// split products (ozaki.cuh): per CTA tile of TGD = 64 rows, every column of X
// and of Y gets a power-of-two scale from its largest entry in the tile
// (shared-memory maxima), each scaled value is split into six bf16 slices,
// and slice s of a tile is stored like the 16-bit tiles above ([row][RW]
// words of (re, im) pairs).  A warp's Gram block accumulates the products of
// slices s, t with s + t = u in D_u: over the tile's 64 rows the terms share
// the grid 2^(ei + ej - 14 - 8u) and stay below 2^24 units (at most
// 64 x 7 x 2^14), so the FP32 sums are exact; after the tile D_0 .. D_5 are
// added in double-float, the scales removed and the result added to the
// warp's double-float accumulators.  Hermitian: only blocks holding an entry
// i <= j; X == Y (a Gram of one block) stages one set of slices.
constexpr int TGD = 64;  // rows per CTA tile

template <int N, bool SAME>
__global__ void __launch_bounds__(TC_WARPS * 32, N == 16 ? (SAME ? 3 : 2) : 1)
    k_gram_tc_df(const float4* __restrict__ X, const float4* __restrict__ Y, int Vh,
                 double2* __restrict__ partials, Gate gate) {
  using GB = GramBlocks<N, true>;
  constexpr int RW = N + 4;
  constexpr int NSL = 6;
  constexpr int PER = TGD * N / (TC_WARPS * 32);  // entries of a tile per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* sX = reinterpret_cast<uint32_t*>(smem_raw);  // [NSL][TGD][RW]
  uint32_t* sY = SAME ? sX : sX + NSL * TGD * RW;
  __shared__ unsigned sMx[N], sMy[N];
  __shared__ int sEx[N], sEy[N];
  if (gate_closed(gate)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nrows = 3LL * Vh;
  dfacc gacc[GB::PER_WARP][4];
#pragma unroll
  for (int b = 0; b < GB::PER_WARP; ++b)
#pragma unroll
    for (int e = 0; e < 4; ++e) gacc[b][e] = CompDF::zero();
  for (long long tile = blockIdx.x; tile * TGD < nrows; tile += gridDim.x) {
    if (threadIdx.x < N) sMx[threadIdx.x] = sMy[threadIdx.x] = 0u;
    __syncthreads();  // also: the previous tile's slices have been read
    float4 xv[PER], yv[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * TC_WARPS * 32;  // column idx % N (N divides 256)
      const long long r = tile * TGD + idx / N;
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      xv[k] = r < nrows ? X[r * N + idx % N] : z;
      yv[k] = SAME ? xv[k] : (r < nrows ? Y[r * N + idx % N] : z);
    }
    {
      float mx = 0.f, my = 0.f;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        mx = fmaxf(mx, fmaxf(fabsf(xv[k].x), fabsf(xv[k].y)));
        my = fmaxf(my, fmaxf(fabsf(yv[k].x), fabsf(yv[k].y)));
      }
      atomicMax(&sMx[threadIdx.x % N], __float_as_uint(mx));
      if (!SAME) atomicMax(&sMy[threadIdx.x % N], __float_as_uint(my));
    }
    __syncthreads();
    if (threadIdx.x < N) {
      sEx[threadIdx.x] = ozaki::pow2_above(sMx[threadIdx.x]);
      sEy[threadIdx.x] = SAME ? sEx[threadIdx.x] : ozaki::pow2_above(sMy[threadIdx.x]);
    }
    __syncthreads();
    {
      const int c = threadIdx.x % N;
      const float scx = ozaki::exp2i(-sEx[c]), scy = ozaki::exp2i(-sEy[c]);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int row = (threadIdx.x + k * TC_WARPS * 32) / N;
        float sr[NSL], si[NSL];
        ozaki::split6(__fmul_rn(xv[k].x, scx), __fmul_rn(xv[k].z, scx), sr);
        ozaki::split6(__fmul_rn(xv[k].y, scx), __fmul_rn(xv[k].w, scx), si);
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl)
          sX[(sl * TGD + row) * RW + c] = ozaki::pack_bf16(sr[sl], si[sl]);
        if (!SAME) {
          ozaki::split6(__fmul_rn(yv[k].x, scy), __fmul_rn(yv[k].z, scy), sr);
          ozaki::split6(__fmul_rn(yv[k].y, scy), __fmul_rn(yv[k].w, scy), si);
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl)
            sY[(sl * TGD + row) * RW + c] = ozaki::pack_bf16(sr[sl], si[sl]);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < GB::PER_WARP; ++bb) {
      const int b = warp + bb * TC_WARPS;
      if (b >= GB::COUNT) break;  // uniform per warp
      int mt, nt;
      GB::at(b, mt, nt);
      float d[6][4];
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[u][e] = 0.f;
      const int q = lane >> 3, rr = lane & 7;
#pragma unroll 1
      for (int ks = 0; ks < TGD / 16; ++ks) {
        // A = X^T, B = Y fragments of every slice (as in gram_tc_tile)
        const int arow = 16 * ks + (q >> 1) * 8 + rr;
        const int acol = 8 * mt + (q & 1) * 4;
        const int brow = 16 * ks + (q & 1) * 8 + rr;
        uint32_t a[NSL][4];
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl) ldsm_x4_t(a[sl], sX + (sl * TGD + arow) * RW + acol);
#pragma unroll
        for (int tt = 0; tt < NSL; ++tt) {
          uint32_t bf[2];
          ldsm_x2_t(bf, sY + (tt * TGD + brow) * RW + 4 * nt);
#pragma unroll
          for (int sl = 0; sl + tt < NSL; ++sl) ozaki::mma_bf16(d[sl + tt], a[sl], bf[0], bf[1]);
        }
      }
      // element e of the block: G row 16 mt + g (+ 8 for e >= 2), column
      // 8 nt + 2 t (+ 1 for odd e); complex indices are half of those
      const int g = lane >> 2, t = lane & 3;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = (16 * mt + g + 8 * (e >> 1)) >> 1, j = (8 * nt + 2 * t + (e & 1)) >> 1;
        const dfacc v = ozaki::combine6(d[0][e], d[1][e], d[2][e], d[3][e], d[4][e], d[5][e]);
        const float fa = ozaki::exp2i(sEx[i]), fb = ozaki::exp2i(sEy[j]);
        const df w = CompDF::fin(dfacc{__fmul_rn(__fmul_rn(v.s, fa), fb),
                                       __fmul_rn(__fmul_rn(v.e, fa), fb)});
        CompDF::add(gacc[bb][e], w);
      }
    }
  }
  gram_tc_write<N, true>(partials + (long long)blockIdx.x * N * N, gacc, 1.0, warp, lane);
}

template <int N, bool SAME>
static cudaError_t launch_gram_tc_df(const void* X, const void* Y, int Vh, double2* partials,
                                     int nblocks, Gate gate, cudaStream_t s) {
  const size_t sm = (SAME ? 1 : 2) * (size_t)6 * TGD * (N + 4) * sizeof(uint32_t);
  auto kern = k_gram_tc_df<N, SAME>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, TC_WARPS * 32, sm, s>>>((const float4*)X, (const float4*)Y, Vh, partials, gate);
  return cudaGetLastError();
}

// Hermitian Grams only (P^dag AP of the iteration)
cudaError_t gram_partials_tc(FieldKind k, const void* X, const void* Y, int N, int Vh,
                             double2* partials, int nblocks, Gate gate, cudaStream_t s) {
  if (k == FK_DF && N == 16)
    return X == Y ? launch_gram_tc_df<16, true>(X, Y, Vh, partials, nblocks, gate, s)
                  : launch_gram_tc_df<16, false>(X, Y, Vh, partials, nblocks, gate, s);
  if (k == FK_DF && N == 32)
    return X == Y ? launch_gram_tc_df<32, true>(X, Y, Vh, partials, nblocks, gate, s)
                  : launch_gram_tc_df<32, false>(X, Y, Vh, partials, nblocks, gate, s);
  if (k == FK_H16) {
    if (N == 16) return launch_gram_tc<StoreH16, 16>(X, Y, Vh, partials, nblocks, gate, s);
    if (N == 32) return launch_gram_tc<StoreH16, 32>(X, Y, Vh, partials, nblocks, gate, s);
  } else if (k == FK_BF16) {
    if (N == 16) return launch_gram_tc<StoreBF16, 16>(X, Y, Vh, partials, nblocks, gate, s);
    if (N == 32) return launch_gram_tc<StoreBF16, 32>(X, Y, Vh, partials, nblocks, gate, s);
  }
  return cudaErrorInvalidValue;
}

bool w_gram_tc_supported(FieldKind k, int N) {
  return (k == FK_DF || k == FK_H16 || k == FK_BF16) && (N == 16 || N == 32);
}

cudaError_t w_update_gram_tc(FieldKind k, void* Q, const void* AP, const double2* beta, int N,
                             int Vh, double2* partials, int nblocks, Gate gate, cudaStream_t s) {
  if (k == FK_DF && (N == 16 || N == 32)) {
    // double-float: W = Q - AP beta, then the Gram of the stored W (two passes)
    cudaError_t e = w_update_tc_df(Q, AP, beta, N, Vh, gate, s);
    if (e != cudaSuccess) return e;
    return N == 16 ? launch_gram_tc_df<16, true>(Q, Q, Vh, partials, nblocks, gate, s)
                   : launch_gram_tc_df<32, true>(Q, Q, Vh, partials, nblocks, gate, s);
  }
  if (k == FK_H16) {
    if (N == 16) return launch_w_gram_tc<StoreH16, 16>(Q, AP, beta, Vh, partials, nblocks, gate, s);
    if (N == 32) return launch_w_gram_tc<StoreH16, 32>(Q, AP, beta, Vh, partials, nblocks, gate, s);
  } else if (k == FK_BF16) {
    if (N == 16) return launch_w_gram_tc<StoreBF16, 16>(Q, AP, beta, Vh, partials, nblocks, gate, s);
    if (N == 32) return launch_w_gram_tc<StoreBF16, 32>(Q, AP, beta, Vh, partials, nblocks, gate, s);
  }
  return cudaErrorInvalidValue;
}

bool bcg_update_tc_supported(FieldKind sk, FieldKind xk, int N) {
  if (sk == FK_DF) return xk == FK_DF && bcg_update_tc_df_supported(N);
  return (sk == FK_H16 || sk == FK_BF16) && xk == FK_DF && (N == 16 || N == 32);
}

cudaError_t bcg_update_tc(FieldKind sk, void* Q, void* P, void* X, const double2* Sinv,
                          const double2* BC, const double2* SH, int N, int Vh, Gate gate,
                          cudaStream_t s) {
  if (sk == FK_DF) return bcg_update_tc_df(Q, P, X, Sinv, BC, SH, N, Vh, gate, s);
  if (sk == FK_H16) {
    if (N == 16) return launch_bcg_update_tc<StoreH16, 16>(Q, P, X, Sinv, BC, SH, Vh, gate, s);
    if (N == 32) return launch_bcg_update_tc<StoreH16, 32>(Q, P, X, Sinv, BC, SH, Vh, gate, s);
  } else if (sk == FK_BF16) {
    if (N == 16) return launch_bcg_update_tc<StoreBF16, 16>(Q, P, X, Sinv, BC, SH, Vh, gate, s);
    if (N == 32) return launch_bcg_update_tc<StoreBF16, 32>(Q, P, X, Sinv, BC, SH, Vh, gate, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bcg
