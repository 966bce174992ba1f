// Tensor-core form of the fused blockCGrQ update (Algorithm 1: Q = W S^-1,
// X += P (beta C), P = Q + P S^dag; the streaming multi-BLAS of Sec. 6.3) for
// the double-float kind of the FP64-accurate form, N = 16, and in its W mode
// the W update W = Q - AP beta of Algorithm 1 (its Gram W^dag W follows in
// k_gram_tc_df).
//
// On the FP32 pipes this update costs 12 instructions per double-float
// multiply-add (24 N^2 multiply-adds per row) and is bound by instruction
// issue.  Here the three N x N products run as exact split products on the
// bf16 tensor cores (ozaki.cuh): each row of W and P is scaled by a power of
// two (its largest entry, from the four threads that hold the row) and split
// into six bf16 slices; each coefficient column likewise (its largest entry
// in the matrix's triangular pattern).  For an output (row r, column j) the
// products W_s[r][k] M_t[k][j] with s + t = u are accumulated in one FP32
// accumulator D_u: they share the grid 2^(er + ej - 14 - 8u), and 2N x 6
// terms of at most 2^14.6 units stay below 2^24, so the accumulation is
// exact.  The epilogue adds D_0 .. D_5 in double-float, removes the scales
// and adds Q (for P) or the old X (for X) in double-float.
//
// Work split as in the 16-bit tensor-core update (blas_tc.cu): a warp owns 16
// rows, the A fragments of a thread are 4 consecutive complex numbers of its
// rows ra, rb (k order permuted consistently in A and B), and the B fragments
// of all slices of the three matrices are built once per CTA in shared
// memory in fragment order.  The A slices of the matrix being multiplied
// (first W, then P) go to a per-warp shared-memory area and serve every
// output column tile; P = Q + P S^dag reads back the Q the same thread has
// just written.
#include "internal.h"
#include "ozaki.cuh"

namespace bcg {

using namespace ozaki;

namespace {

constexpr int TCD_WARPS = 8;  // warps per CTA
constexpr int TCD_NSL = 6;    // slices per value

// coefficient entry (i, j) of matrix m in its triangular pattern: 0 = S^-1
// (upper), 1 = beta C (full), 2 = S^dag (lower)
__device__ __forceinline__ bool tcd_in_pattern(int m, int i, int j) {
  return m == 1 || (m == 0 ? i <= j : i >= j);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// (x + y) * 2^ea * 2^eb for a double-float sum held as (s, e)
__device__ __forceinline__ df tcd_scale(dfacc v, int ea, int eb) {
  const float fa = exp2i(ea), fb = exp2i(eb);
  const dfacc w{__fmul_rn(__fmul_rn(v.s, fa), fb), __fmul_rn(__fmul_rn(v.e, fa), fb)};
  return CompDF::fin(w);
}

template <int N, int NM>
struct TcdGeom {
  static constexpr int KS = N / 8;   // k steps of 16 reals
  static constexpr int NT = N / 4;   // output tiles of 8 reals (4 complex columns)
  static constexpr int MB = N / 16;  // k blocks of 16 complex numbers
  static constexpr int FR = KS * NT * 32;
  // shared memory: B fragments [3][NSL][KS][NT][32] uint2, then the A
  // slices of the matrix being multiplied, [warp][KS][NSL][32] uint4
  static constexpr size_t b_bytes = (size_t)NM * TCD_NSL * FR * sizeof(uint2);
  static constexpr size_t a_bytes = (size_t)TCD_WARPS * KS * TCD_NSL * 32 * sizeof(uint4);
  static constexpr size_t smem = b_bytes + a_bytes;
};

}  // namespace

// WMODE: the W update of Algorithm 1 instead, W = Q - AP beta over Q (AP
// passed as P, beta as Sinv; one full coefficient matrix, phase 1 only)
template <int N, bool WMODE>
__global__ void __launch_bounds__(TCD_WARPS * 32, N == 16 ? (WMODE ? 3 : 2) : 1)
    k_bcg_update_tc_df(float4* __restrict__ Q, float4* __restrict__ P, float4* __restrict__ X,
                       const double2* __restrict__ Sinv, const double2* __restrict__ BC,
                       const double2* __restrict__ SH, int Vh, Gate gate) {
  constexpr int NM = WMODE ? 1 : 3;  // coefficient matrices
  using G = TcdGeom<N, NM>;
  constexpr int KS = G::KS, NT = G::NT, MB = G::MB, FR = G::FR, NSL = TCD_NSL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint2* sB = reinterpret_cast<uint2*>(smem_raw);
  uint4* sA = reinterpret_cast<uint4*>(smem_raw + G::b_bytes);
  __shared__ int sE[3 * N];  // column exponents: |column| < 2^e
  if (gate_closed(gate)) return;
  const bool keepP = gate.st != nullptr && ((const volatile SolverStatus*)gate.st)->ru_pending;
  auto Ms = [&](int m) { return m == 0 ? Sinv : m == 1 ? BC : SH; };
  // the full matrix beta in the W update, else the patterns of tcd_in_pattern
  auto in_pattern = [&](int m, int i, int j) { return WMODE || tcd_in_pattern(m, i, j); };

  for (int c = threadIdx.x; c < NM * N; c += blockDim.x) {
    const int m = c / N, j = c - m * N;
    double mx = 0.0;
    for (int i = 0; i < N; ++i) {
      if (!in_pattern(m, i, j)) continue;
      const double2 v = Ms(m)[i * N + j];
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    int e = 0;
    if (mx > 0.0 && mx < 1e300) frexp(mx, &e);  // mx in [2^(e-1), 2^e)
    sE[c] = e < -120 ? -120 : e > 120 ? 120 : e;
  }
  __syncthreads();
  // B fragments: k step ks (k block ks / 2, half ks % 2), lane (g, t): b.x
  // holds rows (re, im) of input i0 = 16 (ks / 2) + 4 t + 2 (ks % 2), b.y
  // those of i0 + 1; column n = 8 nt + g, complex column n / 2, real part
  // when n is even
  for (int idx = threadIdx.x; idx < NM * FR; idx += blockDim.x) {
    const int m = idx / FR;
    int r = idx - m * FR;
    const int ks = r / (NT * 32);
    r -= ks * NT * 32;
    const int nt = r / 32, lane = r - nt * 32;
    const int g = lane >> 2, t = lane & 3;
    const int i0 = 16 * (ks >> 1) + 4 * t + 2 * (ks & 1);
    const int n = 8 * nt + g, j = n >> 1, part = n & 1;
    const double sc = ldexp(1.0, -sE[m * N + j]);
    float sl[2][2][NSL];  // [input i0 / i0 + 1][re row, im row][slice]
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + q;
      double re = 0.0, im = 0.0;
      if (in_pattern(m, i, j)) {
        const double2 v = Ms(m)[i * N + j];
        re = v.x * sc;
        im = v.y * sc;
      }
      const df e0 = df_from_double(part ? im : re), e1 = df_from_double(part ? re : -im);
      split6(e0.hi, e0.lo, sl[q][0]);
      split6(e1.hi, e1.lo, sl[q][1]);
    }
    for (int s = 0; s < NSL; ++s) {
      uint2 b;
      b.x = pack_bf16(sl[0][0][s], sl[0][1][s]);
      b.y = pack_bf16(sl[1][0][s], sl[1][1][s]);
      sB[((m * NSL + s) * KS + ks) * NT * 32 + nt * 32 + lane] = b;
    }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint4* myA = sA + (size_t)warp * KS * NSL * 32;  // [ks][slice][lane]
  const long long nrows = 3LL * Vh;
  const long long ntiles = (nrows + 15) / 16;
  for (long long tile = (long long)blockIdx.x * TCD_WARPS + warp; tile < ntiles;
       tile += (long long)gridDim.x * TCD_WARPS) {
    const long long ra = tile * 16 + g, rb = ra + 8;
    const bool va = ra < nrows, vb = rb < nrows;
    // the P rows of this tile and the W rows of the next are fetched towards
    // L2 while this tile's W is split and multiplied
    if (va) prefetch_l2(P + ra * N + 4 * t);
    if (vb) prefetch_l2(P + rb * N + 4 * t);
    {
      const long long nra = ra + 16 * (long long)gridDim.x * TCD_WARPS;
      if (nra < nrows) prefetch_l2(Q + nra * N + 4 * t);
      if (nra + 8 < nrows) prefetch_l2(Q + (nra + 8) * N + 4 * t);
    }
    // load rows ra, rb of `src` (this thread's 4 complex numbers per k block),
    // split them into the warp's A slices; returns the row exponents
    auto stage = [&](const float4* src, int (&er)[2]) {
      float4 xa[MB][4], xb[MB][4];
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      float ma = 0.f, mb2 = 0.f;
#pragma unroll
      for (int mb = 0; mb < MB; ++mb)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col = 16 * mb + 4 * t + c;
          xa[mb][c] = va ? src[ra * N + col] : z;
          xb[mb][c] = vb ? src[rb * N + col] : z;
          ma = fmaxf(ma, fmaxf(fabsf(xa[mb][c].x), fabsf(xa[mb][c].y)));
          mb2 = fmaxf(mb2, fmaxf(fabsf(xb[mb][c].x), fabsf(xb[mb][c].y)));
        }
      // the four threads t of a row hold its N entries
      ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, 1));
      ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, 2));
      mb2 = fmaxf(mb2, __shfl_xor_sync(0xffffffffu, mb2, 1));
      mb2 = fmaxf(mb2, __shfl_xor_sync(0xffffffffu, mb2, 2));
      er[0] = pow2_above(__float_as_uint(ma));
      er[1] = pow2_above(__float_as_uint(mb2));
      const float sa = exp2i(-er[0]), sb = exp2i(-er[1]);
      // fragment registers of k step ks: a0 = (ra, complex c0), a1 = (rb, c0),
      // a2 = (ra, c0 + 1), a3 = (rb, c0 + 1), c0 = 16 (ks / 2) + 4 t + 2 (ks % 2)
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int mb = ks >> 1, c0 = 2 * (ks & 1);
        const float4 v[4] = {xa[mb][c0], xb[mb][c0], xa[mb][c0 + 1], xb[mb][c0 + 1]};
        uint32_t w[4][NSL];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float sc = (i & 1) ? sb : sa;
          float sr[NSL], si[NSL];
          split6(__fmul_rn(v[i].x, sc), __fmul_rn(v[i].z, sc), sr);
          split6(__fmul_rn(v[i].y, sc), __fmul_rn(v[i].w, sc), si);
#pragma unroll
          for (int s = 0; s < NSL; ++s) w[i][s] = pack_bf16(sr[s], si[s]);
        }
#pragma unroll
        for (int s = 0; s < NSL; ++s)
          myA[(ks * NSL + s) * 32 + lane] = make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]);
      }
    };
    // the staged matrix times coefficient matrix bm, output tile nt, into acc
    auto product = [&](int bm, int nt, float (&acc)[6][4], int kfirst, int klast) {
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[u][i] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        if (ks < kfirst || ks > klast) continue;
        uint32_t a[NSL][4];
#pragma unroll
        for (int s = 0; s < NSL; ++s) {
          const uint4 v = myA[(ks * NSL + s) * 32 + lane];
          a[s][0] = v.x;
          a[s][1] = v.y;
          a[s][2] = v.z;
          a[s][3] = v.w;
        }
#pragma unroll
        for (int tt = 0; tt < NSL; ++tt) {
          const uint2 b = sB[((bm * NSL + tt) * KS + ks) * NT * 32 + nt * 32 + lane];
#pragma unroll
          for (int s = 0; s + tt < NSL; ++s) mma_bf16(acc[s + tt], a[s], b.x, b.y);
        }
      }
    };
    auto value = [&](const float (&acc)[6][4], int i) {
      return combine6(acc[0][i], acc[1][i], acc[2][i], acc[3][i], acc[4][i], acc[5][i]);
    };
    // k steps holding an input i with a nonzero coefficient for output tile
    // nt: S^-1 upper (i <= the tile's last column), S^dag lower (i >= its first)
    auto k_last_upper = [&](int nt) {
      int kl = KS - 1;
#pragma unroll
      for (int ks = KS - 1; ks >= 0; --ks)
        if (16 * (ks >> 1) > 4 * nt + 3) kl = ks - 1;
      return kl;
    };
    auto k_first_lower = [&](int nt) {
      int kf = 0;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
        if (16 * (ks >> 1) + 15 < 4 * nt) kf = ks + 1;
      return kf;
    };
    float acc[6][4];
    int erw[2], erp[2];
    if constexpr (WMODE) {
      // W = Q - AP beta, over Q
      stage(P, erp);
      __syncwarp();
#pragma unroll 1
      for (int nt = 0; nt < NT; ++nt) {
        const int j = 4 * nt + t;
        product(0, nt, acc, 0, KS - 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!(h ? vb : va)) continue;
          float4* qp = Q + (h ? rb : ra) * N + j;
          cpx<dfacc> wv = cacc_from<CompDF>(StoreDF::load_nc(qp));
          const df pr = tcd_scale(value(acc, 2 * h), erp[h], sE[j]);
          const df pi = tcd_scale(value(acc, 2 * h + 1), erp[h], sE[j]);
          CompDF::add(wv.re, df{-pr.hi, -pr.lo});
          CompDF::add(wv.im, df{-pi.hi, -pi.lo});
          StoreDF::store(qp, cfin<CompDF>(wv));
        }
      }
      __syncwarp();
      continue;
    }
    // phase 1: Q = W S^-1 (W is held in the Q buffer and overwritten by Q)
    stage(Q, erw);
    __syncwarp();
#pragma unroll 1
    for (int nt = 0; nt < NT; ++nt) {
      const int j = 4 * nt + t;  // this thread's complex output column
      product(0, nt, acc, 0, k_last_upper(nt));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!(h ? vb : va)) continue;
        cpx<df> q;
        q.re = tcd_scale(value(acc, 2 * h), erw[h], sE[0 * N + j]);
        q.im = tcd_scale(value(acc, 2 * h + 1), erw[h], sE[0 * N + j]);
        StoreDF::store(Q + (h ? rb : ra) * N + j, q);
      }
    }
    __syncwarp();  // W's slices are read before P's overwrite them
    // phase 2: P = Q + P S^dag (Q read back: this thread wrote it) and
    // X += P (beta C), both from the old P's slices
    stage(P, erp);
    __syncwarp();
#pragma unroll 1
    for (int nt = 0; nt < NT; ++nt) {
      const int j = 4 * nt + t;
      if (!keepP) {
        product(2, nt, acc, k_first_lower(nt), KS - 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!(h ? vb : va)) continue;
          const long long o = (h ? rb : ra) * N + j;
          cpx<dfacc> pv = cacc_from<CompDF>(StoreDF::load_nc(Q + o));
          CompDF::add(pv.re, tcd_scale(value(acc, 2 * h), erp[h], sE[2 * N + j]));
          CompDF::add(pv.im, tcd_scale(value(acc, 2 * h + 1), erp[h], sE[2 * N + j]));
          StoreDF::store(P + o, cfin<CompDF>(pv));
        }
      }
      product(1, nt, acc, 0, KS - 1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!(h ? vb : va)) continue;
        float4* xp = X + (h ? rb : ra) * N + j;
        cpx<dfacc> xv = cacc_from<CompDF>(StoreDF::load_nc(xp));
        CompDF::add(xv.re, tcd_scale(value(acc, 2 * h), erp[h], sE[1 * N + j]));
        CompDF::add(xv.im, tcd_scale(value(acc, 2 * h + 1), erp[h], sE[1 * N + j]));
        StoreDF::store(xp, cfin<CompDF>(xv));
      }
    }
    __syncwarp();  // this tile's A slices are read before the next tile writes them
  }
}

bool bcg_update_tc_df_supported(int N) { return N == 16; }

template <int N, bool WMODE>
static cudaError_t launch_update_tc_df(void* Q, void* P, void* X, const double2* Sinv,
                                       const double2* BC, const double2* SH, int Vh, Gate gate,
                                       cudaStream_t s) {
  using G = TcdGeom<N, WMODE ? 1 : 3>;
  auto kern = k_bcg_update_tc_df<N, WMODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TCD_WARPS * 32, G::smem) !=
          cudaSuccess ||
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
  long long blocks = (tiles + TCD_WARPS - 1) / TCD_WARPS;
  if (blocks > (long long)sms * per_sm) blocks = (long long)sms * per_sm;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, TCD_WARPS * 32, G::smem, s>>>((float4*)Q, (float4*)P, (float4*)X, Sinv,
                                                         BC, SH, Vh, gate);
  return cudaGetLastError();
}

cudaError_t bcg_update_tc_df(void* Q, void* P, void* X, const double2* Sinv, const double2* BC,
                             const double2* SH, int N, int Vh, Gate gate, cudaStream_t s) {
  if (N != 16) return cudaErrorInvalidValue;
  return launch_update_tc_df<16, false>(Q, P, X, Sinv, BC, SH, Vh, gate, s);
}

// N = 32 too: one coefficient matrix (48 KB of fragments) and the A slices of
// 8 warps (96 KB) fit one CTA per SM; the three matrices of the fused update
// at N = 32 would not
cudaError_t w_update_tc_df(void* Q, const void* AP, const double2* beta, int N, int Vh, Gate gate,
                           cudaStream_t s) {
  void* A = const_cast<void*>(AP);
  if (N == 16)
    return launch_update_tc_df<16, true>(Q, A, nullptr, beta, nullptr, nullptr, Vh, gate, s);
  if (N == 32)
    return launch_update_tc_df<32, true>(Q, A, nullptr, beta, nullptr, nullptr, Vh, gate, s);
  return cudaErrorInvalidValue;
}

}  // namespace bcg
