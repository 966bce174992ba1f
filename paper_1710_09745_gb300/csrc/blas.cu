// Block BLAS on L x N block vectors (L = 3 Vh complex rows, N right-hand
// sides), stored site-major [site][colour][rhs] (row = (site, colour), the N
// columns of a row contiguous).
//
//  * Reduction multi-BLAS (Sec. 6.4): K = X^dag Y as per-CTA partial sums
//    (gram_partials) followed by a deterministic fixed-order FP64 reduction
//    over CTAs (gram_reduce).  Hermitian Grams compute only the upper
//    triangle and the reduction mirrors it (the Hermitian policy of
//    Sec. 6.4).
//  * Streaming multi-BLAS (Sec. 6.3): every kernel reads each input row once
//    and keeps the N x N work on chip, so traffic is linear in N.  The fused
//    blockCGrQ update (bcg_update) stages a tile of sites of W and P in shared
//    memory and produces, in one pass, Q = W S^-1 (S upper triangular: the
//    zero half is skipped, Sec. 6.3), X += P (beta C) (the X update of
//    Algorithm 1 using the P of this iteration, Sec. 6.2) and the next search
//    block P = Q + P S^dag (Algorithm 1).  Coefficient columns are staged in
//    chunks of JT columns so that N = 64 fits in shared memory.
#include <type_traits>

#include "internal.h"
#include "tma.cuh"

namespace bcg {

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }
// grid for grid-stride kernels: enough CTAs to fill the GPU, never a huge
// grid of trivial CTAs (a gated-off launch then costs a few microseconds)
// streaming multiprocessors of the current device (152 on a GB300)
static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 152;
    }
    n = v;
  }
  return n;
}

static inline unsigned gcap(long long n, int t, unsigned cap = 152 * 8) {
  unsigned b = nblk(n, t);
  return b < cap ? (b ? b : 1) : cap;
}

// ------------------------------------------------------------ layout ----
template <class S>
__global__ void k_to_internal(const double2* __restrict__ user, typename S::elem* __restrict__ in,
                              int N, int Vh) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)Vh * N * 3;
  if (idx >= total) return;
  int j = (int)(idx % N);
  long long t = idx / N;
  int c = (int)(t % 3);
  long long site = t / 3;
  in[idx] = S::from_double2(user[((long long)j * Vh + site) * 3 + c]);
}

template <class S>
__global__ void k_from_internal(const typename S::elem* __restrict__ in, double2* __restrict__ user,
                                int N, int Vh) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)Vh * N * 3;
  if (idx >= total) return;
  int j = (int)(idx % N);
  long long t = idx / N;
  int c = (int)(t % 3);
  long long site = t / 3;
  user[((long long)j * Vh + site) * 3 + c] = S::to_double2(in[idx]);
}

cudaError_t to_internal(FieldKind k, const double2* user, void* internal, int N, int Vh,
                        cudaStream_t s) {
  long long total = (long long)Vh * N * 3;
  switch (k) {
    case FK_DF:
      k_to_internal<StoreDF><<<nblk(total, 256), 256, 0, s>>>(user, (float4*)internal, N, Vh);
      break;
    case FK_F32:
      k_to_internal<StoreF32><<<nblk(total, 256), 256, 0, s>>>(user, (float2*)internal, N, Vh);
      break;
    case FK_F64:
      k_to_internal<StoreF64><<<nblk(total, 256), 256, 0, s>>>(user, (double2*)internal, N, Vh);
      break;
    case FK_H16:
      k_to_internal<StoreH16><<<nblk(total, 256), 256, 0, s>>>(user, (__half2*)internal, N, Vh);
      break;
    case FK_BF16:
      k_to_internal<StoreBF16><<<nblk(total, 256), 256, 0, s>>>(user, (__nv_bfloat162*)internal, N, Vh);
      break;
  }
  return cudaGetLastError();
}

cudaError_t from_internal(FieldKind k, const void* internal, double2* user, int N, int Vh,
                          cudaStream_t s) {
  long long total = (long long)Vh * N * 3;
  switch (k) {
    case FK_DF:
      k_from_internal<StoreDF><<<nblk(total, 256), 256, 0, s>>>((const float4*)internal, user, N, Vh);
      break;
    case FK_F32:
      k_from_internal<StoreF32><<<nblk(total, 256), 256, 0, s>>>((const float2*)internal, user, N, Vh);
      break;
    case FK_F64:
      k_from_internal<StoreF64><<<nblk(total, 256), 256, 0, s>>>((const double2*)internal, user, N, Vh);
      break;
    case FK_H16:
      k_from_internal<StoreH16><<<nblk(total, 256), 256, 0, s>>>((const __half2*)internal, user, N, Vh);
      break;
    case FK_BF16:
      k_from_internal<StoreBF16><<<nblk(total, 256), 256, 0, s>>>((const __nv_bfloat162*)internal, user, N, Vh);
      break;
  }
  return cudaGetLastError();
}

cudaError_t zero_field(FieldKind k, void* f, size_t n_elems, cudaStream_t s) {
  return cudaMemsetAsync(f, 0, n_elems * elem_bytes(k), s);
}

cudaError_t copy_field(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

// -------------------------------------------------------------- Gram ----
static constexpr int GRAM_THREADS = 256;

__host__ __device__ inline int gram_entries(int N, int herm) { return herm ? N * (N + 1) / 2 : N * N; }

__device__ inline void entry_ij(int e, int N, int herm, int& i, int& j) {
  if (!herm) {
    i = e / N;
    j = e - i * N;
    return;
  }
  int r = 0, off = 0;
  while (off + (N - r) <= e) {
    off += N - r;
    ++r;
  }
  i = r;
  j = r + (e - off);
}

int gram_blocks(int N, int rows) {
  // enough CTAs to fill the GPU a few times over, but never fewer rows per
  // CTA than 64
  int b = 4 * 152;
  int maxb = (rows + 63) / 64;
  if (b > maxb) b = maxb;
  if (b < 1) b = 1;
  return b;
}

// Register-blocked Gram: a CTA stages TS sites of X and Y in shared memory
// (coalesced 128-bit loads of whole sites), then each thread accumulates a
// B x B block of entries (i, j) over the rows of its row group, so every
// value read from shared memory feeds B complex multiply-adds.  Hermitian
// Grams visit only the blocks on and above the block diagonal (Sec. 6.4).
// The CTA walks the tiles grid-stride and writes one N x N partial (row-major
// [i][j], only the blocks it computed) for the fixed-order reduction.
template <class S, int B>
__global__ void __launch_bounds__(GRAM_THREADS)
    k_gram(const typename S::elem* __restrict__ X, const typename S::elem* __restrict__ Y, int N,
           int Vh, int herm, int same, int TS, double2* __restrict__ partials, Gate gate) {
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(gate)) return;
  cpx<real>* sX = reinterpret_cast<cpx<real>*>(smem_raw);
  cpx<real>* sY = same ? sX : sX + TS * N * 3;
  const int tid = threadIdx.x;
  const int nb = (N + B - 1) / B;
  const int NB = herm ? nb * (nb + 1) / 2 : nb * nb;
  const int G = NB >= GRAM_THREADS ? 1 : GRAM_THREADS / NB;
  const int grp = tid / NB;
  const int blk = tid - grp * NB;
  const bool active = grp < G && blk < NB;
  int bi = 0, bj = 0;
  if (herm) {
    int r = 0, off = 0;
    while (off + (nb - r) <= blk) {
      off += nb - r;
      ++r;
    }
    bi = r;
    bj = r + (blk - off);
  } else {
    bi = blk / nb;
    bj = blk - bi * nb;
  }
  const int i0 = bi * B, j0 = bj * B;
  cpx<acc> a[B][B];
#pragma unroll
  for (int u = 0; u < B; ++u)
#pragma unroll
    for (int v = 0; v < B; ++v) a[u][v] = czero<C>();

  for (long long tile = blockIdx.x; tile * TS < Vh; tile += gridDim.x) {
    const long long site0 = tile * TS;
    const int ns = (int)min((long long)TS, (long long)Vh - site0);
    const int nel = ns * N * 3;
    const long long base = site0 * N * 3;
    __syncthreads();
    for (int idx = tid; idx < nel; idx += GRAM_THREADS) {
      sX[idx] = S::load(X + base + idx);
      if (!same) sY[idx] = S::load(Y + base + idx);
    }
    __syncthreads();
    if (active) {
      for (int r = grp; r < ns * 3; r += G) {
        const int s = r / 3;
        const int c = r - s * 3;
        const cpx<real>* xr = sX + (s * 3 + c) * N;
        const cpx<real>* yr = sY + (s * 3 + c) * N;
        cpx<real> xv[B], yv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          xv[u] = (i0 + u < N) ? xr[i0 + u] : cpx<real>{C::rzero(), C::rzero()};
          yv[u] = (j0 + u < N) ? yr[j0 + u] : cpx<real>{C::rzero(), C::rzero()};
        }
#pragma unroll
        for (int u = 0; u < B; ++u)
#pragma unroll
          for (int v = 0; v < B; ++v) cmac_conj<C>(a[u][v], xv[u], yv[v]);
      }
    }
  }
  // reduce the row groups of each block through shared memory, one entry of
  // the B x B block at a time, and write this CTA's partial
  __syncthreads();
  double2* red = reinterpret_cast<double2*>(smem_raw);
  double2* out = partials + (long long)blockIdx.x * N * N;
#pragma unroll
  for (int u = 0; u < B; ++u)
#pragma unroll
    for (int v = 0; v < B; ++v) {
      red[tid] = active ? make_double2(C::to_double(a[u][v].re), C::to_double(a[u][v].im))
                        : make_double2(0.0, 0.0);
      __syncthreads();
      if (tid < NB) {
        double2 sacc = red[tid];
        for (int g2 = 1; g2 < G; ++g2) {
          double2 w = red[g2 * NB + tid];
          sacc.x += w.x;
          sacc.y += w.y;
        }
        if (i0 + u < N && j0 + v < N) out[(i0 + u) * N + (j0 + v)] = sacc;
      }
      __syncthreads();
    }
}

// warp per entry of the result (upper triangle when Hermitian); fixed
// summation order over the per-CTA partials -> deterministic
__global__ void k_gram_reduce(const double2* __restrict__ partials, int nblocks, int N, int herm,
                              double2* __restrict__ out, Gate gate) {
  if (gate_closed(gate)) return;
  const int E = gram_entries(N, herm);
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= E) return;
  int i, j;
  entry_ij(warp, N, herm, i, j);
  double sx = 0.0, sy = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    double2 v = partials[(long long)b * N * N + i * N + j];
    sx += v.x;
    sy += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    sy += __shfl_down_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) {
    out[i * N + j] = make_double2(sx, (herm && i == j) ? 0.0 : sy);
    if (herm && i != j) out[j * N + i] = make_double2(sx, -sy);
  }
}

// sites per Gram tile: the requested count, else 256 / N; never more than
// fits 200 KB of shared memory
static int gram_tile(int req, int N, size_t per_site) {
  int TS = req > 0 ? req : 256 / N;
  if (TS < 1) TS = 1;
  while (TS > 1 && (size_t)TS * per_site > 200 * 1024) TS >>= 1;
  return TS;
}

template <class S, int B>
static void launch_gram_b(const void* X, const void* Y, int N, int Vh, int herm, double2* partials,
                          int nblocks, Gate gate, int tile, cudaStream_t s) {
  using real = typename S::comp::real;
  int same = (X == Y);
  const int TS = gram_tile(tile, N, (same ? 1 : 2) * (size_t)N * 3 * sizeof(cpx<real>));
  size_t tiles = (same ? 1 : 2) * (size_t)TS * N * 3 * sizeof(cpx<real>);
  size_t red = GRAM_THREADS * sizeof(double2);
  size_t sm = tiles > red ? tiles : red;
  cudaFuncSetAttribute(k_gram<S, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gram<S, B><<<nblocks, GRAM_THREADS, sm, s>>>((const typename S::elem*)X,
                                                (const typename S::elem*)Y, N, Vh, herm, same, TS,
                                                partials, gate);
}

template <class S>
static void launch_gram(const void* X, const void* Y, int N, int Vh, int herm, double2* partials,
                        int nblocks, Gate gate, int tile, cudaStream_t s) {
  if (N == 1)
    launch_gram_b<S, 1>(X, Y, N, Vh, herm, partials, nblocks, gate, tile, s);
  else if (N <= 16)
    launch_gram_b<S, 2>(X, Y, N, Vh, herm, partials, nblocks, gate, tile, s);
  else
    launch_gram_b<S, 4>(X, Y, N, Vh, herm, partials, nblocks, gate, tile, s);
}

cudaError_t gram_partials(FieldKind k, const void* X, const void* Y, int N, int Vh, int hermitian,
                          double2* partials, int nblocks, Gate gate, cudaStream_t s, int tile) {
  if ((tile & GR_TC) && hermitian && w_gram_tc_supported(k, N))
    return gram_partials_tc(k, X, Y, N, Vh, partials, nblocks, gate, s);
  tile &= ~GR_TC;
  switch (k) {
    case FK_DF: launch_gram<StoreDF>(X, Y, N, Vh, hermitian, partials, nblocks, gate, tile, s); break;
    case FK_F32: launch_gram<StoreF32>(X, Y, N, Vh, hermitian, partials, nblocks, gate, tile, s); break;
    case FK_F64: launch_gram<StoreF64>(X, Y, N, Vh, hermitian, partials, nblocks, gate, tile, s); break;
    case FK_H16: launch_gram<StoreH16>(X, Y, N, Vh, hermitian, partials, nblocks, gate, tile, s); break;
    case FK_BF16: launch_gram<StoreBF16>(X, Y, N, Vh, hermitian, partials, nblocks, gate, tile, s); break;
  }
  return cudaGetLastError();
}

cudaError_t gram_reduce(const double2* partials, int nblocks, int N, int hermitian, double2* out,
                        Gate gate, cudaStream_t s) {
  int E = gram_entries(N, hermitian);
  k_gram_reduce<<<nblk((long long)E * 32, 256), 256, 0, s>>>(partials, nblocks, N, hermitian, out,
                                                             gate);
  return cudaGetLastError();
}

// ------------------------------------------ W = Q - AP beta with W^dag W ----
// The streaming W update of Algorithm 1 (Sec. 6.3) and the reduction that
// follows it (the Gram W^dag W of the thin QR, Algorithm 2; Sec. 6.4) in one
// pass: a CTA stages a tile of TS sites of Q and AP in shared memory, forms
// W = Q - AP beta there (each entry by the one thread that writes it back
// over Q), stores W, and accumulates the tile's Hermitian Gram from the
// staged W with the register blocking of k_gram; the per-CTA partials go to
// the same fixed-order reduction.  W is read from HBM once fewer than with a
// separate Gram pass.
static constexpr int WGJ = 4;  // columns of W per thread in k_w_gram

template <class S, int B>
__global__ void __launch_bounds__(GRAM_THREADS)
    k_w_gram(typename S::elem* __restrict__ Q, const typename S::elem* __restrict__ AP,
             const double2* __restrict__ beta, int N, int Vh, int TS,
             double2* __restrict__ partials, Gate gate) {
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(gate)) return;
  cpx<real>* sW = reinterpret_cast<cpx<real>*>(smem_raw);  // Q, then W
  cpx<real>* sA = sW + TS * N * 3;                           // AP
  cpx<real>* sb = sA + TS * N * 3;                           // beta [N][N]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < N * N; idx += GRAM_THREADS) {
    const double2 v = beta[idx];
    sb[idx] = {C::from_double(v.x), C::from_double(v.y)};
  }
  const int nb = (N + B - 1) / B;
  const int NB = nb * (nb + 1) / 2;
  const int G = NB >= GRAM_THREADS ? 1 : GRAM_THREADS / NB;
  const int grp = tid / NB;
  const int blk = tid - grp * NB;
  const bool active = grp < G && blk < NB;
  int bi = 0, bj = 0;
  {
    int r = 0, off = 0;
    while (off + (nb - r) <= blk) {
      off += nb - r;
      ++r;
    }
    bi = r;
    bj = r + (blk - off);
  }
  const int i0 = bi * B, j0 = bj * B;
  cpx<acc> a[B][B];
#pragma unroll
  for (int u = 0; u < B; ++u)
#pragma unroll
    for (int v = 0; v < B; ++v) a[u][v] = czero<C>();

  for (long long tile = blockIdx.x; tile * TS < Vh; tile += gridDim.x) {
    const long long site0 = tile * TS;
    const int ns = (int)min((long long)TS, (long long)Vh - site0);
    const int nel = ns * N * 3;
    const long long base = site0 * N * 3;
    __syncthreads();
    for (int idx = tid; idx < nel; idx += GRAM_THREADS) {
      sW[idx] = S::load_nc(Q + base + idx);
      sA[idx] = S::load(AP + base + idx);
    }
    __syncthreads();
    // W = Q - AP beta: a thread owns WR rows x WGJ consecutive columns, so
    // each beta value read from shared memory feeds WR multiply-adds and each
    // AP value WGJ of them (WR = 2 for the FP32-arithmetic kinds, whose
    // multiply-adds are cheap enough that shared-memory reads would bound them)
    constexpr int WR = std::is_same<real, float>::value ? 2 : 1;
    const int ng = (N + WGJ - 1) / WGJ;
    const int nrg = (ns * 3 + WR - 1) / WR;
    for (int u = tid; u < nrg * ng; u += GRAM_THREADS) {
      const int rg = u / ng, j0 = (u - rg * ng) * WGJ;
      cpx<acc> w[WR][WGJ];
#pragma unroll
      for (int rr = 0; rr < WR; ++rr) {
        const int row = rg * WR + rr;
#pragma unroll
        for (int v = 0; v < WGJ; ++v)
          w[rr][v] = (row < ns * 3 && j0 + v < N) ? cacc_from<C>(sW[row * N + j0 + v]) : czero<C>();
      }
      for (int i = 0; i < N; ++i) {
        cpx<real> bb[WGJ];
#pragma unroll
        for (int v = 0; v < WGJ; ++v)
          bb[v] = (j0 + v < N) ? sb[i * N + j0 + v] : cpx<real>{C::rzero(), C::rzero()};
#pragma unroll
        for (int rr = 0; rr < WR; ++rr) {
          const int row = min(rg * WR + rr, ns * 3 - 1);  // a ragged group repeats a row
          const cpx<real> ap = sA[row * N + i];
#pragma unroll
          for (int v = 0; v < WGJ; ++v) {
            // w -= ap * bb
            C::msub(w[rr][v].re, ap.re, bb[v].re);
            C::mac(w[rr][v].re, ap.im, bb[v].im);
            C::msub(w[rr][v].im, ap.re, bb[v].im);
            C::msub(w[rr][v].im, ap.im, bb[v].re);
          }
        }
      }
#pragma unroll
      for (int rr = 0; rr < WR; ++rr) {
        const int row = rg * WR + rr;
        if (row >= ns * 3) continue;
#pragma unroll
        for (int v = 0; v < WGJ; ++v) {
          if (j0 + v < N) {
            typename S::elem e;
            S::store(&e, cfin<C>(w[rr][v]));
            Q[base + row * N + j0 + v] = e;
            // the value as stored (rounded to the storage format) feeds the Gram
            sW[row * N + j0 + v] = S::load_nc(&e);
          }
        }
      }
    }
    __syncthreads();
    if (active) {
      for (int r = grp; r < ns * 3; r += G) {
        const cpx<real>* wr = sW + r * N;
        cpx<real> xv[B], yv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          xv[u] = (i0 + u < N) ? wr[i0 + u] : cpx<real>{C::rzero(), C::rzero()};
          yv[u] = (j0 + u < N) ? wr[j0 + u] : cpx<real>{C::rzero(), C::rzero()};
        }
#pragma unroll
        for (int u = 0; u < B; ++u)
#pragma unroll
          for (int v = 0; v < B; ++v) cmac_conj<C>(a[u][v], xv[u], yv[v]);
      }
    }
  }
  __syncthreads();
  double2* red = reinterpret_cast<double2*>(smem_raw);
  double2* out = partials + (long long)blockIdx.x * N * N;
#pragma unroll
  for (int u = 0; u < B; ++u)
#pragma unroll
    for (int v = 0; v < B; ++v) {
      red[tid] = active ? make_double2(C::to_double(a[u][v].re), C::to_double(a[u][v].im))
                        : make_double2(0.0, 0.0);
      __syncthreads();
      if (tid < NB) {
        double2 sacc = red[tid];
        for (int g2 = 1; g2 < G; ++g2) {
          double2 w = red[g2 * NB + tid];
          sacc.x += w.x;
          sacc.y += w.y;
        }
        if (i0 + u < N && j0 + v < N) out[(i0 + u) * N + (j0 + v)] = sacc;
      }
      __syncthreads();
    }
}

template <class S, int B>
static void launch_w_gram_b(void* Q, const void* AP, const double2* beta, int N, int Vh,
                            double2* partials, int nblocks, Gate gate, int tile, cudaStream_t s) {
  using real = typename S::comp::real;
  const int TS = gram_tile(tile, N, 2 * (size_t)N * 3 * sizeof(cpx<real>));
  const size_t tiles = (2 * (size_t)TS * N * 3 + (size_t)N * N) * sizeof(cpx<real>);
  const size_t red = GRAM_THREADS * sizeof(double2);
  const size_t sm = tiles > red ? tiles : red;
  cudaFuncSetAttribute(k_w_gram<S, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_w_gram<S, B><<<nblocks, GRAM_THREADS, sm, s>>>((typename S::elem*)Q,
                                                  (const typename S::elem*)AP, beta, N, Vh, TS,
                                                  partials, gate);
}

template <class S>
static void launch_w_gram(void* Q, const void* AP, const double2* beta, int N, int Vh,
                          double2* partials, int nblocks, Gate gate, int tile, cudaStream_t s) {
  if (N == 1)
    launch_w_gram_b<S, 1>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s);
  else if (N <= 16)
    launch_w_gram_b<S, 2>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s);
  else
    launch_w_gram_b<S, 4>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s);
}

cudaError_t w_update_gram(FieldKind k, void* Q, const void* AP, const double2* beta, int N, int Vh,
                          double2* partials, int nblocks, Gate gate, cudaStream_t s, int tile) {
  if ((tile & WG_TC) && w_gram_tc_supported(k, N))
    return w_update_gram_tc(k, Q, AP, beta, N, Vh, partials, nblocks, gate, s);
  tile &= ~WG_TC;
  switch (k) {
    case FK_DF: launch_w_gram<StoreDF>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s); break;
    case FK_F32: launch_w_gram<StoreF32>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s); break;
    case FK_F64: launch_w_gram<StoreF64>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s); break;
    case FK_H16: launch_w_gram<StoreH16>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s); break;
    case FK_BF16: launch_w_gram<StoreBF16>(Q, AP, beta, N, Vh, partials, nblocks, gate, tile, s); break;
  }
  return cudaGetLastError();
}

// -------------------------------------------------- coefficient stage ----
template <class C>
__device__ __forceinline__ void stage_coef(cpx<typename C::real>* dst, const double2* __restrict__ M,
                                           int N, int j0, int jn, int JT) {
  for (int idx = threadIdx.x; idx < N * jn; idx += blockDim.x) {
    int i = idx / jn, jj = idx - i * jn;
    double2 v = M[i * N + j0 + jj];
    dst[i * JT + jj] = {C::from_double(v.x), C::from_double(v.y)};
  }
}

// ------------------------------------------------------ fused update ----
// Tile geometry: TS sites per CTA, coefficient columns in chunks of JT.
struct TileCfg {
  int TS, JT;
};

static TileCfg tile_cfg(int N, size_t real_cplx_bytes, int n_tiles, int n_coefs,
                        size_t budget = 96 * 1024) {
  // all N coefficient columns at once when they fit 64 KB (staged once per
  // tile pass instead of once per 16-column chunk), else chunks of 16
  int JT = (size_t)n_coefs * N * N * real_cplx_bytes <= 64 * 1024 ? N : 16;
  if (JT > N) JT = N;
  size_t coef = (size_t)n_coefs * N * JT * real_cplx_bytes;
  if (budget < coef + 32 * 1024) budget = coef + 32 * 1024;
  int TS = 32;
  while (TS > 1 && coef + (size_t)n_tiles * TS * N * 3 * real_cplx_bytes > budget) TS >>= 1;
  return {TS, JT};
}

// Each thread produces JB consecutive output columns j of one row (site,
// colour), so every W and P value read from shared memory feeds JB outputs.
// DB: the W, P and X tiles of the next tile are copied with cp.async, as
// stored, into a second shared buffer while the current one is computed, and
// converted when read; without DB the tiles hold converted values.
template <class SS, bool DB>
struct UpdTile {
  using T = cpx<typename SS::comp::real>;
  static __device__ __forceinline__ T get(const T* p) { return *p; }
};
template <class SS>
struct UpdTile<SS, true> {
  using T = typename SS::elem;
  static __device__ __forceinline__ cpx<typename SS::comp::real> get(const T* p) {
    return SS::load_nc(p);  // a plain (generic) read: valid on shared memory
  }
};

// bytes of the W and P tiles of one buffer set, rounded up to 16 so that the
// X tile behind them can take 16-byte asynchronous copies
__host__ __device__ inline size_t upd_wp_bytes(int TS, int N, size_t tile_elem) {
  return (2 * (size_t)TS * 3 * (N + 1) * tile_elem + 15) / 16 * 16;
}
template <class SS, class XS, int JB, bool DB, int RT, bool XSTAGE>
__global__ void __launch_bounds__(256, 3)
    k_bcg_update(typename SS::elem* __restrict__ Q, typename SS::elem* __restrict__ P,
                 typename XS::elem* __restrict__ X, const double2* __restrict__ Sinv,
                 const double2* __restrict__ BC, const double2* __restrict__ SH, int N, int Vh,
                 int TS, int JT, Gate gate) {
  using C = typename SS::comp;
  using CX = typename XS::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(gate)) return;
  const bool keepP = gate.st != nullptr && ((const volatile SolverStatus*)gate.st)->ru_pending;
  // W and P tiles with a row stride of N + 1 complex numbers, so that the
  // rows read by the lanes of a warp fall into different shared-memory banks
  const int RS = N + 1;
  using XE = typename XS::elem;
  // tiles: W, P (padded rows) and, with DB, the X tile; two sets with DB
  using TR = UpdTile<SS, DB>;
  using TT = typename TR::T;
  const int tile_w = TS * 3 * RS;
  // one set = [W tile][P tile][X tile (DB only)]; set b starts b * set_bytes in
  const size_t wp_bytes = upd_wp_bytes(TS, N, sizeof(TT));
  // XSTAGE: the old X is copied into the tile set too (else read from global
  // memory in the epilogue: each thread reads JB consecutive elements, whole
  // sectors, and the smaller tiles allow more resident blocks)
  const size_t set_bytes = wp_bytes + (DB && XSTAGE ? (size_t)TS * 3 * N * sizeof(XE) : 0);
  auto tW = [&](int bsel) { return reinterpret_cast<TT*>(smem_raw + bsel * set_bytes); };
  auto tP = [&](int bsel) { return tW(bsel) + tile_w; };
  auto tX = [&](int bsel) { return reinterpret_cast<XE*>(smem_raw + bsel * set_bytes + wp_bytes); };
  TT* sW = tW(0);
  TT* sP = tP(0);
  XE* sX = tX(0);
  cpx<real>* sA = reinterpret_cast<cpx<real>*>(smem_raw + (DB ? 2 : 1) * set_bytes);  // Sinv chunk [N][JT]
  cpx<real>* sB = sA + N * JT;                         // BC chunk
  cpx<real>* sC = sB + N * JT;                         // SH chunk
  const bool one_chunk = (JT >= N);
  if (one_chunk) {  // all coefficients fit: stage them once per CTA
    stage_coef<C>(sA, Sinv, N, 0, N, JT);
    stage_coef<C>(sB, BC, N, 0, N, JT);
    if (!keepP) stage_coef<C>(sC, SH, N, 0, N, JT);
  }
  // asynchronous copy of tile t into buffer set bsel (DB only): the copied
  // elements are the stored ones, bit-identical to cpx<real> for FP32
  auto issue = [&](long long t, int bsel) {
    const long long s0 = t * TS;
    const int nsi = (int)min((long long)TS, (long long)Vh - s0);
    const long long bs = s0 * N * 3;
    for (int idx = threadIdx.x; idx < nsi * N * 3; idx += blockDim.x) {
      const int rr = idx / N, cc = idx - rr * N;
      cp_async_bytes(tW(bsel) + rr * RS + cc, Q + bs + idx, sizeof(typename SS::elem));
      cp_async_bytes(tP(bsel) + rr * RS + cc, P + bs + idx, sizeof(typename SS::elem));
      if (XSTAGE) cp_async_bytes(tX(bsel) + idx, X + bs + idx, sizeof(XE));
    }
    cp_async_commit();
  };
  int bcur = 0;
  if (DB && (long long)blockIdx.x * TS < Vh) issue(blockIdx.x, 0);
  for (long long tile = blockIdx.x; tile * TS < Vh; tile += gridDim.x, bcur ^= 1) {
    const long long site0 = tile * TS;
    const int ns = (int)min((long long)TS, (long long)Vh - site0);
    const long long base = site0 * N * 3;
    const int nel = ns * N * 3;
    if (DB) {
      // every thread is done with the previous tile's set before the next
      // tile is copied into it; then wait for this tile's copies
      __syncthreads();
      const long long nxt = tile + gridDim.x;
      if (nxt * TS < Vh) issue(nxt, bcur ^ 1);
      else cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      sW = tW(bcur);
      sP = tP(bcur);
      sX = tX(bcur);
    } else {
      __syncthreads();
      if constexpr (!DB) {
        for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
          const int rr = idx / N, cc = idx - rr * N;
          sW[rr * RS + cc] = SS::load_nc(Q + base + idx);
          sP[rr * RS + cc] = SS::load_nc(P + base + idx);
        }
      }
    }
    for (int j0 = 0; j0 < N; j0 += JT) {
      const int jn = min(JT, N - j0);
      if (!one_chunk) {
        __syncthreads();
        stage_coef<C>(sA, Sinv, N, j0, jn, JT);
        stage_coef<C>(sB, BC, N, j0, jn, JT);
        if (!keepP) stage_coef<C>(sC, SH, N, j0, jn, JT);
      }
      __syncthreads();
      const int ng = (jn + JB - 1) / JB;  // column groups
      const int nrows = ns * 3;
      const int nrg = (nrows + RT - 1) / RT;  // groups of RT rows
      const int nout = nrg * ng;
      // column group major: the lanes of a warp share the group (and hence
      // the triangular loop bounds) and differ only in the rows.  A thread
      // owns RT rows x JB columns, so every coefficient read from shared
      // memory feeds RT multiply-adds and every W, P value JB of them.
      for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int jg = o / nrg;
        const int row0 = (o - jg * nrg) * RT;  // first (site, colour) row
        const int jj0 = jg * JB;
        const TT* w[RT];
        const TT* p[RT];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) {
          const int row = (row0 + rr < nrows) ? row0 + rr : row0;  // a ragged group repeats a row
          w[rr] = sW + row * RS;
          p[rr] = sP + row * RS;
        }
        cpx<acc> q[RT][JB], x[RT][JB], pn[RT][JB];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr)
#pragma unroll
          for (int u = 0; u < JB; ++u) {
            q[rr][u] = czero<C>();
            x[rr][u] = czero<C>();
            pn[rr][u] = czero<C>();
          }
        // i ranges: [0, jlo) feeds Q and X of every column of the group;
        // [jlo, jlo + JB) is the diagonal band (per-column conditions);
        // [jlo + JB, N) feeds X and P S^dag of every column
        const int jlo = j0 + jj0;
        const bool full = (jj0 + JB <= jn);
        const int i_band_end = min(N, jlo + JB);
        if (full) {
          for (int i = 0; i < jlo; ++i) {
            cpx<real> ca[JB], cb[JB];
#pragma unroll
            for (int u = 0; u < JB; ++u) {
              ca[u] = sA[i * JT + jj0 + u];
              cb[u] = sB[i * JT + jj0 + u];
            }
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) {
              const cpx<real> wi = TR::get(w[rr] + i);
              const cpx<real> pi = TR::get(p[rr] + i);
#pragma unroll
              for (int u = 0; u < JB; ++u) {
                cmac<C>(q[rr][u], wi, ca[u]);
                cmac<C>(x[rr][u], pi, cb[u]);
              }
            }
          }
          for (int i = jlo; i < i_band_end; ++i) {
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) {
              const cpx<real> wi = TR::get(w[rr] + i);
              const cpx<real> pi = TR::get(p[rr] + i);
#pragma unroll
              for (int u = 0; u < JB; ++u) {
                const int j = jlo + u;
                if (i <= j) cmac<C>(q[rr][u], wi, sA[i * JT + jj0 + u]);
                cmac<C>(x[rr][u], pi, sB[i * JT + jj0 + u]);
                if (!keepP && i >= j) cmac<C>(pn[rr][u], pi, sC[i * JT + jj0 + u]);
              }
            }
          }
          if (!keepP) {
            for (int i = i_band_end; i < N; ++i) {
              cpx<real> cb[JB], cc[JB];
#pragma unroll
              for (int u = 0; u < JB; ++u) {
                cb[u] = sB[i * JT + jj0 + u];
                cc[u] = sC[i * JT + jj0 + u];
              }
#pragma unroll
              for (int rr = 0; rr < RT; ++rr) {
                const cpx<real> pi = TR::get(p[rr] + i);
#pragma unroll
                for (int u = 0; u < JB; ++u) {
                  cmac<C>(x[rr][u], pi, cb[u]);
                  cmac<C>(pn[rr][u], pi, cc[u]);
                }
              }
            }
          } else {
            for (int i = i_band_end; i < N; ++i) {
              cpx<real> cb[JB];
#pragma unroll
              for (int u = 0; u < JB; ++u) cb[u] = sB[i * JT + jj0 + u];
#pragma unroll
              for (int rr = 0; rr < RT; ++rr) {
                const cpx<real> pi = TR::get(p[rr] + i);
#pragma unroll
                for (int u = 0; u < JB; ++u) cmac<C>(x[rr][u], pi, cb[u]);
              }
            }
          }
        } else {  // ragged last group
          for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) {
              const cpx<real> wi = TR::get(w[rr] + i);
              const cpx<real> pi = TR::get(p[rr] + i);
#pragma unroll
              for (int u = 0; u < JB; ++u) {
                const int jj = jj0 + u;
                if (jj < jn) {
                  const int j = j0 + jj;
                  if (i <= j) cmac<C>(q[rr][u], wi, sA[i * JT + jj]);
                  cmac<C>(x[rr][u], pi, sB[i * JT + jj]);
                  if (!keepP && i >= j) cmac<C>(pn[rr][u], pi, sC[i * JT + jj]);
                }
              }
            }
          }
        }
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) {
          const int row = row0 + rr;
          if (row >= nrows) continue;
          const long long gbase = base + (long long)row * N + j0;
#pragma unroll
          for (int u = 0; u < JB; ++u) {
            const int jj = jj0 + u;
            if (jj < jn) {
              const long long gi = gbase + jj;
              cpx<real> qn = cfin<C>(q[rr][u]);
              cpx<real> xs = cfin<C>(x[rr][u]);
              // the old X: from the prefetched tile with DB (plain shared read)
              cpx<typename CX::acc> xa = cacc_from<CX>(
                  DB && XSTAGE ? XS::load_nc(sX + (long long)row * N + j0 + jj) : XS::load_nc(X + gi));
              CX::add(xa.re, conv<CX, C>::f(xs.re));
              CX::add(xa.im, conv<CX, C>::f(xs.im));
              XS::store(X + gi, cfin<CX>(xa));
              SS::store(Q + gi, qn);
              if (!keepP) {
                // P = Q + P S^dag
                cpx<acc> pf = pn[rr][u];
                C::add(pf.re, qn.re);
                C::add(pf.im, qn.im);
                SS::store(P + gi, cfin<C>(pf));
              }
            }
          }
        }
      }
    }
  }
}

template <class SS, class XS, int RT, bool XSTAGE>
static cudaError_t launch_bcg_update_rt(void* Q, void* P, void* X, const double2* Sinv,
                                        const double2* BC, const double2* SH, int N, int Vh,
                                        Gate gate, int tile, cudaStream_t s) {
  using real = typename SS::comp::real;
  // double-float: 2 output columns per thread keep the accumulators within the
  // register budget of four resident blocks (no spills); other kinds use 4
  constexpr int JB = (std::is_same<SS, StoreDF>::value || std::is_same<SS, StoreF64>::value) ? 2 : 4;
  // all kinds but double-float (ALU-bound, and its shared memory is spent on
  // 4 resident blocks): double-buffered tiles (W, P, X) filled by cp.async
  constexpr bool DB = !std::is_same<SS, StoreDF>::value;
  const size_t cb = sizeof(cpx<real>), xb = sizeof(typename XS::elem);
  const size_t tb = DB ? sizeof(typename SS::elem) : cb;  // tile element bytes
  // coefficient columns staged per chunk: all N when the three N x N
  // matrices fit 64 KB (then once per CTA, not once per tile), else 32 or 16
  int JT = N;
  while (JT > 16 && 3ull * N * JT * cb > 64 * 1024) JT = JT > 32 ? 32 : 16;
  if (JT < N && JT < 16) JT = 16;
  const size_t coef = 3ull * N * JT * cb;
  auto tile_bytes = [&](int ts) {
    size_t one = upd_wp_bytes(ts, N, tb) + (DB && XSTAGE ? (size_t)ts * 3 * N * xb : 0);
    return (DB ? 2 : 1) * one;
  };
  int TS = 32;
  if (tile > 0) {
    TS = tile;  // the tuner's choice (sites per tile)
    while (TS > 1 && coef + tile_bytes(TS) > 200 * 1024) TS >>= 1;
  } else {
    const size_t budget = (N <= 16 ? 56 * 1024 : 96 * 1024) + coef;
    while (TS > 1 && coef + tile_bytes(TS) > budget) TS >>= 1;
  }
  const size_t sm = coef + tile_bytes(TS);
  cudaFuncSetAttribute(k_bcg_update<SS, XS, JB, DB, RT, XSTAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  // a block size that divides a tile's (row, column group) work units, so no
  // pass over a tile runs with part of the block idle
  const int jt = JT < N ? JT : N;
  const int units = ((TS * 3 + RT - 1) / RT) * ((jt + JB - 1) / JB);
  int threads = 256;
  if (units <= 256) {
    threads = (units + 31) / 32 * 32;
  } else {
    for (int th = 256; th >= 64; th -= 32)
      if (units % th == 0) {
        threads = th;
        break;
      }
  }
  // a persistent grid of exactly the resident blocks (no partial last wave)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcg_update<SS, XS, JB, DB, RT, XSTAGE>, threads,
                                                    sm) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  unsigned blocks = gcap(Vh, TS, num_sms() * per_sm);
  k_bcg_update<SS, XS, JB, DB, RT, XSTAGE><<<blocks, threads, sm, s>>>(
      (typename SS::elem*)Q, (typename SS::elem*)P, (typename XS::elem*)X, Sinv, BC, SH, N, Vh, TS,
      JT, gate);
  return cudaGetLastError();
}

// tile = sites per tile (bits 0..5, 0 = default) + UPD_TWO_ROWS: two rows per
// thread (FP32-arithmetic kinds; shared-memory reads bound a one-row thread
// at large N, but the larger thread footprint can cost occupancy, so the
// tuner decides) + UPD_X_GLOBAL: the old X read from global memory rather
// than staged (FP32-arithmetic kinds)
template <class SS, class XS>
static cudaError_t launch_bcg_update(void* Q, void* P, void* X, const double2* Sinv,
                                     const double2* BC, const double2* SH, int N, int Vh,
                                     Gate gate, int tile, cudaStream_t s) {
  const int ts = tile & (UPD_TWO_ROWS - 1);
  if constexpr (std::is_same<typename SS::comp::real, float>::value) {
    const bool xg = (tile & UPD_X_GLOBAL) != 0;
    if (tile & UPD_TWO_ROWS)
      return xg ? launch_bcg_update_rt<SS, XS, 2, false>(Q, P, X, Sinv, BC, SH, N, Vh, gate, ts, s)
                : launch_bcg_update_rt<SS, XS, 2, true>(Q, P, X, Sinv, BC, SH, N, Vh, gate, ts, s);
    if (xg) return launch_bcg_update_rt<SS, XS, 1, false>(Q, P, X, Sinv, BC, SH, N, Vh, gate, ts, s);
  }
  return launch_bcg_update_rt<SS, XS, 1, true>(Q, P, X, Sinv, BC, SH, N, Vh, gate, ts, s);
}

cudaError_t bcg_update(FieldKind sk, FieldKind xk, void* Q, void* P, void* X, const double2* Sinv,
                       const double2* BC, const double2* SH, int N, int Vh, Gate gate,
                       cudaStream_t s, int tile) {
  if ((tile & UPD_TC) && bcg_update_tc_supported(sk, xk, N))
    return bcg_update_tc(sk, Q, P, X, Sinv, BC, SH, N, Vh, gate, s);
  tile &= ~UPD_TC;
  if (sk == FK_DF && xk == FK_DF)
    return launch_bcg_update<StoreDF, StoreDF>(Q, P, X, Sinv, BC, SH, N, Vh, gate, tile, s);
  if (sk == FK_F32 && xk == FK_DF)
    return launch_bcg_update<StoreF32, StoreDF>(Q, P, X, Sinv, BC, SH, N, Vh, gate, tile, s);
  if (sk == FK_F64 && xk == FK_F64)
    return launch_bcg_update<StoreF64, StoreF64>(Q, P, X, Sinv, BC, SH, N, Vh, gate, tile, s);
  if (sk == FK_H16 && xk == FK_DF)
    return launch_bcg_update<StoreH16, StoreDF>(Q, P, X, Sinv, BC, SH, N, Vh, gate, tile, s);
  if (sk == FK_BF16 && xk == FK_DF)
    return launch_bcg_update<StoreBF16, StoreDF>(Q, P, X, Sinv, BC, SH, N, Vh, gate, tile, s);
  return cudaErrorInvalidValue;
}

// --------------------------------------------------- restart update ----
// Q = R Cinv (R in the fine kind, Q, P in the sloppy kind); P = Q + P SH or P = Q
template <class RS, class SS>
__global__ void __launch_bounds__(256)
    k_restart_update(const typename RS::elem* __restrict__ R, typename SS::elem* __restrict__ Q,
                     typename SS::elem* __restrict__ P, const double2* __restrict__ Cinv,
                     const double2* __restrict__ SH, int init, int N, int Vh, int TS, int JT,
                     Gate gate) {
  using CR = typename RS::comp;
  using C = typename SS::comp;
  using rreal = typename CR::real;
  using real = typename C::real;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(gate)) return;
  cpx<rreal>* sR = reinterpret_cast<cpx<rreal>*>(smem_raw);
  cpx<rreal>* sA = sR + TS * N * 3;                                 // Cinv chunk (fine)
  cpx<real>* sP = reinterpret_cast<cpx<real>*>(sA + N * JT);       // P tile (sloppy)
  cpx<real>* sC = sP + TS * N * 3;                                  // SH chunk (sloppy)
  const bool one_chunk = JT >= N;  // all coefficients staged once per CTA
  if (one_chunk) {
    stage_coef<CR>(sA, Cinv, N, 0, N, JT);
    if (!init) stage_coef<C>(sC, SH, N, 0, N, JT);
  }
  for (long long tile = blockIdx.x; tile * TS < Vh; tile += gridDim.x) {
    const long long site0 = tile * TS;
    const int ns = (int)min((long long)TS, (long long)Vh - site0);
    const long long base = site0 * N * 3;
    const int nel = ns * N * 3;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
      sR[idx] = RS::load_nc(R + base + idx);
      if (!init) sP[idx] = SS::load_nc(P + base + idx);
    }
    for (int j0 = 0; j0 < N; j0 += JT) {
      const int jn = min(JT, N - j0);
      if (!one_chunk) {
        __syncthreads();
        stage_coef<CR>(sA, Cinv, N, j0, jn, JT);
        if (!init) stage_coef<C>(sC, SH, N, j0, jn, JT);
      }
      __syncthreads();
      const int nrows = ns * 3;
      const int nout = nrows * jn;
      for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int jj = o / nrows;  // column major: uniform triangular bounds per warp
        const int rw = o - jj * nrows;
        const int sidx = rw / 3;
        const int c = rw - sidx * 3;
        const int j = j0 + jj;
        const cpx<rreal>* r = sR + (sidx * 3 + c) * N;
        cpx<typename CR::acc> q = czero<CR>();
        for (int i = 0; i <= j; ++i) cmac<CR>(q, r[i], sA[i * JT + jj]);
        cpx<rreal> qf = cfin<CR>(q);
        cpx<real> qn = {conv<C, CR>::f(qf.re), conv<C, CR>::f(qf.im)};
        const long long gi = base + ((long long)sidx * 3 + c) * N + j;
        SS::store(Q + gi, qn);
        cpx<typename C::acc> pn = cacc_from<C>(qn);
        if (!init) {
          const cpx<real>* p = sP + (sidx * 3 + c) * N;
          for (int i = 0; i < N; ++i) cmac<C>(pn, p[i], sC[i * JT + jj]);
        }
        SS::store(P + gi, cfin<C>(pn));
      }
    }
  }
}

template <class RS, class SS>
static cudaError_t launch_restart(const void* R, void* Q, void* P, const double2* Cinv,
                                  const double2* SH, int init, int N, int Vh, Gate gate,
                                  cudaStream_t s) {
  using rreal = typename RS::comp::real;
  using real = typename SS::comp::real;
  size_t big = sizeof(cpx<rreal>) > sizeof(cpx<real>) ? sizeof(cpx<rreal>) : sizeof(cpx<real>);
  TileCfg t = tile_cfg(N, big, 2, 2);
  size_t sm = ((size_t)t.TS * N * 3 + (size_t)N * t.JT) * sizeof(cpx<rreal>) +
              ((size_t)t.TS * N * 3 + (size_t)N * t.JT) * sizeof(cpx<real>);
  cudaFuncSetAttribute(k_restart_update<RS, SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  k_restart_update<RS, SS><<<gcap(Vh, t.TS, 152 * 4), 256, sm, s>>>(
      (const typename RS::elem*)R, (typename SS::elem*)Q, (typename SS::elem*)P, Cinv, SH, init, N,
      Vh, t.TS, t.JT, gate);
  return cudaGetLastError();
}

cudaError_t restart_update(FieldKind rk, FieldKind sk, const void* R, void* Q, void* P,
                           const double2* Cinv, const double2* SH, int init, int N, int Vh,
                           Gate gate, cudaStream_t s) {
  if (rk == FK_F64 && sk == FK_DF)
    return launch_restart<StoreF64, StoreDF>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_F64 && sk == FK_F32)
    return launch_restart<StoreF64, StoreF32>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_F64 && sk == FK_F64)
    return launch_restart<StoreF64, StoreF64>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_F64 && sk == FK_H16)
    return launch_restart<StoreF64, StoreH16>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_F64 && sk == FK_BF16)
    return launch_restart<StoreF64, StoreBF16>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_DF && sk == FK_DF)
    return launch_restart<StoreDF, StoreDF>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_DF && sk == FK_F32)
    return launch_restart<StoreDF, StoreF32>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_DF && sk == FK_H16)
    return launch_restart<StoreDF, StoreH16>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  if (rk == FK_DF && sk == FK_BF16)
    return launch_restart<StoreDF, StoreBF16>(R, Q, P, Cinv, SH, init, N, Vh, gate, s);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------ accumulate ----
// Y (full precision) += X (iterated update) ; X = 0
template <class YS, class XS>
__global__ void k_accumulate(typename YS::elem* __restrict__ Y, typename XS::elem* __restrict__ X,
                             long long n, Gate gate) {
  using CY = typename YS::comp;
  using CX = typename XS::comp;
  if (gate_closed(gate)) return;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    cpx<typename CX::real> x = XS::load_nc(X + idx);
    cpx<typename CY::acc> y = cacc_from<CY>(YS::load_nc(Y + idx));
    CY::add(y.re, conv<CY, CX>::f(x.re));
    CY::add(y.im, conv<CY, CX>::f(x.im));
    YS::store(Y + idx, cfin<CY>(y));
    cpx<typename CX::real> z = {CX::rzero(), CX::rzero()};
    XS::store(X + idx, z);
  }
}

// grid of a streaming kernel: reliable-update launches (gated off in most
// iterations) use 2 blocks per SM, others up to 8
static unsigned stream_grid(size_t n, const Gate& gate) {
  return gcap(n, 256, gate_mostly_off(gate) ? 152 * 2 : 152 * 8);
}

cudaError_t accumulate(FieldKind yk, FieldKind xk, void* Y, void* X, size_t n, Gate gate,
                       cudaStream_t s) {
  if (yk == FK_F64 && xk == FK_DF)
    k_accumulate<StoreF64, StoreDF><<<stream_grid(n, gate), 256, 0, s>>>((double2*)Y, (float4*)X, n, gate);
  else if (yk == FK_F64 && xk == FK_F64)
    k_accumulate<StoreF64, StoreF64><<<stream_grid(n, gate), 256, 0, s>>>((double2*)Y, (double2*)X, n, gate);
  else if (yk == FK_DF && xk == FK_DF)
    k_accumulate<StoreDF, StoreDF><<<stream_grid(n, gate), 256, 0, s>>>((float4*)Y, (float4*)X, n, gate);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------- kind conversion ----
template <class DS, class SS>
__global__ void k_convert(const typename SS::elem* __restrict__ in, typename DS::elem* __restrict__ out,
                          long long n, const double* __restrict__ scale, Gate gate) {
  if (gate_closed(gate)) return;
  const double f = scale ? *scale : 1.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    double2 v = SS::to_double2(in[idx]);
    v.x *= f;
    v.y *= f;
    out[idx] = DS::from_double2(v);
  }
}

cudaError_t convert_field(FieldKind from, FieldKind to, const void* in, void* out, size_t n,
                          const double* scale, Gate gate, cudaStream_t s) {
  if (from == FK_F64 && to == FK_DF)
    k_convert<StoreDF, StoreF64><<<stream_grid(n, gate), 256, 0, s>>>((const double2*)in, (float4*)out, n, scale, gate);
  else if (from == FK_F64 && to == FK_F32)
    k_convert<StoreF32, StoreF64><<<stream_grid(n, gate), 256, 0, s>>>((const double2*)in, (float2*)out, n, scale, gate);
  else if (from == FK_F64 && to == FK_H16)
    k_convert<StoreH16, StoreF64><<<stream_grid(n, gate), 256, 0, s>>>((const double2*)in, (__half2*)out, n, scale, gate);
  else if (from == FK_F64 && to == FK_BF16)
    k_convert<StoreBF16, StoreF64><<<stream_grid(n, gate), 256, 0, s>>>((const double2*)in, (__nv_bfloat162*)out, n, scale, gate);
  else if (from == FK_F64 && to == FK_F64)
    k_convert<StoreF64, StoreF64><<<stream_grid(n, gate), 256, 0, s>>>((const double2*)in, (double2*)out, n, scale, gate);
  else if (from == FK_DF && to == FK_F64)
    k_convert<StoreF64, StoreDF><<<stream_grid(n, gate), 256, 0, s>>>((const float4*)in, (double2*)out, n, scale, gate);
  else if (from == to && !scale)
    return cudaMemcpyAsync(out, in, n * elem_bytes(to), cudaMemcpyDeviceToDevice, s);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------- generic block caxpy / trmul ----
// mode 0: Y += X a ; mode 1: Y = X a with a upper triangular
template <class S>
__global__ void __launch_bounds__(256)
    k_block_mul(const typename S::elem* __restrict__ X, const double2* __restrict__ a,
                typename S::elem* __restrict__ Y, int N, int Vh, int TS, int JT, int mode) {
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<real>* sX = reinterpret_cast<cpx<real>*>(smem_raw);
  cpx<real>* sA = sX + TS * N * 3;
  const long long site0 = (long long)blockIdx.x * TS;
  const int ns = (int)min((long long)TS, (long long)Vh - site0);
  const long long base = site0 * N * 3;
  for (int idx = threadIdx.x; idx < ns * N * 3; idx += blockDim.x) sX[idx] = S::load_nc(X + base + idx);
  for (int j0 = 0; j0 < N; j0 += JT) {
    const int jn = min(JT, N - j0);
    __syncthreads();
    stage_coef<C>(sA, a, N, j0, jn, JT);
    __syncthreads();
    const int nrows = ns * 3;
    for (int o = threadIdx.x; o < nrows * jn; o += blockDim.x) {
      const int jj = o / nrows;  // column major: uniform triangular bounds per warp
      const int rw = o - jj * nrows;
      const int sidx = rw / 3;
      const int c = rw - sidx * 3;
      const int j = j0 + jj;
      const long long gi = base + ((long long)sidx * 3 + c) * N + j;
      const cpx<real>* x = sX + (sidx * 3 + c) * N;
      cpx<acc> y = (mode == 0) ? cacc_from<C>(S::load_nc(Y + gi)) : czero<C>();
      const int iend = (mode == 1) ? j + 1 : N;
      for (int i = 0; i < iend; ++i) cmac<C>(y, x[i], sA[i * JT + jj]);
      S::store(Y + gi, cfin<C>(y));
    }
  }
}

template <class S>
static cudaError_t launch_block_mul(const void* X, const double2* a, void* Y, int N, int Vh,
                                    int mode, cudaStream_t s) {
  using real = typename S::comp::real;
  TileCfg t = tile_cfg(N, sizeof(cpx<real>), 1, 1);
  size_t sm = ((size_t)t.TS * N * 3 + (size_t)N * t.JT) * sizeof(cpx<real>);
  cudaFuncSetAttribute(k_block_mul<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_block_mul<S><<<nblk(Vh, t.TS), 256, sm, s>>>((const typename S::elem*)X, a,
                                                 (typename S::elem*)Y, N, Vh, t.TS, t.JT, mode);
  return cudaGetLastError();
}

cudaError_t block_caxpy(FieldKind k, const void* X, const double2* a, void* Y, int N, int Vh,
                        cudaStream_t s) {
  switch (k) {
    case FK_DF: return launch_block_mul<StoreDF>(X, a, Y, N, Vh, 0, s);
    case FK_F32: return launch_block_mul<StoreF32>(X, a, Y, N, Vh, 0, s);
    case FK_H16: return launch_block_mul<StoreH16>(X, a, Y, N, Vh, 0, s);
    case FK_BF16: return launch_block_mul<StoreBF16>(X, a, Y, N, Vh, 0, s);
    default: return launch_block_mul<StoreF64>(X, a, Y, N, Vh, 0, s);
  }
}

cudaError_t block_trmul(FieldKind k, const void* M, const double2* Rinv, void* Q, int N, int Vh,
                        cudaStream_t s) {
  switch (k) {
    case FK_DF: return launch_block_mul<StoreDF>(M, Rinv, Q, N, Vh, 1, s);
    case FK_F32: return launch_block_mul<StoreF32>(M, Rinv, Q, N, Vh, 1, s);
    case FK_H16: return launch_block_mul<StoreH16>(M, Rinv, Q, N, Vh, 1, s);
    case FK_BF16: return launch_block_mul<StoreBF16>(M, Rinv, Q, N, Vh, 1, s);
    default: return launch_block_mul<StoreF64>(M, Rinv, Q, N, Vh, 1, s);
  }
}

// ---------------------------------------------------------- CG, N = 1 ----
// x += alpha p ; r -= alpha Ap ; per-CTA partial of |r|^2
// (x in the update kind, r, p, Ap in the iteration's kind)
template <class S, class XS>
__global__ void __launch_bounds__(256)
    k_cg_axpy_norm(typename XS::elem* __restrict__ x, typename S::elem* __restrict__ r,
                   const typename S::elem* __restrict__ p, const typename S::elem* __restrict__ Ap,
                   const double* __restrict__ alpha_p, const double* __restrict__ alpha_x,
                   double2* __restrict__ partials, long long n, Gate gate) {
  using C = typename S::comp;
  using CX = typename XS::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  __shared__ double red[256];
  if (gate_closed(gate)) return;
  const typename CX::real alphax = CX::from_double(*alpha_x);
  const real nalpha = C::from_double(-*alpha_p);
  acc nrm = C::zero();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cpx<real> pv = S::load(p + i);
    cpx<real> av = S::load(Ap + i);
    cpx<typename CX::acc> xv = cacc_from<CX>(XS::load_nc(x + i));
    cpx<acc> rv = cacc_from<C>(S::load_nc(r + i));
    CX::mac(xv.re, alphax, conv<CX, C>::f(pv.re));
    CX::mac(xv.im, alphax, conv<CX, C>::f(pv.im));
    C::mac(rv.re, nalpha, av.re);
    C::mac(rv.im, nalpha, av.im);
    XS::store(x + i, cfin<CX>(xv));
    cpx<real> rf = cfin<C>(rv);
    S::store(r + i, rf);
    C::mac(nrm, rf.re, rf.re);
    C::mac(nrm, rf.im, rf.im);
  }
  red[threadIdx.x] = C::to_double(nrm);
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(red[0], 0.0);
}

template <class S>
__global__ void k_cg_xpay(typename S::elem* __restrict__ p, const typename S::elem* __restrict__ r,
                          const double* __restrict__ beta_p, long long n, Gate gate) {
  using C = typename S::comp;
  using real = typename C::real;
  if (gate_closed(gate)) return;
  const real beta = C::from_double(*beta_p);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cpx<typename C::acc> v = cacc_from<C>(S::load(r + i));
    cpx<real> pv = S::load_nc(p + i);
    C::mac(v.re, beta, pv.re);
    C::mac(v.im, beta, pv.im);
    S::store(p + i, cfin<C>(v));
  }
}

cudaError_t cg_axpy_norm(FieldKind k, FieldKind xk, void* x, void* r, const void* p,
                         const void* Ap, const double* alpha, const double* alpha_x,
                         double2* partials, int nblocks, int Vh, Gate gate, cudaStream_t s) {
  long long n = 3LL * Vh;
  if (k == FK_DF && xk == FK_DF)
    k_cg_axpy_norm<StoreDF, StoreDF><<<nblocks, 256, 0, s>>>(
        (float4*)x, (float4*)r, (const float4*)p, (const float4*)Ap, alpha, alpha_x, partials, n, gate);
  else if (k == FK_F32 && xk == FK_DF)
    k_cg_axpy_norm<StoreF32, StoreDF><<<nblocks, 256, 0, s>>>(
        (float4*)x, (float2*)r, (const float2*)p, (const float2*)Ap, alpha, alpha_x, partials, n, gate);
  else if (k == FK_H16 && xk == FK_DF)
    k_cg_axpy_norm<StoreH16, StoreDF><<<nblocks, 256, 0, s>>>(
        (float4*)x, (__half2*)r, (const __half2*)p, (const __half2*)Ap, alpha, alpha_x, partials, n, gate);
  else if (k == FK_BF16 && xk == FK_DF)
    k_cg_axpy_norm<StoreBF16, StoreDF><<<nblocks, 256, 0, s>>>(
        (float4*)x, (__nv_bfloat162*)r, (const __nv_bfloat162*)p, (const __nv_bfloat162*)Ap, alpha, alpha_x,
        partials, n, gate);
  else if (k == FK_F64 && xk == FK_F64)
    k_cg_axpy_norm<StoreF64, StoreF64><<<nblocks, 256, 0, s>>>(
        (double2*)x, (double2*)r, (const double2*)p, (const double2*)Ap, alpha, alpha_x, partials, n, gate);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t cg_xpay(FieldKind k, void* p, const void* r, const double* beta, int Vh, Gate gate,
                    cudaStream_t s) {
  long long n = 3LL * Vh;
  switch (k) {
    case FK_DF:
      k_cg_xpay<StoreDF><<<gcap(n, 256), 256, 0, s>>>((float4*)p, (const float4*)r, beta, n, gate);
      break;
    case FK_F32:
      k_cg_xpay<StoreF32><<<gcap(n, 256), 256, 0, s>>>((float2*)p, (const float2*)r, beta, n, gate);
      break;
    case FK_F64:
      k_cg_xpay<StoreF64><<<gcap(n, 256), 256, 0, s>>>((double2*)p, (const double2*)r, beta, n, gate);
      break;
    case FK_H16:
      k_cg_xpay<StoreH16><<<gcap(n, 256), 256, 0, s>>>((__half2*)p, (const __half2*)r, beta, n, gate);
      break;
    case FK_BF16:
      k_cg_xpay<StoreBF16><<<gcap(n, 256), 256, 0, s>>>((__nv_bfloat162*)p, (const __nv_bfloat162*)r, beta, n, gate);
      break;
  }
  return cudaGetLastError();
}

}  // namespace bcg
