// Stencil kernels and their launch helpers, included once per storage kind
// by stencil_<kind>.cu so that the kinds compile in parallel: the block
// stencil of Sec. 6.2 (the hopping term of Eq. 2 applied to N right-hand
// sides with every link loaded once per site), in three variants (plain,
// per-thread cp.async prefetch, bulk-copy pipelined) and with the fused
// epilogues of the normal operator (Sec. 3.2).
#pragma once
#include <type_traits>

#include "internal.h"
#include "tma.cuh"

namespace bcg {

static constexpr int LINK_W = 32;  // sites per link block

// streaming multiprocessors of the current device (looked up once)
static int stencil_sms() {
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

// number of link blocks per parity (the last one may be partly used)
__host__ __device__ inline long long link_blocks(const Geom& g) {
  return ((long long)g.Vh + LINK_W - 1) / LINK_W;
}

// element offset of (parity p, site cb, hop 0, element 0); E elements per
// hop matrix (9, or 6 for two-row storage)
__host__ __device__ __forceinline__ long long link_offset(const Geom& g, int p, int cb, int E = 9) {
  return ((long long)p * link_blocks(g) + cb / LINK_W) * (16 * E * LINK_W) + (cb % LINK_W);
}

// third row of a hop matrix stored as two rows: conj(row0 x row1) times the
// inverse of the matrix's real scale (see Geom)
template <class R>
__device__ __forceinline__ void rebuild_row2(cpx<R>* U, R inv) {
  auto cmulsub = [](cpx<R> a, cpx<R> b, cpx<R> c, cpx<R> d) {  // a b - c d
    return cpx<R>{a.re * b.re - a.im * b.im - (c.re * d.re - c.im * d.im),
                  a.re * b.im + a.im * b.re - (c.re * d.im + c.im * d.re)};
  };
  const cpx<R> w0 = cmulsub(U[1], U[5], U[2], U[4]);
  const cpx<R> w1 = cmulsub(U[2], U[3], U[0], U[5]);
  const cpx<R> w2 = cmulsub(U[0], U[4], U[1], U[3]);
  U[6] = cpx<R>{w0.re * inv, -w0.im * inv};
  U[7] = cpx<R>{w1.re * inv, -w1.im * inv};
  U[8] = cpx<R>{w2.re * inv, -w2.im * inv};
}

// One thread: output site `site`, vector slots j = k, k + T, ... (< N / V) of
// its right-hand sides, each slot V consecutive right-hand sides read with
// one load (V = 2: one 128-bit load of two FP32 complex numbers).  RV slots
// per thread, so R = RV * V right-hand sides share each link load.
template <class S, int V>
struct VecLoad;
template <class S>
struct VecLoad<S, 1> {
  static __device__ __forceinline__ void get(const typename S::elem* p,
                                             cpx<typename S::comp::real>* v) {
    v[0] = S::load_raw(p);
  }
};
template <>
struct VecLoad<StoreF32, 2> {
  static __device__ __forceinline__ void get(const float2* p, cpx<float>* v) {
    StoreF32::load2(p, v[0], v[1]);
  }
};
// 16-bit kinds: 2 complex numbers per 64-bit load, 4 per 128-bit load
template <class S>
struct VecLoad16 {
  template <int V>
  static __device__ __forceinline__ void get(const typename S::elem* p, cpx<float>* v) {
    if (V == 4) {
      uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
      const typename S::elem* e = reinterpret_cast<const typename S::elem*>(&u);
      v[0] = S::cvt_raw(e[0]);
      v[1] = S::cvt_raw(e[1]);
      v[2] = S::cvt_raw(e[2]);
      v[3] = S::cvt_raw(e[3]);
    } else {
      uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      const typename S::elem* e = reinterpret_cast<const typename S::elem*>(&u);
      v[0] = S::cvt_raw(e[0]);
      v[1] = S::cvt_raw(e[1]);
    }
  }
};
template <>
struct VecLoad<StoreH16, 2> {
  static __device__ __forceinline__ void get(const __half2* p, cpx<float>* v) {
    VecLoad16<StoreH16>::get<2>(p, v);
  }
};
template <>
struct VecLoad<StoreH16, 4> {
  static __device__ __forceinline__ void get(const __half2* p, cpx<float>* v) {
    VecLoad16<StoreH16>::get<4>(p, v);
  }
};
template <>
struct VecLoad<StoreBF16, 2> {
  static __device__ __forceinline__ void get(const __nv_bfloat162* p, cpx<float>* v) {
    VecLoad16<StoreBF16>::get<2>(p, v);
  }
};
template <>
struct VecLoad<StoreBF16, 4> {
  static __device__ __forceinline__ void get(const __nv_bfloat162* p, cpx<float>* v) {
    VecLoad16<StoreBF16>::get<4>(p, v);
  }
};

#ifndef BCG_DSLASH_TPB
#define BCG_DSLASH_TPB 128
#endif

// Resident blocks per SM requested from the compiler for the plain kernel,
// and hop unrolling: the FP32 kernel is latency-bound on its gathers;
// capping it at six 128-thread blocks per SM (at most 85 registers a thread)
// without hop unrolling raised its HBM fraction at 32^4 from 0.30 to 0.34
// (N = 16) and from 0.44 to 0.51 (N = 8) with four right-hand sides per
// thread, and no unrolling alone from 0.27 to 0.30 (N = 16) with eight; the
// other kinds showed no gain and keep the compiler's choice.
template <class S, int RV>
struct PlainBounds {
  static constexpr int minb = 1;
  static constexpr int unroll = 1;  // hops unrolled per direction
};
template <int RV>
struct PlainBounds<StoreF32, RV> {
  static constexpr int minb = RV == 2 ? 6 : 1;      // R = 4 (two 128-bit slots)
  static constexpr int unroll = RV >= 2 ? 0 : 1;    // R = 8 also gains without unrolling
};

// The hop loops multiply raw loads (StoreH16 keeps 2^4 x value): remove the
// factor RAW_SCALE^2 from an output accumulator once (exact, a power of two)
template <class S, class A>
__device__ __forceinline__ void unscale_raw(cpx<A>& v) {
  if constexpr (S::RAW_SCALE != 1.f) {
    constexpr float k = 1.f / (S::RAW_SCALE * S::RAW_SCALE);
    v.re *= k;
    v.im *= k;
  }
}

template <class S, int RV, int V, int EPI, int UNROLL_HOPS, bool RC = false>
__global__ void __launch_bounds__(BCG_DSLASH_TPB, (PlainBounds<S, RV>::minb))
    k_dslash(const typename S::elem* __restrict__ links, const typename S::elem* __restrict__ in,
             typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
             const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity, int N,
             int T, long long span, Gate gate) {
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  if (gate_closed(gate)) return;
  const int NS = N / V;
  const long long total = (long long)g.Vh * T;
  const real m2 = C::from_double(m2d);
  // span = 0: grid-stride over (site, slot) pairs; span > 0: this block walks
  // the contiguous range [blockIdx.x * span, (blockIdx.x + 1) * span) in order,
  // so that the neighbours a block reads in y (and partly z) were loaded by
  // the same block shortly before and can still be in its SM's L1
  const long long g0 = span ? (long long)blockIdx.x * span : (long long)blockIdx.x * blockDim.x;
  const long long gend = span ? min(total, g0 + span) : total;
  const long long gstep = span ? (long long)blockDim.x : (long long)gridDim.x * blockDim.x;
  for (long long gid = g0 + threadIdx.x; gid < gend; gid += gstep) {
    const int site = (int)(gid / T);
    const int k = (int)(gid - (long long)site * T);
    int x, y, z, t;
    site_xyzt(g, site, parity, x, y, z, t);
    const int lex = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
    const int nr = (NS - k + T - 1) / T;  // slots k + r*T < NS

    cpx<acc> a[RV][V][3];
#pragma unroll
    for (int r = 0; r < RV; ++r)
#pragma unroll
      for (int w = 0; w < V; ++w)
#pragma unroll
        for (int i = 0; i < 3; ++i) a[r][w][i] = czero<C>();

    constexpr int LE = RC ? 6 : 9;  // stored elements per hop matrix
    const typename S::elem* lp = links + link_offset(g, parity, site, LE);
    // operands of hop d: the hop matrix and this thread's neighbour slots
    auto fetch = [&](int d, cpx<real>* U, cpx<real> (*v)[3][V]) {
      const int mu = d >> 2, kk = hop_k(d & 3);
      const int nb = neighbour_cb_s(g, lex, x, y, z, t, mu, kk);
#pragma unroll
      for (int e = 0; e < LE; ++e) U[e] = S::load_raw(lp + (d * LE + e) * LINK_W);
      if constexpr (RC) {
        // sign of the stored matrix's scale: staggered phase, boundary, backward hop
        const int ps = mu == 0 ? 0 : mu == 1 ? x : mu == 2 ? x + y : x + y + z;
        int sg = (ps & 1) ? -1 : 1;
        if (kk < 0) sg = -sg;
        if (g.antiperiodic && mu == 3 && (t + kk < 0 || t + kk >= g.L[3])) sg = -sg;
        const real inv = (real)sg * (real)g.inv_c[(d & 2) ? 1 : 0];
        // rows 0 and 1 were loaded raw (times RAW_SCALE): keep row 2 raw too
        rebuild_row2<real>(U, inv / (real)S::RAW_SCALE);
      }
      const typename S::elem* ip = in + (long long)nb * N * 3 + k * V;
#pragma unroll
      for (int r = 0; r < RV; ++r)
        if (r < nr)
#pragma unroll
          for (int b = 0; b < 3; ++b) VecLoad<S, V>::get(ip + b * N + r * T * V, v[r][b]);
    };
    auto apply = [&](const cpx<real>* U, const cpx<real> (*v)[3][V]) {
#pragma unroll
      for (int r = 0; r < RV; ++r) {
        if (r < nr) {
#pragma unroll
          for (int w = 0; w < V; ++w)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              cmac<C>(a[r][w][i], U[i * 3 + 0], v[r][0][w]);
              cmac<C>(a[r][w][i], U[i * 3 + 1], v[r][1][w]);
              cmac<C>(a[r][w][i], U[i * 3 + 2], v[r][2][w]);
            }
        }
      }
    };
    auto hop = [&](int d) {
      cpx<real> U[9];
      cpx<real> v[RV][3][V];
      fetch(d, U, v);
      apply(U, v);
    };
    if (UNROLL_HOPS == 2) {
#pragma unroll
      for (int d = 0; d < 16; ++d) hop(d);
    } else if (UNROLL_HOPS == 1) {
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int q = 0; q < 4; ++q) hop(mu * 4 + q);
      }
    } else {
#pragma unroll 1
      for (int d = 0; d < 16; ++d) hop(d);
    }
    const long long ob = (long long)site * N * 3 + k * V;
#pragma unroll
    for (int r = 0; r < RV; ++r) {
      if (r < nr) {
#pragma unroll
        for (int w = 0; w < V; ++w)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const long long oi = ob + i * N + r * T * V + w;
            cpx<acc> v = a[r][w][i];
            unscale_raw<S>(v);
            if (EPI != EPI_NONE) {
              // m2 * c1 - D in
              C::neg(v.re);
              C::neg(v.im);
              cpx<real> cc = S::load(c1 + oi);
              C::mac(v.re, m2, cc.re);
              C::mac(v.im, m2, cc.im);
              if (EPI == EPI_RESIDUAL) {  // c2 - (m2 c1 - D in)
                C::neg(v.re);
                C::neg(v.im);
                cpx<real> bb = S::load(c2 + oi);
                C::add(v.re, bb.re);
                C::add(v.im, bb.im);
              }
            }
            S::store(out + oi, cfin<C>(v));
          }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Bulk-copy pipelined stencil (producer / consumer).  A CTA owns link blocks
// of LINK_W = 32 consecutive output sites: T consumer warps (T threads per
// site, R = RV * V right-hand sides each) and one producer warp.  Its work is
// the stream of (block, hop) tasks.  For each task the producer waits until
// the consumers have released the task's stage (empty mbarrier, one arrival
// per consumer warp), posts the expected bytes on the stage's full mbarrier
// and copies the hop's 9 x 32 link words (one cp.async.bulk) and the 32
// neighbour spinor rows, one bulk copy per run of consecutive rows: for hops
// in y, z and t the rows of 32 consecutive sites are consecutive unless the
// hop wraps, and for x hops they form at most a few runs.  The rows land
// unpadded (3N elements each, slot = site); a consumer thread visits its
// right-hand-side slots in an order rotated by its site, so that the 8 lanes
// of a quarter-warp (two or more sites) read different banks.  Consumers
// wait on full, multiply from shared memory, release the stage and
// accumulate in registers; after hop 15 they write their outputs.  No CTA
// barrier inside the pipeline.
//
// Every wait is bounded by a watchdog deadline: Geom::wait_ns (default 4 s)
// after the CTA started.  Once it has passed, the CTA records
// BLOCKCG_ERR_TIMEOUT in the status word and, before it returns, waits for
// the last issued phase of every stage (at most one phase per stage can be
// outstanding: the producer refills a stage only after the consumers saw its
// previous copies land), so that no bulk copy is still writing into its
// shared memory when it exits.  That drain has its own limit of
// TMA_DRAIN_LIMIT (copies of a few KB land in microseconds; the limit only
// keeps a broken copy from hanging the kernel).
static constexpr uint64_t TMA_WAIT_LIMIT = 4000000000ull;   // 4 s of wall-clock time
static constexpr uint64_t TMA_DRAIN_LIMIT = 4000000000ull;  // 4 s
static constexpr int TMA_MAX_T = 8;                         // consumer warps per CTA

template <class S, int RV, int V, int EPI, int STAGES>
__global__ void __launch_bounds__((TMA_MAX_T + 1) * 32)
    k_dslash_tma(const typename S::elem* __restrict__ links, const typename S::elem* __restrict__ in,
                 typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
                 const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity, int N,
                 int T, Gate gate, SolverStatus* errst) {
  using E = typename S::elem;
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ __align__(8) uint64_t empty[STAGES];
  __shared__ int abort_flag;
  __shared__ long long sh_issued;
  if (gate_closed(gate)) return;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int nconsumer = T * LINK_W;
  const bool producer = tid >= nconsumer;
  const int NS = N / V;
  const int row = 3 * N;  // elements per spinor row (one site, all right-hand sides)
  const int link_elems = 9 * LINK_W;
  const int stage_elems = link_elems + LINK_W * row;
  E* sbase = reinterpret_cast<E*>(smem_raw);
  const long long units = link_blocks(g);
  const long long my_units =
      units > (long long)blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long ntasks = my_units * 16;
  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], T);
    }
    abort_flag = 0;
    sh_issued = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const uint64_t deadline =
      global_ns() + (g.wait_ns ? (uint64_t)g.wait_ns : TMA_WAIT_LIMIT);
  const uint32_t row_bytes = (uint32_t)(row * sizeof(E));

  if (producer) {
    long long q = 0;
    for (; q < ntasks; ++q) {
      const int st = (int)(q % STAGES);
      if (q >= STAGES) {
        int ok = 1;
        if (lane == 0)
          ok = mbar_wait_until(&empty[st], (uint32_t)(((q / STAGES) - 1) & 1), deadline) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok || *(volatile int*)&abort_flag) {
          if (lane == 0) abort_flag = 1;
          break;
        }
      }
      const long long unit = blockIdx.x + (q >> 4) * (long long)gridDim.x;
      const int d = (int)(q & 15);
      E* base = sbase + (size_t)st * stage_elems;
      const long long site0 = unit * LINK_W;
      const int nvalid = (int)min((long long)LINK_W, (long long)g.Vh - site0);
      int nb = 0;
      if (lane < nvalid) {
        int x, y, z, t;
        site_xyzt(g, (int)site0 + lane, parity, x, y, z, t);
        const int lex = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
        nb = neighbour_cb_s(g, lex, x, y, z, t, d >> 2, hop_k(d & 3));
      }
      const int prev = __shfl_up_sync(0xffffffffu, nb, 1);
      const bool start = lane < nvalid && (lane == 0 || nb != prev + 1);
      const unsigned m = __ballot_sync(0xffffffffu, start);
      if (lane == 0)
        mbar_arrive_expect_tx(&full[st], (uint32_t)(link_elems * sizeof(E)) + nvalid * row_bytes);
      __syncwarp();
      if (lane == 0)
        bulk_g2s(base, links + link_offset(g, parity, (int)site0) + d * 9 * LINK_W,
                 (uint32_t)(link_elems * sizeof(E)), &full[st]);
      if (start) {
        const unsigned higher = m & ~((2u << lane) - 1u);
        const int next = higher ? __ffs(higher) - 1 : nvalid;
        bulk_g2s(base + link_elems + lane * row, in + (long long)nb * row,
                 (uint32_t)(next - lane) * row_bytes, &full[st]);
      }
    }
    if (lane == 0) sh_issued = q;
  } else {
    const int warp = tid >> 5;
    (void)warp;
    const int sl = tid / T;  // local site
    const int k = tid - sl * T;
    const int nr = (NS - k + T - 1) / T;  // valid slots: slot index < nr
    const real m2 = C::from_double(m2d);
    cpx<acc> a[RV][V][3];
    for (long long tau = 0; tau < ntasks; ++tau) {
      const int d = (int)(tau & 15);
      const int st = (int)(tau % STAGES);
      if (d == 0) {
#pragma unroll
        for (int r = 0; r < RV; ++r)
#pragma unroll
          for (int w = 0; w < V; ++w)
#pragma unroll
            for (int i = 0; i < 3; ++i) a[r][w][i] = czero<C>();
      }
      const bool ok = mbar_wait_until(&full[st], (uint32_t)((tau / STAGES) & 1), deadline);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      const long long unit = blockIdx.x + (tau >> 4) * (long long)gridDim.x;
      const long long site = unit * LINK_W + sl;
      const bool valid = site < g.Vh;
      const E* base = sbase + (size_t)st * stage_elems;
      if (valid) {
        cpx<real> U[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) U[e] = S::load_nc_raw(base + e * LINK_W + sl);
        const E* ip = base + link_elems + sl * row + k * V;
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          const int sr = (r + sl) & (RV - 1);  // rotated slot: quarter-warp lanes hit distinct banks
          if (sr < nr) {
            cpx<real> v[3][V];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
              for (int w = 0; w < V; ++w) v[b][w] = S::load_nc_raw(ip + b * N + sr * T * V + w);
#pragma unroll
            for (int w = 0; w < V; ++w)
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                cmac<C>(a[r][w][i], U[i * 3 + 0], v[0][w]);
                cmac<C>(a[r][w][i], U[i * 3 + 1], v[1][w]);
                cmac<C>(a[r][w][i], U[i * 3 + 2], v[2][w]);
              }
          }
        }
      }
      // release the stage to the producer (its next copies into it are async-proxy writes)
      fence_proxy_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (d == 15 && valid) {
        const long long ob = site * N * 3 + k * V;
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          const int sr = (r + sl) & (RV - 1);
          if (sr < nr) {
#pragma unroll
            for (int w = 0; w < V; ++w)
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                const long long oi = ob + i * N + sr * T * V + w;
                cpx<acc> vv = a[r][w][i];
                unscale_raw<S>(vv);
                if (EPI != EPI_NONE) {
                  C::neg(vv.re);
                  C::neg(vv.im);
                  cpx<real> cc = S::load(c1 + oi);
                  C::mac(vv.re, m2, cc.re);
                  C::mac(vv.im, m2, cc.im);
                  if (EPI == EPI_RESIDUAL) {
                    C::neg(vv.re);
                    C::neg(vv.im);
                    cpx<real> bb = S::load(c2 + oi);
                    C::add(vv.re, bb.re);
                    C::add(vv.im, bb.im);
                  }
                }
                S::store(out + oi, cfin<C>(vv));
              }
          }
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    // record the failure, then wait for the last issued phase of every stage
    if (tid == 0) {
      if (errst) atomicExch(&errst->error, (int)7 /* BLOCKCG_ERR_TIMEOUT */);
      const long long issued = sh_issued;
      for (long long q = issued - STAGES; q < issued; ++q)
        if (q >= 0)
          mbar_wait_bounded(&full[q % STAGES], (uint32_t)((q / STAGES) & 1), TMA_DRAIN_LIMIT);
    }
    __syncthreads();
  }
}

template <class S, int RV, int V, int EPI, int STAGES>
static bool launch_tma_t(const void* links, const void* in, void* out, const void* c1,
                         const void* c2, double m2, const Geom& g, int parity, int N, Gate gate,
                         SolverStatus* errst, cudaStream_t s) {
  using E = typename S::elem;
  const size_t eb = sizeof(E);
  const int NS = N / V;
  const int T = (NS + RV - 1) / RV;
  if (T > TMA_MAX_T) return false;
  if ((3 * N * eb) % 16) return false;                // rows must be 16-byte multiples
  if (RV & (RV - 1)) return false;                    // slot rotation needs a power of two
  const size_t stage_bytes = (9 * LINK_W + (size_t)LINK_W * 3 * N) * eb;
  const size_t sm = STAGES * stage_bytes;
  if (sm > 200 * 1024) return false;
  auto kern = k_dslash_tma<S, RV, V, EPI, STAGES>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return false;
  const int threads = T * LINK_W + 32;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, sm) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  const long long units = link_blocks(g);
  const long long want = (long long)stencil_sms() * per_sm;
  unsigned blocks = (unsigned)(units < want ? units : want);
  kern<<<blocks, threads, sm, s>>>((const E*)links, (const E*)in, (E*)out, (const E*)c1,
                                   (const E*)c2, m2, g, parity, N, T, gate, errst);
  return true;
}

template <class S, int RV, int V>
static bool launch_tma_r(int epi, const void* links, const void* in, void* out, const void* c1,
                         const void* c2, double m2, const Geom& g, int parity, int N, Gate gate,
                         SolverStatus* errst, cudaStream_t s) {
  // four stages when they fit, else three, else two
  switch (epi) {
    case EPI_NONE:
      return launch_tma_t<S, RV, V, EPI_NONE, 4>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_NONE, 3>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_NONE, 2>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    case EPI_NORMAL:
      return launch_tma_t<S, RV, V, EPI_NORMAL, 4>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_NORMAL, 3>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_NORMAL, 2>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    default:
      return launch_tma_t<S, RV, V, EPI_RESIDUAL, 4>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_RESIDUAL, 3>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_RESIDUAL, 2>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
  }
}

template <class S>
static bool launch_tma_s(int R, int epi, const void* links, const void* in, void* out,
                     const void* c1, const void* c2, double m2, const Geom& g, int parity,
                     int N, Gate gate, SolverStatus* errst, cudaStream_t s) {
  // vector width V: complex numbers per load (FP32: 2 per 128 bits; 16-bit
  // kinds: 4 per 128 bits or 2 per 64 bits); RV = R / V slots per thread
  constexpr bool F32 = std::is_same<S, StoreF32>::value;
  constexpr bool H = std::is_same<S, StoreH16>::value || std::is_same<S, StoreBF16>::value;
  constexpr int V2 = (F32 || H) ? 2 : 1;
  constexpr int V4 = H ? 4 : 1;
  if (H && (N % 4) == 0 && R >= 4) {
    if (R == 4) return launch_tma_r<S, 1, V4>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    return launch_tma_r<S, 2, V4>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
  }
  if ((F32 || H) && (N % 2) == 0 && R >= 2) {
    switch (R) {
      case 2: return launch_tma_r<S, 1, V2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
      case 4: return launch_tma_r<S, 2, V2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
      default: return launch_tma_r<S, 4, V2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    }
  }
  switch (R) {
    case 1: return launch_tma_r<S, 1, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    case 2: return launch_tma_r<S, 2, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    case 4: return launch_tma_r<S, 4, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    default: return launch_tma_r<S, 8, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
  }
}

// ---------------------------------------------------------------------------
// Per-thread asynchronous prefetch stencil.  Same work split as k_dslash, but
// every thread keeps DEPTH - 1 hops of its own operands in flight with
// cp.async into a private shared-memory ring (the T threads of a site share
// the site's nine link elements, each copying every T-th one), so the loads
// of later hops overlap the arithmetic of the current one without a
// CTA-wide barrier.  Requires T to divide the block size.
static constexpr int ASYNC_TPB = 128;

template <class S, int RV, int V, int EPI, int DEPTH>
__global__ void __launch_bounds__(ASYNC_TPB)
    k_dslash_async(const typename S::elem* __restrict__ links, const typename S::elem* __restrict__ in,
                   typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
                   const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity, int N,
                   int T, Gate gate) {
  using E = typename S::elem;
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (gate_closed(gate)) return;
  const int NS = N / V;
  const int SPT = 3 * RV * V;                 // spinor elements per thread per hop
  const int sites_cta = ASYNC_TPB / T;
  // ring: [DEPTH][sites_cta][9] links, then [DEPTH][ASYNC_TPB][SPT] spinors
  E* sL = reinterpret_cast<E*>(smem_raw);
  E* sS = sL + DEPTH * sites_cta * 9;
  const int tid = threadIdx.x;
  const int ls = tid / T;  // local site in the block
  const int k = tid - ls * T;
  const long long total = (long long)g.Vh * T;
  const real m2 = C::from_double(m2d);
  const int nr = (NS - k + T - 1) / T;
  for (long long gid0 = (long long)blockIdx.x * ASYNC_TPB; gid0 < total;
       gid0 += (long long)gridDim.x * ASYNC_TPB) {
    const long long gid = gid0 + tid;
    const bool live = gid < total;
    const int site = live ? (int)(gid / T) : 0;
    int x, y, z, t;
    site_xyzt(g, site, parity, x, y, z, t);
    const int lex = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
    const typename S::elem* lp = links + link_offset(g, parity, site);
    auto issue = [&](int d) {
      if (live) {
        const int buf = d % DEPTH;
        E* l = sL + (buf * sites_cta + ls) * 9;
        for (int e = k; e < 9; e += T) cp_async_bytes(l + e, lp + (d * 9 + e) * LINK_W, sizeof(E));
        const int nb = neighbour_cb_s(g, lex, x, y, z, t, d >> 2, hop_k(d & 3));
        const E* ip = in + (long long)nb * N * 3 + k * V;
        E* sp = sS + ((long long)buf * ASYNC_TPB + tid) * SPT;
#pragma unroll
        for (int r = 0; r < RV; ++r)
          if (r < nr)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              cp_async_bytes(sp + (r * 3 + b) * V, ip + b * N + r * T * V, V * sizeof(E));
      }
      cp_async_commit();
    };
    cpx<acc> a[RV][V][3];
#pragma unroll
    for (int r = 0; r < RV; ++r)
#pragma unroll
      for (int w = 0; w < V; ++w)
#pragma unroll
        for (int i = 0; i < 3; ++i) a[r][w][i] = czero<C>();
#pragma unroll
    for (int d = 0; d < DEPTH - 1; ++d) issue(d);
#pragma unroll 1
    for (int d = 0; d < 16; ++d) {
      if (d + DEPTH - 1 < 16) issue(d + DEPTH - 1);
      else cp_async_commit();
      cp_async_wait<DEPTH - 1>();
      __syncwarp();
      if (live) {
        const int buf = d % DEPTH;
        const E* l = sL + (buf * sites_cta + ls) * 9;
        cpx<real> U[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) U[e] = S::load_nc_raw(l + e);
        const E* sp = sS + ((long long)buf * ASYNC_TPB + tid) * SPT;
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          if (r < nr) {
            cpx<real> v[3][V];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
              for (int w = 0; w < V; ++w) v[b][w] = S::load_nc_raw(sp + (r * 3 + b) * V + w);
#pragma unroll
            for (int w = 0; w < V; ++w)
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                cmac<C>(a[r][w][i], U[i * 3 + 0], v[0][w]);
                cmac<C>(a[r][w][i], U[i * 3 + 1], v[1][w]);
                cmac<C>(a[r][w][i], U[i * 3 + 2], v[2][w]);
              }
          }
        }
      }
      __syncwarp();
    }
    if (live) {
      const long long ob = (long long)site * N * 3 + k * V;
#pragma unroll
      for (int r = 0; r < RV; ++r) {
        if (r < nr) {
#pragma unroll
          for (int w = 0; w < V; ++w)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const long long oi = ob + i * N + r * T * V + w;
              cpx<acc> vv = a[r][w][i];
                unscale_raw<S>(vv);
              if (EPI != EPI_NONE) {
                C::neg(vv.re);
                C::neg(vv.im);
                cpx<real> cc = S::load(c1 + oi);
                C::mac(vv.re, m2, cc.re);
                C::mac(vv.im, m2, cc.im);
                if (EPI == EPI_RESIDUAL) {
                  C::neg(vv.re);
                  C::neg(vv.im);
                  cpx<real> bb = S::load(c2 + oi);
                  C::add(vv.re, bb.re);
                  C::add(vv.im, bb.im);
                }
              }
              S::store(out + oi, cfin<C>(vv));
            }
        }
      }
    }
  }
}

template <class S, int RV, int V, int EPI>
static bool launch_async_t(const void* links, const void* in, void* out, const void* c1,
                           const void* c2, double m2, const Geom& g, int parity, int N, Gate gate,
                           cudaStream_t s) {
  using E = typename S::elem;
  const int NS = N / V;
  const int T = (NS + RV - 1) / RV;
  if (T > ASYNC_TPB || ASYNC_TPB % T) return false;
  if ((V * sizeof(E)) != 4 && (V * sizeof(E)) != 8 && (V * sizeof(E)) != 16) return false;
  constexpr int DEPTH = 3;
  const size_t sm = ((size_t)DEPTH * (ASYNC_TPB / T) * 9 + (size_t)DEPTH * ASYNC_TPB * 3 * RV * V) * sizeof(E);
  auto kern = k_dslash_async<S, RV, V, EPI, DEPTH>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return false;
  long long total = (long long)g.Vh * T;
  long long want = (total + ASYNC_TPB - 1) / ASYNC_TPB;
  unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
  if (gate_mostly_off(gate) && blocks > (unsigned)stencil_sms() * 4)
    blocks = (unsigned)stencil_sms() * 4;  // reliable-update stencil: persistent grid
  kern<<<blocks, ASYNC_TPB, sm, s>>>((const E*)links, (const E*)in, (E*)out, (const E*)c1,
                                     (const E*)c2, m2, g, parity, N, T, gate);
  return true;
}

template <class S, int RV, int V>
static bool launch_async_r(int epi, const void* links, const void* in, void* out, const void* c1,
                           const void* c2, double m2, const Geom& g, int parity, int N, Gate gate,
                           cudaStream_t s) {
  switch (epi) {
    case EPI_NONE: return launch_async_t<S, RV, V, EPI_NONE>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
    case EPI_NORMAL: return launch_async_t<S, RV, V, EPI_NORMAL>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
    default: return launch_async_t<S, RV, V, EPI_RESIDUAL>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
  }
}

template <class S>
static bool launch_async_s(int R, int epi, const void* links, const void* in, void* out,
                     const void* c1, const void* c2, double m2, const Geom& g, int parity,
                     int N, Gate gate, cudaStream_t s) {
  // vector width V: complex numbers per load (FP32: 2 per 128 bits; 16-bit
  // kinds: 4 per 128 bits or 2 per 64 bits); RV = R / V slots per thread
  constexpr bool F32 = std::is_same<S, StoreF32>::value;
  constexpr bool H = std::is_same<S, StoreH16>::value || std::is_same<S, StoreBF16>::value;
  constexpr int V2 = (F32 || H) ? 2 : 1;
  constexpr int V4 = H ? 4 : 1;
  if (H && (N % 4) == 0 && R >= 4) {
    if (R == 4) return launch_async_r<S, 1, V4>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    return launch_async_r<S, 2, V4>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
  }
  if ((F32 || H) && (N % 2) == 0 && R >= 2) {
    switch (R) {
      case 2: return launch_async_r<S, 1, V2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      case 4: return launch_async_r<S, 2, V2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      default: return launch_async_r<S, 4, V2>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    }
  }
  switch (R) {
    case 1: return launch_async_r<S, 1, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    case 2: return launch_async_r<S, 2, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    case 4: return launch_async_r<S, 4, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    default: return launch_async_r<S, 8, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
  }
}


template <class S, int RV, int V, int EPI, bool RC = false>
static void launch_dslash_t(const void* links, const void* in, void* out, const void* c1,
                            const void* c2, double m2, const Geom& g, int parity, int N,
                            Gate gate, bool blocked, cudaStream_t s) {
  using E = typename S::elem;
#ifndef BCG_UNROLL_DF
#define BCG_UNROLL_DF 0
#endif
  constexpr int UNROLL =
      std::is_same<S, StoreDF>::value ? BCG_UNROLL_DF : PlainBounds<S, RV>::unroll;
  const int NS = N / V;
  int T = (NS + RV - 1) / RV;
  long long threads_total = (long long)g.Vh * T;
  int threads = BCG_DSLASH_TPB;
  long long want = (threads_total + threads - 1) / threads;
  unsigned blocks = (unsigned)(want < 152 * 32 ? want : 152 * 32);
  long long span = 0;
  if (gate_mostly_off(gate)) {
    // a reliable-update stencil: a persistent grid (see gate_mostly_off)
    const long long cap = (long long)stencil_sms() * 4;
    if (blocks > cap) blocks = (unsigned)cap;
  }
  if (blocked) {
    // a persistent grid of the resident blocks, each owning one contiguous
    // range of (site, slot) pairs, a whole number of blocks of threads long
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash<S, RV, V, EPI, UNROLL, RC>,
                                                      threads, 0) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    long long nb = (long long)stencil_sms() * per_sm;
    if (nb > want) nb = want;
    const long long per = (want + nb - 1) / nb;  // thread blocks' worth of pairs per CTA
    span = per * threads;
    blocks = (unsigned)((threads_total + span - 1) / span);
  }
  k_dslash<S, RV, V, EPI, UNROLL, RC><<<blocks, threads, 0, s>>>(
      (const E*)links, (const E*)in, (E*)out, (const E*)c1, (const E*)c2, m2, g, parity, N, T, span,
      gate);
}

template <class S, int RV, int V, bool RC = false>
static void launch_dslash_r(int epi, const void* links, const void* in, void* out, const void* c1,
                            const void* c2, double m2, const Geom& g, int parity, int N,
                            Gate gate, bool blocked, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE:
      launch_dslash_t<S, RV, V, EPI_NONE, RC>(links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
      break;
    case EPI_NORMAL:
      launch_dslash_t<S, RV, V, EPI_NORMAL, RC>(links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
      break;
    default:
      launch_dslash_t<S, RV, V, EPI_RESIDUAL, RC>(links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
      break;
  }
}

// R = right-hand sides per thread.  FP32 with even N and R >= 2 uses 128-bit
// loads of two right-hand sides (V = 2, RV = R / 2 slots).
template <class S, bool RC = false>
static void launch_dslash_s(int R, int epi, const void* links, const void* in, void* out,
                     const void* c1, const void* c2, double m2, const Geom& g, int parity,
                     int N, Gate gate, bool blocked, cudaStream_t s) {
  // vector width V: complex numbers per load (FP32: 2 per 128 bits; 16-bit
  // kinds: 4 per 128 bits or 2 per 64 bits); RV = R / V slots per thread
  constexpr bool F32 = std::is_same<S, StoreF32>::value;
  constexpr bool H = std::is_same<S, StoreH16>::value || std::is_same<S, StoreBF16>::value;
  constexpr int V2 = (F32 || H) ? 2 : 1;
  constexpr int V4 = H ? 4 : 1;
  if (H && (N % 4) == 0 && R >= 4) {
    if (R == 4) return launch_dslash_r<S, 1, V4, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
    return launch_dslash_r<S, 2, V4, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
  }
  if ((F32 || H) && (N % 2) == 0 && R >= 2) {
    switch (R) {
      case 2: return launch_dslash_r<S, 1, V2, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
      case 4: return launch_dslash_r<S, 2, V2, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
      default: return launch_dslash_r<S, 4, V2, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
    }
  }
  switch (R) {
    case 1: return launch_dslash_r<S, 1, 1, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
    case 2: return launch_dslash_r<S, 2, 1, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
    case 4: return launch_dslash_r<S, 4, 1, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
    default: return launch_dslash_r<S, 8, 1, RC>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, blocked, s);
  }
}


// One storage kind: the cp.async prefetch kernel (R | DSLASH_ASYNC), the
// bulk-copy pipelined kernel (R | DSLASH_TMA) or the plain kernel; a
// pipelined request that cannot run for this N falls back to the plain one.
template <class S>
static cudaError_t dslash_kind(int R, int epi, const void* links, const void* in, void* out,
                               const void* c1, const void* c2, double m2, const Geom& g,
                               int out_parity, int N, Gate gate, cudaStream_t s) {
  if (R & DSLASH_RECON) {  // two-row links: plain kernel, 32- and 16-bit kinds only
    if constexpr (std::is_same<typename S::comp::real, float>::value) {
      launch_dslash_s<S, true>(R & 0xff, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate,
                               (R & DSLASH_BLOCKED) != 0, s);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (R & DSLASH_ASYNC) {
    const int r = R & 0xff;
    if (launch_async_s<S>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s))
      return cudaGetLastError();
    cudaGetLastError();
    R = r;
  }
  if (R & DSLASH_TMA) {
    const int r = R & 0xff;
    SolverStatus* errst = const_cast<SolverStatus*>(gate.st);
    if (launch_tma_s<S>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, errst, s))
      return cudaGetLastError();
    cudaGetLastError();
    R = r;
  }
  launch_dslash_s<S>(R & 0xff, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate,
                     (R & DSLASH_BLOCKED) != 0, s);
  return cudaGetLastError();
}

}  // namespace bcg
