// Multi-RHS improved-staggered stencil (Sec. 5.2, Eq. 1).
//
// Links are repacked once per gauge field (pack_links) into, for each output
// parity p and each of the 16 hops d = 4*mu + q (q: +1, -1, +3, -3 along mu),
// the matrix that multiplies psi(x + k_q mu) in Eq. 1 with everything folded
// in: 1/2, the staggered phase eta_mu(x), the boundary sign, and for the
// backward hops the dagger and the minus sign of the anti-Hermitian reading.
// Layout [p][site / LW][d * 9 + e][site % LW] (e = 0..8 matrix element,
// LW = 32 sites per block): the loads of one matrix element by consecutive
// sites are contiguous, and all 144 link words a group of sites needs lie in
// one LW * 144-element block instead of 144 streams a parity apart.
//
// One thread owns one output site and a register tile of R right-hand sides
// (the register tiling of Sec. 5.2); the T = ceil(N/R) threads of a site sit
// next to each other in a warp, so each link element is fetched once per
// warp and broadcast (the cache tiling of Sec. 5.2 maps onto the broadcast of
// a warp-wide load).  Spinor blocks are site-major [site][colour][rhs] and
// thread k of a site owns the right-hand sides k, k + T, k + 2T, ...: for one
// (colour, r) the T threads of a site read T consecutive elements, so every
// warp-wide load uses whole 32-byte sectors.
#include <type_traits>

#include "internal.h"
#include "tma.cuh"

namespace bcg {

static constexpr int LINK_W = 32;  // sites per link block

// number of link blocks per parity (the last one may be partly used)
__host__ __device__ inline long long link_blocks(const Geom& g) {
  return ((long long)g.Vh + LINK_W - 1) / LINK_W;
}

// element offset of (parity p, site cb, hop 0, element 0)
__device__ __forceinline__ long long link_offset(const Geom& g, int p, int cb) {
  return ((long long)p * link_blocks(g) + cb / LINK_W) * (16 * 9 * LINK_W) + (cb % LINK_W);
}

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
  typename S::elem* o = out + link_offset(g, p, cb) + (long long)d * 9 * LINK_W;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double2 u = back ? make_double2(U[b * 3 + a].x, -U[b * 3 + a].y) : U[a * 3 + b];
      u.x *= factor;
      u.y *= factor;
      o[(long long)(a * 3 + b) * LINK_W] = S::from_double2(u);
    }
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
    v[0] = S::load(p);
  }
};
template <>
struct VecLoad<StoreF32, 2> {
  static __device__ __forceinline__ void get(const float2* p, cpx<float>* v) {
    StoreF32::load2(p, v[0], v[1]);
  }
};

#ifndef BCG_DSLASH_TPB
#define BCG_DSLASH_TPB 128
#endif
#ifndef BCG_DSLASH_MINB
#define BCG_DSLASH_MINB 1
#endif

template <class S, int RV, int V, int EPI, int UNROLL_HOPS>
__global__ void __launch_bounds__(BCG_DSLASH_TPB, BCG_DSLASH_MINB)
    k_dslash(const typename S::elem* __restrict__ links, const typename S::elem* __restrict__ in,
             typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
             const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity, int N,
             int T, Gate gate) {
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  if (gate_closed(gate)) return;
  const int NS = N / V;
  const long long total = (long long)g.Vh * T;
  const real m2 = C::from_double(m2d);
  for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
       gid += (long long)gridDim.x * blockDim.x) {
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

    const typename S::elem* lp = links + link_offset(g, parity, site);
    auto hop = [&](int d) {
      const int nb = neighbour_cb_s(g, lex, x, y, z, t, d >> 2, hop_k(d & 3));
      cpx<real> U[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) U[e] = S::load(lp + (d * 9 + e) * LINK_W);
      const typename S::elem* ip = in + (long long)nb * N * 3 + k * V;
#pragma unroll
      for (int r = 0; r < RV; ++r) {
        if (r < nr) {
          cpx<real> v[3][V];
#pragma unroll
          for (int b = 0; b < 3; ++b) VecLoad<S, V>::get(ip + b * N + r * T * V, v[b]);
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
// Bulk-copy pipelined stencil.  A CTA owns blocks of LINK_W = 32 consecutive
// output sites (one link block) with T threads per site; its work is the
// stream of (block, hop) tasks.  Warp 0 keeps STAGES - 1 hops ahead: for each
// task it posts the expected byte count on the stage's mbarrier, copies the
// hop's 9 x 32 link words (contiguous in the blocked link layout) with one
// cp.async.bulk and the 32 neighbour spinor blocks (3N complex each) with one
// cp.async.bulk per lane into the stage.  All threads wait for the stage,
// multiply from shared memory and accumulate in registers; after hop 15 they
// write their outputs.  Loads for later hops are in flight while a hop is
// computed, so the kernel no longer waits on one hop's loads at a time.
// Every wait is bounded: on time-out the CTA records BLOCKCG_ERR_TIMEOUT in
// the status word, waits (bounded) for copies it issued and returns.
static constexpr uint64_t TMA_WAIT_LIMIT = 4000000000ull;  // 4 s of wall-clock time

template <class S, int RV, int V, int EPI, int STAGES>
__global__ void __launch_bounds__(256)
    k_dslash_tma(const typename S::elem* __restrict__ links, const typename S::elem* __restrict__ in,
                 typename S::elem* __restrict__ out, const typename S::elem* __restrict__ c1,
                 const typename S::elem* __restrict__ c2, double m2d, Geom g, int parity, int N,
                 int T, int sstride, Gate gate, SolverStatus* errst) {
  using E = typename S::elem;
  using C = typename S::comp;
  using real = typename C::real;
  using acc = typename C::acc;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ int abort_flag;
  if (gate_closed(gate)) return;
  const int tid = threadIdx.x;
  const int NS = N / V;
  const int sl = tid / T;  // local site
  const int k = tid - sl * T;
  const int link_elems = 9 * LINK_W;
  const int stage_elems = link_elems + LINK_W * sstride;
  E* sbase = reinterpret_cast<E*>(smem_raw);
  const long long units = link_blocks(g);
  const long long my_units =
      units > (long long)blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long ntasks = my_units * 16;
  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(&full[i], 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t spin_bytes = 3u * N * sizeof(E);

  auto issue = [&](long long task) {  // warp 0
    const long long unit = blockIdx.x + (task >> 4) * (long long)gridDim.x;
    const int d = (int)(task & 15);
    const int st = (int)(task % STAGES);
    E* base = sbase + (size_t)st * stage_elems;
    const int lane = tid;
    const long long site0 = unit * LINK_W;
    const int nvalid = (int)min((long long)LINK_W, (long long)g.Vh - site0);
    if (lane == 0)
      mbar_arrive_expect_tx(&full[st], (uint32_t)(link_elems * sizeof(E)) + nvalid * spin_bytes);
    __syncwarp();
    if (lane == 0)
      bulk_g2s(base, links + link_offset(g, parity, (int)site0) + d * 9 * LINK_W,
               (uint32_t)(link_elems * sizeof(E)), &full[st]);
    if (lane < nvalid) {
      int x, y, z, t;
      const int site = (int)site0 + lane;
      site_xyzt(g, site, parity, x, y, z, t);
      const int lex = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
      const int nb = neighbour_cb_s(g, lex, x, y, z, t, d >> 2, hop_k(d & 3));
      bulk_g2s(base + link_elems + lane * sstride, in + (long long)nb * N * 3, spin_bytes, &full[st]);
    }
  };

  long long issued = 0;
  if (tid < 32) {
    for (; issued < STAGES - 1 && issued < ntasks; ++issued) issue(issued);
  }
  const real m2 = C::from_double(m2d);
  cpx<acc> a[RV][V][3];
  const int nr = (NS - k + T - 1) / T;  // slots k + r*T < NS
  long long tau = 0;
  for (; tau < ntasks; ++tau) {
    if (tid < 32 && tau + STAGES - 1 < ntasks) {
      issue(tau + STAGES - 1);
    }
    if (tid < 32) issued = min(ntasks, tau + STAGES);
    const int d = (int)(tau & 15);
    const int st = (int)(tau % STAGES);
    const long long unit = blockIdx.x + (tau >> 4) * (long long)gridDim.x;
    const long long site = unit * LINK_W + sl;
    const bool valid = site < g.Vh && sl < LINK_W;
    if (d == 0) {
#pragma unroll
      for (int r = 0; r < RV; ++r)
#pragma unroll
        for (int w = 0; w < V; ++w)
#pragma unroll
          for (int i = 0; i < 3; ++i) a[r][w][i] = czero<C>();
    }
    if (!mbar_wait_bounded(&full[st], (uint32_t)((tau / STAGES) & 1), TMA_WAIT_LIMIT)) {
      abort_flag = 1;
    } else if (valid) {
      const E* base = sbase + (size_t)st * stage_elems;
      cpx<real> U[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) U[e] = S::load_nc(base + e * LINK_W + sl);
      const E* ip = base + link_elems + sl * sstride + k * V;
#pragma unroll
      for (int r = 0; r < RV; ++r) {
        if (r < nr) {
          cpx<real> v[3][V];
#pragma unroll
          for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int w = 0; w < V; ++w) v[b][w] = S::load_nc(ip + b * N + r * T * V + w);
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
      if (d == 15) {
        const long long ob = site * N * 3 + k * V;
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          if (r < nr) {
#pragma unroll
            for (int w = 0; w < V; ++w)
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                const long long oi = ob + i * N + r * T * V + w;
                cpx<acc> vv = a[r][w][i];
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
    fence_proxy_async_shared();
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag) {
    // record the failure, then wait (bounded) for the copies still in flight
    if (tid == 0) {
      if (errst) atomicExch(&errst->error, (int)7 /* BLOCKCG_ERR_TIMEOUT */);
      for (long long q = tau + 1; q < issued; ++q)
        mbar_wait_bounded(&full[q % STAGES], (uint32_t)((q / STAGES) & 1), TMA_WAIT_LIMIT);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Per-thread asynchronous prefetch stencil.  Same work split as k_dslash, but
// every thread keeps DEPTH - 1 hops of its own operands in flight with
// cp.async into a private shared-memory ring (the T threads of a site share
// the site's nine link elements, each copying every T-th one), so the loads
// of later hops overlap the arithmetic of the current one without a
// CTA-wide barrier.  Requires T to divide the block size.
__device__ __forceinline__ void cp_async_bytes(void* dst, const void* src, int bytes) {
  const uint32_t d = smem_u32(dst);
  if (bytes == 16)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N_>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N_) : "memory");
}

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
        for (int e = 0; e < 9; ++e) U[e] = S::load_nc(l + e);
        const E* sp = sS + ((long long)buf * ASYNC_TPB + tid) * SPT;
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          if (r < nr) {
            cpx<real> v[3][V];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
              for (int w = 0; w < V; ++w) v[b][w] = S::load_nc(sp + (r * 3 + b) * V + w);
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
  if ((V * sizeof(E)) != 8 && (V * sizeof(E)) != 16) return false;
  constexpr int DEPTH = 3;
  const size_t sm = ((size_t)DEPTH * (ASYNC_TPB / T) * 9 + (size_t)DEPTH * ASYNC_TPB * 3 * RV * V) * sizeof(E);
  auto kern = k_dslash_async<S, RV, V, EPI, DEPTH>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return false;
  long long total = (long long)g.Vh * T;
  long long want = (total + ASYNC_TPB - 1) / ASYNC_TPB;
  unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
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
  constexpr bool F32 = std::is_same<S, StoreF32>::value;
  if (F32 && (N % 2) == 0 && R >= 2) {
    switch (R) {
      case 2: return launch_async_r<S, 1, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      case 4: return launch_async_r<S, 2, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
      default: return launch_async_r<S, 4, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    }
  }
  switch (R) {
    case 1: return launch_async_r<S, 1, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    case 2: return launch_async_r<S, 2, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    case 4: return launch_async_r<S, 4, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
    default: return launch_async_r<S, 8, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s);
  }
}

// smem site stride (elements): 3N padded so that consecutive sites start 16
// banks apart, and a multiple of 16 bytes
static int tma_site_stride(size_t eb, int N) {
  const int wpe = (int)(eb / 4);
  for (int p = 0; p < 64; ++p) {
    int s = 3 * N + p;
    if ((s * eb) % 16) continue;
    if (((s * wpe) % 32) == 16) return s;
  }
  return 3 * N + (eb == 8 ? ((3 * N) & 1) : 0);
}

template <class S, int RV, int V, int EPI, int STAGES>
static bool launch_tma_t(const void* links, const void* in, void* out, const void* c1,
                         const void* c2, double m2, const Geom& g, int parity, int N, Gate gate,
                         SolverStatus* errst, cudaStream_t s) {
  using E = typename S::elem;
  const size_t eb = sizeof(E);
  const int NS = N / V;
  const int T = (NS + RV - 1) / RV;
  if (T * LINK_W > 256) return false;
  if ((3 * N * eb) % 16) return false;
  const int sstride = tma_site_stride(eb, N);
  const size_t stage_bytes = (9 * LINK_W + (size_t)LINK_W * sstride) * eb;
  const size_t sm = STAGES * stage_bytes;
  if (sm > 200 * 1024) return false;
  auto kern = k_dslash_tma<S, RV, V, EPI, STAGES>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return false;
  long long units = link_blocks(g);
  int per_sm = (int)((220 * 1024) / (sm + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  long long want = 152LL * per_sm;
  unsigned blocks = (unsigned)(units < want ? units : want);
  kern<<<blocks, T * LINK_W, sm, s>>>((const E*)links, (const E*)in, (E*)out, (const E*)c1,
                                      (const E*)c2, m2, g, parity, N, T, sstride, gate, errst);
  return true;
}

template <class S, int RV, int V>
static bool launch_tma_r(int epi, const void* links, const void* in, void* out, const void* c1,
                         const void* c2, double m2, const Geom& g, int parity, int N, Gate gate,
                         SolverStatus* errst, cudaStream_t s) {
  // three stages when they fit, else two
  switch (epi) {
    case EPI_NONE:
      return launch_tma_t<S, RV, V, EPI_NONE, 3>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_NONE, 2>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    case EPI_NORMAL:
      return launch_tma_t<S, RV, V, EPI_NORMAL, 3>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_NORMAL, 2>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    default:
      return launch_tma_t<S, RV, V, EPI_RESIDUAL, 3>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s) ||
             launch_tma_t<S, RV, V, EPI_RESIDUAL, 2>(links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
  }
}

template <class S>
static bool launch_tma_s(int R, int epi, const void* links, const void* in, void* out,
                         const void* c1, const void* c2, double m2, const Geom& g, int parity,
                         int N, Gate gate, SolverStatus* errst, cudaStream_t s) {
  constexpr bool F32 = std::is_same<S, StoreF32>::value;
  if (F32 && (N % 2) == 0 && R >= 2) {
    switch (R) {
      case 2: return launch_tma_r<S, 1, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
      case 4: return launch_tma_r<S, 2, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
      default: return launch_tma_r<S, 4, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    }
  }
  switch (R) {
    case 1: return launch_tma_r<S, 1, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    case 2: return launch_tma_r<S, 2, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    case 4: return launch_tma_r<S, 4, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
    default: return launch_tma_r<S, 8, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, errst, s);
  }
}

size_t links_bytes(FieldKind k, const Geom& g) {
  return 2ull * link_blocks(g) * 16 * 9 * LINK_W * elem_bytes(k);
}

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

template <class S, int RV, int V, int EPI>
static void launch_dslash_t(const void* links, const void* in, void* out, const void* c1,
                            const void* c2, double m2, const Geom& g, int parity, int N,
                            Gate gate, cudaStream_t s) {
  using E = typename S::elem;
#ifndef BCG_UNROLL_F32
#define BCG_UNROLL_F32 1
#endif
#ifndef BCG_UNROLL_DF
#define BCG_UNROLL_DF 0
#endif
  constexpr int UNROLL = std::is_same<S, StoreDF>::value ? BCG_UNROLL_DF : BCG_UNROLL_F32;
  const int NS = N / V;
  int T = (NS + RV - 1) / RV;
  long long threads_total = (long long)g.Vh * T;
  int threads = BCG_DSLASH_TPB;
  long long want = (threads_total + threads - 1) / threads;
  unsigned blocks = (unsigned)(want < 152 * 32 ? want : 152 * 32);
  k_dslash<S, RV, V, EPI, UNROLL><<<blocks, threads, 0, s>>>(
      (const E*)links, (const E*)in, (E*)out, (const E*)c1, (const E*)c2, m2, g, parity, N, T, gate);
}

template <class S, int RV, int V>
static void launch_dslash_r(int epi, const void* links, const void* in, void* out, const void* c1,
                            const void* c2, double m2, const Geom& g, int parity, int N,
                            Gate gate, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE:
      launch_dslash_t<S, RV, V, EPI_NONE>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    case EPI_NORMAL:
      launch_dslash_t<S, RV, V, EPI_NORMAL>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
    default:
      launch_dslash_t<S, RV, V, EPI_RESIDUAL>(links, in, out, c1, c2, m2, g, parity, N, gate, s);
      break;
  }
}

// R = right-hand sides per thread.  FP32 with even N and R >= 2 uses 128-bit
// loads of two right-hand sides (V = 2, RV = R / 2 slots).
template <class S>
static void launch_dslash_s(int R, int epi, const void* links, const void* in, void* out,
                            const void* c1, const void* c2, double m2, const Geom& g, int parity,
                            int N, Gate gate, cudaStream_t s) {
  constexpr bool F32 = std::is_same<S, StoreF32>::value;
  if (F32 && (N % 2) == 0 && R >= 2) {
    switch (R) {
      case 2: launch_dslash_r<S, 1, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); return;
      case 4: launch_dslash_r<S, 2, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); return;
      default: launch_dslash_r<S, 4, F32 ? 2 : 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); return;
    }
  }
  switch (R) {
    case 1: launch_dslash_r<S, 1, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); break;
    case 2: launch_dslash_r<S, 2, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); break;
    case 4: launch_dslash_r<S, 4, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); break;
    default: launch_dslash_r<S, 8, 1>(epi, links, in, out, c1, c2, m2, g, parity, N, gate, s); break;
  }
}

cudaError_t dslash(FieldKind k, int R, int epi, const void* links, const void* in, void* out,
                   const void* c1, const void* c2, double m2, const Geom& g, int out_parity,
                   int N, Gate gate, cudaStream_t s) {
  if (R & DSLASH_ASYNC) {
    const int r = R & 0xff;
    bool ok = false;
    switch (k) {
      case FK_DF: ok = launch_async_s<StoreDF>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s); break;
      case FK_F32: ok = launch_async_s<StoreF32>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s); break;
      case FK_F64: ok = launch_async_s<StoreF64>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, s); break;
    }
    if (ok) return cudaGetLastError();
    cudaGetLastError();
    R = r;
  }
  if (R & DSLASH_TMA) {
    const int r = R & 0xff;
    SolverStatus* errst = const_cast<SolverStatus*>(gate.st);
    bool ok = false;
    switch (k) {
      case FK_DF: ok = launch_tma_s<StoreDF>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, errst, s); break;
      case FK_F32: ok = launch_tma_s<StoreF32>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, errst, s); break;
      case FK_F64: ok = launch_tma_s<StoreF64>(r, epi, links, in, out, c1, c2, m2, g, out_parity, N, gate, errst, s); break;
    }
    if (ok) return cudaGetLastError();
    cudaGetLastError();
    R = r;  // the pipelined kernel cannot run for this kind / N: plain kernel
  }
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
