// Device-side building blocks shared by the block-CGrQ kernels: arithmetic
// policies, complex types, storage formats and lattice geometry.
//
// Arithmetic policies ("Comp"):
//   CompDF  double-float: a real is an unevaluated pair hi + lo of FP32
//           numbers (about 48 significant bits).  Products use the exact
//           FMA-based TwoProd, sums use Knuth's TwoSum; accumulators keep a
//           running sum and a separate error term that is folded in once at
//           the end.  This runs on the FP32 pipes, which on GB300 execute
//           72x more FMAs per second than the FP64 pipe, and is the arithmetic
//           of the FP64-accurate solver form.
//   CompF32 plain FP32 (sloppy arithmetic of the mixed-precision form).
//   CompF64 native FP64 (verification and the final true residual).
// All FP32 steps of the error-free transformations use the __f*_rn
// intrinsics so that the compiler never contracts them into an FMA.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace bcg {

// ------------------------------------------------------------------ df --
struct df {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ df df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// accumulator: value = s + e, e not normalised
struct dfacc {
  float s, e;
};

// ---------------------------------------------------------- policies ----
struct CompDF {
  using real = df;
  using acc = dfacc;
  static __device__ __forceinline__ acc zero() { return {0.f, 0.f}; }
  // c += a * b
  static __device__ __forceinline__ void mac(acc& c, real a, real b) {
    float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, e;
    two_sum(c.s, p, s, e);
    c.s = s;
    c.e = __fadd_rn(c.e, __fadd_rn(e, pe));
  }
  // c -= a * b
  static __device__ __forceinline__ void msub(acc& c, real a, real b) {
    mac(c, real{-a.hi, -a.lo}, b);
  }
  // c += a
  static __device__ __forceinline__ void add(acc& c, real a) {
    float s, e;
    two_sum(c.s, a.hi, s, e);
    c.s = s;
    c.e = __fadd_rn(c.e, __fadd_rn(e, a.lo));
  }
  static __device__ __forceinline__ void neg(acc& c) {
    c.s = -c.s;
    c.e = -c.e;
  }
  static __device__ __forceinline__ real fin(acc c) {
    float s, e;
    two_sum(c.s, c.e, s, e);
    return {s, e};
  }
  static __device__ __forceinline__ double to_double(acc c) { return (double)c.s + (double)c.e; }
  static __device__ __forceinline__ real from_double(double x) { return df_from_double(x); }
  static __device__ __forceinline__ double real_to_double(real x) { return df_to_double(x); }
  static __device__ __forceinline__ real rzero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ acc acc_from(real a) { return {a.hi, a.lo}; }
};

struct CompF32 {
  using real = float;
  using acc = float;
  static __device__ __forceinline__ acc zero() { return 0.f; }
  static __device__ __forceinline__ void mac(acc& c, real a, real b) { c = fmaf(a, b, c); }
  static __device__ __forceinline__ void msub(acc& c, real a, real b) { c = fmaf(-a, b, c); }
  static __device__ __forceinline__ void add(acc& c, real a) { c += a; }
  static __device__ __forceinline__ void neg(acc& c) { c = -c; }
  static __device__ __forceinline__ real fin(acc c) { return c; }
  static __device__ __forceinline__ double to_double(acc c) { return (double)c; }
  static __device__ __forceinline__ real from_double(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ double real_to_double(real x) { return (double)x; }
  static __device__ __forceinline__ real rzero() { return 0.f; }
  static __device__ __forceinline__ acc acc_from(real a) { return a; }
};

struct CompF64 {
  using real = double;
  using acc = double;
  static __device__ __forceinline__ acc zero() { return 0.0; }
  static __device__ __forceinline__ void mac(acc& c, real a, real b) { c = fma(a, b, c); }
  static __device__ __forceinline__ void msub(acc& c, real a, real b) { c = fma(-a, b, c); }
  static __device__ __forceinline__ void add(acc& c, real a) { c += a; }
  static __device__ __forceinline__ void neg(acc& c) { c = -c; }
  static __device__ __forceinline__ real fin(acc c) { return c; }
  static __device__ __forceinline__ double to_double(acc c) { return c; }
  static __device__ __forceinline__ real from_double(double x) { return x; }
  static __device__ __forceinline__ double real_to_double(real x) { return x; }
  static __device__ __forceinline__ real rzero() { return 0.0; }
  static __device__ __forceinline__ acc acc_from(real a) { return a; }
};

template <class R>
struct cpx {
  R re, im;
};

// c += a * b (complex)
template <class C>
__device__ __forceinline__ void cmac(cpx<typename C::acc>& c, const cpx<typename C::real>& a,
                                     const cpx<typename C::real>& b) {
  C::mac(c.re, a.re, b.re);
  C::msub(c.re, a.im, b.im);
  C::mac(c.im, a.re, b.im);
  C::mac(c.im, a.im, b.re);
}

// c += conj(a) * b (complex)
template <class C>
__device__ __forceinline__ void cmac_conj(cpx<typename C::acc>& c, const cpx<typename C::real>& a,
                                          const cpx<typename C::real>& b) {
  C::mac(c.re, a.re, b.re);
  C::mac(c.re, a.im, b.im);
  C::mac(c.im, a.re, b.im);
  C::msub(c.im, a.im, b.re);
}

template <class C>
__device__ __forceinline__ cpx<typename C::acc> czero() {
  return {C::zero(), C::zero()};
}

template <class C>
__device__ __forceinline__ cpx<typename C::acc> cacc_from(const cpx<typename C::real>& a) {
  return {C::acc_from(a.re), C::acc_from(a.im)};
}

template <class C>
__device__ __forceinline__ cpx<typename C::real> cfin(const cpx<typename C::acc>& a) {
  return {C::fin(a.re), C::fin(a.im)};
}

// ----------------------------------------------------------- storage ----
// Complex element formats in HBM.  Every field is a block of N columns in
// site-major order [site][rhs][colour] (one 3-vector of complex numbers per
// site and right-hand side).
struct StoreDF {  // {re.hi, im.hi, re.lo, im.lo}: one 128-bit word per complex
  using elem = float4;
  using comp = CompDF;
  static constexpr float RAW_SCALE = 1.f;  // see StoreH16
  static __device__ __forceinline__ cpx<df> load_raw(const elem* p) { return load(p); }
  static __device__ __forceinline__ cpx<df> load_nc_raw(const elem* p) { return load_nc(p); }
  static __device__ __forceinline__ cpx<df> load(const elem* p) {
    float4 v = __ldg(p);
    return {{v.x, v.z}, {v.y, v.w}};
  }
  static __device__ __forceinline__ cpx<df> load_nc(const elem* p) {
    float4 v = *p;
    return {{v.x, v.z}, {v.y, v.w}};
  }
  static __device__ __forceinline__ void store(elem* p, const cpx<df>& a) {
    *p = make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo);
  }
  static __device__ __forceinline__ elem from_double2(double2 z) {
    df r = df_from_double(z.x), i = df_from_double(z.y);
    return make_float4(r.hi, i.hi, r.lo, i.lo);
  }
  static __device__ __forceinline__ double2 to_double2(elem v) {
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
};

struct StoreF32 {
  using elem = float2;
  using comp = CompF32;
  static constexpr float RAW_SCALE = 1.f;
  // two consecutive complex numbers with one 128-bit load (16-byte aligned)
  static __device__ __forceinline__ void load2(const elem* p, cpx<float>& a, cpx<float>& b) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a = {v.x, v.y};
    b = {v.z, v.w};
  }
  static __device__ __forceinline__ cpx<float> load(const elem* p) {
    float2 v = __ldg(p);
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cpx<float> load_nc(const elem* p) {
    float2 v = *p;
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cpx<float> load_raw(const elem* p) { return load(p); }
  static __device__ __forceinline__ cpx<float> load_nc_raw(const elem* p) { return load_nc(p); }
  static __device__ __forceinline__ void store(elem* p, const cpx<float>& a) {
    *p = make_float2(a.re, a.im);
  }
  static __device__ __forceinline__ elem from_double2(double2 z) {
    return make_float2(__double2float_rn(z.x), __double2float_rn(z.y));
  }
  static __device__ __forceinline__ double2 to_double2(elem v) {
    return make_double2((double)v.x, (double)v.y);
  }
};

struct StoreF64 {
  using elem = double2;
  using comp = CompF64;
  static constexpr float RAW_SCALE = 1.f;
  static __device__ __forceinline__ cpx<double> load_raw(const elem* p) { return load(p); }
  static __device__ __forceinline__ cpx<double> load_nc_raw(const elem* p) { return load_nc(p); }
  static __device__ __forceinline__ cpx<double> load(const elem* p) {
    double2 v = __ldg(p);
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cpx<double> load_nc(const elem* p) {
    double2 v = *p;
    return {v.x, v.y};
  }
  static __device__ __forceinline__ void store(elem* p, const cpx<double>& a) {
    *p = make_double2(a.re, a.im);
  }
  static __device__ __forceinline__ elem from_double2(double2 z) { return z; }
  static __device__ __forceinline__ double2 to_double2(elem v) { return v; }
};

// 16-bit sloppy storage with FP32 arithmetic.  FP16 stores 2^4 x value:
// Krylov block vectors are normalised, so the components of Q are ~L^-1/2
// (1e-3 .. 1e-4 here); the fixed power-of-two factor lifts them well above
// FP16's subnormal range while leaving ~10^5 of headroom for the growth of
// the search block P (|P| ~ |r_k| / min_j |r_j| when the residual
// oscillates) and for A P, without per-site scale arrays; the factor is
// exact in both directions.  BF16 has FP32's exponent range and needs no
// factor.
struct StoreH16 {
  using elem = __half2;
  using comp = CompF32;
  static constexpr float SCALE = 16.f;
  static constexpr float INV = 1.f / 16.f;
  // The raw loads keep the stored 2^4 factor: kernels that multiply stored
  // values by stored values (the stencil: links times spinors) take the
  // products in the scaled domain and remove RAW_SCALE^2 once per output,
  // saving two multiplications per loaded element (exact: powers of two).
  static constexpr float RAW_SCALE = SCALE;
  static __device__ __forceinline__ cpx<float> cvt(__half2 h) {
    float2 f = __half22float2(h);
    return {f.x * INV, f.y * INV};
  }
  static __device__ __forceinline__ cpx<float> cvt_raw(__half2 h) {
    float2 f = __half22float2(h);
    return {f.x, f.y};
  }
  static __device__ __forceinline__ cpx<float> load_raw(const elem* p) { return cvt_raw(__ldg(p)); }
  static __device__ __forceinline__ cpx<float> load_nc_raw(const elem* p) { return cvt_raw(*p); }
  static __device__ __forceinline__ cpx<float> load(const elem* p) { return cvt(__ldg(p)); }
  static __device__ __forceinline__ cpx<float> load_nc(const elem* p) { return cvt(*p); }
  static __device__ __forceinline__ void store(elem* p, const cpx<float>& a) {
    *p = __floats2half2_rn(a.re * SCALE, a.im * SCALE);
  }
  static __device__ __forceinline__ elem from_double2(double2 z) {
    return __floats2half2_rn(__double2float_rn(z.x) * SCALE, __double2float_rn(z.y) * SCALE);
  }
  static __device__ __forceinline__ double2 to_double2(elem v) {
    float2 f = __half22float2(v);
    return make_double2((double)f.x * INV, (double)f.y * INV);
  }
};

struct StoreBF16 {
  using elem = __nv_bfloat162;
  using comp = CompF32;
  static constexpr float RAW_SCALE = 1.f;
  static __device__ __forceinline__ cpx<float> cvt(__nv_bfloat162 h) {
    float2 f = __bfloat1622float2(h);
    return {f.x, f.y};
  }
  static __device__ __forceinline__ cpx<float> cvt_raw(__nv_bfloat162 h) { return cvt(h); }
  static __device__ __forceinline__ cpx<float> load_raw(const elem* p) { return cvt(__ldg(p)); }
  static __device__ __forceinline__ cpx<float> load_nc_raw(const elem* p) { return cvt(*p); }
  static __device__ __forceinline__ cpx<float> load(const elem* p) { return cvt(__ldg(p)); }
  static __device__ __forceinline__ cpx<float> load_nc(const elem* p) { return cvt(*p); }
  static __device__ __forceinline__ void store(elem* p, const cpx<float>& a) {
    *p = __floats2bfloat162_rn(a.re, a.im);
  }
  static __device__ __forceinline__ elem from_double2(double2 z) {
    return __floats2bfloat162_rn(__double2float_rn(z.x), __double2float_rn(z.y));
  }
  static __device__ __forceinline__ double2 to_double2(elem v) {
    float2 f = __bfloat1622float2(v);
    return make_double2((double)f.x, (double)f.y);
  }
};

// Conversions between compute types (used where a sloppy block meets a
// full-precision one, e.g. X += P (beta C) with P in FP32 and X in df).
template <class To, class From>
struct conv;
template <class C>
struct conv<C, C> {
  static __device__ __forceinline__ typename C::real f(typename C::real x) { return x; }
};
template <>
struct conv<CompDF, CompF32> {
  static __device__ __forceinline__ df f(float x) { return {x, 0.f}; }
};
template <>
struct conv<CompF32, CompDF> {
  static __device__ __forceinline__ float f(df x) { return __fadd_rn(x.hi, x.lo); }
};
template <>
struct conv<CompDF, CompF64> {
  static __device__ __forceinline__ df f(double x) { return df_from_double(x); }
};
template <>
struct conv<CompF64, CompDF> {
  static __device__ __forceinline__ double f(df x) { return df_to_double(x); }
};
template <>
struct conv<CompF32, CompF64> {
  static __device__ __forceinline__ float f(double x) { return __double2float_rn(x); }
};
template <>
struct conv<CompF64, CompF32> {
  static __device__ __forceinline__ double f(float x) { return (double)x; }
};

// ---------------------------------------------------------- geometry ----
struct Geom {
  int L[4];  // Lx, Ly, Lz, Lt (all even)
  int hx;    // Lx / 2
  int Vh;    // sites per parity
  // links stored as two rows (stencil calls flagged DSLASH_RECON): the third
  // row is conj(row0 x row1) * eta_mu(x) * boundary sign * backward sign *
  // inv_c[kind], inv_c = 1 / (c / 2) for the fat (0) and long (1) link scale c
  int antiperiodic;
  float inv_c[2];
  // bounded device waits (bulk-copy stencil) give up after this many ns
  unsigned long long wait_ns;
  // the tensor-core double-float stencil's per-column maxima (64 words of the
  // handle's workspace; null until a workspace is set)
  unsigned* tc_colmax;
};

// coordinates of the site with checkerboard index cb on parity p
__device__ __forceinline__ void site_coords(const Geom& g, int cb, int p, int c[4]) {
  int xh = cb % g.hx;
  int r = cb / g.hx;
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

// checkerboard index of c + k * mu (periodic)
__device__ __forceinline__ int neighbour_cb(const Geom& g, const int c[4], int mu, int k) {
  int y[4] = {c[0], c[1], c[2], c[3]};
  int v = y[mu] + k;
  int L = g.L[mu];
  while (v >= L) v -= L;
  while (v < 0) v += L;
  y[mu] = v;
  int lex = y[0] + g.L[0] * (y[1] + g.L[1] * (y[2] + g.L[2] * y[3]));
  return lex >> 1;
}

// Coordinates as scalars (no arrays, so nothing is indexed at run time and
// nothing spills to local memory).
__device__ __forceinline__ void site_xyzt(const Geom& g, int cb, int p, int& x, int& y, int& z,
                                          int& t) {
  int xh = cb % g.hx;
  int r = cb / g.hx;
  y = r % g.L[1];
  r /= g.L[1];
  z = r % g.L[2];
  t = r / g.L[2];
  x = 2 * xh + ((y + z + t + p) & 1);
}

// checkerboard index of (x,y,z,t) + k * mu (periodic), lex = lexicographic
// index of (x,y,z,t)
__device__ __forceinline__ int neighbour_cb_s(const Geom& g, int lex, int x, int y, int z, int t,
                                              int mu, int k) {
  const int c = mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t;
  const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
  const int st = mu == 0 ? 1 : mu == 1 ? g.L[0] : mu == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
  int v = c + k;
  while (v >= L) v -= L;
  while (v < 0) v += L;
  return (lex + (v - c) * st) >> 1;
}

// hop table: direction d = 4*mu + q, q = 0..3 -> k = +1, -1, +3, -3
__device__ __forceinline__ int hop_k(int q) { return (q == 0) ? 1 : (q == 1) ? -1 : (q == 2) ? 3 : -3; }

// Solver status word of the device-driven iteration: written by the N x N
// kernels of dense.cu (convergence, reliable-update trigger, breakdown) and by
// bounded waits (time-out), read by the gated kernels and polled by api.cu.
struct SolverStatus {
  int converged_iter;  // iteration at which the iterated residual met tol (or INT_MAX)
  int done;            // 1: true residual verified <= tol
  int ru_pending;      // 1: a reliable update runs after this iteration
  int error;           // blockcg_status code of a device-detected failure
  int iters;           // iterations performed
  int reliable_updates;
  int stopped;         // 1: max_iter iterations done; the gated kernels stop
  int trips;           // device-side loop trips (batched solves)
  double res_max;      // max relative iterated residual after the last iteration
  double res_at_ru;    // max relative residual at the last reliable update
  double true_res_max; // max relative true residual at the last check
  int verified;        // 1: done rests on a native-FP64 true residual
  int fp64_only;       // 1: a double-float convergence failed its FP64
                       // confirmation; all later reliable updates are FP64
};

}  // namespace bcg
