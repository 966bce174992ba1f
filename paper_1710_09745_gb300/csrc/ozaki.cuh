// Exact split products on the bf16 tensor cores (Ozaki's scheme) for the
// double-float kernels: a scaled double-float value in (-1, 1) is written as
// six bf16 slices on the grids 2^(-7-8k); products of slices are exact in
// bf16 x bf16 -> FP32, and the products whose slice indices sum to u share
// one power-of-two grid, so their FP32 sum is exact while it stays below
// 2^24 units.  Used by the tensor-core stencil (stencil_tc.cu) and the
// tensor-core double-float block update (blas_tc.cu).
#pragma once
#include "common.cuh"

namespace bcg {
namespace ozaki {

__device__ __forceinline__ float rnd_grid(float x, float c) {  // x to the grid ulp(c)
  return __fsub_rn(__fadd_rn(x, c), c);
}

// six bf16-exact slices of a scaled double-float value h + l, |h + l| < 1:
// slice k on the grid 2^(-7-8k) (rounding to nearest by adding and removing
// c_k = 1.5 * 2^(16-8k)); every step but the (hi remainder + lo) sum is exact
__device__ __forceinline__ void split6(float h, float l, float (&s)[6]) {
  s[0] = rnd_grid(h, 98304.f);  // 1.5 * 2^16
  float r = __fsub_rn(h, s[0]);
  s[1] = rnd_grid(r, 384.f);  // 1.5 * 2^8
  r = __fsub_rn(r, s[1]);
  s[2] = rnd_grid(r, 1.5f);
  r = __fsub_rn(r, s[2]);
  r = __fadd_rn(r, l);
  s[3] = rnd_grid(r, 0.005859375f);  // 1.5 * 2^-8
  r = __fsub_rn(r, s[3]);
  s[4] = rnd_grid(r, 2.288818359375e-05f);  // 1.5 * 2^-16
  r = __fsub_rn(r, s[4]);
  s[5] = rnd_grid(r, 8.940696716308594e-08f);  // 1.5 * 2^-24
}

// (lo, hi) -> one register of two bf16 (lo in the low half: the element
// with the smaller k of an MMA fragment pair); exact for slice values
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// smallest e with |v| < 2^e for the non-negative float with bit pattern b,
// clamped to [-120, 120] (0 and denormals give -126 -> -120; inf/NaN 120,
// which keeps them non-finite after scaling)
__device__ __forceinline__ int pow2_above(unsigned b) {
  const int e = (int)((b >> 23) & 0xffu) - 126;
  return e < -120 ? -120 : e > 120 ? 120 : e;
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

// D = sum_u D_u in double-float
__device__ __forceinline__ dfacc combine6(float d0, float d1, float d2, float d3, float d4,
                                          float d5) {
  float h, l, e2;
  two_sum(d0, d1, h, l);
  two_sum(h, d2, h, e2);
  l = __fadd_rn(l, __fadd_rn(e2, __fadd_rn(__fadd_rn(d5, d4), d3)));
  const float s = __fadd_rn(h, l);  // fast two-sum: |h| >= |l|
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}

}  // namespace ozaki
}  // namespace bcg
