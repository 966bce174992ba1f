// blockcg_bench_alu: measured arithmetic issue rates of the current GPU, the
// denominators behind the double-float stencil's arithmetic roofline.
//
// The FP64-accurate solver form computes in double-float on the FP32 pipes
// (common.cuh); its stencil is bound by FP32 instruction issue, not by HBM.
// This probe times long chains of independent fused multiply-adds per thread
// (8 chains, so that the pipeline latency is hidden) on a grid of several
// resident blocks per SM, once in FP32 and once in FP64, and returns the
// multiply-adds per second of each.  A chain's result is stored only if it
// equals an impossible value, so the compiler keeps every multiply-add.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/blockcg.h"

namespace bcg {

static __device__ float g_probe_sink_f;
static __device__ double g_probe_sink_d;

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b) {
  T c[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = fma(c[k], a, b);
  }
  T s = c[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) s += c[k];
  if (s == (T)-1.2345e-30) {
    if (sizeof(T) == 4) g_probe_sink_f = (float)s;
    else g_probe_sink_d = (double)s;
  }
}

// multiply-adds per second of one chain kernel, timed with events
template <class T>
static cudaError_t time_chains(cudaStream_t s, int blocks, int iters, double* per_s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    // a ~1.0 multiplier keeps the chains finite over any iteration count
    const T a = (T)0.99999, b = (T)1e-7;
    k_fma_chains<T><<<blocks, 256, 0, s>>>(iters / 8, a, b);  // warm-up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) k_fma_chains<T><<<blocks, 256, 0, s>>>(iters, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) *per_s = (double)blocks * 256 * 8 * (double)iters / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace bcg

extern "C" blockcg_status blockcg_bench_alu(void* stream, double* fp32_fma_per_s,
                                            double* fp64_fma_per_s, int* sm_count) {
  using namespace bcg;
  if (!fp32_fma_per_s || !fp64_fma_per_s || !sm_count) return BLOCKCG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return BLOCKCG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // 8 blocks of 256 threads per SM: 64 warps, the SM's full complement
  const int blocks = sms * 8;
  if (time_chains<float>(s, blocks, 1 << 16, fp32_fma_per_s) != cudaSuccess) return BLOCKCG_ERR_CUDA;
  if (time_chains<double>(s, blocks, 1 << 12, fp64_fma_per_s) != cudaSuccess) return BLOCKCG_ERR_CUDA;
  *sm_count = sms;
  return BLOCKCG_OK;
}

// ---------------------------------------------------------------------------
// blockcg_bench_mma: measured rate of the warp-level bf16 tensor-core
// product (mma.sync m16n8k16, FP32 accumulation), the instruction the
// tensor-core double-float stencil issues.  Each warp runs 4 independent
// accumulator chains on register operands (no memory traffic), 8 blocks of
// 256 threads per SM; a chain's result is stored only if it equals an
// impossible value.
namespace bcg {

static __device__ float g_probe_sink_mma;

__global__ void __launch_bounds__(256) k_mma_chains(int iters, uint32_t a0, uint32_t b0) {
  float d[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) d[c][i] = 0.f;
  const uint32_t a1 = a0 ^ (threadIdx.x & 1u), b1 = b0 ^ (threadIdx.x & 2u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};\n"
          : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
          : "r"(a0), "r"(a1), "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) s += d[c][i];
  if (s == -1.2345e-30f) g_probe_sink_mma = s;
}

}  // namespace bcg

extern "C" blockcg_status blockcg_bench_mma(void* stream, double* bf16_flop_per_s) {
  using namespace bcg;
  if (!bf16_flop_per_s) return BLOCKCG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return BLOCKCG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sms * 8, iters = 1 << 14;
  // bf16 operands 1.0 and 2^-20 (bit patterns): the sums stay finite
  const uint32_t a = 0x3f803f80u, b = 0x35803580u;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_mma_chains<<<blocks, 256, 0, s>>>(iters / 8, a, b);  // warm-up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) k_mma_chains<<<blocks, 256, 0, s>>>(iters, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.f)) return BLOCKCG_ERR_CUDA;
  // 16 x 8 x 16 multiply-adds = 4096 flops per warp instruction
  *bf16_flop_per_s = (double)blocks * 8 /* warps */ * 4 /* chains */ * (double)iters * 4096.0 /
                     (ms * 1e-3);
  return BLOCKCG_OK;
}
