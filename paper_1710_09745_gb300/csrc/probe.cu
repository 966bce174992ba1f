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
