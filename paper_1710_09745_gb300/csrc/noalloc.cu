// blockcg_block_cdot_noalloc: K = X^dag Y with no device allocation at all.
//
// Some callers cannot allocate device memory: code that runs inside a memory
// pool it does not own, plug-ins of host applications that hand over only
// their own buffers, or programs that must not call cudaMalloc because it can
// synchronise the device.  For them this entry point keeps its scratch (the
// per-CTA partial sums of the Gram reduction) in a fixed array in the
// library's own device image, so the caller provides only X, Y, K and a
// stream.  Every GPU that loads the library holds that array (4 MiB) until
// the process exits.
//
// Host code must not hand the kernels the array's name: on the host it is a
// stand-in symbol, not a device address.  The device address is looked up
// once per device with cudaGetSymbolAddress, with that device current, on the
// first call made while it is current, and cached with the device's SM count.
// The cache is not invalidated: after cudaDeviceReset the cached address
// belongs to a context that no longer exists, so a process that resets a
// device must not call this entry point on it again.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/blockcg.h"
#include "internal.h"

namespace bcg {

static constexpr int NOALLOC_SCRATCH_ELEMS = 262144;  // double2 -> 4 MiB
static constexpr int NOALLOC_THREADS = 256;
static constexpr int NOALLOC_MAX_EPT = 16;
static constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH_ELEMS];

// Per-CTA partial sums of K = X^dag Y on the user layout [N][Vh][3]
// complex128, native FP64.  Each CTA writes all N*N of its entries, so the
// scratch needs no clearing between calls.
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_cdot_user(const double2* __restrict__ X, const double2* __restrict__ Y, int N, long long rows,
                double2* __restrict__ partials) {
  __shared__ double2 red[NOALLOC_THREADS];
  const int E = N * N;
  const int tid = threadIdx.x;
  const int G = (E >= NOALLOC_THREADS) ? 1 : (NOALLOC_THREADS / E);
  const int grp = tid / (E < NOALLOC_THREADS ? E : NOALLOC_THREADS);
  const long long rpb = (rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * rpb;
  const long long r1 = min(rows, r0 + rpb);
  int ne = 0;
  int ei[NOALLOC_MAX_EPT], ej[NOALLOC_MAX_EPT];
  double2 acc[NOALLOC_MAX_EPT];
  if (grp < G) {
    int e0 = (E < NOALLOC_THREADS) ? (tid % E) : tid;
    for (int e = e0; e < E && ne < NOALLOC_MAX_EPT; e += NOALLOC_THREADS) {
      ei[ne] = e / N;
      ej[ne] = e % N;
      acc[ne] = make_double2(0.0, 0.0);
      ++ne;
    }
    for (long long r = r0 + grp; r < r1; r += G) {
      for (int q = 0; q < ne; ++q) {
        double2 x = X[(long long)ei[q] * rows + r];
        double2 y = Y[(long long)ej[q] * rows + r];
        acc[q].x = fma(x.x, y.x, fma(x.y, y.y, acc[q].x));
        acc[q].y = fma(x.x, y.y, fma(-x.y, y.x, acc[q].y));
      }
    }
  }
  double2* out = partials + (long long)blockIdx.x * E;
  if (G == 1) {
    for (int q = 0; q < ne; ++q) out[tid + q * NOALLOC_THREADS] = acc[q];
    return;
  }
  red[tid] = (grp < G && ne > 0) ? acc[0] : make_double2(0.0, 0.0);
  __syncthreads();
  if (tid < E) {
    double2 s = red[tid];
    for (int g2 = 1; g2 < G; ++g2) {
      s.x += red[g2 * E + tid].x;
      s.y += red[g2 * E + tid].y;
    }
    out[tid] = s;
  }
}

static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];
static int g_noalloc_sms[NOALLOC_MAX_DEVICES];

// Device address of the scratch array and SM count of the current device
// (looked up once per device).
static cudaError_t noalloc_scratch_address(void** out, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_noalloc_sms[dev] = n > 0 ? n : 1;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  *sms = g_noalloc_sms[dev];
  return cudaSuccess;
}

}  // namespace bcg

extern "C" blockcg_status blockcg_block_cdot_noalloc(const void* X, const void* Y, int n_rhs,
                                                     long long vh, void* K, void* stream) {
  using namespace bcg;
  if (!X || !Y || !K || vh < 1) return BLOCKCG_ERR_ARG;
  if (n_rhs < 1 || n_rhs > 64) return BLOCKCG_ERR_ARG;  // 64 x 64 partials per CTA at most
  const int N = n_rhs;
  const long long rows = 3LL * vh;
  void* scratch = nullptr;
  int sms = 1;
  if (noalloc_scratch_address(&scratch, &sms) != cudaSuccess) return BLOCKCG_ERR_CUDA;
  // as many CTAs as the scratch holds partial matrices for, up to 4 per SM
  int nblocks = NOALLOC_SCRATCH_ELEMS / (N * N);
  if (nblocks > 4 * sms) nblocks = 4 * sms;
  long long by_rows = (rows + 63) / 64;
  if (nblocks > by_rows) nblocks = (int)by_rows;
  if (nblocks < 1) nblocks = 1;
  cudaStream_t s = (cudaStream_t)stream;
  k_cdot_user<<<nblocks, NOALLOC_THREADS, 0, s>>>((const double2*)X, (const double2*)Y, N, rows,
                                                  (double2*)scratch);
  if (cudaGetLastError() != cudaSuccess) return BLOCKCG_ERR_CUDA;
  Gate g0{nullptr, GATE_ALWAYS};
  if (gram_reduce((const double2*)scratch, nblocks, N, 0, (double2*)K, g0, s) != cudaSuccess)
    return BLOCKCG_ERR_CUDA;
  return BLOCKCG_OK;
}
