// Vector-pipe throughput probe: the denominator of the atom kernel's roofline.
// The fused atom kernel is bound by the FP32 (mixed path) or FP64 (FP64 path)
// fused multiply-add pipes, whose peak is not a published figure for this part;
// this kernel measures it on the device at hand.  Every thread runs CHAINS
// independent FMA chains (enough to hide the pipe latency) for `iters`
// iterations; the result is stored only under a condition the inputs never meet,
// so the work cannot be elided.
#include <cuda_runtime.h>

#include "pod_internal.h"

using namespace fastpod;

static __device__ float g_fma_sink;

namespace {
constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 8;

__global__ void __launch_bounds__(PEAK_THREADS) fma_f32_kernel(int iters, float x, float y) {
  float a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) a[c] = fmaf(a[c], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  if (s == -1.0f) g_fma_sink = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) fma_f32x2_kernel(int iters, float x, float y) {
  float2 a[CHAINS / 2];
#pragma unroll
  for (int c = 0; c < CHAINS / 2; ++c) a[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
  const float2 xx = make_float2(x, x), yy = make_float2(y, y);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS / 2; ++c) a[c] = __ffma2_rn(a[c], xx, yy);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS / 2; ++c) s += a[c].x + a[c].y;
  if (s == -1.0f) g_fma_sink = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) fma_f64_kernel(int iters, double x, double y) {
  double a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  if (s == -1.0) g_fma_sink = (float)s;
}
}  // namespace

extern "C" int pod_fma_probe(int kind, int iters, double* flops, void* stream) {
  if (kind < 0 || kind > 2 || iters < 1 || !flops) return POD_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return POD_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return POD_ECUDA;
  const int blocks = nsm * (2048 / PEAK_THREADS);
  cudaStream_t st = (cudaStream_t)stream;
  const float xf = 0.999999f, yf = 1e-7f;
  if (kind == 0)
    fma_f32_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, xf, yf);
  else if (kind == 1)
    fma_f32x2_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, xf, yf);
  else
    fma_f64_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.999999999, 1e-12);
  if (cudaGetLastError() != cudaSuccess) return POD_ECUDA;
  *flops = 2.0 * 16.0 * CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
  return POD_OK;
}
