// Deterministic force gather, per-atom virial and fixed-order FP64 reductions.
//   F_k = sum_{t in N(k)} ( g[k, t] - g[rev(k, t)] )   (F = -dE/dr, no atomics)
//   W_k = - sum_{t in N(k)} d_kt (x) g[k, t]            (pair virial, summed later)
#include "pod_common.cuh"
#include "pod_kernels.h"

namespace fastpod {

// Warp per atom k, lane per neighbour slot t (coalesced):
//   F_k = sum_t ( g[k, t] - gT[k, t] )
// g[k, t] = dE_k/dr_kt and gT[k, t] = dE_j/dr_jk of the reverse pair, written by
// the atom kernel (no atomics).  Per-block FP64 partials of E = sum_i E_i and of
// the virial partials are summed in a fixed order by the last block to finish,
// so every result is bitwise reproducible.
constexpr int WPB_GATHER = 8;

template <typename T>
__global__ void __launch_bounds__(WPB_GATHER * 32)
    gather_reduce_kernel(int N, int cap, const int* __restrict__ nbr_count, const Q4<T>* __restrict__ g,
                         const Q4<T>* __restrict__ gT, const double* __restrict__ Ei,
                         const double* __restrict__ wpart, int n_wpart, double* __restrict__ F, double fscale,
                         double* __restrict__ part, unsigned* __restrict__ ticket, double* __restrict__ E_out,
                         double* __restrict__ W_out, int* __restrict__ status) {
  __shared__ double sred[WPB_GATHER][10];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q] = 0.0;
  for (int k = blockIdx.x * WPB_GATHER + warp; k < N; k += gridDim.x * WPB_GATHER) {
    const int n = min(nbr_count[k], cap);
    T f0 = T(0), f1 = T(0), f2 = T(0);
    for (int t = lane; t < n; t += 32) {
      const size_t p = (size_t)k * cap + t;
      const Q4<T> a = g[p], b = gT[p];
      f0 += a.x - b.x;
      f1 += a.y - b.y;
      f2 += a.z - b.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f0 += __shfl_xor_sync(0xffffffffu, f0, o);
      f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    }
    if (lane == 0) {
      if (F) {
        F[k] = fscale * (double)f0;
        F[(size_t)N + k] = fscale * (double)f1;
        F[(size_t)2 * N + k] = fscale * (double)f2;
      }
      if (!(isfinite((double)f0) && isfinite((double)f1) && isfinite((double)f2))) atomicOr(status, ST_NONFINITE);
      acc[0] += Ei[k];
    }
  }
  // virial partials of the atom kernel, a fixed subset per warp of this block
  if (lane < 9)
    for (int w = blockIdx.x * WPB_GATHER + warp; w < n_wpart; w += gridDim.x * WPB_GATHER)
      acc[1 + lane] += wpart[(size_t)w * 9 + lane];
  // fold the per-lane virial components into lane 0's slot order
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const double v = __shfl_sync(0xffffffffu, acc[1 + q], q);
    if (lane == 0) acc[1 + q] = v;
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 10; ++q) sred[warp][q] = acc[q];
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double s = 0.0;
    for (int wv = 0; wv < WPB_GATHER; ++wv) s += sred[wv][threadIdx.x];
    part[(size_t)blockIdx.x * 10 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order parallel sum of the block partials: thread t adds blocks
  // t, t + blockDim, ... in order (independent L2 loads), then one fixed tree
  double s[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) s[q] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < 10; ++q) s[q] += __ldcg(part + (size_t)b * 10 + q);
  }
  __shared__ double fin2[10][WPB_GATHER * 32];
#pragma unroll
  for (int q = 0; q < 10; ++q) fin2[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 10; ++q) fin2[q][threadIdx.x] += fin2[q][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) E_out[0] = fin2[0][0];
  if (W_out && threadIdx.x >= 1 && threadIdx.x < 10) W_out[threadIdx.x - 1] = fin2[threadIdx.x][0];
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch (graph replays)
}

template <typename T>
cudaError_t launch_gather_reduce(int N, int cap, const int* nbr_count, const Q4<T>* g, const Q4<T>* gT,
                                 const double* Ei, const double* wpart, int n_wpart, double* F, double fscale,
                                 double* part, int nblocks, unsigned* ticket, double* E, double* W, int* status,
                                 cudaStream_t st) {
  gather_reduce_kernel<T><<<nblocks, WPB_GATHER * 32, 0, st>>>(N, cap, nbr_count, g, gT, Ei, wpart, n_wpart, F,
                                                               fscale, part, ticket, E, W, status);
  return cudaGetLastError();
}

int gather_blocks(int N) {
  const int want = (N + WPB_GATHER - 1) / WPB_GATHER;
  return want < 8 * 152 ? (want > 0 ? want : 1) : 8 * 152;
}

template cudaError_t launch_gather_reduce<float>(int, int, const int*, const Q4<float>*, const Q4<float>*,
                                                 const double*, const double*, int, double*, double, double*, int,
                                                 unsigned*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_gather_reduce<double>(int, int, const int*, const Q4<double>*, const Q4<double>*,
                                                  const double*, const double*, int, double*, double, double*, int,
                                                  unsigned*, double*, double*, int*, cudaStream_t);

}  // namespace fastpod
