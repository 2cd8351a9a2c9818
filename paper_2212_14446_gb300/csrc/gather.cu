// Deterministic force gather, per-atom virial and fixed-order FP64 reductions.
//   F_k = sum_{t in N(k)} ( g[k, t] - g[rev(k, t)] )   (F = -dE/dr, no atomics)
//   W_k = - sum_{t in N(k)} d_kt (x) g[k, t]            (pair virial, summed later)
#include "pod_common.cuh"
#include "pod_kernels.h"

namespace fastpod {

template <typename T>
__device__ __forceinline__ void gather_disp(int N, int i, int j, int code, const double* wpos, const float4* phi,
                                            const float4* plo, const double* L, const float* Lh, const float* Ll,
                                            T& dx, T& dy, T& dz);

template <>
__device__ __forceinline__ void gather_disp<double>(int N, int i, int j, int code, const double* wpos,
                                                    const float4*, const float4*, const double* L, const float*,
                                                    const float*, double& dx, double& dy, double& dz) {
  int sx, sy, sz;
  shift_unpack(code, sx, sy, sz);
  dx = disp_fp64(wpos[i], wpos[j], sx, L[0]);
  dy = disp_fp64(wpos[(size_t)N + i], wpos[(size_t)N + j], sy, L[1]);
  dz = disp_fp64(wpos[(size_t)2 * N + i], wpos[(size_t)2 * N + j], sz, L[2]);
}

template <>
__device__ __forceinline__ void gather_disp<float>(int, int i, int j, int code, const double*, const float4* phi,
                                                   const float4* plo, const double*, const float* Lh,
                                                   const float* Ll, float& dx, float& dy, float& dz) {
  int sx, sy, sz;
  shift_unpack(code, sx, sy, sz);
  const float4 hi = phi[i], li = plo[i], hj = phi[j], lj = plo[j];
  dx = disp_f32(hi.x, li.x, hj.x, lj.x, sx, Lh[0], Ll[0]);
  dy = disp_f32(hi.y, li.y, hj.y, lj.y, sy, Lh[1], Ll[1]);
  dz = disp_f32(hi.z, li.z, hj.z, lj.z, sz, Lh[2], Ll[2]);
}

struct BoxArgs {
  double L[3];
  float Lh[3], Ll[3];
};

template <typename T>
__global__ void gather_kernel(int N, int cap, const int* __restrict__ nbr_count, const int* __restrict__ nbr_j,
                              const int* __restrict__ nbr_s, const int* __restrict__ rev,
                              const Q4<T>* __restrict__ g, const double* __restrict__ wpos,
                              const float4* __restrict__ phi, const float4* __restrict__ plo, BoxArgs bx,
                              double* __restrict__ F, double* __restrict__ Wat, int* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int n = min(nbr_count[k], cap);
  double fx = 0, fy = 0, fz = 0;
  T w[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) w[q] = T(0);
  bool finite = true;
  for (int t = 0; t < n; ++t) {
    const size_t p = (size_t)k * cap + t;
    const Q4<T> a = g[p];
    const Q4<T> b = g[rev[p]];
    fx += (double)a.x - (double)b.x;
    fy += (double)a.y - (double)b.y;
    fz += (double)a.z - (double)b.z;
    T dx, dy, dz;
    gather_disp<T>(N, k, nbr_j[p], nbr_s[p], wpos, phi, plo, bx.L, bx.Lh, bx.Ll, dx, dy, dz);
    w[0] -= dx * a.x; w[1] -= dx * a.y; w[2] -= dx * a.z;
    w[3] -= dy * a.x; w[4] -= dy * a.y; w[5] -= dy * a.z;
    w[6] -= dz * a.x; w[7] -= dz * a.y; w[8] -= dz * a.z;
  }
  finite = isfinite(fx) && isfinite(fy) && isfinite(fz);
  if (!finite) atomicOr(status, ST_NONFINITE);
  if (F) {
    F[k] = fx;
    F[(size_t)N + k] = fy;
    F[(size_t)2 * N + k] = fz;
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) Wat[(size_t)k * 9 + q] = (double)w[q];
}

// One block per configuration: E = sum_i E_i and W = sum_i W_i in FP64, each
// thread summing a strided subsequence in order, then a fixed tree.
__global__ void reduce_kernel(const int* __restrict__ offs, const double* __restrict__ Ei,
                              const double* __restrict__ Wat, double* __restrict__ E, double* __restrict__ W) {
  __shared__ double red[10][256];
  const int c = blockIdx.x;
  const int a0 = offs[c], a1 = offs[c + 1];
  double acc[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q] = 0.0;
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    acc[0] += Ei[i];
    if (Wat) {
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[1 + q] += Wat[(size_t)i * 9 + q];
    }
  }
#pragma unroll
  for (int q = 0; q < 10; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 10; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    E[c] = red[0][0];
    if (W) {
#pragma unroll
      for (int q = 0; q < 9; ++q) W[(size_t)c * 9 + q] = red[1 + q][0];
    }
  }
}

template <typename T>
cudaError_t launch_gather(int N, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s,
                          const int* rev, const Q4<T>* g, const double* wpos, const float4* phi, const float4* plo,
                          const double L[3], double* F, double* Wat, int* status, cudaStream_t st) {
  BoxArgs bx;
  for (int d = 0; d < 3; ++d) {
    bx.L[d] = L[d];
    bx.Lh[d] = (float)L[d];
    bx.Ll[d] = (float)(L[d] - (double)bx.Lh[d]);
  }
  const int tb = 128;
  gather_kernel<T><<<(N + tb - 1) / tb, tb, 0, st>>>(N, cap, nbr_count, nbr_j, nbr_s, rev, g, wpos, phi, plo, bx,
                                                     F, Wat, status);
  return cudaGetLastError();
}

template cudaError_t launch_gather<float>(int, int, const int*, const int*, const int*, const int*,
                                          const Q4<float>*, const double*, const float4*, const float4*,
                                          const double*, double*, double*, int*, cudaStream_t);
template cudaError_t launch_gather<double>(int, int, const int*, const int*, const int*, const int*,
                                           const Q4<double>*, const double*, const float4*, const float4*,
                                           const double*, double*, double*, int*, cudaStream_t);

cudaError_t launch_reduce(int n_cfg, const int* cfg_offs, const double* Ei, const double* Wat, double* E, double* W,
                          cudaStream_t st) {
  reduce_kernel<<<n_cfg, 256, 0, st>>>(cfg_offs, Ei, Wat, E, W);
  return cudaGetLastError();
}

}  // namespace fastpod
