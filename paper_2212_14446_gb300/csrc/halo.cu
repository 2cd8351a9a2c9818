// Spatial decomposition of one periodic system into slabs along an axis (one GPU
// per slab): the device side of the halo exchange.  Not a step of the paper's
// method -- the per-atom evaluation of Sec. 2 split over GPUs.
//
//   pod_halo_select  the atoms whose wrapped coordinate along the axis lies in
//                    [x0, x1), in ascending index order (a stable compaction),
//                    with their positions as the receiving domain lays them out
//                    (the axis coordinate moved by a periodic image shift and the
//                    domain's origin): a rank's own atoms, or the layer within
//                    the list radius of a slab face that a neighbour needs as
//                    ghosts;
//   pod_halo_add     F[:, idx[k]] += G[:, k]: the ghost forces a neighbour sent
//                    back, added onto the owning atoms.
#include <cuda_runtime.h>

#include <cmath>

#include "pod_internal.h"

namespace fastpod {

constexpr int HALO_THREADS = 1024;

// One block walks the atoms in tiles of HALO_THREADS: a block-wide exclusive
// scan of the predicate gives every selected atom its output slot, so the
// output is in ascending atom order whatever the thread count.
__global__ void __launch_bounds__(HALO_THREADS)
    halo_select_kernel(int N, const double* __restrict__ pos, int axis, double L, double x0, double x1, double shift,
                       double offset, int cap, int* __restrict__ idx, double* __restrict__ out,
                       int* __restrict__ count) {
  __shared__ int wsum[HALO_THREADS / 32];
  __shared__ int base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) base = 0;
  __syncthreads();
  for (int t0 = 0; t0 < N; t0 += HALO_THREADS) {
    const int i = t0 + tid;
    double xw = 0.0;
    bool sel = false;
    if (i < N) {
      const double v = pos[(size_t)axis * N + i];
      xw = (v >= 0.0 && v < L) ? v : __dsub_rn(v, __dmul_rn(L, floor(__ddiv_rn(v, L))));
      sel = xw >= x0 && xw < x1;
    }
    const unsigned m = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the warp counts
      int x = lane < HALO_THREADS / 32 ? wsum[lane] : 0;
      int inc = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane < HALO_THREADS / 32) wsum[lane] = inc - x;
    }
    __syncthreads();
    if (sel) {
      const int k = base + wsum[warp] + __popc(m & ((1u << lane) - 1u));
      if (k < cap) {
        idx[k] = i;
        for (int d = 0; d < 3; ++d)
          out[(size_t)d * cap + k] = d == axis ? (xw + shift) - offset : pos[(size_t)d * N + i];
      }
    }
    __syncthreads();
    if (tid == HALO_THREADS - 1) base += wsum[warp] + __popc(m);
    __syncthreads();
  }
  if (tid == 0) *count = base;
}

__global__ void halo_add_kernel(int n, int N, const double* __restrict__ G, const int* __restrict__ idx,
                                double* __restrict__ F, int* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = idx[k];
  if (i < 0 || i >= N) {
    atomicOr(status, ST_REV);
    return;
  }
  for (int d = 0; d < 3; ++d) F[(size_t)d * N + i] += G[(size_t)d * n + k];
}

}  // namespace fastpod

using namespace fastpod;

extern "C" {

int pod_halo_select(pod_handle* h, const double* pos, int n_atoms, int axis, double L, double x0, double x1,
                    double shift, double offset, int cap, int* idx, double* out, int* count, void* stream) {
  NvtxRange nvtx_("pod_halo_select");
  if (!h) return POD_EINVAL;
  if (!pos || !idx || !out || !count) return h->fail(POD_EINVAL, "pod_halo_select: NULL argument");
  if (n_atoms < 0 || cap < 0 || axis < 0 || axis > 2) return h->fail(POD_EINVAL, "pod_halo_select: bad size or axis");
  if (!(L > 0) || !std::isfinite(L)) return h->fail(POD_EINVAL, "pod_halo_select: the box length must be positive");
  if (h->device >= 0) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device)
      return h->fail(POD_EINVAL, "the handle was created on device %d but device %d is current", h->device, cur);
  }
  int rc = h->ensure(h->halo_cnt, sizeof(int), "halo count");
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  halo_select_kernel<<<1, HALO_THREADS, 0, st>>>(n_atoms, pos, axis, L, x0, x1, shift, offset, cap, idx, out,
                                                 (int*)h->halo_cnt.p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h->cuda_fail(e, "halo select kernel");
  int n = 0;
  e = cudaMemcpyAsync(&n, h->halo_cnt.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return h->cuda_fail(e, "halo count read");
  *count = n;
  if (n > cap) return h->fail(POD_ENEIGH, "pod_halo_select: %d atoms selected, capacity %d", n, cap);
  return POD_OK;
}

int pod_halo_add(pod_handle* h, const double* G, const int* idx, int n, double* F, int n_atoms, void* stream) {
  NvtxRange nvtx_("pod_halo_add");
  if (!h) return POD_EINVAL;
  if (n < 0 || n_atoms < 0) return h->fail(POD_EINVAL, "pod_halo_add: bad size");
  if (n == 0) return POD_OK;
  if (!G || !idx || !F) return h->fail(POD_EINVAL, "pod_halo_add: NULL argument");
  if (!h->status.p) {  // the status word starts cleared (read_status clears it after each report)
    int rc = h->ensure(h->status, sizeof(int) * 4, "status");
    if (rc) return rc;
    cudaError_t e0 = cudaMemset(h->status.p, 0, sizeof(int) * 4);
    if (e0 != cudaSuccess) return h->cuda_fail(e0, "status init");
  }
  const int tb = 256;
  halo_add_kernel<<<(n + tb - 1) / tb, tb, 0, (cudaStream_t)stream>>>(n, n_atoms, G, idx, F, (int*)h->status.p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h->cuda_fail(e, "halo add kernel");
  return h->sync ? h->read_status((cudaStream_t)stream) : POD_OK;
}

}  // extern "C"
