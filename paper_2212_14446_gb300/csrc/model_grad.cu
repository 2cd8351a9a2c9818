// Parameter gradients of a force-matching loss (Eq. 63b) for the linear,
// quadratic and embedding models, from per-atom descriptors D_i (Eq. 12b, 26a,
// 27a, 30a) and their directional derivatives Ddot_i = sum_k (dD_i/dr_k) . v_k.
//
// For a loss L(theta) = sum_c w_E^2 ((E_c - E_c^ref) / N_c)^2
//                     + w_F^2 sum_k |F_k - F_k^ref|^2
// the gradient is dL/dtheta = sum_i w_i dE_i/dtheta + t d/de[dE/dtheta](r + e v)
// with v = F - F^ref, w_i = 2 w_E^2 (E_c - E_c^ref) / N_c^2 for the atoms i of
// configuration c and t = -2 w_F^2 (F = -dE/dr, so the force term is minus the
// directional derivative of dE/dtheta along v).  Per model:
//   linear     dE_i/dc_m = D_im
//   quadratic  dE_i/dbeta_mn = D_im D_in (m <= n)
//   embedding  dE_i/da_m = F'(rho_i) D_im, dE_i/dalpha_k = rho_i^k, rho_i = a . D_i
// and the directional derivatives follow by the product and chain rules with
// Ddot_i and rhodot_i = a . Ddot_i.
//
// Every output is a sum over atoms: blocks take chunks of atoms and write
// per-block partial sums, reduced afterwards in block order (deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "pod_internal.h"

namespace fastpod {

constexpr int MG_THREADS = 256;
constexpr int MG_ROWS = 16;  // atoms staged in shared memory per step

// part[bx][e] over the atoms of chunk bx (grid.x) for the outputs e of tile by
// (grid.y, one output per thread): e < M the linear part, then the quadratic
// upper triangle (model 1) or the embedding terms (model 2: a, then alpha).
// Shared memory: MG_ROWS rows of D and Ddot (2 MG_ROWS M doubles).
__global__ void __launch_bounds__(MG_THREADS)
    model_grad_partial_kernel(int N, int M, int model, int deg, const double* __restrict__ D,
                              const double* __restrict__ Dd, const double* __restrict__ w, double t,
                              const double* __restrict__ emb, int nout, int rows_per_block,
                              double* __restrict__ part) {
  extern __shared__ double mg[];
  double* sD = mg;
  double* sDd = mg + (size_t)MG_ROWS * M;
  __shared__ double sw[MG_ROWS], sF1[MG_ROWS], sF2[MG_ROWS], srho[MG_ROWS], srd[MG_ROWS];
  const int tid = threadIdx.x;
  const int e = blockIdx.y * MG_THREADS + tid;
  const int i0 = blockIdx.x * rows_per_block;
  const int i1 = min(N, i0 + rows_per_block);
  // what output e is: 0 linear c_e; 1 quadratic (m, n); 2 embedding a_m; 3 embedding alpha_pw
  int kind = 0, m = e, n = 0, pw = 0;
  if (e >= M) {
    if (model == 1) {
      kind = 1;
      int k = e - M;
      m = 0;
      while (m < M && k >= M - m) {
        k -= M - m;
        ++m;
      }
      n = m + k;
    } else if (e - M < M) {
      kind = 2;
      m = e - M;
    } else {
      kind = 3;
      pw = e - 2 * M;
    }
  }
  const bool live = e < nout;
  double s = 0.0;
  for (int r0 = i0; r0 < i1; r0 += MG_ROWS) {
    const int nr = min(MG_ROWS, i1 - r0);
    __syncthreads();
    for (int q = tid; q < nr * M; q += MG_THREADS) {
      sD[q] = D[(size_t)r0 * M + q];
      sDd[q] = Dd[(size_t)r0 * M + q];
    }
    if (tid < nr) sw[tid] = w[r0 + tid];
    __syncthreads();
    if (model == 2 && tid < nr) {  // rho, rhodot, F'(rho), F''(rho) by Horner's rule
      double rho = 0.0, rd = 0.0;
      for (int c = 0; c < M; ++c) {
        rho = fma(emb[c], sD[tid * M + c], rho);
        rd = fma(emb[c], sDd[tid * M + c], rd);
      }
      const double* al = emb + M;
      double f1 = 0.0, f2 = 0.0;
      for (int k = deg; k >= 1; --k) f1 = fma(f1, rho, k * al[k]);
      for (int k = deg; k >= 2; --k) f2 = fma(f2, rho, (double)k * (k - 1) * al[k]);
      srho[tid] = rho;
      srd[tid] = rd;
      sF1[tid] = f1;
      sF2[tid] = f2;
    }
    __syncthreads();
    if (!live) continue;
    for (int r = 0; r < nr; ++r) {
      const double wi = sw[r];
      const double* Dr = sD + r * M;
      const double* Ddr = sDd + r * M;
      if (kind == 0) {
        s = fma(wi, Dr[m], fma(t, Ddr[m], s));
      } else if (kind == 1) {
        s = fma(wi, Dr[m] * Dr[n], fma(t, fma(Ddr[m], Dr[n], Dr[m] * Ddr[n]), s));
      } else if (kind == 2) {
        s = fma(wi * sF1[r], Dr[m], fma(t, fma(sF2[r] * srd[r], Dr[m], sF1[r] * Ddr[m]), s));
      } else {
        double rp = 1.0, rpm1 = 0.0;  // rho^pw and rho^(pw - 1)
        for (int u = 0; u < pw; ++u) {
          rpm1 = rp;
          rp *= srho[r];
        }
        s = fma(wi, rp, fma(t, pw * rpm1 * srd[r], s));
      }
    }
  }
  if (live) part[(size_t)blockIdx.x * nout + e] = s;
}

__global__ void model_grad_reduce_kernel(int nblk, int nout, const double* __restrict__ part,
                                         double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nout) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * nout + e];
  out[e] = s;
}

}  // namespace fastpod

using namespace fastpod;

extern "C" {

int pod_descriptors_tangent(pod_handle* h, const pod_system* sys, const double* v, double* Ddot, void* stream) {
  NvtxRange nvtx_("pod_descriptors_tangent");
  if (!h) return POD_EINVAL;
  if (!v || !Ddot) return h->fail(POD_EINVAL, "direction v and Ddot are required");
  return h->global_desc(sys, v, nullptr, (cudaStream_t)stream, Ddot);
}

int pod_model_gradients(pod_handle* h, int n_atoms, const double* D, const double* Ddot, const double* w, double t,
                        double* grad, void* stream) {
  NvtxRange nvtx_("pod_model_gradients");
  if (!h) return POD_EINVAL;
  if (n_atoms < 1 || !D || !Ddot || !w || !grad) return h->fail(POD_EINVAL, "pod_model_gradients: bad argument");
  if (!std::isfinite(t)) return h->fail(POD_EINVAL, "pod_model_gradients: t must be finite");
  if (h->device >= 0) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device)
      return h->fail(POD_EINVAL, "the handle was created on device %d but device %d is current", h->device, cur);
  }
  const int M = h->M;
  const int model = h->quad ? 1 : (h->emb_deg > 0 ? 2 : 0);
  const int deg = h->emb_deg;
  const int nout = M + (model == 1 ? M * (M + 1) / 2 : (model == 2 ? M + deg + 1 : 0));
  const int rows_per_block = 256;
  const int nblk = (n_atoms + rows_per_block - 1) / rows_per_block;
  int rc = h->ensure(h->mgrad, sizeof(double) * ((size_t)nblk * nout + nout), "model gradient partials");
  if (rc) return rc;
  double* part = (double*)h->mgrad.p;
  double* out = part + (size_t)nblk * nout;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = sizeof(double) * 2 * (size_t)MG_ROWS * M;
  static size_t granted[64] = {};
  cudaError_t e = grant_smem((const void*)model_grad_partial_kernel, smem, granted);
  if (e == cudaSuccess) {
    const dim3 grid(nblk, (nout + MG_THREADS - 1) / MG_THREADS);
    model_grad_partial_kernel<<<grid, MG_THREADS, smem, st>>>(n_atoms, M, model, deg, D, Ddot, w, t,
                                                              (const double*)h->embW.p, nout, rows_per_block, part);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    model_grad_reduce_kernel<<<(nout + 255) / 256, 256, 0, st>>>(nblk, nout, part, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return h->cuda_fail(e, "model gradients");
  return POD_OK;
}

}  // extern "C"
