// Batches of independent configurations stored back to back (training sets):
// per-atom wrap with the atom's own box, a neighbour search restricted to the
// atom's configuration (all images within r_cut), and per-configuration sums.
#include "pod_common.cuh"
#include "pod_kernels.h"

namespace fastpod {

__global__ void batch_wrap_kernel(int N, const double* __restrict__ pos, const int* __restrict__ cfg_of,
                                  const CfgBox* __restrict__ cbox, double* __restrict__ wpos,
                                  float4* __restrict__ phi, float4* __restrict__ plo, int* __restrict__ status,
                                  unsigned long long* __restrict__ facc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (facc) {  // fixed-point force, energy and virial accumulators of this call start at zero
    ulonglong2* fz = reinterpret_cast<ulonglong2*>(facc + 4 * (size_t)i);
    fz[0] = make_ulonglong2(0ull, 0ull);
    fz[1] = make_ulonglong2(0ull, 0ull);
    ulonglong2* tz = reinterpret_cast<ulonglong2*>(facc + 4 * (size_t)N);
    for (int q = i; q < FACC_TAIL / 2; q += N) tz[q] = make_ulonglong2(0ull, 0ull);
  }
  const CfgBox& b = cbox[cfg_of[i]];
  double x[3];
  bool finite = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = pos[(size_t)d * N + i];
    finite = finite && isfinite(v);
    if (b.pbc[d]) v = __dsub_rn(v, __dmul_rn(b.L[d], floor(__ddiv_rn(v, b.L[d]))));
    x[d] = v;
    wpos[(size_t)d * N + i] = v;
  }
  if (!finite) atomicOr(status, ST_NONFINITE);
  float h[3], l[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    h[d] = __double2float_rn(x[d]);
    l[d] = __double2float_rn(x[d] - (double)h[d]);
  }
  phi[i] = make_float4(h[0], h[1], h[2], 0.f);
  plo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// Warp per atom: every atom j of the same configuration and every image s with
// |s_d| <= S_d is a candidate; FP32 prefilter, exact FP64 decision in the band
// (the same definition as the cell-list kernels), hits sorted by (j, s).
__global__ void __launch_bounds__(WPB_NEIGH * 32)
    batch_neigh_kernel(int N, const int* __restrict__ cfg_of, const CfgBox* __restrict__ cbox,
                       const double* __restrict__ wpos, const float4* __restrict__ phi, double rc2, float rc2_lo,
                       float rc2_hi, int cap, int keycap, int* __restrict__ nbr_count, int* __restrict__ nbr_j,
                       int* __restrict__ nbr_s, int* __restrict__ status) {
  extern __shared__ unsigned long long bsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* keys = bsm + (size_t)warp * keycap;
  const int i = blockIdx.x * WPB_NEIGH + warp;
  if (i >= N) return;
  const CfgBox b = cbox[cfg_of[i]];
  const float4 hi = phi[i];
  const float Lh[3] = {(float)b.L[0], (float)b.L[1], (float)b.L[2]};
  // images whose box comes within r_cut of this atom (a conservative superset:
  // the margin covers the FP32 position and the band; the exact test decides)
  int smin[3], smax[3];
  {
    const float rcm = sqrtf(rc2_hi) * 1.0001f + 1e-4f;
    const float xi[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (b.S[d] == 0) {
        smin[d] = smax[d] = 0;
      } else {
        smin[d] = max(-b.S[d], (int)floorf((xi[d] - rcm) / Lh[d]));
        smax[d] = min(b.S[d], (int)floorf((xi[d] + rcm) / Lh[d]));
      }
    }
  }
  const int wx = smax[0] - smin[0] + 1, wy = smax[1] - smin[1] + 1, wz = smax[2] - smin[2] + 1;
  const int nimg = wx * wy * wz;
  const int nat = b.a1 - b.a0;
  const int total = nimg * nat;
  const int zero = shift_pack(0, 0, 0);
  int nhit = 0;
  // candidate j under image (sx, sy, sz): the FP32 prefilter, the exact FP64 band
  // decision, and its key
  auto test = [&](int j, int sx, int sy, int sz, int code, unsigned long long& key) {
    if (j == i && code == zero) return false;
    const float4 hj = phi[j];
    const float dx = (hj.x + (float)sx * Lh[0]) - hi.x;
    const float dy = (hj.y + (float)sy * Lh[1]) - hi.y;
    const float dz = (hj.z + (float)sz * Lh[2]) - hi.z;
    const float r2f = dx * dx + dy * dy + dz * dz;
    bool hit = false;
    if (r2f < rc2_lo) {
      hit = true;
    } else if (r2f < rc2_hi) {
      const double ddx = disp_fp64(wpos[i], wpos[j], sx, b.L[0]);
      const double ddy = disp_fp64(wpos[(size_t)N + i], wpos[(size_t)N + j], sy, b.L[1]);
      const double ddz = disp_fp64(wpos[(size_t)2 * N + i], wpos[(size_t)2 * N + j], sz, b.L[2]);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
      hit = r2 < rc2;
    }
    key = ((unsigned long long)j << 24) | (unsigned long long)code;
    return hit;
  };
  // hits are appended in candidate order (image-major, then atom) either way
  auto append = [&](bool hit, unsigned long long key) {
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int pos = nhit + __popc(m & ((1u << lane) - 1u));
      if (pos < keycap) keys[pos] = key;
    }
    nhit += __popc(m);
  };
  if (nat >= 32) {
    // image by image, lanes over the configuration's atoms: no division per candidate
    for (int img = 0; img < nimg; ++img) {
      const int sx = img % wx + smin[0], sy = (img / wx) % wy + smin[1], sz = img / (wx * wy) + smin[2];
      const int code = shift_pack(sx, sy, sz);
      for (int j0 = 0; j0 < nat; j0 += 32) {
        unsigned long long key = 0;
        const bool hit = j0 + lane < nat && test(b.a0 + j0 + lane, sx, sy, sz, code, key);
        append(hit, key);
      }
    }
  } else {
    // small configurations: 32 consecutive (image, atom) candidates per round;
    // 32-bit indices (a 64-bit division per candidate runs on the FP64 pipe, 1/64
    // of the FP32 rate on this part; a batch whose count does not fit is refused
    // on the host)
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      unsigned long long key = 0;
      bool hit = false;
      if (f < total) {
        const int img = f / nat;
        const int sx = img % wx + smin[0], sy = (img / wx) % wy + smin[1], sz = img / (wx * wy) + smin[2];
        hit = test(b.a0 + (f - img * nat), sx, sy, sz, shift_pack(sx, sy, sz), key);
      }
      append(hit, key);
    }
  }
  __syncwarp();
  const int n = min(nhit, keycap);
  int np = 1;
  while (np < n) np <<= 1;
  for (int t = n + lane; t < np; t += 32) keys[t] = ~0ull;
  __syncwarp();
  for (int k = 2; k <= np; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < np; t += 32) {
        const int u = t ^ j;
        if (u > t) {
          const unsigned long long a = keys[t], c = keys[u];
          const bool up = (t & k) == 0;
          if ((a > c) == up) { keys[t] = c; keys[u] = a; }
        }
      }
      __syncwarp();
    }
  const int nw = min(n, cap);
  for (int t = lane; t < cap; t += 32) {
    if (t < nw) {
      const unsigned long long key = keys[t];
      nbr_j[(size_t)i * cap + t] = (int)(key >> 24);
      nbr_s[(size_t)i * cap + t] = (int)(key & 0xFFFFFFull);
    } else {
      nbr_j[(size_t)i * cap + t] = 0x7fffffff;  // sentinel: rows stay sorted to cap
    }
  }
  if (lane == 0) {
    nbr_count[i] = nhit;
    if (nhit > cap) atomicOr(status, ST_NEIGH);
  }
}

// Block per configuration: out[c] = scale_c * sum_{i in c} v[i] in a fixed
// order (strided per thread, then a fixed tree); scale_c = w / n_c when
// per_atom != 0, else w.
__global__ void segsum_kernel(const CfgBox* __restrict__ cbox, const double* __restrict__ v, double w, int per_atom,
                              double* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  const int a0 = cbox[c].a0, a1 = cbox[c].a1;
  double s = 0.0;
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0] * (per_atom ? w / (double)(a1 - a0) : w);
}

// Column sums of a row-major [rows][M] array per configuration, fixed order:
// block b sums the rows of chunk b (<= 256 rows, never crossing a configuration)
// with one thread per column; block c of the second kernel adds its
// configuration's chunk partials in chunk order.
__global__ void colsum_chunk_kernel(const int* __restrict__ chunk_rows, int M, const double* __restrict__ D,
                                    double* __restrict__ part) {
  const int b = blockIdx.x;
  const int r0 = chunk_rows[2 * b], r1 = chunk_rows[2 * b + 1];
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double s = 0.0;
    for (int r = r0; r < r1; ++r) s += D[(size_t)r * M + m];
    part[(size_t)b * M + m] = s;
  }
}

__global__ void colsum_cfg_kernel(const int* __restrict__ cfg_chunks, int M, const double* __restrict__ part,
                                  double* __restrict__ G) {
  const int c = blockIdx.x;
  const int k0 = cfg_chunks[c], k1 = cfg_chunks[c + 1];
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double s = 0.0;
    for (int k = k0; k < k1; ++k) s += part[(size_t)k * M + m];
    G[(size_t)c * M + m] = s;
  }
}

cudaError_t launch_colsum(int n_chunks, const int* chunk_rows, int n_cfg, const int* cfg_chunks, int M,
                          const double* D, double* part, double* G, cudaStream_t st) {
  colsum_chunk_kernel<<<n_chunks, 128, 0, st>>>(chunk_rows, M, D, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  colsum_cfg_kernel<<<n_cfg, 128, 0, st>>>(cfg_chunks, M, part, G);
  return cudaGetLastError();
}

cudaError_t launch_batch_wrap(int N, const double* pos, const int* cfg_of, const CfgBox* cbox, double* wpos,
                              float4* phi, float4* plo, int* status, cudaStream_t st, unsigned long long* facc) {
  const int tb = 256;
  batch_wrap_kernel<<<(N + tb - 1) / tb, tb, 0, st>>>(N, pos, cfg_of, cbox, wpos, phi, plo, status, facc);
  return cudaGetLastError();
}

cudaError_t launch_batch_neigh(int N, const int* cfg_of, const CfgBox* cbox, const double* wpos, const float4* phi,
                               double rcut, double Lmax, int Smax, int cap, int* nbr_count, int* nbr_j, int* nbr_s,
                               int* status, cudaStream_t st) {
  const double rc2 = rcut * rcut;
  const double err_d = 4.0 * Lmax * 1.1920928955078125e-7 * (1 + 3 * Smax);
  const double err_r2 = 2.0 * 1.7320508075688772 * rcut * err_d + 3.0 * err_d * err_d + 8.0 * rc2 * 1.1920928955078125e-7;
  const double band = fmax(4.0 * err_r2, 1e-6 * rc2);
  int keycap = 32;
  while (keycap < cap) keycap <<= 1;
  const size_t smem = (size_t)WPB_NEIGH * keycap * sizeof(unsigned long long);
  static size_t granted[64] = {};
  if (cudaError_t e = grant_smem((const void*)batch_neigh_kernel, smem, granted)) return e;
  batch_neigh_kernel<<<(N + WPB_NEIGH - 1) / WPB_NEIGH, WPB_NEIGH * 32, smem, st>>>(
      N, cfg_of, cbox, wpos, phi, rc2, (float)(rc2 - band), (float)(rc2 + band), cap, keycap, nbr_count, nbr_j,
      nbr_s, status);
  return cudaGetLastError();
}

cudaError_t launch_segsum(int n_cfg, const CfgBox* cbox, const double* v, double w, int per_atom, double* out,
                          cudaStream_t st) {
  segsum_kernel<<<n_cfg, 256, 0, st>>>(cbox, v, w, per_atom, out);
  return cudaGetLastError();
}

}  // namespace fastpod
