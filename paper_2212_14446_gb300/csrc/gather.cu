// Deterministic force gather, per-atom virial and fixed-order FP64 reductions.
//   F_k = sum_{t in N(k)} ( g[k, t] - g[rev(k, t)] )   (F = -dE/dr, no atomics)
//   W_k = - sum_{t in N(k)} d_kt (x) g[k, t]            (pair virial, summed later)
#include "pod_common.cuh"
#include "pod_kernels.h"

namespace fastpod {

// Lower bounds of atom i0 in row j0 and of i1 in row j1, searched in lockstep
// (branch-free binary search over the sentinel-padded sorted rows, so the two
// chains of dependent loads overlap), then the scans over equal indices for the
// negated shifts.  q = -1 if absent; an invalid query (v = false) returns -1 and
// reads row 0 only.
__device__ __forceinline__ void find_reverse2(const int* __restrict__ nbr_j, const int* __restrict__ nbr_s, int cap,
                                              bool v0, int i0, int j0, int c0, bool v1, int i1, int j1, int c1,
                                              int& q0, int& q1) {
  const size_t b0 = (size_t)(v0 ? j0 : 0) * cap, b1 = (size_t)(v1 ? j1 : 0) * cap;
  int lo0 = 0, lo1 = 0;
  int step = 1;
  while (2 * step <= cap) step *= 2;
  for (; step > 0; step >>= 1) {
    const bool t0 = lo0 + step <= cap && __ldg(nbr_j + b0 + lo0 + step - 1) < i0;
    const bool t1 = lo1 + step <= cap && __ldg(nbr_j + b1 + lo1 + step - 1) < i1;
    lo0 += t0 ? step : 0;
    lo1 += t1 ? step : 0;
  }
  q0 = -1;
  q1 = -1;
  if (v0) {
    const int want = shift_negate(c0);
    for (int t = lo0; t < cap && __ldg(nbr_j + b0 + t) == i0; ++t)
      if (__ldg(nbr_s + b0 + t) == want) { q0 = (int)(b0 + t); break; }
  }
  if (v1) {
    const int want = shift_negate(c1);
    for (int t = lo1; t < cap && __ldg(nbr_j + b1 + t) == i1; ++t)
      if (__ldg(nbr_s + b1 + t) == want) { q1 = (int)(b1 + t); break; }
  }
}

// Warp per atom k, lane per neighbour slot t (coalesced own slots):
//   F_k = sum_t ( g[k, t] - g[rev(k, t)] )
// g[k, t] = dE_k/dr_kt, written by the atom kernel; rev(k, t) is the slot of the
// reverse pair in j's row, read from rev_in or searched (and then stored in
// rev_out when given, for steps that reuse the list).  Each warp takes two atoms
// per iteration so that their dependent loads overlap.  No atomics.  Per-block
// FP64 partials of E = sum_i E_i and of the virial partials are summed in a fixed
// order by the last block to finish, so every result is bitwise reproducible.
constexpr int GATHER_MIN_BLOCKS = 3;  // 16-warp blocks: 40 registers

template <typename T>
__global__ void __launch_bounds__(GATHER_MAX_WPB * 32, GATHER_MIN_BLOCKS)
    gather_reduce_kernel(int N, int n_eval, int cap, const int* __restrict__ nbr_count, const int* __restrict__ nbr_j,
                         const int* __restrict__ nbr_s, const int* __restrict__ rev_in, int* __restrict__ rev_out,
                         const Q4<T>* __restrict__ g, const double* __restrict__ Ei,
                         const double* __restrict__ wpart, int n_wpart, double* __restrict__ F, double fscale,
                         double* __restrict__ part, unsigned* __restrict__ ticket, double* __restrict__ E_out,
                         double* __restrict__ W_out, int* __restrict__ status) {
  __shared__ double sred[GATHER_MAX_WPB][10];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int stride = gridDim.x * nwarps;
  double eacc = 0.0, wacc = 0.0;  // lane 0: atom energies; lane q < 9: virial component q
  for (int k0 = blockIdx.x * nwarps + warp; k0 < N; k0 += 2 * stride) {
    const int k1 = k0 + stride;
    const bool has1 = k1 < N;
    const int n0 = min(nbr_count[k0], cap);
    const int n1 = has1 ? min(nbr_count[k1], cap) : 0;
    T f0 = T(0), f1 = T(0), f2 = T(0), h0 = T(0), h1 = T(0), h2 = T(0);
    const int nmax = max(n0, n1);
    for (int t = lane; t < nmax; t += 32) {
      const bool v0 = t < n0, v1 = t < n1;
      const size_t p0 = (size_t)k0 * cap + t, p1 = (size_t)(has1 ? k1 : k0) * cap + t;
      int q0 = -1, q1 = -1;
      if (rev_in) {
        if (v0) q0 = rev_in[p0];
        if (v1) q1 = rev_in[p1];
      } else {
        const int j0 = v0 ? nbr_j[p0] : 0, c0 = v0 ? nbr_s[p0] : 0;
        const int j1 = v1 ? nbr_j[p1] : 0, c1 = v1 ? nbr_s[p1] : 0;
        find_reverse2(nbr_j, nbr_s, cap, v0, k0, j0, c0, v1, k1, j1, c1, q0, q1);
        if (rev_out) {
          if (v0) rev_out[p0] = q0;
          if (v1) rev_out[p1] = q1;
        }
      }
      if ((v0 && q0 < 0) || (v1 && q1 < 0))
        atomicOr(status, ST_REV);  // a list without its reverse pair: reported, never read out of bounds
      // only atoms below n_eval have pair gradients (the rest are ghost atoms)
      const size_t qmax = (size_t)n_eval * cap;
      if (v0 && k0 < n_eval) {
        const Q4<T> a = g[p0];
        f0 += a.x;
        f1 += a.y;
        f2 += a.z;
      }
      if (v1 && k1 < n_eval) {
        const Q4<T> a = g[p1];
        h0 += a.x;
        h1 += a.y;
        h2 += a.z;
      }
      if (q0 >= 0 && (size_t)q0 < qmax) {
        const Q4<T> b = g[q0];
        f0 -= b.x;
        f1 -= b.y;
        f2 -= b.z;
      }
      if (q1 >= 0 && (size_t)q1 < qmax) {
        const Q4<T> b = g[q1];
        h0 -= b.x;
        h1 -= b.y;
        h2 -= b.z;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f0 += __shfl_xor_sync(0xffffffffu, f0, o);
      f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      h0 += __shfl_xor_sync(0xffffffffu, h0, o);
      h1 += __shfl_xor_sync(0xffffffffu, h1, o);
      h2 += __shfl_xor_sync(0xffffffffu, h2, o);
    }
    // lane c < 6 stores component c % 3 of atom c < 3 ? k0 : k1 (one conversion
    // instruction per warp instead of six)
    if (lane < 6 && (lane < 3 || has1)) {
      const int k = lane < 3 ? k0 : k1, d = lane < 3 ? lane : lane - 3;
      const T v = lane == 0 ? f0 : lane == 1 ? f1 : lane == 2 ? f2 : lane == 3 ? h0 : lane == 4 ? h1 : h2;
      if (F) F[(size_t)d * N + k] = fscale * (double)v;
      if (!isfinite(v)) atomicOr(status, ST_NONFINITE);
    }
    if (lane == 0) {
      if (k0 < n_eval) eacc += Ei[k0];
      if (has1 && k1 < n_eval) eacc += Ei[k1];
    }
  }
  // virial partials of the atom kernel, a fixed subset per warp of this block
  if (lane < 9)
    for (int w = blockIdx.x * nwarps + warp; w < n_wpart; w += stride) wacc += wpart[(size_t)w * 9 + lane];
  if (lane == 0) sred[warp][0] = eacc;
  if (lane < 9) sred[warp][1 + lane] = wacc;
  __syncthreads();
  if (threadIdx.x < 10) {
    double s = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) s += sred[wv][threadIdx.x];
    part[(size_t)blockIdx.x * 10 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order sum of the block partials: component q is added by warp q mod
  // (warps per block); lane l adds blocks l, l + 32, ... in order, then a fixed
  // butterfly across the lanes
  for (int q = warp; q < 10; q += nwarps) {
    double s = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(part + (size_t)b * 10 + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (q == 0) E_out[0] = s;
      else if (W_out) W_out[q - 1] = s;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch (graph replays)
}

// FP32 path: forces from the fixed-point accumulators the atom kernel filled
// (F = fscale * acc * 2^-32), and E and the virial from the fixed-point totals
// after the force rows (2^-36).  Integer sums do not depend on the order of the
// atomics, so every result is bitwise reproducible.
// With cell_count set it also clears the ncells counts of the cell list for the
// next call's binning (the neighbour search of this call has read them).
__global__ void __launch_bounds__(256)
    finalize_kernel(int N, const unsigned long long* __restrict__ facc, double* __restrict__ F, double fscale,
                    double* __restrict__ E_out, double* __restrict__ W_out, int* __restrict__ cell_count,
                    int ncells, int* __restrict__ status, int* __restrict__ status_out) {
  const double sc = fscale * FIX_INV_SCALE;
  // as the step's last kernel: hand the status word of this call (every earlier
  // kernel has finished) to status_out and clear it for the next call
  if (status_out && blockIdx.x == 0 && threadIdx.x == 0) {
    status_out[0] = status[0];
    status[0] = 0;
  }
  if (cell_count)
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) cell_count[c] = 0;
  if (blockIdx.x == 0) {  // warp w sums quantities w, w + 8 (0: E, 1..9: W)
    const int lane = threadIdx.x & 31;
    for (int q = threadIdx.x >> 5; q < 10; q += blockDim.x >> 5) {
      const double v = ew_value_warp(facc + 4 * (size_t)N + 2 * q, lane);
      if (lane == 0) {
        if (q == 0)
          E_out[0] = v;
        else if (W_out)
          W_out[q - 1] = v;
      }
    }
  }
  if (!F) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(facc + 4 * (size_t)k);
    const unsigned long long b = facc[4 * (size_t)k + 2];
    if (fscale == 1.0) {  // x 2^-32 by integer operations (the same bits, off the FP64 pipe)
      F[k] = fixed_to_double((long long)a.x, -32);
      F[(size_t)N + k] = fixed_to_double((long long)a.y, -32);
      F[(size_t)2 * N + k] = fixed_to_double((long long)b, -32);
    } else {
      F[k] = sc * (double)(long long)a.x;
      F[(size_t)N + k] = sc * (double)(long long)a.y;
      F[(size_t)2 * N + k] = sc * (double)(long long)b;
    }
  }
}

constexpr int FINALIZE_THREADS = 256;
// One atom per thread (a streaming pass: every thread's loads in flight at once),
// at most 64 blocks per SM's worth, striding beyond that.
int finalize_blocks(int N) {
  const int want = (N + FINALIZE_THREADS - 1) / FINALIZE_THREADS;
  return want < 64 * 152 ? (want > 0 ? want : 1) : 64 * 152;
}

cudaError_t launch_finalize(int N, const unsigned long long* facc, double* F, double fscale, int nblocks, double* E,
                            double* W, cudaStream_t st, int* cell_count, int ncells, int* status, int* status_out) {
  finalize_kernel<<<nblocks, FINALIZE_THREADS, 0, st>>>(N, facc, F, fscale, E, W, cell_count, ncells, status,
                                                        status_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_reduce(int N, int n_eval, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s,
                                 const int* rev_in, int* rev_out, const Q4<T>* g, const double* Ei,
                                 const double* wpart, int n_wpart, double* F, double fscale, double* part,
                                 int nblocks, unsigned* ticket, double* E, double* W, int* status, cudaStream_t st,
                                 int wpb) {
  if (wpb < 1 || wpb > GATHER_MAX_WPB) return cudaErrorInvalidValue;
  gather_reduce_kernel<T><<<nblocks, wpb * 32, 0, st>>>(N, n_eval, cap, nbr_count, nbr_j, nbr_s, rev_in, rev_out, g,
                                                               Ei, wpart, n_wpart, F, fscale, part, ticket, E, W,
                                                               status);
  return cudaGetLastError();
}

// One wave of fat blocks (bps per SM at most) striding over the atoms keeps the
// number of block partials, and so the last block's fixed-order sum, small.
int gather_blocks(int N, int wpb, int bps) {
  const int want = (N + wpb - 1) / wpb;
  const int full = bps * 152;
  return want < full ? (want > 0 ? want : 1) : full;
}

template cudaError_t launch_gather_reduce<float>(int, int, int, const int*, const int*, const int*, const int*, int*,
                                                 const Q4<float>*, const double*, const double*, int, double*,
                                                 double, double*, int, unsigned*, double*, double*, int*,
                                                 cudaStream_t, int);
template cudaError_t launch_gather_reduce<double>(int, int, int, const int*, const int*, const int*, const int*, int*,
                                                  const Q4<double>*, const double*, const double*, int, double*,
                                                  double, double*, int, unsigned*, double*, double*, int*,
                                                  cudaStream_t, int);

}  // namespace fastpod
