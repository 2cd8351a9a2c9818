// Householder QR of the weighted design matrix of the fit (Eq. 63a), the
// fallback of the normal-equations solve: min || [A; sqrt(gamma) I] c - [b; 0] ||
// is solved from the QR factors of the augmented matrix, so the condition number
// is that of A itself rather than its square (as in A^T A).
//
// Tall-skinny QR as a reduction tree, all in FP64 with a fixed order of
// operations (deterministic):
//   rows    each block absorbs a contiguous range of rows of A (and b) into a
//           running upper-triangular factor R held in shared memory, cmax rows
//           at a time;
//   merge   each block absorbs g factors of the previous level into one;
//   final   one block absorbs the last factors and the rows sqrt(gamma) I, then
//           solves R c = Q^T b by back substitution.
// A step that absorbs c new rows into R applies M Householder reflections that
// act only on row k of R and the new rows: column k of R is zero below its
// diagonal, so the reflection that annihilates the new rows' column k leaves the
// other rows of R untouched.
#include <cuda_runtime.h>

#include "pod_kernels.h"

namespace fastpod {

constexpr int QR_THREADS = 256;
constexpr int QR_MAXM = 256;  // descriptors handled by the final solve

// Panel P in shared memory, column-major with leading dimension ld: columns
// [0, M) of the matrix and column M for the right-hand side; rows [0, M) hold
// the running factor R (and Q^T b), rows [M, M + c) the new rows.
__device__ void qr_absorb(double* P, int ld, int M, int c) {
  __shared__ double s_v0, s_beta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int k = 0; k < M; ++k) {
    const double* colk = P + (size_t)k * ld;
    if (warp == 0) {
      double s = 0.0;
      for (int i = lane; i < c; i += 32) s = fma(colk[M + i], colk[M + i], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const double x0 = colk[k];
        if (s == 0.0) {  // the new rows are already zero in this column
          s_beta = 0.0;
          s_v0 = 0.0;
        } else {
          const double nrm = sqrt(fma(x0, x0, s));
          const double alpha = x0 >= 0.0 ? -nrm : nrm;
          const double v0 = x0 - alpha;
          s_v0 = v0;
          s_beta = 2.0 / fma(v0, v0, s);  // H = I - beta v v^T, v = (v0 at row k, new rows)
          P[(size_t)k * ld + k] = alpha;
        }
      }
    }
    __syncthreads();
    const double beta = s_beta, v0 = s_v0;
    if (beta != 0.0) {
      for (int j = k + 1 + warp; j <= M; j += nwarp) {
        double* colj = P + (size_t)j * ld;
        double w = 0.0;
        for (int i = lane; i < c; i += 32) w = fma(colk[M + i], colj[M + i], w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        const double f = beta * fma(v0, colj[k], w);
        __syncwarp();
        if (lane == 0) colj[k] = fma(-f, v0, colj[k]);
        for (int i = lane; i < c; i += 32) colj[M + i] = fma(-f, colk[M + i], colj[M + i]);
      }
    }
    __syncthreads();
  }
}

// Rows of A (column-major AT[m][row], rows [r0, r1) of this block) and b into
// one factor per block: out[block] = rows [0, M) of the panel's M + 1 columns,
// column-major ([M + 1][M]).
__global__ void __launch_bounds__(QR_THREADS)
    tsqr_rows_kernel(int M, long long R, const double* __restrict__ AT, const double* __restrict__ b,
                     long long rows_per_block, int cmax, double* __restrict__ out) {
  extern __shared__ double P[];
  const int ld = M + cmax;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < (M + 1) * M; e += nthr) P[(size_t)(e / M) * ld + e % M] = 0.0;
  const long long r0 = (long long)blockIdx.x * rows_per_block;
  const long long r1 = r0 + rows_per_block < R ? r0 + rows_per_block : R;
  for (long long q = r0; q < r1; q += cmax) {
    const int c = (int)(r1 - q < cmax ? r1 - q : cmax);
    __syncthreads();
    for (int e = tid; e < (M + 1) * c; e += nthr) {
      const int j = e / c, i = e - j * c;
      P[(size_t)j * ld + M + i] = j < M ? AT[(size_t)j * R + q + i] : b[q + i];
    }
    __syncthreads();
    qr_absorb(P, ld, M, c);
  }
  __syncthreads();
  double* o = out + (size_t)blockIdx.x * (M + 1) * M;
  for (int e = tid; e < (M + 1) * M; e += nthr) o[e] = P[(size_t)(e / M) * ld + e % M];
}

// Block b absorbs the factors in[g b .. g b + g) (each [M + 1][M]) into one.
// With c_out set (one block): then absorbs sqrt(gamma) I (right-hand side 0) and
// solves R c = Q^T b; info = k + 1 when R_kk = 0 (rank deficient), else 0.
__global__ void __launch_bounds__(QR_THREADS)
    tsqr_merge_kernel(int M, int nin, int g, const double* __restrict__ in, int cmax, double sqrt_gamma,
                      double* __restrict__ out, double* __restrict__ c_out, int* __restrict__ info) {
  extern __shared__ double P[];
  const int ld = M + cmax;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int first = blockIdx.x * g;
  const int last = first + g < nin ? first + g : nin;
  const double* f0 = in + (size_t)first * (M + 1) * M;
  for (int e = tid; e < (M + 1) * M; e += nthr) P[(size_t)(e / M) * ld + e % M] = f0[e];
  for (int p = first + 1; p < last; ++p) {
    const double* fp = in + (size_t)p * (M + 1) * M;
    for (int r0 = 0; r0 < M; r0 += cmax) {
      const int c = M - r0 < cmax ? M - r0 : cmax;
      __syncthreads();
      for (int e = tid; e < (M + 1) * c; e += nthr) {
        const int j = e / c, i = e - j * c;
        P[(size_t)j * ld + M + i] = fp[(size_t)j * M + r0 + i];
      }
      __syncthreads();
      qr_absorb(P, ld, M, c);
    }
  }
  if (!c_out) {
    __syncthreads();
    double* o = out + (size_t)blockIdx.x * (M + 1) * M;
    for (int e = tid; e < (M + 1) * M; e += nthr) o[e] = P[(size_t)(e / M) * ld + e % M];
    return;
  }
  if (sqrt_gamma > 0.0) {
    for (int r0 = 0; r0 < M; r0 += cmax) {
      const int c = M - r0 < cmax ? M - r0 : cmax;
      __syncthreads();
      for (int e = tid; e < (M + 1) * c; e += nthr) {
        const int j = e / c, i = e - j * c;
        P[(size_t)j * ld + M + i] = (j == r0 + i) ? sqrt_gamma : 0.0;
      }
      __syncthreads();
      qr_absorb(P, ld, M, c);
    }
  }
  __syncthreads();
  // back substitution R c = y by one warp, rows from the bottom up
  __shared__ double sc[QR_MAXM];
  if (tid < 32) {
    const int lane = tid;
    int bad = 0;
    for (int k = M - 1; k >= 0; --k) {
      double s = 0.0;
      for (int j = k + 1 + lane; j < M; j += 32) s = fma(P[(size_t)j * ld + k], sc[j], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double rkk = P[(size_t)k * ld + k];
      if (rkk == 0.0 || !isfinite(rkk)) bad = k + 1;
      if (lane == 0) sc[k] = bad ? 0.0 : (P[(size_t)M * ld + k] - s) / rkk;
      __syncwarp();
    }
    for (int k = lane; k < M; k += 32) c_out[k] = sc[k];
    if (lane == 0) *info = bad;
  }
}

size_t tsqr_smem_bytes(int M, int cmax) { return sizeof(double) * (size_t)(M + 1) * (M + cmax); }

cudaError_t launch_tsqr_rows(int M, long long R, const double* AT, const double* b, int nblocks,
                             long long rows_per_block, int cmax, double* out, cudaStream_t st) {
  const size_t smem = tsqr_smem_bytes(M, cmax);
  static size_t granted[64] = {};
  if (cudaError_t e = grant_smem((const void*)tsqr_rows_kernel, smem, granted)) return e;
  tsqr_rows_kernel<<<nblocks, QR_THREADS, smem, st>>>(M, R, AT, b, rows_per_block, cmax, out);
  return cudaGetLastError();
}

cudaError_t launch_tsqr_merge(int M, int nin, int g, const double* in, int cmax, double sqrt_gamma, double* out,
                              double* c_out, int* info, cudaStream_t st) {
  const size_t smem = tsqr_smem_bytes(M, cmax);
  static size_t granted[64] = {};
  if (cudaError_t e = grant_smem((const void*)tsqr_merge_kernel, smem, granted)) return e;
  const int nblocks = c_out ? 1 : (nin + g - 1) / g;
  tsqr_merge_kernel<<<nblocks, QR_THREADS, smem, st>>>(M, nin, c_out ? nin : g, in, cmax, sqrt_gamma, out, c_out,
                                                         info);
  return cudaGetLastError();
}

}  // namespace fastpod
