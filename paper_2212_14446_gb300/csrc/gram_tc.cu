// Normal-equation matrix G = A^T A of the fit (Eq. 63a) on the tensor cores,
// exactly.  Every column m of A is written as a sum of SLICES 8-bit integer
// slices on a grid fixed by the column's largest magnitude,
//   A_rm = 2^e_m sum_s v_s[r][m] 2^(-8 (s + 1)) + rest,  |v_s| <= 255,
// stored as BF16 (exact for such integers).  For each slice pair (s, t) with
// s <= t and s + t < SLICES the products V_s^T V_t are formed by BF16 MMAs with
// FP32 accumulation over chunks of 256 rows -- every partial sum is an integer
// below 2^24, so the FP32 accumulator holds it exactly whatever its rounding --
// and the chunk sums are added as 64-bit integers.  The dropped slice pairs and
// the rest are below 2^(-59) of the column maxima, so G carries no summation
// error beyond that (the FP64 SYRK it replaces rounds once per row).  G_mn is
// then assembled in FP64 from the integer sums, smallest slice pairs first.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "pod_internal.h"

namespace fastpod {

constexpr int TC_CHUNK = 256;  // rows per exact FP32 accumulation
constexpr int TC_SPLITS_MAX = 64;

constexpr int TC_COLBLK = 32;  // row blocks per column for the column scans

// Largest magnitude of column m over row block blockIdx.y, as the bit pattern
// of the double (ordered like the values for non-negative doubles).
__global__ void gram_colmax_kernel(long long R, const double* __restrict__ AT, unsigned long long* __restrict__ pmax) {
  __shared__ unsigned long long smax[256];
  const int m = blockIdx.x;
  const long long r0 = R * blockIdx.y / gridDim.y, r1 = R * (blockIdx.y + 1) / gridDim.y;
  const unsigned long long* col = reinterpret_cast<const unsigned long long*>(AT + (size_t)m * R);
  unsigned long long v = 0;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) v = max(v, __ldg(col + r) & 0x7fffffffffffffffull);
  smax[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) pmax[(size_t)m * gridDim.y + blockIdx.y] = smax[0];
}

// e_m: the smallest integer with max_r |A_rm| < 2^e_m (0 for an all-zero column).
__global__ void gram_colexp_kernel(int M, int nblk, const unsigned long long* __restrict__ pmax, int* __restrict__ ex) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  unsigned long long v = 0;
  for (int k = 0; k < nblk; ++k) v = max(v, pmax[(size_t)m * nblk + k]);
  const int ef = (int)(v >> 52);        // biased exponent of the largest magnitude
  ex[m] = ef == 0 ? 0 : ef - 1022;      // max = f 2^(ef - 1022), f in [0.5, 1)
}

// VT[s][m][r] (r contiguous, RP rows, Mp columns, zero padded): the slices.
// X = floor(|A_rm| 2^(64 - e_m)) (< 2^64) is formed from the double's bits by
// integer shifts; slice s is byte 7 - s of X with the sign of A_rm.  Values
// below the smallest normal double count as zero.
__global__ void gram_slice_kernel(int M, int Mp, long long R, long long RP, int slices, const double* __restrict__ AT,
                                  const int* __restrict__ ex, __nv_bfloat16* __restrict__ VT) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Mp * RP) return;
  const int m = (int)(idx / RP);
  const long long r = idx - (long long)m * RP;
  unsigned long long X = 0;
  bool neg = false;
  if (m < M && r < R) {
    const unsigned long long bits = __double_as_longlong(__ldg(AT + (size_t)m * R + r));
    neg = (bits >> 63) != 0;
    const int ef = (int)((bits >> 52) & 0x7ff);
    if (ef != 0) {
      const unsigned long long mant = (bits & 0xfffffffffffffull) | (1ull << 52);  // |a| = mant 2^(ef - 1075)
      const int sh = ef - 1075 + 64 - ex[m];                                        // <= 11 as |a| < 2^e_m
      X = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
    }
  }
  for (int s = 0; s < slices; ++s) {
    const int v = (int)((X >> (56 - 8 * s)) & 0xff);
    VT[((size_t)s * Mp + m) * RP + r] = __float2bfloat16_rn((float)(neg ? -v : v));  // exact: |v| <= 255
  }
}

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

constexpr int TC_STAGES = 8;  // 32-row steps in flight (cp.async ring)

// One block per (slice pair, row split), Mp = 16 NJ: warp w computes the
// 16 x 8 NJ tile of V_s^T V_t at rows 16 (w % NJ) and columns 8 NJ (w / NJ) (NJ
// m-tiles x 2 column halves of NJ n-tiles).  The block stages each 32-row step
// of the two slices (Mp rows x 64 bytes each) in shared memory through a
// cp.async ring of TC_STAGES steps.  Lane (g, t) = (lane / 4, lane % 4) reads
// rows k0 + 8t .. k0 + 8t + 7 of its A and B rows with one 16-byte load each;
// the MMA's k positions (2t, 2t + 1, 2t + 8, 2t + 9) are mapped to rows (8t,
// 8t + 1, 8t + 2, 8t + 3) in the first MMA and to the next four in the second,
// the same mapping for A and B, so each pair of MMAs sums exactly the 32 rows of
// the step.  part[(pair * splits + split)][Mp][Mp] gets the 64-bit integer sums.
template <int NJ>
__global__ void __launch_bounds__(2 * NJ * 32)
    gram_tc_kernel(int Mp, long long RP, int splits, const int2* __restrict__ pairs,
                   const __nv_bfloat16* __restrict__ VT, long long* __restrict__ part) {
  extern __shared__ uint4 gstage[];  // [TC_STAGES][2][Mp][4] 16-byte words
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = warp % NJ, nh = warp / NJ;
  const int m0 = 16 * mt, n0 = nh * 8 * NJ;
  const int2 st = pairs[blockIdx.x];
  const int split = blockIdx.y;
  const long long nstep = RP / 32;
  const long long k0s = nstep * split / splits, k1s = nstep * (split + 1) / splits;
  const uint4* Asrc = reinterpret_cast<const uint4*>(VT + (size_t)st.x * Mp * RP);
  const uint4* Bsrc = reinterpret_cast<const uint4*>(VT + (size_t)st.y * Mp * RP);
  const size_t row_q = (size_t)RP / 8;  // 16-byte words per slice row
  const int nthr = blockDim.x;
  const int words = 2 * Mp * 4;  // 16-byte words per stage
  auto issue = [&](long long step, int slot) {
    if (step < k1s) {
      uint4* dst = gstage + (size_t)slot * words;
      for (int q = threadIdx.x; q < words; q += nthr) {
        const int which = q / (Mp * 4), rem = q - which * Mp * 4, row = rem >> 2, wq = rem & 3;
        const uint4* src = (which ? Bsrc : Asrc) + (size_t)row * row_q + (size_t)step * 4 + wq;
        cp_async16(dst + q, src);
      }
    }
    cp_async_commit();
  };
  long long acc64[NJ][4];
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc64[j][q] = 0;
  float acc[NJ][4];
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
#pragma unroll
  for (int sidx = 0; sidx < TC_STAGES - 1; ++sidx) issue(k0s + sidx, sidx);
  for (long long k = k0s; k < k1s; ++k) {
    const int slot = (int)((k - k0s) % TC_STAGES);
    cp_async_wait<TC_STAGES - 2>();
    __syncthreads();  // step k is in shared memory; the slot refilled below is free
    issue(k + TC_STAGES - 1, (int)((k - k0s + TC_STAGES - 1) % TC_STAGES));
    const uint4* sA = gstage + (size_t)slot * words;
    const uint4* sB = sA + Mp * 4;
    const uint4 alo = sA[(m0 + g) * 4 + t];
    const uint4 ahi = sA[(m0 + g + 8) * 4 + t];
    const unsigned a1[4] = {alo.x, ahi.x, alo.y, ahi.y};
    const unsigned a2[4] = {alo.z, ahi.z, alo.w, ahi.w};
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const uint4 bv = sB[(n0 + 8 * j + g) * 4 + t];
      const unsigned b1[2] = {bv.x, bv.y};
      const unsigned b2[2] = {bv.z, bv.w};
      mma_bf16(acc[j], a1, b1);
      mma_bf16(acc[j], a2, b2);
    }
    if (((k + 1) & (TC_CHUNK / 32 - 1)) == 0 || k + 1 == k1s) {  // end of a 256-row chunk: exact integers
#pragma unroll
      for (int j = 0; j < NJ; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc64[j][q] += (long long)__float2ll_rn(acc[j][q]);
          acc[j][q] = 0.f;
        }
    }
  }
  cp_async_wait<0>();
  long long* out = part + ((size_t)blockIdx.x * splits + split) * Mp * Mp;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int col = n0 + 8 * j + 2 * t;
    out[(size_t)(m0 + g) * Mp + col] = acc64[j][0];
    out[(size_t)(m0 + g) * Mp + col + 1] = acc64[j][1];
    out[(size_t)(m0 + g + 8) * Mp + col] = acc64[j][2];
    out[(size_t)(m0 + g + 8) * Mp + col + 1] = acc64[j][3];
  }
}

// G_mn = sum over slice pairs (largest s + t, i.e. smallest terms, first) of
// 2^(e_m + e_n - 8 (s + t + 2)) (P_st[m][n] (+ P_st[n][m] for s != t)), the
// integer split sums exact; gamma on the diagonal.
__global__ void gram_tc_combine_kernel(int M, int Mp, int npairs, int splits, const int2* __restrict__ pairs,
                                       const long long* __restrict__ part, const int* __restrict__ ex, double gamma,
                                       double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  const int m = e / M, n = e - m * M;
  double s = 0.0;
  for (int p = npairs - 1; p >= 0; --p) {  // pairs come in ascending s + t
    const int2 st = pairs[p];
    long long v = 0;
    for (int k = 0; k < splits; ++k) {
      const long long* P = part + ((size_t)p * splits + k) * Mp * Mp;
      v += P[(size_t)m * Mp + n];
      if (st.x != st.y) v += P[(size_t)n * Mp + m];
    }
    s += ldexp((double)v, ex[m] + ex[n] - 8 * (st.x + st.y + 2));
  }
  if (m == n) s += gamma;
  G[e] = s;
}

// r = A^T b in FP64: block (m, k) sums its row block with a fixed-order tree,
// then the row blocks are added in order.
__global__ void atb_partial_kernel(long long R, const double* __restrict__ AT, const double* __restrict__ b,
                                   double* __restrict__ part) {
  __shared__ double sred[256];
  const int m = blockIdx.x;
  const long long r0 = R * blockIdx.y / gridDim.y, r1 = R * (blockIdx.y + 1) / gridDim.y;
  const double* col = AT + (size_t)m * R;
  double v = 0.0;
  for (long long k = r0 + threadIdx.x; k < r1; k += blockDim.x) v = fma(col[k], b[k], v);
  sred[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sred[threadIdx.x] += sred[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)m * gridDim.y + blockIdx.y] = sred[0];
}

__global__ void atb_final_kernel(int M, int nblk, const double* __restrict__ part, double* __restrict__ r) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += part[(size_t)m * nblk + k];
  r[m] = s;
}

}  // namespace fastpod

using namespace fastpod;

// Stage 2 on the tensor cores: G = A^T A + gamma I and r = A^T b into dG, dr.
int pod_handle::fit_gram_tc(double gamma, double* dG, double* dr) {
  const int Mp = M <= 112 ? 112 : 128;
  if (M > 128) return fail(POD_EINVAL, "the tensor-core Gram handles at most 128 descriptors");
  const long long R = fit_R;
  const long long RP = (R + TC_CHUNK - 1) / TC_CHUNK * TC_CHUNK;
  constexpr int SLICES = 8;
  int hp[2 * 64], np = 0;
  for (int sum = 0; sum < SLICES; ++sum)  // ascending s + t
    for (int s = 0; 2 * s <= sum; ++s) {
      hp[2 * np] = s;
      hp[2 * np + 1] = sum - s;
      ++np;
    }
  // one block per SM (the kernel holds 128 registers a thread): splits fill one wave
  const int splits = (int)std::max<long long>(1, std::min<long long>(TC_SPLITS_MAX, 152 / np));
  const size_t vt_bytes = sizeof(__nv_bfloat16) * SLICES * (size_t)Mp * RP;
  const size_t part_bytes = sizeof(long long) * (size_t)np * splits * Mp * Mp;
  int rc_;
  const size_t scan_bytes = sizeof(double) * (size_t)M * TC_COLBLK;
  if ((rc_ = ensure(fitG, vt_bytes + part_bytes + sizeof(int) * (2 * 64 + 128) + 2 * scan_bytes + 1024, "Gram slices")))
    return rc_;
  unsigned char* base = (unsigned char*)fitG.p;
  __nv_bfloat16* VT = (__nv_bfloat16*)base;
  long long* part = (long long*)(base + (vt_bytes + 255) / 256 * 256);
  int* dex = (int*)((unsigned char*)part + part_bytes);
  int2* dpairs = (int2*)(dex + 128);
  unsigned long long* pmax = (unsigned long long*)((unsigned char*)(dpairs + 64) + 256);
  double* apart = (double*)(pmax + (size_t)M * TC_COLBLK);
  cudaError_t e = cudaMemcpy(dpairs, hp, sizeof(int) * 2 * np, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "Gram slice pairs");
  const double* AT = (const double*)fitA.p;
  gram_colmax_kernel<<<dim3((unsigned)M, TC_COLBLK), 256, 0, nullptr>>>(R, AT, pmax);
  gram_colexp_kernel<<<(M + 127) / 128, 128, 0, nullptr>>>(M, TC_COLBLK, pmax, dex);
  const long long nel = (long long)Mp * RP;
  gram_slice_kernel<<<(unsigned)((nel + 255) / 256), 256, 0, nullptr>>>(M, Mp, R, RP, SLICES, AT, dex, VT);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "Gram slicing");
  const dim3 grid((unsigned)np, (unsigned)splits);
  const size_t smem = (size_t)TC_STAGES * 2 * Mp * 64;
  static size_t granted7[64] = {}, granted8[64] = {};
  if (Mp == 112) {
    if ((e = grant_smem((const void*)gram_tc_kernel<7>, smem, granted7)) != cudaSuccess)
      return cuda_fail(e, "Gram shared memory");
    gram_tc_kernel<7><<<grid, 2 * 7 * 32, smem, nullptr>>>(Mp, RP, splits, dpairs, VT, part);
  } else {
    if ((e = grant_smem((const void*)gram_tc_kernel<8>, smem, granted8)) != cudaSuccess)
      return cuda_fail(e, "Gram shared memory");
    gram_tc_kernel<8><<<grid, 2 * 8 * 32, smem, nullptr>>>(Mp, RP, splits, dpairs, VT, part);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "Gram tensor-core kernel");
  gram_tc_combine_kernel<<<(M * M + 255) / 256, 256, 0, nullptr>>>(M, Mp, np, splits, dpairs, part, dex, gamma, dG);
  atb_partial_kernel<<<dim3((unsigned)M, TC_COLBLK), 256, 0, nullptr>>>(R, AT, (const double*)fitb.p, apart);
  atb_final_kernel<<<(M + 127) / 128, 128, 0, nullptr>>>(M, TC_COLBLK, apart, dr);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "Gram assembly");
  return POD_OK;
}
