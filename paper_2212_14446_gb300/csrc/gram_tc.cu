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
// Two forms of the slice products, with identical integer sums: tcgen05 MMAs
// with TMEM accumulators (gram_umma_kernel, the default) and warp-level mma.sync
// (gram_tc_kernel).
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

// ---------------------------------------------------------------------------
// The same slice products on the fifth-generation tensor cores (tcgen05).
//
// Slices are stored tiled for the MMA: VU[s][kb][mg][kg][mr][kr] holds row
// r = 64 kb + 8 kg + kr of column m = 8 mg + mr, so one 64-row step of a slice
// (a "tile", Mp x 64 BF16 = Mp x 128 bytes) is contiguous and is already the
// K-major, unswizzled operand layout of tcgen05.mma: 8 x 8 core matrices of 128
// bytes, 128 bytes apart along K and 1,024 bytes apart along M/N.  One block
// per (slice pair, row split); warp roles:
//   warp 8 lane 0   copies the A and B tiles of each step into a ring of
//                   U_STAGES shared-memory stages (cp.async.bulk, completion on
//                   an mbarrier with the byte count);
//   warp 9 lane 0   issues four M128 x N(Mp) x K16 BF16 MMAs per step into one of
//                   two TMEM accumulators (FP32), restarting the accumulator at
//                   every 256-row chunk (every partial sum an integer below
//                   2^24, exact), and commits the chunk to an mbarrier;
//   warps 0..7      drain each finished chunk from TMEM (warp w reads TMEM lanes
//                   32 (w % 4) .. + 31, columns half w / 4), convert the exact
//                   FP32 integers to int32 and add them in registers; at the end
//                   they add the block's sums to P[pair][m][n] with 64-bit
//                   integer atomics (order-independent, so deterministic).
// A block covers at most U_MAX_ROWS rows, so its int32 sums stay below
// U_MAX_ROWS * 255^2 < 2^31.  Every wait is bounded (about two seconds of
// global time); a wait that runs out sets ST_TIMEOUT, tells the other roles to
// stop, and the block still waits for its own copies and MMAs before freeing
// TMEM.
constexpr int U_KB = 64;                    // rows per step (one stage)
constexpr int U_STAGES = 6;                 // shared-memory ring
constexpr int U_CHUNK_KB = TC_CHUNK / U_KB;  // steps per exact FP32 chunk
constexpr int U_EPI_WARPS = 8;
constexpr int U_THREADS = (U_EPI_WARPS + 2) * 32;
constexpr long long U_MAX_ROWS = 32768;     // 32768 * 255^2 < 2^31
constexpr unsigned U_TMEM_COLS = 256;       // two accumulators of up to 128 columns

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the completion of phase `parity`; false if limit_ns of global time
// pass (about two seconds by default) or (when stop is given) another role has
// set *stop.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, const volatile int* stop,
                                          unsigned long long limit_ns = 2000000000ull) {
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (stop && *stop) return false;
      const unsigned long long t = global_ns();
      if (it == 0)
        t0 = t;
      else if (t - t0 > limit_ns)
        return false;
    }
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at and reports ST_TIMEOUT when the limit runs out.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int* __restrict__ status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const unsigned b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  if (!mbar_wait(b, 0u, nullptr, limit_ns)) atomicOr(status, ST_TIMEOUT);
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets, descriptor version 1,
// no swizzle.
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
constexpr unsigned umma_idesc(int Mm, int Nn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(Nn >> 3) << 17) | ((unsigned)(Mm >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                          unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
// 32 TMEM lanes x 8 columns of 32-bit words; the values are valid after tmem_wait8.
__device__ __forceinline__ void tmem_ld8(unsigned taddr, unsigned* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
// Waits for this thread's TMEM loads; the operands tie the loaded registers to
// the wait so no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait8(unsigned* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

// X = floor(|a| 2^(64 - e)) from the double's bits (integer shifts; values below
// the smallest normal double count as zero); the sign is returned separately.
__device__ __forceinline__ unsigned long long slice_bits(double a, int e, bool& neg) {
  const unsigned long long bits = __double_as_longlong(a);
  neg = (bits >> 63) != 0;
  const int ef = (int)((bits >> 52) & 0x7ff);
  if (ef == 0) return 0ull;
  const unsigned long long mant = (bits & 0xfffffffffffffull) | (1ull << 52);  // |a| = mant 2^(ef - 1075)
  const int sh = ef - 1075 + 64 - e;                                           // <= 11 as |a| < 2^e
  return sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
}

// VU (tiled slices, layout above) from A: thread per (column m, 8-row group), so
// each thread stores one 16-byte core-matrix row per slice and 64 consecutive
// threads store one contiguous 1,024-byte group.
__global__ void gram_slice_tiled_kernel(int M, int Mp, long long R, long long RP, int slices,
                                        const double* __restrict__ AT, const int* __restrict__ ex,
                                        __nv_bfloat16* __restrict__ VU) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int MG = Mp >> 3;
  const long long nKB = RP / U_KB;
  if (t >= nKB * MG * 64) return;
  const int mr = (int)(t & 7), kg = (int)((t >> 3) & 7);
  const long long rest = t >> 6;
  const int mg = (int)(rest % MG);
  const long long kb = rest / MG;
  const int m = mg * 8 + mr;
  const long long r0 = kb * U_KB + kg * 8;
  unsigned long long X[8];
  unsigned negmask = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    X[k] = 0ull;
    if (m < M && r0 + k < R) {
      bool neg;
      X[k] = slice_bits(__ldg(AT + (size_t)m * R + r0 + k), ex[m], neg);
      negmask |= (neg ? 1u : 0u) << k;
    }
  }
  uint4* dst = reinterpret_cast<uint4*>(VU + (size_t)kb * Mp * U_KB) + (size_t)(mg * 8 + kg) * 8 + mr;
  const size_t slice_words = (size_t)nKB * Mp * U_KB / 8;  // 16-byte words per slice
  for (int s = 0; s < slices; ++s) {
    unsigned w[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      const int v0 = (int)((X[k] >> (56 - 8 * s)) & 0xff), v1 = (int)((X[k + 1] >> (56 - 8 * s)) & 0xff);
      const __nv_bfloat162 h = __floats2bfloat162_rn((float)((negmask >> k) & 1 ? -v0 : v0),
                                                     (float)((negmask >> (k + 1)) & 1 ? -v1 : v1));  // exact
      w[k / 2] = *reinterpret_cast<const unsigned*>(&h);
    }
    dst[s * slice_words] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int MP>
__global__ void __launch_bounds__(U_THREADS, 1)
    gram_umma_kernel(long long nKB, int splits, const int2* __restrict__ pairs, const __nv_bfloat16* __restrict__ VU,
                     unsigned long long* __restrict__ P, int* __restrict__ status) {
  static_assert(MP % 16 == 0 && MP <= 128, "N of the MMA");
  constexpr unsigned TILE = MP * 128;  // one 64-row step of one slice
  constexpr unsigned ATILE = 128 * 128;  // A operand: 128 MMA rows, zero beyond MP
  constexpr unsigned STAGE = ATILE + TILE;
  constexpr int HALF = MP / 2;  // accumulator columns per epilogue thread
  constexpr unsigned IDESC = umma_idesc(128, MP);
  extern __shared__ unsigned char usm_raw[];
  unsigned char* usm = usm_raw + ((1024u - (smem_u32(usm_raw) & 1023u)) & 1023u);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(usm + U_STAGES * STAGE);
  // bars: full[U_STAGES], empty[U_STAGES], tfull[2], tempty[2], fin
  unsigned* tslot = reinterpret_cast<unsigned*>(bars + 2 * U_STAGES + 5);
  volatile int* stop = reinterpret_cast<volatile int*>(tslot + 1);
  const unsigned sbase = smem_u32(usm), bbase = smem_u32(bars);
  auto full = [&](int s) { return bbase + 8u * s; };
  auto empty = [&](int s) { return bbase + 8u * (U_STAGES + s); };
  auto tfull = [&](int b) { return bbase + 8u * (2 * U_STAGES + b); };
  auto tempty = [&](int b) { return bbase + 8u * (2 * U_STAGES + 2 + b); };
  const unsigned fin = bbase + 8u * (2 * U_STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 st = pairs[blockIdx.x];
  const long long kb0 = nKB * blockIdx.y / splits, kb1 = nKB * (blockIdx.y + 1) / splits;
  const int nkb = (int)(kb1 - kb0);
  const int nch = (nkb + U_CHUNK_KB - 1) / U_CHUNK_KB;

  if constexpr (ATILE > TILE) {  // MMA rows MP..127 of every A stage read zeros
    constexpr int W = (ATILE - TILE) / 16;
    for (int i = threadIdx.x; i < U_STAGES * W; i += blockDim.x)
      reinterpret_cast<uint4*>(usm + (i / W) * STAGE + TILE)[i % W] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < U_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), U_EPI_WARPS);
    }
    mbar_init(fin, 1);
    *stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the zero rows, for the tensor cores
  if (warp == U_EPI_WARPS + 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(U_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = *tslot;

  if (warp == U_EPI_WARPS) {
    if (lane == 0) {  // ---- copies
      const unsigned char* srcA = reinterpret_cast<const unsigned char*>(VU) + ((size_t)st.x * nKB + kb0) * TILE;
      const unsigned char* srcB = reinterpret_cast<const unsigned char*>(VU) + ((size_t)st.y * nKB + kb0) * TILE;
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int s = i % U_STAGES;
        if (i >= U_STAGES && !mbar_wait(empty(s), (unsigned)((i / U_STAGES - 1) & 1), stop)) {
          if (!*stop) atomicOr(status, ST_TIMEOUT);
          *stop = 1;
          break;
        }
        mbar_expect_tx(full(s), 2 * TILE);
        bulk_g2s(sbase + s * STAGE, srcA + (size_t)i * TILE, TILE, full(s));
        bulk_g2s(sbase + s * STAGE + ATILE, srcB + (size_t)i * TILE, TILE, full(s));
        issued = i + 1;
      }
      // the last copies of every stage have landed before the block ends
      for (int i = max(0, issued - U_STAGES); i < issued; ++i)
        if (!mbar_wait(full(i % U_STAGES), (unsigned)((i / U_STAGES) & 1), nullptr)) atomicOr(status, ST_TIMEOUT);
    }
  } else if (warp == U_EPI_WARPS + 1) {
    if (lane == 0) {  // ---- MMAs
      int i = 0;
      bool ok = true;
      for (int c = 0; c < nch && ok; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(tempty(b), (unsigned)(((c >> 1) - 1) & 1), stop)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const unsigned d = tbase + (unsigned)b * 128u;
        const int kend = min(nkb, (c + 1) * U_CHUNK_KB);
        for (; i < kend; ++i) {
          const int s = i % U_STAGES;
          if (!mbar_wait(full(s), (unsigned)((i / U_STAGES) & 1), stop)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const unsigned a0 = sbase + s * STAGE, b0 = a0 + ATILE;
#pragma unroll
          for (int kk = 0; kk < U_KB / 16; ++kk)
            umma_bf16(d, umma_desc(a0 + kk * 256u, 128u, 1024u), umma_desc(b0 + kk * 256u, 128u, 1024u), IDESC,
                      (i > c * U_CHUNK_KB || kk > 0) ? 1u : 0u);
          umma_commit(empty(s));  // the stage is free once these MMAs have read it
        }
        if (ok) umma_commit(tfull(b));
      }
      if (!ok) {
        if (!*stop) atomicOr(status, ST_TIMEOUT);
        *stop = 1;
      }
      umma_commit(fin);  // every MMA of this thread has completed before TMEM is freed
      if (!mbar_wait(fin, 0u, nullptr)) atomicOr(status, ST_TIMEOUT);
    }
  } else {  // ---- drain: warps 0..7
    const int quad = warp & 3, half = warp >> 2;
    int acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0;
    for (int c = 0; c < nch; ++c) {
      const int b = c & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull(b), (unsigned)((c >> 1) & 1), stop));
      if (!ok) {  // warp-uniform, so the aligned TMEM loads below stay convergent
        if (lane == 0 && !*stop) atomicOr(status, ST_TIMEOUT);
        *stop = 1;
        break;
      }
      tc_fence_after();
      const unsigned taddr = tbase + ((unsigned)(quad * 32) << 16) + (unsigned)b * 128u + (unsigned)(half * HALF);
      unsigned r[HALF];
#pragma unroll
      for (int g = 0; g < HALF / 8; ++g) tmem_ld8(taddr + 8u * g, r + 8 * g);
#pragma unroll
      for (int g = 0; g < HALF / 8; ++g) tmem_wait8(r + 8 * g);
#pragma unroll
      for (int j = 0; j < HALF; ++j) acc[j] += __float2int_rn(__uint_as_float(r[j]));
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(b));
    }
    const int m = quad * 32 + lane;
    if (m < MP && !*stop) {
      unsigned long long* out = P + ((size_t)blockIdx.x * MP + m) * MP + half * HALF;
#pragma unroll
      for (int j = 0; j < HALF; ++j)
        if (acc[j]) atomicAdd(out + j, (unsigned long long)(long long)acc[j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == U_EPI_WARPS + 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(U_TMEM_COLS) : "memory");
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

// Stage 2 on the tensor cores: G = A^T A + gamma I and r = A^T b into dG, dr
// (tcgen05 kernel, or the mma.sync kernel when legacy_mma).
int pod_handle::fit_gram_tc(double gamma, double* dG, double* dr, bool legacy_mma) {
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
  // mma.sync: one block per SM (128 registers a thread), splits fill one wave.
  // tcgen05: about four waves of one block per SM, at most U_MAX_ROWS rows a block.
  const long long nKB = RP / U_KB;
  int splits;
  if (legacy_mma) {
    splits = (int)std::max<long long>(1, std::min<long long>(TC_SPLITS_MAX, 152 / np));
  } else {
    const long long need = (nKB * U_KB + U_MAX_ROWS - 1) / U_MAX_ROWS;
    splits = (int)std::max<long long>(need, std::min<long long>(nKB, std::max(1, 4 * 152 / np)));
  }
  const int psplits = legacy_mma ? splits : 1;  // tcgen05 blocks add into one integer sum per pair
  const size_t vt_bytes = sizeof(__nv_bfloat16) * SLICES * (size_t)Mp * RP;
  const size_t part_bytes = sizeof(long long) * (size_t)np * psplits * Mp * Mp;
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
  cudaError_t e = cudaSuccess;
  if (!fit_capturing) {  // (a recorded fit reuses the pairs its first run uploaded)
    e = cudaMemcpy(dpairs, hp, sizeof(int) * 2 * np, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "Gram slice pairs");
  }
  const double* AT = (const double*)fitA.p;
  gram_colmax_kernel<<<dim3((unsigned)M, TC_COLBLK), 256, 0, fit_st>>>(R, AT, pmax);
  gram_colexp_kernel<<<(M + 127) / 128, 128, 0, fit_st>>>(M, TC_COLBLK, pmax, dex);
  const long long nel = (long long)Mp * RP;
  if (legacy_mma)
    gram_slice_kernel<<<(unsigned)((nel + 255) / 256), 256, 0, fit_st>>>(M, Mp, R, RP, SLICES, AT, dex, VT);
  else
    gram_slice_tiled_kernel<<<(unsigned)((nel / 8 + 255) / 256), 256, 0, fit_st>>>(M, Mp, R, RP, SLICES, AT, dex,
                                                                                       VT);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "Gram slicing");
  const dim3 grid((unsigned)np, (unsigned)splits);
  if (legacy_mma) {
    const size_t smem = (size_t)TC_STAGES * 2 * Mp * 64;
    static size_t granted7[64] = {}, granted8[64] = {};
    if (Mp == 112) {
      if ((e = grant_smem((const void*)gram_tc_kernel<7>, smem, granted7)) != cudaSuccess)
        return cuda_fail(e, "Gram shared memory");
      gram_tc_kernel<7><<<grid, 2 * 7 * 32, smem, fit_st>>>(Mp, RP, splits, dpairs, VT, part);
    } else {
      if ((e = grant_smem((const void*)gram_tc_kernel<8>, smem, granted8)) != cudaSuccess)
        return cuda_fail(e, "Gram shared memory");
      gram_tc_kernel<8><<<grid, 2 * 8 * 32, smem, fit_st>>>(Mp, RP, splits, dpairs, VT, part);
    }
  } else {
    if ((e = cudaMemsetAsync(part, 0, part_bytes, fit_st)) != cudaSuccess) return cuda_fail(e, "Gram sums clear");
    // stages, 1,024 bytes of alignment slack, barriers, TMEM address and stop flag
    const size_t smem = (size_t)U_STAGES * (128 * 128 + Mp * 128) + 1024 + 8 * (2 * U_STAGES + 5) + 16;
    static size_t grantedu7[64] = {}, grantedu8[64] = {};
    unsigned long long* P = (unsigned long long*)part;
    if (Mp == 112) {
      if ((e = grant_smem((const void*)gram_umma_kernel<112>, smem, grantedu7)) != cudaSuccess)
        return cuda_fail(e, "Gram shared memory");
      gram_umma_kernel<112><<<grid, U_THREADS, smem, fit_st>>>(nKB, splits, dpairs, VT, P, (int*)status.p);
    } else {
      if ((e = grant_smem((const void*)gram_umma_kernel<128>, smem, grantedu8)) != cudaSuccess)
        return cuda_fail(e, "Gram shared memory");
      gram_umma_kernel<128><<<grid, U_THREADS, smem, fit_st>>>(nKB, splits, dpairs, VT, P, (int*)status.p);
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "Gram tensor-core kernel");
  gram_tc_combine_kernel<<<(M * M + 255) / 256, 256, 0, fit_st>>>(M, Mp, np, psplits, dpairs, part, dex, gamma, dG);
  atb_partial_kernel<<<dim3((unsigned)M, TC_COLBLK), 256, 0, fit_st>>>(R, AT, (const double*)fitb.p, apart);
  atb_final_kernel<<<(M + 127) / 128, 128, 0, fit_st>>>(M, TC_COLBLK, apart, dr);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "Gram assembly");
  return POD_OK;
}

extern "C" int pod_selftest_wait(long long limit_ns, int* status_out) {
  if (!status_out || limit_ns < 0 || limit_ns > 10000000000LL) return POD_EINVAL;
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return POD_ENOMEM;
  e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32>>>((unsigned long long)limit_ns, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(status_out, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? POD_OK : POD_ECUDA;
}
