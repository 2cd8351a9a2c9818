// Internal definitions shared by the fastpod CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace fastpod {

// ---------------------------------------------------------------- limits
constexpr int MAXA = 8;    // alpha values per beta
constexpr int MAXB = 2;    // beta values
constexpr int MAXG = 8;    // gamma values
constexpr int MAXK = 16;   // radial modes (= lanes per atom in the atom kernels)
constexpr int MAXROWS = MAXA * MAXB + MAXG;
constexpr int PAMAX = 4;   // highest angular degree compiled
// FP32 path: forces accumulate as 64-bit fixed-point integers with 32 fraction
// bits (integer addition is associative, so the sums are reproducible whatever
// the order of the atomic adds); |F| up to 2^30 eV/A, resolution 2.3e-10 eV/A.
constexpr float FIX_SCALE_F = 4294967296.0f;     // 2^32
constexpr double FIX_INV_SCALE = 1.0 / 4294967296.0;
constexpr float FIX_GMAX = 1073741824.0f;        // 2^30: larger pair gradients are reported
// Energy and virial totals of the FP32 path, fixed point with 2^-36 resolution,
// in the accumulators after the N force rows.  A contribution X (an energy or a
// virial component times 2^36) is added as its low 32 bits (unsigned) to one
// 64-bit sum and its high part X >> 32 (signed) to another, so the totals are
// exact, independent of the order of the atomics, and cannot overflow for any
// system the device holds.  Entry 2q is the low sum of quantity q and 2q + 1 the
// high sum (q = 0: E, q = 1..9: the virial, row major); EW_COPIES copies of these
// 32 entries (warp w adds to copy w mod EW_COPIES) keep the atomics on any one
// address few.
constexpr int EW_STRIDE = 32;
constexpr int EW_COPIES = 64;
constexpr int FACC_TAIL = EW_STRIDE * EW_COPIES;
constexpr float EW_SCALE_F = 68719476736.0f;     // 2^36
constexpr float EW_MAX_ATOM = 2097152.0f;        // 2^21: larger atom energies are reported
constexpr float EW_MAX_WARP = 67108864.0f;       // 2^26: larger per-warp virial sums are reported

__device__ __forceinline__ void ew_add(unsigned long long* acc, long long X) {
  atomicAdd(acc, (unsigned long long)(X & 0xffffffffll));
  atomicAdd(acc + 1, (unsigned long long)(X >> 32));
}

// Value of one fixed-point total over the copies, summed by the 32 lanes of a
// warp (lane l takes copies l, l + 32, ...): (high + carry of low) * 2^-4 +
// (low mod 2^32) * 2^-36, the integer sums exact in any order.  All lanes
// return the value.
__device__ __forceinline__ double ew_value_warp(const unsigned long long* acc, int lane) {
  unsigned long long lo = 0, hs = 0;
#pragma unroll
  for (int c = lane; c < EW_COPIES; c += 32) {
    const unsigned long long l = acc[c * EW_STRIDE], h = acc[c * EW_STRIDE + 1];
    hs += h + (l >> 32);
    lo += l & 0xffffffffull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    hs += __shfl_xor_sync(0xffffffffu, hs, o);
    lo += __shfl_xor_sync(0xffffffffu, lo, o);
  }
  const long long hi = (long long)hs + (long long)(lo >> 32);
  return (double)hi * 0.0625 + (double)(lo & 0xffffffffull) * (1.0 / 68719476736.0);
}
constexpr int MAXM = 1 + MAXK + MAXK * (PAMAX + 1) + MAXK * 11;  // descriptors (11 = four-body K_a at P = 4)
constexpr int CH = 32;     // pairs per atom staged in shared memory at a time
constexpr int WPB_ATOM = 2;   // warps per block, atom kernels (default launch shape)
constexpr int WPB_NEIGH = 4;  // warps per block, neighbour kernels (default launch shape)
constexpr int ATOM_MAX_WPB = 4;   // launch shapes the kernels accept (autotuned per system size)
constexpr int NEIGH_MAX_WPB = 8;
constexpr int GATHER_MAX_WPB = 16;

// device status bits (OR-ed into a status word, read by the host)
constexpr int ST_NEIGH = 1;      // more neighbours than the list capacity
constexpr int ST_CELL = 2;       // more atoms in a cell than the cell capacity
constexpr int ST_RANGE = 4;      // pair with r <= r_in
constexpr int ST_NONFINITE = 8;  // NaN / Inf in positions
constexpr int ST_REV = 16;       // reverse pair not found (broken list symmetry)
constexpr int ST_OVERFLOW = 32;  // a force, energy or virial beyond the mixed path's fixed-point range
constexpr int ST_TIMEOUT = 64;   // a bounded wait inside a kernel ran out (the kernel stopped early)

// ------------------------------------------------ small vector of 4 T
template <typename T>
struct alignas(4 * sizeof(T)) Q4 {
  T x, y, z, w;
};

// ------------------------------------------------ radial parameters
// Snapshot rows: phi(alpha_a, beta_b) at row a * n_beta + b, then varphi(gamma_g)
// at row n_alpha * n_beta + g (Eq. 3, Eq. 11).  Q rows padded to MAXK columns.
template <typename T>
struct RadialConst {
  T r_in, inv_h;
  T alpha[MAXA];
  T beta[MAXB];
  T inv_ebm1[MAXB];  // 1 / (exp(-beta) - 1)
  T gamma[MAXG];
  T Q[MAXROWS][MAXK];
  int n_alpha, n_beta, n_gamma, K;
  int alpha_seq;  // alpha == {1, 2, ..., n_alpha}: sin(k pi x) by angle addition
  int gamma_seq;  // gamma == {1, 2, ..., n_gamma}: r^-g by repeated products
  // Optional tabulated basis: cubic Hermite pieces of R_k on tab_n equal
  // intervals of (r_in, r_cut), built in FP64 from the same snapshots and Q;
  // piece (g, k) holds (a, b, c, d) with R_k = a + t (b + t (c + t d)),
  // t = (r - r_in) / h - g in [0, 1].  NULL -> evaluate the snapshots directly.
  const Q4<T>* tab;
  T tab_inv_h;
  int tab_n;
};

// ------------------------------------------------ cell grid
struct CellGrid {
  int nc[3];      // cells per direction
  int S[3];       // cell offsets searched per direction
  int pbc[3];
  double L[3];    // box lengths
  float Lf[3];    // box lengths rounded to FP32 (image offsets of the FP32 prefilter)
  float Ll[3];    // L - Lf rounded to FP32 (low part of the box for double-float displacements)
  double inv_cs[3];
  int ncells;
  int cap;        // atoms per cell
};

// ------------------------------------------------ one configuration of a batch
struct CfgBox {
  double L[3];
  float Lh[3], Ll[3];  // FP32 hi / lo split of L
  int pbc[3];
  int S[3];            // images searched per direction
  int a0, a1;          // atom range [a0, a1)
};

// ------------------------------------------------ packed image shift
// x * 2^e as a double, rounded to nearest even exactly as (double)x * 2^e is
// (x a 64-bit integer with |x| < 2^63; e such that nonzero results stay normal),
// with integer operations only: the FP64 pipe, slow on this part, bounds a
// streaming pass that converts three fixed-point values per atom through it.
__host__ __device__ __forceinline__ double fixed_to_double(long long x, int e) {
  if (x == 0) return 0.0;
  const unsigned long long sign = x < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
#ifdef __CUDA_ARCH__
  int p = 63 - __clzll((long long)m);  // position of the leading one
#else
  int p = 63 - __builtin_clzll(m);
#endif
  unsigned long long q;
  if (p <= 52) {
    q = m << (52 - p);
  } else {  // round the bits below the 53 kept ones to nearest even
    const int sh = p - 52;
    const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q = m >> sh;
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    if (q >> 53) {  // the rounding carried into a new leading bit
      q >>= 1;
      ++p;
    }
  }
  const unsigned long long bits = sign | ((unsigned long long)(p + 1023 + e) << 52) | (q & ((1ull << 52) - 1ull));
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  static_assert(sizeof(d) == sizeof(bits), "64-bit double");
  __builtin_memcpy(&d, &bits, sizeof(d));
  return d;
#endif
}

__host__ __device__ __forceinline__ int shift_pack(int sx, int sy, int sz) {
  return ((sx + 128) << 16) | ((sy + 128) << 8) | (sz + 128);
}
__host__ __device__ __forceinline__ void shift_unpack(int code, int& sx, int& sy, int& sz) {
  sx = ((code >> 16) & 0xFF) - 128;
  sy = ((code >> 8) & 0xFF) - 128;
  sz = (code & 0xFF) - 128;
}
__host__ __device__ __forceinline__ int shift_negate(int code) {
  int sx, sy, sz;
  shift_unpack(code, sx, sy, sz);
  return shift_pack(-sx, -sy, -sz);
}

// Slot of the reverse pair (j, i, -s) in j's row: lower bound on the atom index
// over the sentinel-padded sorted row, then a scan over equal indices for the
// negated shift.  -1 if absent.
__device__ __forceinline__ int find_reverse(const int* __restrict__ nbr_j, const int* __restrict__ nbr_s, int cap,
                                            int i, int j, int code) {
  const int want = shift_negate(code);
  const int* row = nbr_j + (size_t)j * cap;
  int lo = 0, hi = cap;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(row + mid) < i) lo = mid + 1; else hi = mid;
  }
  for (int t = lo; t < cap && __ldg(row + t) == i; ++t)
    if (__ldg(nbr_s + (size_t)j * cap + t) == want) return (int)((size_t)j * cap + t);
  return -1;
}

// ------------------------------------------------ displacements
// FP64: d = (x_j + s L) - x_i, every operation rounded separately (no FMA), the
// expression the neighbour test is defined on.
__device__ __forceinline__ double disp_fp64(double xi, double xj, int s, double L) {
  return __dsub_rn(__dadd_rn(xj, __dmul_rn((double)s, L)), xi);
}

// FP32 from a double-float split x = hi + lo of both positions and of L: the
// large terms are added with exact error terms (two-sum) so the small
// displacement keeps FP32 relative accuracy even when |x| ~ L >> |d|.
__device__ __forceinline__ float disp_f32(float hi_i, float lo_i, float hi_j, float lo_j, int s, float Lh,
                                          float Ll) {
  const float a = hi_j, b = -hi_i;
  const float t = __fadd_rn(a, b);
  const float bb = __fsub_rn(t, a);
  const float e1 = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
  const float sf = (float)s;
  const float sL = __fmul_rn(sf, Lh);
  const float e3 = __fmaf_rn(sf, Lh, -sL);  // exact rounding error of s * Lh
  const float t2 = __fadd_rn(t, sL);
  const float bb2 = __fsub_rn(t2, t);
  const float e2 = __fadd_rn(__fsub_rn(t, __fsub_rn(t2, bb2)), __fsub_rn(sL, bb2));
  const float lo = __fadd_rn(__fsub_rn(lo_j, lo_i), __fmul_rn(sf, Ll));
  return __fadd_rn(t2, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(lo, e3)));
}

// ------------------------------------------------ math wrappers
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double d_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void d_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void d_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ float d_exp2(float x) { return exp2f(x); }
__device__ __forceinline__ double d_exp2(double x) { return exp2(x); }
__device__ __forceinline__ float d_log2(float x) { return log2f(x); }
__device__ __forceinline__ double d_log2(double x) { return log2(x); }

__device__ __forceinline__ Q4<float> ldg_q4(const Q4<float>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  Q4<float> q;
  q.x = v.x;
  q.y = v.y;
  q.z = v.z;
  q.w = v.w;
  return q;
}
__device__ __forceinline__ Q4<double> ldg_q4(const Q4<double>* p) { return *p; }

// Two consecutive table entries with one 256-bit read-only load (sm_100 and
// later; p 32-byte aligned): half the load instructions, and half the L1
// wavefronts, of two 128-bit loads of lanes that each read a different row.
__device__ __forceinline__ void ldg_q4x2(const Q4<float>* p, Q4<float>& a, Q4<float>& b) {
  asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
               : "l"(p));
}

// ------------------------------------------------ radial basis of one pair
// R_k(r) = sum_l Q_lk Phi_l(r) and R'_k(r), Phi_l = f_c psi_l (Eq. 3-12).
// KT is a compile-time bound on K (K = KT in the specialised kernels).
template <typename T, int KT>
__device__ __forceinline__ void radial_pair(const RadialConst<T>& rc, T r, T* R, T* Rp) {
  if (rc.tab) {
    const T tr = (r - rc.r_in) * rc.tab_inv_h;
    const int g = min((int)tr, rc.tab_n - 1);
    const T t = tr - T(g);
    const Q4<T>* row = rc.tab + (size_t)g * rc.K;
    if constexpr (std::is_same<T, float>::value && KT != MAXK && KT % 2 == 0) {
      // rows of an even number of 16-byte entries start on 32 bytes (the table
      // itself is 256-byte aligned): entries in pairs
#pragma unroll
      for (int k = 0; k < KT; k += 2) {
        Q4<T> q0, q1;
        ldg_q4x2(row + k, q0, q1);
        R[k] = fma(t, fma(t, fma(t, q0.w, q0.z), q0.y), q0.x);
        Rp[k] = fma(t, fma(t * T(3), q0.w, T(2) * q0.z), q0.y) * rc.tab_inv_h;
        R[k + 1] = fma(t, fma(t, fma(t, q1.w, q1.z), q1.y), q1.x);
        Rp[k + 1] = fma(t, fma(t * T(3), q1.w, T(2) * q1.z), q1.y) * rc.tab_inv_h;
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      if (KT == MAXK && k >= rc.K) {
        R[k] = T(0);
        Rp[k] = T(0);
        continue;
      }
      const Q4<T> q = ldg_q4(row + k);
      R[k] = fma(t, fma(t, fma(t, q.w, q.z), q.y), q.x);
      Rp[k] = fma(t, fma(t * T(3), q.w, T(2) * q.z), q.y) * rc.tab_inv_h;
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < KT; ++k) { R[k] = T(0); Rp[k] = T(0); }
  const T s = r - rc.r_in;
  const T inv_s = T(1) / s;
  const T t = s * rc.inv_h;
  const T t2 = t * t;
  const T u3 = T(1) - t2 * t;
  const T y = fma(u3, u3, T(1e-6));   // epsilon of Eq. 8
  const T rs = d_rsqrt(y);
  const T fc = d_exp(T(1) - rs);
  const T dfc = fc * (u3 * (T(-3) * t2 * rc.inv_h)) * (rs * rs * rs);
  const int K = rc.K;
  auto accum = [&](int row, T phi, T dphi) {
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      if (KT == MAXK && k >= K) break;
      const T q = rc.Q[row][k];
      R[k] = fma(q, phi, R[k]);
      Rp[k] = fma(q, dphi, Rp[k]);
    }
  };
  for (int ib = 0; ib < rc.n_beta; ++ib) {
    const T be = rc.beta[ib];
    const T et = d_exp(-be * t);
    const T x = (et - T(1)) * rc.inv_ebm1[ib];
    const T dx = -be * rc.inv_h * et * rc.inv_ebm1[ib];
    if (rc.alpha_seq) {
      T s1, c1;
      d_sincospi(x, &s1, &c1);
      T sk = s1, ck = c1;
      for (int ia = 0; ia < rc.n_alpha; ++ia) {
        const T apdx = T(ia + 1) * T(3.14159265358979323846) * dx;
        const T f = sk * inv_s;
        const T df = (apdx * ck - f) * inv_s;
        accum(ia * rc.n_beta + ib, fc * f, fma(dfc, f, fc * df));
        const T sn = fma(sk, c1, ck * s1);  // sin((k+1) pi x)
        const T cn = fma(ck, c1, -sk * s1); // cos((k+1) pi x)
        sk = sn;
        ck = cn;
      }
    } else {
      for (int ia = 0; ia < rc.n_alpha; ++ia) {
        const T al = rc.alpha[ia];
        T sk, ck;
        d_sincospi(al * x, &sk, &ck);
        const T f = sk * inv_s;
        const T df = (al * T(3.14159265358979323846) * dx * ck - f) * inv_s;
        accum(ia * rc.n_beta + ib, fc * f, fma(dfc, f, fc * df));
      }
    }
  }
  const int row0 = rc.n_alpha * rc.n_beta;
  const T ir = T(1) / r;
  if (rc.gamma_seq) {
    T f = T(1);
    for (int ig = 0; ig < rc.n_gamma; ++ig) {
      f *= ir;
      const T df = -T(ig + 1) * f * ir;
      accum(row0 + ig, fc * f, fma(dfc, f, fc * df));
    }
  } else {
    const T lr = d_log2(r);
    for (int ig = 0; ig < rc.n_gamma; ++ig) {
      const T ga = rc.gamma[ig];
      const T f = d_exp2(-ga * lr);
      const T df = -ga * f * ir;
      accum(row0 + ig, fc * f, fma(dfc, f, fc * df));
    }
  }
}

}  // namespace fastpod
