// Fused per-atom kernel: radial snapshots + POD projection (Eq. 3-12), atomic
// basis B_imnl (Eq. 24b), contraction into D2 / D3 / D4 (Eq. 12b, 26a, 27a, 30a),
// energy E_i = c . D_i (Eq. 57a), adjoint dE_i/dB and the adjoint pair pass
// g_ij = dE_i/dr_ij (Eq. 24c, 26c) -- one launch, all intermediates on chip.
//
// Work mapping (one warp holds A = 32 / K atoms):
//   pair pass      lanes over the flattened (atom, neighbour) pairs of the warp;
//                  each lane evaluates one pair's snapshots, R_k and R'_k and
//                  stages (u, r, R, R') in shared memory;
//   B and contraction  lane (atom, m) owns B_m[0..N_a) in registers, so every
//                  D3/D4 product and the whole adjoint run in registers;
//   adjoint pair pass  lanes over pairs again, reading dE/dB_m from shared memory.
//
// Modes: 0 descriptors, 1 linear energy and forces, 2 descriptor tangent, 3
// design-matrix pair gradients, 4 quadratic model, 5 embedding model.
#pragma once
#include <type_traits>

#include "contract_gen.cuh"
#include "pod_common.cuh"
#include "pod_kernels.h"

namespace fastpod {

// (u, r) of a displacement: r = |d|, u = d / r.  Every kernel forming pair
// geometry uses this one expression, so they agree bit for bit.
template <typename T>
__device__ __forceinline__ Q4<T> pair_unit(T dx, T dy, T dz) {
  const T r = d_sqrt(dx * dx + dy * dy + dz * dz);
  const T ir = T(1) / r;
  Q4<T> q;
  q.x = dx * ir;
  q.y = dy * ir;
  q.z = dz * ir;
  q.w = r;
  return q;
}

template <typename T>
__device__ __forceinline__ void pair_disp(const AtomArgs<T>& p, int i, int j, int sx, int sy, int sz, T& dx, T& dy,
                                          T& dz);

template <>
__device__ __forceinline__ void pair_disp<double>(const AtomArgs<double>& p, int i, int j, int sx, int sy, int sz,
                                                  double& dx, double& dy, double& dz) {
  const size_t N = p.N;
  const double* L = p.cfg_of ? p.cbox[p.cfg_of[i]].L : p.L;
  dx = disp_fp64(p.wpos[i], p.wpos[j], sx, L[0]);
  dy = disp_fp64(p.wpos[N + i], p.wpos[N + j], sy, L[1]);
  dz = disp_fp64(p.wpos[2 * N + i], p.wpos[2 * N + j], sz, L[2]);
}

template <>
__device__ __forceinline__ void pair_disp<float>(const AtomArgs<float>& p, int i, int j, int sx, int sy, int sz,
                                                 float& dx, float& dy, float& dz) {
  const float4 hi = p.phi[i], li = p.plo[i], hj = p.phi[j], lj = p.plo[j];
  const float* Lh = p.Lh;
  const float* Ll = p.Ll;
  if (p.cfg_of) {
    const CfgBox& b = p.cbox[p.cfg_of[i]];
    Lh = b.Lh;
    Ll = b.Ll;
  }
  dx = disp_f32(hi.x, li.x, hj.x, lj.x, sx, Lh[0], Ll[0]);
  dy = disp_f32(hi.y, li.y, hj.y, lj.y, sy, Lh[1], Ll[1]);
  dz = disp_f32(hi.z, li.z, hj.z, lj.z, sz, Lh[2], Ll[2]);
}

__device__ __forceinline__ int chunk_count(int n, int ch) { return min(max(n - ch * CH, 0), CH); }

// Stage chunk `ch` of the warp's pairs: (u, r) and R, R' per pair.
template <typename T, int KT, bool TANGENT = false>
__device__ __forceinline__ void pair_pass(const AtomArgs<T>& p, const AtomLayout& lay, Q4<T>* geo, T* sR, T* sRp,
                                          const int* scnt, int atom0, int A, int K, int ch, int lane,
                                          Q4<T>* sV = nullptr, int* sj = nullptr) {
  int tot = 0;
  for (int a = 0; a < A; ++a) tot += chunk_count(scnt[a], ch);
  for (int f = lane; f < tot; f += 32) {
    int a = 0, base = 0;
    for (; a < A; ++a) {
      const int nca = chunk_count(scnt[a], ch);
      if (f < base + nca) break;
      base += nca;
    }
    const int jj = f - base, slot = ch * CH + jj, i = atom0 + a;
    const size_t pidx = (size_t)i * p.cap + slot;
    T dx, dy, dz;
    int j;
    if (std::is_same<T, float>::value && p.pd) {
      // displacement formed by the neighbour search (same arithmetic, same bits)
      const float4 q = __ldg(p.pd + pidx);
      dx = (T)q.x;
      dy = (T)q.y;
      dz = (T)q.z;
      j = __float_as_int(q.w);
    } else {
      j = p.nbr_j[pidx];
      const int code = p.nbr_s[pidx];
      int sx, sy, sz;
      shift_unpack(code, sx, sy, sz);
      pair_disp<T>(p, i, j, sx, sy, sz, dx, dy, dz);
    }
    if (sj) sj[a * lay.GA + jj] = j;
    const Q4<T> gq = pair_unit(dx, dy, dz);
    const T r = gq.w;
    geo[a * lay.GA + jj] = gq;
    T R[KT], Rp[KT];
    if (r > p.rad.r_in && r < p.rmask) {
      radial_pair<T, KT>(p.rad, r, R, Rp);
    } else {
      if (!(r > p.rad.r_in)) atomicOr(p.status, ST_RANGE);
#pragma unroll
      for (int k = 0; k < KT; ++k) { R[k] = T(0); Rp[k] = T(0); }
    }
    T* Rrow = sR + a * lay.SA + jj * lay.KS;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      if (KT == MAXK && k >= K) break;
      Rrow[k] = R[k];
    }
    if (TANGENT) {  // relative displacement direction of the pair
      const size_t N = p.N;
      Q4<T> vq;
      vq.x = (T)(p.vdir[j] - p.vdir[i]);
      vq.y = (T)(p.vdir[N + j] - p.vdir[N + i]);
      vq.z = (T)(p.vdir[2 * N + j] - p.vdir[2 * N + i]);
      vq.w = T(0);
      sV[a * lay.GA + jj] = vq;
    }
    if (!p.rad.tab || TANGENT || p.keep_rp) {  // keep R' for the adjoint / tangent pass
      T* Rprow = sRp + a * lay.SA + jj * lay.KS;
#pragma unroll
      for (int k = 0; k < KT; ++k) {
        if (KT == MAXK && k >= K) break;
        Rprow[k] = Rp[k];
      }
    }
  }
}

// Pair gradient g_ij = sum_{m,x} a_mx dB_mx/dr_ij of one pair (Eq. 24c): u = (unit
// vector, r), R and R' of the pair, adj = the atom's rows dE/dB_m (K rows of NAP,
// shared memory), s3m = dE/dS3 per mode for the exclusive three-body set (or
// NULL).  dA/dr = (grad_u A - (u . grad_u A) u) / r for homogeneous A (Euler).
// Both the fused atom kernel and the separate adjoint kernel call this, so the
// two give the same bits.
template <typename T, int PA, int KT>
__device__ __forceinline__ Q4<T> pair_gradient(const Q4<T>& u, const T* Rv, const T* Rpv, const T* adj, int K,
                                               const T* s3m) {
  constexpr int NA = Mono<PA>::NA;
  constexpr int NAP = (NA + 3) / 4 * 4;
  T Am[NAP];
  T e[NAP];
  T ps = T(0);
  if constexpr (std::is_same<T, float>::value) {
    // paired FP32 multiply-add over the basis components (a_m loaded as float4)
    float2 A2[NAP / 2], e2[NAP / 2];
    Mono<PA>::eval2(u.x, u.y, u.z, A2);
#pragma unroll
    for (int k = Mono<PA>::NA2; k < NAP / 2; ++k) A2[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NAP / 2; ++k) e2[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int mm = 0; mm < KT; ++mm) {
      if (KT == MAXK && mm >= K) break;
      const float2 R2 = make_float2(Rv[mm], Rv[mm]);
      const float4* a4 = reinterpret_cast<const float4*>(adj + mm * NAP);
      float2 u2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int x4 = 0; x4 < NAP / 4; ++x4) {
        const float4 av = a4[x4];
        const float2 lo = make_float2(av.x, av.y), hi = make_float2(av.z, av.w);
        u2 = __ffma2_rn(lo, A2[2 * x4], u2);
        u2 = __ffma2_rn(hi, A2[2 * x4 + 1], u2);
        e2[2 * x4] = __ffma2_rn(lo, R2, e2[2 * x4]);
        e2[2 * x4 + 1] = __ffma2_rn(hi, R2, e2[2 * x4 + 1]);
      }
      ps = fma(Rpv[mm], u2.x + u2.y, ps);
      if (s3m) ps = fma(T(2) * s3m[mm] * Rv[mm], Rpv[mm], ps);  // dS3/dr = 2 R R'
    }
#pragma unroll
    for (int x = 0; x < NAP; ++x) {
      Am[x] = (x & 1) ? A2[x >> 1].y : A2[x >> 1].x;
      e[x] = (x & 1) ? e2[x >> 1].y : e2[x >> 1].x;
    }
  } else {
    Mono<PA>::eval(u.x, u.y, u.z, Am);
#pragma unroll
    for (int x = NA; x < NAP; ++x) Am[x] = T(0);
#pragma unroll
    for (int x = 0; x < NAP; ++x) e[x] = T(0);
#pragma unroll
    for (int mm = 0; mm < KT; ++mm) {
      if (KT == MAXK && mm >= K) break;
      const T Rm = Rv[mm], Rpm = Rpv[mm];
      const Q4<T>* a4 = reinterpret_cast<const Q4<T>*>(adj + mm * NAP);
      T um = T(0);
#pragma unroll
      for (int x4 = 0; x4 < NAP / 4; ++x4) {
        const Q4<T> av = a4[x4];
        um = fma(av.x, Am[4 * x4 + 0], um);
        um = fma(av.y, Am[4 * x4 + 1], um);
        um = fma(av.z, Am[4 * x4 + 2], um);
        um = fma(av.w, Am[4 * x4 + 3], um);
        e[4 * x4 + 0] = fma(av.x, Rm, e[4 * x4 + 0]);
        e[4 * x4 + 1] = fma(av.y, Rm, e[4 * x4 + 1]);
        e[4 * x4 + 2] = fma(av.z, Rm, e[4 * x4 + 2]);
        e[4 * x4 + 3] = fma(av.w, Rm, e[4 * x4 + 3]);
      }
      ps = fma(Rpm, um, ps);
      if (s3m) ps = fma(T(2) * s3m[mm] * Rm, Rpm, ps);  // dS3/dr = 2 R R'
    }
  }
  T gx, gy, gz;
  Mono<PA>::grad(e, Am, gx, gy, gz);
  // dA/dr = (grad_u A - (u . grad_u A) u) / r for homogeneous A (Euler)
  const T ug = u.x * gx + u.y * gy + u.z * gz;
  const T ir = T(1) / u.w;
  Q4<T> out;
  out.x = fma(ps, u.x, (gx - ug * u.x) * ir);
  out.y = fma(ps, u.y, (gy - ug * u.y) * ir);
  out.z = fma(ps, u.z, (gz - ug * u.z) * ir);
  out.w = T(0);
  return out;
}

// FP32 specialised kernels are held to 128 registers (4 blocks of 4 warps per SM): the
// paired multiply-add operands otherwise push them past that without a gain.
template <typename T, int MODE, int KT>
constexpr int atom_min_blocks() {
  // the design mode is held to 6 blocks of 2 warps per SM by its shared memory,
  // so it takes up to 168 registers at no cost in occupancy
  return (std::is_same<T, float>::value && MODE != 2 && KT != MAXK) ? (MODE == 3 ? 3 : 4) : 1;
}

template <typename T, int PA, bool HAS4, int MODE, int KT>
__global__ void __launch_bounds__(ATOM_MAX_WPB * 32, atom_min_blocks<T, MODE, KT>())
    atom_kernel(const AtomArgs<T> p, const AtomLayout lay) {
  constexpr int NA = Mono<PA>::NA;
  constexpr int NAP = (NA + 3) / 4 * 4;
  constexpr int KA = HAS4 ? Four<PA>::KA : 1;
  extern __shared__ __align__(32) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wb = sm + (size_t)warp * lay.warp_bytes;
  Q4<T>* geo = reinterpret_cast<Q4<T>*>(wb + lay.off_geo);
  T* sR = reinterpret_cast<T*>(wb + lay.off_R);
  T* sRp = reinterpret_cast<T*>(wb + lay.off_Rp);
  T* sadj = reinterpret_cast<T*>(wb + lay.off_adj);
  T* se = reinterpret_cast<T*>(wb + lay.off_e);
  int* scnt = reinterpret_cast<int*>(wb + lay.off_cnt);
  Q4<T>* sV = reinterpret_cast<Q4<T>*>(wb + lay.off_V);
  // neighbour index of each staged pair (energy modes with a displacement list)
  int* sj = (std::is_same<T, float>::value && p.pd && lay.off_J) ? reinterpret_cast<int*>(wb + lay.off_J) : nullptr;

  const int K = (KT == MAXK) ? p.K : KT;
  const int A = (KT == MAXK) ? lay.A : 32 / KT;
  const int a_loc = lane / K;
  const int m = lane - a_loc * K;
  const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;  // global warp index
  const int atom0 = gwarp * A;
  // energy modes (1: linear model, 4: quadratic model): the block converts the
  // coefficients to T once (shared memory)
  constexpr bool EMODE = (MODE == 1 || MODE == 4 || MODE == 5);
  __shared__ T sc[MAXM];
  if (EMODE) {
    for (int q = threadIdx.x; q < p.M; q += blockDim.x) sc[q] = (T)p.c[q];
    __syncthreads();
  }
  // FP32 energy modes: E and the virial accumulate in fixed point (the tail of
  // the force accumulators); FP64: per-warp virial partials for the gather
  constexpr bool FIXP = EMODE && std::is_same<T, float>::value;
  if (atom0 >= p.n_eval) {  // uniform per warp
    if (EMODE && !FIXP && lane < 9) p.wpart[(size_t)gwarp * 9 + lane] = 0.0;
    return;
  }
  if (lane < A) {
    const int i = atom0 + lane;
    scnt[lane] = (i < p.n_eval) ? min(p.nbr_count[i], p.cap) : 0;
  }
  __syncwarp();
  int nmax = 0;
  for (int a = 0; a < A; ++a) nmax = max(nmax, scnt[a]);
  const int nchunks = (nmax + CH - 1) / CH;
  const bool am = (a_loc < A) && (atom0 + a_loc < p.n_eval);
  const int my_n = am ? scnt[a_loc] : 0;

  if (MODE == 2) {
    // ---------------- tangent: dD_i along relative displacements (v_j - v_i) per pair
    T B[NA], Bd[NA];
#pragma unroll
    for (int x = 0; x < NA; ++x) { B[x] = T(0); Bd[x] = T(0); }
    for (int ch = 0; ch < nchunks; ++ch) {
      pair_pass<T, KT, true>(p, lay, geo, sR, sRp, scnt, atom0, A, K, ch, lane, sV);
      __syncwarp();
      if (am) {
        const int nc = chunk_count(my_n, ch);
        for (int jj = 0; jj < nc; ++jj) {
          const Q4<T> u = geo[a_loc * lay.GA + jj];
          const Q4<T> v = sV[a_loc * lay.GA + jj];
          const T R = sR[a_loc * lay.SA + jj * lay.KS + m];
          const T Rp = sRp[a_loc * lay.SA + jj * lay.KS + m];
          const T sdot = u.x * v.x + u.y * v.y + u.z * v.z;  // d r / d eps
          const T ir = T(1) / u.w;
          // d u / d eps = (v - (u . v) u) / r
          T Am[NA], dA[NA];
          Mono<PA>::eval_d(u.x, u.y, u.z, (v.x - sdot * u.x) * ir, (v.y - sdot * u.y) * ir,
                           (v.z - sdot * u.z) * ir, Am, dA);
          const T Rs = Rp * sdot;
#pragma unroll
          for (int x = 0; x < NA; ++x) {
            B[x] = fma(R, Am[x], B[x]);
            Bd[x] = fma(Rs, Am[x], fma(R, dA[x], Bd[x]));
          }
        }
      }
      __syncwarp();
    }
    if (am) {
      const int i = atom0 + a_loc;
      double* Di = p.D + (size_t)i * p.M;
      if (m == 0) Di[0] = 0.0;
      if (m < p.K2) Di[1 + m] = (double)Bd[0];
      T d3[PA + 1], d3d[PA + 1];
      Mono<PA>::d3(B, d3);
      Mono<PA>::d3_tangent(B, Bd, d3d);
      if (m < p.K3) {
#pragma unroll
        for (int n = 0; n <= PA; ++n)
          if (n <= p.P3) Di[p.col3 + m * (p.P3 + 1) + n] = (double)d3d[n];
      }
      if (HAS4 && m < p.K4) {
        T Dd[KA];
        Four<PA>::tangent(B, Bd, d3, d3d, Dd);
#pragma unroll
        for (int q = 0; q < KA; ++q)
          if (q < p.KA4) Di[p.col4 + m * p.KA4 + q] = (double)Dd[q];
      }
    }
    return;
  }

  // ---------------- forward: B_m[x] = sum_j R_m(r_ij) A_x(u_ij)   (Eq. 24b),
  // and S3 = sum_j R_m(r_ij)^2 for the exclusive three-body set (Eq. 15b)
  T S3 = T(0);
  T B[NA];
#pragma unroll
  for (int x = 0; x < NA; ++x) B[x] = T(0);
  float2 B2[Mono<PA>::NA2];  // FP32 path: B accumulated in pairs
#pragma unroll
  for (int k = 0; k < Mono<PA>::NA2; ++k) B2[k] = make_float2(0.f, 0.f);
  for (int ch = 0; ch < nchunks; ++ch) {
    pair_pass<T, KT, false>(p, lay, geo, sR, sRp, scnt, atom0, A, K, ch, lane, nullptr, sj);
    __syncwarp();
    if (am) {
      const int nc = chunk_count(my_n, ch);
      const Q4<T>* ga = geo + a_loc * lay.GA;
      const T* Ra = sR + a_loc * lay.SA + m;
      if constexpr (std::is_same<T, float>::value) {
        // paired FP32 multiply-add: two basis components per instruction (two pairs
        // per iteration, so that their shared-memory reads overlap)
#pragma unroll 2
        for (int jj = 0; jj < nc; ++jj) {
          const Q4<T> u = ga[jj];
          const float R = Ra[jj * lay.KS];
          float2 A2[Mono<PA>::NA2];
          Mono<PA>::eval2(u.x, u.y, u.z, A2);
          const float2 R2 = make_float2(R, R);
#pragma unroll
          for (int k = 0; k < Mono<PA>::NA2; ++k) B2[k] = __ffma2_rn(A2[k], R2, B2[k]);
          S3 = fmaf(R, R, S3);
        }
      } else {
        for (int jj = 0; jj < nc; ++jj) {
          const Q4<T> u = ga[jj];
          const T R = Ra[jj * lay.KS];
          T Am[NA];
          Mono<PA>::eval(u.x, u.y, u.z, Am);
#pragma unroll
          for (int x = 0; x < NA; ++x) B[x] = fma(R, Am[x], B[x]);
          S3 = fma(R, R, S3);
        }
      }
    }
    __syncwarp();
  }
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int x = 0; x < NA; ++x) B[x] = (x & 1) ? B2[x >> 1].y : B2[x >> 1].x;
  }

  if (MODE == 0 || (MODE == 3 && p.D)) {
    // ---------------- descriptors (Eq. 12b, 26a, 27a, 30a)
    if (am) {
      const int i = atom0 + a_loc;
      double* Di = p.D + (size_t)i * p.M;
      if (m == 0) Di[0] = 1.0;
      if (m < p.K2) Di[1 + m] = (double)B[0];
      T d3[PA + 1];
      Mono<PA>::d3(B, d3);
      if (m < p.K3) {
        // exclusive set (Eq. 15b, pairs k > j): (D3 - sum_j R_m^2) / 2, as (u_j . u_j)^n = 1
#pragma unroll
        for (int n = 0; n <= PA; ++n)
          if (n <= p.P3) Di[p.col3 + m * (p.P3 + 1) + n] = (double)(p.excl3 ? T(0.5) * (d3[n] - S3) : d3[n]);
      }
      if (HAS4 && m < p.K4) {
        T D4[KA];
        Four<PA>::desc(B, d3, D4);
#pragma unroll
        for (int q = 0; q < KA; ++q)
          if (q < p.KA4) Di[p.col4 + m * p.KA4 + q] = (double)D4[q];
      }
    }
    if (MODE == 0) return;
  }

  if (MODE == 3) {
    // ---------------- design-matrix pair gradients.  Descriptor q of mode m is
    // the column col(q, m) of the linear model; its pair gradient
    // dD_{i,col}/dr_ij is the adjoint pair pass (Eq. 24c) with c = e_col: the
    // lane (atom, m) forms a = dD_{i,col}/dB_m (one row of the sparse Jacobian of
    // Eq. 12b, 26a, 27a, 30a), then lanes over pairs contract it with dB_m/dr_ij.
    T d3v[PA + 1];
    Mono<PA>::d3(B, d3v);
    const int n3 = p.P3 + 1;
    const int Qd = 1 + n3 + p.KA4;
    // Columns whose adjoint rows live on single degrees of the monomials -- D2
    // (a = e_0), D3_n (a_x = 2 mu_x B_x for deg x = n, Eq. 26a) and the
    // partitions (n, 0, 0) of D4 = B_0 D3_n (Eq. 27a: a = B_0 times the D3_n row
    // plus D3_n e_0) -- come out of one pass over the pairs: per pair and mode
    // the degree-resolved sums s_n = sum_{deg x = n} 2 mu_x B_x A_x and their
    // gradients, combined per column.  The general partitions (Eq. 30a) have
    // dense rows and keep a pass each (first, below).
    auto sparse_q = [&](int q) {
      if (q <= n3) return true;
      if (!HAS4) return false;
      const int pp = q - 1 - n3;
      bool hit = false;
#pragma unroll
      for (int n = 0; n <= PA; ++n) hit |= Four<PA>::p_n00(n) == pp;
      return hit;
    };
    bool any_sparse = false;
    for (int q = p.q0; q < p.q1 && q < Qd; ++q) any_sparse |= sparse_q(q);
    for (int q = p.q0; q < p.q1 && q < Qd; ++q) {
      if (sparse_q(q)) continue;  // in the pass below
      __syncwarp();
      if (am) {
        T a[NAP];
#pragma unroll
        for (int x = 0; x < NAP; ++x) a[x] = T(0);
        if (q == 0) {
          if (m < p.K2) a[0] = T(1);  // D2 = B_m00
        } else if (q <= n3) {
          if (m < p.K3) {  // D3_mn = sum_x mu_x B_x^2 over degree n
            T h[PA + 1];
#pragma unroll
            for (int n = 0; n <= PA; ++n) h[n] = (n == q - 1) ? T(1) : T(0);
            Mono<PA>::d3_adjoint(B, h, a);
          }
        } else if (HAS4) {
          const int pp = q - 1 - n3;
          if (m < p.K4 && pp < p.KA4) {
            int n00 = -1;
#pragma unroll
            for (int n = 0; n <= PA; ++n)
              if (Four<PA>::p_n00(n) == pp) n00 = n;
            if (n00 >= 0) {  // D4 = B_0 D3_n (Eq. 27a)
              T h[PA + 1];
#pragma unroll
              for (int n = 0; n <= PA; ++n) h[n] = (n == n00) ? B[0] : T(0);
              Mono<PA>::d3_adjoint(B, h, a);
#pragma unroll
              for (int n = 0; n <= PA; ++n)
                if (n == n00) a[0] += d3v[n];
            } else {  // general partition (Eq. 30a)
              T w4[KA];
#pragma unroll
              for (int qq = 0; qq < KA; ++qq) w4[qq] = (qq == pp) ? T(1) : T(0);
              Four<PA>::adjoint(B, w4, a);
            }
          }
        }
        T* adst = sadj + a_loc * lay.AS + m * NAP;
#pragma unroll
        for (int x = 0; x < NAP; ++x) adst[x] = a[x];
      }
      __syncwarp();
      for (int ch = 0; ch < nchunks; ++ch) {
        if (nchunks > 1) {
          __syncwarp();
          pair_pass<T, KT, false>(p, lay, geo, sR, sRp, scnt, atom0, A, K, ch, lane);
          __syncwarp();
        }
        int tot = 0;
        for (int a = 0; a < A; ++a) tot += chunk_count(scnt[a], ch);
        for (int f = lane; f < tot; f += 32) {
          int a = 0, base = 0;
          for (; a < A; ++a) {
            const int nca = chunk_count(scnt[a], ch);
            if (f < base + nca) break;
            base += nca;
          }
          const int jj = f - base, slot = ch * CH + jj, i = atom0 + a;
          const Q4<T> u = geo[a * lay.GA + jj];
          T Rv[KT], Rpv[KT];
          if (p.rad.tab && !p.keep_rp) {
            if (u.w > p.rad.r_in && u.w < p.rmask) {
              radial_pair<T, KT>(p.rad, u.w, Rv, Rpv);
            } else {
#pragma unroll
              for (int k = 0; k < KT; ++k) { Rv[k] = T(0); Rpv[k] = T(0); }
            }
          } else {
            const T* Rrow = sR + a * lay.SA + jj * lay.KS;
            const T* Rprow = sRp + a * lay.SA + jj * lay.KS;
#pragma unroll
            for (int k = 0; k < KT; ++k) {
              if (KT == MAXK && k >= K) break;
              Rv[k] = Rrow[k];
              Rpv[k] = Rprow[k];
            }
          }
          T Am[NAP];
          Mono<PA>::eval(u.x, u.y, u.z, Am);
#pragma unroll
          for (int x = NA; x < NAP; ++x) Am[x] = T(0);
          const T ir = T(1) / u.w;
          const T* adj = sadj + a * lay.AS;
          T* out = p.gdm + (((size_t)(q - p.q0) * p.N + i) * p.cap + slot) * (size_t)K * 3;
          // modes one at a time (a rolled loop: the unrolled body overflowed the
          // instruction cache); R and R' of the mode selected, not indexed
#pragma unroll 1
          for (int mm = 0; mm < K; ++mm) {
            T Rsel = Rv[0], Rpsel = Rpv[0];
#pragma unroll
            for (int k = 1; k < KT; ++k)
              if (k == mm) {
                Rsel = Rv[k];
                Rpsel = Rpv[k];
              }
            T am_[NAP];
            const Q4<T>* a4 = reinterpret_cast<const Q4<T>*>(adj + mm * NAP);
#pragma unroll
            for (int x4 = 0; x4 < NAP / 4; ++x4) {
              const Q4<T> av = a4[x4];
              am_[4 * x4 + 0] = av.x;
              am_[4 * x4 + 1] = av.y;
              am_[4 * x4 + 2] = av.z;
              am_[4 * x4 + 3] = av.w;
            }
            T dot = T(0);
#pragma unroll
            for (int x = 0; x < NA; ++x) dot = fma(am_[x], Am[x], dot);
            T gx, gy, gz;
            Mono<PA>::grad(am_, Am, gx, gy, gz);
            const T ug = u.x * gx + u.y * gy + u.z * gz;
            const T s1 = Rpsel * dot, s2 = Rsel * ir;
            out[3 * mm + 0] = fma(s1, u.x, s2 * (gx - ug * u.x));
            out[3 * mm + 1] = fma(s1, u.y, s2 * (gy - ug * u.y));
            out[3 * mm + 2] = fma(s1, u.z, s2 * (gz - ug * u.z));
          }
        }
      }
    }
    // (after the general columns, which still need B in registers)
    T* sd3 = reinterpret_cast<T*>(wb + lay.off_d3);
    if (any_sparse) {
      __syncwarp();
      if (am) {
        T h[NAP], one[PA + 1];
#pragma unroll
        for (int x = 0; x < NAP; ++x) h[x] = T(0);
#pragma unroll
        for (int n = 0; n <= PA; ++n) one[n] = T(1);
        Mono<PA>::d3_adjoint(B, one, h);  // h_x = 2 mu_x B_x
        T* adst = sadj + a_loc * lay.AS + m * NAP;
#pragma unroll
        for (int x = 0; x < NAP; ++x) adst[x] = h[x];
#pragma unroll
        for (int n = 0; n <= PA; ++n) sd3[(a_loc * K + m) * (PA + 1) + n] = d3v[n];
      }
      __syncwarp();
      for (int ch = 0; ch < nchunks; ++ch) {
        if (nchunks > 1) {
          __syncwarp();
          pair_pass<T, KT, false>(p, lay, geo, sR, sRp, scnt, atom0, A, K, ch, lane);
          __syncwarp();
        }
        int tot = 0;
        for (int a = 0; a < A; ++a) tot += chunk_count(scnt[a], ch);
        for (int f = lane; f < tot; f += 32) {
          int a = 0, base = 0;
          for (; a < A; ++a) {
            const int nca = chunk_count(scnt[a], ch);
            if (f < base + nca) break;
            base += nca;
          }
          const int jj = f - base, slot = ch * CH + jj, i = atom0 + a;
          const Q4<T> u = geo[a * lay.GA + jj];
          T Rv[KT], Rpv[KT];
          if (p.rad.tab && !p.keep_rp) {
            if (u.w > p.rad.r_in && u.w < p.rmask) {
              radial_pair<T, KT>(p.rad, u.w, Rv, Rpv);
            } else {
#pragma unroll
              for (int k = 0; k < KT; ++k) { Rv[k] = T(0); Rpv[k] = T(0); }
            }
          } else {
            const T* Rrow = sR + a * lay.SA + jj * lay.KS;
            const T* Rprow = sRp + a * lay.SA + jj * lay.KS;
#pragma unroll
            for (int k = 0; k < KT; ++k) {
              if (KT == MAXK && k >= K) break;
              Rv[k] = Rrow[k];
              Rpv[k] = Rprow[k];
            }
          }
          T Am[NAP];
          Mono<PA>::eval(u.x, u.y, u.z, Am);
#pragma unroll
          for (int x = NA; x < NAP; ++x) Am[x] = T(0);
          const T ir = T(1) / u.w;
          const size_t pbase = ((size_t)i * p.cap + slot) * (size_t)K * 3;
          const size_t plane = (size_t)p.N * p.cap * (size_t)K * 3;
#pragma unroll 1
          for (int mm = 0; mm < K; ++mm) {
            T R = Rv[0], Rp = Rpv[0];  // (selected, so that Rv and Rpv stay in registers)
#pragma unroll
            for (int k = 1; k < KT; ++k)
              if (k == mm) {
                R = Rv[k];
                Rp = Rpv[k];
              }
            T hm[NAP];
            const Q4<T>* h4 = reinterpret_cast<const Q4<T>*>(sadj + a * lay.AS + mm * NAP);
#pragma unroll
            for (int x4 = 0; x4 < NAP / 4; ++x4) {
              const Q4<T> hv = h4[x4];
              hm[4 * x4 + 0] = hv.x;
              hm[4 * x4 + 1] = hv.y;
              hm[4 * x4 + 2] = hv.z;
              hm[4 * x4 + 3] = hv.w;
            }
            T sn[PA + 1], gxn[PA + 1], gyn[PA + 1], gzn[PA + 1];
            Mono<PA>::dot_grad_deg(hm, Am, sn, gxn, gyn, gzn);
            const T B0 = T(0.5) * hm[0];
            const T s2 = R * ir;
            // g = R' (a . A) u + (R / r) (G - (u . G) u) for a column with a . A = dot, a . grad A = G
            auto emit = [&](int q, T dot, T Gx, T Gy, T Gz) {
              if (q < p.q0 || q >= p.q1) return;
              T* out = p.gdm + (size_t)(q - p.q0) * plane + pbase + 3 * mm;
              const T ug = u.x * Gx + u.y * Gy + u.z * Gz;
              const T s1 = Rp * dot;
              out[0] = fma(s1, u.x, s2 * (Gx - ug * u.x));
              out[1] = fma(s1, u.y, s2 * (Gy - ug * u.y));
              out[2] = fma(s1, u.z, s2 * (Gz - ug * u.z));
            };
            emit(0, mm < p.K2 ? T(1) : T(0), T(0), T(0), T(0));  // D2 = B_m,0, A_0 = 1
#pragma unroll
            for (int n = 0; n <= PA; ++n) {
              if (n <= p.P3) {
                const bool on = mm < p.K3;
                emit(1 + n, on ? sn[n] : T(0), on ? gxn[n] : T(0), on ? gyn[n] : T(0), on ? gzn[n] : T(0));
              }
              if (HAS4) {
                const int pp = Four<PA>::p_n00(n);
                if (pp < p.KA4) {
                  const bool on = mm < p.K4;
                  const T d3n = sd3[(a * K + mm) * (PA + 1) + n];
                  emit(1 + n3 + pp, on ? fma(B0, sn[n], d3n) : T(0), on ? B0 * gxn[n] : T(0),
                       on ? B0 * gyn[n] : T(0), on ? B0 * gzn[n] : T(0));
                }
              }
            }
          }
        }
      }
    }
    return;
  }

  if (MODE == 4) {
    // ---------------- quadratic model: stage this atom's descriptors (all
    // columns) so each lane can form dE_i/dD_col = c_col + sum_n S_col,n D_in
    T* sDa = reinterpret_cast<T*>(wb + lay.off_D) + a_loc * lay.MS;
    if (am) {
      T d3[PA + 1];
      Mono<PA>::d3(B, d3);
      if (m == 0) sDa[0] = T(1);
      if (m < p.K2) sDa[1 + m] = B[0];
      if (m < p.K3) {
#pragma unroll
        for (int n = 0; n <= PA; ++n)
          if (n <= p.P3) sDa[p.col3 + m * (p.P3 + 1) + n] = d3[n];
      }
      if (HAS4 && m < p.K4) {
        T D4[KA];
        Four<PA>::desc(B, d3, D4);
#pragma unroll
        for (int q = 0; q < KA; ++q)
          if (q < p.KA4) sDa[p.col4 + m * p.KA4 + q] = D4[q];
      }
    }
    __syncwarp();
    if constexpr (KT != MAXK) {
      // dE_i/dD = c + S D_i for the warp's atoms at once: lanes over columns,
      // each S element loaded once per warp and applied to every atom (the
      // descriptors are shared-memory broadcasts)
      constexpr int AW = 32 / KT;
      const T* sD0 = reinterpret_cast<const T*>(wb + lay.off_D);
      T* sCe = reinterpret_cast<T*>(wb + lay.off_D) + AW * lay.MS;
      for (int col0 = 0; col0 < p.M; col0 += 32) {
        const int col = col0 + lane;
        if (col < p.M) {
          T acc[AW];
#pragma unroll
          for (int a = 0; a < AW; ++a) acc[a] = T(0);
          const int M4 = p.M & ~3;
          for (int n = 0; n < M4; n += 4) {
            // S is symmetric: rows n..n+3 at column col, coalesced over lanes
            const T s0 = p.qbeta[(size_t)n * p.M + col], s1 = p.qbeta[(size_t)(n + 1) * p.M + col];
            const T s2 = p.qbeta[(size_t)(n + 2) * p.M + col], s3 = p.qbeta[(size_t)(n + 3) * p.M + col];
#pragma unroll
            for (int a = 0; a < AW; ++a) {
              const Q4<T> d = *reinterpret_cast<const Q4<T>*>(sD0 + a * lay.MS + n);
              acc[a] = fma(s0, d.x, fma(s1, d.y, fma(s2, d.z, fma(s3, d.w, acc[a]))));
            }
          }
          for (int n = M4; n < p.M; ++n) {
            const T sv = p.qbeta[(size_t)n * p.M + col];
#pragma unroll
            for (int a = 0; a < AW; ++a) acc[a] = fma(sv, sD0[a * lay.MS + n], acc[a]);
          }
          const T cc = sc[col];
#pragma unroll
          for (int a = 0; a < AW; ++a) sCe[a * lay.MS + col] = cc + acc[a];
        }
      }
      __syncwarp();
    }
  }

  // ---------------- embedding model (Sec. 3: EAM and MEAM written with POD
  // descriptors, a polynomial embedding of a density that is a linear
  // combination of descriptors): rho_i = a . D_i summed over the atom's lanes,
  // then F(rho_i) and F'(rho_i) by Horner's rule
  T emb_rho = T(0), emb_F = T(0), emb_Fp = T(0);
  if (MODE == 5) {
    T part = T(0);
    if (am) {
      const double* ea = p.emb_a;
      if (m == 0) part = (T)ea[0];  // one-body column, D_i0 = 1
      T d3[PA + 1];
      Mono<PA>::d3(B, d3);
      if (m < p.K2) part = fma((T)ea[1 + m], B[0], part);
#pragma unroll
      for (int n = 0; n <= PA; ++n)
        if (n <= p.P3 && m < p.K3) part = fma((T)ea[p.col3 + m * (p.P3 + 1) + n], d3[n], part);
      if (HAS4 && m < p.K4) {
        T D4[KA];
        Four<PA>::desc(B, d3, D4);
#pragma unroll
        for (int q = 0; q < KA; ++q)
          if (q < p.KA4) part = fma((T)ea[p.col4 + m * p.KA4 + q], D4[q], part);
      }
    }
    se[lane] = part;
    __syncwarp();
    if (am) {
      for (int mm = 0; mm < K; ++mm) emb_rho += se[a_loc * K + mm];
      emb_F = (T)p.emb_alpha[p.emb_deg];
      for (int k = p.emb_deg - 1; k >= 0; --k) {
        emb_Fp = fma(emb_Fp, emb_rho, emb_F);
        emb_F = fma(emb_F, emb_rho, (T)p.emb_alpha[k]);
      }
    }
    __syncwarp();
  }

  // ---------------- energy and adjoint a = dE_i/dB_m  (Eq. 26c generalised)
  T E = T(0);
  T s3 = T(0);  // exclusive three-body set: dE_i/dS3 of this lane's mode
  {
    T a[NAP];
#pragma unroll
    for (int x = 0; x < NAP; ++x) a[x] = T(0);
    if (am) {
      const T* c = sc;
      T c2 = (m < p.K2) ? c[1 + m] : T(0);
      T c0 = c[0];
      T h[PA + 1];
#pragma unroll
      for (int n = 0; n <= PA; ++n)
        h[n] = (n <= p.P3 && m < p.K3) ? c[p.col3 + m * (p.P3 + 1) + n] : T(0);
      T w4[KA];
#pragma unroll
      for (int q = 0; q < KA; ++q) w4[q] = (HAS4 && q < p.KA4 && m < p.K4) ? c[p.col4 + m * p.KA4 + q] : T(0);
      if (p.excl3) {
        // sum_n c_n (D3_n - S3) / 2: weights c_n / 2 on the inclusive D3_n and
        // -sum_n c_n / 2 on S3
#pragma unroll
        for (int n = 0; n <= PA; ++n) {
          s3 = fma(T(-0.5), h[n], s3);
          h[n] *= T(0.5);
        }
      }
      T Elin = T(0);  // quadratic model: the linear part c . D of this lane's columns
      if (MODE == 4) {
        const T* Da = reinterpret_cast<const T*>(wb + lay.off_D) + a_loc * lay.MS;
        auto ceff = [&](int col) {
          if constexpr (KT != MAXK) {  // formed above for the whole warp
            return reinterpret_cast<const T*>(wb + lay.off_D)[(32 / KT) * lay.MS + a_loc * lay.MS + col];
          } else {
            const T* row = p.qbeta + (size_t)col * p.M;
            T s = c[col];
            for (int n = 0; n < p.M; ++n) s = fma(row[n], Da[n], s);
            return s;
          }
        };
        if (m < p.K2) {
          Elin = fma(c2, Da[1 + m], Elin);
          c2 = ceff(1 + m);
        }
#pragma unroll
        for (int n = 0; n <= PA; ++n)
          if (n <= p.P3 && m < p.K3) {
            const int col = p.col3 + m * (p.P3 + 1) + n;
            Elin = fma(h[n], Da[col], Elin);
            h[n] = ceff(col);
          }
#pragma unroll
        for (int q = 0; q < KA; ++q)
          if (HAS4 && q < p.KA4 && m < p.K4) {
            const int col = p.col4 + m * p.KA4 + q;
            Elin = fma(w4[q], Da[col], Elin);
            w4[q] = ceff(col);
          }
        if (m == 0) {
          Elin += c0;
          c0 = ceff(0);
        }
      }
      if (MODE == 5) {  // dE_i/dD_col = c_col + F'(rho_i) a_col
        const double* ea = p.emb_a;
        if (m < p.K2) c2 = fma(emb_Fp, (T)ea[1 + m], c2);
#pragma unroll
        for (int n = 0; n <= PA; ++n)
          if (n <= p.P3 && m < p.K3) h[n] = fma(emb_Fp, (T)ea[p.col3 + m * (p.P3 + 1) + n], h[n]);
#pragma unroll
        for (int q = 0; q < KA; ++q)
          if (HAS4 && q < p.KA4 && m < p.K4) w4[q] = fma(emb_Fp, (T)ea[p.col4 + m * p.KA4 + q], w4[q]);
        if (m == 0) c0 = fma(emb_Fp, (T)ea[0], c0);
      }
      T d3[PA + 1];
      Mono<PA>::d3(B, d3);
      T a0 = c2;
      if (HAS4) {
        // general partitions (Eq. 30a): cubic form, E4 = (1/3) sum_x B_x dE4/dB_x
        Four<PA>::adjoint(B, w4, a);
        T E4 = T(0);
#pragma unroll
        for (int x = 0; x < NA; ++x) E4 = fma(a[x], B[x], E4);
        E = E4 * (T(1) / T(3));
        // b = c = 0 partitions (Eq. 27a): D4 = D2 * D3_n folds into the D3 weights
#pragma unroll
        for (int n = 0; n <= PA; ++n) {
          const T wn = w4[Four<PA>::p_n00(n)];
          a0 = fma(wn, d3[n], a0);
          h[n] = fma(wn, B[0], h[n]);
        }
      }
      E = fma(c2, B[0], E);
#pragma unroll
      for (int n = 0; n <= PA; ++n) E = fma(h[n], d3[n], E);
      Mono<PA>::d3_adjoint(B, h, a);
      a[0] += a0;
      if (m == 0) E += c0;
      E = fma(s3, S3, E);
      // quadratic model: E above is sum_col (dE/dD_col) D_col = c.D + 2 E_quad, so
      // E_i = (c.D + that) / 2
      if (MODE == 4) E = T(0.5) * (E + Elin);
      // embedding model: E above is (c + F' a) . D = c . D + F' rho, so
      // E_i = that - F' rho + F(rho)
      if (MODE == 5 && m == 0) E += emb_F - emb_Fp * emb_rho;
      T* adst = sadj + a_loc * lay.AS + m * NAP;
#pragma unroll
      for (int x = 0; x < NAP; ++x) adst[x] = a[x];
    }
  }
  se[lane] = E;
  __syncwarp();
  long long efix = 0;  // FP32 path: this lane's atom energy in fixed point
  if (am && m == 0) {
    T s = T(0);
    for (int mm = 0; mm < K; ++mm) s += se[lane + mm];
    p.Ei[atom0 + a_loc] = (double)s;
    if constexpr (FIXP) {
      if (fabsf(s) < EW_MAX_ATOM)
        efix = __float2ll_rn(s * EW_SCALE_F);
      else
        atomicOr(p.status, isfinite(s) ? ST_OVERFLOW : ST_NONFINITE);
    }
  }
  if constexpr (FIXP) {
    // the warp's energy (exact integer sum of its atoms' fixed-point values)
    // joins the fixed-point total: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) efix += __shfl_xor_sync(0xffffffffu, efix, o);
    if (lane == 0) ew_add(p.facc + 4 * (size_t)p.N + (gwarp % EW_COPIES) * EW_STRIDE, efix);
  }
  if (p.excl3) {  // dE_i/dS3 of every (atom, mode) for the pair pass
    __syncwarp();
    se[lane] = s3;
    __syncwarp();
  }
  if (MODE == 1 && p.adj_out) {
    // the adjoint pair pass runs as its own kernel: hand it dE_i/dB_m (and dE_i/dS3)
    if (am) {
      const int i = atom0 + a_loc;
      const Q4<T>* asrc = reinterpret_cast<const Q4<T>*>(sadj + a_loc * lay.AS + m * NAP);
      Q4<T>* adst = reinterpret_cast<Q4<T>*>(p.adj_out + ((size_t)i * K + m) * NAP);
#pragma unroll
      for (int x4 = 0; x4 < NAP / 4; ++x4) adst[x4] = asrc[x4];
      if (p.excl3) p.s3_out[(size_t)i * K + m] = s3;
    }
    return;
  }

  // ---------------- adjoint pair pass: g_ij = sum_{m,x} a_mx dB_mx/dr_ij  (Eq. 24c)
  T wv[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) wv[q] = T(0);
  for (int ch = 0; ch < nchunks; ++ch) {
    if (nchunks > 1) {
      __syncwarp();
      pair_pass<T, KT, false>(p, lay, geo, sR, sRp, scnt, atom0, A, K, ch, lane, nullptr, sj);
      __syncwarp();
    }
    int tot = 0;
    for (int a = 0; a < A; ++a) tot += chunk_count(scnt[a], ch);
    for (int f = lane; f < tot; f += 32) {
      int a = 0, base = 0;
      for (; a < A; ++a) {
        const int nca = chunk_count(scnt[a], ch);
        if (f < base + nca) break;
        base += nca;
      }
      const int jj = f - base, slot = ch * CH + jj, i = atom0 + a;
      const Q4<T> u = geo[a * lay.GA + jj];
      T Rv[KT], Rpv[KT];
      if (p.rad.tab && !p.keep_rp) {
        // tabulated basis: re-evaluate R, R' (or read them staged, keep_rp)
        if (u.w > p.rad.r_in && u.w < p.rmask) {
          radial_pair<T, KT>(p.rad, u.w, Rv, Rpv);
        } else {
#pragma unroll
          for (int k = 0; k < KT; ++k) { Rv[k] = T(0); Rpv[k] = T(0); }
        }
      } else {
        const T* Rrow = sR + a * lay.SA + jj * lay.KS;
        const T* Rprow = sRp + a * lay.SA + jj * lay.KS;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
          if (KT == MAXK && k >= K) break;
          Rv[k] = Rrow[k];
          Rpv[k] = Rprow[k];
        }
      }
      const Q4<T> out =
          pair_gradient<T, PA, KT>(u, Rv, Rpv, sadj + a * lay.AS, K, p.excl3 ? se + a * K : static_cast<T*>(nullptr));
      const size_t pidx = (size_t)i * p.cap + slot;
      if constexpr (std::is_same<T, float>::value) {
        // F_i += g_ij, F_j -= g_ij as fixed-point integers (order-independent sums)
        const int j = sj ? sj[a * lay.GA + jj] : p.nbr_j[pidx];
        if (!(fabsf(out.x) < FIX_GMAX && fabsf(out.y) < FIX_GMAX && fabsf(out.z) < FIX_GMAX)) {
          atomicOr(p.status, isfinite(out.x) && isfinite(out.y) && isfinite(out.z) ? ST_OVERFLOW : ST_NONFINITE);
        } else {
          const long long fx = __float2ll_rn(out.x * FIX_SCALE_F);
          const long long fy = __float2ll_rn(out.y * FIX_SCALE_F);
          const long long fz = __float2ll_rn(out.z * FIX_SCALE_F);
          atomicAdd(p.facc + 4 * (size_t)i + 0, (unsigned long long)fx);
          atomicAdd(p.facc + 4 * (size_t)i + 1, (unsigned long long)fy);
          atomicAdd(p.facc + 4 * (size_t)i + 2, (unsigned long long)fz);
          atomicAdd(p.facc + 4 * (size_t)j + 0, (unsigned long long)(-fx));
          atomicAdd(p.facc + 4 * (size_t)j + 1, (unsigned long long)(-fy));
          atomicAdd(p.facc + 4 * (size_t)j + 2, (unsigned long long)(-fz));
        }
      } else {
        p.g[pidx] = out;
      }
      // pair virial  W -= r_ij (x) g_ij
      const T dx = u.x * u.w, dy = u.y * u.w, dz = u.z * u.w;
      wv[0] -= dx * out.x; wv[1] -= dx * out.y; wv[2] -= dx * out.z;
      wv[3] -= dy * out.x; wv[4] -= dy * out.y; wv[5] -= dy * out.z;
      wv[6] -= dz * out.x; wv[7] -= dz * out.y; wv[8] -= dz * out.z;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 9; ++q) wv[q] += __shfl_xor_sync(0xffffffffu, wv[q], o);
  }
  if constexpr (FIXP) {
    // the warp's virial joins the fixed-point totals: one atomic per component
    if (lane < 9) {
      T w = wv[0];
#pragma unroll
      for (int q = 1; q < 9; ++q)
        if (lane == q) w = wv[q];
      long long v = 0;
      if (fabsf(w) < EW_MAX_WARP)
        v = __float2ll_rn(w * EW_SCALE_F);
      else
        atomicOr(p.status, isfinite(w) ? ST_OVERFLOW : ST_NONFINITE);
      ew_add(p.facc + 4 * (size_t)p.N + (gwarp % EW_COPIES) * EW_STRIDE + 2 * (1 + lane), v);
    }
  } else if (lane < 9) {
    T v = wv[0];
#pragma unroll
    for (int q = 1; q < 9; ++q)
      if (lane == q) v = wv[q];
    p.wpart[(size_t)gwarp * 9 + lane] = (double)v;
  }
}

// ------------------------------------------------------------------ layout
template <typename T>
AtomLayout make_layout(int K, int PA, bool table, bool tangent = false, int quadM = 0, bool pair_j = false,
                       bool design = false) {
  if (tangent) table = false;  // the tangent pass reads R' from shared memory
  AtomLayout L{};
  const int NA = (PA + 1) * (PA + 2) * (PA + 3) / 6;
  const int NAP = (NA + 3) / 4 * 4;
  L.A = 32 / K;
  L.KS = K | 1;
  L.SA = CH * L.KS + K;
  L.GA = CH + 1;
  int AS = (K * NAP + 3) / 4 * 4;
  if (((AS / 4) & 1) == 0) AS += 4;
  L.AS = AS;
  auto al = [](size_t v, size_t a) { return (v + a - 1) / a * a; };
  size_t off = 0;
  L.off_geo = off;
  off = al(off + sizeof(Q4<T>) * (size_t)L.A * L.GA, 32);
  L.off_R = off;
  off = al(off + sizeof(T) * (size_t)L.A * L.SA, 32);
  L.off_Rp = off;
  if (!table) off = al(off + sizeof(T) * (size_t)L.A * L.SA, 32);
  L.off_adj = off;
  off = al(off + sizeof(T) * (size_t)L.A * L.AS, 32);
  L.off_e = off;
  off = al(off + sizeof(T) * 32, 32);
  L.off_cnt = off;
  off = al(off + sizeof(int) * 32, 32);
  L.off_V = off;
  if (tangent) off = al(off + sizeof(Q4<T>) * (size_t)L.A * L.GA, 32);
  L.off_D = off;  // quadratic model: descriptors of the warp's atoms, then dE/dD
  L.MS = quadM > 0 ? (quadM + 3) / 4 * 4 : 0;  // rows of 16-byte multiples (float4 reads)
  off = al(off + 2 * sizeof(T) * (size_t)L.A * L.MS, 32);
  L.off_J = 0;
  if (pair_j) {  // neighbour index per staged pair (displacement lists)
    L.off_J = off;
    off = al(off + sizeof(int) * (size_t)L.A * L.GA, 32);
  }
  L.off_d3 = 0;
  if (design) {  // design mode: D3_n of every (atom, mode) of the warp
    L.off_d3 = off;
    off = al(off + sizeof(T) * (size_t)L.A * K * (PA + 1), 32);
  }
  L.warp_bytes = off;
  return L;
}

template <typename T, int PA, bool HAS4, int MODE, int KT>
static cudaError_t launch_one(const AtomArgs<T>& p, const AtomLayout& lay, cudaStream_t st) {
  auto kern = atom_kernel<T, PA, HAS4, MODE, KT>;
  const int wpb = p.wpb > 0 ? p.wpb : WPB_ATOM;
  if (wpb > ATOM_MAX_WPB) return cudaErrorInvalidValue;
  const size_t smem = (size_t)wpb * lay.warp_bytes;
  // raise the dynamic shared-memory limit once per instantiation, device and size
  // (not a stream operation, so it stays out of captured graphs after the first call)
  static size_t granted[64] = {};
  if (cudaError_t e = grant_smem((const void*)kern, smem, granted)) return e;
  const int atoms_per_block = wpb * lay.A;
  const int grid = (p.n_eval + atoms_per_block - 1) / atoms_per_block;
  if (grid > 0) kern<<<grid, wpb * 32, smem, st>>>(p, lay);
  return cudaGetLastError();
}

// Warps launched by the atom kernels for N atoms with K radial modes (one
// virial partial per warp).
inline int atom_warps_t(int N, int K, int wpb) {
  const int A = 32 / K;
  const int apb = wpb * A;
  return (N + apb - 1) / apb * wpb;
}

template <typename T, int MODE>
static cudaError_t dispatch_generic(const AtomArgs<T>& p, const AtomLayout& lay, int PA, bool has4,
                                    cudaStream_t st) {
  switch (PA * 2 + (has4 ? 1 : 0)) {
    case 0: return launch_one<T, 0, false, MODE, MAXK>(p, lay, st);
    case 1: return launch_one<T, 0, true, MODE, MAXK>(p, lay, st);
    case 2: return launch_one<T, 1, false, MODE, MAXK>(p, lay, st);
    case 3: return launch_one<T, 1, true, MODE, MAXK>(p, lay, st);
    case 4: return launch_one<T, 2, false, MODE, MAXK>(p, lay, st);
    case 5: return launch_one<T, 2, true, MODE, MAXK>(p, lay, st);
    case 6: return launch_one<T, 3, false, MODE, MAXK>(p, lay, st);
    case 7: return launch_one<T, 3, true, MODE, MAXK>(p, lay, st);
    case 8: return launch_one<T, 4, false, MODE, MAXK>(p, lay, st);
    case 9: return launch_one<T, 4, true, MODE, MAXK>(p, lay, st);
    default: return cudaErrorInvalidValue;
  }
}

// Embedding model (mode 5): its own entry so that it is compiled separately.
template <typename T>
cudaError_t launch_atom_emb_t(const AtomArgs<T>& p, int PA, bool has4, cudaStream_t st) {
  if (!p.emb_a || !p.emb_alpha || p.emb_deg < 1) return cudaErrorInvalidValue;
  const AtomLayout lay = make_layout<T>(p.K, PA, p.rad.tab != nullptr && !p.keep_rp, false, 0, p.pd != nullptr);
  if (p.K == 6 && PA == 4 && has4) return launch_one<T, 4, true, 5, 6>(p, lay, st);
  if (p.K == 3 && PA == 3 && !has4) return launch_one<T, 3, false, 5, 3>(p, lay, st);
  return dispatch_generic<T, 5>(p, lay, PA, has4, st);
}

// Specialised instantiations for the two workloads the library is tuned for
// (K = 3, P = 3, no 4-body; K = 6, P = 4, 4-body), generic K <= 16 otherwise.
template <typename T>
cudaError_t launch_atom_t(int mode, const AtomArgs<T>& p, int PA, bool has4, cudaStream_t st) {
  const AtomLayout lay = make_layout<T>(p.K, PA, p.rad.tab != nullptr && !p.keep_rp, mode == 2, mode == 4 ? p.M : 0,
                                        p.pd != nullptr, mode == 3);
  const bool spec6 = (p.K == 6 && PA == 4 && has4);
  const bool spec3 = (p.K == 3 && PA == 3 && !has4);
  if (mode == 2) {
    if (spec6) return launch_one<T, 4, true, 2, 6>(p, lay, st);
    if (spec3) return launch_one<T, 3, false, 2, 3>(p, lay, st);
    return dispatch_generic<T, 2>(p, lay, PA, has4, st);
  }
  if (mode == 0) {
    if (spec6) return launch_one<T, 4, true, 0, 6>(p, lay, st);
    if (spec3) return launch_one<T, 3, false, 0, 3>(p, lay, st);
    return dispatch_generic<T, 0>(p, lay, PA, has4, st);
  }
  if (mode == 3) {
    if (spec6) return launch_one<T, 4, true, 3, 6>(p, lay, st);
    if (spec3) return launch_one<T, 3, false, 3, 3>(p, lay, st);
    return dispatch_generic<T, 3>(p, lay, PA, has4, st);
  }
  if (mode == 4) {
    if (!p.qbeta) return cudaErrorInvalidValue;
    if (spec6) return launch_one<T, 4, true, 4, 6>(p, lay, st);
    if (spec3) return launch_one<T, 3, false, 4, 3>(p, lay, st);
    return dispatch_generic<T, 4>(p, lay, PA, has4, st);
  }
  if (spec6) return launch_one<T, 4, true, 1, 6>(p, lay, st);
  if (spec3) return launch_one<T, 3, false, 1, 3>(p, lay, st);
  return dispatch_generic<T, 1>(p, lay, PA, has4, st);
}

}  // namespace fastpod
