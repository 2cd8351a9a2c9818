// Adjoint pair pass of the linear mixed-precision path as a kernel of its own:
// g_ij = sum_{m,x} a_mx dB_mx/dr_ij (Eq. 24c) for every pair, from the per-atom
// adjoint a = dE_i/dB (Eq. 26c generalised) that the atom kernel wrote in its
// forward-only form.  One warp per atom, one lane per pair: the atom's K rows of
// a are staged once in shared memory and read as broadcasts, so a warp holds
// few registers and many warps fit on an SM -- the latency of the pass is hidden
// by occupancy instead of being one long chain inside the fused kernel.  The
// per-pair arithmetic is the fused kernel's own (pair_unit, radial_pair,
// pair_gradient), so forces are the same bits either way.
#include "atom_impl.cuh"

namespace fastpod {

constexpr int ADJ_WPB = 4;

template <int PA, int KT>
__global__ void __launch_bounds__(ADJ_WPB * 32) pair_adjoint_kernel(const AtomArgs<float> p) {
  constexpr int NA = Mono<PA>::NA;
  constexpr int NAP = (NA + 3) / 4 * 4;
  extern __shared__ __align__(16) float asm_[];
  const int K = (KT == MAXK) ? p.K : KT;
  const int row = K * NAP;
  const int wstride = (row + K + 3) / 4 * 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * ADJ_WPB + warp;
  const int i = gwarp;
  float wv[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) wv[q] = 0.f;
  if (i < p.n_eval) {
    float* sa = asm_ + (size_t)warp * wstride;
    const float4* src = reinterpret_cast<const float4*>(p.adj_out + (size_t)i * row);
    for (int t = lane; t < row / 4; t += 32) reinterpret_cast<float4*>(sa)[t] = __ldg(src + t);
    const float* s3m = nullptr;
    if (p.excl3) {
      if (lane < K) sa[row + lane] = p.s3_out[(size_t)i * K + lane];
      s3m = sa + row;
    }
    __syncwarp();
    const int n = min(p.nbr_count[i], p.cap);
    for (int slot = lane; slot < n; slot += 32) {
      const size_t pidx = (size_t)i * p.cap + slot;
      float dx, dy, dz;
      int j;
      if (p.pd) {
        const float4 q = __ldg(p.pd + pidx);
        dx = q.x;
        dy = q.y;
        dz = q.z;
        j = __float_as_int(q.w);
      } else {
        j = p.nbr_j[pidx];
        int sx, sy, sz;
        shift_unpack(p.nbr_s[pidx], sx, sy, sz);
        pair_disp<float>(p, i, j, sx, sy, sz, dx, dy, dz);
      }
      const Q4<float> u = pair_unit(dx, dy, dz);
      float Rv[KT], Rpv[KT];
      if (u.w > p.rad.r_in && u.w < p.rmask) {
        radial_pair<float, KT>(p.rad, u.w, Rv, Rpv);
      } else {
#pragma unroll
        for (int k = 0; k < KT; ++k) { Rv[k] = 0.f; Rpv[k] = 0.f; }
      }
      const Q4<float> out = pair_gradient<float, PA, KT>(u, Rv, Rpv, sa, K, s3m);
      // F_i += g_ij, F_j -= g_ij as fixed-point integers (order-independent sums)
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
      // pair virial  W -= r_ij (x) g_ij
      const float rx = u.x * u.w, ry = u.y * u.w, rz = u.z * u.w;
      wv[0] -= rx * out.x; wv[1] -= rx * out.y; wv[2] -= rx * out.z;
      wv[3] -= ry * out.x; wv[4] -= ry * out.y; wv[5] -= ry * out.z;
      wv[6] -= rz * out.x; wv[7] -= rz * out.y; wv[8] -= rz * out.z;
    }
  }
  if (gwarp >= p.n_eval) return;  // uniform per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 9; ++q) wv[q] += __shfl_xor_sync(0xffffffffu, wv[q], o);
  }
  // the warp's virial joins the fixed-point totals: one atomic per component
  if (lane < 9) {
    float w = wv[0];
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
}

template <int PA, int KT>
static cudaError_t launch_adj(const AtomArgs<float>& p, cudaStream_t st) {
  constexpr int NAP = (Mono<PA>::NA + 3) / 4 * 4;
  const int K = (KT == MAXK) ? p.K : KT;
  const size_t smem = sizeof(float) * (size_t)ADJ_WPB * ((K * NAP + K + 3) / 4 * 4);
  const int grid = (p.n_eval + ADJ_WPB - 1) / ADJ_WPB;
  if (grid > 0) pair_adjoint_kernel<PA, KT><<<grid, ADJ_WPB * 32, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pair_adjoint_f32(const AtomArgs<float>& p, int PA, bool has4, cudaStream_t st) {
  if (!p.adj_out || (p.excl3 && !p.s3_out) || !p.facc) return cudaErrorInvalidValue;
  if (p.K == 6 && PA == 4 && has4) return launch_adj<4, 6>(p, st);
  if (p.K == 3 && PA == 3 && !has4) return launch_adj<3, 3>(p, st);
  switch (PA) {
    case 0: return launch_adj<0, MAXK>(p, st);
    case 1: return launch_adj<1, MAXK>(p, st);
    case 2: return launch_adj<2, MAXK>(p, st);
    case 3: return launch_adj<3, MAXK>(p, st);
    case 4: return launch_adj<4, MAXK>(p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fastpod
