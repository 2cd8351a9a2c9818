// Ridge least-squares fit of the linear POD model (Eq. 63a):
//   min || A c - b ||^2 + gamma || c ||^2
// A has one row per configuration energy, w_E G_m / N_c (G_m = sum_i D_im,
// Eq. 58a), and one row per force component, -w_F dG_m / dr_ka; b holds
// w_E E_ref / N_c and w_F F_ref.
//
// Column m of A is assembled with the energy/force kernels themselves: with the
// coefficient vector e_m the atom energies are E_i = D_im, their per-configuration
// sum is G_m, and the "forces" are -dG_m/dr, so the adjoint pair pass and the
// coalesced gather write column m directly (A is stored column-major, AT[m][row]).
// The normal equations (A^T A + gamma I) c = A^T b are formed in FP64 by a
// blocked SYRK with a fixed-order reduction of per-block partials, then solved
// by Cholesky on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pod_internal.h"

namespace fastpod {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_RT = 32;   // rows of A staged per step
constexpr int GRAM_MP = 128;  // maximum (padded) number of descriptors handled by the Gram kernel

// Block b accumulates rows [b * chunk, (b + 1) * chunk) of A: 4 x 4 tiles of the
// upper triangle of A^T A per thread, plus A^T b.  part[b] = (G (Mp x Mp), r (Mp)).
__global__ void __launch_bounds__(GRAM_THREADS)
    gram_partial_kernel(int M, int Mp, long long R, const double* __restrict__ AT, const double* __restrict__ bvec,
                        long long chunk, double* __restrict__ part) {
  extern __shared__ double gsm[];
  double* S = gsm;                       // [Mp][GRAM_RT]
  double* bs = gsm + (size_t)Mp * GRAM_RT; // [GRAM_RT]
  const int tid = threadIdx.x;
  const int nb = Mp / 4;
  const int ntile = nb * (nb + 1) / 2;
  const long long r0 = (long long)blockIdx.x * chunk;
  const long long r1 = min(R, r0 + chunk);
  constexpr int TPT = 3;  // tiles per thread: (32 * 33 / 2) / 256 rounded up
  double acc[TPT][16];
  int ta[TPT], tb[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = tid + u * GRAM_THREADS;
    int a = 0, rem = t;
    while (a < nb && rem >= nb - a) {
      rem -= nb - a;
      ++a;
    }
    ta[u] = (t < ntile) ? a : -1;
    tb[u] = (t < ntile) ? a + rem : -1;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[u][q] = 0.0;
  }
  double racc = 0.0;
  for (long long rs = r0; rs < r1; rs += GRAM_RT) {
    const int nr = (int)min((long long)GRAM_RT, r1 - rs);
    for (int e = tid; e < Mp * GRAM_RT; e += GRAM_THREADS) {
      const int a = e / GRAM_RT, rr = e - a * GRAM_RT;
      S[e] = (a < M && rr < nr) ? AT[(size_t)a * R + rs + rr] : 0.0;
    }
    if (tid < GRAM_RT) bs[tid] = tid < nr ? bvec[rs + tid] : 0.0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (ta[u] < 0) continue;
      const double* Sa = S + (size_t)(4 * ta[u]) * GRAM_RT;
      const double* Sb = S + (size_t)(4 * tb[u]) * GRAM_RT;
      for (int rr = 0; rr < GRAM_RT; ++rr) {
        double xa[4], xb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xa[q] = Sa[q * GRAM_RT + rr];
          xb[q] = Sb[q * GRAM_RT + rr];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][p * 4 + q] = fma(xa[p], xb[q], acc[u][p * 4 + q]);
      }
    }
    if (tid < Mp) {
      for (int rr = 0; rr < GRAM_RT; ++rr) racc = fma(S[(size_t)tid * GRAM_RT + rr], bs[rr], racc);
    }
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.x * ((size_t)Mp * Mp + Mp);
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    if (ta[u] < 0) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) out[(size_t)(4 * ta[u] + p) * Mp + 4 * tb[u] + q] = acc[u][p * 4 + q];
  }
  if (tid < Mp) out[(size_t)Mp * Mp + tid] = racc;
}

// G[a][b] (a <= b, mirrored) and r[a]: sum of the block partials in block order.
__global__ void gram_reduce_kernel(int M, int Mp, int nblk, const double* __restrict__ part, double gamma,
                                   double* __restrict__ G, double* __restrict__ r) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = M * M + M;
  if (e >= n) return;
  const size_t stride = (size_t)Mp * Mp + Mp;
  if (e < M * M) {
    const int a = e / M, b = e - a * M;
    const int lo = min(a, b), hi = max(a, b);
    // tile (lo / 4, hi / 4) holds entry (lo, hi) when lo / 4 <= hi / 4, which always holds
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k * stride + (size_t)lo * Mp + hi];
    if (a == b) s += gamma;
    G[e] = s;
  } else {
    const int a = e - M * M;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k * stride + (size_t)Mp * Mp + a];
    r[a] = s;
  }
}

// In-place Cholesky G = L L^T (lower triangle) and the two triangular solves,
// one block, fixed order.  info = 0 on success, k + 1 if pivot k is not positive.
__global__ void cholesky_solve_kernel(int M, double* __restrict__ G, double* __restrict__ r, double* __restrict__ c,
                                      int* __restrict__ info) {
  __shared__ double piv;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      const double d = G[(size_t)k * M + k];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = k + 1;
        piv = 1.0;
      } else {
        piv = sqrt(d);
      }
      G[(size_t)k * M + k] = piv;
    }
    __syncthreads();
    if (bad) break;
    for (int i = k + 1 + tid; i < M; i += blockDim.x) G[(size_t)i * M + k] /= piv;
    __syncthreads();
    const int m = M - k - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) G[(size_t)i * M + j] -= G[(size_t)i * M + k] * G[(size_t)j * M + k];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) *info = bad;
    return;
  }
  // L y = r (y overwrites r)
  for (int k = 0; k < M; ++k) {
    if (tid == 0) r[k] /= G[(size_t)k * M + k];
    __syncthreads();
    for (int i = k + 1 + tid; i < M; i += blockDim.x) r[i] -= G[(size_t)i * M + k] * r[k];
    __syncthreads();
  }
  // L^T c = y
  for (int k = M - 1; k >= 0; --k) {
    if (tid == 0) c[k] = r[k] / G[(size_t)k * M + k];
    __syncthreads();
    for (int i = tid; i < k; i += blockDim.x) r[i] -= G[(size_t)k * M + i] * c[k];
    __syncthreads();
  }
  if (tid == 0) *info = 0;
}

// Residuals of the fitted model: per block, sum |A c - b| over energy rows
// (row < n_e) and over force rows.  out[blk] = (sum_e, sum_f).
__global__ void residual_kernel(int M, long long R, long long n_e, const double* __restrict__ AT,
                                const double* __restrict__ bvec, const double* __restrict__ c,
                                double* __restrict__ out) {
  __shared__ double se[256], sf[256];
  double e_acc = 0.0, f_acc = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (long long)gridDim.x * blockDim.x) {
    double p = 0.0;
    for (int a = 0; a < M; ++a) p = fma(AT[(size_t)a * R + r], c[a], p);
    const double d = fabs(p - bvec[r]);
    if (r < n_e) e_acc += d; else f_acc += d;
  }
  se[threadIdx.x] = e_acc;
  sf[threadIdx.x] = f_acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      se[threadIdx.x] += se[threadIdx.x + k];
      sf[threadIdx.x] += sf[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = se[0];
    out[2 * blockIdx.x + 1] = sf[0];
  }
}

// b: energy rows w_E E_ref[c] (/ N_c), force rows w_F F_ref (SoA [3][N]).
__global__ void fit_rhs_kernel(int n_cfg, int N, const CfgBox* __restrict__ cbox, const double* __restrict__ E_ref,
                               const double* __restrict__ F_ref, double wE, double wF, int per_atom,
                               double* __restrict__ b) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_cfg) {
    const int n = cbox[e].a1 - cbox[e].a0;
    b[e] = wE * E_ref[e] / (per_atom ? (double)n : 1.0);
  } else if (e < n_cfg + 3LL * N) {
    b[e] = wF * F_ref[e - n_cfg];
  }
}

}  // namespace fastpod

using namespace fastpod;

// Stage 1: neighbour lists of the batch, design matrix A (column-major) and b.
int pod_handle::fit_build(const pod_system* bsys, const double* E_ref, const double* F_ref, const pod_fit_opts& o) {
  int rc_ = validate_system(bsys);
  if (rc_) return rc_;
  if (!E_ref || !F_ref) return fail(POD_EINVAL, "E_ref and F_ref are required");
  if (!(o.w_E >= 0) || !(o.w_F >= 0) || !(o.gamma_reg >= 0)) return fail(POD_EINVAL, "weights and gamma must be >= 0");
  const int Mp = (M + 3) / 4 * 4;
  if (Mp > GRAM_MP) return fail(POD_EINVAL, "the fit supports at most %d descriptors", GRAM_MP);
  pod_system sys = *bsys;  // a single configuration is a batch of one
  int offs1[2] = {0, bsys->n_atoms};
  if (sys.n_configs <= 1) {
    sys.n_configs = 1;
    sys.atom_offs = offs1;
    sys.boxes = bsys->box;
    sys.pbcs = nullptr;
  }
  cudaStream_t st = nullptr;
  const int N = sys.n_atoms;
  const int keep_sync = this->sync;
  this->sync = 1;
  Plan pl;
  retries = 0;
  for (;;) {
    if ((rc_ = plan_batch(&sys, pl))) break;
    if ((rc_ = build_neighbors(sys.pos, pl, true, st))) break;
    bool retry;
    if ((rc_ = finish(st, pl, retry))) break;
    if (!retry) break;
  }
  this->sync = keep_sync;
  if (rc_) return rc_;
  const int nc = pl.n_cfg;
  const long long R = (long long)nc + 3LL * N;
  const size_t gbytes = (precision == POD_MIXED ? sizeof(Q4<float>) : sizeof(Q4<double>)) * (size_t)N * pl.cap;
  if ((rc_ = ensure(g, gbytes, "pair gradients"))) return rc_;
  const int nwarp = atom_warps(N, K, pl.shape.atom_wpb);
  if ((rc_ = ensure(wpart, sizeof(double) * 9 * (size_t)nwarp, "virial partials"))) return rc_;
  if ((rc_ = ensure(Ei, sizeof(double) * (size_t)N, "atom energies"))) return rc_;
  const int nblk = gather_blocks(N, pl.shape.gather_wpb, pl.shape.gather_bps);
  if ((rc_ = ensure(Wat, sizeof(double) * 10 * (size_t)nblk, "block partial sums"))) return rc_;
  if (!offs.p) {
    if ((rc_ = ensure(offs, sizeof(unsigned) * 4, "ticket"))) return rc_;
    cudaError_t e0 = cudaMemset(offs.p, 0, sizeof(unsigned) * 4);
    if (e0 != cudaSuccess) return cuda_fail(e0, "ticket init");
  }
  if ((rc_ = ensure(fitA, sizeof(double) * (size_t)M * R, "design matrix"))) return rc_;
  if ((rc_ = ensure(fitb, sizeof(double) * (size_t)R, "right-hand side"))) return rc_;
  const size_t work_bytes = sizeof(double) * ((size_t)M * M + (size_t)M * M + 4 * (size_t)M + 2 * 1024 + 8) + 64;
  if ((rc_ = ensure(fitwork, work_bytes, "fit workspace"))) return rc_;
  std::vector<double> eye((size_t)M * M, 0.0);
  for (int m = 0; m < M; ++m) eye[(size_t)m * M + m] = 1.0;
  double* dI = (double*)fitwork.p;
  double* dtot = dI + (size_t)M * M * 2 + 2 * (size_t)M + 2 * 1024;
  cudaError_t e = cudaMemcpy(dI, eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "identity upload");
  double* AT = (double*)fitA.p;
  double* bvec = (double*)fitb.p;
  const int* rev_in = (const int*)rev.p;  // the batch's reverse index, built once above
  for (int m = 0; m < M; ++m) {
    if ((rc_ = run_atoms(1, pl, nullptr, dI + (size_t)m * M, (double*)Ei.p, st))) return rc_;
    double* col = AT + (size_t)m * R;
    if (precision == POD_MIXED)
      e = launch_gather_reduce<float>(N, pl.cap, (const int*)nbr_count.p, (const int*)nbr_j.p, (const int*)nbr_s.p,
                                      rev_in, nullptr, (const Q4<float>*)g.p, (const double*)Ei.p,
                                      (const double*)wpart.p, nwarp, col + nc, o.w_F, (double*)Wat.p, nblk,
                                      (unsigned*)offs.p, dtot, nullptr, (int*)status.p, st, pl.shape.gather_wpb);
    else
      e = launch_gather_reduce<double>(N, pl.cap, (const int*)nbr_count.p, (const int*)nbr_j.p,
                                       (const int*)nbr_s.p, rev_in, nullptr, (const Q4<double>*)g.p,
                                       (const double*)Ei.p, (const double*)wpart.p, nwarp, col + nc, o.w_F,
                                       (double*)Wat.p, nblk, (unsigned*)offs.p, dtot, nullptr, (int*)status.p, st,
                                       pl.shape.gather_wpb);
    if (e != cudaSuccess) return cuda_fail(e, "design-matrix force rows");
    e = launch_segsum(nc, (const CfgBox*)boxes.p, (const double*)Ei.p, o.w_E, o.per_atom_energy, col, st);
    if (e != cudaSuccess) return cuda_fail(e, "design-matrix energy rows");
  }
  const int tb = 256;
  fit_rhs_kernel<<<(unsigned)((R + tb - 1) / tb), tb, 0, st>>>(nc, N, (const CfgBox*)boxes.p, E_ref, F_ref, o.w_E,
                                                               o.w_F, o.per_atom_energy, bvec);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "rhs kernel");
  fit_R = R;
  fit_nc = nc;
  fit_N = N;
  fit_wE = o.w_E;
  fit_wF = o.w_F;
  return POD_OK;
}

// Stage 2: G = A^T A + gamma I and r = A^T b on the device (fitwork).
int pod_handle::fit_gram(double gamma) {
  const int Mp = (M + 3) / 4 * 4;
  const long long R = fit_R;
  const size_t gram_blocks = (size_t)std::max<long long>(1, std::min<long long>(2 * 152, (R + 4095) / 4096));
  const size_t part_bytes = sizeof(double) * gram_blocks * ((size_t)Mp * Mp + Mp);
  int rc_;
  if ((rc_ = ensure(fitG, part_bytes, "Gram partials"))) return rc_;
  double* dG = (double*)fitwork.p + (size_t)M * M;
  double* dr = dG + (size_t)M * M;
  const long long chunk = (R + (long long)gram_blocks - 1) / (long long)gram_blocks;
  const size_t gsmem = sizeof(double) * ((size_t)Mp * GRAM_RT + GRAM_RT);
  cudaError_t e;
  if (gsmem > 48 * 1024) {
    e = cudaFuncSetAttribute(gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
    if (e != cudaSuccess) return cuda_fail(e, "gram smem");
  }
  gram_partial_kernel<<<(unsigned)gram_blocks, GRAM_THREADS, gsmem, nullptr>>>(
      M, Mp, R, (const double*)fitA.p, (const double*)fitb.p, chunk, (double*)fitG.p);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gram kernel");
  gram_reduce_kernel<<<(M * M + M + 255) / 256, 256, 0, nullptr>>>(M, Mp, (int)gram_blocks, (const double*)fitG.p,
                                                                  gamma, dG, dr);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gram reduce");
  return POD_OK;
}

// Stage 3: Cholesky solve of the device G, r into the device c.
int pod_handle::fit_solve_dev() {
  double* dG = (double*)fitwork.p + (size_t)M * M;
  double* dr = dG + (size_t)M * M;
  double* dc = dr + M;
  int* dinfo = (int*)(dc + M + 2 * 1024 + 8);
  cholesky_solve_kernel<<<1, 256, 0, nullptr>>>(M, dG, dr, dc, dinfo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cholesky kernel");
  int info = 0;
  e = cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cholesky status");
  if (info) return fail(POD_ESINGULAR, "normal equations are not positive definite (pivot %d)", info - 1);
  return POD_OK;
}

// Stage 4: sums of |A c - b| over the energy rows and the force rows (unweighted back by w).
int pod_handle::fit_residual_dev(double* sumE, double* sumF) {
  double* dc = (double*)fitwork.p + 2 * (size_t)M * M + M;
  double* dres = dc + M;
  const int rblocks = 1024;
  residual_kernel<<<rblocks, 256, 0, nullptr>>>(M, fit_R, fit_nc, (const double*)fitA.p, (const double*)fitb.p, dc,
                                                dres);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "residual kernel");
  std::vector<double> res(2 * rblocks);
  e = cudaMemcpy(res.data(), dres, sizeof(double) * res.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "residual read");
  double se = 0.0, sf = 0.0;
  for (int b = 0; b < rblocks; ++b) {
    se += res[2 * b];
    sf += res[2 * b + 1];
  }
  *sumE = fit_wE > 0 ? se / fit_wE : 0.0;
  *sumF = fit_wF > 0 ? sf / fit_wF : 0.0;
  return POD_OK;
}

int pod_handle::fit(const pod_system* bsys, const double* E_ref, const double* F_ref, const pod_fit_opts* opts,
                    double* c_out, double* mae_E, double* mae_F) {
  if (!c_out) return fail(POD_EINVAL, "c_out is required");
  pod_fit_opts o{100.0, 1.0, 1e-12, 1};
  if (opts) o = *opts;
  int rc_;
  if ((rc_ = fit_build(bsys, E_ref, F_ref, o))) return rc_;
  if ((rc_ = fit_gram(o.gamma_reg))) return rc_;
  if ((rc_ = fit_solve_dev())) return rc_;
  double se = 0, sf = 0;
  if ((rc_ = fit_residual_dev(&se, &sf))) return rc_;
  double* dc = (double*)fitwork.p + 2 * (size_t)M * M + M;
  cudaError_t e = cudaMemcpy(c_out, dc, sizeof(double) * M, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "coefficients read");
  if ((rc_ = read_status(nullptr))) return rc_;
  if (mae_E) *mae_E = se / fit_nc;
  if (mae_F) *mae_F = fit_N > 0 ? sf / (3.0 * fit_N) : 0.0;
  return POD_OK;
}

extern "C" {

int pod_fit(pod_handle* h, const pod_system* batch, const double* E_ref, const double* F_ref,
            const pod_fit_opts* opts, double* c_out, double* mae_E, double* mae_F) {
  if (!h) return POD_EINVAL;
  return h->fit(batch, E_ref, F_ref, opts, c_out, mae_E, mae_F);
}

int pod_fit_normal(pod_handle* h, const pod_system* batch, const double* E_ref, const double* F_ref,
                   const pod_fit_opts* opts, double* G_out, double* r_out) {
  if (!h) return POD_EINVAL;
  if (!G_out || !r_out) return h->fail(POD_EINVAL, "G_out and r_out are required");
  pod_fit_opts o{100.0, 1.0, 1e-12, 1};
  if (opts) o = *opts;
  int rc;
  if ((rc = h->fit_build(batch, E_ref, F_ref, o))) return rc;
  if ((rc = h->fit_gram(o.gamma_reg))) return rc;
  const int M = h->M;
  double* dG = (double*)h->fitwork.p + (size_t)M * M;
  cudaError_t e = cudaMemcpy(G_out, dG, sizeof(double) * M * M, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(r_out, dG + (size_t)M * M, sizeof(double) * M, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "normal equations read");
  return h->read_status(nullptr);
}

int pod_fit_solve(pod_handle* h, const double* G, const double* r, double* c_out) {
  if (!h) return POD_EINVAL;
  if (!G || !r || !c_out) return h->fail(POD_EINVAL, "G, r and c_out are required");
  const int M = h->M;
  const size_t work_bytes = sizeof(double) * ((size_t)M * M + (size_t)M * M + 4 * (size_t)M + 2 * 1024 + 8) + 64;
  int rc;
  if ((rc = h->ensure(h->fitwork, work_bytes, "fit workspace"))) return rc;
  double* dG = (double*)h->fitwork.p + (size_t)M * M;
  cudaError_t e = cudaMemcpy(dG, G, sizeof(double) * M * M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dG + (size_t)M * M, r, sizeof(double) * M, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return h->cuda_fail(e, "normal equations upload");
  if ((rc = h->fit_solve_dev())) return rc;
  e = cudaMemcpy(c_out, dG + (size_t)M * M + M, sizeof(double) * M, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return h->cuda_fail(e, "coefficients read");
  return POD_OK;
}

int pod_fit_residual(pod_handle* h, const double* c, double* sum_abs_E, double* sum_abs_F, int* n_E, int* n_F) {
  if (!h) return POD_EINVAL;
  if (!c || !sum_abs_E || !sum_abs_F) return h->fail(POD_EINVAL, "c and the sums are required");
  if (h->fit_R == 0) return h->fail(POD_EINVAL, "pod_fit_residual needs a design matrix from pod_fit_normal");
  const int M = h->M;
  double* dc = (double*)h->fitwork.p + 2 * (size_t)M * M + M;
  cudaError_t e = cudaMemcpy(dc, c, sizeof(double) * M, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return h->cuda_fail(e, "coefficients upload");
  int rc;
  if ((rc = h->fit_residual_dev(sum_abs_E, sum_abs_F))) return rc;
  if (n_E) *n_E = h->fit_nc;
  if (n_F) *n_F = 3 * h->fit_N;
  return POD_OK;
}

}  // extern "C"
