// Kernel argument blocks and launcher declarations (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <cmath>

#include "pod_common.cuh"

namespace fastpod {

// Shared-memory layout of one warp in the atom kernels (byte offsets).
// Raises a kernel's dynamic shared-memory limit when a launch needs more than the
// default 48 KB.  The attribute belongs to the current device, so the largest
// size granted is remembered per device (granted: [64]); it is not a stream
// operation.
inline cudaError_t grant_smem(const void* kern, size_t smem, size_t* granted) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && smem <= granted[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) granted[dev] = smem;
  return e;
}

// Launch shape of the step's kernels (warps per block; gather blocks per SM).
struct LaunchShape {
  int atom_wpb = WPB_ATOM;
  int neigh_wpb = WPB_NEIGH;
  int gather_wpb = 16;
  int gather_bps = 3;
  int atom_rp = 0;  // table path: stage R' in shared memory in the pair pass (else re-evaluate it)
  int atom_split = -1;  // mixed linear path: 1 adjoint pair pass as its own kernel, 0 fused, -1 by size
  int neigh_blockwide = -1;  // block-per-cell search: 1 block-wide candidate tests, 0 a warp per atom, -1 by size
  int design_wpb = 8;        // fit: warps per block of the force-row gather
};

struct AtomLayout {
  int A;    // atoms per warp
  int KS;   // row stride of the staged R / R' (odd, >= K)
  int SA;   // per-atom stride of R / R' (CH * KS + K: lanes (atom, m) hit distinct banks)
  int GA;   // per-atom stride of the staged (u, r), in Q4 units
  int AS;   // per-atom stride of the adjoint dE/dB (multiple of 4, odd number of 16-byte units)
  size_t off_geo, off_R, off_Rp, off_adj, off_e, off_cnt, off_V, off_D, off_J, warp_bytes;
  size_t off_d3;   // design mode: D3_n per (atom, mode) of the warp
  int MS;   // per-atom stride of the staged descriptors (quadratic model)
};

template <typename T>
struct AtomArgs {
  int N, cap;
  int n_eval;           // atoms [0, n_eval) are evaluated; the rest only appear as neighbours (ghosts)
  int wpb;              // warps per block of the launch (0: default)
  int keep_rp;          // table path: R' staged in shared memory for the adjoint pass
  const int* nbr_count;
  const int* nbr_j;
  const int* nbr_s;
  const float4* pd;     // FP32 path (optional): per-slot displacement x_j + s L - x_i, j in .w (N * cap)
  const double* wpos;   // wrapped positions [3][N] (FP64 path)
  const float4* phi;    // FP32 hi part of the wrapped positions (mixed path)
  const float4* plo;    // FP32 lo part
  double L[3];
  float Lh[3], Ll[3];
  int K, K2, K3, K4, P3, P4, KA4, M, col3, col4;
  double* D;            // mode 0: descriptors [N][M]
  const double* c;      // modes 1, 4: coefficients [M]
  const T* qbeta;       // mode 4: symmetric quadratic weights S [M][M], S_mn = beta_mn + beta_nm
  const double* emb_a;      // mode 5: density weights a [M] (rho_i = a . D_i)
  const double* emb_alpha;  // mode 5: embedding polynomial F(rho) = sum_k alpha_k rho^k, [emb_deg + 1]
  int emb_deg;
  int excl3;            // modes 0, 1: three-body columns as the exclusive sums of Eq. 15b
  double* Ei;           // mode 1: atom energies [N]
  Q4<T>* g;             // mode 1, FP64 path: dE_i/dr_ij per pair slot [N * cap]
  unsigned long long* facc;  // mode 1, FP32 path: fixed-point force accumulators [N][4]
  T* adj_out;           // mode 1 (optional): stop after the adjoint, writing dE_i/dB [N][K][NAP] here
  T* s3_out;            //   and dE_i/dS3 [N][K] (exclusive three-body set); the pair pass then runs
                        //   as launch_pair_adjoint_f32
  double* wpart;        // mode 1: per-warp virial partials [warps][9]
  const double* vdir;   // mode 2: displacement direction per atom [3][N] (tangent of D written to D)
  T* gdm;               // mode 3: design-matrix pair gradients [q - q0][N * cap][K][3]
  int q0, q1;           // mode 3: range of per-mode descriptor indices q (0: 2-body, 1..P3+1: 3-body, then 4-body)
  T rmask;              // pairs with r >= rmask contribute nothing (lists built with a skin; +inf: none)
  const int* cfg_of;    // batch: configuration of each atom (NULL: one configuration, box L)
  const CfgBox* cbox;   // batch: per-configuration boxes
  int* status;
  RadialConst<T> rad;
};

// Mask radius in the pair arithmetic's type: the smallest T >= r (so that, for
// every T value x, x < result exactly when x < r), or +inf when r <= 0 (no mask).
template <typename T>
inline T mask_radius(double r) {
  if (!(r > 0)) return (T)INFINITY;
  T v = (T)r;
  if ((double)v < r) v = std::nextafter(v, (T)INFINITY);
  return v;
}

cudaError_t launch_bin(int N, const double* pos, const CellGrid& cg, double* wpos, float4* phi, float4* plo,
                       int* cell_count, float4* cell_pos, int* status, cudaStream_t st, int* wrapk = nullptr,
                       unsigned long long* facc = nullptr, int* nbr_count = nullptr, const double* csrc = nullptr,
                       double* cdst = nullptr, int cn = 0);
cudaError_t launch_rewrap(int N, const double* pos, const int* wrapk, const double L[3], double* wpos, float4* phi,
                          float4* plo, int* status, cudaStream_t st, unsigned long long* facc = nullptr);
cudaError_t launch_kick(int N3, double* v, const double* F, double half_dt_over_m, double* x, double dt,
                        cudaStream_t st);
// Neighbour search over the binned atoms.  pad: fill each row with a sentinel up
// to cap (needed by the reverse-slot search); pd (optional): also write each
// slot's FP32 displacement with j in .w -- *wrote_pd says whether the kernel
// that ran did (the block-per-cell search does, the general search does not).
// Block-per-cell neighbour search, candidate tests when no shape says otherwise:
// block-wide (all threads over candidates x own atoms) for small systems, a warp
// per own atom for large ones (measured crossover between 8,192 and 1,024,000 atoms).
inline bool neigh_blockwide_default(int N) { return N <= 131072; }

cudaError_t launch_neigh(int N, const CellGrid& cg, const double* wpos, const float4* phi, const float4* plo,
                         const int* cell_count, const float4* cell_pos, double rcut, int cap, int* nbr_count,
                         int* nbr_j, int* nbr_s, int* status, cudaStream_t st, int wpb = WPB_NEIGH,
                         float4* pd = nullptr, bool pad = true, bool* wrote_pd = nullptr, bool blockwide = true);
cudaError_t launch_rev(int N, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s, int* rev,
                       int* status, cudaStream_t st);
cudaError_t launch_export_neighbors(int N, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s,
                                    int cap_out, int* count_out, int* j_out, int* s_out, cudaStream_t st);

cudaError_t launch_batch_wrap(int N, const double* pos, const int* cfg_of, const CfgBox* cbox, double* wpos,
                              float4* phi, float4* plo, int* status, cudaStream_t st,
                              unsigned long long* facc = nullptr);
cudaError_t launch_batch_neigh(int N, const int* cfg_of, const CfgBox* cbox, const double* wpos, const float4* phi,
                               double rcut, double Lmax, int Smax, int cap, int* nbr_count, int* nbr_j, int* nbr_s,
                               int* status, cudaStream_t st);
cudaError_t launch_segsum(int n_cfg, const CfgBox* cbox, const double* v, double w, int per_atom, double* out,
                          cudaStream_t st);

cudaError_t launch_atom_f32(int mode, const AtomArgs<float>& p, int PA, bool has4, cudaStream_t st);
cudaError_t launch_atom_f64(int mode, const AtomArgs<double>& p, int PA, bool has4, cudaStream_t st);
// Adjoint pair pass of the linear FP32 path as its own kernel (warp per atom, lane
// per pair), after launch_atom_f32 in mode 1 with adj_out set: g_ij from dE_i/dB,
// fixed-point forces, energy-free virial totals.
cudaError_t launch_pair_adjoint_f32(const AtomArgs<float>& p, int PA, bool has4, cudaStream_t st);
// Embedding model (energy mode 5), compiled in translation units of their own.
cudaError_t launch_atom_emb_f32(const AtomArgs<float>& p, int PA, bool has4, cudaStream_t st);
cudaError_t launch_atom_emb_f64(const AtomArgs<double>& p, int PA, bool has4, cudaStream_t st);

template <typename T>
cudaError_t launch_gather_reduce(int N, int n_eval, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s,
                                 const int* rev_in, int* rev_out, const Q4<T>* g, const double* Ei,
                                 const double* wpart, int n_wpart, double* F, double fscale, double* part,
                                 int nblocks, unsigned* ticket, double* E, double* W, int* status, cudaStream_t st,
                                 int wpb);
int atom_warps(int N, int K, int wpb);
cudaError_t launch_colsum(int n_chunks, const int* chunk_rows /*[n_chunks][2]*/, int n_cfg, const int* cfg_chunks,
                          int M, const double* D, double* part, double* G, cudaStream_t st);
// Tall-skinny Householder QR of the fit's design matrix (qr.cu): shared memory of
// one panel (M + 1 columns of M + cmax rows); the row stage (one factor per block
// from rows of A and b), the merge stage (g factors into one per block) and the
// final stage (c_out set: one block absorbs every factor and sqrt(gamma) I, then
// back substitution; info = k + 1 for a zero pivot R_kk, else 0).
size_t tsqr_smem_bytes(int M, int cmax);
cudaError_t launch_tsqr_rows(int M, long long R, const double* AT, const double* b, int nblocks,
                             long long rows_per_block, int cmax, double* out, cudaStream_t st);
cudaError_t launch_tsqr_merge(int M, int nin, int g, const double* in, int cmax, double sqrt_gamma, double* out,
                              double* c_out, int* info, cudaStream_t st);
int gather_blocks(int N, int wpb, int bps);
int finalize_blocks(int N);
cudaError_t launch_finalize(int N, const unsigned long long* facc, double* F, double fscale, int nblocks, double* E,
                            double* W, cudaStream_t st, int* cell_count = nullptr, int ncells = 0,
                            int* status = nullptr, int* status_out = nullptr);

}  // namespace fastpod
