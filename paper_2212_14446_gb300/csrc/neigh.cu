// Cell-list neighbour builder: full list of every atom within r_cut, with
// periodic images, sorted by (j, s_x, s_y, s_z); plus the reverse-pair index used
// by the deterministic force gather.
#include "pod_common.cuh"
#include "pod_kernels.h"

namespace fastpod {

// One thread per atom: wrap into [0, L) (x - L floor(x / L), each operation
// rounded separately), split into FP32 hi + lo, bin into a cell: the cell slot
// holds the FP32 hi position and the atom index (in .w), so the search reads a
// candidate with one load; phi[i].w holds the atom's own cell index.
// A coordinate already in [0, L) has floor(x / L) = 0 exactly (the rounded
// quotient of x < L by L stays below 1), so the FP64 division, slow on this
// part, only runs for atoms outside the box.
__global__ void bin_kernel(int N, const double* __restrict__ pos, CellGrid cg, double* __restrict__ wpos,
                           float4* __restrict__ phi, float4* __restrict__ plo, int* __restrict__ cell_count,
                           float4* __restrict__ cell_pos, int* __restrict__ wrapk, int* __restrict__ status,
                           unsigned long long* __restrict__ facc, int* __restrict__ nbr_count,
                           const double* __restrict__ csrc, double* __restrict__ cdst, int cn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // an optional copy of cn values (the coefficients of a host-buffer call, read
  // through the pinned buffer's device address) rides on this launch
  for (int q = i; q < cn; q += gridDim.x * blockDim.x) cdst[q] = csrc[q];
  if (i >= N) return;
  if (facc) {  // fixed-point force, energy and virial accumulators of this call start at zero
    ulonglong2* fz = reinterpret_cast<ulonglong2*>(facc + 4 * (size_t)i);
    fz[0] = make_ulonglong2(0ull, 0ull);
    fz[1] = make_ulonglong2(0ull, 0ull);
    ulonglong2* tz = reinterpret_cast<ulonglong2*>(facc + 4 * (size_t)N);
    for (int q = i; q < FACC_TAIL / 2; q += N) tz[q] = make_ulonglong2(0ull, 0ull);
  }
  double x[3];
  int c[3];
  bool finite = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = pos[(size_t)d * N + i];
    finite = finite && isfinite(v);
    double k = 0.0;
    if (cg.pbc[d] && !(v >= 0.0 && v < cg.L[d])) {
      k = floor(__ddiv_rn(v, cg.L[d]));
      v = __dsub_rn(v, __dmul_rn(cg.L[d], k));
    }
    if (wrapk) wrapk[(size_t)d * N + i] = finite ? (int)k : 0;
    x[d] = v;
    int ci = (int)floor(v * cg.inv_cs[d]);
    ci = ci < 0 ? 0 : (ci >= cg.nc[d] ? cg.nc[d] - 1 : ci);
    c[d] = finite ? ci : 0;
    wpos[(size_t)d * N + i] = v;
  }
  if (!finite) atomicOr(status, ST_NONFINITE);
  float h[3], l[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    h[d] = __double2float_rn(x[d]);
    l[d] = __double2float_rn(x[d] - (double)h[d]);
  }
  const int cell = (c[2] * cg.nc[1] + c[1]) * cg.nc[0] + c[0];
  phi[i] = make_float4(h[0], h[1], h[2], __int_as_float(cell));
  plo[i] = make_float4(l[0], l[1], l[2], 0.f);
  const int slot = atomicAdd(&cell_count[cell], 1);
  if (slot < cg.cap) {
    cell_pos[(size_t)cell * cg.cap + slot] = make_float4(h[0], h[1], h[2], __int_as_float(i));
  } else {
    // a full cell: the call is reported and retried with larger cells; the
    // block-per-cell search never sees this atom, so give it an empty row now
    atomicOr(status, ST_CELL);
    if (nbr_count) nbr_count[i] = 0;
  }
}

constexpr int NEIGH_PREFETCH = 4;
constexpr unsigned long long BAND_MARK = 1ull << 62;

// Finish atom i's row from the warp's candidate keys (nhit of them, at most
// keycap stored): decide the band candidates exactly in FP64 (R6) and drop the
// misses, sort the keys (j, s) ascending, write the row padded with a sentinel,
// and the count (a count above cap raises ST_NEIGH).
__device__ __forceinline__ void neigh_finish_row(int N, const CellGrid& cg, const double* __restrict__ wpos,
                                                 double rc2, int cap, int keycap, int i, int lane, int nhit,
                                                 unsigned long long* keys, int* __restrict__ nbr_count,
                                                 int* __restrict__ nbr_j, int* __restrict__ nbr_s,
                                                 int* __restrict__ status) {
  __syncwarp();
  int n = min(nhit, keycap);
  int dropped_all = 0;  // band keys dropped among the n kept
  // decide the band candidates exactly in FP64 (R6): drop the misses
  {
    const double xi0 = wpos[i], xi1 = wpos[(size_t)N + i], xi2 = wpos[(size_t)2 * N + i];
    int dropped = 0;
    for (int t = lane; t < n; t += 32) {
      unsigned long long key = keys[t];
      bool drop = false;
      if (key & BAND_MARK) {
        key &= ~BAND_MARK;
        const int j = (int)(key >> 24);
        int sx, sy, sz;
        shift_unpack((int)(key & 0xFFFFFFull), sx, sy, sz);
        const double ddx = disp_fp64(xi0, wpos[j], sx, cg.L[0]);
        const double ddy = disp_fp64(xi1, wpos[(size_t)N + j], sy, cg.L[1]);
        const double ddz = disp_fp64(xi2, wpos[(size_t)2 * N + j], sz, cg.L[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
        drop = !(r2 < rc2);
        keys[t] = drop ? ~0ull : key;
      }
      dropped += drop ? 1 : 0;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) dropped += __shfl_xor_sync(0xffffffffu, dropped, d);
    dropped_all = dropped;
    // an overflowed key buffer lost candidates: keep the preliminary count (> cap)
    // so the call reports it and retries with a larger capacity
    if (nhit <= keycap) nhit -= dropped;
    __syncwarp();
  }
  if (n <= 32) {
    // bitonic sort of one key per lane in registers (dropped keys sort last)
    unsigned long long v = lane < n ? keys[lane] : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0;
        const bool lower = (lane & j) == 0;
        v = (lower == up) ? (v < w ? v : w) : (v < w ? w : v);
      }
    if (lane < n) keys[lane] = v;
    __syncwarp();
  } else {
    int np = 1;
    while (np < n) np <<= 1;
    for (int t = n + lane; t < np; t += 32) keys[t] = ~0ull;
    __syncwarp();
    for (int k = 2; k <= np; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < np; t += 32) {
          const int u = t ^ j;
          if (u > t) {
            const unsigned long long a = keys[t], b = keys[u];
            const bool up = (t & k) == 0;
            if ((a > b) == up) { keys[t] = b; keys[u] = a; }
          }
        }
        __syncwarp();
      }
  }
  // The valid keys lead the sorted array.  The kernels that read the list take
  // min(count, cap) slots, so every one of them must hold a valid pair: after an
  // overflow (count above cap, the call is retried) slots past the valid keys
  // repeat the last valid one (or, with none, the atom itself: r = 0, reported).
  const int nvalid = n - dropped_all;
  const int nfill = min(nhit, cap);
  const unsigned long long fill_key =
      nvalid > 0 ? keys[nvalid - 1] : (((unsigned long long)i << 24) | (unsigned long long)shift_pack(0, 0, 0));
  for (int t = lane; t < cap; t += 32) {
    if (t < nfill) {
      const unsigned long long key = t < nvalid ? keys[t] : fill_key;
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

// Warp per atom.  Candidates of the (2S+1)^3 neighbouring cells are tested in
// FP32 on the hi parts; those inside r_cut^2 - band are hits, those within the
// thin band around r_cut^2 are kept with a mark and decided afterwards by the
// exact FP64 expression, so the list equals the FP64 definition bit for bit
// while the scan loop holds no FP64 state.  Hits are sorted by key (j, s) with a
// bitonic sort (registers for <= 32 keys, else shared memory).

__global__ void __launch_bounds__(NEIGH_MAX_WPB * 32)
    neigh_kernel(int N, CellGrid cg, const double* __restrict__ wpos, const float4* __restrict__ phi,
                 const float4* __restrict__ plo, const int* __restrict__ cell_count,
                 const float4* __restrict__ cell_pos, double rc2, float rc2_lo, float rc2_hi, int cap,
                 int keycap, int* __restrict__ nbr_count, int* __restrict__ nbr_j, int* __restrict__ nbr_s,
                 int* __restrict__ status) {
  extern __shared__ unsigned long long nsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* keys = nsm + (size_t)warp * keycap;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= N) return;

  const float4 hi_i = phi[i];
  const int own = __float_as_int(hi_i.w);  // the atom's cell, from the bin kernel
  const int ci[3] = {own % cg.nc[0], (own / cg.nc[0]) % cg.nc[1], own / (cg.nc[0] * cg.nc[1])};
  const int wx = 2 * cg.S[0] + 1, wy = 2 * cg.S[1] + 1, wz = 2 * cg.S[2] + 1;
  const int noff = wx * wy * wz;
  const bool s1 = cg.S[0] == 1 && cg.S[1] == 1 && cg.S[2] == 1;
  const int zero = shift_pack(0, 0, 0);
  int nhit = 0;
  for (int ob = 0; ob < noff; ob += 32) {
    // lane -> one (cell, image) of this batch; every lane then walks its own cell
    const int o = ob + lane;
    int cnt = 0, cell = 0, code = zero;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (o < noff) {
      int oc[3];
      if (s1) {  // one cell of search depth: constant divisors
        oc[0] = o % 3 - 1;
        oc[1] = (o / 3) % 3 - 1;
        oc[2] = o / 9 - 1;
      } else {
        oc[0] = o % wx - cg.S[0];
        oc[1] = (o / wx) % wy - cg.S[1];
        oc[2] = o / (wx * wy) - cg.S[2];
      }
      int tc[3], sh[3];
      bool ok = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int t = ci[d] + oc[d];
        int sd = 0;
        if (cg.pbc[d]) {
          if (s1)  // |offset| <= 1 <= nc: at most one box length to wrap
            sd = t < 0 ? -1 : (t >= cg.nc[d] ? 1 : 0);
          else
            sd = (t >= 0) ? t / cg.nc[d] : -((-t + cg.nc[d] - 1) / cg.nc[d]);
          t -= sd * cg.nc[d];
        } else if (t < 0 || t >= cg.nc[d]) {
          ok = false;
        }
        tc[d] = t;
        sh[d] = sd;
      }
      if (ok) {
        cell = (tc[2] * cg.nc[1] + tc[1]) * cg.nc[0] + tc[0];
        cnt = min(cell_count[cell], cg.cap);
        code = shift_pack(sh[0], sh[1], sh[2]);
        px = (float)sh[0] * cg.Lf[0] - hi_i.x;
        py = (float)sh[1] * cg.Lf[1] - hi_i.y;
        pz = (float)sh[2] * cg.Lf[2] - hi_i.z;
      }
    }
    int cmax = cnt;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, d));
    const float4* cp = cell_pos + (size_t)cell * cg.cap;
    for (int k0 = 0; k0 < cmax; k0 += NEIGH_PREFETCH) {
      float4 q[NEIGH_PREFETCH];
#pragma unroll
      for (int u = 0; u < NEIGH_PREFETCH; ++u)
        q[u] = (k0 + u < cnt) ? cp[k0 + u] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
#pragma unroll
      for (int u = 0; u < NEIGH_PREFETCH; ++u) {
        const int j = __float_as_int(q[u].w);
        bool hit = false;
        unsigned long long key = 0;
        if (j >= 0 && !(j == i && code == zero)) {
          // FP32 prefilter on the hi parts only; its error is far inside the band
          const float dx = q[u].x + px, dy = q[u].y + py, dz = q[u].z + pz;
          const float r2f = dx * dx + dy * dy + dz * dz;
          hit = r2f < rc2_hi;
          key = ((unsigned long long)j << 24) | (unsigned long long)code | (r2f < rc2_lo ? 0ull : BAND_MARK);
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int pos = nhit + __popc(m & ((1u << lane) - 1u));
          if (pos < keycap) keys[pos] = key;
        }
        nhit += __popc(m);
      }
    }
  }
  neigh_finish_row(N, cg, wpos, rc2, cap, keycap, i, lane, nhit, keys, nbr_count, nbr_j, nbr_s, status);
}

// Block per cell, for a search depth of one cell in every direction (image
// shifts in {-1, 0, 1}).  The candidates of the 27 neighbouring (cell, image)
// pairs are staged once in shared memory as image-shifted FP32 positions with
// their image id (one coalesced copy per neighbouring cell).  Every thread of the
// block then takes candidates and tests each against all of the cell's own
// atoms (the candidate stays in registers, the own atoms are shared-memory
// broadcasts), appending hits to the own atom's key list; afterwards a warp per
// own atom decides its band keys, sorts them and writes its row.  Keys are
// 32-bit, (j << 5) | image id with id = 9 (s_x + 1) + 3 (s_y + 1) + (s_z + 1),
// so their order is the list order (j, s_x, s_y, s_z); bit 31 marks a band
// candidate until the exact FP64 decision (R6) keeps or drops it.  The order in
// which hits are appended does not matter: each row is sorted.  The row is
// written as (j, packed shift), padded with a sentinel up to cap when the
// reverse-slot search will read it (pad), and, when pd is given, as the pair
// displacement x_j + s L - x_i in FP32 from the double-float split of both
// positions (the arithmetic of the atom kernels, so the same bits) with j in the
// fourth word.  Requires N < 2^26.  Atoms that did not fit in their cell are
// given an empty row by the bin kernel (and the call is retried).
constexpr unsigned KEY_BAND = 0x80000000u;

template <bool BLOCKWIDE>
__global__ void __launch_bounds__(NEIGH_MAX_WPB * 32)
    neigh_cell_kernel(int N, CellGrid cg, const double* __restrict__ wpos, const float4* __restrict__ phi,
                      const float4* __restrict__ plo, const int* __restrict__ cell_count,
                      const float4* __restrict__ cell_pos, double rc2, float rc2_lo, float rc2_hi, int cap,
                      int keycap, int pad, int* __restrict__ nbr_count, int* __restrict__ nbr_j,
                      int* __restrict__ nbr_s, float4* __restrict__ pd, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ int soff[28], scell[27], sid[27];
  __shared__ float spx[27], spy[27], spz[27];
  const int ccap = 27 * cg.cap;
  float4* cand = reinterpret_cast<float4*>(csm);
  unsigned char* cid = reinterpret_cast<unsigned char*>(cand + ccap);
  int* ncnt = reinterpret_cast<int*>(csm + (sizeof(float4) * (size_t)ccap + (size_t)ccap + 15) / 16 * 16);
  unsigned* kbuf = reinterpret_cast<unsigned*>(ncnt + (cg.cap + 3) / 4 * 4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int cell = blockIdx.x;
  if (warp == 0) {
    const int ci[3] = {cell % cg.nc[0], (cell / cg.nc[0]) % cg.nc[1], cell / (cg.nc[0] * cg.nc[1])};
    int cnt = 0, tcell = 0, id = 13;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (lane < 27) {
      const int oc[3] = {lane / 9 - 1, (lane / 3) % 3 - 1, lane % 3 - 1};
      int tc[3], sh[3];
      bool ok = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int t = ci[d] + oc[d];
        int sd = 0;
        if (cg.pbc[d]) {
          sd = t < 0 ? -1 : (t >= cg.nc[d] ? 1 : 0);
          t -= sd * cg.nc[d];
        } else if (t < 0 || t >= cg.nc[d]) {
          ok = false;
        }
        tc[d] = t;
        sh[d] = sd;
      }
      if (ok) {
        tcell = (tc[2] * cg.nc[1] + tc[1]) * cg.nc[0] + tc[0];
        cnt = min(cell_count[tcell], cg.cap);
        px = (float)sh[0] * cg.Lf[0];
        py = (float)sh[1] * cg.Lf[1];
        pz = (float)sh[2] * cg.Lf[2];
        id = (sh[0] + 1) * 9 + (sh[1] + 1) * 3 + (sh[2] + 1);  // the image shift decides the key
      }
    }
    int x = cnt;  // inclusive prefix sum over the stencil entries
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < 27) {
      soff[lane] = x - cnt;
      scell[lane] = tcell;
      sid[lane] = id;
      spx[lane] = px;
      spy[lane] = py;
      spz[lane] = pz;
    }
    if (lane == 26) soff[27] = x;
  }
  __syncthreads();
  const int ncand = soff[27];
  // the cell's own atoms are the centre stencil entry (offset 0, image 0: id 13)
  const int own0 = soff[13], own_n = soff[14] - soff[13];
  auto entry_of = [&](int f) {
    int lo = 0, hi = 27;  // soff[lo] <= f < soff[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (soff[mid] <= f)
        lo = mid;
      else
        hi = mid;
    }
    return lo;
  };
  // copy the candidates with all threads, two per thread per round (both loads
  // in flight before either is stored)
  for (int f0 = threadIdx.x; f0 < ncand; f0 += 2 * blockDim.x) {
    const int f1 = f0 + blockDim.x;
    const int e0 = entry_of(f0), e1 = f1 < ncand ? entry_of(f1) : 0;
    const float4 q0 = cell_pos[(size_t)scell[e0] * cg.cap + (f0 - soff[e0])];
    float4 q1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (f1 < ncand) q1 = cell_pos[(size_t)scell[e1] * cg.cap + (f1 - soff[e1])];
    cand[f0] = make_float4(q0.x + spx[e0], q0.y + spy[e0], q0.z + spz[e0], q0.w);
    cid[f0] = (unsigned char)sid[e0];
    if (f1 < ncand) {
      cand[f1] = make_float4(q1.x + spx[e1], q1.y + spy[e1], q1.z + spz[e1], q1.w);
      cid[f1] = (unsigned char)sid[e1];
    }
  }
  const unsigned below = (1u << lane) - 1u;
  if (BLOCKWIDE) {
    for (int a = threadIdx.x; a < own_n; a += blockDim.x) ncnt[a] = 0;
    __syncthreads();
    // every candidate against every own atom; hits appended to the atom's keys
    for (int f = threadIdx.x; f < ncand; f += blockDim.x) {
      const float4 q = cand[f];
      const int j = __float_as_int(q.w);
      const unsigned kj = ((unsigned)j << 5) | (unsigned)cid[f];
      const bool self_img = cid[f] == 13;
      for (int a = 0; a < own_n; ++a) {
        const float4 qi = cand[own0 + a];
        const float dx = q.x - qi.x, dy = q.y - qi.y, dz = q.z - qi.z;
        const float r2f = dx * dx + dy * dy + dz * dz;
        if (r2f < rc2_hi && !(self_img && j == __float_as_int(qi.w))) {
          const int pos = atomicAdd(&ncnt[a], 1);
          if (pos < keycap) kbuf[(size_t)a * keycap + pos] = kj | (r2f < rc2_lo ? 0u : KEY_BAND);
        }
      }
    }
    __syncthreads();
  } else {
    __syncthreads();
  }
  // (the box's low part comes with the grid: formed per thread in FP64 it had
  // occupied the slow FP64 pipe of every block)
  const float* Ll = cg.Ll;
  for (int a = warp; a < own_n; a += nwarps) {
    const int i = __float_as_int(cand[own0 + a].w);
    // BLOCKWIDE: the atom's own key list; else this warp's list, filled here by
    // the warp testing every candidate with lanes over candidates
    unsigned* keys = BLOCKWIDE ? kbuf + (size_t)a * keycap : kbuf + (size_t)warp * keycap;
    int nhit = 0;
    if (BLOCKWIDE) {
      nhit = ncnt[a];
    } else {
      const float4 qi = cand[own0 + a];
      auto test = [&](int f, unsigned& key) {  // FP32 test of candidate f (band keys marked)
        bool hit = false;
        key = 0;
        if (f < ncand) {
          const float4 q = cand[f];
          const int j = __float_as_int(q.w);
          const int id = cid[f];
          if (!(j == i && id == 13)) {
            const float dx = q.x - qi.x, dy = q.y - qi.y, dz = q.z - qi.z;
            const float r2f = dx * dx + dy * dy + dz * dz;
            hit = r2f < rc2_hi;
            key = ((unsigned)j << 5) | (unsigned)id | (r2f < rc2_lo ? 0u : KEY_BAND);
          }
        }
        return hit;
      };
      for (int f0 = 0; f0 < ncand; f0 += 64) {  // two rounds of 32 candidates per iteration
        unsigned key0, key1;
        const bool hit0 = test(f0 + lane, key0);
        const bool hit1 = test(f0 + 32 + lane, key1);
        const unsigned m0 = __ballot_sync(0xffffffffu, hit0);
        const unsigned m1 = __ballot_sync(0xffffffffu, hit1);
        if (hit0) {
          const int pos = nhit + __popc(m0 & below);
          if (pos < keycap) keys[pos] = key0;
        }
        if (hit1) {
          const int pos = nhit + __popc(m0) + __popc(m1 & below);
          if (pos < keycap) keys[pos] = key1;
        }
        nhit += __popc(m0) + __popc(m1);
      }
      __syncwarp();
    }
    const int n = min(nhit, keycap);
    int dropped_all = 0;  // band keys dropped among the n kept
    unsigned anyband = 0;
    for (int t = lane; t < n; t += 32) anyband |= keys[t] & KEY_BAND;
    if (__any_sync(0xffffffffu, anyband != 0)) {
      // decide the band candidates exactly in FP64 (R6): drop the misses
      const double xi0 = wpos[i], xi1 = wpos[(size_t)N + i], xi2 = wpos[(size_t)2 * N + i];
      int dropped = 0;
      for (int t = lane; t < n; t += 32) {
        unsigned key = keys[t];
        if (key & KEY_BAND) {
          key &= ~KEY_BAND;
          const int j = (int)(key >> 5), id = (int)(key & 31u);
          const int sx = id / 9 - 1, sy = (id / 3) % 3 - 1, sz = id % 3 - 1;
          const double ddx = disp_fp64(xi0, wpos[j], sx, cg.L[0]);
          const double ddy = disp_fp64(xi1, wpos[(size_t)N + j], sy, cg.L[1]);
          const double ddz = disp_fp64(xi2, wpos[(size_t)2 * N + j], sz, cg.L[2]);
          const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
          const bool drop = !(r2 < rc2);
          keys[t] = drop ? 0xffffffffu : key;
          dropped += drop ? 1 : 0;
        }
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) dropped += __shfl_xor_sync(0xffffffffu, dropped, d);
      dropped_all = dropped;
      // an overflowed key buffer lost candidates: keep the preliminary count (> cap)
      // so the call reports it and retries with a larger capacity
      if (nhit <= keycap) nhit -= dropped;
      __syncwarp();
    }
    if (n <= 32) {
      // bitonic sort of one key per lane in registers (dropped keys sort last)
      unsigned v = lane < n ? keys[lane] : 0xffffffffu;
#pragma unroll
      for (int kk = 2; kk <= 32; kk <<= 1)
#pragma unroll
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
          const unsigned w = __shfl_xor_sync(0xffffffffu, v, jj);
          const bool up = (lane & kk) == 0;
          const bool lower = (lane & jj) == 0;
          v = (lower == up) ? min(v, w) : max(v, w);
        }
      __syncwarp();
      if (lane < n) keys[lane] = v;
      __syncwarp();
    } else {
      int np = 1;
      while (np < n) np <<= 1;
      for (int t = n + lane; t < np; t += 32) keys[t] = 0xffffffffu;
      __syncwarp();
      for (int kk = 2; kk <= np; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
          for (int t = lane; t < np; t += 32) {
            const int u = t ^ jj;
            if (u > t) {
              const unsigned x = keys[t], y = keys[u];
              const bool up = (t & kk) == 0;
              if ((x > y) == up) { keys[t] = y; keys[u] = x; }
            }
          }
          __syncwarp();
        }
    }
    // The valid keys lead the sorted array.  The kernels that read the list take
    // min(count, cap) slots, so every one of them must hold a valid pair: after
    // an overflow (count above cap, the call is retried) slots past the valid
    // keys repeat the last valid one (or, with none, the atom itself: r = 0,
    // reported).
    const int nvalid = n - dropped_all;
    const int nw = min(nhit, cap);
    const unsigned fill_key = nvalid > 0 ? keys[nvalid - 1] : (((unsigned)i << 5) | 13u);
    float4 hi_i = make_float4(0.f, 0.f, 0.f, 0.f), lo_i = hi_i;
    if (pd) {
      hi_i = phi[i];
      lo_i = plo[i];
    }
    const int tend = pad ? cap : nw;
    for (int t = lane; t < tend; t += 32) {
      if (t < nw) {
        const unsigned key = t < nvalid ? keys[t] : fill_key;
        const int j = (int)(key >> 5), id = (int)(key & 31u);
        const int sx = id / 9 - 1, sy = (id / 3) % 3 - 1, sz = id % 3 - 1;
        if (!pd || pad) {  // with displacement rows only (and no padding) the index rows are not read
          nbr_j[(size_t)i * cap + t] = j;
          nbr_s[(size_t)i * cap + t] = shift_pack(sx, sy, sz);
        }
        if (pd) {
          const float4 hj = phi[j], lj = plo[j];
          const float dx = disp_f32(hi_i.x, lo_i.x, hj.x, lj.x, sx, cg.Lf[0], Ll[0]);
          const float dy = disp_f32(hi_i.y, lo_i.y, hj.y, lj.y, sy, cg.Lf[1], Ll[1]);
          const float dz = disp_f32(hi_i.z, lo_i.z, hj.z, lj.z, sz, cg.Lf[2], Ll[2]);
          pd[(size_t)i * cap + t] = make_float4(dx, dy, dz, __int_as_float(j));
        }
      } else {
        nbr_j[(size_t)i * cap + t] = 0x7fffffff;  // sentinel: rows stay sorted to cap
      }
    }
    if (lane == 0) {
      nbr_count[i] = nhit;
      if (nhit > cap) atomicOr(status, ST_NEIGH);
    }
    __syncwarp();
  }
}

// Thread per pair slot: index of the reverse pair (j, i, -s) in j's list.  Rows
// are sorted and padded with a sentinel to cap, so a lower bound on the atom
// index over the whole row needs no count; equal indices (several images of
// the same atom) are then scanned for the negated shift.
__global__ void rev_kernel(int N, int cap, const int* __restrict__ nbr_count, const int* __restrict__ nbr_j,
                           const int* __restrict__ nbr_s, int* __restrict__ rev, int* __restrict__ status) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (size_t)N * cap) return;
  const int j = nbr_j[p];
  if (j >= N) return;  // sentinel slot
  // a 32-bit division where the slot index fits (a 64-bit one runs on the FP64 pipe)
  const int i = p < 0x80000000ull ? (int)((unsigned)p / (unsigned)cap) : (int)(p / cap);
  const int q = find_reverse(nbr_j, nbr_s, cap, i, j, nbr_s[p]);
  if (q < 0) atomicOr(status, ST_REV);
  rev[p] = q;  // -1: the gather skips it (and the status reports the broken list)
}

// Copy the internal list into the caller's [N][cap_out] / [N][cap_out][3] layout.
__global__ void export_neighbors_kernel(int N, int cap, const int* __restrict__ nbr_count,
                                        const int* __restrict__ nbr_j, const int* __restrict__ nbr_s, int cap_out,
                                        int* __restrict__ count_out, int* __restrict__ j_out,
                                        int* __restrict__ s_out) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (size_t)N * cap_out) return;
  const int i = p < 0x80000000ull ? (int)((unsigned)p / (unsigned)cap_out) : (int)(p / cap_out);
  const int t = (int)(p - (size_t)i * cap_out);
  const int n = nbr_count[i];
  if (t == 0) count_out[i] = n;
  if (t >= min(n, cap)) return;
  const int code = nbr_s[(size_t)i * cap + t];
  int sx, sy, sz;
  shift_unpack(code, sx, sy, sz);
  j_out[p] = nbr_j[(size_t)i * cap + t];
  s_out[3 * p] = sx;
  s_out[3 * p + 1] = sy;
  s_out[3 * p + 2] = sz;
}

// ------------------------------------------------------------ launchers
cudaError_t launch_bin(int N, const double* pos, const CellGrid& cg, double* wpos, float4* phi, float4* plo,
                       int* cell_count, float4* cell_pos, int* status, cudaStream_t st, int* wrapk,
                       unsigned long long* facc, int* nbr_count, const double* csrc, double* cdst, int cn) {
  const int tb = 64;  // small blocks spread the FP64 work of small systems over all SMs
  bin_kernel<<<(N + tb - 1) / tb, tb, 0, st>>>(N, pos, cg, wpos, phi, plo, cell_count, cell_pos, wrapk, status,
                                               facc, nbr_count, csrc, cdst, cn);
  return cudaGetLastError();
}

// Between rebuilds of a list built with a skin: positions are shifted by the
// box multiples frozen at the last build (x - k L, the same rounding as the
// wrap), so an atom that crossed the box edge keeps its images consistent with
// the stored shifts.
__global__ void rewrap_kernel(int N, const double* __restrict__ pos, const int* __restrict__ wrapk, double L0, double L1,
                              double L2, double* __restrict__ wpos, float4* __restrict__ phi,
                              float4* __restrict__ plo, int* __restrict__ status,
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
  const double L[3] = {L0, L1, L2};
  double x[3];
  bool finite = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = pos[(size_t)d * N + i];
    finite = finite && isfinite(v);
    const int k = wrapk[(size_t)d * N + i];
    if (k != 0) v = __dsub_rn(v, __dmul_rn(L[d], (double)k));
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

cudaError_t launch_rewrap(int N, const double* pos, const int* wrapk, const double L[3], double* wpos, float4* phi,
                          float4* plo, int* status, cudaStream_t st, unsigned long long* facc) {
  const int tb = 256;
  rewrap_kernel<<<(N + tb - 1) / tb, tb, 0, st>>>(N, pos, wrapk, L[0], L[1], L[2], wpos, phi, plo, status, facc);
  return cudaGetLastError();
}

// Velocity Verlet halves: v += a dt / 2 with a = F conv / m, then optionally
// x += v dt (kick_drift), all FP64.
__global__ void kick_kernel(int N3, double* __restrict__ v, const double* __restrict__ F, double half_dt_over_m,
                            double* __restrict__ x, double dt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N3) return;
  const double vn = fma(F[e], half_dt_over_m, v[e]);
  v[e] = vn;
  if (x) x[e] = fma(vn, dt, x[e]);
}

cudaError_t launch_kick(int N3, double* v, const double* F, double half_dt_over_m, double* x, double dt,
                        cudaStream_t st) {
  const int tb = 256;
  kick_kernel<<<(N3 + tb - 1) / tb, tb, 0, st>>>(N3, v, F, half_dt_over_m, x, dt);
  return cudaGetLastError();
}

static size_t neigh_smem_bytes(int keycap, int wpb) { return (size_t)wpb * keycap * sizeof(unsigned long long); }

cudaError_t launch_neigh(int N, const CellGrid& cg, const double* wpos, const float4* phi, const float4* plo,
                         const int* cell_count, const float4* cell_pos, double rcut, int cap, int* nbr_count,
                         int* nbr_j, int* nbr_s, int* status, cudaStream_t st, int wpb, float4* pd, bool pad,
                         bool* wrote_pd, bool blockwide) {
  if (wrote_pd) *wrote_pd = false;
  if (wpb < 1 || wpb > NEIGH_MAX_WPB) return cudaErrorInvalidValue;
  const double rc2 = rcut * rcut;
  // Error of the FP32 prefilter: each displacement component is formed from
  // FP32-rounded positions (|x| < L) and s * L_h, so |d_f32 - d| <= 4 ulp(L_max)
  // per component with margin; r^2 then moves by at most 2 sqrt(3) r_cut err_d
  // plus the rounding of r^2 itself.  Pairs whose FP32 r^2 falls within the band
  // are decided by the exact FP64 expression.
  const double Lmax = fmax(fmax(cg.L[0], cg.L[1]), fmax(cg.L[2], rcut));
  const double err_d = 4.0 * Lmax * 1.1920928955078125e-7 * (1 + cg.S[0] + cg.S[1] + cg.S[2]);
  const double err_r2 = 2.0 * 1.7320508075688772 * rcut * err_d + 3.0 * err_d * err_d + 8.0 * rc2 * 1.1920928955078125e-7;
  const double band = fmax(4.0 * err_r2, 1e-6 * rc2);
  const float rc2_lo = (float)(rc2 - band);
  const float rc2_hi = (float)(rc2 + band);
  const bool s1 = cg.S[0] == 1 && cg.S[1] == 1 && cg.S[2] == 1;
  // block per cell when there are enough cells to fill the GPU (two per SM)
  if (s1 && cg.ncells >= 2 * 152 && N < (1 << 26)) {
    int keycap = 32;
    while (keycap < cap) keycap <<= 1;
    // candidates and their image ids, hit counts and key lists: per own atom of
    // the cell (block-wide tests) or per warp
    const int nlists = blockwide ? cg.cap : wpb;
    const size_t cell_smem = (sizeof(float4) * 27 * (size_t)cg.cap + 27 * (size_t)cg.cap + 15) / 16 * 16 +
                             sizeof(int) * (size_t)((cg.cap + 3) / 4 * 4) +
                             (size_t)nlists * keycap * sizeof(unsigned);
    if (cell_smem <= 96 * 1024) {
      static size_t cgranted[2][64] = {};
      const void* kern = blockwide ? (const void*)neigh_cell_kernel<true> : (const void*)neigh_cell_kernel<false>;
      if (cudaError_t e = grant_smem(kern, cell_smem, cgranted[blockwide ? 1 : 0])) return e;
      if (blockwide)
        neigh_cell_kernel<true><<<cg.ncells, wpb * 32, cell_smem, st>>>(
            N, cg, wpos, phi, plo, cell_count, cell_pos, rc2, rc2_lo, rc2_hi, cap, keycap, pad ? 1 : 0, nbr_count,
            nbr_j, nbr_s, pd, status);
      else
        neigh_cell_kernel<false><<<cg.ncells, wpb * 32, cell_smem, st>>>(
            N, cg, wpos, phi, plo, cell_count, cell_pos, rc2, rc2_lo, rc2_hi, cap, keycap, pad ? 1 : 0, nbr_count,
            nbr_j, nbr_s, pd, status);
      if (wrote_pd) *wrote_pd = pd != nullptr;
      return cudaGetLastError();
    }
  }
  int keycap = 32;
  while (keycap < cap) keycap <<= 1;
  const size_t smem = neigh_smem_bytes(keycap, wpb);
  static size_t granted[64] = {};
  if (cudaError_t e = grant_smem((const void*)neigh_kernel, smem, granted)) return e;
  neigh_kernel<<<(N + wpb - 1) / wpb, wpb * 32, smem, st>>>(
      N, cg, wpos, phi, plo, cell_count, cell_pos, rc2, rc2_lo, rc2_hi, cap, keycap, nbr_count, nbr_j, nbr_s,
      status);
  return cudaGetLastError();
}

cudaError_t launch_rev(int N, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s, int* rev,
                       int* status, cudaStream_t st) {
  const size_t tot = (size_t)N * cap;
  const int tb = 256;
  rev_kernel<<<(unsigned)((tot + tb - 1) / tb), tb, 0, st>>>(N, cap, nbr_count, nbr_j, nbr_s, rev, status);
  return cudaGetLastError();
}

cudaError_t launch_export_neighbors(int N, int cap, const int* nbr_count, const int* nbr_j, const int* nbr_s,
                                    int cap_out, int* count_out, int* j_out, int* s_out, cudaStream_t st) {
  const size_t tot = (size_t)N * cap_out;
  const int tb = 256;
  export_neighbors_kernel<<<(unsigned)((tot + tb - 1) / tb), tb, 0, st>>>(N, cap, nbr_count, nbr_j, nbr_s,
                                                                           cap_out, count_out, j_out, s_out);
  return cudaGetLastError();
}

}  // namespace fastpod
