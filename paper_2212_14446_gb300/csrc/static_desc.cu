// pod_descriptors_static: the descriptor pipeline (wrap and bin, neighbour
// search, fused atom kernel in descriptor mode) for one configuration, with every
// intermediate buffer carved out of one statically allocated device array
// instead of the handle's workspace.  Nothing here allocates device or pinned
// host memory.
//
// Why it exists: some callers cannot let a library allocate device memory --
// molecular-dynamics engines and plugins that manage all device memory through
// their own pool with a fixed budget, and forbid other code from calling
// cudaMalloc / cudaFree (which synchronise the device and fragment the pool).
// They can still call this entry point, passing their own input and output
// buffers.
//
// Limits: at most STATIC_MAX_ATOMS atoms, STATIC_NBR_CAP neighbours per atom,
// STATIC_MAX_CELLS cells of STATIC_CELL_CAP atoms; larger inputs are rejected
// with POD_EINVAL, more neighbours or a fuller cell with POD_ENEIGH.  The
// scratch array (about 6.3 MB) is part of every GPU that loads the library and
// stays allocated until the process exits.  All calls share it: calls that
// overlap on the GPU (other streams, other host threads) race, so serialise
// them.  The first call on each device looks up the array's device address
// (cudaGetSymbolAddress) with that device current and caches it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pod_internal.h"

using namespace fastpod;

namespace {
constexpr int STATIC_MAX_ATOMS = 4096;
constexpr int STATIC_NBR_CAP = 64;
constexpr int STATIC_MAX_CELLS = 8192;
constexpr int STATIC_CELL_CAP = 32;
constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_WPOS = 0;
constexpr size_t OFF_PHI = al256(OFF_WPOS + sizeof(double) * 3 * STATIC_MAX_ATOMS);
constexpr size_t OFF_PLO = al256(OFF_PHI + sizeof(float4) * STATIC_MAX_ATOMS);
constexpr size_t OFF_CNT = al256(OFF_PLO + sizeof(float4) * STATIC_MAX_ATOMS);
constexpr size_t OFF_NBRJ = al256(OFF_CNT + sizeof(int) * STATIC_MAX_ATOMS);
constexpr size_t OFF_NBRS = al256(OFF_NBRJ + sizeof(int) * (size_t)STATIC_MAX_ATOMS * STATIC_NBR_CAP);
constexpr size_t OFF_CELLC = al256(OFF_NBRS + sizeof(int) * (size_t)STATIC_MAX_ATOMS * STATIC_NBR_CAP);
constexpr size_t OFF_CELLA = al256(OFF_CELLC + sizeof(int) * STATIC_MAX_CELLS);
constexpr size_t OFF_STATUS = al256(OFF_CELLA + sizeof(float4) * (size_t)STATIC_MAX_CELLS * STATIC_CELL_CAP);
constexpr size_t SCRATCH_BYTES = al256(OFF_STATUS + 256);
}  // namespace

static __device__ __align__(256) unsigned char g_pod_static_scratch[SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
constexpr int MAX_DEVICES = 256;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per
// device; the host-side symbol is only a stand-in and must not be passed on).
int scratch_address(pod_handle* h, unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return h->cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return h->fail(POD_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pod_static_scratch);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return POD_OK;
}

template <typename T>
void static_args(const pod_handle* h, const Plan& pl, const unsigned char* base, double* D, AtomArgs<T>& a) {
  std::memset(&a, 0, sizeof(a));
  a.N = pl.N;
  a.n_eval = pl.N;
  a.cap = pl.cap;
  a.nbr_count = reinterpret_cast<const int*>(base + OFF_CNT);
  a.nbr_j = reinterpret_cast<const int*>(base + OFF_NBRJ);
  a.nbr_s = reinterpret_cast<const int*>(base + OFF_NBRS);
  a.wpos = reinterpret_cast<const double*>(base + OFF_WPOS);
  a.phi = reinterpret_cast<const float4*>(base + OFF_PHI);
  a.plo = reinterpret_cast<const float4*>(base + OFF_PLO);
  for (int d = 0; d < 3; ++d) {
    a.L[d] = pl.cg.L[d];
    a.Lh[d] = (float)pl.cg.L[d];
    a.Ll[d] = (float)(pl.cg.L[d] - (double)a.Lh[d]);
  }
  a.K = h->K;
  a.K2 = h->P.K2;
  a.K3 = h->P.K3;
  a.K4 = h->P.K4;
  a.P3 = h->P.P3;
  a.P4 = h->P.P4;
  a.KA4 = h->KA4;
  a.M = h->M;
  a.col3 = 1 + h->P.K2;
  a.col4 = a.col3 + h->P.K3 * (h->P.P3 + 1);
  a.D = D;
  a.status = reinterpret_cast<int*>(const_cast<unsigned char*>(base) + OFF_STATUS);
  a.rmask = mask_radius<T>(h->skin > 0 ? h->P.r_cut : 0.0);  // a list built with a skin keeps only pairs inside r_cut
}
}  // namespace

extern "C" int pod_descriptors_static(pod_handle* h, const pod_system* sys, double* D, void* stream) {
  NvtxRange nvtx_("pod_descriptors_static");
  if (!h) return POD_EINVAL;
  if (!sys || !sys->pos || !D) return h->fail(POD_EINVAL, "system, positions and D are required");
  if (sys->n_configs > 1) return h->fail(POD_EINVAL, "pod_descriptors_static takes a single configuration");
  if (h->excl3) return h->fail(POD_EINVAL, "pod_descriptors_static takes the fast POD descriptor set");
  const int N = sys->n_atoms;
  if (N < 1 || N > STATIC_MAX_ATOMS)
    return h->fail(POD_EINVAL, "pod_descriptors_static handles 1..%d atoms (got %d)", STATIC_MAX_ATOMS, N);
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  int rc = h->plan_single(N, sys->box, sys->pbc, pl);
  if (rc) return rc;
  // fixed capacities of the scratch layout; coarsen the cell grid to fit
  pl.cap = STATIC_NBR_CAP;
  pl.cg.cap = STATIC_CELL_CAP;
  long long ncells = (long long)pl.cg.nc[0] * pl.cg.nc[1] * pl.cg.nc[2];
  while (ncells > STATIC_MAX_CELLS) {
    int dmax = 0;
    for (int d = 1; d < 3; ++d)
      if (pl.cg.nc[d] > pl.cg.nc[dmax]) dmax = d;
    CellGrid& cg = pl.cg;
    cg.nc[dmax] = std::max(1, cg.nc[dmax] / 2);
    cg.inv_cs[dmax] = cg.nc[dmax] / cg.L[dmax];
    const double cs = cg.L[dmax] / cg.nc[dmax];
    cg.S[dmax] = cg.pbc[dmax] ? (int)std::ceil(h->P.r_cut / cs * (1.0 + 1e-12)) : (cg.nc[dmax] > 1 ? 1 : 0);
    ncells = (long long)cg.nc[0] * cg.nc[1] * cg.nc[2];
  }
  pl.cg.ncells = (int)ncells;
  unsigned char* base = nullptr;
  if ((rc = scratch_address(h, &base))) return rc;
  int* status = reinterpret_cast<int*>(base + OFF_STATUS);
  int* cellc = reinterpret_cast<int*>(base + OFF_CELLC);
  // the array keeps the previous call's contents: clear what must start at zero
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cellc, 0, sizeof(int) * (size_t)ncells, st);
  if (e != cudaSuccess) return h->cuda_fail(e, "static scratch clear");
  e = launch_bin(N, sys->pos, pl.cg, reinterpret_cast<double*>(base + OFF_WPOS), reinterpret_cast<float4*>(base + OFF_PHI),
                 reinterpret_cast<float4*>(base + OFF_PLO), cellc, reinterpret_cast<float4*>(base + OFF_CELLA), status, st,
                 nullptr, nullptr, reinterpret_cast<int*>(base + OFF_CNT));
  if (e != cudaSuccess) return h->cuda_fail(e, "bin kernel");
  e = launch_neigh(N, pl.cg, reinterpret_cast<const double*>(base + OFF_WPOS),
                   reinterpret_cast<const float4*>(base + OFF_PHI), reinterpret_cast<const float4*>(base + OFF_PLO),
                   cellc, reinterpret_cast<const float4*>(base + OFF_CELLA), h->P.r_cut, pl.cap,
                   reinterpret_cast<int*>(base + OFF_CNT), reinterpret_cast<int*>(base + OFF_NBRJ),
                   reinterpret_cast<int*>(base + OFF_NBRS), status, st);
  if (e != cudaSuccess) return h->cuda_fail(e, "neighbour kernel");
  const bool has4 = h->P.P4 >= 0;
  if (h->precision == POD_MIXED) {
    AtomArgs<float> a;
    static_args(h, pl, base, D, a);
    a.rad = h->rad32;  // per-pair evaluation of the snapshots (no radial table in the scratch)
    a.rad.tab = nullptr;
    e = launch_atom_f32(0, a, h->PA, has4, st);
  } else {
    AtomArgs<double> a;
    static_args(h, pl, base, D, a);
    a.rad = h->rad64;
    e = launch_atom_f64(0, a, h->PA, has4, st);
  }
  if (e != cudaSuccess) return h->cuda_fail(e, "atom kernel");
  int hs = 0;
  e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return h->cuda_fail(e, "static status read");
  if (hs & (ST_NEIGH | ST_CELL))
    return h->fail(POD_ENEIGH, "more than %d neighbours per atom or %d atoms per cell (status 0x%x)", STATIC_NBR_CAP,
                   STATIC_CELL_CAP, hs);
  if (hs & ST_NONFINITE) return h->fail(POD_ENONFINITE, "non-finite positions");
  if (hs & ST_RANGE) return h->fail(POD_ERANGE, "a pair is closer than r_in");
  return POD_OK;
}
