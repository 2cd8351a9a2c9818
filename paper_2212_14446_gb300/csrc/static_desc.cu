// pod_descriptors_static: the descriptor pipeline (wrap and bin, neighbour
// search, fused atom kernel in descriptor mode) for one configuration, with every
// intermediate buffer -- the mixed path's radial table included -- carved out of
// one statically allocated device array instead of the handle's workspace.  The
// entry point calls no cudaMalloc, cudaFree or other allocating routine.
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
// scratch array (about 6.8 MB) is part of every GPU that loads the library and
// stays allocated until the process exits.  All calls share it: calls that
// overlap on the GPU (other streams, other host threads) race, so serialise
// them.  Set-up: pod_create looks up the array's device address
// (cudaGetSymbolAddress) on its device, with that device current, and caches it;
// with CUDA's lazy module loading that lookup is also what loads the array, so
// the entry point itself finds it in place.
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
constexpr size_t OFF_TAB = al256(OFF_CELLA + sizeof(float4) * (size_t)STATIC_MAX_CELLS * STATIC_CELL_CAP);
constexpr size_t OFF_STATUS = al256(OFF_TAB + sizeof(Q4<float>) * (size_t)pod_handle::TAB_N * MAXK);
constexpr size_t SCRATCH_BYTES = al256(OFF_STATUS + 256);
}  // namespace

static __device__ __align__(256) unsigned char g_pod_static_scratch[SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
constexpr int MAX_DEVICES = 256;
void* g_scratch_addr[MAX_DEVICES] = {};
// uid of the handle whose radial table is in the array on each device (0: none)
unsigned long long g_tab_owner[MAX_DEVICES] = {};

// Device address of the scratch array on device `dev` (which must be current);
// the host-side symbol is only a stand-in and must not be passed on.
cudaError_t lookup_locked(int dev) {
  if (g_scratch_addr[dev]) return cudaSuccess;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_pod_static_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[dev] = p;
  return cudaSuccess;
}

int scratch_address(pod_handle* h, unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return h->cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return h->fail(POD_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  e = lookup_locked(dev);
  if (e != cudaSuccess) return h->cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return POD_OK;
}
}  // namespace

int static_scratch_setup(int device) {
  if (device < 0 || device >= MAX_DEVICES) return (int)cudaErrorInvalidDevice;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess || cur != device) return (int)(e != cudaSuccess ? e : cudaErrorInvalidDevice);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  e = lookup_locked(device);
  if (e != cudaSuccess) cudaGetLastError();  // leave no sticky error behind; the entry point reports it
  return (int)e;
}

namespace {
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
  int rc = h->validate_system(sys);  // also: the handle's device must be current
  if (rc) return rc;
  if (!D) return h->fail(POD_EINVAL, "D is NULL");
  if (sys->n_configs > 1) return h->fail(POD_EINVAL, "pod_descriptors_static takes a single configuration");
  if (sys->n_local > 0 && sys->n_local < sys->n_atoms)
    return h->fail(POD_EINVAL, "pod_descriptors_static evaluates every atom: no ghost atoms (n_local)");
  if (h->excl3) return h->fail(POD_EINVAL, "pod_descriptors_static takes the fast POD descriptor set");
  const int N = sys->n_atoms;
  if (N > STATIC_MAX_ATOMS)
    return h->fail(POD_EINVAL, "pod_descriptors_static handles 1..%d atoms (got %d)", STATIC_MAX_ATOMS, N);
  if (h->K > MAXK) return h->fail(POD_EINVAL, "too many radial modes for the static radial table");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  rc = h->plan_single(N, sys->box, sys->pbc, pl);
  if (rc) return rc;
  // fixed capacities of the scratch layout; coarsen the cell grid to fit (the
  // search depth follows the list radius, r_cut plus any skin, as in plan_single)
  pl.cap = STATIC_NBR_CAP;
  pl.cg.cap = STATIC_CELL_CAP;
  const double rc_list = h->rlist();
  long long ncells = (long long)pl.cg.nc[0] * pl.cg.nc[1] * pl.cg.nc[2];
  while (ncells > STATIC_MAX_CELLS) {
    int dmax = 0;
    for (int d = 1; d < 3; ++d)
      if (pl.cg.nc[d] > pl.cg.nc[dmax]) dmax = d;
    CellGrid& cg = pl.cg;
    cg.nc[dmax] = std::max(1, cg.nc[dmax] / 2);
    cg.inv_cs[dmax] = cg.nc[dmax] / cg.L[dmax];
    const double cs = cg.L[dmax] / cg.nc[dmax];
    cg.S[dmax] = cg.pbc[dmax] ? (int)std::ceil(rc_list / cs * (1.0 + 1e-12)) : (cg.nc[dmax] > 1 ? 1 : 0);
    ncells = (long long)cg.nc[0] * cg.nc[1] * cg.nc[2];
  }
  pl.cg.ncells = (int)ncells;
  unsigned char* base = nullptr;
  if ((rc = scratch_address(h, &base))) return rc;
  int* status = reinterpret_cast<int*>(base + OFF_STATUS);
  int* cellc = reinterpret_cast<int*>(base + OFF_CELLC);
  const bool mixed = h->precision == POD_MIXED;
  const bool table = mixed && h->radial_mode == 0;
  Q4<float>* tab = reinterpret_cast<Q4<float>*>(base + OFF_TAB);
  // the array keeps the previous call's contents: clear what must start at zero,
  // and upload this handle's radial table unless it is the one already there
  // (from pageable host memory: staged by the driver, no device allocation)
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cellc, 0, sizeof(int) * (size_t)ncells, st);
  if (e != cudaSuccess) return h->cuda_fail(e, "static scratch clear");
  if (table) {
    h->build_table_host();
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return h->cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (g_tab_owner[dev] != h->uid) {
      e = cudaMemcpyAsync(tab, h->h_tab.data(), sizeof(Q4<float>) * h->h_tab.size(), cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return h->cuda_fail(e, "static radial table upload");
      g_tab_owner[dev] = h->uid;
    }
  }
  e = launch_bin(N, sys->pos, pl.cg, reinterpret_cast<double*>(base + OFF_WPOS), reinterpret_cast<float4*>(base + OFF_PHI),
                 reinterpret_cast<float4*>(base + OFF_PLO), cellc, reinterpret_cast<float4*>(base + OFF_CELLA), status, st,
                 nullptr, nullptr, reinterpret_cast<int*>(base + OFF_CNT));
  if (e != cudaSuccess) return h->cuda_fail(e, "bin kernel");
  e = launch_neigh(N, pl.cg, reinterpret_cast<const double*>(base + OFF_WPOS),
                   reinterpret_cast<const float4*>(base + OFF_PHI), reinterpret_cast<const float4*>(base + OFF_PLO),
                   cellc, reinterpret_cast<const float4*>(base + OFF_CELLA), rc_list, pl.cap,
                   reinterpret_cast<int*>(base + OFF_CNT), reinterpret_cast<int*>(base + OFF_NBRJ),
                   reinterpret_cast<int*>(base + OFF_NBRS), status, st, WPB_NEIGH, nullptr, true, nullptr,
                   neigh_blockwide_default(N));
  if (e != cudaSuccess) return h->cuda_fail(e, "neighbour kernel");
  const bool has4 = h->P.P4 >= 0;
  if (mixed) {
    AtomArgs<float> a;
    static_args(h, pl, base, D, a);
    a.rad = h->rad32;
    if (table) {  // the FP64-built cubic table, as in pod_descriptors
      a.rad.tab = tab;
      a.rad.tab_inv_h = (float)(pod_handle::TAB_N / (h->P.r_cut - h->P.r_in));
      a.rad.tab_n = pod_handle::TAB_N;
    } else {
      a.rad.tab = nullptr;  // POD_OPT_RADIAL = 1: snapshots evaluated per pair
    }
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
