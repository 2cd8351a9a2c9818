// C ABI of the fastpod library: handle life cycle, POD basis, workspace and the
// orchestration of the neighbour / atom / gather / reduce kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pod.h"
#include "pod_common.cuh"
#include "pod_internal.h"
#include "pod_kernels.h"

using namespace fastpod;

// ============================================================ small helpers
namespace {

int num_partitions_upto(int P) {
  int cnt = 0;
  for (int n = 0; n <= P; ++n)
    for (int a = n; a >= 0; --a)
      for (int b = std::min(a, n - a); b >= 0; --b) {
        const int c = n - a - b;
        if (c >= 0 && c <= b) ++cnt;
      }
  return cnt;
}

// Radial snapshots Phi_l(r) on the host, FP64 (Eq. 3-11), rows ordered
// phi(alpha_a, beta_b) for a (outer), b (inner), then varphi(gamma_g).
void host_snapshots(const HostParams& P, double r, double* out) {
  const double h = P.r_cut - P.r_in;
  const double s = r - P.r_in;
  const double t = s / h;
  const double u = 1.0 - t * t * t;
  const double fc = std::exp(1.0 - 1.0 / std::sqrt(u * u + 1e-6));
  int row = 0;
  for (size_t a = 0; a < P.alpha.size(); ++a)
    for (size_t b = 0; b < P.beta.size(); ++b) {
      const double x = (std::exp(-P.beta[b] * t) - 1.0) / (std::exp(-P.beta[b]) - 1.0);
      out[row++] = fc * std::sin(P.alpha[a] * M_PI * x) / s;
    }
  for (size_t g = 0; g < P.gamma.size(); ++g) out[row++] = fc * std::pow(r, -P.gamma[g]);
}

// POD of the snapshot family (Section 2.2, Eq. 12): one-sided (Hestenes)
// Jacobi on X = sqrt(h) Phi (n_grid x Ns); the right singular vectors are the
// eigenvectors of C = X^T X and sigma^2 its eigenvalues.  Sorted descending,
// largest-magnitude entry positive, Q_lk = v_lk / sigma_k.
int pod_basis(const HostParams& P, int n_grid, int K, std::vector<double>& Q, std::vector<double>& eig) {
  const int Ns = (int)(P.alpha.size() * P.beta.size() + P.gamma.size());
  const double h = (P.r_cut - P.r_in) / n_grid;
  std::vector<double> X((size_t)Ns * n_grid);  // column-major: column a = snapshot a
  std::vector<double> row(Ns);
  for (int g = 0; g < n_grid; ++g) {
    host_snapshots(P, P.r_in + (g + 0.5) * h, row.data());
    for (int a = 0; a < Ns; ++a) X[(size_t)a * n_grid + g] = std::sqrt(h) * row[a];
  }
  std::vector<double> V((size_t)Ns * Ns, 0.0);
  for (int a = 0; a < Ns; ++a) V[(size_t)a * Ns + a] = 1.0;  // column-major too
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int a = 0; a < Ns - 1; ++a)
      for (int b = a + 1; b < Ns; ++b) {
        double* xa = &X[(size_t)a * n_grid];
        double* xb = &X[(size_t)b * n_grid];
        double al = 0, be = 0, ga = 0;
        for (int g = 0; g < n_grid; ++g) {
          al += xa[g] * xa[g];
          be += xb[g] * xb[g];
          ga += xa[g] * xb[g];
        }
        if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
        rotated = true;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int g = 0; g < n_grid; ++g) {
          const double p = xa[g], q = xb[g];
          xa[g] = c * p - s * q;
          xb[g] = s * p + c * q;
        }
        double* va = &V[(size_t)a * Ns];
        double* vb = &V[(size_t)b * Ns];
        for (int l = 0; l < Ns; ++l) {
          const double p = va[l], q = vb[l];
          va[l] = c * p - s * q;
          vb[l] = s * p + c * q;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> lam(Ns);
  for (int a = 0; a < Ns; ++a) {
    double s2 = 0;
    for (int g = 0; g < n_grid; ++g) s2 += X[(size_t)a * n_grid + g] * X[(size_t)a * n_grid + g];
    lam[a] = s2;
  }
  std::vector<int> idx(Ns);
  for (int a = 0; a < Ns; ++a) idx[a] = a;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return lam[x] > lam[y]; });
  eig.assign(Ns, 0.0);
  Q.assign((size_t)Ns * K, 0.0);
  for (int k = 0; k < Ns; ++k) eig[k] = lam[idx[k]];
  for (int k = 0; k < K; ++k) {
    const int col = idx[k];
    if (!(lam[col] > 0)) return -1;
    const double* v = &V[(size_t)col * Ns];
    int am = 0;
    for (int l = 1; l < Ns; ++l)
      if (std::fabs(v[l]) > std::fabs(v[am])) am = l;
    const double sc = (v[am] < 0 ? -1.0 : 1.0) / std::sqrt(lam[col]);
    for (int l = 0; l < Ns; ++l) Q[(size_t)l * K + k] = v[l] * sc;
  }
  return 0;
}

// Phi_l(r) and dPhi_l/dr on the host, FP64, same row order as host_snapshots.
void host_snapshots_d(const HostParams& P, double r, double* phi, double* dphi) {
  const double h = P.r_cut - P.r_in;
  const double s = r - P.r_in;
  const double t = s / h;
  const double u = 1.0 - t * t * t;
  const double y = u * u + 1e-6;
  const double fc = std::exp(1.0 - 1.0 / std::sqrt(y));
  const double dfc = fc * (u * (-3.0 * t * t / h)) / (y * std::sqrt(y));
  int row = 0;
  for (size_t a = 0; a < P.alpha.size(); ++a)
    for (size_t b = 0; b < P.beta.size(); ++b) {
      const double be = P.beta[b], al = P.alpha[a];
      const double em1 = std::exp(-be) - 1.0, et = std::exp(-be * t);
      const double x = (et - 1.0) / em1, dx = -be / h * et / em1;
      const double sn = std::sin(al * M_PI * x), cs = std::cos(al * M_PI * x);
      const double f = sn / s, df = (al * M_PI * cs * dx * s - sn) / (s * s);
      phi[row] = fc * f;
      dphi[row] = dfc * f + fc * df;
      ++row;
    }
  for (size_t g = 0; g < P.gamma.size(); ++g) {
    const double f = std::pow(r, -P.gamma[g]), df = -P.gamma[g] * f / r;
    phi[row] = fc * f;
    dphi[row] = dfc * f + fc * df;
    ++row;
  }
}

bool is_seq(const std::vector<double>& v) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] != (double)(i + 1)) return false;
  return true;
}

template <typename T>
void fill_radial(const pod_handle* h, RadialConst<T>& rc) {
  std::memset(&rc, 0, sizeof(rc));
  const HostParams& P = h->P;
  rc.r_in = (T)P.r_in;
  rc.inv_h = (T)(1.0 / (P.r_cut - P.r_in));
  rc.n_alpha = (int)P.alpha.size();
  rc.n_beta = (int)P.beta.size();
  rc.n_gamma = (int)P.gamma.size();
  rc.K = h->K;
  for (int a = 0; a < rc.n_alpha; ++a) rc.alpha[a] = (T)P.alpha[a];
  for (int b = 0; b < rc.n_beta; ++b) {
    rc.beta[b] = (T)P.beta[b];
    rc.inv_ebm1[b] = (T)(1.0 / (std::exp(-P.beta[b]) - 1.0));
  }
  for (int g = 0; g < rc.n_gamma; ++g) rc.gamma[g] = (T)P.gamma[g];
  for (int l = 0; l < h->Ns; ++l)
    for (int k = 0; k < h->K; ++k) rc.Q[l][k] = (T)h->Q[(size_t)l * h->K + k];
  rc.alpha_seq = is_seq(P.alpha) ? 1 : 0;
  rc.gamma_seq = is_seq(P.gamma) ? 1 : 0;
}

}  // namespace

// ============================================================ handle helpers
int pod_handle::fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  err = buf;
  return code;
}

int pod_handle::cuda_fail(cudaError_t e, const char* what) {
  return fail(POD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int pod_handle::ensure(DevBuf& b, size_t bytes, const char* what) {
  if (bytes <= b.bytes && b.p) return POD_OK;
  size_t nb = std::max<size_t>(bytes, 256);
  nb = nb + nb / 4;
  if (ws_limit) {  // POD_OPT_WORKSPACE_LIMIT_MB: refuse growth past the cap, before freeing anything
    size_t others = 0;
    for (DevBuf* o : all_bufs())
      if (o != &b) others += o->bytes;
    if (others + nb > ws_limit) nb = std::max<size_t>(bytes, 256);  // without the growth margin
    if (others + nb > ws_limit)
      return fail(POD_ENOMEM, "%s: %zu bytes would take the workspace to %zu, above its limit of %zu", what, nb,
                  others + nb, ws_limit);
  }
  if (b.p) {
    drop_host_graph();  // a captured host graph may hold this buffer's address
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, nb);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(POD_ENOMEM, "cudaMalloc(%zu) for %s failed: %s", nb, what, cudaGetErrorString(e));
  }
  b.bytes = nb;
  return POD_OK;
}

pod_handle::~pod_handle() {
  for (DevBuf* b : all_bufs()) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
  }
  if (h_status) cudaFreeHost(h_status);
  for (cudaEvent_t& e : ev)
    if (e) cudaEventDestroy(e);
  drop_host_graph();
  if (fhost) cudaFreeHost(fhost);
  if (fcap_st) cudaStreamDestroy(fcap_st);
}

bool pod_handle::HostKey::operator==(const HostKey& o) const {
  for (int k = 0; k < 6; ++k)
    if (ptr[k] != o.ptr[k]) return false;
  for (int d = 0; d < 3; ++d)
    if (pbc[d] != o.pbc[d] || box[d] != o.box[d]) return false;
  return N == o.N && precision == o.precision && quad == o.quad && radial == o.radial && tune_gen == o.tune_gen &&
         emb_deg == o.emb_deg && excl3 == o.excl3 && n_local == o.n_local;
}

void pod_handle::drop_host_graph() {
  if (hgraph) cudaGraphExecDestroy(hgraph);
  hgraph = nullptr;
  hkey_valid = false;
  fit_graph_drop();  // a recorded fit holds buffer addresses too
}

int pod_handle::mark(int k, cudaStream_t st) {
  if (!timing) return POD_OK;
  if (!ev[k]) {
    cudaError_t e = cudaEventCreate(&ev[k]);
    if (e != cudaSuccess) return cuda_fail(e, "event create");
  }
  cudaError_t e = cudaEventRecord(ev[k], st);
  if (e != cudaSuccess) return cuda_fail(e, "event record");
  return POD_OK;
}

int pod_handle::timing_collect() {
  if (!timing) return POD_OK;
  cudaError_t e = cudaEventSynchronize(ev[4]);
  if (e != cudaSuccess) return cuda_fail(e, "event sync");
  for (int k = 0; k < 4; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "event elapsed");
    t_acc[k] += ms;
  }
  ++t_calls;
  return POD_OK;
}

// Launch-shape autotuner: times the step's three phases (neighbour build, atom
// kernel, gather) with CUDA events for each candidate shape on the caller's
// system and keeps, per phase, the fastest (coordinate search; the phases are
// independent kernels).  The winner is stored for the system's size class and
// used by every later call on systems of that class.
int pod_handle::autotune(const pod_system* sys, const double* c, int reps, cudaStream_t st, LaunchShape& best,
                         double ms[3]) {
  int rc_ = validate_system(sys);
  if (rc_) return rc_;
  if (sys->n_configs > 1) return autotune_fit(sys, reps, best, ms);
  if (!c) return fail(POD_EINVAL, "coefficients are required");
  if (reps < 1) reps = 5;
  if ((rc_ = ensure(E_out, sizeof(double), "energy"))) return rc_;
  double* E = (double*)E_out.p;
  const int cls = size_class(sys->n_atoms);
  const int keep_sync = sync, keep_timing = timing, keep_nbr = nbr_mode;
  const double keep_acc[4] = {t_acc[0], t_acc[1], t_acc[2], t_acc[3]};
  const int keep_calls = t_calls;
  sync = 1;
  timing = 1;
  nbr_mode = 0;  // every timed call builds its list
  auto measure = [&](const LaunchShape& s, double out[3]) -> int {
    tuned[cls] = s;
    int r = energy_forces(sys, c, E, nullptr, nullptr, nullptr, st);  // warm-up (sizes the workspace)
    if (r) return r;
    for (int k = 0; k < 4; ++k) t_acc[k] = 0;
    t_calls = 0;
    for (int i = 0; i < reps && !r; ++i) r = energy_forces(sys, c, E, nullptr, nullptr, nullptr, st);
    for (int k = 0; k < 3; ++k) out[k] = t_calls ? t_acc[k] / t_calls : 0.0;
    return r;
  };
  LaunchShape cur{};
  double t[3];
  static const int atom_c[] = {1, 2, 4};
  static const int neigh_c[] = {2, 4, 6, 8};
  static const int gather_c[][2] = {{16, 3}, {16, 2}, {8, 6}, {8, 4}, {4, 12}};
  double best_atom = 1e30, best_neigh = 1e30, best_gather = 1e30;
  LaunchShape win = cur;
  // the separate adjoint kernel exists for the linear mixed path only
  const bool can_split = precision == POD_MIXED && !quad && emb_deg == 0 && adj_force < 0;
  for (int sp = 0; sp < (can_split ? 2 : 1) && !rc_; ++sp)
    for (int a : atom_c)
      for (int rp = 0; rp < 2 && !rc_; ++rp) {
        if (rp && (precision != POD_MIXED || radial_mode != 0 || sp)) break;  // R' staging: fused table path only
        LaunchShape s = win;
        s.atom_wpb = a;
        s.atom_rp = rp;
        s.atom_split = can_split ? sp : -1;
        if ((rc_ = measure(s, t))) break;
        if (t[1] < best_atom) {
          best_atom = t[1];
          win.atom_wpb = a;
          win.atom_rp = rp;
          win.atom_split = s.atom_split;
        }
      }
  for (int bw = 0; !rc_ && bw < 2; ++bw)
    for (int n = 0; !rc_ && n < 4; ++n) {
      LaunchShape s = win;
      s.neigh_wpb = neigh_c[n];
      s.neigh_blockwide = bw;
      if ((rc_ = measure(s, t))) break;
      if (t[0] < best_neigh) {
        best_neigh = t[0];
        win.neigh_wpb = neigh_c[n];
        win.neigh_blockwide = bw;
      }
    }
  // the FP32 path sums forces in the atom kernel (fixed point) and has no gather
  for (int g = 0; !rc_ && precision != POD_MIXED && g < 5; ++g) {
    LaunchShape s = win;
    s.gather_wpb = gather_c[g][0];
    s.gather_bps = gather_c[g][1];
    if ((rc_ = measure(s, t))) break;
    if (t[2] < best_gather) {
      best_gather = t[2];
      win.gather_wpb = gather_c[g][0];
      win.gather_bps = gather_c[g][1];
    }
  }
  sync = keep_sync;
  timing = keep_timing;
  nbr_mode = keep_nbr;
  for (int k = 0; k < 4; ++k) t_acc[k] = keep_acc[k];
  t_calls = keep_calls;
  reuse_ok = false;
  if (rc_) {
    tuned.erase(cls);
    return rc_;
  }
  tuned[cls] = win;
  ++tune_gen;
  best = win;
  ms[0] = best_neigh;
  ms[1] = best_atom;
  ms[2] = best_gather < 1e29 ? best_gather : t[2];
  return POD_OK;
}

// Batch form of the tuner: the fit's design pass (atom kernel in design mode and
// the force-row gather), timed with CUDA events around the design-matrix stage
// of pod_fit (zero labels) for atom-kernel warps per block {1, 2, 4} and gather
// warps per block {2, 4, 8} (coordinate search); the winner serves later fits
// of batches of the same size class.
int pod_handle::autotune_fit(const pod_system* sys, int reps, LaunchShape& best, double ms[3]) {
  if (reps < 1) reps = 3;
  const int cls = size_class(sys->n_atoms);
  const long long rows = (long long)sys->n_configs + 3LL * sys->n_atoms;
  int rc_;
  if ((rc_ = ensure(tune_ref, sizeof(double) * (size_t)rows, "tuning labels"))) return rc_;
  cudaError_t e = cudaMemset(tune_ref.p, 0, sizeof(double) * (size_t)rows);
  if (e != cudaSuccess) return cuda_fail(e, "tuning labels");
  const double* Er = (const double*)tune_ref.p;
  const double* Fr = Er + sys->n_configs;
  const pod_fit_opts o{100.0, 1.0, 1e-12, 1, 0};
  const int keep_timing = timing;
  timing = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
    if (t0) cudaEventDestroy(t0);
    timing = keep_timing;
    return cuda_fail(cudaGetLastError(), "tuning events");
  }
  auto measure = [&](const LaunchShape& s, double& out) -> int {
    tuned_fit[cls] = s;
    int r = fit_build(sys, Er, Fr, o);  // warm-up (sizes the workspace)
    if (r) return r;
    float acc = 0.f;
    for (int i = 0; i < reps && !r; ++i) {
      cudaEventRecord(t0, nullptr);
      r = fit_build(sys, Er, Fr, o);
      cudaEventRecord(t1, nullptr);
      if (cudaEventSynchronize(t1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "tuning events");
      float m = 0.f;
      cudaEventElapsedTime(&m, t0, t1);
      acc += m;
    }
    out = acc / reps;
    return r;
  };
  static const int atom_c[] = {1, 2, 4};
  static const int gather_c[] = {2, 4, 8};  // the gather is bounded to 256 threads a block
  LaunchShape win{};
  double best_ms = 1e30, t = 0;
  for (int a : atom_c) {
    LaunchShape s = win;
    s.atom_wpb = a;
    if ((rc_ = measure(s, t))) break;
    if (t < best_ms) { best_ms = t; win.atom_wpb = a; }
  }
  for (int k = 0; !rc_ && k < 3; ++k) {
    LaunchShape s = win;
    s.design_wpb = gather_c[k];
    if ((rc_ = measure(s, t))) break;
    if (t < best_ms) { best_ms = t; win.design_wpb = gather_c[k]; }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  timing = keep_timing;
  fit_R = 0;  // the tuning design matrices are not a fit's
  if (rc_) {
    tuned_fit.erase(cls);
    return rc_;
  }
  tuned_fit[cls] = win;
  ++tune_gen;
  best = win;
  ms[0] = 0.0;
  ms[1] = best_ms;
  ms[2] = 0.0;
  return POD_OK;
}

std::vector<DevBuf*> pod_handle::all_bufs() {
  return {&cell_count, &cell_atoms, &wpos, &phi, &plo, &nbr_count, &nbr_j, &nbr_s, &rev, &g, &Ei,
          &Wat, &status, &offs, &pos_in, &c_in, &E_out, &F_out, &W_out, &Ei_out, &fitA, &fitG, &fitb,
          &fitwork, &cfg_of, &boxes, &rtab, &wpart, &Dws, &chunks, &cpart, &wrapk, &gdm, &dmG, &facc, &qS32, &qS64, &pdisp, &adjb, &qrw, &halo_cnt, &mgrad, &tune_ref,
          &embW};
}

// ============================================================ C ABI
extern "C" {

int pod_create(const pod_params* prm, pod_handle** out) {
  NvtxRange nvtx_("pod_create");
  if (!out) return POD_EINVAL;
  *out = nullptr;
  if (!prm) return POD_EINVAL;
  pod_handle* h = new (std::nothrow) pod_handle();
  if (!h) return POD_ENOMEM;
  static std::atomic<unsigned long long> next_uid{1};
  h->uid = next_uid.fetch_add(1);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    h->device = -1;
  }
  auto bad = [&](const char* msg) {
    h->err = msg;
    int code = POD_EINVAL;
    // keep the handle alive so the caller can read the message
    *out = h;
    return code;
  };
  if (!(prm->r_in > 0) || !(prm->r_cut > prm->r_in)) return bad("require 0 < r_in < r_cut");
  if (prm->n_alpha < 1 || prm->n_alpha > MAXA || !prm->alpha) return bad("n_alpha must be in 1..8");
  if (prm->n_beta < 1 || prm->n_beta > MAXB || !prm->beta) return bad("n_beta must be in 1..2");
  if (prm->n_gamma < 0 || prm->n_gamma > MAXG || (prm->n_gamma > 0 && !prm->gamma))
    return bad("n_gamma must be in 0..8");
  for (int b = 0; b < prm->n_beta; ++b)
    if (!(prm->beta[b] > 0)) return bad("every beta must be > 0");
  if (prm->P3 < -1 || prm->P3 > PAMAX || prm->P4 < -1 || prm->P4 > PAMAX)
    return bad("P3 and P4 must be in -1..4");
  if (prm->K2 < 0 || prm->K3 < 0 || prm->K4 < 0 || prm->K2 > MAXK || prm->K3 > MAXK || prm->K4 > MAXK)
    return bad("K2, K3, K4 must be in 0..16");
  if (prm->precision != POD_FP64 && prm->precision != POD_MIXED) return bad("precision must be POD_FP64 or POD_MIXED");
  HostParams& P = h->P;
  P.r_in = prm->r_in;
  P.r_cut = prm->r_cut;
  P.alpha.assign(prm->alpha, prm->alpha + prm->n_alpha);
  P.beta.assign(prm->beta, prm->beta + prm->n_beta);
  if (prm->n_gamma) P.gamma.assign(prm->gamma, prm->gamma + prm->n_gamma);
  P.K2 = prm->K2;
  P.P3 = prm->P3;
  P.P4 = prm->P4;
  P.K3 = prm->P3 >= 0 ? prm->K3 : 0;
  P.K4 = prm->P4 >= 0 ? prm->K4 : 0;
  h->precision = prm->precision;
  h->Ns = prm->n_alpha * prm->n_beta + prm->n_gamma;
  h->K = std::max(P.K2, std::max(P.K3, P.K4));
  if (h->K < 1) return bad("at least one of K2, K3, K4 must be positive");
  if (h->K > h->Ns) return bad("radial modes K must not exceed the number of snapshots");
  h->PA = std::max(0, std::max(P.P3, P.P4));
  h->KA4 = P.P4 >= 0 ? num_partitions_upto(P.P4) : 0;
  h->M = 1 + P.K2 + P.K3 * (P.P3 + 1) + P.K4 * h->KA4;
  const int n_grid = prm->n_grid > 0 ? prm->n_grid : 2000;
  if (n_grid < h->Ns) return bad("n_grid must be at least Ns");
  if (prm->Q) {
    h->Q.assign(prm->Q, prm->Q + (size_t)h->Ns * h->K);
    h->eig.assign(h->Ns, 0.0);
  } else if (pod_basis(P, n_grid, h->K, h->Q, h->eig) != 0) {
    return bad("POD basis: snapshot family is rank deficient for the requested K");
  }
  fill_radial<float>(h, h->rad32);
  fill_radial<double>(h, h->rad64);
  // set-up of the allocation-free entry point on this device (address of its
  // static scratch array); a failure here is reported by that entry point
  if (h->device >= 0) static_scratch_setup(h->device);
  *out = h;
  return POD_OK;
}

int pod_destroy(pod_handle* h) {
  delete h;
  return POD_OK;
}

int pod_info(const pod_handle* h, int* M, int* Ns, int* K, double* Q_out, double* eig_out) {
  if (!h) return POD_EINVAL;
  if (M) *M = h->M;
  if (Ns) *Ns = h->Ns;
  if (K) *K = h->K;
  if (Q_out && !h->Q.empty()) std::memcpy(Q_out, h->Q.data(), sizeof(double) * h->Q.size());
  if (eig_out && !h->eig.empty()) std::memcpy(eig_out, h->eig.data(), sizeof(double) * h->eig.size());
  return POD_OK;
}

int pod_set_option(pod_handle* h, int option, int value) {
  if (!h) return POD_EINVAL;
  if (option == POD_OPT_SYNC) {
    h->sync = value ? 1 : 0;
    return POD_OK;
  }
  if (option == POD_OPT_RADIAL) {
    if (value != 0 && value != 1) return h->fail(POD_EINVAL, "radial mode must be 0 (table) or 1 (direct)");
    h->radial_mode = value;
    return POD_OK;
  }
  if (option == POD_OPT_NEIGHBOR_REUSE) {
    h->nbr_mode = value ? 1 : 0;
    return POD_OK;
  }
  if (option == POD_OPT_TIMING) {
    h->timing = value ? 1 : 0;
    return POD_OK;
  }
  if (option == POD_OPT_GRAM) {
    if (value < 0 || value > 2) return h->fail(POD_EINVAL, "Gram mode must be 0, 1 or 2");
    h->gram_mode = value;
    return POD_OK;
  }
  if (option == POD_OPT_DESCRIPTORS) {
    if (value != 0 && value != 1) return h->fail(POD_EINVAL, "descriptor set must be 0 (fast POD) or 1");
    h->excl3 = value;
    return POD_OK;
  }
  if (option == POD_OPT_ADJOINT) {
    if (value < -1 || value > 1) return h->fail(POD_EINVAL, "adjoint kernel must be -1 (by shape), 0 or 1");
    h->adj_force = value;
    return POD_OK;
  }
  if (option == POD_OPT_WORKSPACE_LIMIT_MB) {
    if (value < 0) return h->fail(POD_EINVAL, "workspace limit must be >= 0 MiB (0: none)");
    h->ws_limit = (size_t)value << 20;
    return POD_OK;
  }
  if (option == POD_OPT_HOST_MAPPED) {
    if (value != 0 && value != 1) return h->fail(POD_EINVAL, "host mapping must be 0 or 1");
    h->host_mapped_off = value == 0;
    h->drop_host_graph();
    return POD_OK;
  }
  if (option == POD_OPT_FIT_GRAPH) {
    if (value != 0 && value != 1) return h->fail(POD_EINVAL, "fit recording must be 0 or 1");
    h->fit_off = value == 0;
    if (h->fit_off) h->fit_graph_drop();
    return POD_OK;
  }
  if (option == POD_OPT_NEIGHBOR_TESTS) {
    if (value < -1 || value > 1) return h->fail(POD_EINVAL, "neighbour tests must be -1 (by shape), 0 or 1");
    h->neigh_force = value;
    return POD_OK;
  }
  if (option == POD_OPT_PRECISION) {
    if (value != POD_FP64 && value != POD_MIXED) return h->fail(POD_EINVAL, "precision must be POD_FP64 or POD_MIXED");
    h->precision = value;
    return POD_OK;
  }
  return h->fail(POD_EINVAL, "unknown option %d", option);
}

int pod_set_quadratic(pod_handle* h, const double* beta) {
  if (!h) return POD_EINVAL;
  if (!beta) {
    h->quad = false;
    return POD_OK;
  }
  h->emb_deg = 0;
  const int M = h->M;
  std::vector<double> S((size_t)M * M);
  std::vector<float> S32((size_t)M * M);
  for (int m = 0; m < M; ++m)
    for (int n = 0; n < M; ++n) {
      // S_mn = beta_mn + beta_nm over the upper triangle (diagonal: 2 beta_mm)
      const double v = m == n ? 2.0 * beta[(size_t)m * M + m] : beta[(size_t)std::min(m, n) * M + std::max(m, n)];
      if (!std::isfinite(v)) return h->fail(POD_EINVAL, "quadratic weights must be finite");
      S[(size_t)m * M + n] = v;
      S32[(size_t)m * M + n] = (float)v;
    }
  int rc;
  if ((rc = h->ensure(h->qS64, sizeof(double) * S.size(), "quadratic weights"))) return rc;
  if ((rc = h->ensure(h->qS32, sizeof(float) * S32.size(), "quadratic weights"))) return rc;
  cudaError_t e = cudaMemcpy(h->qS64.p, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->qS32.p, S32.data(), sizeof(float) * S32.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return h->cuda_fail(e, "quadratic weights upload");
  h->quad = true;
  return POD_OK;
}

int pod_set_embedding(pod_handle* h, const double* a, int degree, const double* alpha) {
  if (!h) return POD_EINVAL;
  if (!a) {
    h->emb_deg = 0;
    return POD_OK;
  }
  if (degree < 1 || degree > POD_EMB_MAX_DEGREE || !alpha)
    return h->fail(POD_EINVAL, "the embedding polynomial needs 1 <= degree <= %d and its coefficients",
                   POD_EMB_MAX_DEGREE);
  const int M = h->M;
  std::vector<double> w((size_t)M + degree + 1);
  for (int m = 0; m < M; ++m) w[m] = a[m];
  for (int k = 0; k <= degree; ++k) w[(size_t)M + k] = alpha[k];
  for (double v : w)
    if (!std::isfinite(v)) return h->fail(POD_EINVAL, "embedding weights must be finite");
  int rc;
  if ((rc = h->ensure(h->embW, sizeof(double) * w.size(), "embedding weights"))) return rc;
  cudaError_t e = cudaMemcpy(h->embW.p, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return h->cuda_fail(e, "embedding weights upload");
  h->quad = false;
  h->emb_deg = degree;
  return POD_OK;
}

int pod_autotune(pod_handle* h, const pod_system* sys, const double* c, int reps, int* shape, double* ms,
                 void* stream) {
  NvtxRange nvtx_("pod_autotune");
  if (!h) return POD_EINVAL;
  LaunchShape best{};
  double t[3] = {0, 0, 0};
  const int rc = h->autotune(sys, c, reps, (cudaStream_t)stream, best, t);
  if (rc) return rc;
  if (shape && sys && sys->n_configs > 1) {  // batch: the fit's design pass
    shape[0] = 0;
    shape[1] = best.atom_wpb;
    shape[2] = best.design_wpb;
    shape[3] = shape[4] = shape[5] = 0;
  } else if (shape) {
    shape[0] = best.neigh_wpb;
    shape[1] = best.atom_wpb;
    shape[2] = best.gather_wpb;
    shape[3] = best.gather_bps;
    shape[4] = best.atom_split == 1 ? 2 : best.atom_rp;
    shape[5] = best.neigh_blockwide == 1 ? 1 : 0;
  }
  if (ms)
    for (int k = 0; k < 3; ++k) ms[k] = t[k];
  return POD_OK;
}

const char* pod_last_error(const pod_handle* h) { return h ? h->err.c_str() : "null handle"; }

int pod_set_skin(pod_handle* h, double skin) {
  if (!h) return POD_EINVAL;
  if (!(skin >= 0) || !std::isfinite(skin)) return h->fail(POD_EINVAL, "skin must be >= 0");
  h->skin = skin;
  h->reuse_ok = false;
  return POD_OK;
}

int pod_md_step(pod_handle* h, const pod_system* sys, double* pos, double* v, double* F, const double* c,
                double mass, double dt, double* E, void* stream) {
  NvtxRange nvtx_("pod_md_step");
  if (!h) return POD_EINVAL;
  return h->md_step(sys, pos, v, F, c, mass, dt, E, (cudaStream_t)stream);
}

int pod_timing(pod_handle* h, double* ms, int* calls) {
  if (!h) return POD_EINVAL;
  if (ms)
    for (int k = 0; k < 4; ++k) ms[k] = h->t_acc[k];
  if (calls) *calls = h->t_calls;
  for (int k = 0; k < 4; ++k) h->t_acc[k] = 0;
  h->t_calls = 0;
  return POD_OK;
}

int pod_status(pod_handle* h, void* stream) {
  if (!h) return POD_EINVAL;
  return h->read_status((cudaStream_t)stream);
}

}  // extern "C"

// ============================================================ orchestration
int pod_handle::read_status(cudaStream_t st) {
  if (!status.p) return POD_OK;
  if (!h_status) {
    cudaError_t ea = cudaMallocHost(&h_status, sizeof(int) * 4);
    if (ea != cudaSuccess) {
      h_status = nullptr;
      return cuda_fail(ea, "pinned status word");
    }
  }
  cudaError_t e = cudaMemcpyAsync(h_status, status.p, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  const int s = *h_status;
  last_status = s;
  e = cudaMemsetAsync(status.p, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "status clear");
  return status_error(s);
}

// The error a device status word stands for (POD_OK for 0).
int pod_handle::status_error(int s) {
  if (s & (ST_NEIGH | ST_CELL)) return fail(POD_ENEIGH, "neighbour or cell capacity exceeded (status 0x%x)", s);
  if (s & ST_REV) return fail(POD_ENEIGH, "neighbour list is not symmetric (status 0x%x)", s);
  if (s & ST_NONFINITE) return fail(POD_ENONFINITE, "non-finite positions or results");
  if (s & ST_RANGE) return fail(POD_ERANGE, "a pair is closer than r_in");
  if (s & ST_OVERFLOW)
    return fail(POD_ERANGE, "a force, atom energy or virial exceeds the fixed-point range of the mixed path");
  if (s & ST_TIMEOUT) return fail(POD_ECUDA, "a bounded wait inside a kernel ran out (status 0x%x)", s);
  return POD_OK;
}

int pod_handle::plan_single(int N, const double box[3], const int pbc[3], Plan& pl) {
  const double rc = rlist();
  pl.N = N;
  double vol = 1.0;
  long long ncells = 1;
  for (int d = 0; d < 3; ++d) {
    CellGrid& cg = pl.cg;
    cg.pbc[d] = pbc[d] ? 1 : 0;
    double L = box[d];
    if (pbc[d] && !(L > 0)) return fail(POD_EINVAL, "periodic direction %d needs a positive box length", d);
    if (!(L >= 0) || !std::isfinite(L)) return fail(POD_EINVAL, "box length %d is not finite", d);
    cg.L[d] = L;
    cg.Lf[d] = (float)L;
    cg.Ll[d] = (float)(L - (double)cg.Lf[d]);
    int nc = L > 0 ? (int)std::floor(L / (rc * (1.0 + 1e-9))) : 1;
    nc = std::max(1, std::min(nc, 1024));
    cg.nc[d] = nc;
    const double cs = L > 0 ? L / nc : 0.0;
    cg.inv_cs[d] = L > 0 ? nc / L : 0.0;
    if (pbc[d])
      cg.S[d] = (int)std::ceil(rc / cs * (1.0 + 1e-12));
    else
      cg.S[d] = nc > 1 ? 1 : 0;
    if (pbc[d] && cg.S[d] > 60) return fail(POD_EINVAL, "box length %d too small for r_cut", d);
    ncells *= nc;
    vol *= std::max(L, rc);
  }
  // keep the cell count modest for sparse systems
  while (ncells > 8LL * N + 64) {
    int dmax = 0;
    for (int d = 1; d < 3; ++d)
      if (pl.cg.nc[d] > pl.cg.nc[dmax]) dmax = d;
    CellGrid& cg = pl.cg;
    ncells /= cg.nc[dmax];
    cg.nc[dmax] = std::max(1, cg.nc[dmax] / 2);
    ncells *= cg.nc[dmax];
    const double cs = cg.L[dmax] / cg.nc[dmax];
    cg.inv_cs[dmax] = cg.nc[dmax] / cg.L[dmax];
    cg.S[dmax] = cg.pbc[dmax] ? (int)std::ceil(rc / cs * (1.0 + 1e-12)) : (cg.nc[dmax] > 1 ? 1 : 0);
  }
  pl.cg.ncells = (int)ncells;
  // cell capacity: mean occupancy plus four standard deviations of a Poisson count
  // plus a margin (a fuller cell is reported and the call retried with twice it);
  // it sizes the neighbour search's shared memory, so it is kept tight
  const double expect_cell = (double)N / ncells;
  int capc = (int)(expect_cell + 4.0 * std::sqrt(expect_cell) + 8.0);
  capc = (capc + 7) / 8 * 8;
  pl.cg.cap = std::max(capc, cap_cell);
  const double expect = N / vol * (4.0 / 3.0) * M_PI * rc * rc * rc;
  int cap = (int)(1.5 * expect + 16);
  cap = (cap + 7) / 8 * 8;
  pl.cap = std::max(std::max(cap, 16), cap_nbr);
  return POD_OK;
}

int pod_handle::plan_batch(const pod_system* sys, Plan& pl) {
  fit_graph_drop();  // the batch layout buffers below change under a recorded fit
  const int nc = sys->n_configs;
  const double rc = rlist();
  pl.N = sys->n_atoms;
  pl.batched = true;
  pl.n_cfg = nc;
  pl.Lmax = rc;
  pl.Smax = 0;
  h_cbox.assign(nc, CfgBox{});
  h_cfg_of.assign(pl.N, 0);
  double max_expect = 0;
  if (sys->atom_offs[0] != 0 || sys->atom_offs[nc] != pl.N) return fail(POD_EINVAL, "atom_offs must run from 0 to n_atoms");
  for (int c = 0; c < nc; ++c) {
    CfgBox& b = h_cbox[c];
    b.a0 = sys->atom_offs[c];
    b.a1 = sys->atom_offs[c + 1];
    if (b.a1 < b.a0) return fail(POD_EINVAL, "atom_offs must be non-decreasing");
    double vol = 1.0;
    for (int d = 0; d < 3; ++d) {
      const double L = sys->boxes[3 * c + d];
      const int pb = sys->pbcs ? sys->pbcs[3 * c + d] : sys->pbc[d];
      if (pb && !(L > 0)) return fail(POD_EINVAL, "configuration %d: periodic direction %d needs a positive box", c, d);
      if (!(L >= 0) || !std::isfinite(L)) return fail(POD_EINVAL, "configuration %d: box is not finite", c);
      b.L[d] = L;
      b.Lh[d] = (float)L;
      b.Ll[d] = (float)(L - (double)b.Lh[d]);
      b.pbc[d] = pb ? 1 : 0;
      b.S[d] = pb ? (int)std::ceil(rc / L * (1.0 + 1e-12)) : 0;
      if (b.S[d] > 60) return fail(POD_EINVAL, "configuration %d: box too small for r_cut", c);
      pl.Smax = std::max(pl.Smax, b.S[d]);
      pl.Lmax = std::max(pl.Lmax, L);
      vol *= std::max(L, rc);
    }
    // the batch search indexes an atom's candidates (images x atoms) with 32-bit ints
    const long long ncand =
        (long long)(2 * b.S[0] + 1) * (2 * b.S[1] + 1) * (2 * b.S[2] + 1) * (long long)(b.a1 - b.a0);
    if (ncand > (1LL << 31) - 64)
      return fail(POD_EINVAL, "configuration %d: %lld periodic-image candidates per atom, more than 2^31", c, ncand);
    for (int i = b.a0; i < b.a1; ++i) h_cfg_of[i] = c;
    max_expect = std::max(max_expect, (b.a1 - b.a0) / vol * (4.0 / 3.0) * M_PI * rc * rc * rc);
  }
  int cap = (int)(1.5 * max_expect + 16);
  cap = (cap + 7) / 8 * 8;
  pl.cap = std::max(std::max(cap, 16), cap_nbr);
  int rc_;
  if ((rc_ = ensure(boxes, sizeof(CfgBox) * (size_t)nc, "configuration boxes"))) return rc_;
  if ((rc_ = ensure(cfg_of, sizeof(int) * (size_t)pl.N, "configuration index"))) return rc_;
  cudaError_t e = cudaMemcpy(boxes.p, h_cbox.data(), sizeof(CfgBox) * (size_t)nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(cfg_of.p, h_cfg_of.data(), sizeof(int) * (size_t)pl.N, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch upload");
  return POD_OK;
}

int pod_handle::size_class(int N) {
  int c = 0;
  while ((2LL << c) <= N) ++c;
  return c;
}

int pod_handle::plan(const pod_system* sys, Plan& pl) {
  const int rc_ = sys->n_configs > 1 ? plan_batch(sys, pl) : plan_single(sys->n_atoms, sys->box, sys->pbc, pl);
  auto it = tuned.find(size_class(sys->n_atoms));
  pl.shape = it != tuned.end() ? it->second : LaunchShape{};
  return rc_;
}

int pod_handle::build_neighbors(const double* pos, Plan& pl, bool need_rev, cudaStream_t st,
                                unsigned long long* facc_zero, float4* pd, bool pad, bool* wrote_pd) {
  pd_ok = false;  // a new list makes any earlier displacement rows stale
  if (wrote_pd) *wrote_pd = false;
  const int N = pl.N;
  int rc_;
  reuse_ok = false;
  if (!pl.batched) {
    const void* before = cell_count.p;
    if ((rc_ = ensure(cell_count, sizeof(int) * (size_t)pl.cg.ncells, "cell counts"))) return rc_;
    if (cell_count.p != before) cells_clean = 0;  // a new buffer holds no known zeros
    if ((rc_ = ensure(cell_atoms, sizeof(float4) * (size_t)pl.cg.ncells * pl.cg.cap, "cell slots"))) return rc_;
  }
  if ((rc_ = ensure(wpos, sizeof(double) * 3 * (size_t)N, "wrapped positions"))) return rc_;
  if ((rc_ = ensure(phi, sizeof(float4) * (size_t)N, "positions hi"))) return rc_;
  if ((rc_ = ensure(plo, sizeof(float4) * (size_t)N, "positions lo"))) return rc_;
  if ((rc_ = ensure(nbr_count, sizeof(int) * (size_t)N, "neighbour counts"))) return rc_;
  if ((rc_ = ensure(nbr_j, sizeof(int) * (size_t)N * pl.cap, "neighbour list"))) return rc_;
  if ((rc_ = ensure(nbr_s, sizeof(int) * (size_t)N * pl.cap, "neighbour shifts"))) return rc_;
  if (!status.p) {
    // the status word accumulates device conditions until read_status() reads and clears it
    if ((rc_ = ensure(status, sizeof(int) * 4, "status"))) return rc_;
    cudaError_t e0 = cudaMemset(status.p, 0, sizeof(int) * 4);
    if (e0 != cudaSuccess) return cuda_fail(e0, "status init");
  }
  cudaError_t e;
  if (pl.batched) {
    e = launch_batch_wrap(N, pos, (const int*)cfg_of.p, (const CfgBox*)boxes.p, (double*)wpos.p, (float4*)phi.p,
                          (float4*)plo.p, (int*)status.p, st, facc_zero);
    if (e != cudaSuccess) return cuda_fail(e, "batch wrap kernel");
    e = launch_batch_neigh(N, (const int*)cfg_of.p, (const CfgBox*)boxes.p, (const double*)wpos.p,
                           (const float4*)phi.p, rlist(), pl.Lmax, pl.Smax, pl.cap, (int*)nbr_count.p,
                           (int*)nbr_j.p, (int*)nbr_s.p, (int*)status.p, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch neighbour kernel");
  } else {
  if (cells_clean < pl.cg.ncells) {  // the previous call's clear did not cover these counts
    e = cudaMemsetAsync(cell_count.p, 0, sizeof(int) * (size_t)pl.cg.ncells, st);
    if (e != cudaSuccess) return cuda_fail(e, "cell count clear");
  }
  cells_clean = 0;  // binning fills them; the caller's clear restores the invariant
  last_ncells = pl.cg.ncells;
  if ((rc_ = ensure(wrapk, sizeof(int) * 3 * (size_t)N, "wrap offsets"))) return rc_;
  e = launch_bin(N, pos, pl.cg, (double*)wpos.p, (float4*)phi.p, (float4*)plo.p, (int*)cell_count.p,
                 (float4*)cell_atoms.p, (int*)status.p, st, (int*)wrapk.p, facc_zero, (int*)nbr_count.p, bin_csrc,
                 bin_cdst, bin_cn);
  if (bin_cn > 0) bin_cdone = true;
  if (e != cudaSuccess) return cuda_fail(e, "bin kernel");
  e = launch_neigh(N, pl.cg, (const double*)wpos.p, (const float4*)phi.p, (const float4*)plo.p,
                   (const int*)cell_count.p, (const float4*)cell_atoms.p, rlist(), pl.cap, (int*)nbr_count.p,
                   (int*)nbr_j.p, (int*)nbr_s.p, (int*)status.p, st, pl.shape.neigh_wpb, pd, pad || need_rev,
                   wrote_pd, neigh_blockwide(pl, N));
  if (e != cudaSuccess) return cuda_fail(e, "neighbour kernel");
  }
  if (need_rev) {
    if ((rc_ = ensure(rev, sizeof(int) * (size_t)N * pl.cap, "reverse index"))) return rc_;
    e = launch_rev(N, pl.cap, (const int*)nbr_count.p, (const int*)nbr_j.p, (const int*)nbr_s.p, (int*)rev.p,
                   (int*)status.p, st);
    if (e != cudaSuccess) return cuda_fail(e, "reverse-index kernel");
  }
  return POD_OK;
}

// Restores the zero cell counts after a call that binned (memset on the stream).
int pod_handle::clear_cells(const Plan& pl, cudaStream_t st) {
  if (pl.batched || !cell_count.p) return POD_OK;
  cudaError_t e = cudaMemsetAsync(cell_count.p, 0, sizeof(int) * (size_t)pl.cg.ncells, st);
  if (e != cudaSuccess) return cuda_fail(e, "cell count clear");
  cells_clean = pl.cg.ncells;
  return POD_OK;
}

template <typename T>
void pod_handle::fill_args(AtomArgs<T>& a, const Plan& pl) {
  std::memset(&a, 0, sizeof(a));
  a.N = pl.N;
  a.n_eval = n_eval_cur > 0 ? n_eval_cur : pl.N;
  a.cap = pl.cap;
  a.nbr_count = (const int*)nbr_count.p;
  a.nbr_j = (const int*)nbr_j.p;
  a.nbr_s = (const int*)nbr_s.p;
  a.wpos = (const double*)wpos.p;
  a.phi = (const float4*)phi.p;
  a.plo = (const float4*)plo.p;
  for (int d = 0; d < 3; ++d) {
    a.L[d] = pl.cg.L[d];
    a.Lh[d] = (float)pl.cg.L[d];
    a.Ll[d] = (float)(pl.cg.L[d] - (double)a.Lh[d]);
  }
  a.K = K;
  a.K2 = P.K2;
  a.K3 = P.K3;
  a.K4 = P.K4;
  a.P3 = P.P3;
  a.P4 = P.P4;
  a.KA4 = KA4;
  a.M = M;
  a.excl3 = excl3;
  a.col3 = 1 + P.K2;
  a.col4 = a.col3 + P.K3 * (P.P3 + 1);
  a.status = (int*)status.p;
  a.cfg_of = pl.batched ? (const int*)cfg_of.p : nullptr;
  a.cbox = pl.batched ? (const CfgBox*)boxes.p : nullptr;
  a.vdir = vdir_cur;
  a.rmask = mask_radius<T>(skin > 0 ? P.r_cut : 0.0);
  a.wpb = pl.shape.atom_wpb;
  a.keep_rp = pl.shape.atom_rp;
}

// Cubic Hermite pieces of R_k on TAB_N equal intervals of (r_in, r_cut), from
// FP64 values and derivatives of the snapshot projection at the nodes (the first
// node is taken 1e-4 h inside the interval, where phi has its removable 0/0).
// Built once per handle on the host (h_tab) and uploaded on first use.
void pod_handle::build_table_host() {
  if (!h_tab.empty()) return;
  const int n = TAB_N;
  const double h = (P.r_cut - P.r_in) / n;
  std::vector<double> R((size_t)(n + 1) * K), dR((size_t)(n + 1) * K), phi(Ns), dphi(Ns);
  for (int g = 0; g <= n; ++g) {
    double r = P.r_in + g * h;
    if (g == 0) r += 1e-4 * h;
    host_snapshots_d(P, r, phi.data(), dphi.data());
    for (int k = 0; k < K; ++k) {
      double a = 0, b = 0;
      for (int l = 0; l < Ns; ++l) {
        a += Q[(size_t)l * K + k] * phi[l];
        b += Q[(size_t)l * K + k] * dphi[l];
      }
      R[(size_t)g * K + k] = a;
      dR[(size_t)g * K + k] = b;
    }
  }
  std::vector<Q4<float>> tab((size_t)n * K);
  for (int g = 0; g < n; ++g)
    for (int k = 0; k < K; ++k) {
      const double f0 = R[(size_t)g * K + k], f1 = R[(size_t)(g + 1) * K + k];
      const double d0 = h * dR[(size_t)g * K + k], d1 = h * dR[(size_t)(g + 1) * K + k];
      Q4<float>& q = tab[(size_t)g * K + k];
      q.x = (float)f0;
      q.y = (float)d0;
      q.z = (float)(3.0 * (f1 - f0) - 2.0 * d0 - d1);
      q.w = (float)(2.0 * (f0 - f1) + d0 + d1);
    }
  h_tab.swap(tab);
}

int pod_handle::ensure_table(cudaStream_t st) {
  if (tab_ready) return POD_OK;
  build_table_host();
  int rc_;
  if ((rc_ = ensure(rtab, sizeof(Q4<float>) * h_tab.size(), "radial table"))) return rc_;
  cudaError_t e = cudaMemcpy(rtab.p, h_tab.data(), sizeof(Q4<float>) * h_tab.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "radial table upload");
  (void)st;
  tab_ready = true;
  return POD_OK;
}

// Whether the linear mixed path runs its adjoint pair pass as a kernel of its own
// (warp per atom, lane per pair) after a forward-only atom kernel, instead of
// inside the fused kernel: the option when set, else the launch shape, else by
// size -- small systems, where the fused kernel is one latency-bound wave.
bool pod_handle::split_adjoint(const Plan& pl) const {
  if (adj_force >= 0) return adj_force == 1;
  if (pl.shape.atom_split >= 0) return pl.shape.atom_split == 1;
  return false;  // the fused pass measured faster at every size tried
}

// Candidate tests of the block-per-cell neighbour search: block-wide (every
// thread of the block over candidates x own atoms) or a warp per own atom; the
// option when set, the launch shape when tuned, else block-wide for small systems (fewer cells than
// SMs' worth of warps per atom) and a warp per atom for large ones.
bool pod_handle::neigh_blockwide(const Plan& pl, int N) const {
  if (neigh_force >= 0) return neigh_force == 1;
  if (pl.shape.neigh_blockwide >= 0) return pl.shape.neigh_blockwide == 1;
  return neigh_blockwide_default(N);
}

int pod_handle::run_atoms(int mode, const Plan& pl, double* D, const double* c, double* Ei_dst, cudaStream_t st) {
  cudaError_t e;
  const bool has4 = P.P4 >= 0;
  if (precision == POD_MIXED) {
    AtomArgs<float> a;
    fill_args(a, pl);
    a.rad = rad32;
    if (radial_mode == 0) {
      int rc_ = ensure_table(st);
      if (rc_) return rc_;
      a.rad.tab = (const Q4<float>*)rtab.p;
      a.rad.tab_inv_h = (float)(TAB_N / (P.r_cut - P.r_in));
      a.rad.tab_n = TAB_N;
    }
    a.D = D;
    a.c = c;
    a.Ei = Ei_dst;
    a.g = nullptr;
    // displacement rows: energy modes only, of the list built by this call
    a.pd = (pd_ok && (mode == 1 || mode == 4 || mode == 5)) ? (const float4*)pdisp.p : nullptr;
    a.facc = (unsigned long long*)facc.p;
    a.qbeta = (const float*)qS32.p;
    a.emb_a = (const double*)embW.p;
    a.emb_alpha = (const double*)embW.p + M;
    a.emb_deg = emb_deg;
    a.wpart = (double*)wpart.p;
    a.gdm = (float*)gdm.p;
    a.q0 = dm_q0;
    a.q1 = dm_q1;
    if (mode == 3) a.keep_rp = 1;  // the design pass reads R, R' of every pair once per descriptor index
    const bool split = mode == 1 && split_adjoint(pl);
    if (split) {
      const int nap = ((PA + 1) * (PA + 2) * (PA + 3) / 6 + 3) / 4 * 4;
      const size_t rows = (size_t)a.n_eval * K;
      int rc_ = ensure(adjb, sizeof(float) * rows * (nap + 1), "atom adjoints");
      if (rc_) return rc_;
      a.adj_out = (float*)adjb.p;
      a.s3_out = (float*)adjb.p + rows * nap;
      a.keep_rp = 0;  // the forward-only kernel needs no R'
    }
    e = mode == 5 ? launch_atom_emb_f32(a, PA, has4, st) : launch_atom_f32(mode, a, PA, has4, st);
    if (e == cudaSuccess && split) e = launch_pair_adjoint_f32(a, PA, has4, st);
  } else {
    AtomArgs<double> a;
    fill_args(a, pl);
    a.rad = rad64;
    a.D = D;
    a.c = c;
    a.Ei = Ei_dst;
    a.g = (Q4<double>*)g.p;
    a.qbeta = (const double*)qS64.p;
    a.emb_a = (const double*)embW.p;
    a.emb_alpha = (const double*)embW.p + M;
    a.emb_deg = emb_deg;
    a.wpart = (double*)wpart.p;
    a.gdm = (double*)gdm.p;
    a.q0 = dm_q0;
    a.q1 = dm_q1;
    e = mode == 5 ? launch_atom_emb_f64(a, PA, has4, st) : launch_atom_f64(mode, a, PA, has4, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "atom kernel");
  return POD_OK;
}

int pod_handle::finish(cudaStream_t st, Plan& pl, bool& retry) {
  retry = false;
  if (!sync) return POD_OK;
  int rc_ = read_status(st);
  if (rc_ == POD_ENEIGH && (last_status & (ST_NEIGH | ST_CELL)) && retries < 4) {
    if (last_status & ST_NEIGH) cap_nbr = std::max(cap_nbr, pl.cap * 2);
    if (last_status & ST_CELL) cap_cell = std::max(cap_cell, pl.cg.cap * 2);
    ++retries;
    retry = true;
    err.clear();
    return POD_OK;
  }
  return rc_;
}

int pod_handle::validate_system(const pod_system* sys) {
  if (!sys) return fail(POD_EINVAL, "system is NULL");
  if (sys->n_atoms < 1) return fail(POD_EINVAL, "n_atoms must be >= 1");
  if (!sys->pos) return fail(POD_EINVAL, "positions are NULL");
  if (sys->n_configs > 1 && (!sys->atom_offs || !sys->boxes))
    return fail(POD_EINVAL, "a batch needs atom_offs and boxes");
  if (sys->n_local < 0 || sys->n_local > sys->n_atoms) return fail(POD_EINVAL, "n_local must be in [0, n_atoms]");
  if (device >= 0) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != device)
      return fail(POD_EINVAL, "the handle was created on device %d but device %d is current", device, cur);
  }
  return POD_OK;
}

int pod_handle::energy_forces(const pod_system* sys, const double* c, double* E, double* Ei_user, double* F,
                              double* W, cudaStream_t st) {
  int rc_ = validate_system(sys);
  if (rc_) return rc_;
  if (!c || !E) return fail(POD_EINVAL, "c and E are required");
  const int N = sys->n_atoms;
  retries = 0;
  for (;;) {
    Plan pl;
    if ((rc_ = plan(sys, pl))) return rc_;
    if (pl.batched && W) return fail(POD_EINVAL, "the virial is not available for batches of configurations");
    if (excl3 && (quad || emb_deg > 0))
      return fail(POD_EINVAL, "the quadratic and embedding models take the fast POD descriptor set");
    if (pl.batched && sys->n_local > 0 && sys->n_local != N)
      return fail(POD_EINVAL, "local and ghost atoms apply to a single configuration");
    // atoms [0, n_eval) carry energy terms; the rest are ghosts that receive forces
    const int n_eval = (sys->n_local > 0 && sys->n_local < N) ? sys->n_local : N;
    if ((rc_ = mark(0, st))) return rc_;
    const bool reuse = nbr_mode == 1 && reuse_ok && !pl.batched && last_pl.N == N && last_pl.cg.L[0] == pl.cg.L[0] &&
                       last_pl.cg.L[1] == pl.cg.L[1] && last_pl.cg.L[2] == pl.cg.L[2];
    // FP32 path: forces accumulate in fixed point, zeroed by this call's wrap
    // kernel; FP64 path: pair gradients per slot and the gather
    const bool fixp = precision == POD_MIXED;
    if (fixp && (rc_ = ensure(facc, sizeof(unsigned long long) * (4 * (size_t)N + FACC_TAIL), "force accumulators")))
      return rc_;
    unsigned long long* fa = fixp ? (unsigned long long*)facc.p : nullptr;
    if (reuse) {
      pl = last_pl;
      cudaError_t ew = launch_rewrap(N, sys->pos, (const int*)wrapk.p, pl.cg.L, (double*)wpos.p, (float4*)phi.p,
                                     (float4*)plo.p, (int*)status.p, st, fa);
      if (ew != cudaSuccess) return cuda_fail(ew, "rewrap kernel");
    } else {
      // the FP64 gather searches the reverse slots; when the list may be reused
      // (a skin, or reuse switched on) it also stores them for the reusing steps.
      // The mixed path rebuilding every call takes each pair's displacement from
      // the neighbour search (rows without sentinel padding; not kept for reuse).
      const bool want_pd = fixp && !pl.batched && skin == 0.0 && nbr_mode == 0;
      if (want_pd && (rc_ = ensure(pdisp, sizeof(float4) * (size_t)N * pl.cap, "pair displacements"))) return rc_;
      if ((rc_ = build_neighbors(sys->pos, pl, false, st, fa, want_pd ? (float4*)pdisp.p : nullptr, !want_pd,
                                 &pd_ok)))
        return rc_;
    }
    if (reuse) pd_ok = false;
    const bool keep_rev = !fixp && !reuse && !pl.batched && (skin > 0 || nbr_mode == 1);
    if (keep_rev && (rc_ = ensure(rev, sizeof(int) * (size_t)N * pl.cap, "reverse index"))) return rc_;
    const int* rev_in = reuse ? (const int*)rev.p : nullptr;
    int* rev_out = keep_rev ? (int*)rev.p : nullptr;
    if (!fixp && (rc_ = ensure(g, sizeof(Q4<double>) * (size_t)N * pl.cap, "pair gradients"))) return rc_;
    const int nwarp = atom_warps(n_eval, K, pl.shape.atom_wpb);
    if (!fixp && (rc_ = ensure(wpart, sizeof(double) * 9 * (size_t)nwarp, "virial partials"))) return rc_;
    double* Ei_dst = Ei_user;
    if (!Ei_dst) {
      if ((rc_ = ensure(Ei, sizeof(double) * (size_t)N, "atom energies"))) return rc_;
      Ei_dst = (double*)Ei.p;
    }
    const int nblk = fixp ? finalize_blocks(N) : gather_blocks(N, pl.shape.gather_wpb, pl.shape.gather_bps);
    if ((rc_ = ensure(Wat, sizeof(double) * 10 * (size_t)nblk, "block partial sums"))) return rc_;
    if (!offs.p) {
      if ((rc_ = ensure(offs, sizeof(unsigned) * 4, "ticket"))) return rc_;
      cudaError_t e0 = cudaMemset(offs.p, 0, sizeof(unsigned) * 4);
      if (e0 != cudaSuccess) return cuda_fail(e0, "ticket init");
    }
    if ((rc_ = mark(1, st))) return rc_;
    if (n_eval < N) {  // ghost atoms have no energy of their own
      cudaError_t ez = cudaMemsetAsync(Ei_dst + n_eval, 0, sizeof(double) * (size_t)(N - n_eval), st);
      if (ez != cudaSuccess) return cuda_fail(ez, "ghost atom energies");
    }
    n_eval_cur = n_eval;
    const bool pd_used = pd_ok;
    rc_ = run_atoms(quad ? 4 : (emb_deg > 0 ? 5 : 1), pl, nullptr, c, Ei_dst, st);
    n_eval_cur = 0;
    pd_ok = false;
    if (rc_) return rc_;
    if ((rc_ = mark(2, st))) return rc_;
    cudaError_t e;
    const bool clear_in_finalize = fixp && !pl.batched && cell_count.p && !reuse;
    if (fixp) {
      // the finalize is this step's last kernel when it clears the cell counts
      int* sout = (clear_in_finalize && fin_status_out) ? fin_status_out : nullptr;
      e = launch_finalize(N, fa, F, 1.0, nblk, E, W, st, clear_in_finalize ? (int*)cell_count.p : nullptr,
                          pl.cg.ncells, (int*)status.p, sout);
      if (sout) fin_status_done = true;
    } else {
      e = launch_gather_reduce<double>(N, n_eval, pl.cap, (const int*)nbr_count.p, (const int*)nbr_j.p,
                                       (const int*)nbr_s.p, rev_in, rev_out, (const Q4<double>*)g.p, Ei_dst,
                                       (const double*)wpart.p, nwarp, F, 1.0, (double*)Wat.p, nblk,
                                       (unsigned*)offs.p, E, W, (int*)status.p, st, pl.shape.gather_wpb);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gather kernel");
    if (clear_in_finalize)
      cells_clean = pl.cg.ncells;
    else if (!reuse && (rc_ = clear_cells(pl, st)))
      return rc_;
    if (pl.batched) {  // per-configuration energies (the gather wrote the batch total into E[0])
      e = launch_segsum(pl.n_cfg, (const CfgBox*)boxes.p, Ei_dst, 1.0, 0, E, st);
      if (e != cudaSuccess) return cuda_fail(e, "per-configuration energy");
    }
    if ((rc_ = mark(3, st))) return rc_;
    if ((rc_ = mark(4, st))) return rc_;
    if ((rc_ = timing_collect())) return rc_;
    bool retry;
    if ((rc_ = finish(st, pl, retry))) return rc_;
    if (!retry) {
      // a list can be reused (FP64 path: once its reverse slots are stored)
      if (!pl.batched && (fixp || reuse || rev_out) && !pd_used) {
        last_pl = pl;
        reuse_ok = true;
      }
      return POD_OK;
    }
  }
}

// One velocity-Verlet step: v += F dt / 2m, x += v dt, F <- F(x), v += F dt / 2m.
// Units: mass in amu, dt in fs, forces in eV/A (1 eV/(A amu) = 9.648533212e-3 A/fs^2).
int pod_handle::md_step(const pod_system* sys, double* pos, double* v, double* F, const double* c, double mass,
                        double dt, double* E, cudaStream_t st) {
  if (sys && sys->n_local > 0 && sys->n_local != sys->n_atoms)
    return fail(POD_EINVAL, "md_step integrates every atom: no ghost atoms");
  if (!sys || !pos || !v || !F || !c || !E) return fail(POD_EINVAL, "md_step: NULL argument");
  if (sys->n_configs > 1) return fail(POD_EINVAL, "md_step takes a single configuration");
  if (!(mass > 0) || !(dt > 0)) return fail(POD_EINVAL, "mass and dt must be positive");
  const int N3 = 3 * sys->n_atoms;
  const double h = 0.5 * dt * 9.648533212e-3 / mass;
  cudaError_t e = launch_kick(N3, v, F, h, pos, dt, st);
  if (e != cudaSuccess) return cuda_fail(e, "kick-drift kernel");
  pod_system s2 = *sys;
  s2.pos = pos;
  int rc_ = energy_forces(&s2, c, E, nullptr, F, nullptr, st);
  if (rc_) return rc_;
  e = launch_kick(N3, v, F, h, nullptr, dt, st);
  if (e != cudaSuccess) return cuda_fail(e, "kick kernel");
  return POD_OK;
}

int pod_handle::descriptors(const pod_system* sys, double* D, cudaStream_t st) {
  int rc_ = validate_system(sys);
  if (rc_) return rc_;
  if (!D) return fail(POD_EINVAL, "D is NULL");
  retries = 0;
  for (;;) {
    Plan pl;
    if ((rc_ = plan(sys, pl))) return rc_;
    if ((rc_ = build_neighbors(sys->pos, pl, false, st))) return rc_;
    if ((rc_ = run_atoms(0, pl, D, nullptr, nullptr, st))) return rc_;
    if ((rc_ = clear_cells(pl, st))) return rc_;
    bool retry;
    if ((rc_ = finish(st, pl, retry))) return rc_;
    if (!retry) return POD_OK;
  }
}

int pod_handle::neighbors(const pod_system* sys, int cap_out, int* count, int* nbr_out, int* shift_out,
                          cudaStream_t st) {
  int rc_ = validate_system(sys);
  if (rc_) return rc_;
  if (cap_out < 1 || !count || !nbr_out || !shift_out) return fail(POD_EINVAL, "bad neighbour output arguments");
  retries = 0;
  for (;;) {
    Plan pl;
    if ((rc_ = plan(sys, pl))) return rc_;
    pl.cap = (std::max(pl.cap, cap_out) + 7) / 8 * 8;
    if ((rc_ = build_neighbors(sys->pos, pl, false, st))) return rc_;
    cudaError_t e = launch_export_neighbors(sys->n_atoms, pl.cap, (const int*)nbr_count.p, (const int*)nbr_j.p,
                                            (const int*)nbr_s.p, cap_out, count, nbr_out, shift_out, st);
    if (e != cudaSuccess) return cuda_fail(e, "neighbour export");
    if ((rc_ = clear_cells(pl, st))) return rc_;
    bool retry;
    if ((rc_ = finish(st, pl, retry))) return rc_;
    if (!retry) break;
  }
  return POD_OK;
}

// Global descriptors G_m = sum_i D_im per configuration (Eq. 58a), or with vdir
// their directional derivative sum_k dG_m/dr_k . v_k (tangent mode).
// Chunk table of the per-configuration column sums: <= 256 rows per chunk,
// chunks never cross a configuration (rows: [nch][2], then configuration chunk
// offsets [n_cfg + 1]; nrows2 = 2 nch).
int pod_handle::colsum_table(const Plan& pl, int& nch, int& nrows2) {
  std::vector<int> rows, cfgc;
  const int ncfg = pl.batched ? pl.n_cfg : 1;
  cfgc.push_back(0);
  for (int c = 0; c < ncfg; ++c) {
    const int a0 = pl.batched ? h_cbox[c].a0 : 0, a1 = pl.batched ? h_cbox[c].a1 : pl.N;
    for (int r = a0; r < a1; r += 256) {
      rows.push_back(r);
      rows.push_back(std::min(a1, r + 256));
    }
    cfgc.push_back((int)rows.size() / 2);
  }
  nch = (int)rows.size() / 2;
  nrows2 = (int)rows.size();
  int rc_;
  if ((rc_ = ensure(chunks, sizeof(int) * (rows.size() + cfgc.size()), "chunk table"))) return rc_;
  if ((rc_ = ensure(cpart, sizeof(double) * (size_t)std::max(nch, 1) * M, "column partials"))) return rc_;
  cudaError_t e = cudaMemcpy(chunks.p, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy((int*)chunks.p + rows.size(), cfgc.data(), sizeof(int) * cfgc.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "chunk table upload");
  return POD_OK;
}

int pod_handle::global_desc(const pod_system* sys, const double* vdir, double* Gout, cudaStream_t st,
                            double* per_atom) {
  int rc_ = validate_system(sys);
  if (rc_) return rc_;
  if (!Gout && !per_atom) return fail(POD_EINVAL, "output is NULL");
  if (vdir && excl3) return fail(POD_EINVAL, "the descriptor tangent takes the fast POD descriptor set");
  const int N = sys->n_atoms;
  retries = 0;
  for (;;) {
    Plan pl;
    if ((rc_ = plan(sys, pl))) return rc_;
    if ((rc_ = build_neighbors(sys->pos, pl, false, st))) return rc_;
    double* rows = per_atom;  // per-atom rows to the caller, or to the workspace for the sums
    if (!rows) {
      if ((rc_ = ensure(Dws, sizeof(double) * (size_t)N * M, "descriptor workspace"))) return rc_;
      rows = (double*)Dws.p;
    }
    vdir_cur = vdir;
    rc_ = run_atoms(vdir ? 2 : 0, pl, rows, nullptr, nullptr, st);
    vdir_cur = nullptr;
    if (rc_) return rc_;
    if ((rc_ = clear_cells(pl, st))) return rc_;
    if (Gout) {
      int nch = 0, nrows2 = 0;
      if ((rc_ = colsum_table(pl, nch, nrows2))) return rc_;
      const int ncfg = pl.batched ? pl.n_cfg : 1;
      cudaError_t e = launch_colsum(nch, (const int*)chunks.p, ncfg, (const int*)chunks.p + nrows2, M,
                                    (const double*)rows, (double*)cpart.p, Gout, st);
      if (e != cudaSuccess) return cuda_fail(e, "column sums");
    }
    bool retry;
    if ((rc_ = finish(st, pl, retry))) return rc_;
    if (!retry) return POD_OK;
  }
}

extern "C" {

int pod_global_descriptors(pod_handle* h, const pod_system* sys, double* G, void* stream) {
  NvtxRange nvtx_("pod_global_descriptors");
  if (!h) return POD_EINVAL;
  return h->global_desc(sys, nullptr, G, (cudaStream_t)stream);
}

int pod_descriptors_jvp(pod_handle* h, const pod_system* sys, const double* v, double* Gdot, void* stream) {
  NvtxRange nvtx_("pod_descriptors_jvp");
  if (!h) return POD_EINVAL;
  if (!v) return h->fail(POD_EINVAL, "direction v is NULL");
  return h->global_desc(sys, v, Gdot, (cudaStream_t)stream);
}

int pod_neighbors(pod_handle* h, const pod_system* sys, int cap, int* count, int* nbr, int* shift, void* stream) {
  NvtxRange nvtx_("pod_neighbors");
  if (!h) return POD_EINVAL;
  int rc = h->neighbors(sys, cap, count, nbr, shift, (cudaStream_t)stream);
  if (rc == POD_OK && h->sync) {
    // report atoms with more neighbours than the caller's capacity
    std::vector<int> hc(sys->n_atoms);
    cudaError_t e = cudaMemcpy(hc.data(), count, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return h->cuda_fail(e, "count read");
    for (int v : hc)
      if (v > cap) return h->fail(POD_ENEIGH, "an atom has %d neighbours, more than cap = %d", v, cap);
  }
  return rc;
}

int pod_descriptors(pod_handle* h, const pod_system* sys, double* D, void* stream) {
  NvtxRange nvtx_("pod_descriptors");
  if (!h) return POD_EINVAL;
  return h->descriptors(sys, D, (cudaStream_t)stream);
}

int pod_energy_forces(pod_handle* h, const pod_system* sys, const double* c, double* E, double* Ei, double* F,
                      double* W, void* stream) {
  NvtxRange nvtx_("pod_energy_forces");
  if (!h) return POD_EINVAL;
  return h->energy_forces(sys, c, E, Ei, F, W, (cudaStream_t)stream);
}

namespace {
bool host_pinned(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}
// The device address of pinned host memory (NULL stays NULL); false when p is
// not pinned host memory mapped into the device's address space.
bool mapped_ptr(const void* p, void** d) {
  *d = nullptr;
  if (!p) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
  *d = a.devicePointer;
  return true;
}
}  // namespace

// Host-buffer energy and forces.  Copies in, one evaluation, copies out.  When
// calls repeat with the same (pinned) buffers, size, box and settings on a
// non-default stream, the second such call captures the step and a read of the
// status word into a CUDA graph (with the copies, or with the kernels reading
// and writing the pinned buffers directly: the mapped form above) and later
// calls replay it (one launch instead of one per kernel and copy); a status
// other than OK after a replay drops the graph and re-runs the call on the
// direct path (capacity retries, or the error).
int pod_energy_forces_host(pod_handle* h, const pod_system* sys, const double* c, double* E, double* Ei, double* F,
                           double* W, void* stream) {
  NvtxRange nvtx_("pod_energy_forces_host");
  if (!h) return POD_EINVAL;
  int rc = h->validate_system(sys);
  if (rc) return rc;
  if (!c || !E) return h->fail(POD_EINVAL, "c and E are required");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = sys->n_atoms;
  if ((rc = h->ensure(h->pos_in, sizeof(double) * 3 * (size_t)N, "staged positions"))) return rc;
  if ((rc = h->ensure(h->c_in, sizeof(double) * (size_t)h->M, "staged coefficients"))) return rc;
  if ((rc = h->ensure(h->E_out, sizeof(double) * 16, "staged energy"))) return rc;
  if (F && (rc = h->ensure(h->F_out, sizeof(double) * 3 * (size_t)N, "staged forces"))) return rc;
  if (W && (rc = h->ensure(h->W_out, sizeof(double) * 9, "staged virial"))) return rc;
  if (Ei && (rc = h->ensure(h->Ei_out, sizeof(double) * (size_t)N, "staged atom energies"))) return rc;
  pod_system dsys = *sys;
  dsys.pos = (const double*)h->pos_in.p;

  pod_handle::HostKey key{};
  key.ptr[0] = sys->pos;
  key.ptr[1] = c;
  key.ptr[2] = E;
  key.ptr[3] = Ei;
  key.ptr[4] = F;
  key.ptr[5] = W;
  key.N = N;
  for (int d = 0; d < 3; ++d) {
    key.pbc[d] = sys->pbc[d];
    key.box[d] = sys->box[d];
  }
  key.precision = h->precision;
  key.quad = h->quad ? 1 : 0;
  key.emb_deg = h->emb_deg;
  key.excl3 = h->excl3;
  key.n_local = sys->n_local;
  key.radial = h->radial_mode;
  key.tune_gen = h->tune_gen;
  const bool graphable = !h->hgraph_off && st != nullptr && !h->timing && h->nbr_mode == 0 && h->skin == 0 &&
                         sys->n_configs <= 1;

  auto enqueue_step = [&](int sync_mode) -> int {
    cudaError_t e = cudaMemcpyAsync(h->pos_in.p, sys->pos, sizeof(double) * 3 * (size_t)N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->c_in.p, c, sizeof(double) * h->M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return h->cuda_fail(e, "host-to-device copy");
    const int keep_sync = h->sync;
    h->sync = sync_mode;
    const int r = h->energy_forces(&dsys, (const double*)h->c_in.p, (double*)h->E_out.p,
                                   Ei ? (double*)h->Ei_out.p : nullptr, F ? (double*)h->F_out.p : nullptr,
                                   W ? (double*)h->W_out.p : nullptr, st);
    h->sync = keep_sync;
    if (r) return r;
    e = cudaMemcpyAsync(E, h->E_out.p, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && F) e = cudaMemcpyAsync(F, h->F_out.p, sizeof(double) * 3 * (size_t)N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && W) e = cudaMemcpyAsync(W, h->W_out.p, sizeof(double) * 9, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && Ei) e = cudaMemcpyAsync(Ei, h->Ei_out.p, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return h->cuda_fail(e, "device-to-host copy");
    return POD_OK;
  };

  if (graphable && h->hgraph && h->hkey_valid && h->hkey == key) {
    cudaError_t e = cudaSuccess;
    if (h->cells_clean < h->hgraph_ncells)  // another call left its cell counts behind
      e = cudaMemsetAsync(h->cell_count.p, 0, sizeof(int) * (size_t)h->hgraph_ncells, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(h->hgraph, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return h->cuda_fail(e, "host graph replay");
    h->cells_clean = h->hgraph_ncells;  // the replayed step clears what it binned
    if (*h->h_status == 0) return POD_OK;
    h->drop_host_graph();  // capacity overflow or an error: redo the call on the direct path
  }
  rc = enqueue_step(1);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return h->cuda_fail(e, "device-to-host copy");
  if (!graphable) return POD_OK;
  if (!(host_pinned(sys->pos) && host_pinned(c) && host_pinned(E) && host_pinned(Ei) && host_pinned(F) &&
        host_pinned(W))) {
    return POD_OK;
  }
  if (!(h->hkey_prev == key)) {  // capture on the second call with the same key
    h->hkey_prev = key;
    return POD_OK;
  }
  if (!h->h_status || !h->status.p) return POD_OK;
  // Mapped form (on Grace, pinned host memory is coherent with the GPU over
  // NVLink-C2C): the step reads the positions and writes E, Ei, F and W through
  // the pinned buffers' device addresses, and the bin kernel copies c, so the
  // graph holds no copy but the status word's.  Otherwise copies in and out.
  // The mixed path's finalize also hands over the status word (no copy node).
  void *pos_d = nullptr, *c_d = nullptr, *E_d = nullptr, *Ei_d = nullptr, *F_d = nullptr, *W_d = nullptr;
  void* hs_d = nullptr;
  const bool mapped = !h->host_mapped_off && (sys->n_local == 0 || sys->n_local == N) &&
                      mapped_ptr(sys->pos, &pos_d) && mapped_ptr(c, &c_d) && mapped_ptr(E, &E_d) &&
                      mapped_ptr(Ei, &Ei_d) && mapped_ptr(F, &F_d) && mapped_ptr(W, &W_d) &&
                      mapped_ptr(h->h_status, &hs_d);
  bool status_by_finalize = false;
  auto enqueue_mapped = [&]() -> int {
    pod_system msys = *sys;
    msys.pos = (const double*)pos_d;
    h->bin_csrc = (const double*)c_d;
    h->bin_cdst = (double*)h->c_in.p;
    h->bin_cn = h->M;
    h->bin_cdone = false;
    h->fin_status_out = (int*)hs_d;
    h->fin_status_done = false;
    const int keep_sync = h->sync;
    h->sync = 0;
    int r = h->energy_forces(&msys, (const double*)h->c_in.p, (double*)E_d, (double*)Ei_d, (double*)F_d,
                             (double*)W_d, st);
    h->sync = keep_sync;
    const bool copied = h->bin_cdone;
    status_by_finalize = h->fin_status_done;
    h->bin_csrc = nullptr;
    h->bin_cdst = nullptr;
    h->bin_cn = 0;
    h->bin_cdone = false;
    h->fin_status_out = nullptr;
    h->fin_status_done = false;
    if (r == POD_OK && !copied) r = POD_EINVAL;  // no bin kernel took the coefficients: not this form
    return r;
  };
  // capture: (copies in,) the asynchronous step, (copies out,) status word out and clear
  h->drop_host_graph();
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->hgraph_off = true;
    return POD_OK;
  }
  rc = mapped ? enqueue_mapped() : enqueue_step(0);
  cudaError_t ec = cudaSuccess;
  if (rc == POD_OK && !status_by_finalize) {
    ec = cudaMemcpyAsync(h->h_status, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ec == cudaSuccess) ec = cudaMemsetAsync(h->status.p, 0, sizeof(int), st);
  }
  cudaError_t ee = cudaStreamEndCapture(st, &g);
  if (rc != POD_OK || ec != cudaSuccess || ee != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    h->err.clear();
    h->hgraph_off = true;  // this handle stays on the direct path
    return POD_OK;
  }
  cudaGraphExec_t ex = nullptr;
  ee = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ee != cudaSuccess || !ex) {
    cudaGetLastError();
    h->hgraph_off = true;
    return POD_OK;
  }
  h->hgraph = ex;
  h->hkey = key;
  h->hkey_valid = true;
  h->hgraph_ncells = h->last_ncells;
  return POD_OK;
}

}  // extern "C"
