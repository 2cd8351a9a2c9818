// Library-internal handle definition.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <map>
#include <string>
#include <vector>

#include "../../include/pod.h"
#include "pod_common.cuh"
#include "pod_kernels.h"

// NVTX range over one ABI call (visible in Nsight Systems timelines; a no-op
// unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct HostParams {
  double r_in = 0, r_cut = 0;
  std::vector<double> alpha, beta, gamma;
  int K2 = 0, K3 = 0, K4 = 0, P3 = -1, P4 = -1;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Plan {
  int N = 0;
  int cap = 0;  // neighbour capacity per atom
  fastpod::CellGrid cg{};
  // batches of configurations (n_cfg > 1): per-atom configuration and boxes
  bool batched = false;
  int n_cfg = 1;
  double Lmax = 0;
  int Smax = 0;
  fastpod::LaunchShape shape{};  // launch shape for this system size (autotuned or default)
};

struct pod_handle {
  HostParams P;
  int precision = 0;
  int Ns = 0, K = 0, PA = 0, KA4 = 0, M = 0;
  std::vector<double> Q, eig;
  fastpod::RadialConst<float> rad32{};
  fastpod::RadialConst<double> rad64{};
  std::string err;
  int sync = 1;
  int device = -1;  // the device current at pod_create (its workspace lives there)
  int retries = 0;
  int last_status = 0;
  int cap_nbr = 0, cap_cell = 0;  // grown after overflows
  int* h_status = nullptr;        // pinned
  int timing = 0;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::map<int, fastpod::LaunchShape> tuned;  // autotuned launch shapes by size class (floor log2 N)
  std::map<int, fastpod::LaunchShape> tuned_fit;  // the fit's design-pass shapes by size class of the batch
  DevBuf tune_ref;  // zero labels for timing the fit's design pass
  int autotune_fit(const pod_system* sys, int reps, fastpod::LaunchShape& best, double ms[3]);
  int tune_gen = 0;                            // bumped by every autotune (invalidates host graphs)
  // host-buffer entry point: one CUDA graph (copies in, step, copies out, status)
  // replayed while calls repeat with the same buffers, sizes, box and settings
  struct HostKey {
    const void* ptr[6];
    int N, pbc[3], precision, quad, radial, tune_gen, emb_deg, excl3, n_local;
    double box[3];
    bool operator==(const HostKey& o) const;
  };
  HostKey hkey{}, hkey_prev{};
  bool hkey_valid = false, hgraph_off = false;
  bool host_mapped_off = false;  // POD_OPT_HOST_MAPPED = 0: the graph copies in and out
  size_t ws_limit = 0;           // POD_OPT_WORKSPACE_LIMIT_MB in bytes (0: no limit)
  // a copy that the next bin kernel performs (the mapped host graph's coefficients)
  const double* bin_csrc = nullptr;
  double* bin_cdst = nullptr;
  int bin_cn = 0;
  bool bin_cdone = false;
  // where the next finalize hands the status word (the mapped host graph's)
  int* fin_status_out = nullptr;
  bool fin_status_done = false;
  cudaGraphExec_t hgraph = nullptr;
  void drop_host_graph();
  static int size_class(int N);
  int autotune(const pod_system* sys, const double* c, int reps, cudaStream_t st, fastpod::LaunchShape& best,
               double ms[3]);
  double t_acc[4] = {0, 0, 0, 0};
  int t_calls = 0;
  int mark(int k, cudaStream_t st);
  int timing_collect();
  DevBuf cell_count, cell_atoms, wpos, phi, plo, nbr_count, nbr_j, nbr_s, rev, g, Ei, Wat, status, offs;
  DevBuf pos_in, c_in, E_out, F_out, W_out, Ei_out;       // host-buffer entry point staging
  DevBuf fitA, fitG, fitb, fitwork, cfg_of, boxes;        // fit
  DevBuf rtab;                                            // tabulated radial basis (mixed path)
  DevBuf wpart;                                           // virial partials
  static constexpr int TAB_N = 2048;
  int radial_mode = 0;  // mixed path: 0 = tabulated R_k, 1 = snapshots evaluated per pair
  bool tab_ready = false;
  std::vector<fastpod::Q4<float>> h_tab;  // the table's host copy ([TAB_N][K] cubic pieces)
  void build_table_host();
  int ensure_table(cudaStream_t st);
  unsigned long long uid = 0;  // unique per handle for the process lifetime (never reused)

  ~pod_handle();
  std::vector<DevBuf*> all_bufs();
  int fail(int code, const char* fmt, ...);
  int cuda_fail(cudaError_t e, const char* what);
  int ensure(DevBuf& b, size_t bytes, const char* what);
  int read_status(cudaStream_t st);
  int validate_system(const pod_system* sys);
  int plan_single(int N, const double box[3], const int pbc[3], Plan& pl);
  int plan_batch(const pod_system* sys, Plan& pl);
  int plan(const pod_system* sys, Plan& pl);
  std::vector<fastpod::CfgBox> h_cbox;
  std::vector<int> h_cfg_of;
  int fit(const pod_system* batch, const double* E_ref, const double* F_ref, const pod_fit_opts* opts,
          double* c_out, double* mae_E, double* mae_F);
  // neighbour lists with a skin, reused between rebuilds (single configurations)
  double skin = 0.0;
  int nbr_mode = 0;       // 0: rebuild every call, 1: reuse the last energy/force list
  bool reuse_ok = false;
  Plan last_pl;
  DevBuf wrapk;
  double rlist() const { return P.r_cut + skin; }
  int md_step(const pod_system* sys, double* pos, double* v, double* F, const double* c, double mass, double dt,
              double* E, cudaStream_t st);
  int global_desc(const pod_system* sys, const double* vdir, double* G, cudaStream_t st, double* per_atom = nullptr);
  const double* vdir_cur = nullptr;
  DevBuf Dws, chunks, cpart;
  DevBuf gdm, dmG;
  DevBuf facc;  // FP32 path: fixed-point force accumulators [N][4]
  DevBuf qS32, qS64;  // quadratic model: symmetric weights S = beta + beta^T (FP32 and FP64 copies)
  bool quad = false;
  DevBuf embW;        // embedding model: density weights a [M], then the polynomial alpha [deg + 1]
  int emb_deg = 0;    // 0: no embedding model
  int excl3 = 0;      // 1: three-body descriptors as the exclusive sums of Eq. 15b
  int n_eval_cur = 0; // energy calls: atoms evaluated (the system's n_local; 0 = all)  // fit: design-matrix pair gradients, per-configuration descriptor sums
  int dm_q0 = 0, dm_q1 = 0;  // fit: descriptor-index range of the current design pass
  int colsum_table(const Plan& pl, int& nch, int& nrows2);
  int fit_build(const pod_system* batch, const double* E_ref, const double* F_ref, const pod_fit_opts& o);
  int fit_gram(double gamma);
  int fit_gram_tc(double gamma, double* dG, double* dr, bool legacy_mma);
  int gram_mode = 0;  // exact slice products: 0 tcgen05, 2 mma.sync; 1: FP64 SYRK
  int fit_solve_dev();
  int fit_solve_qr(double gamma);
  DevBuf qrw;  // QR solve: factors of the row and merge stages
  DevBuf halo_cnt;  // pod_halo_select: count of the selected atoms
  DevBuf mgrad;     // pod_model_gradients: per-block partial sums, then the result
  int fit_residual_dev(double* sumE, double* sumF);
  // The plan of the last fit_build, from which its launches can be issued again
  // (fit_design_launch) and recorded into a CUDA graph.
  struct FitCtx {
    Plan pl;
    const double* pos = nullptr;
    const double* E_ref = nullptr;
    const double* F_ref = nullptr;
    pod_fit_opts o{};
    int qchunk = 1, nch = 0, nrows2 = 0;
    long long R = 0;
  } fctx;
  int fit_design_launch();
  int* fit_info_dev();
  int fit_solve_launch();
  int fit_qr_launch(double gamma);
  int fit_residual_launch();
  void fit_residual_sums(const double* res, double* sumE, double* sumF) const;
  cudaStream_t fit_st = nullptr;  // stream of the fit's launches: the legacy stream, or the recording stream
  bool fit_capturing = false;     // recording: no host synchronisation, no uploads
  // Recorded fit: repeated pod_fit calls with the same batch layout, buffers,
  // options and settings replay one CUDA graph of the whole device chain.
  cudaGraphExec_t fgraph = nullptr;
  cudaStream_t fcap_st = nullptr;
  std::vector<unsigned long long> fkey;
  void* fhost = nullptr;  // pinned: status, pivot status, residual sums, c
  int fit_replays = 0;    // fits served by a replay (pod_fit_replays)
  bool fit_off = false;   // POD_OPT_FIT_GRAPH = 0: no recording
  std::vector<unsigned long long> fit_key(const pod_system* b, const double* E_ref, const double* F_ref,
                                          const pod_fit_opts& o) const;
  int fit_record(const std::vector<unsigned long long>& key);
  int fit_replay(const pod_fit_opts& o, double* c_out, double* mae_E, double* mae_F, bool& redo);
  void fit_graph_drop();
  int status_error(int s);
  long long fit_R = 0;
  int fit_nc = 0, fit_N = 0;
  double fit_wE = 0, fit_wF = 0;
  int build_neighbors(const double* pos, Plan& pl, bool need_rev, cudaStream_t st,
                      unsigned long long* facc = nullptr, float4* pd = nullptr, bool pad = true,
                      bool* wrote_pd = nullptr);
  // Cell counts are zero between calls: each call that bins clears them again at
  // its end (the mixed energy path in its finalize kernel, the others with a
  // memset); cells_clean is the number of leading entries known to be zero
  // (0 after a binning whose clear has not been enqueued, or a new buffer).
  long long cells_clean = 0;
  long long last_ncells = 0;    // cells binned by the last single-configuration call
  long long hgraph_ncells = 0;  // cells binned by the captured host-buffer step
  int clear_cells(const Plan& pl, cudaStream_t st);
  DevBuf pdisp;        // mixed path: per-slot pair displacements from the neighbour search
  DevBuf adjb;         // mixed linear path, separate adjoint kernel: dE_i/dB [N][K][NAP], then dE_i/dS3 [N][K]
  int adj_force = -1;  // POD_OPT_ADJOINT: -1 launch shape / size, 0 fused, 1 separate kernel
  bool split_adjoint(const Plan& pl) const;
  bool neigh_blockwide(const Plan& pl, int N) const;
  int neigh_force = -1;  // POD_OPT_NEIGHBOR_TESTS: -1 launch shape / size, 0 warp per atom, 1 block-wide
  bool pd_ok = false;  // pdisp holds the current list's displacements (for the next atom-kernel launch)
  template <typename T>
  void fill_args(fastpod::AtomArgs<T>& a, const Plan& pl);
  int run_atoms(int mode, const Plan& pl, double* D, const double* c, double* Ei_dst, cudaStream_t st);
  int finish(cudaStream_t st, Plan& pl, bool& retry);
  int energy_forces(const pod_system* sys, const double* c, double* E, double* Ei, double* F, double* W,
                    cudaStream_t st);
  int descriptors(const pod_system* sys, double* D, cudaStream_t st);
  int neighbors(const pod_system* sys, int cap_out, int* count, int* nbr, int* shift, cudaStream_t st);
};

// Looks up (once per device, with that device current) the device address of
// the static scratch array of pod_descriptors_static; returns a cudaError_t.
int static_scratch_setup(int device);
