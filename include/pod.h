/*
 * fastpod -- C ABI of the GB300 (sm_103a) implementation of fast proper
 * orthogonal descriptors (N.-C. Nguyen, "Fast proper orthogonal descriptors for
 * many-body interatomic potentials", arXiv:2212.14446).
 *
 * The library computes, for every atom i of an atomic configuration,
 *   - the POD radial basis R_k(r) = sum_l Q_lk Phi_l(r) built from parametrized
 *     radial snapshots with a smooth cut-off              (Section 2.2, Eq. 3-12)
 *   - the atomic basis B_imnl = sum_j R_m(r_ij) A_nl(rhat_ij)     (Eq. 24b)
 *   - the inclusive 2-, 3- and 4-body descriptors via Eq. 12b, Eq. 26a,
 *     Eq. 27a and Eq. 30a (equal to the naive sums Eq. 15 / Eq. 18a)
 *   - the linear energy E_i = sum_m c_m D_im, E = sum_i E_i     (Eq. 57a, 58a)
 *   - forces F_k = -dE/dr_k and the virial by an adjoint of Eq. 24c / Eq. 26c
 *   - the ridge least-squares fit of Eq. 63a.
 *
 * Conventions common to every call
 *   - All lengths are in Angstrom; energies in the units of the coefficients c.
 *   - Positions are structure-of-arrays: pos[0..N) = x, pos[N..2N) = y,
 *     pos[2N..3N) = z (FP64).  Boxes are orthorhombic, [0, L_d) in periodic
 *     directions.  Forces use the same [3][N] layout.
 *   - Descriptor order per atom (M columns):
 *       [ 1 | D2_m (m < K2) | D3_mn (m < K3 major, n = 0..P3) |
 *         D4_mp (m < K4 major, p in the order of Table 1: degree ascending,
 *                then (a, b, c) lexicographically descending) ]
 *     with M = 1 + K2 + K3 (P3 + 1) + K4 K_a(P4)  (Table 6 caption).
 *   - Device pointers are CUDA device memory on the current device; the caller
 *     owns every buffer passed in.  The library owns the handle, Q, its tables
 *     and a workspace that grows on demand and is freed by pod_destroy.
 *   - Calls taking `stream` (a cudaStream_t, NULL = legacy default stream)
 *     enqueue their kernels on it.  With the synchronous-status option on (the
 *     default), each call waits for its stream at the end and turns device-side
 *     conditions into return codes; with it off, calls return as soon as the
 *     work is enqueued and pod_status() reports later.
 *   - Return value: POD_OK (0) or a negative POD_E* code; pod_last_error()
 *     gives the message.  No call throws or aborts; invalid arguments never
 *     reach a kernel.
 *   - A handle is not thread-safe; use one handle per host thread/stream.
 */
#ifndef FASTPOD_POD_H
#define FASTPOD_POD_H

#ifdef __cplusplus
extern "C" {
#endif

#define POD_OK 0
#define POD_EINVAL (-1)     /* bad parameter, NULL pointer, unsupported size      */
#define POD_ENOMEM (-2)     /* device or host allocation failed                   */
#define POD_ECUDA (-3)      /* a CUDA runtime call failed, or a bounded wait inside
                               a kernel ran out (the kernel stopped early)        */
#define POD_ERANGE (-4)     /* a pair closer than r_in (outside (r_in, r_cut)); on
                               the mixed path also a value outside its fixed-point
                               range: a pair gradient of 2^30 eV/A or more, an atom
                               energy of 2^21 eV or more, or a per-warp virial sum
                               of 2^26 eV or more                                   */
#define POD_ENONFINITE (-5) /* NaN/Inf in positions or results                    */
#define POD_ESINGULAR (-6)  /* fit: normal equations not positive definite        */
#define POD_ENEIGH (-7)     /* neighbour or cell capacity exceeded after retry    */
#define POD_EIO (-8)        /* a model file could not be read or written          */

#define POD_FP64 0  /* every step in FP64 (reference path)                        */
#define POD_MIXED 1 /* FP32 pair/contraction/adjoint, FP64 reductions and fit     */

typedef struct pod_handle pod_handle;

/* Hyper-parameters mu = (r_in, r_cut, alpha, beta, gamma) of Section 2.2 and
 * the radial/angular sizes of Sections 2.3-2.4.  The snapshot family is
 * phi(r; alpha_a, beta_b) for every pair (a, b) (alpha outer, beta inner),
 * followed by varphi(r; gamma_g) for every g, each times the cut-off f_c
 * (Eq. 6, Eq. 11); Ns = n_alpha * n_beta + n_gamma.  Arrays are copied. */
typedef struct {
  double r_in, r_cut;      /* 0 < r_in < r_cut                                  */
  int n_alpha;             /* 1..8                                              */
  const double* alpha;
  int n_beta;              /* 1..2, every beta > 0                              */
  const double* beta;
  int n_gamma;             /* 0..8                                              */
  const double* gamma;
  int K2, K3, K4;          /* radial modes per body order, 0..16, <= Ns         */
  int P3;                  /* three-body angular degree, -1 (none) .. 4         */
  int P4;                  /* four-body angular degree, -1 (none) .. 4          */
  int n_grid;              /* POD midpoint-grid points (0 -> 2000)              */
  int precision;           /* POD_FP64 or POD_MIXED                             */
  const double* Q;         /* optional Ns x K_r projection (row-major) used
                              instead of the library's own POD; NULL -> compute */
} pod_params;

/* One configuration (n_configs <= 1) or a batch of configurations stored back
 * to back (n_configs > 1, used by pod_fit and the batched calls). */
typedef struct {
  int n_atoms;             /* total atoms, >= 1                                 */
  const double* pos;       /* [3][n_atoms] SoA (device, or host for *_host)     */
  double box[3];           /* box lengths for a single configuration            */
  int pbc[3];              /* 1 = periodic, 0 = open                            */
  int n_configs;           /* 0 or 1: single configuration                      */
  const int* atom_offs;    /* HOST [n_configs + 1] atom offsets (batch only)    */
  const double* boxes;     /* HOST [n_configs][3] box lengths   (batch only)    */
  const int* pbcs;         /* HOST [n_configs][3] or NULL (= pbc for all)       */
  int n_local;             /* single configuration, pod_energy_forces(_host):
                              atoms [0, n_local) are local -- their energies E_i
                              and pair gradients are evaluated -- and atoms
                              [n_local, n_atoms) are ghosts (periodic or
                              neighbouring-domain copies) that only appear as
                              neighbours; forces are returned on every atom
                              (ghosts get the reactions of local atoms' terms)
                              and E, W sum the local terms only.  0 = every atom
                              is local.  The building block of a spatial domain
                              decomposition: summing each domain's local-plus-
                              ghost forces onto the owning atoms gives the forces
                              of the whole system.  Other entry points evaluate
                              every atom; pod_md_step refuses ghosts.           */
} pod_system;

/* Creates a handle: validates params, builds the POD basis on the host (the
 * snapshot Gram matrix on an n_grid midpoint grid over (r_in, r_cut),
 * eigenvectors sorted by decreasing eigenvalue, each with its largest entry
 * positive, scaled by 1/sqrt(lambda) so R_k has unit L2 norm; Section 2.2,
 * Eq. 12) unless params->Q is given, and the angular tables (Table 3-5).
 * *out receives the handle.  The handle belongs to the CUDA device current at
 * this call (its workspace is allocated there): call it with that device
 * current; a call with another device current fails with POD_EINVAL.
 * Errors: POD_EINVAL, POD_ENOMEM, POD_ECUDA. */
int pod_create(const pod_params* params, pod_handle** out);

/* Frees the handle, its device tables and workspace.  NULL is allowed. */
int pod_destroy(pod_handle* h);

/* Model files (the paper defines no format; a deployment feature).  pod_save
 * writes the handle's parameters (r_in, r_cut, alpha, beta, gamma, K2..K4, P3, P4),
 * its projection Q and, if c (host [M]) is not NULL, the coefficients of a linear
 * model, as versioned text with round-trip precision; the file is written under a
 * temporary name and renamed, so it appears whole or not at all.  Errors:
 * POD_EINVAL (NULL, non-finite c), POD_EIO.
 * pod_load creates a handle (precision POD_FP64 or POD_MIXED) from such a file
 * with the saved Q, so it evaluates bit for bit like the saved handle; if the
 * file holds coefficients and c_out is not NULL they are copied to c_out (host,
 * capacity c_capacity >= M), and *n_c (if not NULL) is set to their number (0
 * when the file holds none).  Errors: POD_EIO (cannot open), POD_EINVAL
 * (malformed file, bad parameters, c_capacity too small); on errors after the
 * handle was created *out holds it for pod_last_error and must be destroyed. */
int pod_save(const pod_handle* h, const char* path, const double* c);
int pod_load(const char* path, int precision, pod_handle** out, double* c_out, int c_capacity, int* n_c);

/* Sizes and basis of a handle.  Any output pointer may be NULL.
 * M: descriptors per atom; Ns: snapshots; K: radial modes K_r;
 * Q_out: host [Ns][K] projection; eig_out: host [Ns] eigenvalues (descending;
 * zeros when Q was supplied). */
int pod_info(const pod_handle* h, int* M, int* Ns, int* K, double* Q_out, double* eig_out);

/* Sets a handle option.  POD_OPT_SYNC (default 1): wait for the stream at the
 * end of each call and report device-side conditions as return codes.
 * POD_OPT_PRECISION: POD_FP64 or POD_MIXED for subsequent calls. */
#define POD_OPT_SYNC 1
#define POD_OPT_PRECISION 2
#define POD_OPT_TIMING 3 /* 1: time each phase of pod_energy_forces with CUDA events */
#define POD_OPT_RADIAL 4 /* mixed path only: 0 (default) R_k from a 2048-interval cubic
                            Hermite table built in FP64 at first use (relative error
                            ~1e-7); 1 = snapshots evaluated per pair in FP32 and
                            projected (Eq. 3-12; POD cancellation costs ~1e-5)  */
#define POD_OPT_NEIGHBOR_REUSE 5 /* 1: pod_energy_forces reuses the list of its previous call
                                   (single configuration, same size and box) instead of
                                   rebuilding it; requires a skin (pod_set_skin) that
                                   covers the displacements since that call */
#define POD_OPT_DESCRIPTORS 6 /* three-body columns: 0 (default) the fast POD sums over all
                                 (j, k) (Eq. 23a/26a); 1 the exclusive sums over pairs
                                 k > j of the original POD (Eq. 15b), formed as
                                 (D3_mn - sum_j R_m(r_ij)^2) / 2 (Eq. 15c).  Honoured by
                                 pod_descriptors, pod_global_descriptors and the linear
                                 model's pod_energy_forces (its adjoint carries the
                                 extra two-body term); the quadratic and embedding models,
                                 the descriptor tangent, the fit entry points and
                                 pod_descriptors_static return POD_EINVAL while it is 1 */
#define POD_OPT_GRAM 7 /* normal equations of the fit: 0 (default) G = A^T A from exact
                          8-bit slice products on the BF16 tensor cores (tcgen05 MMAs
                          with TMEM accumulators; integer sums, no rounding beyond
                          2^-59 of the column maxima); 1 an FP64 SYRK on the FP64
                          pipes; 2 the same exact slice products through mma.sync
                          (bit-identical to 0) */
#define POD_OPT_ADJOINT 8 /* mixed path, linear model: where the adjoint pair pass g_ij of
                             Eq. 24c runs. -1 (default) by the autotuned launch shape, else
                             inside the fused kernel, which measured faster); 0 inside the
                             fused atom kernel; 1 as its own kernel (warp per atom, lane per
                             pair) after a forward-only atom kernel.  Forces and atom
                             energies are the same bits either way; E and W differ only in
                             the grouping of their exact fixed-point sums */
#define POD_OPT_NEIGHBOR_TESTS 9 /* candidate tests of the block-per-cell neighbour search:
                                    -1 (default) by the autotuned launch shape, else by size
                                    (block-wide up to 131,072 atoms); 1 block-wide (every
                                    thread of a cell's block over candidates x the cell's own
                                    atoms, shared-memory atomics per atom); 0 a warp per own
                                    atom (lanes over candidates, ballot compaction).  The lists
                                    are the same either way (sorted rows) */
#define POD_OPT_FIT_GRAPH 10 /* pod_fit: 1 (default) a fit records its device chain (neighbour
                                lists, design matrix, normal equations or QR, solve, residual)
                                into a CUDA graph after it has run, and a later pod_fit with the
                                same batch layout (sizes, offsets, boxes, periodicity), the same
                                device arrays, options and handle settings replays the graph
                                instead of issuing ~20 launches with host synchronisations
                                between them; results are the same bits.  A replay whose lists
                                no longer fit the recorded capacities falls back to the ordinary
                                path.  Phase timing (POD_OPT_TIMING) disables recording.  0: off */
#define POD_OPT_HOST_MAPPED 11 /* pod_energy_forces_host replays: 1 (default) the kernels read
                                  and write mapped pinned host buffers directly (on Grace,
                                  coherent over NVLink-C2C); 0 copy nodes into and out of
                                  library-owned device buffers.  Results are the same bits */
#define POD_OPT_WORKSPACE_LIMIT_MB 12 /* a cap, in MiB, on the device workspace this handle
                                         allocates (0, the default: none).  A call whose
                                         buffers would grow past it returns POD_ENOMEM before
                                         freeing or allocating anything, and the handle stays
                                         usable (raise or clear the cap and call again); a cap
                                         below what is already held frees nothing */
int pod_set_option(pod_handle* h, int option, int value);

/* Neighbour-list skin (A, default 0): lists are built with r_cut + skin and pairs
 * beyond r_cut contribute nothing, so a list stays valid while no atom has moved
 * more than skin / 2 since it was built (standard MD practice; the paper's
 * cut-off of Section 2.2 is unchanged).  Between rebuilds positions are shifted
 * by the box multiples frozen at the build, so atoms may cross the box edge.
 * Errors: POD_EINVAL. */
int pod_set_skin(pod_handle* h, double skin);

/* One velocity-Verlet step of the linear POD potential for a single
 * configuration: v += F dt / 2m; pos += v dt; F <- F(pos) (pod_energy_forces,
 * honouring POD_OPT_NEIGHBOR_REUSE); v += F dt / 2m.  pos, v, F: device [3][N],
 * updated in place (F must hold the forces at the input positions); sys gives N,
 * box and pbc (sys->pos is ignored); c device [M]; E device [1] receives the
 * potential energy at the new positions.  mass in atomic mass units, dt in fs,
 * energies in eV and lengths in A (1 eV/(A amu) = 9.648533212e-3 A/fs^2).
 * Errors as pod_energy_forces. */
int pod_md_step(pod_handle* h, const pod_system* sys, double* pos, double* v, double* F, const double* c,
                double mass, double dt, double* E, void* stream);

/* Per-phase device time of the pod_energy_forces calls made while
 * POD_OPT_TIMING was on, measured with CUDA events recorded on the call's stream
 * around each phase: ms[0] neighbour list (binning, search, sort), ms[1] fused
 * atom kernel, ms[2] force gather with the fused energy/virial reduction,
 * ms[3] reserved (0) (totals in milliseconds; ms is host [4]).  *calls receives the number of
 * calls timed.  Resets the totals.  With timing on, each call waits for its
 * last event. */
int pod_timing(pod_handle* h, double* ms, int* calls);

/* Waits for `stream` and returns the device-side status accumulated since the
 * last report (POD_OK, POD_ERANGE, POD_ENONFINITE, POD_ENEIGH, or POD_ECUDA when a
 * bounded wait inside a kernel ran out), then clears it. */
int pod_status(pod_handle* h, void* stream);

/* Full neighbour list of one configuration (the cut-off region of Section 2.2):
 * every (j, s) with |x_j + s L - x_i| < r_cut, excluding (i, 0), positions
 * wrapped into [0, L) in periodic directions, the squared distance formed in
 * FP64 as (dx*dx + dy*dy) + dz*dz without fused multiply-add, each atom's list
 * sorted by (j, s_x, s_y, s_z).
 *   count: device [N] number of neighbours per atom (may exceed cap)
 *   nbr:   device [N][cap] neighbour index j
 *   shift: device [N][cap][3] image shift s (int)
 * Errors: POD_EINVAL; POD_ENEIGH if an atom has more than cap neighbours (the
 * first cap entries are still written, count holds the true number). */
int pod_neighbors(pod_handle* h, const pod_system* sys, int cap, int* count, int* nbr, int* shift,
                  void* stream);

/* Descriptors D (device [N][M], FP64) of every atom: Eq. 12b, Eq. 26a, Eq. 27a,
 * Eq. 30a.  The mixed path computes in FP32 and stores FP64.  Batched systems
 * are supported.  Errors: POD_EINVAL, POD_ERANGE, POD_ENEIGH, POD_ECUDA. */
int pod_descriptors(pod_handle* h, const pod_system* sys, double* D, void* stream);

/* Linear POD energy and its derivatives (Eq. 57a, 58a; forces by the adjoint
 * of Eq. 24c / 26c):
 *   c:  device [M] coefficients (FP64)
 *   E:  device [max(1, n_configs)] total energy per configuration (FP64;
 *       order-independent: fixed-order sums, except a single configuration on
 *       the mixed path, whose E and W are exact fixed-point integer sums with
 *       2^-36 resolution), required
 *   Ei: device [N] atom energies or NULL
 *   F:  device [3][N] forces F_k = -dE/dr_k or NULL
 *   W:  device [max(1, n_configs)][9] virial W_ab = -sum_ij (r_ij)_a dE_i/d(r_ij)_b
 *       (row-major 3x3) or NULL
 * Errors: POD_EINVAL, POD_ERANGE, POD_ENEIGH, POD_ENONFINITE, POD_ECUDA. */
int pod_energy_forces(pod_handle* h, const pod_system* sys, const double* c, double* E, double* Ei, double* F,
                      double* W, void* stream);

/* Global descriptors G_m = sum_{i in config} D_im (Eq. 58a): device
 * [max(1, n_configs)][M].  dE/dc = G for the linear model.  Errors as
 * pod_descriptors. */
int pod_global_descriptors(pod_handle* h, const pod_system* sys, double* G, void* stream);

/* Directional derivative of the global descriptors along per-atom displacements:
 * Gdot_m = sum_k (dG_m/dr_k) . v_k, v device [3][N] (same layout as positions),
 * Gdot device [max(1, n_configs)][M], computed in one forward-mode pass through
 * Eq. 24b / 26a / 27a / 30a (dB/dr of Eq. 24c along r_j - r_i).  Since the
 * forces are linear in c, the gradient of any force loss L(F) with respect to c
 * is dL/dc = -Gdot evaluated at v = dL/dF.  Errors as pod_descriptors. */
int pod_descriptors_jvp(pod_handle* h, const pod_system* sys, const double* v, double* Gdot, void* stream);

/* Per-atom directional derivatives of the descriptors along per-atom
 * displacements: Ddot[i][m] = sum_k (dD_im/dr_k) . v_k (v device [3][N], Ddot
 * device [N][M]), the forward-mode pass of pod_descriptors_jvp (Eq. 24b / 26a /
 * 27a / 30a with dB/dr of Eq. 24c) without the sum over atoms.  Batches are
 * supported.  Errors as pod_descriptors. */
int pod_descriptors_tangent(pod_handle* h, const pod_system* sys, const double* v, double* Ddot, void* stream);

/* Gradient of a force-matching loss (Eq. 63b) with respect to the parameters of
 * the handle's current model, from per-atom descriptors D and their directional
 * derivatives Ddot along v = F - F_ref (device [n_atoms][M] each, from
 * pod_descriptors and pod_descriptors_tangent):
 *   grad = sum_i w_i dE_i/dtheta + t (d/de) [sum_i dE_i/dtheta](r + e v)
 * with w (device [n_atoms]) the weight of each atom's energy term -- for
 * L = sum_c w_E^2 ((E_c - E_c^ref) / N_c)^2 + w_F^2 |F - F^ref|^2 it is
 * 2 w_E^2 (E_c - E_c^ref) / N_c^2 on the atoms of configuration c -- and t the
 * weight of the force term (-2 w_F^2 for that loss).  grad (host) receives:
 *   linear model     dL/dc (M)
 *   quadratic model  dL/dc (M), then dL/dbeta_mn for m <= n, row-major (M (M + 1) / 2)
 *   embedding model  dL/dc (M), dL/da (M), dL/dalpha_k for k = 0..degree
 * FP64, sums in a fixed order; synchronous.  Errors: POD_EINVAL, POD_ENOMEM,
 * POD_ECUDA. */
int pod_model_gradients(pod_handle* h, int n_atoms, const double* D, const double* Ddot, const double* w, double t,
                        double* grad, void* stream);

/* pod_energy_forces with HOST buffers: sys->pos, c, E, Ei, F, W are host
 * pointers (pinned memory is fastest).  Copies inputs to library-owned device
 * buffers, computes, copies results back and waits for the stream.  Calls that
 * repeat with the same pinned buffers, size, box and settings on a non-default
 * stream replay a CUDA graph from the third call on; with POD_OPT_HOST_MAPPED
 * (default) and buffers mapped into the device's address space (pinned memory
 * under unified addressing), that graph's kernels read the positions and
 * coefficients and write E, Ei, F and W through the buffers' device addresses
 * instead of copying them (same bits).  The buffers must hold the documented
 * sizes either way, and buffers passed again at the same addresses must still
 * be allocated and pinned: a replay reads and writes them without re-checking
 * (a call with other pointers takes the direct path and records anew). */
int pod_energy_forces_host(pod_handle* h, const pod_system* sys, const double* c, double* E, double* Ei,
                           double* F, double* W, void* stream);

/* Options of the ridge least-squares fit of Eq. 63a. */
typedef struct {
  double w_E;         /* energy-row weight (paper: 100)                          */
  double w_F;         /* force-row weight (paper: 1)                             */
  double gamma_reg;   /* ridge parameter (paper: 1e-12)                          */
  int per_atom_energy;/* 1: energy rows are G_m / N against E / N (default)      */
  int solver;         /* 0 (default): Cholesky of the normal equations, and when
                         a pivot is not positive a Householder QR of the weighted
                         design matrix [A; sqrt(gamma_reg) I] (condition number
                         of A instead of its square); 1: Cholesky only
                         (POD_ESINGULAR on a non-positive pivot); 2: QR only      */
} pod_fit_opts;

/* Fits c (host [M]) to reference energies and forces of a batch of
 * configurations: rows w_E G_m(cfg) / N_cfg against w_E E_ref / N_cfg and rows
 * -w_F dG_m/dr_ka against w_F F_ref, plus gamma_reg I.  Normal equations
 * (A^T A + gamma I) c = A^T b with G = A^T A formed exactly from 8-bit slice
 * products on the tensor cores (POD_OPT_GRAM 0, default; rounding below 2^-59 of
 * the column maxima) or by an FP64 SYRK (POD_OPT_GRAM 1), solved by FP64
 * Cholesky; with opts->solver 0 or 2 a tall-skinny FP64 Householder QR of the
 * weighted design matrix instead (fallback on a non-positive pivot, or always).
 *   E_ref: device [n_configs]; F_ref: device [3][N]; mae_E (per atom) and
 *   mae_F (per component) receive the training errors (host, may be NULL).
 * Synchronous.  Errors: POD_EINVAL, POD_ESINGULAR, POD_ERANGE, POD_ENEIGH,
 * POD_ECUDA. */
int pod_fit(pod_handle* h, const pod_system* batch, const double* E_ref, const double* F_ref,
            const pod_fit_opts* opts, double* c_out, double* mae_E, double* mae_F);

/* Number of pod_fit calls on this handle that replayed a recorded fit
 * (POD_OPT_FIT_GRAPH).  POD_EINVAL on a null argument. */
int pod_fit_replays(const pod_handle* h, int* replays);

/* The fit in stages, for sharding configurations over several GPUs or processes
 * (the normal equations are additive over configurations):
 *   pod_fit_normal   builds A and b for this batch and returns G = A^T A +
 *                    gamma_reg I and r = A^T b (host [M][M] and [M]); A stays
 *                    in the handle's workspace.  Pass gamma_reg = 0 on all but
 *                    one shard (or add gamma once after summing).
 *   pod_fit_solve    solves G c = r by Cholesky on the GPU (host inputs/output);
 *                    POD_ESINGULAR if G is not positive definite.
 *   pod_fit_residual sums |A c - b| over the energy rows (divided by w_E) and the
 *                    force rows (divided by w_F) of the last pod_fit_normal batch;
 *                    *n_E / *n_F receive the row counts (MAE = sum / n).
 * Synchronous.  Errors as pod_fit. */
int pod_fit_normal(pod_handle* h, const pod_system* batch, const double* E_ref, const double* F_ref,
                   const pod_fit_opts* opts, double* G_out, double* r_out);
int pod_fit_solve(pod_handle* h, const double* G, const double* r, double* c_out);
int pod_fit_residual(pod_handle* h, const double* c, double* sum_abs_E, double* sum_abs_F, int* n_E, int* n_F);

/* pod_descriptors without any memory allocation.  The paper has no counterpart:
 * this is a deployment variant for callers that cannot let a library allocate
 * device memory -- for example molecular-dynamics engines and plugins that keep
 * all device memory in their own pool with a fixed budget and forbid other code
 * from calling cudaMalloc / cudaFree (which synchronise the device and fragment
 * the pool).  The caller passes the positions (device [3][N]) and the output D
 * (device [N][M]), as for pod_descriptors; every intermediate buffer, the mixed
 * path's radial table included, lives in one file-scope device array of about
 * 6.8 MB that each GPU loading the library holds until the process exits.  The
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   Limits: one configuration of 1..4096 atoms (POD_EINVAL beyond), at most 64
 *   neighbours per atom and 32 atoms per cell (POD_ENEIGH beyond); every atom is
 *   evaluated (n_local in (0, N) is refused with POD_EINVAL).  The handle's
 *   device must be current (POD_EINVAL otherwise), as for every other call.
 *   Results: the same kernels and radial evaluation as pod_descriptors on the
 *   handle (mixed path: the FP64-built radial table by default, per-pair
 *   snapshots under POD_OPT_RADIAL = 1; FP64 path unchanged).
 *   Set-up: pod_create, on its device and with that device current, looks up
 *   the array's device address (cudaGetSymbolAddress) and caches it; under
 *   CUDA's lazy module loading this is where the array is loaded.  Should that
 *   lookup fail there, the first call repeats it (it then belongs before any
 *   stream capture).  The first call of a handle copies its radial table (mixed
 *   path, up to 512 KB) into the array from host memory.
 *   All calls share the array and it keeps the previous call's contents (the
 *   call clears what must start at zero): calls that overlap on the GPU (other
 *   streams or host threads) race and must be serialised by the caller.  Waits
 *   for `stream` before returning. */
int pod_descriptors_static(pod_handle* h, const pod_system* sys, double* D, void* stream);

/* Spatial decomposition of one periodic system into slabs along an axis, one GPU
 * per slab (the per-atom evaluation of Sec. 2 split over GPUs; the paper has no
 * multi-GPU counterpart).  Each domain is evaluated by pod_energy_forces with
 * its own atoms first and the ghosts after them (pod_system.n_local), the axis
 * open; these two calls are the device side of the exchange between domains.
 *
 * pod_halo_select: the atoms i of pos (device [3][n_atoms]) whose coordinate
 * along `axis`, wrapped into [0, L) as x - L floor(x / L), lies in [x0, x1), in
 * ascending index order: idx (device [cap]) receives i, out (device [3][cap])
 * the position with the axis coordinate replaced by (x + shift) - offset (shift:
 * a periodic image, -L, 0 or L; offset: the origin of the receiving domain) and
 * the other two coordinates unchanged, *count (host) the number selected.
 * Synchronous.  POD_ENEIGH if more than cap atoms are selected (*count holds the
 * number; nothing beyond cap is written); POD_EINVAL on bad arguments or when
 * the handle's device is not current. */
int pod_halo_select(pod_handle* h, const double* pos, int n_atoms, int axis, double L, double x0, double x1,
                    double shift, double offset, int cap, int* idx, double* out, int* count, void* stream);

/* pod_halo_add: F[d][idx[k]] += G[d][k] for k < n (G device [3][n], idx device
 * [n] of distinct atom indices in [0, n_atoms), F device [3][n_atoms]): ghost
 * forces returned by a neighbouring domain added onto the owning atoms.  An index
 * out of range is skipped and reported (POD_ENEIGH, when POD_OPT_SYNC is on). */
int pod_halo_add(pod_handle* h, const double* G, const int* idx, int n, double* F, int n_atoms, void* stream);

/* Quadratic POD model (Sec. 4, the extension of Eq. 57a with products of
 * descriptors): E_i = sum_m c_m D_im + sum_m sum_{n >= m} beta_mn D_im D_in.
 * beta: host [M][M] row-major; only the entries with m <= n are read (the
 * one-body column 0 included); copied to the device.  NULL returns the handle to
 * the linear model.  While set, pod_energy_forces, pod_energy_forces_host and
 * pod_md_step evaluate the quadratic model (forces by the same adjoint pass with
 * dE_i/dD_im = c_m + sum_n (beta_mn + beta_nm) D_in per atom); the fit entry
 * points fit the linear model only.  POD_EINVAL for non-finite weights. */
int pod_set_quadratic(pod_handle* h, const double* beta);

/* Embedding model (Sec. 3: EAM and MEAM expressed with POD descriptors -- a
 * polynomial embedding of an atom density that is a linear combination of the
 * two-, three- and four-body descriptors):
 *   E_i = sum_m c_m D_im + F(rho_i),  rho_i = sum_m a_m D_im,
 *   F(rho) = sum_{k=0..degree} alpha_k rho^k.
 * With a on the two-body columns only this is an EAM-type potential, with the
 * three-body columns too a MEAM-type one; degree 2 is the quadratic model with
 * beta = alpha_2 a a^T (upper triangle doubled off the diagonal).
 *   a: host [M] density weights (one-body column 0 included), or NULL to return
 *      the handle to the linear model;  degree: 1..POD_EMB_MAX_DEGREE;
 *   alpha: host [degree + 1], alpha_0 first.
 * Copied to the device.  While set, pod_energy_forces, pod_energy_forces_host and
 * pod_md_step evaluate this model (forces by the same adjoint pass with
 * dE_i/dD_im = c_m + F'(rho_i) a_m per atom); it replaces a quadratic model
 * and is replaced by one; the fit entry points fit the linear model only.
 * POD_EINVAL for a bad degree or non-finite weights. */
#define POD_EMB_MAX_DEGREE 8
int pod_set_embedding(pod_handle* h, const double* a, int degree, const double* alpha);

/* Launch-shape autotuner (a deployment feature; the paper has no counterpart).
 * Times the three phases of pod_energy_forces on `sys` (one configuration,
 * device positions as for pod_energy_forces; c: device [M]) for a small set of
 * candidate launch shapes -- warps per block of the neighbour search {2, 4, 6, 8}
 * each with block-wide candidate tests and with a warp per own atom,
 * of the fused atom kernel {1, 2, 4} (FP32 table path: each with and without R'
 * staged in shared memory), and, on the FP64 path, warps per block x blocks per
 * SM of the gather {16x3, 16x2, 8x6, 8x4, 4x12} -- with CUDA events on `stream`, `reps`
 * timed calls each (after one warm-up call), and keeps the fastest per phase.
 * The result is stored in the handle for the system's size class (floor(log2
 * N)) and used by later calls on systems of that class; the other classes keep
 * the default shape (4, 2, 16x3).  Results do not depend on the shape except
 * for the rounding order of the energy and virial sums.  Synchronous (calls
 * pod_energy_forces about 25 x (reps + 1) times); not for use during stream
 * capture.
 *   shape (host int[6], or NULL): neighbour wpb, atom wpb, gather wpb, gather
 *   blocks per SM, and the form of the adjoint pair pass: 0 inside the fused atom
 *   kernel, re-evaluating R'; 1 the same with R' staged in shared memory (FP32
 *   table path); 2 as its own kernel after a forward-only atom kernel (FP32 linear
 *   model; see POD_OPT_ADJOINT) -- all candidates of the atom-phase search; and
 *   the neighbour search's candidate tests: 1 block-wide (every thread of the
 *   cell's block over candidates x the cell's own atoms), 0 a warp per own atom.
 *   ms (host double[3], or NULL): mean times of the neighbour, atom and gather
 *   phases with the chosen shape.
 * A batch (n_configs > 1) tunes the fit's design pass instead: the atom kernel in
 * design mode {1, 2, 4} warps per block and the force-row gather {2, 4, 8}, timed
 * around the design-matrix stage of pod_fit with zero labels (c may be NULL);
 * shape then holds (0, atom wpb, gather wpb, 0, 0, 0) and ms[1] the stage's time;
 * later fits of batches of that size class use it (results do not depend on it).
 * Errors as pod_energy_forces / pod_fit. */
int pod_autotune(pod_handle* h, const pod_system* sys, const double* c, int reps, int* shape, double* ms,
                 void* stream);

/* Throughput probe for the vector pipes that bound the fused atom kernel (not a
 * step of the method; the paper has no counterpart).  Launches, on `stream`, one
 * grid of independent fused multiply-add chains filling every SM of the current
 * device and stores in *flops the floating-point operations it performs (an FMA
 * counts 2).  kind: 0 = FP32 fmaf, 1 = FP32 paired FMA (two lanes of float2 per
 * instruction), 2 = FP64 fma.  The caller times the launch on `stream` (CUDA
 * events) and divides.  Touches no caller memory; iters >= 1; POD_EINVAL on a
 * bad kind/iters/null flops, POD_ECUDA on a launch failure. */
int pod_fma_probe(int kind, int iters, double* flops, void* stream);

/* Self-test of the bounded waits that the tensor-core kernels use (not a step of
 * the method): one thread of a one-block launch on the current device waits on an
 * mbarrier that nothing arrives at, gives up after limit_ns nanoseconds of global
 * time (0 .. 1e10) and reports it as the status bit ST_TIMEOUT (64) in
 * *status_out; the context stays usable.  Synchronous (default stream).
 * POD_EINVAL on a bad limit or a null status_out, POD_ENOMEM / POD_ECUDA on a
 * failed allocation or launch. */
int pod_selftest_wait(long long limit_ns, int* status_out);

/* Message of the last error on this handle ("" if none).  Owned by the handle. */
const char* pod_last_error(const pod_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* FASTPOD_POD_H */
