/*
 * Plain FP64 CPU oracle for fast proper orthogonal descriptors
 * (N.-C. Nguyen, "Fast proper orthogonal descriptors for many-body interatomic
 * potentials", arXiv:2212.14446).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or table with the CUDA library.
 *
 * Everything is double precision, compiled with -ffp-contract=off, written as
 * the plain definitions of the paper:
 *   - radial snapshots and smooth cut-off ............... Eq. 3-11 (Section 2.2)
 *   - POD basis R_k = sum_l Q_lk Phi_l ................... Eq. 12
 *   - two-body descriptors D2_k = sum_j R_k(r_ij) ........ Eq. 12b
 *   - inclusive three-body sums (j = k included) ......... Eq. 15 / Eq. 22a
 *   - inclusive four-body sums over all ordered (j,k,l) .. Eq. 18a / Eq. 23a
 *   - analytic derivatives of those sums ................. Section 2.7
 * plus, as a second and separately derived form of the same quantities, the
 * atom-density algorithm:
 *   - angular monomials in the order of Table 3 ......... Eq. 23b
 *   - atomic basis B_imnl ............................... Eq. 24b
 *   - three-body contraction with Table 4 coefficients .. Eq. 26a
 *   - four-body products (b = c = 0) .................... Eq. 27a
 *   - four-body trinomial contraction .................... Eq. 30a
 *   - descriptor derivatives via dB/dr .................. Eq. 26c / Eq. 24c
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *   - snapshot set: phi(alpha, beta) for every alpha x beta in the lists (kappa = 1)
 *     followed by varphi(gamma) for every gamma (kappa = 0); the convex
 *     combination psi spans the same space (Eq. 5).
 *   - POD: Gram matrix C = h Phi^T Phi on a midpoint grid of n_grid points over
 *     (r_in, r_cut); eigenvalues descending; each eigenvector's largest-magnitude
 *     entry made positive; Q_lk = v_lk / sqrt(lambda_k) so that R_k has unit L2 norm.
 *   - neighbours: positions wrapped x <- x - L floor(x / L) in periodic
 *     directions; pair (j, s) included when |x_j + s L - x_i|^2 < r_cut^2 with the
 *     squared distance formed as (dx*dx + dy*dy) + dz*dz; the list is sorted by
 *     (j, s_x, s_y, s_z).
 *   - descriptor order: [1 | D2 (m) | D3 (m major, n = 0..P3) | D4 (m major,
 *     p in Table 1 order)], Table 1 order = n ascending, then (a, b, c)
 *     lexicographically descending.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EPS_CUT 1e-6   /* epsilon inside the cut-off function, Eq. 8 */
#define ORC_MAXS 64        /* max number of snapshots */
#define ORC_MAXK 32        /* max number of radial modes */
#define ORC_MAXP 10        /* max angular degree */

typedef struct {
  double r_in, r_cut;
  int n_alpha;
  const double* alpha;
  int n_beta;
  const double* beta;
  int n_gamma;
  const double* gamma;
  int K2, K3, K4, P3, P4;
} orc_params;

typedef struct {
  int N;
  const double* pos; /* N x 3, atom-major */
  double box[3];
  int pbc[3];
} orc_system;

/* ------------------------------------------------------------------ sizes */

int orc_num_snapshots(const orc_params* p) { return p->n_alpha * p->n_beta + p->n_gamma; }

static int imax(int a, int b) { return a > b ? a : b; }

int orc_num_radial(const orc_params* p) {
  int k = imax(p->K2, p->P3 >= 0 ? p->K3 : 0);
  if (p->P4 >= 0) k = imax(k, p->K4);
  return k;
}

int orc_max_degree(const orc_params* p) { return imax(p->P3, p->P4); }

/* number of monomials of degree exactly n in three variables */
static int orc_nmono_deg(int n) { return (n + 1) * (n + 2) / 2; }

/* number of monomials of degree <= P: (P+1)(P+2)(P+3)/6 */
int orc_num_monomials(int P) { return P < 0 ? 0 : (P + 1) * (P + 2) * (P + 3) / 6; }

/* Partitions n = a + b + c with a >= b >= c >= 0, in lexicographically descending
 * order of (a, b, c).  Used both for Table 1 and for the exponent patterns of
 * Table 3.  Returns the count; writes triples when out != NULL. */
static int orc_partitions(int n, int* out) {
  int cnt = 0;
  for (int a = n; a >= 0; --a)
    for (int b = (n - a < a ? n - a : a); b >= 0; --b) {
      int c = n - a - b;
      if (c < 0 || c > b) continue;
      if (out) { out[3 * cnt] = a; out[3 * cnt + 1] = b; out[3 * cnt + 2] = c; }
      ++cnt;
    }
  return cnt;
}

/* Four-body angular functions of Table 1 for degrees 0..P4: (a, b, c) triples. */
int orc_fourbody_table(int P4, int* abc) {
  int cnt = 0;
  for (int n = 0; n <= P4; ++n) cnt += orc_partitions(n, abc ? abc + 3 * cnt : NULL);
  return cnt;
}

int orc_num_fourbody(int P4) { return P4 < 0 ? 0 : orc_fourbody_table(P4, NULL); }

int orc_num_descriptors(const orc_params* p) {
  int M = 1 + p->K2;
  if (p->P3 >= 0) M += p->K3 * (p->P3 + 1);
  if (p->P4 >= 0) M += p->K4 * orc_num_fourbody(p->P4);
  return M;
}

/* Angular monomials of Table 3 for degrees 0..P: exponent triples and the
 * multinomial coefficients n!/(e1! e2! e3!) of Table 4.  Within a degree the
 * exponent patterns (partitions) come in descending order; for each pattern the
 * variable carrying the first part runs over x, y, z, then the variable carrying
 * the second part over the remaining ones, equal parts being assigned to
 * variables in increasing order. */
int orc_monomial_table(int P, int* exps, double* coef) {
  int cnt = 0;
  for (int n = 0; n <= P; ++n) {
    int parts[3 * 64];
    int np = orc_partitions(n, parts);
    for (int q = 0; q < np; ++q) {
      const int* lam = parts + 3 * q;
      for (int v1 = 0; v1 < 3; ++v1)
        for (int v2 = 0; v2 < 3; ++v2) {
          if (v2 == v1) continue;
          int v3 = 3 - v1 - v2;
          if (lam[0] == lam[1] && !(v1 < v2)) continue;
          if (lam[1] == lam[2] && !(v2 < v3)) continue;
          int e[3];
          e[v1] = lam[0];
          e[v2] = lam[1];
          e[v3] = lam[2];
          if (exps) { exps[3 * cnt] = e[0]; exps[3 * cnt + 1] = e[1]; exps[3 * cnt + 2] = e[2]; }
          if (coef) {
            double f = 1.0;
            for (int t = 2; t <= n; ++t) f *= t;
            for (int d = 0; d < 3; ++d)
              for (int t = 2; t <= e[d]; ++t) f /= t;
            coef[cnt] = f;
          }
          ++cnt;
        }
    }
  }
  return cnt;
}

/* ------------------------------------------------- radial snapshots (Eq. 3-11) */

/* Phi_l(r) = f_c(r) psi(r; mu_l) and dPhi_l/dr for every snapshot l. */
int orc_snapshots(const orc_params* p, double r, double* phi, double* dphi) {
  const double h = p->r_cut - p->r_in;
  const double s = r - p->r_in;
  const double t = s / h;
  /* smooth cut-off, Eq. 8 */
  const double u = 1.0 - t * t * t;
  const double y = u * u + ORC_EPS_CUT;
  const double fc = exp(1.0 - 1.0 / sqrt(y));
  /* d/dr exp(1 - y^-1/2) = fc * (1/2) y^-3/2 * dy/dr,  dy/dr = 2 u (-3 t^2 / h) */
  const double dfc = fc * (u * (-3.0 * t * t / h)) / (y * sqrt(y));
  int l = 0;
  for (int ia = 0; ia < p->n_alpha; ++ia)
    for (int ib = 0; ib < p->n_beta; ++ib) {
      const double al = p->alpha[ia], be = p->beta[ib];
      /* scaled distance x (Eq. 4) and its derivative */
      const double eb = exp(-be), et = exp(-be * t);
      const double x = (et - 1.0) / (eb - 1.0);
      const double dx = (-be / h) * et / (eb - 1.0);
      const double arg = al * M_PI * x;
      const double sn = sin(arg), cs = cos(arg);
      const double f = sn / s;                                  /* phi, Eq. 3 */
      const double df = (al * M_PI * cs * dx * s - sn) / (s * s);
      phi[l] = fc * f;
      dphi[l] = dfc * f + fc * df;
      ++l;
    }
  for (int ig = 0; ig < p->n_gamma; ++ig) {
    const double ga = p->gamma[ig];
    const double f = pow(r, -ga);                               /* varphi, Eq. 3 */
    const double df = -ga * f / r;
    phi[l] = fc * f;
    dphi[l] = dfc * f + fc * df;
    ++l;
  }
  return l;
}

/* ------------------------------------------------------------- POD (Eq. 12) */

/* Cyclic Jacobi eigen-solver for a symmetric n x n matrix A (destroyed).
 * On return w holds the eigenvalues and V (n x n, row-major) the eigenvectors in
 * its columns.  Rotation angles follow the classical symmetric Schur
 * decomposition of a 2 x 2 block. */
static int orc_jacobi(int n, double* A, double* V, double* w) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  int sweep;
  for (sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        const double app = A[p * n + p], aqq = A[q * n + q];
        if (fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
        rotated = 1;
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = t * c;
        for (int k = 0; k < n; ++k) { /* columns p, q of A J */
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* rows p, q of J^T (A J) */
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        A[p * n + q] = A[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    if (!rotated) break;
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  return sweep;
}

/* Snapshot Gram matrix on the midpoint grid, its eigen-decomposition and the
 * projection Q (Ns x K, row-major).  eig receives all Ns eigenvalues
 * (descending).  gram (Ns x Ns) receives C if non-NULL. */
int orc_basis(const orc_params* p, int n_grid, int K, double* Q, double* eig, double* gram) {
  const int Ns = orc_num_snapshots(p);
  if (Ns <= 0 || Ns > ORC_MAXS || K < 1 || K > Ns || n_grid < Ns) return -1;
  const double h = (p->r_cut - p->r_in) / n_grid;
  double* C = (double*)calloc((size_t)Ns * Ns, sizeof(double));
  double* V = (double*)calloc((size_t)Ns * Ns, sizeof(double));
  double w[ORC_MAXS], phi[ORC_MAXS], dphi[ORC_MAXS];
  for (int g = 0; g < n_grid; ++g) {
    const double r = p->r_in + (g + 0.5) * h;
    orc_snapshots(p, r, phi, dphi);
    for (int a = 0; a < Ns; ++a)
      for (int b = 0; b < Ns; ++b) C[a * Ns + b] += phi[a] * phi[b];
  }
  for (int a = 0; a < Ns * Ns; ++a) C[a] *= h;
  if (gram) memcpy(gram, C, sizeof(double) * Ns * Ns);
  orc_jacobi(Ns, C, V, w);
  /* sort descending (selection sort on indices) */
  int idx[ORC_MAXS];
  for (int i = 0; i < Ns; ++i) idx[i] = i;
  for (int i = 0; i < Ns; ++i)
    for (int j = i + 1; j < Ns; ++j)
      if (w[idx[j]] > w[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  for (int k = 0; k < Ns; ++k) eig[k] = w[idx[k]];
  for (int k = 0; k < K; ++k) {
    const int col = idx[k];
    int amax = 0;
    for (int l = 1; l < Ns; ++l)
      if (fabs(V[l * Ns + col]) > fabs(V[amax * Ns + col])) amax = l;
    const double sgn = V[amax * Ns + col] < 0 ? -1.0 : 1.0;
    const double scale = sgn / sqrt(w[col]);
    for (int l = 0; l < Ns; ++l) Q[l * K + k] = V[l * Ns + col] * scale;
  }
  free(C);
  free(V);
  return 0;
}

/* R_k(r) = sum_l Q_lk Phi_l(r) and its derivative (Eq. 12). */
static void orc_radial(const orc_params* p, const double* Q, int K, double r, double* R, double* dR) {
  double phi[ORC_MAXS], dphi[ORC_MAXS];
  const int Ns = orc_snapshots(p, r, phi, dphi);
  for (int k = 0; k < K; ++k) {
    double a = 0.0, b = 0.0;
    for (int l = 0; l < Ns; ++l) {
      a += Q[l * K + k] * phi[l];
      b += Q[l * K + k] * dphi[l];
    }
    R[k] = a;
    dR[k] = b;
  }
}

void orc_radial_eval(const orc_params* p, const double* Q, int K, int n, const double* r, double* R,
                     double* dR) {
  for (int i = 0; i < n; ++i) orc_radial(p, Q, K, r[i], R + (size_t)i * K, dR + (size_t)i * K);
}

/* ---------------------------------------------------- neighbours (brute force) */

static double orc_wrap(double x, double L) { return x - L * floor(x / L); }

/* All (j, s) with |x_j + s L - x_i| < r_cut, excluding (i, 0), sorted by
 * (j, s_x, s_y, s_z).  Returns the count (entries beyond cap are not written). */
int orc_neighbors_of(const orc_system* sy, double rcut, int i, int cap, int* js, int* sh, double* d) {
  double xi[3];
  int S[3];
  for (int a = 0; a < 3; ++a) {
    const double x = sy->pos[3 * i + a];
    xi[a] = sy->pbc[a] ? orc_wrap(x, sy->box[a]) : x;
    S[a] = sy->pbc[a] ? (int)ceil(rcut / sy->box[a]) : 0;
  }
  const double rc2 = rcut * rcut;
  int cnt = 0;
  for (int j = 0; j < sy->N; ++j) {
    double xj[3];
    for (int a = 0; a < 3; ++a) {
      const double x = sy->pos[3 * j + a];
      xj[a] = sy->pbc[a] ? orc_wrap(x, sy->box[a]) : x;
    }
    for (int sx = -S[0]; sx <= S[0]; ++sx)
      for (int syy = -S[1]; syy <= S[1]; ++syy)
        for (int sz = -S[2]; sz <= S[2]; ++sz) {
          if (j == i && sx == 0 && syy == 0 && sz == 0) continue;
          const double dx = (xj[0] + sx * sy->box[0]) - xi[0];
          const double dy = (xj[1] + syy * sy->box[1]) - xi[1];
          const double dz = (xj[2] + sz * sy->box[2]) - xi[2];
          const double r2 = (dx * dx + dy * dy) + dz * dz;
          if (!(r2 < rc2)) continue;
          if (cnt < cap) {
            if (js) js[cnt] = j;
            if (sh) { sh[3 * cnt] = sx; sh[3 * cnt + 1] = syy; sh[3 * cnt + 2] = sz; }
            if (d) { d[3 * cnt] = dx; d[3 * cnt + 1] = dy; d[3 * cnt + 2] = dz; }
          }
          ++cnt;
        }
  }
  return cnt;
}

/* Cell-list form of the same neighbour search (a second, faster route to the
 * list above, for large systems and the timed CPU baseline).  Cells are at
 * least r_cut wide; every (cell, image) whose unwrapped cell index lies within
 * ceil(r_cut / cell) + 1 of the atom's cell is scanned (one cell of margin
 * against rounding in the cell assignment), each candidate is tested with the
 * same FP64 expression as orc_neighbors_of, and the hits are sorted by
 * (j, s_x, s_y, s_z), so both routes give the same list entry for entry. */
typedef struct {
  int N, nc[3], S[3], pbc[3];
  double lo[3], cs[3], box[3];
  double* xw;      /* N x 3 wrapped (periodic) or raw (open) positions */
  int* start;      /* ncells + 1 */
  int* atoms;      /* N, ascending atom index within each cell */
} orc_cells;

void orc_cells_free(orc_cells* cl) {
  if (!cl) return;
  free(cl->xw);
  free(cl->start);
  free(cl->atoms);
  free(cl);
}

static int orc_cell_of(const orc_cells* cl, int a, double x) {
  int c = (int)floor((x - cl->lo[a]) / cl->cs[a]);
  if (c < 0) c = 0;
  if (c >= cl->nc[a]) c = cl->nc[a] - 1;
  return c;
}

orc_cells* orc_cells_build(const orc_system* sy, double rcut) {
  orc_cells* cl = (orc_cells*)calloc(1, sizeof(orc_cells));
  if (!cl) return NULL;
  const int N = sy->N;
  cl->N = N;
  cl->xw = (double*)malloc(sizeof(double) * 3 * (size_t)(N + 1));
  if (!cl->xw) { orc_cells_free(cl); return NULL; }
  long long ncells = 1;
  for (int a = 0; a < 3; ++a) {
    cl->pbc[a] = sy->pbc[a] ? 1 : 0;
    cl->box[a] = sy->box[a];
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < N; ++i) {
      const double x = sy->pos[3 * i + a];
      const double v = cl->pbc[a] ? orc_wrap(x, sy->box[a]) : x;
      cl->xw[3 * i + a] = v;
      if (i == 0 || v < lo) lo = v;
      if (i == 0 || v > hi) hi = v;
    }
    if (cl->pbc[a]) {
      lo = 0.0;
      hi = sy->box[a];
    }
    int nc = (int)floor((hi - lo) / rcut);
    if (nc < 1) nc = 1;
    if (nc > 256) nc = 256;
    cl->nc[a] = nc;
    cl->lo[a] = lo;
    cl->cs[a] = hi > lo ? (hi - lo) / nc : 1.0;
    cl->S[a] = (int)ceil(rcut / cl->cs[a]) + 1;
    ncells *= nc;
  }
  cl->start = (int*)calloc((size_t)ncells + 1, sizeof(int));
  cl->atoms = (int*)malloc(sizeof(int) * (size_t)(N + 1));
  int* cell = (int*)malloc(sizeof(int) * (size_t)(N + 1));
  if (!cl->start || !cl->atoms || !cell) { free(cell); orc_cells_free(cl); return NULL; }
  for (int i = 0; i < N; ++i) {
    const int cx = orc_cell_of(cl, 0, cl->xw[3 * i]);
    const int cy = orc_cell_of(cl, 1, cl->xw[3 * i + 1]);
    const int cz = orc_cell_of(cl, 2, cl->xw[3 * i + 2]);
    cell[i] = (cz * cl->nc[1] + cy) * cl->nc[0] + cx;
    cl->start[cell[i] + 1]++;
  }
  for (long long c = 0; c < ncells; ++c) cl->start[c + 1] += cl->start[c];
  int* fill = (int*)malloc(sizeof(int) * (size_t)(ncells + 1));
  if (!fill) { free(cell); orc_cells_free(cl); return NULL; }
  memcpy(fill, cl->start, sizeof(int) * (size_t)ncells);
  for (int i = 0; i < N; ++i) cl->atoms[fill[cell[i]]++] = i;  /* ascending within a cell */
  free(fill);
  free(cell);
  return cl;
}

typedef struct {
  int j, s[3];
  double d[3];
} orc_hit;

static int orc_hit_cmp(const void* pa, const void* pb) {
  const orc_hit* a = (const orc_hit*)pa;
  const orc_hit* b = (const orc_hit*)pb;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  for (int t = 0; t < 3; ++t)
    if (a->s[t] != b->s[t]) return a->s[t] < b->s[t] ? -1 : 1;
  return 0;
}

/* Neighbours of atom i through the cell list; same output contract as
 * orc_neighbors_of (returns the true count, writes at most cap entries). */
int orc_cells_neighbors_of(const orc_cells* cl, double rcut, int i, int cap, int* js, int* sh, double* d) {
  const double* xi = cl->xw + 3 * i;
  int ci[3], lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    ci[a] = orc_cell_of(cl, a, xi[a]);
    lo[a] = ci[a] - cl->S[a];
    hi[a] = ci[a] + cl->S[a];
    if (!cl->pbc[a]) {
      if (lo[a] < 0) lo[a] = 0;
      if (hi[a] > cl->nc[a] - 1) hi[a] = cl->nc[a] - 1;
    }
  }
  const double rc2 = rcut * rcut;
  int nhit = 0, hcap = 64;
  orc_hit* hits = (orc_hit*)malloc(sizeof(orc_hit) * hcap);
  if (!hits) return -1;
  for (int tz = lo[2]; tz <= hi[2]; ++tz)
    for (int ty = lo[1]; ty <= hi[1]; ++ty)
      for (int tx = lo[0]; tx <= hi[0]; ++tx) {
        const int t[3] = {tx, ty, tz};
        int c[3], s[3];
        for (int a = 0; a < 3; ++a) {
          /* unwrapped cell index t -> (cell in [0, nc), image shift floor(t / nc)) */
          const int nc = cl->nc[a];
          s[a] = t[a] >= 0 ? t[a] / nc : -((-t[a] + nc - 1) / nc);
          c[a] = t[a] - s[a] * nc;
        }
        const int cell = (c[2] * cl->nc[1] + c[1]) * cl->nc[0] + c[0];
        for (int q = cl->start[cell]; q < cl->start[cell + 1]; ++q) {
          const int j = cl->atoms[q];
          if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
          const double* xj = cl->xw + 3 * j;
          const double dx = (xj[0] + s[0] * cl->box[0]) - xi[0];
          const double dy = (xj[1] + s[1] * cl->box[1]) - xi[1];
          const double dz = (xj[2] + s[2] * cl->box[2]) - xi[2];
          const double r2 = (dx * dx + dy * dy) + dz * dz;
          if (!(r2 < rc2)) continue;
          if (nhit == hcap) {
            hcap *= 2;
            orc_hit* nh = (orc_hit*)realloc(hits, sizeof(orc_hit) * hcap);
            if (!nh) { free(hits); return -1; }
            hits = nh;
          }
          orc_hit* h = hits + nhit++;
          h->j = j;
          h->s[0] = s[0]; h->s[1] = s[1]; h->s[2] = s[2];
          h->d[0] = dx; h->d[1] = dy; h->d[2] = dz;
        }
      }
  qsort(hits, nhit, sizeof(orc_hit), orc_hit_cmp);
  for (int k = 0; k < nhit && k < cap; ++k) {
    if (js) js[k] = hits[k].j;
    if (sh) { sh[3 * k] = hits[k].s[0]; sh[3 * k + 1] = hits[k].s[1]; sh[3 * k + 2] = hits[k].s[2]; }
    if (d) { d[3 * k] = hits[k].d[0]; d[3 * k + 1] = hits[k].d[1]; d[3 * k + 2] = hits[k].d[2]; }
  }
  free(hits);
  return nhit;
}

/* ----------------------------------------------------- per-atom geometry */

typedef struct {
  int n, K;
  double* r;   /* n */
  double* u;   /* n x 3 unit vectors */
  double* R;   /* n x K */
  double* dR;  /* n x K */
} orc_geom;

static void orc_geom_init(orc_geom* g, const orc_params* p, const double* Q, int n, const double* d) {
  g->n = n;
  g->K = orc_num_radial(p);
  g->r = (double*)malloc(sizeof(double) * (n + 1));
  g->u = (double*)malloc(sizeof(double) * 3 * (n + 1));
  g->R = (double*)malloc(sizeof(double) * g->K * (n + 1));
  g->dR = (double*)malloc(sizeof(double) * g->K * (n + 1));
  for (int j = 0; j < n; ++j) {
    const double x = d[3 * j], y = d[3 * j + 1], z = d[3 * j + 2];
    const double r = sqrt(x * x + y * y + z * z);
    g->r[j] = r;
    g->u[3 * j] = x / r;
    g->u[3 * j + 1] = y / r;
    g->u[3 * j + 2] = z / r;
    orc_radial(p, Q, g->K, r, g->R + (size_t)j * g->K, g->dR + (size_t)j * g->K);
  }
}

static void orc_geom_free(orc_geom* g) {
  free(g->r);
  free(g->u);
  free(g->R);
  free(g->dR);
}

static double orc_dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double orc_ipow(double x, int n) {
  double v = 1.0;
  for (int t = 0; t < n; ++t) v *= x;
  return v;
}

/* d w / d r_a where w = u_a . u_b :  (u_b - w u_a) / r_a */
static void orc_dw(const double* ua, const double* ub, double w, double ra, double* out) {
  for (int t = 0; t < 3; ++t) out[t] = (ub[t] - w * ua[t]) / ra;
}

/* ------------------------------------------- naive descriptors (Eq. 12b, 15, 18a) */

int orc_atom_descriptors_naive(const orc_params* p, const double* Q, int n, const double* d, double* D) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  const int K = g.K;
  int col = 0;
  D[col++] = 1.0; /* one-body descriptor */
  for (int m = 0; m < p->K2; ++m) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += g.R[j * K + m];
    D[col++] = s;
  }
  if (p->P3 >= 0) {
    for (int m = 0; m < p->K3; ++m)
      for (int nn = 0; nn <= p->P3; ++nn) {
        double s = 0.0;
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) {
            const double w = orc_dot3(g.u + 3 * j, g.u + 3 * k);
            s += g.R[j * K + m] * g.R[k * K + m] * orc_ipow(w, nn);
          }
        D[col++] = s;
      }
  }
  if (p->P4 >= 0) {
    int abc[3 * 512];
    const int Ka = orc_fourbody_table(p->P4, abc);
    for (int m = 0; m < p->K4; ++m)
      for (int q = 0; q < Ka; ++q) {
        const int a = abc[3 * q], b = abc[3 * q + 1], c = abc[3 * q + 2];
        double s = 0.0;
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) {
            const double w1 = orc_dot3(g.u + 3 * j, g.u + 3 * k);
            for (int l = 0; l < n; ++l) {
              const double w2 = orc_dot3(g.u + 3 * j, g.u + 3 * l);
              const double w3 = orc_dot3(g.u + 3 * k, g.u + 3 * l);
              s += g.R[j * K + m] * g.R[k * K + m] * g.R[l * K + m] * orc_ipow(w1, a) * orc_ipow(w2, b) *
                   orc_ipow(w3, c);
            }
          }
        D[col++] = s;
      }
  }
  orc_geom_free(&g);
  return col;
}

/* Derivatives of the naive sums with respect to each neighbour's relative
 * position r_ij: dD[j][col][3].  Each summand is differentiated with respect to
 * each of its vector arguments and the result added to that argument's slot, so
 * repeated indices (j = k, ...) are handled by the product rule. */
int orc_atom_dD_naive(const orc_params* p, const double* Q, int n, const double* d, double* dD) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  const int K = g.K;
  const int M = orc_num_descriptors(p);
  memset(dD, 0, sizeof(double) * (size_t)n * M * 3);
#define DD(j, c, t) dD[((size_t)(j) * M + (c)) * 3 + (t)]
  int col0 = 1;
  for (int m = 0; m < p->K2; ++m)
    for (int j = 0; j < n; ++j)
      for (int t = 0; t < 3; ++t) DD(j, col0 + m, t) += g.dR[j * K + m] * g.u[3 * j + t];
  col0 += p->K2;
  if (p->P3 >= 0) {
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        const double* uj = g.u + 3 * j;
        const double* uk = g.u + 3 * k;
        const double w = orc_dot3(uj, uk);
        double dwj[3], dwk[3];
        orc_dw(uj, uk, w, g.r[j], dwj);
        orc_dw(uk, uj, w, g.r[k], dwk);
        for (int m = 0; m < p->K3; ++m) {
          const double Rj = g.R[j * K + m], Rk = g.R[k * K + m];
          const double dRj = g.dR[j * K + m], dRk = g.dR[k * K + m];
          for (int nn = 0; nn <= p->P3; ++nn) {
            const int c = col0 + m * (p->P3 + 1) + nn;
            const double wn = orc_ipow(w, nn);
            const double dwn = nn > 0 ? nn * orc_ipow(w, nn - 1) : 0.0;
            for (int t = 0; t < 3; ++t) {
              DD(j, c, t) += dRj * uj[t] * Rk * wn + Rj * Rk * dwn * dwj[t];
              DD(k, c, t) += Rj * dRk * uk[t] * wn + Rj * Rk * dwn * dwk[t];
            }
          }
        }
      }
    col0 += p->K3 * (p->P3 + 1);
  }
  if (p->P4 >= 0) {
    int abc[3 * 512];
    const int Ka = orc_fourbody_table(p->P4, abc);
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
          const double *uj = g.u + 3 * j, *uk = g.u + 3 * k, *ul = g.u + 3 * l;
          const double w1 = orc_dot3(uj, uk), w2 = orc_dot3(uj, ul), w3 = orc_dot3(uk, ul);
          double d1j[3], d1k[3], d2j[3], d2l[3], d3k[3], d3l[3];
          orc_dw(uj, uk, w1, g.r[j], d1j);
          orc_dw(uk, uj, w1, g.r[k], d1k);
          orc_dw(uj, ul, w2, g.r[j], d2j);
          orc_dw(ul, uj, w2, g.r[l], d2l);
          orc_dw(uk, ul, w3, g.r[k], d3k);
          orc_dw(ul, uk, w3, g.r[l], d3l);
          for (int q = 0; q < Ka; ++q) {
            const int a = abc[3 * q], b = abc[3 * q + 1], c = abc[3 * q + 2];
            const double f = orc_ipow(w1, a) * orc_ipow(w2, b) * orc_ipow(w3, c);
            const double f1 = a ? a * orc_ipow(w1, a - 1) * orc_ipow(w2, b) * orc_ipow(w3, c) : 0.0;
            const double f2 = b ? b * orc_ipow(w1, a) * orc_ipow(w2, b - 1) * orc_ipow(w3, c) : 0.0;
            const double f3 = c ? c * orc_ipow(w1, a) * orc_ipow(w2, b) * orc_ipow(w3, c - 1) : 0.0;
            for (int m = 0; m < p->K4; ++m) {
              const int cc = col0 + m * Ka + q;
              const double Rj = g.R[j * K + m], Rk = g.R[k * K + m], Rl = g.R[l * K + m];
              const double RRR = Rj * Rk * Rl;
              for (int t = 0; t < 3; ++t) {
                DD(j, cc, t) += g.dR[j * K + m] * uj[t] * Rk * Rl * f + RRR * (f1 * d1j[t] + f2 * d2j[t]);
                DD(k, cc, t) += Rj * g.dR[k * K + m] * uk[t] * Rl * f + RRR * (f1 * d1k[t] + f3 * d3k[t]);
                DD(l, cc, t) += Rj * Rk * g.dR[l * K + m] * ul[t] * f + RRR * (f2 * d2l[t] + f3 * d3l[t]);
              }
            }
          }
        }
  }
#undef DD
  orc_geom_free(&g);
  return M;
}

/* ------------------------------- atom-density form (Eq. 24b, 26a, 27a, 30a) */

typedef struct {
  int P, NA;
  int exps[3 * 400];
  double mu[400];
  int deg[400];
  int index[ORC_MAXP + 1][ORC_MAXP + 1][ORC_MAXP + 1]; /* exponent triple -> monomial index */
} orc_mono;

static void orc_mono_init(orc_mono* mo, int P) {
  mo->P = P;
  mo->NA = orc_monomial_table(P, mo->exps, mo->mu);
  for (int x = 0; x < mo->NA; ++x) {
    const int* e = mo->exps + 3 * x;
    mo->deg[x] = e[0] + e[1] + e[2];
    mo->index[e[0]][e[1]][e[2]] = x;
  }
}

static double orc_mono_eval(const int* e, const double* u) {
  return orc_ipow(u[0], e[0]) * orc_ipow(u[1], e[1]) * orc_ipow(u[2], e[2]);
}

/* d A_e(u(r)) / d r  =  (grad_u A_e - n A_e u) / r  (u = r / |r|, A homogeneous of degree n) */
static void orc_mono_grad(const int* e, const double* u, double r, double* out) {
  const int n = e[0] + e[1] + e[2];
  const double A = orc_mono_eval(e, u);
  for (int t = 0; t < 3; ++t) {
    double ga = 0.0;
    if (e[t] > 0) {
      int el[3] = {e[0], e[1], e[2]};
      el[t] -= 1;
      ga = e[t] * orc_mono_eval(el, u);
    }
    out[t] = (ga - n * A * u[t]) / r;
  }
}

/* B[m][x] = sum_j R_m(r_ij) A_x(u_ij), Eq. 24b. */
static void orc_atomic_basis(const orc_geom* g, const orc_mono* mo, double* B) {
  const int K = g->K, NA = mo->NA;
  memset(B, 0, sizeof(double) * K * NA);
  for (int j = 0; j < g->n; ++j)
    for (int x = 0; x < NA; ++x) {
      const double A = orc_mono_eval(mo->exps + 3 * x, g->u + 3 * j);
      for (int m = 0; m < K; ++m) B[m * NA + x] += g->R[j * K + m] * A;
    }
}

/* D3_mn = sum_{x of degree n} mu_x B_mx^2, Eq. 26a */
static double orc_fast_d3(const orc_mono* mo, const double* Bm, int n) {
  double s = 0.0;
  for (int x = 0; x < mo->NA; ++x)
    if (mo->deg[x] == n) s += mo->mu[x] * Bm[x] * Bm[x];
  return s;
}

/* D4 for partition (a, b, c); with G != NULL also accumulate wt * dD4/dB_m into G. */
static double orc_fast_d4(const orc_mono* mo, const double* Bm, int a, int b, int c, double wt, double* G) {
  if (b == 0 && c == 0) { /* Eq. 27a: D4 = D2 * D3_a */
    const double d3 = orc_fast_d3(mo, Bm, a);
    if (G) {
      G[0] += wt * d3;
      for (int x = 0; x < mo->NA; ++x)
        if (mo->deg[x] == a) G[x] += wt * Bm[0] * 2.0 * mo->mu[x] * Bm[x];
    }
    return Bm[0] * d3;
  }
  /* Eq. 30a: sum over monomials q (deg a), s (deg b), t (deg c) */
  double s = 0.0;
  for (int q = 0; q < mo->NA; ++q) {
    if (mo->deg[q] != a) continue;
    for (int sidx = 0; sidx < mo->NA; ++sidx) {
      if (mo->deg[sidx] != b) continue;
      for (int t = 0; t < mo->NA; ++t) {
        if (mo->deg[t] != c) continue;
        const int *eq = mo->exps + 3 * q, *es = mo->exps + 3 * sidx, *et = mo->exps + 3 * t;
        const int x1 = mo->index[eq[0] + es[0]][eq[1] + es[1]][eq[2] + es[2]];
        const int x2 = mo->index[eq[0] + et[0]][eq[1] + et[1]][eq[2] + et[2]];
        const int x3 = mo->index[es[0] + et[0]][es[1] + et[1]][es[2] + et[2]];
        const double cf = mo->mu[q] * mo->mu[sidx] * mo->mu[t];
        s += cf * Bm[x1] * Bm[x2] * Bm[x3];
        if (G) {
          G[x1] += wt * cf * Bm[x2] * Bm[x3];
          G[x2] += wt * cf * Bm[x1] * Bm[x3];
          G[x3] += wt * cf * Bm[x1] * Bm[x2];
        }
      }
    }
  }
  return s;
}

int orc_atom_descriptors_fast(const orc_params* p, const double* Q, int n, const double* d, double* D) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  orc_mono mo;
  orc_mono_init(&mo, imax(0, orc_max_degree(p)));  /* D2 = B_m00 needs degree 0 */
  const int K = g.K, NA = mo.NA;
  double* B = (double*)malloc(sizeof(double) * K * NA);
  orc_atomic_basis(&g, &mo, B);
  int col = 0;
  D[col++] = 1.0;
  for (int m = 0; m < p->K2; ++m) D[col++] = B[m * NA + 0];
  if (p->P3 >= 0)
    for (int m = 0; m < p->K3; ++m)
      for (int nn = 0; nn <= p->P3; ++nn) D[col++] = orc_fast_d3(&mo, B + m * NA, nn);
  if (p->P4 >= 0) {
    int abc[3 * 512];
    const int Ka = orc_fourbody_table(p->P4, abc);
    for (int m = 0; m < p->K4; ++m)
      for (int q = 0; q < Ka; ++q)
        D[col++] = orc_fast_d4(&mo, B + m * NA, abc[3 * q], abc[3 * q + 1], abc[3 * q + 2], 0.0, NULL);
  }
  free(B);
  orc_geom_free(&g);
  return col;
}

/* Adjoint of the linear energy E_i = sum_col c_col D_col with respect to B:
 * G[m][x] = dE_i / dB_mx (Eq. 26c generalised to every body order). */
static double orc_fast_energy_adjoint(const orc_params* p, const orc_mono* mo, int K, const double* B,
                                      const double* c, double* G) {
  const int NA = mo->NA;
  memset(G, 0, sizeof(double) * K * NA);
  int col = 0;
  double E = c[col++];
  for (int m = 0; m < p->K2; ++m) {
    E += c[col] * B[m * NA];
    G[m * NA] += c[col];
    ++col;
  }
  if (p->P3 >= 0)
    for (int m = 0; m < p->K3; ++m)
      for (int nn = 0; nn <= p->P3; ++nn) {
        const double* Bm = B + m * NA;
        E += c[col] * orc_fast_d3(mo, Bm, nn);
        for (int x = 0; x < NA; ++x)
          if (mo->deg[x] == nn) G[m * NA + x] += c[col] * 2.0 * mo->mu[x] * Bm[x];
        ++col;
      }
  if (p->P4 >= 0) {
    int abc[3 * 512];
    const int Ka = orc_fourbody_table(p->P4, abc);
    for (int m = 0; m < p->K4; ++m)
      for (int q = 0; q < Ka; ++q) {
        E += c[col] * orc_fast_d4(mo, B + m * NA, abc[3 * q], abc[3 * q + 1], abc[3 * q + 2], c[col],
                                  G + m * NA);
        ++col;
      }
  }
  return E;
}

/* g_j = sum_{m,x} G_mx dB_mx / dr_ij  with  dB/dr = R' A u + R dA/dr  (Eq. 24c). */
static void orc_pair_contract(const orc_geom* g, const orc_mono* mo, const double* G, double* out) {
  const int K = g->K, NA = mo->NA;
  for (int j = 0; j < g->n; ++j) {
    const double* u = g->u + 3 * j;
    double acc[3] = {0, 0, 0};
    for (int x = 0; x < NA; ++x) {
      const double A = orc_mono_eval(mo->exps + 3 * x, u);
      double dA[3];
      orc_mono_grad(mo->exps + 3 * x, u, g->r[j], dA);
      for (int m = 0; m < K; ++m) {
        const double gm = G[m * NA + x];
        if (gm == 0.0) continue;
        const double R = g->R[j * K + m], dR = g->dR[j * K + m];
        for (int t = 0; t < 3; ++t) acc[t] += gm * (dR * A * u[t] + R * dA[t]);
      }
    }
    out[3 * j] = acc[0];
    out[3 * j + 1] = acc[1];
    out[3 * j + 2] = acc[2];
  }
}

/* Atom energy E_i and dE_i/dr_ij for every neighbour (atom-density form). */
double orc_atom_energy_grad_fast(const orc_params* p, const double* Q, const double* c, int n, const double* d,
                                 double* grad) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  orc_mono mo;
  orc_mono_init(&mo, imax(0, orc_max_degree(p)));  /* D2 = B_m00 needs degree 0 */
  const int K = g.K, NA = mo.NA;
  double* B = (double*)malloc(sizeof(double) * K * NA);
  double* G = (double*)malloc(sizeof(double) * K * NA);
  orc_atomic_basis(&g, &mo, B);
  const double E = orc_fast_energy_adjoint(p, &mo, K, B, c, G);
  if (grad) orc_pair_contract(&g, &mo, G, grad);
  free(B);
  free(G);
  orc_geom_free(&g);
  return E;
}

/* Linear-model atom energies and forces over the atoms [i0, i1) of a system,
 * through the cell list and the atom-density form above: Ei[i] = E_i, and every
 * pair gradient g_ij = dE_i/dr_ij added to F[i] and subtracted from F[j]
 * (F: N x 3, accumulated, not cleared), W -= r_ij (x) g_ij (3 x 3, accumulated).
 * With escale != NULL also escale[i] = sum_m |c_m D_im| (the scale of the
 * energy tolerance), from the atom's descriptors.
 * Returns the largest neighbour count, or -1 when it exceeds cap. */
int orc_energy_forces_range(const orc_params* p, const double* Q, const double* c, const orc_cells* cl,
                            double rcut, int i0, int i1, int cap, double* Ei, double* F, double* W,
                            double* escale) {
  const int M = orc_num_descriptors(p);
  double* Dv = escale ? (double*)malloc(sizeof(double) * M) : NULL;
  int* js = (int*)malloc(sizeof(int) * cap);
  double* d = (double*)malloc(sizeof(double) * 3 * cap);
  double* g = (double*)malloc(sizeof(double) * 3 * cap);
  int nmax = 0;
  if (!js || !d || !g) { free(js); free(d); free(g); return -1; }
  for (int i = i0; i < i1; ++i) {
    const int n = orc_cells_neighbors_of(cl, rcut, i, cap, js, NULL, d);
    if (n < 0 || n > cap) { nmax = -1; break; }
    if (n > nmax) nmax = n;
    Ei[i] = orc_atom_energy_grad_fast(p, Q, c, n, d, g);
    if (escale) {
      orc_atom_descriptors_fast(p, Q, n, d, Dv);
      double sc = 0.0;
      for (int q = 0; q < M; ++q) sc += fabs(c[q] * Dv[q]);
      escale[i] = sc;
    }
    for (int k = 0; k < n; ++k)
      for (int t = 0; t < 3; ++t) {
        F[3 * i + t] += g[3 * k + t];
        F[3 * js[k] + t] -= g[3 * k + t];
        for (int a = 0; a < 3; ++a) W[3 * a + t] -= d[3 * k + a] * g[3 * k + t];
      }
  }
  free(js);
  free(d);
  free(g);
  free(Dv);
  return nmax;
}

/* Explicit descriptor derivatives dD[j][col][3] in the atom-density form: for
 * each column the adjoint dD_col/dB is formed and contracted with dB/dr_ij. */
int orc_atom_dD_fast(const orc_params* p, const double* Q, int n, const double* d, double* dD) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  orc_mono mo;
  orc_mono_init(&mo, imax(0, orc_max_degree(p)));  /* D2 = B_m00 needs degree 0 */
  const int K = g.K, NA = mo.NA;
  const int M = orc_num_descriptors(p);
  double* B = (double*)malloc(sizeof(double) * K * NA);
  double* G = (double*)malloc(sizeof(double) * K * NA);
  double* tmp = (double*)malloc(sizeof(double) * 3 * (n + 1));
  double* cvec = (double*)calloc(M, sizeof(double));
  orc_atomic_basis(&g, &mo, B);
  memset(dD, 0, sizeof(double) * (size_t)n * M * 3);
  for (int col = 1; col < M; ++col) {
    cvec[col] = 1.0;
    orc_fast_energy_adjoint(p, &mo, K, B, cvec, G);
    cvec[col] = 0.0;
    orc_pair_contract(&g, &mo, G, tmp);
    for (int j = 0; j < n; ++j)
      for (int t = 0; t < 3; ++t) dD[((size_t)j * M + col) * 3 + t] = tmp[3 * j + t];
  }
  free(cvec);
  free(tmp);
  free(B);
  free(G);
  orc_geom_free(&g);
  return M;
}

/* Exclusive three-body sums of the original POD (k > j), Eq. 15b -- used only to
 * check the relation of Eq. 15c.  out[m][n] for m < K3, n <= P3. */
void orc_atom_d3_exclusive(const orc_params* p, const double* Q, int n, const double* d, double* out) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  const int K = g.K;
  for (int m = 0; m < p->K3; ++m)
    for (int nn = 0; nn <= p->P3; ++nn) {
      double s = 0.0;
      for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k)
          s += g.R[j * K + m] * g.R[k * K + m] * orc_ipow(orc_dot3(g.u + 3 * j, g.u + 3 * k), nn);
      out[m * (p->P3 + 1) + nn] = s;
    }
  orc_geom_free(&g);
}

/* Symmetrised four-body functions g_p of Table 2 summed over all ordered
 * (j, k, l): out[m][p].  Used only for the check sum_{jkl} g_p = 3 D4_p. */
void orc_atom_g4_sums(const orc_params* p, const double* Q, int n, const double* d, double* out) {
  orc_geom g;
  orc_geom_init(&g, p, Q, n, d);
  const int K = g.K;
  int abc[3 * 512];
  const int Ka = orc_fourbody_table(p->P4, abc);
  for (int m = 0; m < p->K4; ++m)
    for (int q = 0; q < Ka; ++q) {
      const int a = abc[3 * q], b = abc[3 * q + 1], c = abc[3 * q + 2];
      double s = 0.0;
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k)
          for (int l = 0; l < n; ++l) {
            const double w1 = orc_dot3(g.u + 3 * j, g.u + 3 * k);
            const double w2 = orc_dot3(g.u + 3 * j, g.u + 3 * l);
            const double w3 = orc_dot3(g.u + 3 * k, g.u + 3 * l);
            const double gp = orc_ipow(w1, a) * orc_ipow(w2, b) * orc_ipow(w3, c) +
                              orc_ipow(w1, c) * orc_ipow(w2, a) * orc_ipow(w3, b) +
                              orc_ipow(w1, b) * orc_ipow(w2, c) * orc_ipow(w3, a);
            s += g.R[j * K + m] * g.R[k * K + m] * g.R[l * K + m] * gp;
          }
      out[m * Ka + q] = s;
    }
  orc_geom_free(&g);
}
