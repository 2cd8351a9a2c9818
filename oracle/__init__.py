"""Plain FP64 CPU oracle for fast POD descriptors, energies, forces and the fit.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this package.
It shares no code with the CUDA library (``paper_2212_14446_gb300``) and never
imports it.

The arithmetic lives in ``pod_oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module compiles it with gcc, calls it through ctypes and assembles per-atom
results into system quantities with numpy:

* ``descriptors``      -- Eq. 12b / Eq. 15 / Eq. 18a (naive) or Eq. 24b-30a (fast)
* ``energy_forces``    -- E_i = sum_m c_m D_im (Eq. 57a), E = sum_i E_i (Eq. 58a),
                          F_k = -dE/dr_k, virial W = -sum_ij r_ij (x) dE_i/dr_ij
* ``design_matrix`` / ``fit`` -- ridge least squares of Eq. 63a with energy rows
                          G_m / N against E / N (weight 100) and force rows
                          -dG_m / dr_k against F_k (weight 1), gamma = 1e-12
                          (Section 5); solved with numpy's SVD least squares.

Reading of the paper for the virial (the paper is silent):
W_ab = -sum_i sum_j (r_ij)_a dE_i/d(r_ij)_b.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pod_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CAP = 512  # neighbour capacity per atom for the oracle's lists


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("r_in", C.c_double), ("r_cut", C.c_double),
                ("n_alpha", C.c_int), ("alpha", C.POINTER(C.c_double)),
                ("n_beta", C.c_int), ("beta", C.POINTER(C.c_double)),
                ("n_gamma", C.c_int), ("gamma", C.POINTER(C.c_double)),
                ("K2", C.c_int), ("K3", C.c_int), ("K4", C.c_int), ("P3", C.c_int), ("P4", C.c_int)]


class _System(C.Structure):
    _fields_ = [("N", C.c_int), ("pos", C.POINTER(C.c_double)),
                ("box", C.c_double * 3), ("pbc", C.c_int * 3)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, ip, i, d = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int, C.c_double
            P, S = C.POINTER(_Params), C.POINTER(_System)
            sig = {
                "orc_num_snapshots": (i, [P]), "orc_num_radial": (i, [P]), "orc_max_degree": (i, [P]),
                "orc_num_monomials": (i, [i]), "orc_num_fourbody": (i, [i]),
                "orc_num_descriptors": (i, [P]), "orc_fourbody_table": (i, [i, ip]),
                "orc_monomial_table": (i, [i, ip, dp]), "orc_snapshots": (i, [P, d, dp, dp]),
                "orc_basis": (i, [P, i, i, dp, dp, dp]), "orc_radial_eval": (None, [P, dp, i, i, dp, dp, dp]),
                "orc_neighbors_of": (i, [S, d, i, i, ip, ip, dp]),
                "orc_cells_build": (C.c_void_p, [S, d]), "orc_cells_free": (None, [C.c_void_p]),
                "orc_cells_neighbors_of": (i, [C.c_void_p, d, i, i, ip, ip, dp]),
                "orc_energy_forces_range": (i, [P, dp, dp, C.c_void_p, d, i, i, i, dp, dp, dp, dp]),
                "orc_atom_descriptors_naive": (i, [P, dp, i, dp, dp]),
                "orc_atom_descriptors_fast": (i, [P, dp, i, dp, dp]),
                "orc_atom_dD_naive": (i, [P, dp, i, dp, dp]),
                "orc_atom_dD_fast": (i, [P, dp, i, dp, dp]),
                "orc_atom_energy_grad_fast": (d, [P, dp, dp, i, dp, dp]),
                "orc_atom_d3_exclusive": (None, [P, dp, i, dp, dp]),
                "orc_atom_g4_sums": (None, [P, dp, i, dp, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


# --------------------------------------------------------------------- tables

def monomial_table(P: int):
    """Exponents (N_a x 3) in Table 3 order and multinomial coefficients (Table 4)."""
    n = lib().orc_num_monomials(P)
    e = np.zeros((max(n, 1), 3), dtype=np.int32)
    c = np.zeros(max(n, 1))
    lib().orc_monomial_table(P, _ip(e), _dp(c))
    return e[:n], c[:n]


def fourbody_table(P4: int):
    """(a, b, c) of the four-body angular functions f_p (Table 1 order)."""
    n = lib().orc_num_fourbody(P4)
    t = np.zeros((max(n, 1), 3), dtype=np.int32)
    if n:
        lib().orc_fourbody_table(P4, _ip(t))
    return t[:n]


def num_fourbody(P4: int) -> int:
    return lib().orc_num_fourbody(P4)


def num_monomials(P: int) -> int:
    return lib().orc_num_monomials(P)


# ------------------------------------------------------------------- oracle

class _SysData:
    """One configuration as the oracle's C routines take it (atom-major FP64
    positions), with an optional cell list built by the C side."""

    def __init__(self, cfg, r_cut: float, cells: bool):
        self.pos = np.ascontiguousarray(cfg.pos, dtype=np.float64)
        self.s = _System(self.pos.shape[0], _dp(self.pos), (C.c_double * 3)(*cfg.box), (C.c_int * 3)(*cfg.pbc))
        self.cells = None
        if cells:
            self.cells = lib().orc_cells_build(C.byref(self.s), float(r_cut))
            if not self.cells:
                raise MemoryError("oracle cell list")

    def __del__(self):
        if getattr(self, "cells", None):
            lib().orc_cells_free(self.cells)
            self.cells = None


class Oracle:
    """FP64 oracle bound to one parameter set.  Q is computed by the oracle's own
    POD (Gram matrix + cyclic Jacobi) unless given."""

    def __init__(self, params, Q: np.ndarray | None = None):
        self.params = params
        self._alpha = np.ascontiguousarray(params.alpha, dtype=np.float64)
        self._beta = np.ascontiguousarray(params.beta, dtype=np.float64)
        self._gamma = np.ascontiguousarray(params.gamma, dtype=np.float64)
        self._p = _Params(params.r_in, params.r_cut, len(self._alpha), _dp(self._alpha),
                          len(self._beta), _dp(self._beta), len(self._gamma), _dp(self._gamma),
                          params.K2, params.K3, params.K4, params.P3, params.P4)
        self.pp = C.byref(self._p)
        L = lib()
        self.Ns = L.orc_num_snapshots(self.pp)
        self.K = L.orc_num_radial(self.pp)
        self.M = L.orc_num_descriptors(self.pp)
        self.Pa = L.orc_max_degree(self.pp)
        self.eig = np.zeros(self.Ns)
        self.gram = np.zeros((self.Ns, self.Ns))
        Qo = np.zeros((self.Ns, self.K))
        rc = L.orc_basis(self.pp, params.n_grid, self.K, _dp(Qo), _dp(self.eig), _dp(self.gram))
        if rc != 0:
            raise ValueError("oracle basis failed")
        self.Q_own = Qo
        self.Q = np.ascontiguousarray(Q if Q is not None else Qo, dtype=np.float64).reshape(self.Ns, self.K)

    # -- radial pieces
    def snapshots(self, r: float):
        phi = np.zeros(self.Ns)
        dphi = np.zeros(self.Ns)
        lib().orc_snapshots(self.pp, float(r), _dp(phi), _dp(dphi))
        return phi, dphi

    def radial(self, r: np.ndarray):
        r = np.ascontiguousarray(r, dtype=np.float64)
        R = np.zeros((r.size, self.K))
        dR = np.zeros((r.size, self.K))
        lib().orc_radial_eval(self.pp, _dp(self.Q), self.K, r.size, _dp(r), _dp(R), _dp(dR))
        return R, dR

    # -- neighbours
    # Two routes to the same list: the brute-force scan over every atom and image
    # (orc_neighbors_of, the definition), and a cell list (orc_cells_neighbors_of)
    # that the CPU tests pin to it entry for entry; systems of CELLS_MIN atoms or
    # more take the cell list.
    CELLS_MIN = 4096

    def _system(self, cfg, cells=None):
        return _SysData(cfg, self.params.r_cut, (cfg.n >= self.CELLS_MIN) if cells is None else cells)

    def neighbors(self, cfg, i: int, _sys=None):
        sd = _sys if _sys is not None else self._system(cfg)
        js = np.zeros(CAP, dtype=np.int32)
        sh = np.zeros((CAP, 3), dtype=np.int32)
        d = np.zeros((CAP, 3))
        if sd.cells:
            n = lib().orc_cells_neighbors_of(sd.cells, self.params.r_cut, int(i), CAP, _ip(js), _ip(sh), _dp(d))
        else:
            n = lib().orc_neighbors_of(C.byref(sd.s), self.params.r_cut, int(i), CAP, _ip(js), _ip(sh), _dp(d))
        if n < 0:
            raise MemoryError("oracle neighbour search")
        if n > CAP:
            raise ValueError("oracle neighbour capacity exceeded")
        return js[:n].copy(), sh[:n].copy(), d[:n].copy()

    def neighbor_lists(self, cfg, atoms=None, cells=None):
        sysd = self._system(cfg, cells)
        atoms = range(cfg.n) if atoms is None else atoms
        return [self.neighbors(cfg, i, sysd) for i in atoms]

    # -- descriptors of one atom from its displacement list
    def atom_descriptors(self, d: np.ndarray, fast: bool = False) -> np.ndarray:
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        D = np.zeros(self.M)
        fn = lib().orc_atom_descriptors_fast if fast else lib().orc_atom_descriptors_naive
        fn(self.pp, _dp(self.Q), d.shape[0], _dp(d), _dp(D))
        return D

    def atom_dD(self, d: np.ndarray, fast: bool = False) -> np.ndarray:
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((d.shape[0], self.M, 3))
        fn = lib().orc_atom_dD_fast if fast else lib().orc_atom_dD_naive
        fn(self.pp, _dp(self.Q), d.shape[0], _dp(d), _dp(out))
        return out

    def atom_energy_grad(self, d: np.ndarray, c: np.ndarray):
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        c = np.ascontiguousarray(c, dtype=np.float64)
        g = np.zeros((d.shape[0], 3))
        E = lib().orc_atom_energy_grad_fast(self.pp, _dp(self.Q), _dp(c), d.shape[0], _dp(d), _dp(g))
        return E, g

    def atom_d3_exclusive(self, d):
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((self.params.K3, self.params.P3 + 1))
        lib().orc_atom_d3_exclusive(self.pp, _dp(self.Q), d.shape[0], _dp(d), _dp(out))
        return out

    def atom_g4_sums(self, d):
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((self.params.K4, num_fourbody(self.params.P4)))
        lib().orc_atom_g4_sums(self.pp, _dp(self.Q), d.shape[0], _dp(d), _dp(out))
        return out

    # -- system quantities
    def descriptors(self, cfg, atoms=None, fast: bool = False) -> np.ndarray:
        atoms = list(range(cfg.n)) if atoms is None else list(atoms)
        sysd = self._system(cfg)
        out = np.zeros((len(atoms), self.M))
        for a, i in enumerate(atoms):
            _, _, d = self.neighbors(cfg, i, sysd)
            out[a] = self.atom_descriptors(d, fast)
        return out

    def pair_grads(self, cfg, c, atoms, fast: bool = True):
        """For each atom i in ``atoms``: (E_i, js, shifts, d, dE_i/dr_ij)."""
        sysd = self._system(cfg)
        res = {}
        for i in atoms:
            js, sh, d = self.neighbors(cfg, i, sysd)
            if fast:
                E, g = self.atom_energy_grad(d, c)
            else:
                D = self.atom_descriptors(d, fast=False)
                dD = self.atom_dD(d, fast=False)
                E = float(D @ c)
                g = np.einsum("jmt,m->jt", dD, c)
            res[int(i)] = (E, js, sh, d, g)
        return res

    def energy_forces(self, cfg, c, fast: bool = True, force_atoms=None):
        """Atom energies, total energy, forces and virial.

        With ``force_atoms`` given, only those atoms' forces are formed (from the
        pair gradients of every atom whose list touches them) and the virial is
        not computed (returned as None)."""
        c = np.asarray(c, dtype=np.float64)
        if force_atoms is None:
            pg = self.pair_grads(cfg, c, range(cfg.n), fast)
            Ei = np.array([pg[i][0] for i in range(cfg.n)])
            F = np.zeros((cfg.n, 3))
            W = np.zeros((3, 3))
            for i in range(cfg.n):
                _, js, _, d, g = pg[i]
                F[i] += g.sum(axis=0)
                np.subtract.at(F, js, g)
                W -= d.T @ g
            return Ei, math.fsum(Ei), F, W
        force_atoms = [int(k) for k in force_atoms]
        need = set(force_atoms)
        sysd = self._system(cfg)
        for k in force_atoms:
            js, _, _ = self.neighbors(cfg, k, sysd)
            need.update(int(j) for j in js)
        pg = self.pair_grads(cfg, c, sorted(need), fast)
        F = np.zeros((len(force_atoms), 3))
        for a, k in enumerate(force_atoms):
            _, js, _, _, g = pg[k]
            F[a] += g.sum(axis=0)
            for i in need:
                _, jsi, _, _, gi = pg[i]
                sel = jsi == k
                if np.any(sel):
                    F[a] -= gi[sel].sum(axis=0)
        Ei = {i: pg[i][0] for i in need}
        return Ei, None, F, None

    def energy_forces_local(self, cfg, c, n_local: int, fast: bool = True):
        """Atoms [0, n_local) local, the rest ghosts: E and W of the local atoms'
        terms (Eq. 57a), forces on every atom from those terms (a ghost receives
        the reactions -g_ij of its local neighbours' pair gradients)."""
        c = np.asarray(c, dtype=np.float64)
        pg = self.pair_grads(cfg, c, range(n_local), fast)
        Ei = np.zeros(cfg.n)
        F = np.zeros((cfg.n, 3))
        W = np.zeros((3, 3))
        for i in range(n_local):
            Ei[i], js, _, d, g = pg[i]
            F[i] += g.sum(axis=0)
            np.subtract.at(F, js, g)
            W -= d.T @ g
        return Ei, math.fsum(Ei[:n_local]), F, W

    def energy_forces_quadratic(self, cfg, c, beta, fast: bool = True):
        """Quadratic model of Sec. 4 (the extension of Eq. 57a by products of
        descriptors): E_i = sum_m c_m D_im + sum_{m <= n} beta_mn D_im D_in, with
        the upper triangle of ``beta`` read.  Forces from the explicit descriptor
        derivatives: dE_i/dr_ij = sum_m (c_m + sum_n S_mn D_in) dD_im/dr_ij with
        S = beta_upper + beta_upper^T, assembled like ``energy_forces``."""
        c = np.asarray(c, dtype=np.float64)
        bu = np.triu(np.asarray(beta, dtype=np.float64))
        S = bu + bu.T
        sysd = self._system(cfg)
        Ei = np.zeros(cfg.n)
        F = np.zeros((cfg.n, 3))
        W = np.zeros((3, 3))
        for i in range(cfg.n):
            js, _, d = self.neighbors(cfg, i, sysd)
            D = self.atom_descriptors(d, fast)
            Ei[i] = D @ c + D @ bu @ D
            if len(js) == 0:
                continue
            dD = self.atom_dD(d, fast)              # (n_j, M, 3): dD_im / dr_ij
            g = np.einsum("jmt,m->jt", dD, c + S @ D)
            F[i] += g.sum(axis=0)
            np.subtract.at(F, js, g)
            W -= d.T @ g
        return Ei, math.fsum(Ei), F, W

    def exclusive3_descriptors(self, d: np.ndarray, fast: bool = True) -> np.ndarray:
        """Descriptors of one atom with the three-body columns replaced by the
        exclusive sums of the original POD over pairs k > j (Eq. 15b), formed from
        the inclusive ones by Eq. 15c: (D3_mn - sum_j R_m(r_j)^2) / 2."""
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        D = np.array(self.atom_descriptors(d, fast), dtype=np.float64)
        if d.shape[0] == 0:
            return D
        R, _ = self.radial(np.linalg.norm(d, axis=1))
        S = np.sum(R * R, axis=0)
        p = self.params
        col3, n3 = 1 + p.K2, p.P3 + 1
        for m in range(p.K3):
            D[col3 + m * n3: col3 + (m + 1) * n3] = 0.5 * (D[col3 + m * n3: col3 + (m + 1) * n3] - S[m])
        return D

    def energy_forces_exclusive3(self, cfg, c, fast: bool = True):
        """Linear model on the exclusive three-body set (Eq. 15b):
        E_i = c . Dx_i with ``exclusive3_descriptors``.  Forces from the explicit
        derivatives: dDx_i,col/dr_ij = (dD3_i,col/dr_ij - 2 R_m R'_m r_ij / r) / 2 on
        the three-body columns of mode m, assembled like ``energy_forces``."""
        c = np.asarray(c, dtype=np.float64)
        p = self.params
        col3, n3 = 1 + p.K2, p.P3 + 1
        sysd = self._system(cfg)
        Ei = np.zeros(cfg.n)
        F = np.zeros((cfg.n, 3))
        W = np.zeros((3, 3))
        for i in range(cfg.n):
            js, _, d = self.neighbors(cfg, i, sysd)
            Ei[i] = self.exclusive3_descriptors(d, fast) @ c
            if len(js) == 0:
                continue
            dD = np.array(self.atom_dD(d, fast))    # (n_j, M, 3): dD_im / dr_ij
            r = np.linalg.norm(d, axis=1)
            R, dR = self.radial(r)
            u = d / r[:, None]
            for m in range(p.K3):
                dS = 2.0 * (R[:, m] * dR[:, m])[:, None] * u    # (n_j, 3)
                for n in range(n3):
                    dD[:, col3 + m * n3 + n, :] = 0.5 * (dD[:, col3 + m * n3 + n, :] - dS)
            g = np.einsum("jmt,m->jt", dD, c)
            F[i] += g.sum(axis=0)
            np.subtract.at(F, js, g)
            W -= d.T @ g
        return Ei, math.fsum(Ei), F, W

    def energy_forces_embedding(self, cfg, c, a, alpha, fast: bool = True):
        """Embedding model of Sec. 3 (EAM and MEAM written with POD descriptors):
        E_i = sum_m c_m D_im + F(rho_i) with the density rho_i = sum_m a_m D_im and
        the polynomial embedding F(rho) = sum_k alpha_k rho^k.  Forces from the
        explicit descriptor derivatives: dE_i/dr_ij = sum_m (c_m + F'(rho_i) a_m)
        dD_im/dr_ij, assembled like ``energy_forces``."""
        c = np.asarray(c, dtype=np.float64)
        a = np.asarray(a, dtype=np.float64)
        alpha = np.asarray(alpha, dtype=np.float64)
        F_poly = np.polynomial.Polynomial(alpha)
        dF_poly = F_poly.deriv()
        sysd = self._system(cfg)
        Ei = np.zeros(cfg.n)
        F = np.zeros((cfg.n, 3))
        W = np.zeros((3, 3))
        for i in range(cfg.n):
            js, _, d = self.neighbors(cfg, i, sysd)
            D = self.atom_descriptors(d, fast)
            rho = float(D @ a)
            Ei[i] = D @ c + F_poly(rho)
            if len(js) == 0:
                continue
            dD = self.atom_dD(d, fast)              # (n_j, M, 3): dD_im / dr_ij
            g = np.einsum("jmt,m->jt", dD, c + dF_poly(rho) * a)
            F[i] += g.sum(axis=0)
            np.subtract.at(F, js, g)
            W -= d.T @ g
        return Ei, math.fsum(Ei), F, W

    def energy_forces_cells(self, cfg, c, threads: int = 1, cap: int = CAP, atom_range=None, escale=None):
        """Linear-model E_i, E, F and W of every atom through the cell list and the
        atom-density form (Eq. 24b, 26a, 27a, 30a and their adjoint), in C over
        chunks of atoms on `threads` host threads (each with its own force and
        virial accumulators, summed afterwards).  The faster CPU route to the
        quantities of ``energy_forces``; the CPU tests pin the two together.
        With ``atom_range`` = (i0, i1) only those atoms' energy terms are formed
        (their pair gradients still reach every atom's force).  With ``escale``
        an array of N, escale[i] receives sum_m |c_m D_im| (the energy-error scale
        of the tolerances)."""
        import concurrent.futures as cf
        c = np.ascontiguousarray(c, dtype=np.float64)
        sd = self._system(cfg, cells=True)
        N = cfg.n
        i0, i1 = (0, N) if atom_range is None else (int(atom_range[0]), int(atom_range[1]))
        Ei = np.zeros(N)
        T = max(1, min(int(threads), i1 - i0))
        Fs = [np.zeros((N, 3)) for _ in range(T)]
        Ws = [np.zeros((3, 3)) for _ in range(T)]
        bounds = [i0 + (i1 - i0) * t // T for t in range(T + 1)]

        def run(t):
            return lib().orc_energy_forces_range(self.pp, _dp(self.Q), _dp(c), sd.cells, self.params.r_cut,
                                                 bounds[t], bounds[t + 1], int(cap), _dp(Ei), _dp(Fs[t]),
                                                 _dp(Ws[t]), _dp(escale) if escale is not None else None)

        if T == 1:
            res = [run(0)]
        else:
            with cf.ThreadPoolExecutor(max_workers=T) as ex:
                res = list(ex.map(run, range(T)))
        if min(res) < 0:
            raise ValueError("oracle neighbour capacity exceeded")
        F = Fs[0]
        for t in range(1, T):
            F += Fs[t]
        W = Ws[0]
        for t in range(1, T):
            W += Ws[t]
        return Ei, math.fsum(Ei), F, W

    # -- fit (Eq. 63a)
    def config_rows(self, cfg, fast: bool = True):
        """Global descriptors G (M,) and dG/dr_k (N, 3, M) of one configuration."""
        sysd = self._system(cfg)
        G = np.zeros(self.M)
        dG = np.zeros((cfg.n, 3, self.M))
        for i in range(cfg.n):
            js, _, d = self.neighbors(cfg, i, sysd)
            G += self.atom_descriptors(d, fast)
            dD = self.atom_dD(d, fast)              # (n, M, 3)
            dG[i] -= dD.sum(axis=0).T
            np.add.at(dG, js, dD.transpose(0, 2, 1))
        return G, dG

    def design_matrix(self, configs, E_ref, F_ref, w_E=100.0, w_F=1.0, fast=True):
        rows, rhs = [], []
        for cfg, E, F in zip(configs, E_ref, F_ref):
            G, dG = self.config_rows(cfg, fast)
            rows.append(w_E * G[None, :] / cfg.n)
            rhs.append(np.array([w_E * E / cfg.n]))
            rows.append(w_F * (-dG.reshape(-1, self.M)))
            rhs.append(w_F * np.asarray(F, dtype=np.float64).reshape(-1))
        return np.vstack(rows), np.concatenate(rhs)

    def normal_equations(self, configs, E_ref, F_ref, w_E=100.0, w_F=1.0, gamma=1e-12, fast=True, threads=1):
        """A^T A + gamma I and A^T b of ``design_matrix`` (Eq. 63a), each
        configuration's block of rows formed on one of `threads` host threads and
        the blocks' products summed in configuration order."""
        import concurrent.futures as cf

        def block(k):
            A, b = self.design_matrix([configs[k]], [E_ref[k]], [F_ref[k]], w_E, w_F, fast)
            return A.T @ A, A.T @ b

        if threads <= 1:
            parts = [block(k) for k in range(len(configs))]
        else:
            with cf.ThreadPoolExecutor(max_workers=threads) as ex:
                parts = list(ex.map(block, range(len(configs))))
        G = np.zeros((self.M, self.M))
        r = np.zeros(self.M)
        for Gk, rk in parts:
            G += Gk
            r += rk
        G += gamma * np.eye(self.M)
        return G, r

    def fit(self, configs, E_ref, F_ref, w_E=100.0, w_F=1.0, gamma=1e-12, fast=True):
        A, b = self.design_matrix(configs, E_ref, F_ref, w_E, w_F, fast)
        Aa = np.vstack([A, math.sqrt(gamma) * np.eye(self.M)])
        ba = np.concatenate([b, np.zeros(self.M)])
        c, *_ = np.linalg.lstsq(Aa, ba, rcond=None)
        return c, A, b
