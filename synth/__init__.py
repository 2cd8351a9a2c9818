"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws numbers: lattice sites, strains, jitter, random packings,
coefficient vectors and the POD parameter presets.  It holds none of the method's
arithmetic (no radial functions, no basis, no descriptors), so both the CUDA path
and the CPU oracle can take their inputs from here without sharing any code.

The workloads stand in for the FitSNAP tantalum data set that the paper fits
(Section 5: BCC, FCC, A15 crystals, defects and liquid), which is not available.
Every generator is driven by ``numpy.random.Generator(PCG64(seed))``; the
convention used throughout is ``seed = 1000 * config_id + replica``.

Positions are returned as ``(N, 3)`` float64 arrays (atom-major); boxes are
orthorhombic ``(3,)`` arrays in Angstrom; ``pbc`` is a 3-tuple of ints.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Lattice constants (Angstrom) at about 0.055 atoms / A^3.
A_BCC = 3.316
A_FCC = 4.178
A_A15 = 5.259
DENSITY = 0.055

# Fractional sites of the conventional cells.
BCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
A15_BASIS = np.array([
    [0.0, 0.0, 0.0], [0.5, 0.5, 0.5],
    [0.25, 0.0, 0.5], [0.75, 0.0, 0.5],
    [0.0, 0.5, 0.25], [0.0, 0.5, 0.75],
    [0.5, 0.25, 0.0], [0.5, 0.75, 0.0],
])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class PODParams:
    """Plain container for the POD hyper-parameters (no arithmetic)."""
    r_in: float = 1.0
    r_cut: float = 5.0
    alpha: list = field(default_factory=lambda: [1.0, 2.0, 3.0, 4.0])
    beta: list = field(default_factory=lambda: [3.0])
    gamma: list = field(default_factory=lambda: [1.0, 2.0, 3.0, 4.0])
    K2: int = 6
    K3: int = 6
    K4: int = 6
    P3: int = 4
    P4: int = 4
    n_grid: int = 2000

    @property
    def Ns(self) -> int:
        return len(self.alpha) * len(self.beta) + len(self.gamma)

    @property
    def Kr(self) -> int:
        return max(self.K2, self.K3, self.K4 if self.P4 >= 0 else 0)

    @property
    def Pa(self) -> int:
        return max(self.P3, self.P4)


def params_small() -> PODParams:
    """128-atom workload: Ns = 6 snapshots -> K = 3 modes, angular degree 3, no 4-body."""
    return PODParams(alpha=[1.0, 2.0, 3.0], beta=[3.0], gamma=[1.0, 2.0, 3.0],
                     K2=3, K3=3, K4=3, P3=3, P4=-1)


def params_full() -> PODParams:
    """8,192-atom and larger workloads: Ns = 8 -> K = 6, angular degree 4, 2/3/4-body."""
    return PODParams()


@dataclass
class Config:
    pos: np.ndarray          # (N, 3) float64
    box: np.ndarray          # (3,) float64
    pbc: tuple = (1, 1, 1)
    kind: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def lattice(basis: np.ndarray, a: float, n1: int, n2: int, n3: int) -> Config:
    cells = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    cells = cells.reshape(-1, 3).astype(np.float64)
    frac = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac * a
    box = np.array([n1 * a, n2 * a, n3 * a], dtype=np.float64)
    return Config(pos=pos, box=box)


def bcc(ncell: int, a: float = A_BCC) -> Config:
    c = lattice(BCC_BASIS, a, ncell, ncell, ncell)
    c.kind = "bcc"
    return c


def jitter(cfg: Config, sigma: float, g: np.random.Generator) -> Config:
    pos = cfg.pos + g.normal(0.0, sigma, size=cfg.pos.shape)
    return Config(pos=pos, box=cfg.box.copy(), pbc=cfg.pbc, kind=cfg.kind)


def strain_iso(cfg: Config, s: float) -> Config:
    """Isotropic linear strain x -> (1 + s) x."""
    return Config(pos=cfg.pos * (1.0 + s), box=cfg.box * (1.0 + s), pbc=cfg.pbc, kind=cfg.kind)


def coefficients(M: int, seed: int, sigma: float = 1e-2) -> np.ndarray:
    """Linear-model coefficients c ~ N(0, sigma^2) (sigma is a standard deviation)."""
    return rng(seed).normal(0.0, sigma, size=M)


# --------------------------------------------------------------------------- workloads

def config_small(replica: int = 0) -> Config:
    """128-atom BCC Ta, 4x4x4 cubic cells, a = 3.316 A, jitter N(0, 0.05 A)."""
    g = rng(1000 * 1 + replica)
    return jitter(bcc(4), 0.05, g)


def config_full(replica: int = 0, ncell: int = 16) -> Config:
    """BCC Ta ncell^3 cells (16^3 = 8,192 atoms), +-3 % isotropic strain, jitter N(0, 0.1 A)."""
    g = rng(1000 * 2 + replica)
    u = g.uniform(-0.03, 0.03)
    return jitter(strain_iso(bcc(ncell), u), 0.1, g)


def config_md(replica: int = 0, ncell: int = 80) -> Config:
    """BCC Ta ncell^3 cells (80^3 = 1,024,000 atoms), jitter N(0, 0.08 A)."""
    g = rng(1000 * 4 + replica)
    return jitter(bcc(ncell), 0.08, g)


def _supercell_dims(nbasis: int, n_target: int) -> tuple:
    best = None
    lim = max(1, int(math.ceil((n_target / nbasis) ** (1 / 3))) + 3)
    for n1 in range(1, lim + 1):
        for n2 in range(n1, lim + 1):
            for n3 in range(n2, lim + 1):
                cnt = n1 * n2 * n3 * nbasis
                if cnt < n_target:
                    continue
                key = (cnt, n3 - n1)
                if best is None or key < best[0]:
                    best = (key, (n1, n2, n3))
    return best[1]


def liquid(n: int, g: np.random.Generator, density: float = DENSITY, dmin: float = 2.0) -> Config:
    """Random sequential addition in a periodic cube at the given density."""
    L = (n / density) ** (1.0 / 3.0)
    pos = np.zeros((0, 3))
    tries = 0
    while pos.shape[0] < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("random packing failed")
        p = g.uniform(0.0, L, size=3)
        if pos.shape[0]:
            d = pos - p
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin * dmin:
                continue
        pos = np.vstack([pos, p])
    return Config(pos=pos, box=np.array([L, L, L]), kind="liquid")


def config_train(index: int, replica: int = 0) -> Config:
    """One configuration of the batched-fit set (kind, size, vacancies, volume strain, jitter)."""
    g = rng(1000 * 3 + replica * 100003 + index)
    kind = ["bcc", "fcc", "a15", "liquid"][int(g.integers(0, 4))]
    n_target = int(g.integers(2, 251))
    if kind == "liquid":
        cfg = liquid(n_target, g)
    else:
        basis, a = {"bcc": (BCC_BASIS, A_BCC), "fcc": (FCC_BASIS, A_FCC), "a15": (A15_BASIS, A_A15)}[kind]
        n1, n2, n3 = _supercell_dims(basis.shape[0], n_target)
        cfg = lattice(basis, a, n1, n2, n3)
        if cfg.n > n_target:
            keep = np.sort(g.permutation(cfg.n)[:n_target])
            cfg = Config(pos=cfg.pos[keep], box=cfg.box)
        cfg.kind = kind
    vol = g.uniform(0.8, 1.2)
    cfg = strain_iso(cfg, vol ** (1.0 / 3.0) - 1.0)
    return jitter(cfg, 0.1, g)


def training_set(n_configs: int, replica: int = 0) -> list:
    return [config_train(k, replica) for k in range(n_configs)]


def cluster(n: int, seed: int, radius: float = 2.6, dmin: float = 1.6) -> Config:
    """Open-boundary cluster of n atoms inside a ball, pairwise distances >= dmin."""
    g = rng(seed)
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cluster packing failed")
        p = g.uniform(-radius, radius, size=3)
        if np.dot(p, p) > radius * radius:
            continue
        if any(np.dot(p - q, p - q) < dmin * dmin for q in pts):
            continue
        pts.append(p)
    pos = np.array(pts) + 10.0
    return Config(pos=pos, box=np.array([20.0, 20.0, 20.0]), pbc=(0, 0, 0), kind="cluster")


def random_rotation(g: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q
