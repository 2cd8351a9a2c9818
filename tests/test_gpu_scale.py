"""Parity with the FP64 oracle at the full sizes of the two large workloads.

* The 1,024,000-atom BCC Ta system (80^3 cells, jitter N(0, 0.08 A)), both
  precision paths, in the launch shapes the benchmark uses (autotuned): every
  atom energy, every force and the virial against the oracle's cell-list route
  (pinned on the CPU to its brute-force definition), descriptors of atoms at box
  faces, cell faces and random places against the oracle's plain sums.
* The batched fit on the real training-set generator (BCC/FCC/A15 with
  vacancies and liquids, 2..250 atoms): the normal equations G = A^T A + gamma I
  and r = A^T b that pod_fit_normal returns, element by element, against the
  oracle's design matrix for a subset that holds every 200..250-atom
  configuration of the first 120 plus small ones (tens of 256-row chunks and
  many row splits of the tensor-core Gram); and the whole 2,000-configuration set
  against the sum of its shards (the normal equations are additive).

Tolerances (readings of the paper's error statements):
  energy |dE| / sum_i sum_m |c_m D_im| and E_i per atom the same way: 1e-12
  (FP64), 1e-5 (mixed); forces max |dF| <= 1e-10 max|F| (FP64), 1e-4 eV/A
  (mixed); virial relative to max |W| as the energy; descriptors per column
  relative to the column maximum: 1e-12 / 1e-5.
  Normal equations: |dG_mn| <= tau sqrt(G_mm G_nn), |dr_m| <= tau sqrt(G_mm) |b|,
  tau = 1e-12 (FP64 path); mixed path tau = 2e-5, from |dG_mn| <=
  (|dA_m| |A_n| + |A_m| |dA_n|) <= 2 eps_col sqrt(G_mm G_nn) with the column-wise
  relative error eps_col of the design matrix bounded by the 1e-5 descriptor
  (and descriptor-gradient) error of the mixed path.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14446_gb300 import build as b
    b.build()
    import paper_2212_14446_gb300 as p
    return p


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _soa(cfg):
    return torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device="cuda")


# ------------------------------------------------------- 1,024,000 atoms

@pytest.fixture(scope="module")
def md_system():
    p = synth.params_full()
    cfg = synth.config_md(0)
    o = oracle.Oracle(p)
    c = synth.coefficients(o.M, 4001)
    esc = np.zeros(cfg.n)
    Ei, E, F, W = o.energy_forces_cells(cfg, c, threads=_cores(), escale=esc)
    return p, o, cfg, c, (Ei, E, F, W, esc)


def _edge_atoms(cfg, n_rand=8):
    """Atoms closest to the box faces and to the faces of the 53^3 cell grid, plus
    random ones."""
    L = cfg.box
    w = cfg.pos - L * np.floor(cfg.pos / L)
    pick = set()
    for d in range(3):
        pick.add(int(np.argmin(w[:, d])))
        pick.add(int(np.argmax(w[:, d])))
        cs = L[d] / int(np.floor(L[d] / 5.0))
        frac = np.abs(w[:, d] / cs - np.round(w[:, d] / cs))
        pick.add(int(np.argmin(frac + (w[:, d] < 1.0))))
    corner = np.linalg.norm(np.minimum(w, L - w), axis=1)
    pick.add(int(np.argmin(corner)))
    pick.update(int(i) for i in synth.rng(91).choice(cfg.n, size=n_rand, replace=False))
    return sorted(pick)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_md_size_energy_forces_virial(pkg, md_system, prec):
    p, o, cfg, c, (Ei_o, E_o, F_o, W_o, esc) = md_system
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    x = _soa(cfg)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    pod.autotune(x, cfg.box, ct, reps=2)
    out = pod.energy_forces(x, cfg.box, ct)
    E = out["E"].item()
    Ei = out["Ei"].cpu().numpy()
    F = out["F"].cpu().numpy()
    W = out["W"].cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(E - E_o) <= tol * float(np.sum(esc))
    assert np.max(np.abs(Ei - Ei_o) / np.maximum(esc, 1e-300)) <= tol
    if prec == "fp64":
        assert np.max(np.abs(F - F_o)) <= 1e-10 * np.max(np.abs(F_o))
    else:
        assert np.max(np.abs(F - F_o)) <= 1e-4
    assert np.max(np.abs(W - W_o)) <= tol * np.max(np.abs(W_o))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_md_size_descriptors_at_edges(pkg, md_system, prec, tol):
    p, o, cfg, _, _ = md_system
    atoms = _edge_atoms(cfg)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    D = pod.descriptors(_soa(cfg), cfg.box)
    Dg = D[torch.tensor(atoms, device="cuda")].cpu().numpy()
    del D
    Dref = o.descriptors(cfg, atoms=atoms)  # the plain sums of Eq. 12b, 15, 18a
    den = np.max(np.abs(Dref), axis=0)
    den = np.where(den > 0, den, 1.0)
    assert np.max(np.max(np.abs(Dg - Dref), axis=0) / den) <= tol


# ------------------------------------------------------- the training set

def _labels(o, cfgs, c):
    E, F = [], []
    for cf in cfgs:
        _, e, f, _ = o.energy_forces_cells(cf, c)
        E.append(e)
        F.append(f)
    return np.array(E), F


@pytest.fixture(scope="module")
def fit_subset():
    p = synth.params_full()
    o = oracle.Oracle(p)
    first = synth.training_set(120)
    big = [cf for cf in first if cf.n >= 200]
    small = [cf for cf in first if cf.n <= 60][:20]
    cfgs = big + small
    cstar = synth.coefficients(o.M, 5001)
    E_ref, F_ref = _labels(o, cfgs, cstar)
    g = synth.rng(5002)  # noisy labels, as a real fit sees them
    E_ref = E_ref + 1e-3 * np.array([cf.n for cf in cfgs]) * g.normal(size=len(cfgs))
    F_ref = [f + 5e-2 * g.normal(size=f.shape) for f in F_ref]
    G_o, r_o = o.normal_equations(cfgs, E_ref, F_ref, threads=_cores())
    A_b = np.sqrt(sum(100.0 ** 2 * (e / cf.n) ** 2 + float(np.sum(f * f)) for cf, e, f in zip(cfgs, E_ref, F_ref)))
    return p, o, cfgs, E_ref, F_ref, G_o, r_o, A_b


@pytest.mark.parametrize("prec,tau", [("fp64", 1e-12), ("mixed", 2e-5)])
@pytest.mark.parametrize("gram", [0, 1])
def test_fit_normal_equations_elementwise(pkg, fit_subset, prec, tau, gram):
    p, o, cfgs, E_ref, F_ref, G_o, r_o, b_norm = fit_subset
    assert sum(1 + 3 * cf.n for cf in cfgs) > 16000  # many 256-row chunks
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    pkg.pod_set_option(pod.h, pkg.POD_OPT_GRAM, gram)
    G, r = pod.fit_normal(cfgs, E_ref, F_ref)
    d = np.sqrt(np.abs(np.diag(G_o)))
    assert np.max(np.abs(G - G_o) / np.outer(d, d)) <= tau
    assert np.max(np.abs(r - r_o) / (d * b_norm)) <= tau


def test_full_training_set_normal_equations_are_additive(pkg):
    """The 2,000-configuration set of the fit workload: G and r of the whole set
    equal the sums over four shards (each with its own column scaling in the
    exact tensor-core Gram), and the mixed path's G agrees with the FP64 path's
    within the mixed bound."""
    from paper_2212_14446_gb300.parallel import shard_indices
    p = synth.params_full()
    cfgs = synth.training_set(2000)
    pod64 = pkg.POD(p, precision="fp64")
    cstar = torch.tensor(synth.coefficients(pod64.M, 3001), dtype=torch.float64)
    out = pod64.energy_forces_batch(cfgs, cstar)
    E_ref = out["E"].cpu().numpy()
    Fall = out["F"].cpu().numpy()
    offs = out["offs"]
    F_ref = [Fall[offs[k]:offs[k + 1]] for k in range(len(cfgs))]
    pod = pkg.POD(p, precision="mixed", Q=pod64.Q)
    G_all, r_all = pod.fit_normal(cfgs, E_ref, F_ref)
    G = np.zeros_like(G_all)
    r = np.zeros_like(r_all)
    for rank in range(4):
        idx = shard_indices(len(cfgs), rank, 4)
        Gs, rs = pod.fit_normal([cfgs[i] for i in idx], E_ref[idx], [F_ref[i] for i in idx],
                                gamma=1e-12 if rank == 0 else 0.0)
        G += Gs
        r += rs
    d = np.sqrt(np.abs(np.diag(G_all)))
    assert np.max(np.abs(G - G_all) / np.outer(d, d)) <= 1e-13
    assert np.max(np.abs(r - r_all)) <= 1e-13 * np.max(np.abs(r_all))
    G64, _ = pod64.fit_normal(cfgs, E_ref, F_ref)
    d64 = np.sqrt(np.abs(np.diag(G64)))
    assert np.max(np.abs(G_all - G64) / np.outer(d64, d64)) <= 2e-5
