"""Differentiation paths: global descriptors, their forward-mode directional
derivative (descriptor JVP) against the oracle's explicit dD/dr, and the
torch.autograd Functions (energy gradient = -F and G; force-matching loss
gradient with respect to c against central differences, exact for a loss that
is quadratic in c)."""
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


def _soa(cfg):
    return torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device="cuda")


def _jvp_oracle(o, cfg, v, atoms=None):
    """sum_i sum_j dD_i/dr_ij . (v_j - v_i) from the oracle's explicit derivatives."""
    lists = o.neighbor_lists(cfg) if atoms is None else [o.neighbors(cfg, i) for i in atoms]
    idx = range(cfg.n) if atoms is None else atoms
    Gd = np.zeros(o.M)
    for i, (js, _, d) in zip(idx, lists):
        dD = o.atom_dD(d, fast=True)  # (n, M, 3)
        Gd += np.einsum("jmt,jt->m", dD, v[js] - v[i][None, :])
    return Gd


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_global_descriptors_and_jvp_small(pkg, prec, tol):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(31))
    v = synth.rng(32).normal(size=(cfg.n, 3))
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    G = pod.global_descriptors(_soa(cfg), cfg.box).cpu().numpy()[0]
    Gref = o.descriptors(cfg, fast=True).sum(axis=0)
    assert np.max(np.abs(G - Gref) / np.maximum(np.abs(Gref), 1.0)) <= tol
    Gd = pod.descriptors_jvp(_soa(cfg), cfg.box, torch.tensor(v.T.copy(), device="cuda")).cpu().numpy()[0]
    Gdref = _jvp_oracle(o, cfg, v)
    scale = np.maximum(np.abs(Gdref), 1e-3 * np.abs(Gdref).max())
    assert np.max(np.abs(Gd - Gdref) / scale) <= (1e-10 if prec == "fp64" else 1e-4)


def test_jvp_full_size_sampled(pkg):
    """8,192 atoms: a direction supported on three atoms touches only their
    neighbourhoods, so the oracle evaluates dD/dr for those atoms alone."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.config_full()
    v = np.zeros((cfg.n, 3))
    g = synth.rng(40)
    seeds = [17, 4000, 8000]
    for k in seeds:
        v[k] = g.normal(size=3)
    touched = set(seeds)
    for k in seeds:
        js, _, _ = o.neighbors(cfg, k)
        touched.update(int(j) for j in js)
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    Gd = pod.descriptors_jvp(_soa(cfg), cfg.box, torch.tensor(v.T.copy(), device="cuda")).cpu().numpy()[0]
    Gdref = _jvp_oracle(o, cfg, v, atoms=sorted(touched))
    scale = np.maximum(np.abs(Gdref), 1e-3 * np.abs(Gdref).max())
    assert np.max(np.abs(Gd - Gdref) / scale) <= 1e-10


def test_energy_autograd(pkg):
    from paper_2212_14446_gb300.autograd import pod_energy
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(41))
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device="cuda", requires_grad=True)  # (N, 3)
    c = torch.tensor(synth.coefficients(o.M, 42), device="cuda", requires_grad=True)
    E = pod_energy(pos, c, pod, cfg.box)
    E.backward()
    Eo, _ = None, None
    _, E_o, F_o, _ = o.energy_forces(cfg, c.detach().cpu().numpy(), fast=True)
    assert E.item() == pytest.approx(E_o, rel=1e-12)
    assert np.allclose(pos.grad.cpu().numpy(), -F_o, atol=1e-10 * np.abs(F_o).max())
    G = o.descriptors(cfg, fast=True).sum(axis=0)
    assert np.allclose(c.grad.cpu().numpy(), G, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("which", ["small", "full"])
def test_force_matching_gradient(pkg, which):
    """L(c) = sum (F(c) - F_ref)^2 is quadratic in c: its central difference along
    any direction equals the gradient exactly up to rounding."""
    from paper_2212_14446_gb300.autograd import pod_forces
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(43)) if which == "small" else synth.config_full()
    pod = pkg.POD(p, precision="fp64")
    M = pod.M
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device="cuda")
    c0 = torch.tensor(synth.coefficients(M, 44), device="cuda")
    Fref = torch.tensor(synth.rng(45).normal(0, 0.1, size=cfg.pos.shape), device="cuda")
    c = c0.clone().requires_grad_(True)
    L = ((pod_forces(pos, c, pod, cfg.box) - Fref) ** 2).sum()
    L.backward()
    d = torch.tensor(synth.rng(46).normal(size=M), device="cuda")
    eps = 1e-3
    with torch.no_grad():
        Lp = ((pod_forces(pos, c0 + eps * d, pod, cfg.box) - Fref) ** 2).sum()
        Lm = ((pod_forces(pos, c0 - eps * d, pod, cfg.box) - Fref) ** 2).sum()
    fd = (Lp - Lm).item() / (2 * eps)
    an = torch.dot(c.grad, d).item()
    assert an == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(L.item()))


def test_large_batch_energy_forces_sampled(pkg):
    """32 independent 8,192-atom configurations (262,144 atoms) in one batched
    call, mixed precision: sampled forces against the oracle."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = [synth.config_full(replica=r) for r in range(32)]
    c = synth.coefficients(o.M, 47)
    pod = pkg.POD(p, precision="mixed", Q=o.Q)
    out = pod.energy_forces_batch(cfgs, torch.tensor(c))
    F = out["F"].cpu().numpy()
    offs = out["offs"]
    for k, atoms in [(0, [5]), (19, [777]), (31, [8191])]:
        _, _, Fo, _ = o.energy_forces(cfgs[k], c, fast=True, force_atoms=atoms)
        assert np.max(np.abs(F[offs[k] + np.array(atoms)] - Fo)) <= 1e-4
    E = out["E"].cpu().numpy()
    assert E.shape == (32,) and np.all(np.isfinite(E))
