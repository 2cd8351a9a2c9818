"""Exclusive three-body descriptor set (Eq. 15b: the original POD sums over
pairs k > j) on the GPU against the FP64 oracle: descriptors and the linear
model's energy, forces and virial.  Tolerances as for the fast POD set:
descriptors per column <= 1e-12 (FP64) / 1e-5 (mixed) of the column's largest
value; energy <= 1e-12 / 1e-5 of sum_i |E_i|; forces <= 1e-10 max|F| / 1e-4."""
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


def _dev(cfg):
    return torch.tensor(cfg.pos.T.copy(), device="cuda")


def _col_err(D, Dref):
    den = np.max(np.abs(Dref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(D - Dref), axis=0) / den))


@pytest.mark.parametrize("which", ["full", "small"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_exclusive3_descriptors_and_energy_forces(pkg, which, prec):
    p = synth.params_full() if which == "full" else synth.params_small()
    o = oracle.Oracle(p)
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(111))
    c = synth.coefficients(o.M, 112)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    pod.set_descriptor_set("exclusive")
    D = pod.descriptors(_dev(cfg), cfg.box).cpu().numpy()
    sysd = o._system(cfg)
    Dref = np.array([o.exclusive3_descriptors(o.neighbors(cfg, i, sysd)[2]) for i in range(cfg.n)])
    tol_d = 1e-12 if prec == "fp64" else 1e-5
    assert _col_err(D, Dref) <= tol_d
    Ei_o, E_o, F_o, W_o = o.energy_forces_exclusive3(cfg, c)
    out = pod.energy_forces(_dev(cfg), cfg.box, torch.tensor(c, device="cuda"))
    E, F, W, Ei = out["E"].item(), out["F"].cpu().numpy(), out["W"].cpu().numpy(), out["Ei"].cpu().numpy()
    escale = float(np.sum(np.abs(Ei_o)))
    fmax = float(np.max(np.abs(F_o)))
    if prec == "fp64":
        assert abs(E - E_o) <= 1e-12 * escale
        assert np.max(np.abs(Ei - Ei_o)) <= 1e-12 * escale
        assert np.max(np.abs(F - F_o)) <= 1e-10 * fmax
        assert np.max(np.abs(W - W_o)) <= 1e-10 * max(np.max(np.abs(W_o)), escale)
    else:
        assert abs(E - E_o) <= 1e-5 * escale
        assert np.max(np.abs(F - F_o)) <= 1e-4 * max(fmax, 1.0)
        assert np.max(np.abs(W - W_o)) <= 1e-5 * max(np.max(np.abs(W_o)), escale)
    # back to the fast POD set
    pod.set_descriptor_set("fast")
    D2 = pod.descriptors(_dev(cfg), cfg.box).cpu().numpy()
    assert _col_err(D2, o.descriptors(cfg, fast=True)) <= tol_d


def test_exclusive3_refused_where_unsupported(pkg):
    """The quadratic and embedding models, the descriptor tangent, the fit and the
    allocation-free entry take the fast POD set only."""
    p = synth.params_small()
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(113))
    pod = pkg.POD(p, precision="fp64")
    c = torch.tensor(synth.coefficients(pod.M, 114), device="cuda")
    x = _dev(cfg)
    pod.set_descriptor_set("exclusive")
    pod.set_quadratic(np.zeros((pod.M, pod.M)))
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(x, cfg.box, c)
    assert ei.value.code == pkg.POD_EINVAL
    pod.set_quadratic(None)
    pod.set_embedding(np.zeros(pod.M), np.array([0.0, 1.0]))
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(x, cfg.box, c)
    assert ei.value.code == pkg.POD_EINVAL
    pod.set_embedding(None)
    D = torch.empty((cfg.n, pod.M), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_descriptors_static(pod.h, pod.system(x, cfg.box), D)
    assert ei.value.code == pkg.POD_EINVAL
    with pytest.raises(pkg.PodError) as ei:
        pod.descriptors_jvp(x, cfg.box, torch.ones_like(x))
    assert ei.value.code == pkg.POD_EINVAL
    E = pod.energy_forces(x, cfg.box, c)["E"]  # the linear model still runs
    assert torch.isfinite(E).all()
