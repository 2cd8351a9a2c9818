"""Quadratic POD model (Sec. 4: E_i = c.D_i + sum_{m<=n} beta_mn D_im D_in) on
the GPU against the FP64 oracle.  Tolerances as for the linear model: FP64
energy <= 1e-12 of sum_i |E_i|-scale, forces <= 1e-10 max|F|; mixed energy <=
1e-5 relative, forces <= 1e-4 of max|F| (the quadratic terms scale the forces)."""
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


def _beta(M, seed, scale=1e-5):
    return synth.rng(seed).normal(0.0, scale, size=(M, M))


@pytest.mark.parametrize("which", ["full", "small"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quadratic_energy_forces(pkg, which, prec):
    p = synth.params_full() if which == "full" else synth.params_small()
    o = oracle.Oracle(p)
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(81))
    c = synth.coefficients(o.M, 82)
    beta = _beta(o.M, 83)
    Ei_o, E_o, F_o, W_o = o.energy_forces_quadratic(cfg, c, beta)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    pod.set_quadratic(beta)
    out = pod.energy_forces(torch.tensor(cfg.pos.T.copy(), device="cuda"), cfg.box, torch.tensor(c, device="cuda"))
    E = out["E"].item()
    F = out["F"].cpu().numpy()
    W = out["W"].cpu().numpy()
    Ei = out["Ei"].cpu().numpy()
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
    # back to the linear model
    pod.set_quadratic(None)
    lin = pod.energy_forces(torch.tensor(cfg.pos.T.copy(), device="cuda"), cfg.box,
                            torch.tensor(c, device="cuda"))
    _, E_l, F_l, _ = o.energy_forces(cfg, c, fast=True)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(lin["E"].item() - E_l) <= tol * float(np.sum(np.abs(o.descriptors(cfg, fast=True) * c)))


def test_quadratic_zero_beta_is_linear_bitwise(pkg):
    """beta = 0 gives exactly the linear model's forces (FP64 path)."""
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(4), 0.1, synth.rng(84))
    pod = pkg.POD(p, precision="fp64")
    c = torch.tensor(synth.coefficients(pod.M, 85), device="cuda")
    x = torch.tensor(cfg.pos.T.copy(), device="cuda")
    lin = pod.energy_forces(x, cfg.box, c)
    pod.set_quadratic(np.zeros((pod.M, pod.M)))
    q = pod.energy_forces(x, cfg.box, c)
    assert torch.equal(q["F"], lin["F"])
    assert q["E"].item() == pytest.approx(lin["E"].item(), rel=1e-15)
