"""Neighbour lists with a skin reused between rebuilds, and the velocity-Verlet
step (the MD-scale workload).  A list built at x0 with skin 0.4 A and reused at
x1 (displacements <= 0.1 A, some atoms crossing the box edge) must give the
energy and forces of a fresh r_cut list at x1; one md step must equal the
velocity-Verlet update written out with the library's own energy/forces."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
CONV = 9.648533212e-3  # A/fs^2 per eV/(A amu)


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14446_gb300 import build as b
    b.build()
    import paper_2212_14446_gb300 as p
    return p


def _moved_config():
    cfg = synth.jitter(synth.bcc(6), 0.08, synth.rng(51))  # 432 atoms, box 19.9 A
    g = synth.rng(52)
    x0 = cfg.pos.copy()
    x0[:5, 0] = 0.02 * np.arange(5)  # atoms sitting on the lower box face
    x1 = x0 + g.uniform(-0.1, 0.1, size=x0.shape) / np.sqrt(3)
    x1[:5, 0] -= 0.05  # ... that cross it
    return cfg, x0, x1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reuse_with_skin_equals_rebuild(pkg, prec):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg, x0, x1 = _moved_config()
    c = torch.tensor(synth.coefficients(o.M, 53), device="cuda")
    a = pkg.POD(p, precision=prec, Q=o.Q)
    a.set_skin(0.4)
    a.set_neighbor_reuse(True)
    t0 = torch.tensor(x0.T.copy(), device="cuda")
    t1 = torch.tensor(x1.T.copy(), device="cuda")
    a.energy_forces(t0, cfg.box, c)          # builds the skin list at x0
    ra = a.energy_forces(t1, cfg.box, c)     # reuses it at x1
    b = pkg.POD(p, precision=prec, Q=o.Q)
    rb = b.energy_forces(t1, cfg.box, c)     # fresh r_cut list at x1
    Fa, Fb = ra["F"].cpu().numpy(), rb["F"].cpu().numpy()
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert abs(ra["E"].item() - rb["E"].item()) <= tol * abs(rb["E"].item())
    assert np.max(np.abs(Fa - Fb)) <= tol * np.max(np.abs(Fb))
    assert np.allclose(ra["W"].cpu().numpy(), rb["W"].cpu().numpy(), rtol=0, atol=tol * np.abs(rb["W"].cpu().numpy()).max())
    if prec == "fp64":  # and the oracle at x1
        _, E_o, F_o, _ = o.energy_forces(synth.Config(pos=x1, box=cfg.box), c.cpu().numpy(), fast=True)
        assert abs(ra["E"].item() - E_o) <= 1e-11 * abs(E_o)


def test_md_step_is_velocity_verlet(pkg):
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(5), 0.08, synth.rng(54))
    pod = pkg.POD(p, precision="fp64")
    pod.set_skin(0.3)
    c = torch.tensor(synth.coefficients(pod.M, 55), device="cuda")
    mass, dt = 180.94788, 1.0
    x = torch.tensor(cfg.pos.T.copy(), device="cuda")
    v = torch.tensor(synth.rng(56).normal(0, 1.2e-3, size=(3, cfg.n)), device="cuda")
    F = pod.energy_forces(x, cfg.box, c)["F"].t().contiguous()
    x0, v0, F0 = x.clone(), v.clone(), F.clone()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    pod.md_step(x, v, F, c, cfg.box, mass, dt, E)
    h = 0.5 * dt * CONV / mass
    x_ref = x0 + (v0 + h * F0) * dt
    ref = pkg.POD(p, precision="fp64").energy_forces(x_ref, cfg.box, c)
    F1 = ref["F"].t()
    v_ref = v0 + h * (F0 + F1)
    assert torch.allclose(x, x_ref, rtol=0, atol=1e-13)
    assert abs(E.item() - ref["E"].item()) <= 1e-12 * abs(ref["E"].item())
    assert torch.allclose(F, F1, rtol=0, atol=1e-10 * F1.abs().max().item())
    assert torch.allclose(v, v_ref, rtol=0, atol=1e-15 + 1e-12 * v_ref.abs().max().item())
