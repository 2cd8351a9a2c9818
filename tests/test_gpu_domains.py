"""Spatial decomposition on the GPU: the 8,192-atom periodic system split into
slab domains (local atoms + ghost copies within r_cut, pod_system.n_local),
each evaluated by the library, forces summed onto the owning atoms, equals the
whole system evaluated at once.  Tolerances: FP64 as the parity tests (1e-12
energy, 1e-10 max|F| forces and virial); mixed as the mixed path against FP64
(the domains' shifted coordinates round differently): 1e-6 relative energy,
1e-4 eV/A forces, 1e-5 relative virial."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n_slabs", [2, 3])
def test_slab_domains_equal_whole_system(pkg, prec, n_slabs):
    from paper_2212_14446_gb300 import parallel
    p = synth.params_full()
    cfg = synth.config_full(3)
    pod = pkg.POD(p, precision=prec)
    ct = torch.tensor(synth.coefficients(pod.M, 131), device="cuda")
    whole = pod.energy_forces(torch.tensor(cfg.pos.T.copy(), device="cuda"), cfg.box, ct)
    E0, Ei0 = whole["E"].item(), whole["Ei"].cpu().numpy()
    F0, W0 = whole["F"].cpu().numpy(), whole["W"].cpu().numpy()
    ghost_ei = []

    def evaluate(sub, sub_box, pbc, n_local):
        out = pod.energy_forces(torch.tensor(sub.T.copy(), device="cuda"), sub_box, ct, pbc=pbc, n_local=n_local)
        ei = out["Ei"].cpu().numpy()
        ghost_ei.append(np.max(np.abs(ei[n_local:])) if len(ei) > n_local else 0.0)
        return out["E"].item(), ei, out["F"].cpu().numpy(), out["W"].cpu().numpy()

    E, Ei, F, W = parallel.energy_forces_domains(evaluate, cfg.pos, cfg.box, p.r_cut, n_slabs)
    assert max(ghost_ei) == 0.0  # ghosts carry no energy of their own
    fmax, wmax = float(np.max(np.abs(F0))), float(np.max(np.abs(W0)))
    if prec == "fp64":
        assert E == pytest.approx(E0, rel=1e-12)
        assert np.max(np.abs(Ei - Ei0)) <= 1e-12 * np.max(np.abs(Ei0))
        assert np.max(np.abs(F - F0)) <= 1e-10 * fmax
        assert np.max(np.abs(W - W0)) <= 1e-10 * wmax
    else:
        assert E == pytest.approx(E0, rel=1e-6)
        assert np.max(np.abs(F - F0)) <= 1e-4 * max(fmax, 1.0)
        assert np.max(np.abs(W - W0)) <= 1e-5 * wmax


def test_n_local_validation(pkg):
    p = synth.params_small()
    cfg = synth.config_small()
    pod = pkg.POD(p, precision="fp64")
    ct = torch.tensor(synth.coefficients(pod.M, 132), device="cuda")
    x = torch.tensor(cfg.pos.T.copy(), device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(x, cfg.box, ct, n_local=cfg.n + 1)
    assert ei.value.code == pkg.POD_EINVAL
    a = pod.energy_forces(x, cfg.box, ct, n_local=cfg.n)  # every atom local = the plain call
    b = pod.energy_forces(x, cfg.box, ct)
    assert torch.equal(a["F"], b["F"]) and torch.equal(a["E"], b["E"])
