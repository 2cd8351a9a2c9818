"""Launch-shape autotuner (a deployment feature, not a step of the method): it
returns a shape from the candidate sets, the tuned shape is used by later calls,
and the results do not depend on it -- forces and atom energies bit for bit (each
is computed by one lane in a fixed order whatever the block shape), total energy
and virial to rounding (their block partials are summed in a shape-dependent but
fixed order)."""
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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_shape_and_results(pkg, prec):
    p = synth.params_full()
    cfg = synth.config_full()
    pod = pkg.POD(p, precision=prec)
    c = torch.tensor(synth.coefficients(pod.M, 61), device="cuda")
    x = torch.tensor(cfg.pos.T.copy(), device="cuda")
    before = pod.energy_forces(x, cfg.box, c)
    t = pod.autotune(x, cfg.box, c, reps=2)
    assert t["neigh_wpb"] in (2, 4, 8) and t["atom_wpb"] in (1, 2, 4) and t["atom_rp"] in (0, 1)
    assert prec == "mixed" or t["atom_rp"] == 0
    assert (t["gather_wpb"], t["gather_bps"]) in ((16, 3), (16, 2), (8, 6), (8, 4), (4, 12))
    assert all(m > 0 for m in t["ms"])
    for _ in range(2):  # two calls in a row with the tuned shape
        after = pod.energy_forces(x, cfg.box, c)
        assert torch.equal(after["F"], before["F"])
        assert torch.equal(after["Ei"], before["Ei"])
        assert abs(after["E"].item() - before["E"].item()) <= 1e-13 * abs(before["E"].item())
        assert torch.allclose(after["W"], before["W"], rtol=0, atol=1e-13 * before["W"].abs().max().item())


def test_every_candidate_shape_gives_the_same_forces(pkg):
    """Tuning a 2,000-atom system twice (each pass runs every candidate shape)
    keeps its forces bit for bit under whichever shape wins."""
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(10), 0.1, synth.rng(62))
    pod = pkg.POD(p, precision="mixed")
    c = torch.tensor(synth.coefficients(pod.M, 63), device="cuda")
    x = torch.tensor(cfg.pos.T.copy(), device="cuda")
    ref = pod.energy_forces(x, cfg.box, c)["F"].clone()
    for _ in range(2):
        pod.autotune(x, cfg.box, c, reps=1)
        assert torch.equal(pod.energy_forces(x, cfg.box, c)["F"], ref)


def test_autotune_rejects_a_batch(pkg):
    p = synth.params_small()
    pod = pkg.POD(p, precision="fp64")
    cfgs = [synth.config_small(replica=r) for r in range(2)]
    pos, offs, boxes, pbcs = pod.pack_batch(cfgs)
    xs = torch.tensor(pos, device="cuda")
    sysd = pod.batch_system(xs, offs, boxes, pbcs)
    c = torch.tensor(synth.coefficients(pod.M, 64), device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_autotune(pod.h, sysd, c)
    assert ei.value.code == pkg.POD_EINVAL
