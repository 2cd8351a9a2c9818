"""Launch-shape autotuner (a deployment feature, not a step of the method): it
returns a shape from the candidate sets, the tuned shape is used by later calls,
and the results do not depend on it -- forces and atom energies bit for bit (each
is computed by one lane in a fixed order whatever the block shape), total energy
and virial to rounding (their block partials are summed in a shape-dependent but
fixed order; on the mixed path the energy is an exact fixed-point total and the
virial's per-warp FP32 partials depend on the grouping of pairs into warps).
The adjoint pair pass of the mixed linear path runs inside the fused atom kernel
or as its own kernel; both forms give the same forces, atom energies and energy
bit for bit."""
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
    assert t["neigh_wpb"] in (2, 4, 6, 8) and t["atom_wpb"] in (1, 2, 4) and t["atom_rp"] in (0, 1, 2)
    assert prec == "mixed" or t["atom_rp"] == 0
    assert (t["gather_wpb"], t["gather_bps"]) in ((16, 3), (16, 2), (8, 6), (8, 4), (4, 12))
    assert all(m > 0 for m in t["ms"])
    for _ in range(2):  # two calls in a row with the tuned shape
        after = pod.energy_forces(x, cfg.box, c)
        assert torch.equal(after["F"], before["F"])
        assert torch.equal(after["Ei"], before["Ei"])
        assert abs(after["E"].item() - before["E"].item()) <= 1e-13 * abs(before["E"].item())
        wtol = 1e-13 if prec == "fp64" else 1e-5
        assert torch.allclose(after["W"], before["W"], rtol=0, atol=wtol * before["W"].abs().max().item())


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


def test_batch_tuner_refuses_what_the_fit_refuses(pkg):
    """A batch goes to the fit's tuner, which refuses what pod_fit refuses (the
    exclusive three-body set)."""
    p = synth.params_small()
    pod = pkg.POD(p, precision="fp64")
    pod.set_descriptor_set("exclusive")
    cfgs = [synth.config_small(replica=r) for r in range(2)]
    pos, offs, boxes, pbcs = pod.pack_batch(cfgs)
    xs = torch.tensor(pos, device="cuda")
    sysd = pod.batch_system(xs, offs, boxes, pbcs)
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_autotune(pod.h, sysd, None)
    assert ei.value.code == pkg.POD_EINVAL


def _generic_params():
    # K = 4 modes, degree 2, no four-body terms: the generic (run-time K) kernels
    return synth.PODParams(alpha=[1.0, 2.0, 3.0], beta=[3.0], gamma=[1.0, 2.0], K2=4, K3=4, K4=4, P3=2, P4=-1)


@pytest.mark.parametrize("which", ["full", "small", "generic", "exclusive3"])
def test_separate_adjoint_kernel_equals_fused(pkg, which):
    if which == "small":
        p, cfg = synth.params_small(), synth.config_small()
    elif which == "generic":
        p, cfg = _generic_params(), synth.jitter(synth.bcc(8), 0.1, synth.rng(65))
    else:
        p, cfg = synth.params_full(), synth.config_full()
    pod = pkg.POD(p, precision="mixed")
    if which == "exclusive3":
        pod.set_descriptor_set("exclusive")
    c = torch.tensor(synth.coefficients(pod.M, 66), device="cuda")
    x = torch.tensor(cfg.pos.T.copy(), device="cuda")
    pod.set_adjoint_kernel("fused")
    fused = pod.energy_forces(x, cfg.box, c)
    pod.set_adjoint_kernel("separate")
    for _ in range(2):
        sep = pod.energy_forces(x, cfg.box, c)
        assert torch.equal(sep["F"], fused["F"])
        assert torch.equal(sep["Ei"], fused["Ei"])
        assert sep["E"].item() == fused["E"].item()  # exact fixed-point sum of the same E_i
        assert torch.allclose(sep["W"], fused["W"], rtol=0, atol=1e-5 * fused["W"].abs().max().item())


def test_batch_tuner_picks_design_shapes_with_the_same_fit(pkg):
    """pod_autotune on a batch tunes the fit's design pass; the fit afterwards
    gives the same bits as on an untuned handle."""
    p = synth.params_full()
    cfgs = []
    k = 0
    while len(cfgs) < 30:
        cf = synth.config_train(k, 71)
        k += 1
        if cf.n <= 60:
            cfgs.append(cf)
    pod = pkg.POD(p, precision="mixed")
    teacher = pkg.POD(p, precision="fp64", Q=pod.Q)
    out = teacher.energy_forces_batch(cfgs, torch.tensor(synth.coefficients(pod.M, 72)))
    pos, offs, boxes, pbcs = pod.pack_batch(cfgs)
    x = torch.tensor(pos, dtype=torch.float64, device="cuda")
    Er = out["E"].to("cuda").contiguous()
    Fr = out["F"].to("cuda").t().contiguous()
    ref = pkg.POD(p, precision="mixed", Q=pod.Q)
    c_ref, _, _ = ref.fit_device(x, offs, boxes, pbcs, Er, Fr)
    t = pod.autotune_fit(x, offs, boxes, pbcs, reps=1)
    assert t["atom_wpb"] in (1, 2, 4) and t["design_wpb"] in (2, 4, 8) and t["ms"] > 0
    c, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)
    assert np.array_equal(c, c_ref)
