"""Recorded fits (POD_OPT_FIT_GRAPH): a pod_fit on a batch already on the device
records its device chain (neighbour lists, design matrix, normal equations or QR,
solve, residual) into a CUDA graph after it has run; a later pod_fit with the same
layout, device arrays, options and settings replays the graph.

* A replay gives the same bits as the call that recorded it.
* A replay recomputes everything from the arrays' current contents: new positions
  and labels in the same arrays give the same bits as the ordinary path on a
  handle with recording off.
* The Cholesky -> QR fallback and the QR solver work through a replay.
* A changed layout, options, phase timing or recording switched off take the
  ordinary path.
"""
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


def _batch(pkg, pod, cfgs, E_ref, F_ref):
    pos, offs, boxes, pbcs = pod.pack_batch(cfgs)
    x = torch.tensor(pos, dtype=torch.float64, device="cuda")
    Er = torch.tensor(np.asarray(E_ref, dtype=np.float64), device="cuda")
    Fr = torch.tensor(np.ascontiguousarray(np.concatenate(F_ref, axis=0).T), dtype=torch.float64, device="cuda")
    return x, offs, boxes, pbcs, Er, Fr


def _teacher(pkg, p, Q, cfgs, seed):
    t = pkg.POD(p, precision="fp64", Q=Q)
    cstar = torch.tensor(synth.coefficients(t.M, seed), dtype=torch.float64)
    out = t.energy_forces_batch(cfgs, cstar)
    Fall = out["F"].cpu().numpy()
    offs = out["offs"]
    g = synth.rng(seed + 1)
    E = out["E"].cpu().numpy() + 1e-3 * g.normal(size=len(cfgs))
    F = [Fall[offs[k]:offs[k + 1]] + 1e-2 * g.normal(size=(offs[k + 1] - offs[k], 3)) for k in range(len(cfgs))]
    return E, F


def _configs(n, replica, max_atoms):
    out, k = [], 0
    while len(out) < n:
        cfg = synth.config_train(k, replica)
        k += 1
        if cfg.n <= max_atoms:
            out.append(cfg)
    return out


@pytest.mark.parametrize("prec,solver", [("mixed", "auto"), ("fp64", "auto"), ("mixed", "qr")])
def test_replay_equals_recording_and_recomputes_from_inputs(pkg, prec, solver):
    p = synth.params_full()
    cfgs = _configs(40, 31, 60)
    pod = pkg.POD(p, precision=prec)
    E, F = _teacher(pkg, p, pod.Q, cfgs, 3101)
    x, offs, boxes, pbcs, Er, Fr = _batch(pkg, pod, cfgs, E, F)
    c0, mE0, mF0 = pod.fit_device(x, offs, boxes, pbcs, Er, Fr, solver=solver)
    assert pod.fit_replays() == 0
    c1, mE1, mF1 = pod.fit_device(x, offs, boxes, pbcs, Er, Fr, solver=solver)
    assert pod.fit_replays() == 1
    assert np.array_equal(c0, c1) and mE0 == mE1 and mF0 == mF1
    # new positions and labels in the same arrays: the replay recomputes everything
    g = synth.rng(3102)
    moved = [synth.Config(pos=cf.pos + 0.02 * g.normal(size=cf.pos.shape), box=cf.box, pbc=cf.pbc) for cf in cfgs]
    E2, F2 = _teacher(pkg, p, pod.Q, moved, 3103)
    x2, _, _, _, Er2, Fr2 = _batch(pkg, pod, moved, E2, F2)
    x.copy_(x2)
    Er.copy_(Er2)
    Fr.copy_(Fr2)
    c2, mE2, mF2 = pod.fit_device(x, offs, boxes, pbcs, Er, Fr, solver=solver)
    assert pod.fit_replays() == 2
    ref = pkg.POD(p, precision=prec, Q=pod.Q)
    ref.set_fit_graph(False)
    c3, mE3, mF3 = ref.fit_device(x, offs, boxes, pbcs, Er, Fr, solver=solver)
    c4, _, _ = ref.fit_device(x, offs, boxes, pbcs, Er, Fr, solver=solver)
    assert ref.fit_replays() == 0
    assert np.array_equal(c2, c3) and np.array_equal(c3, c4) and mE2 == mE3 and mF2 == mF3
    assert not np.array_equal(c0, c2)


def test_changed_layout_options_or_timing_take_the_ordinary_path(pkg):
    p = synth.params_full()
    cfgs = _configs(20, 32, 50)
    pod = pkg.POD(p, precision="mixed")
    E, F = _teacher(pkg, p, pod.Q, cfgs, 3201)
    x, offs, boxes, pbcs, Er, Fr = _batch(pkg, pod, cfgs, E, F)
    c0, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)
    pod.fit_device(x, offs, boxes, pbcs, Er, Fr, gamma=1e-10)  # other options: records anew
    assert pod.fit_replays() == 0
    b2 = boxes.copy()
    b2[0] = b2[0] * 1.01  # another layout
    pod.fit_device(x, offs, b2, pbcs, Er, Fr)
    assert pod.fit_replays() == 0
    c1, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)  # records the first layout again
    c2, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)  # replays it
    assert pod.fit_replays() == 1
    assert np.array_equal(c0, c1) and np.array_equal(c1, c2)
    pod.set_timing(True)
    c3, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)
    pod.set_timing(False)
    assert pod.fit_replays() == 1 and np.array_equal(c0, c3)


def test_fallback_to_qr_through_a_replay(pkg):
    """Rank-deficient open dimers: Cholesky fails inside the replay and the QR
    fallback runs on the design matrix the replay formed."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    g = synth.rng(3301)
    cfgs = []
    for _ in range(30):
        r = g.uniform(2.2, 4.8)
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0] + r * u])
        cfgs.append(synth.Config(pos=pos, box=np.array([30.0, 30.0, 30.0]), pbc=(0, 0, 0)))
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    E, F = _teacher(pkg, p, pod.Q, cfgs, 3302)
    x, offs, boxes, pbcs, Er, Fr = _batch(pkg, pod, cfgs, E, F)
    with pytest.raises(pkg.PodError) as ei:
        pod.fit_device(x, offs, boxes, pbcs, Er, Fr, solver="cholesky")
    assert ei.value.code == pkg.POD_ESINGULAR
    c0, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)  # Cholesky fails, QR: recorded
    c1, _, _ = pod.fit_device(x, offs, boxes, pbcs, Er, Fr)  # replay, same fallback
    assert pod.fit_replays() == 1
    assert np.array_equal(c0, c1) and np.all(np.isfinite(c1))
