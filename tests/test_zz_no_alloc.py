"""The allocation-free descriptor entry point, pod_descriptors_static, against
the regular pod_descriptors on the same inputs, through the C ABI.

Some callers cannot let a library allocate device memory (engines that keep all
device memory in their own fixed pool); pod_descriptors_static serves them from
one statically allocated device array.  This file is collected last on purpose
(it shares that array across calls): two calls in a row, on different
configurations, must each match the regular entry point within the descriptor
tolerances used throughout the tests (1e-12 FP64, 1e-5 mixed, per column
relative to the column maximum).
"""
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


def _soa(cfg):
    return torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device="cuda")


def _colerr(D, Dref):
    den = np.max(np.abs(Dref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(D - Dref), axis=0) / den))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_static_matches_regular_twice(pkg, prec, tol):
    p = synth.params_full()
    pod = pkg.POD(p, precision=prec)
    if prec == "mixed":
        pod.set_radial("direct")  # the static entry point evaluates the snapshots per pair
    cfgs = [synth.config_full(0, ncell=8), synth.jitter(synth.bcc(5), 0.1, synth.rng(5))]  # 1024 and 250 atoms
    for cfg in cfgs:  # two calls in a row; the second must not see the first call's leftovers
        x = _soa(cfg)
        sysd = pod.system(x, cfg.box)
        D_static = torch.full((cfg.n, pod.M), float("nan"), dtype=torch.float64, device="cuda")
        pkg.pod_descriptors_static(pod.h, sysd, D_static)
        D_ref = pod.descriptors(x, cfg.box)
        assert torch.isfinite(D_static).all()
        assert _colerr(D_static.cpu().numpy(), D_ref.cpu().numpy()) <= tol


def test_static_rejects_oversized_input(pkg):
    p = synth.params_full()
    pod = pkg.POD(p)
    cfg = synth.bcc(13)  # 4394 atoms > 4096
    x = _soa(cfg)
    D = torch.empty((cfg.n, pod.M), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_descriptors_static(pod.h, pod.system(x, cfg.box), D)
    assert ei.value.code == pkg.POD_EINVAL
    assert "4096" in str(ei.value)
