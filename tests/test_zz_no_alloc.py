"""The allocation-free descriptor entry point, pod_descriptors_static, through the
C ABI.

Some callers cannot let a library allocate device memory: engines that keep all
device memory in their own fixed pool and forbid cudaMalloc/cudaFree (both
synchronise the device and fragment the pool).  pod_descriptors_static serves
them from one statically allocated device array.  This file is collected last on
purpose (the calls share that array), and every test here also passes when the
file runs alone in a fresh process.

Checked: two calls in a row on different configurations, each against the FP64
oracle (per-column error relative to the column maximum: 1e-12 on the FP64 path,
1e-5 on the mixed path) and against the regular pod_descriptors on the same
handle (the same kernels: bit for bit); free device memory unchanged across a
call; a sparse box whose cell grid is coarsened to the array's cell limit; a dense
lattice past the 64-neighbour limit (POD_ENEIGH); refused inputs.
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


def _soa(cfg):
    return torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device="cuda")


def _colerr(D, Dref):
    den = np.max(np.abs(Dref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(D - Dref), axis=0) / den))


def _static(pkg, pod, cfg):
    x = _soa(cfg)
    D = torch.full((cfg.n, pod.M), float("nan"), dtype=torch.float64, device="cuda")
    pkg.pod_descriptors_static(pod.h, pod.system(x, cfg.box), D)
    return D, x


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_static_matches_oracle_and_regular_twice(pkg, prec, tol):
    p = synth.params_full()
    pod = pkg.POD(p, precision=prec)
    orc = oracle.Oracle(p, Q=pod.Q)
    cfgs = [synth.config_full(0, ncell=8), synth.jitter(synth.bcc(5), 0.1, synth.rng(5))]  # 1024 and 250 atoms
    for cfg in cfgs:  # two calls in a row; the second must not see the first call's leftovers
        D_static, x = _static(pkg, pod, cfg)
        assert torch.isfinite(D_static).all()
        atoms = np.arange(0, cfg.n, 7)
        D_orc = orc.descriptors(cfg, atoms=atoms)
        assert _colerr(D_static.cpu().numpy()[atoms], D_orc) <= tol
        D_ref = pod.descriptors(x, cfg.box)
        assert torch.equal(D_static, D_ref)


def test_static_call_takes_no_device_memory(pkg):
    p = synth.params_full()
    pod = pkg.POD(p, precision="mixed")
    cfg = synth.config_full(1, ncell=8)
    x = _soa(cfg)
    sysd = pod.system(x, cfg.box)
    D = torch.empty((cfg.n, pod.M), dtype=torch.float64, device="cuda")
    pkg.pod_descriptors_static(pod.h, sysd, D)  # first call: loads kernels, copies the table
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    D1 = D.clone()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    pkg.pod_descriptors_static(pod.h, sysd, D)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1, (free0, free1, free2)
    assert torch.equal(D, D1)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_static_sparse_box_coarsened_grid(pkg, prec, tol):
    # 2,000 atoms in a 200 A periodic box: 40^3 cells of r_cut, coarsened to the
    # array's 8,192-cell limit (20^3 cells of 10 A, search depth one cell)
    g = synth.rng(77)
    cfg = synth.liquid(2000, g, density=2000 / 200.0 ** 3, dmin=2.0)
    p = synth.params_full()
    pod = pkg.POD(p, precision=prec)
    D_static, x = _static(pkg, pod, cfg)
    D_ref = pod.descriptors(x, cfg.box)
    assert torch.equal(D_static, D_ref)
    counts = pod.neighbors(x, cfg.box, cap=64)[0].cpu().numpy()
    busy = np.argsort(-counts, kind="stable")[:20]  # the atoms with the most neighbours
    assert counts[busy[0]] >= 1
    orc = oracle.Oracle(p, Q=pod.Q)
    D_orc = orc.descriptors(cfg, atoms=busy)
    assert _colerr(D_static.cpu().numpy()[busy], D_orc) <= tol


def test_static_dense_lattice_reports_neighbour_limit(pkg):
    # BCC with a = 2.3 A: ~86 neighbours within 5 A, above the 64-neighbour limit
    cfg = synth.bcc(5, a=2.3)
    pod = pkg.POD(synth.params_full())
    x = _soa(cfg)
    D = torch.empty((cfg.n, pod.M), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_descriptors_static(pod.h, pod.system(x, cfg.box), D)
    assert ei.value.code == pkg.POD_ENEIGH
    # the handle and the array stay usable: a regular system right after
    cfg2 = synth.config_small(0)
    pod2 = pkg.POD(synth.params_small(), precision="fp64")
    D2, x2 = _static(pkg, pod2, cfg2)
    assert torch.equal(D2, pod2.descriptors(x2, cfg2.box))


def test_static_rejects_oversized_and_ghost_input(pkg):
    p = synth.params_full()
    pod = pkg.POD(p)
    cfg = synth.bcc(13)  # 4394 atoms > 4096
    x = _soa(cfg)
    D = torch.empty((cfg.n, pod.M), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_descriptors_static(pod.h, pod.system(x, cfg.box), D)
    assert ei.value.code == pkg.POD_EINVAL
    assert "4096" in str(ei.value)
    cfg = synth.config_small(0)
    x = _soa(cfg)
    D = torch.empty((cfg.n, pod.M), dtype=torch.float64, device="cuda")
    sysd = pod.system(x, cfg.box)
    sysd.n_local = 64  # ghost atoms are not taken by the allocation-free entry point
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_descriptors_static(pod.h, sysd, D)
    assert ei.value.code == pkg.POD_EINVAL
