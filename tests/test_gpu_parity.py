"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (stated in the spec contract and the readings of the paper):
  * neighbour lists: bit-exact (same (j, s) lists, same order);
  * descriptors: per column m, max_i |dD_im| / max_i |D_im| <= 1e-12 (FP64 path),
    <= 1e-5 (mixed path);
  * energy: |dE| / sum_i sum_m |c_m D_im| <= 1e-12 (FP64), <= 1e-5 (mixed);
  * forces: max |dF| <= 1e-10 * max|F| (FP64), <= 1e-4 eV/A (mixed);
  * virial: same relative bounds as the energy, scaled by max |W|.
The oracle computes its own POD basis; the CUDA path is given the oracle's Q so
both evaluate the same radial functions (the library's own basis is compared
with the oracle's separately in test_lib_cpu.py).
"""
import math

import time

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


DEV = "cuda:0"


def soa(cfg):
    return torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device=DEV)


def desc_err(D, Dref):
    den = np.max(np.abs(Dref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(D - Dref), axis=0) / den))


@pytest.fixture(scope="module")
def small():
    p = synth.params_small()
    o = oracle.Oracle(p)
    cfg = synth.config_small()
    c = synth.coefficients(o.M, 1001)
    return p, o, cfg, c


@pytest.fixture(scope="module")
def full():
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.config_full()
    c = synth.coefficients(o.M, 2001)
    return p, o, cfg, c


@pytest.fixture(scope="module")
def full_oracle_ef(full):
    p, o, cfg, c = full
    return o.energy_forces(cfg, c, fast=True)


def neighbor_compare(pkg, o, p, cfg, atoms, cap=96, tests="auto"):
    pod = pkg.POD(p, Q=o.Q)
    pod.set_neighbor_tests(tests)
    count, nbr, shift = pod.neighbors(soa(cfg), cfg.box, cfg.pbc, cap=cap)
    count, nbr, shift = count.cpu().numpy(), nbr.cpu().numpy(), shift.cpu().numpy()
    for i in atoms:
        js, sh, _ = o.neighbors(cfg, i)
        assert count[i] == len(js), (i, count[i], len(js))
        assert np.array_equal(nbr[i, : len(js)], js), i
        assert np.array_equal(shift[i, : len(js)], sh), i
    return count


# --------------------------------------------------------------- neighbours

def test_neighbors_bitexact_small(pkg, small):
    p, o, cfg, _ = small
    neighbor_compare(pkg, o, p, cfg, range(cfg.n))


@pytest.mark.parametrize("tests", ["blockwide", "warp"])
def test_neighbors_bitexact_full_sampled(pkg, full, tests):
    """8,192 atoms: the block-per-cell search, with either form of its candidate tests."""
    p, o, cfg, _ = full
    g = synth.rng(5)
    count = neighbor_compare(pkg, o, p, cfg, g.choice(cfg.n, 200, replace=False), tests=tests)
    assert 18 <= count.min() and count.max() <= 40


@pytest.mark.parametrize("tests", ["blockwide", "warp"])
def test_neighbors_cell_search_on_cutoff_band(pkg, full, tests):
    """The block-per-cell search decides pairs at r_cut (1 -+ 1e-7), r_cut and
    r_cut (1 - 1e-15) -- some across the periodic boundary -- in the exact FP64
    band like the oracle."""
    p, o, cfg0, _ = full
    pos = cfg0.pos.copy()
    rc = p.r_cut
    L = cfg0.box
    moved = []
    for k, (f, u) in enumerate([(1 - 1e-7, (1, 0, 0)), (1 + 1e-7, (0, 1, 0)), (1.0, (0, 0, 1)),
                                (1 - 1e-15, (1, 1, 0)), (1 + 1e-7, (-1, 0, 1)), (1 - 1e-7, (0, -1, -1))]):
        i, j = 1000 * k + 3, 1000 * k + 611
        u = np.array(u, dtype=np.float64)
        pos[j] = np.mod(pos[i] + rc * f * u / np.linalg.norm(u), L)
        moved += [i, j]
    pos[moved[-2]] = np.array([0.25, 7.0, 9.0])  # the last pair straddles the x = 0 face
    pos[moved[-1]] = np.mod(pos[moved[-2]] + rc * (1 - 1e-7) * np.array([-1.0, 0.0, 0.0]), L)
    cfg = synth.Config(pos=pos, box=L, pbc=cfg0.pbc)
    g = synth.rng(6)
    neighbor_compare(pkg, o, p, cfg, sorted(set(moved) | set(g.choice(cfg.n, 40, replace=False).tolist())),
                     tests=tests)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 5, 8, 13, 21])
def test_neighbors_bitexact_training_configs(pkg, k):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.config_train(k)
    neighbor_compare(pkg, o, p, cfg, range(cfg.n), cap=160)


def test_neighbors_open_cluster(pkg):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.cluster(12, 44)
    neighbor_compare(pkg, o, p, cfg, range(cfg.n))


def test_neighbors_on_cutoff_band(pkg):
    """Pairs at r = r_cut (1 - 1e-6) and r_cut (1 + 1e-6) decide in the exact FP64 band."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    rc = p.r_cut
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + rc * (1 - 1e-6), 5.0, 5.0], [5.0, 5.0 + rc * (1 + 1e-6), 5.0],
                    [5.0, 5.0, 5.0 + rc], [5.0 - rc * (1 - 1e-15), 5.0, 5.0]])
    cfg = synth.Config(pos=pos, box=np.array([30.0, 30.0, 30.0]), pbc=(0, 0, 0))
    neighbor_compare(pkg, o, p, cfg, range(cfg.n))


# ------------------------------------------------------------- descriptors

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_descriptors_small(pkg, small, prec, tol):
    p, o, cfg, _ = small
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    D = pod.descriptors(soa(cfg), cfg.box).cpu().numpy()
    Dref = o.descriptors(cfg, fast=False)
    assert desc_err(D, Dref) <= tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_descriptors_full_sampled(pkg, full, prec, tol):
    p, o, cfg, _ = full
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    D = pod.descriptors(soa(cfg), cfg.box).cpu().numpy()
    atoms = synth.rng(9).choice(cfg.n, 40, replace=False)
    Dref = o.descriptors(cfg, atoms=atoms, fast=False)
    assert desc_err(D[atoms], Dref) <= tol
    assert np.all(D[:, 0] == 1.0)
    # D3 >= 0 everywhere (Eq. 26a is a sum of squares)
    M3 = slice(1 + p.K2, 1 + p.K2 + p.K3 * (p.P3 + 1))
    assert np.all(D[:, M3] >= 0)


@pytest.mark.parametrize("kw", [
    dict(K2=5, K3=3, K4=3, P3=2, P4=2),                     # Table 6 row 2 sizes, generic kernel
    dict(K2=2, K3=1, K4=1, P3=2, P4=1),                     # Table 6 row 1 sizes
    dict(K2=4, K3=4, K4=0, P3=4, P4=-1),                    # three-body only, P = 4
    dict(K2=3, K3=0, K4=0, P3=-1, P4=-1),                   # two-body only
    dict(alpha=[1.5, 2.5], beta=[2.0, 4.0], gamma=[0.5, 1.5, 2.5], K2=5, K3=5, K4=5, P3=3, P4=3),
])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_descriptors_generic_params(pkg, kw, prec, tol):
    p = synth.PODParams(**{**synth.params_full().__dict__, **kw})
    o = oracle.Oracle(p)
    cfg = synth.config_train(7)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    D = pod.descriptors(soa(cfg), cfg.box).cpu().numpy()
    Dref = o.descriptors(cfg, fast=True)
    assert D.shape == Dref.shape
    assert desc_err(D, Dref) <= tol


def test_mixed_direct_radial_mode(pkg, full):
    """The mixed path can also evaluate the snapshots per pair in FP32 and project
    them (Eq. 3-12); the POD cancellation of the small modes then costs about an
    order of magnitude over the tabulated default (stated bound: 5e-5)."""
    p, o, cfg, _ = full
    pod = pkg.POD(p, precision="mixed", Q=o.Q)
    pod.set_radial("direct")
    D = pod.descriptors(soa(cfg), cfg.box).cpu().numpy()
    atoms = synth.rng(9).choice(cfg.n, 40, replace=False)
    Dref = o.descriptors(cfg, atoms=atoms, fast=True)
    assert desc_err(D[atoms], Dref) <= 5e-5


# --------------------------------------------------------- energy and forces

def energy_scale(o, cfg, c, atoms=None):
    D = o.descriptors(cfg, atoms=atoms, fast=True)
    return float(np.sum(np.abs(D * c[None, :])))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_energy_forces_small(pkg, small, prec):
    p, o, cfg, c = small
    Ei_o, E_o, F_o, W_o = o.energy_forces(cfg, c, fast=True)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    out = pod.energy_forces(soa(cfg), cfg.box, torch.tensor(c, device=DEV))
    check_ef(out, Ei_o, E_o, F_o, W_o, energy_scale(o, cfg, c), prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_energy_forces_full(pkg, full, full_oracle_ef, prec):
    p, o, cfg, c = full
    Ei_o, E_o, F_o, W_o = full_oracle_ef
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    out = pod.energy_forces(soa(cfg), cfg.box, torch.tensor(c, device=DEV))
    check_ef(out, Ei_o, E_o, F_o, W_o, energy_scale(o, cfg, c, atoms=range(0, cfg.n, 7)) * 7, prec)


def check_ef(out, Ei_o, E_o, F_o, W_o, escale, prec):
    E = out["E"].item()
    Ei = out["Ei"].cpu().numpy()
    F = out["F"].cpu().numpy()
    W = out["W"].cpu().numpy()
    tol_e = 1e-12 if prec == "fp64" else 1e-5
    assert abs(E - E_o) / escale <= tol_e
    assert np.max(np.abs(Ei - Ei_o)) / (escale / len(Ei)) <= 50 * tol_e
    fmax = np.max(np.abs(F_o))
    errF = np.max(np.abs(F - F_o))
    if prec == "fp64":
        assert errF <= 1e-10 * fmax, (errF, fmax)
    else:
        assert errF <= 1e-4, (errF, fmax)
    wmax = np.max(np.abs(W_o))
    assert np.max(np.abs(W - W_o)) <= (1e-10 if prec == "fp64" else 1e-5) * max(wmax, escale)


def test_forces_sampled_against_naive_oracle(pkg, full):
    """Forces on a few atoms of the 8,192-atom configuration from the naive
    (triple-sum) oracle derivative, one atom at a time."""
    p, o, cfg, c = full
    atoms = [0, 4097]
    _, _, Fn, _ = o.energy_forces(cfg, c, fast=False, force_atoms=atoms)
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    F = pod.energy_forces(soa(cfg), cfg.box, torch.tensor(c, device=DEV))["F"].cpu().numpy()
    assert np.max(np.abs(F[atoms] - Fn)) <= 1e-10 * max(1.0, np.max(np.abs(Fn)))


def test_forces_fd_on_gpu(pkg):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(12))
    c = torch.tensor(synth.coefficients(o.M, 13), device=DEV)
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    x = soa(cfg)
    F = pod.energy_forces(x, cfg.box, c)["F"].cpu().numpy()
    h = 1e-5
    for k, t in [(0, 0), (7, 1), (30, 2)]:
        xp = x.clone()
        xm = x.clone()
        xp[t, k] += h
        xm[t, k] -= h
        Ep = pod.energy_forces(xp, cfg.box, c)["E"].item()
        Em = pod.energy_forces(xm, cfg.box, c)["E"].item()
        assert F[k, t] == pytest.approx(-(Ep - Em) / (2 * h), abs=1e-6 * max(1.0, abs(F[k, t])))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_deterministic(pkg, full, prec):
    p, o, cfg, c = full
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    x = soa(cfg)
    ct = torch.tensor(c, device=DEV)
    a = pod.energy_forces(x, cfg.box, ct)
    b = pod.energy_forces(x, cfg.box, ct)
    for k in ("E", "Ei", "F", "W"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_one_handle_many_systems(pkg, full, prec):
    """A handle that alternates between systems (cell grids of different sizes;
    the block-per-cell search for 16^3 and 12^3 cells, the warp-per-atom search
    for 4^3) gives, on every call, the results of a fresh handle bit for bit:
    nothing a call leaves in the workspace (cell counts, accumulators, lists)
    leaks into the next."""
    p, o, cfg, c = full
    systems = {"a": cfg, "b": synth.config_full(1, ncell=12), "c": synth.config_full(2, ncell=4)}
    ct = torch.tensor(c, device=DEV)
    fresh = {}
    for name, cf in systems.items():
        pod = pkg.POD(p, precision=prec, Q=o.Q)
        fresh[name] = pod.energy_forces(soa(cf), cf.box, ct)
        pod.close()
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    for name in ("a", "b", "a", "c", "a", "a", "c", "b", "b", "a"):
        cf = systems[name]
        out = pod.energy_forces(soa(cf), cf.box, ct)
        for k in ("E", "Ei", "F", "W"):
            assert torch.equal(out[k], fresh[name][k]), (name, k)


def test_host_entry_point(pkg, small):
    p, o, cfg, c = small
    pod = pkg.POD(p, precision="mixed", Q=o.Q)
    dev = pod.energy_forces(soa(cfg), cfg.box, torch.tensor(c, device=DEV))
    host = pod.energy_forces_host(np.ascontiguousarray(cfg.pos.T), cfg.box, c)
    assert host["E"][0] == dev["E"].item()
    assert np.array_equal(host["F"], dev["F"].cpu().numpy())
    assert np.array_equal(host["W"], dev["W"].cpu().numpy())


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_isolated_atom_and_dimer(pkg, prec):
    p = synth.params_full()
    o = oracle.Oracle(p)
    c = synth.coefficients(o.M, 3)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    one = synth.Config(pos=np.array([[3.0, 3.0, 3.0]]), box=np.array([10.0, 10.0, 10.0]), pbc=(0, 0, 0))
    D = pod.descriptors(soa(one), one.box, one.pbc).cpu().numpy()
    assert D[0, 0] == 1.0 and np.all(D[0, 1:] == 0)
    out = pod.energy_forces(soa(one), one.box, torch.tensor(c, device=DEV), pbc=one.pbc)
    # the mixed path forms E_i in FP32, so c_0 is rounded to single precision
    assert out["E"].item() == pytest.approx(c[0], rel=1e-12 if prec == "fp64" else 1e-7)
    assert np.all(out["F"].cpu().numpy() == 0)
    dim = synth.Config(pos=np.array([[3.0, 3.0, 3.0], [5.1, 3.7, 2.2]]), box=np.array([10.0, 10.0, 10.0]),
                       pbc=(0, 0, 0))
    D = pod.descriptors(soa(dim), dim.box, dim.pbc).cpu().numpy()
    Dref = o.descriptors(dim, fast=False)
    if prec == "fp64":
        assert desc_err(D, Dref) <= 1e-12
    else:
        # One pair: every column's scale is its single value, and some modes are
        # near a zero crossing at this distance (d ln R_k / dr ~ 22 / A for the
        # sixth), so the FP32 rounding of r itself moves a column by more than
        # 1e-5 of its value.  Tolerance: 1e-5 of the value plus the change from 4
        # ulps of r through dD/dr (the oracle's explicit derivative).
        d = dim.pos[1] - dim.pos[0]
        r = float(np.linalg.norm(d))
        dD = o.atom_dD(d.reshape(1, 3))[0]               # (M, 3): dD / dr_ij
        dDdr = np.abs(dD @ (d / r))
        tol = 1e-5 * np.abs(Dref[0]) + 4 * float(np.spacing(np.float32(r))) * dDdr
        assert np.all(np.abs(D - Dref) <= tol[None, :] + 1e-12)


def test_error_codes(pkg):
    p = synth.params_full()
    pod = pkg.POD(p)
    c = torch.zeros(pod.M, dtype=torch.float64, device=DEV)
    close = synth.Config(pos=np.array([[3.0, 3.0, 3.0], [3.5, 3.0, 3.0]]), box=np.array([10.0] * 3), pbc=(0, 0, 0))
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(soa(close), close.box, c, pbc=close.pbc)
    assert ei.value.code == pkg.POD_ERANGE
    nanc = synth.Config(pos=np.array([[3.0, 3.0, float("nan")], [5.5, 3.0, 3.0]]), box=np.array([10.0] * 3),
                        pbc=(1, 1, 1))
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(soa(nanc), nanc.box, c)
    assert ei.value.code == pkg.POD_ENONFINITE
    # the handle stays usable after errors
    ok = synth.config_small()
    pod.energy_forces(soa(ok), ok.box, c)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_workspace_limit_reports_enomem(pkg, full, prec):
    """An allocation failure injected on the host: with a 1 MiB workspace cap the
    8,192-atom call cannot grow its buffers and returns POD_ENOMEM (nothing is
    freed or allocated past the cap, no kernel faults); with the cap cleared the
    same handle gives the bits of a fresh one."""
    p, o, cfg, c = full
    ct = torch.tensor(c, device=DEV)
    pod = pkg.POD(p, precision=prec)
    pod.set_workspace_limit_mb(1)
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(soa(cfg), cfg.box, ct)
    assert ei.value.code == pkg.POD_ENOMEM
    assert "limit" in str(ei.value)
    pod.set_workspace_limit_mb(0)
    a = pod.energy_forces(soa(cfg), cfg.box, ct)
    b = pkg.POD(p, precision=prec).energy_forces(soa(cfg), cfg.box, ct)
    for k in ("E", "F", "W"):
        assert torch.equal(a[k], b[k]), k


def test_bounded_wait_reports_timeout(pkg):
    """The bounded mbarrier wait of the tensor-core kernels, on a barrier that
    nothing arrives at: it gives up after its limit (50 ms here), reports
    ST_TIMEOUT (64) through the status word, and the context stays usable."""
    t0 = time.perf_counter()
    st = pkg.pod_selftest_wait(50_000_000)
    elapsed = time.perf_counter() - t0
    assert st == 64
    assert 0.04 <= elapsed < 5.0
    ok = synth.config_small()
    pod = pkg.POD(synth.params_full())
    c = torch.zeros(pod.M, dtype=torch.float64, device=DEV)
    out = pod.energy_forces(soa(ok), ok.box, c)
    assert float(out["E"]) == 0.0


def test_mixed_energy_virial_totals(pkg, full):
    """Mixed path: E and the virial are exact fixed-point sums (2^-36 grid) of the
    FP32 atom energies and per-warp virial sums.  E equals the exact sum of the
    returned E_i to within half a grid step per atom; W agrees with the FP64 path
    within the mixed tolerance; coefficients that push atom energies past the
    accumulator range are reported (POD_ERANGE) and the handle stays usable."""
    p, o, cfg, c = full
    ct = torch.tensor(c, device=DEV)
    pod = pkg.POD(p, precision="mixed", Q=o.Q)
    out = pod.energy_forces(soa(cfg), cfg.box, ct)
    Ei = out["Ei"].cpu().numpy()
    s = math.fsum(Ei.tolist())
    assert abs(out["E"].item() - s) <= len(Ei) * 2.0 ** -37 + 1e-15 * abs(s)
    ref = pkg.POD(p, precision="fp64", Q=o.Q).energy_forces(soa(cfg), cfg.box, ct)
    W, W64 = out["W"].cpu().numpy(), ref["W"].cpu().numpy()
    assert np.max(np.abs(W - W64)) <= 1e-5 * np.max(np.abs(W64))
    with pytest.raises(pkg.PodError) as ei:
        pod.energy_forces(soa(cfg), cfg.box, ct * 1e9)
    assert ei.value.code == pkg.POD_ERANGE
    again = pod.energy_forces(soa(cfg), cfg.box, ct)
    assert torch.equal(again["E"], out["E"]) and torch.equal(again["F"], out["F"])


@pytest.mark.parametrize("tests", ["blockwide", "warp"])
def test_capacity_retry(pkg, tests):
    """A dense cluster in a large open box: the density-based capacity estimate
    is far too small, the call overflows, grows its lists and succeeds (the
    block-per-cell search, with either form of its candidate tests)."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    g = synth.rng(17)
    pts = []
    while len(pts) < 60:
        q = g.uniform(-3.5, 3.5, size=3)
        if all(np.linalg.norm(q - r) > 1.2 for r in pts):
            pts.append(q)
    cfg = synth.Config(pos=np.array(pts) + 40.0, box=np.array([80.0, 80.0, 80.0]), pbc=(0, 0, 0))
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    pod.set_neighbor_tests(tests)
    D = pod.descriptors(soa(cfg), cfg.box, cfg.pbc).cpu().numpy()
    Dref = o.descriptors(cfg, atoms=range(0, 60, 6), fast=True)
    assert desc_err(D[::6], Dref) <= 1e-12


def test_fma_probe(pkg):
    """The vector-pipe probe launches, reports its flop count and gives a rate
    below any physical ceiling (a far higher one would mean elided work)."""
    s = torch.cuda.Stream()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for kind, iters in ((0, 64), (1, 64), (2, 4)):
        fl = pkg.pod_fma_probe(kind, iters, s)
        assert fl == 2 * 16 * 8 * iters * nsm * 8 * 256
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            t0.record(s)
            pkg.pod_fma_probe(kind, iters * 16, s)
            t1.record(s)
        torch.cuda.synchronize()
        tflops = 16 * fl / (t0.elapsed_time(t1) / 1e3) / 1e12
        assert 0.1 < tflops < 400.0
    with pytest.raises(pkg.PodError):
        pkg.pod_fma_probe(3, 1, s)


@pytest.mark.parametrize("prec,mapped", [("fp64", True), ("mixed", True), ("fp64", False), ("mixed", False)])
def test_host_entry_graph_replay(pkg, prec, mapped):
    """Repeated host-buffer calls with the same pinned buffers on a stream replay a
    captured graph: every call (direct, capturing, replayed) equals the device
    entry point bit for bit, including after the positions and the coefficients
    change in place.  Both graph forms: kernels on the mapped pinned buffers, or
    copies in and out."""
    import ctypes as C
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(4), 0.1, synth.rng(91))
    n = cfg.n
    pod = pkg.POD(p, precision=prec)
    pod.set_host_mapped(mapped)
    c = synth.coefficients(pod.M, 92)
    s = torch.cuda.Stream()
    pos_t = torch.tensor(np.ascontiguousarray(cfg.pos.T)).pin_memory()
    c_t = torch.tensor(c).pin_memory()
    E_t = torch.zeros(1, dtype=torch.float64).pin_memory()
    Ei_t = torch.zeros(n, dtype=torch.float64).pin_memory()
    F_t = torch.zeros((3, n), dtype=torch.float64).pin_memory()
    W_t = torch.zeros(9, dtype=torch.float64).pin_memory()
    pos_h, c_h, E_h, Ei_h, F_h, W_h = (t.numpy() for t in (pos_t, c_t, E_t, Ei_t, F_t, W_t))
    sysd = pkg.make_system(pos_h.ctypes.data_as(C.POINTER(C.c_double)), n, cfg.box)
    rng = synth.rng(93)
    prepared = pkg.HostEnergyForces(pod.h, sysd, c_h, E_h, Ei_h, F_h, W_h, stream=s)
    for call in range(8):
        if call == 4:  # new positions in the same buffer: the replay must take them
            pos_h[...] = np.ascontiguousarray((cfg.pos + rng.normal(0, 0.02, size=cfg.pos.shape)).T)
        if call == 6:  # new coefficients in the same buffer
            c = synth.coefficients(pod.M, 94)
            c_h[...] = c
        if call % 2:  # the prepared repeated-call form, the same entry point
            prepared()
        else:
            pkg.pod_energy_forces_host(pod.h, sysd, c_h, E_h, Ei_h, F_h, W_h, stream=s)
        dev = pod.energy_forces(torch.tensor(pos_h, device=DEV), cfg.box, torch.tensor(c, device=DEV))
        assert E_h[0] == dev["E"].item(), call
        assert np.array_equal(F_h.T, dev["F"].cpu().numpy()), call
        assert np.array_equal(Ei_h, dev["Ei"].cpu().numpy()), call
        assert np.array_equal(W_h, dev["W"].cpu().numpy().ravel()), call


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_host_graph_replay_without_optional_outputs(pkg, prec):
    """Host-buffer replays with E_i and W left NULL (E and F only): the mapped graph
    writes just those, and every call equals the device entry point."""
    import ctypes as C
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(5), 0.08, synth.rng(98))
    n = cfg.n
    pod = pkg.POD(p, precision=prec)
    c = synth.coefficients(pod.M, 99)
    s = torch.cuda.Stream()
    pos_t = torch.tensor(np.ascontiguousarray(cfg.pos.T)).pin_memory()
    c_t = torch.tensor(c).pin_memory()
    E_t = torch.zeros(1, dtype=torch.float64).pin_memory()
    F_t = torch.zeros((3, n), dtype=torch.float64).pin_memory()
    pos_h, c_h, E_h, F_h = (t.numpy() for t in (pos_t, c_t, E_t, F_t))
    sysd = pkg.make_system(pos_h.ctypes.data_as(C.POINTER(C.c_double)), n, cfg.box)
    call = pkg.HostEnergyForces(pod.h, sysd, c_h, E_h, None, F_h, None, stream=s)
    rng = synth.rng(100)
    for k in range(5):
        if k == 3:
            pos_h[...] = np.ascontiguousarray((cfg.pos + rng.normal(0, 0.02, size=cfg.pos.shape)).T)
        call()
        dev = pod.energy_forces(torch.tensor(pos_h, device=DEV), cfg.box, torch.tensor(c, device=DEV))
        assert E_h[0] == dev["E"].item(), k
        assert np.array_equal(F_h.T, dev["F"].cpu().numpy()), k


@pytest.mark.parametrize("mapped", [True, False])
def test_host_graph_replay_redoes_an_overflowing_call(pkg, mapped):
    """A replayed host-buffer call whose cell and neighbour lists overflow (the
    positions changed in place into a dense cluster) reports it through the status
    word the graph hands back, drops the graph and redoes the call on the direct
    path with larger capacities: every call equals the device entry point."""
    import ctypes as C
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(4), 0.05, synth.rng(95))  # 128 atoms, 2 x 2 x 2 cells
    n, L = cfg.n, cfg.box
    pod = pkg.POD(p, precision="mixed")
    pod.set_host_mapped(mapped)
    c = synth.coefficients(pod.M, 96)
    s = torch.cuda.Stream()
    pos_t = torch.tensor(np.ascontiguousarray(cfg.pos.T)).pin_memory()
    c_t = torch.tensor(c).pin_memory()
    E_t = torch.zeros(1, dtype=torch.float64).pin_memory()
    F_t = torch.zeros((3, n), dtype=torch.float64).pin_memory()
    W_t = torch.zeros(9, dtype=torch.float64).pin_memory()
    pos_h, c_h, E_h, F_h, W_h = (t.numpy() for t in (pos_t, c_t, E_t, F_t, W_t))
    sysd = pkg.make_system(pos_h.ctypes.data_as(C.POINTER(C.c_double)), n, L)
    call = pkg.HostEnergyForces(pod.h, sysd, c_h, E_h, None, F_h, W_h, stream=s)
    # atoms 0..59 moved into one 6 A cube (one cell), at least 1.2 A (> r_in) from
    # every other atom and periodic image
    g = synth.rng(97)
    dense = cfg.pos.copy()
    placed = [q for q in dense[60:]]
    for i in range(60):
        while True:
            q = g.uniform(0.3, 6.3, size=3)
            d = np.asarray(placed) - q
            d -= L * np.round(d / L)
            if np.min(np.linalg.norm(d, axis=1)) > 1.2:
                break
        dense[i] = q
        placed.append(q)

    def check(x, tag):
        dev = pod.energy_forces(torch.tensor(np.ascontiguousarray(x.T), device=DEV), L, torch.tensor(c, device=DEV))
        assert E_h[0] == dev["E"].item(), tag
        assert np.array_equal(F_h.T, dev["F"].cpu().numpy()), tag
        assert np.array_equal(W_h, dev["W"].cpu().numpy().ravel()), tag

    for k in range(3):  # direct, capturing, replayed
        call()
        check(cfg.pos, k)
    pos_h[...] = np.ascontiguousarray(dense.T)
    for k in range(3, 7):  # the replay overflows and is redone; then direct, capture, replay
        call()
        check(dense, k)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_model_file_evaluates_like_the_saved_handle(pkg, full, prec, tmp_path):
    """A handle loaded from a model file (parameters, Q, c) gives the saved
    handle's energies and forces bit for bit."""
    p, o, cfg, c = full
    pod = pkg.POD(p, precision=prec)
    path = str(tmp_path / "ta.pod")
    pod.save(path, c)
    pod2, c2 = pkg.POD.load(path, prec)
    x = soa(cfg)
    a = pod.energy_forces(x, cfg.box, torch.tensor(c, device=DEV))
    b = pod2.energy_forces(x, cfg.box, torch.tensor(c2, device=DEV))
    for k in ("E", "Ei", "F", "W"):
        assert torch.equal(a[k], b[k]), k
