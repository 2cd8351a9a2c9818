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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("world", [1, 2, 3])
def test_halo_exchange_on_the_device(pkg, prec, world):
    """The device-resident decomposition: each slab (a thread with its own handle)
    keeps its atoms' positions and forces on the GPU, selects its halo layers
    with pod_halo_select, exchanges them with its neighbours (mailboxes between
    the threads standing in for point-to-point messages), evaluates its domain
    and adds the returned ghost forces with pod_halo_add; the owned forces,
    atom energies, E and W equal the whole system's (tolerances as above)."""
    import threading
    from paper_2212_14446_gb300 import parallel
    p = synth.params_full()
    cfg = synth.config_full(3)
    pod0 = pkg.POD(p, precision=prec)
    ct = torch.tensor(synth.coefficients(pod0.M, 131), device="cuda")
    whole = pod0.energy_forces(torch.tensor(cfg.pos.T.copy(), device="cuda"), cfg.box, ct)
    E0, Ei0 = whole["E"].item(), whole["Ei"].cpu().numpy()
    F0, W0 = whole["F"].cpu().numpy(), whole["W"].cpu().numpy()
    tc = parallel.ThreadComm(world)
    pods = [pkg.POD(p, precision=prec, Q=pod0.Q) for _ in range(world)]
    out, errs = [None] * world, []

    def run(r):
        try:
            dom = parallel.SlabDomain(cfg.box, p.r_cut, axis=0, rank=r, world=world)
            own = parallel.owned_atoms(dom, cfg.pos)
            x = torch.tensor(np.ascontiguousarray(cfg.pos[own].T), device="cuda")
            comm = tc.rank(dom) if world > 1 else parallel.LoopComm()
            E, Ei, F, W = parallel.slab_energy_forces(dom, parallel.DeviceOps(pods[r]), x, ct, comm)
            out[r] = (own, E.item(), Ei.cpu().numpy(), F.cpu().numpy(), W.cpu().numpy())
        except Exception as ex:  # surfaced below
            errs.append(ex)

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    F = np.zeros((cfg.n, 3))
    Ei = np.zeros(cfg.n)
    seen = np.zeros(cfg.n, dtype=int)
    for own, _, ei, f, _ in out:
        F[own] = f.T
        Ei[own] = ei
        seen[own] += 1
    assert np.all(seen == 1)
    fmax, wmax = float(np.max(np.abs(F0))), float(np.max(np.abs(W0)))
    for _, E, _, _, W in out:
        W = W.reshape(3, 3)
        if prec == "fp64":
            assert E == pytest.approx(E0, rel=1e-12)
            assert np.max(np.abs(W - W0)) <= 1e-10 * wmax
        else:
            assert E == pytest.approx(E0, rel=1e-6)
            assert np.max(np.abs(W - W0)) <= 1e-5 * wmax
    if prec == "fp64":
        assert np.max(np.abs(Ei - Ei0)) <= 1e-12 * np.max(np.abs(Ei0))
        assert np.max(np.abs(F - F0)) <= 1e-10 * fmax
    else:
        assert np.max(np.abs(F - F0)) <= 1e-4 * max(fmax, 1.0)


def test_halo_select_and_add(pkg):
    """pod_halo_select: ascending selection by the wrapped axis coordinate, the
    image shift and origin applied to that axis only; capacity overflow reported
    with the count; pod_halo_add adds onto the indexed atoms only."""
    p = synth.params_small()
    pod = pkg.POD(p)
    g = synth.rng(141)
    N, L = 2000, 20.0
    pos = g.uniform(-L, 2 * L, size=(3, N))  # some outside the box: wrapped
    x = torch.tensor(pos, device="cuda")
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    out = torch.empty((3, N), dtype=torch.float64, device="cuda")
    k = pkg.pod_halo_select(pod.h, x, 1, L, 3.0, 8.0, L, 1.5, N, idx, out)
    xw = np.mod(pos[1], L)
    want = np.nonzero((xw >= 3.0) & (xw < 8.0))[0]
    assert k == len(want)
    assert np.array_equal(idx[:k].cpu().numpy(), want)
    o = out[:, :k].cpu().numpy()
    assert np.array_equal(o[0], pos[0, want]) and np.array_equal(o[2], pos[2, want])
    assert np.allclose(o[1], xw[want] + L - 1.5, rtol=0, atol=1e-12)
    small = torch.empty(4, dtype=torch.int32, device="cuda")
    small_out = torch.empty((3, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.PodError) as ei:
        pkg.pod_halo_select(pod.h, x, 1, L, 3.0, 8.0, 0.0, 0.0, 4, small, small_out)
    assert ei.value.code == pkg.POD_ENEIGH
    F = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    G = torch.tensor(g.normal(size=(3, k)), device="cuda")
    pkg.pod_halo_add(pod.h, G, idx, k, F)
    Fh = F.cpu().numpy()
    assert np.array_equal(Fh[:, want], G.cpu().numpy())
    rest = np.ones(N, dtype=bool)
    rest[want] = False
    assert np.all(Fh[:, rest] == 0.0)
