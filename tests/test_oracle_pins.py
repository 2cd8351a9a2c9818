"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the printed
tables, closed forms for dimers and trimers, identities between the two forms
of the descriptors (Eq. 15c, Eq. 27a, Table 2 sums), invariances, a library
eigen-solver, and finite differences.  None of them needs a GPU.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def _N(n):
    return (n + 1) * (n + 2) // 2


# ----------------------------------------------------------------- tables

def test_table3_monomial_order():
    gold = np.array(read_golden("table3_monomials_p4.txt", int))
    e, _ = oracle.monomial_table(4)
    assert e.shape == (35, 3)
    assert np.array_equal(e.sum(1), gold[:, 0])
    assert np.array_equal(e, gold[:, 1:])


def test_table4_multinomial_coefficients():
    gold = read_golden("table4_multinomial_p4.txt", int)
    e, c = oracle.monomial_table(4)
    deg = e.sum(1)
    for n, row in enumerate(gold):
        assert list(c[deg == n].astype(int)) == row
        assert sum(row) == 3 ** n  # (1 + 1 + 1)^n


def test_table1_fourbody_functions():
    gold = np.array(read_golden("table1_fourbody_p4.txt", int))
    assert np.array_equal(oracle.fourbody_table(4), gold)


def test_table5_counts():
    for P, Ka, Na, Ca, ratio in read_golden("table5_complexity.txt", int):
        assert oracle.num_fourbody(P) == Ka
        assert oracle.num_monomials(P) == Na
        # C_a = number of (q, s, t) products of Eq. 30a over all partitions a >= b >= c
        ca = sum(_N(a) * _N(b) * _N(c) for a, b, c in oracle.fourbody_table(P))
        assert ca == Ca
        # The printed ratio for P = 10 is 75 while 21304 / 286 = 74.49 rounds to 74:
        # a misprint in the table (C_a and N_a themselves are reproduced exactly).
        if P == 10:
            assert ratio == 75 and int(math.floor(Ca / Na + 0.5)) == 74
        else:
            assert int(math.floor(Ca / Na + 0.5)) == ratio


def test_table6_descriptor_counts():
    for K2, K3, P3, M3, K4, P4, M4 in read_golden("table6_descriptor_counts.txt", int):
        p3 = synth.PODParams(K2=K2, K3=K3, K4=1, P3=P3, P4=-1,
                             alpha=[1.0] * 1, beta=[3.0], gamma=list(range(1, 40)))
        p4 = synth.PODParams(K2=K2, K3=K3, K4=K4, P3=P3, P4=P4,
                             alpha=[1.0] * 1, beta=[3.0], gamma=list(range(1, 40)))
        assert oracle.lib().orc_num_descriptors(_pp(p3)) == M3
        assert oracle.lib().orc_num_descriptors(_pp(p4)) == M4


def _pp(p):
    import ctypes as C
    a = np.asarray(p.alpha, float)
    b = np.asarray(p.beta, float)
    g = np.asarray(p.gamma, float)
    _pp.keep = (a, b, g)
    s = oracle._Params(p.r_in, p.r_cut, len(a), oracle._dp(a), len(b), oracle._dp(b), len(g), oracle._dp(g),
                       p.K2, p.K3, p.K4, p.P3, p.P4)
    _pp.s = s
    return C.byref(s)


def test_multinomial_identity():
    g = synth.rng(7)
    e, c = oracle.monomial_table(10)
    deg = e.sum(1)
    for _ in range(20):
        u = g.normal(size=3)
        v = g.normal(size=3)
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        Au = np.prod(u[None, :] ** e, axis=1)
        Av = np.prod(v[None, :] ** e, axis=1)
        for n in range(11):
            s = np.sum((c * Au * Av)[deg == n])
            assert s == pytest.approx(np.dot(u, v) ** n, rel=1e-13, abs=1e-14)


# ------------------------------------------------------ radial functions

@pytest.fixture(scope="module")
def orc_full():
    return oracle.Oracle(synth.params_full())


@pytest.fixture(scope="module")
def orc_small():
    return oracle.Oracle(synth.params_small())


def test_snapshot_special_values(orc_full):
    p = orc_full.params
    beta = p.beta[0]
    h = p.r_cut - p.r_in
    # x(r) = 1/2  <=>  exp(-beta t) = (1 + exp(-beta)) / 2
    t = -math.log((1 + math.exp(-beta)) / 2) / beta
    r = p.r_in + t * h
    phi, _ = orc_full.snapshots(r)
    # phi_alpha = f_c sin(alpha pi / 2) / (r - r_in): alpha = 1, 2, 3, 4 -> +1, 0, -1, 0
    assert phi[2] / phi[0] == pytest.approx(-1.0, rel=1e-13)
    assert abs(phi[1] / phi[0]) < 1e-14 and abs(phi[3] / phi[0]) < 1e-14
    # f_c = (r - r_in) * phi_1 here, so varphi_gamma / f_c = r^-gamma
    fc = (r - p.r_in) * phi[0]
    for k, gam in enumerate(p.gamma):
        assert phi[4 + k] / fc == pytest.approx(r ** -gam, rel=1e-13)
    # cut-off limits: f_c(r_in) = exp(1 - (1 + eps)^-1/2), f_c -> 0 at r_cut
    phi_in, _ = orc_full.snapshots(p.r_in + 1e-9)
    fc_in = phi_in[4] * (p.r_in + 1e-9)  # gamma = 1
    assert fc_in == pytest.approx(math.exp(1 - 1 / math.sqrt(1 + 1e-6)), rel=1e-8)
    phi_out, _ = orc_full.snapshots(p.r_cut)
    assert np.all(np.abs(phi_out) < 1e-300)


def test_snapshot_derivatives_fd(orc_full):
    h = 1e-6
    for r in np.linspace(1.05, 4.95, 17):
        phi_p, _ = orc_full.snapshots(r + h)
        phi_m, _ = orc_full.snapshots(r - h)
        _, dphi = orc_full.snapshots(r)
        fd = (phi_p - phi_m) / (2 * h)
        assert np.allclose(dphi, fd, rtol=1e-7, atol=1e-8 * np.max(np.abs(dphi)) + 1e-12)


@pytest.mark.parametrize("which", ["small", "full"])
def test_pod_basis_against_library_eigensolver(which):
    params = synth.params_small() if which == "small" else synth.params_full()
    o = oracle.Oracle(params)
    n = params.n_grid
    h = (params.r_cut - params.r_in) / n
    rg = params.r_in + (np.arange(n) + 0.5) * h
    Phi = np.array([o.snapshots(r)[0] for r in rg])  # (n, Ns)
    Cm = h * Phi.T @ Phi
    assert np.allclose(Cm, o.gram, rtol=1e-13, atol=1e-15 * np.abs(Cm).max())
    lam = np.sort(np.linalg.eigvalsh(Cm))[::-1]
    assert np.allclose(o.eig, lam, rtol=1e-9, atol=1e-14 * lam[0])
    # R_k orthonormal on the grid:  h R^T R = I
    R = Phi @ o.Q
    assert np.allclose(h * R.T @ R, np.eye(o.K), atol=1e-10)
    # eigen residual C v = lambda v for the kept modes
    V = o.Q * np.sqrt(o.eig[: o.K])[None, :]
    assert np.allclose(Cm @ V, V * o.eig[None, : o.K], atol=1e-11 * lam[0])
    # sign convention: largest-magnitude entry of each eigenvector is positive
    for k in range(o.K):
        assert V[np.argmax(np.abs(V[:, k])), k] > 0


def test_radial_derivative_fd(orc_full):
    r = np.linspace(1.1, 4.9, 11)
    h = 1e-6
    R, dR = orc_full.radial(r)
    Rp, _ = orc_full.radial(r + h)
    Rm, _ = orc_full.radial(r - h)
    assert np.allclose(dR, (Rp - Rm) / (2 * h), rtol=1e-6, atol=1e-7)


# ------------------------------------------------------------ neighbours

def test_bcc_neighbor_shells():
    o = oracle.Oracle(synth.params_small())
    cfg = synth.bcc(3)
    a = synth.A_BCC
    for i in [0, 1, 17, 53]:
        js, sh, d = o.neighbors(cfg, i)
        r = np.linalg.norm(d, axis=1)
        assert len(js) == 26
        assert np.sum(np.isclose(r, a * math.sqrt(3) / 2)) == 8
        assert np.sum(np.isclose(r, a)) == 6
        assert np.sum(np.isclose(r, a * math.sqrt(2))) == 12


def test_tiny_box_images_give_bulk_neighbors():
    o = oracle.Oracle(synth.params_small())
    cfg = synth.bcc(1)  # 2 atoms, box 3.316 A < r_cut: many images
    for i in range(2):
        js, sh, d = o.neighbors(cfg, i)
        assert len(js) == 26
        r = np.linalg.norm(d, axis=1)
        assert np.sum(np.isclose(r, synth.A_BCC * math.sqrt(2))) == 12
        assert np.sum(np.all(sh == 0, axis=1)) == 1  # only the other basis atom is in-cell


def test_neighbor_list_symmetric_and_sorted():
    o = oracle.Oracle(synth.params_small())
    cfg = synth.config_train(5)
    lists = o.neighbor_lists(cfg)
    pairs = set()
    for i, (js, sh, d) in enumerate(lists):
        keys = [(int(j), *map(int, s)) for j, s in zip(js, sh)]
        assert keys == sorted(keys)
        for j, s in zip(js, sh):
            pairs.add((i, int(j), *map(int, s)))
    for (i, j, sx, sy, sz) in pairs:
        assert (j, i, -sx, -sy, -sz) in pairs


def test_neighbor_count_against_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    o = oracle.Oracle(synth.params_small())
    cfg = synth.config_small()
    L = cfg.box
    wrapped = cfg.pos - L * np.floor(cfg.pos / L)
    tree = spatial.cKDTree(wrapped, boxsize=L)
    for i in range(0, cfg.n, 9):
        js, _, _ = o.neighbors(cfg, i)
        ref = [j for j in tree.query_ball_point(wrapped[i], 5.0) if j != i]
        assert sorted(ref) == sorted(js.tolist())


def _lists_equal(a, b):
    for (ja, sa, da), (jb, sb, db) in zip(a, b):
        assert np.array_equal(ja, jb)
        assert np.array_equal(sa, sb)
        assert np.array_equal(da, db)  # same FP64 expression: identical bits


def _band_config():
    """Pairs placed 1e-9 A inside, on, and outside r_cut along each axis."""
    rc = 5.0
    pos = [[10.0, 10.0, 10.0], [10.0 + rc - 1e-9, 10.0, 10.0], [10.0, 10.0 + rc, 10.0],
           [10.0, 10.0, 10.0 + rc + 1e-9], [10.0 - rc + 1e-12, 10.0, 10.0]]
    return synth.Config(pos=np.array(pos), box=np.array([30.0, 30.0, 30.0]), pbc=(1, 1, 1))


@pytest.mark.parametrize("which", ["small", "train", "cluster", "mixed_pbc", "band", "full_sample", "gas"])
def test_cell_list_equals_brute_force(which):
    """The cell-list neighbour pass gives the brute-force list entry for entry
    (indices, image shifts and displacement bits) on every kind of geometry:
    minimum-image boxes, training boxes shorter than r_cut (many images), open
    clusters, a box periodic in one direction only, pairs within 1e-9 A of r_cut,
    and atoms of the 8,192-atom system."""
    o = oracle.Oracle(synth.params_small())
    if which == "small":
        cfgs, atoms = [synth.config_small(0)], None
    elif which == "train":
        cfgs, atoms = [synth.config_train(k) for k in range(24)], None
    elif which == "cluster":
        cfgs, atoms = [synth.cluster(12, 7)], None
    elif which == "mixed_pbc":
        c = synth.config_train(3)
        cfgs, atoms = [synth.Config(pos=c.pos, box=c.box, pbc=(1, 0, 1))], None
    elif which == "band":
        cfgs, atoms = [_band_config()], None
    elif which == "gas":
        cfgs, atoms = [synth.liquid(300, synth.rng(9), density=300 / 60.0 ** 3)], None
    else:
        cfgs, atoms = [synth.config_full(0)], list(range(0, 8192, 97))
    for cfg in cfgs:
        brute = o.neighbor_lists(cfg, atoms, cells=False)
        cells = o.neighbor_lists(cfg, atoms, cells=True)
        _lists_equal(brute, cells)
    if which == "band":
        js, _, _ = o.neighbors(cfgs[0], 0, o._system(cfgs[0], cells=True))
        assert sorted(js.tolist()) == [1, 4]  # strictly inside r_cut only


@pytest.mark.parametrize("threads", [1, 3])
def test_cell_list_energy_forces_equal_brute_force(threads):
    """The threaded cell-list energy/force route equals the brute-force assembly
    of ``energy_forces`` (same per-atom arithmetic; forces and virial summed in
    another order)."""
    for p, cfg in [(synth.params_small(), synth.config_small(0)),
                   (synth.params_full(), synth.config_train(11))]:
        o = oracle.Oracle(p)
        c = synth.coefficients(o.M, 17)
        Ei0, E0, F0, W0 = o.energy_forces(cfg, c)
        Ei1, E1, F1, W1 = o.energy_forces_cells(cfg, c, threads=threads)
        assert np.array_equal(Ei0, Ei1)
        assert E0 == E1
        fmax = np.max(np.abs(F0))
        assert np.max(np.abs(F1 - F0)) <= 1e-13 * fmax
        assert np.max(np.abs(W1 - W0)) <= 1e-13 * np.max(np.abs(W0))


# ---------------------------------------------------- descriptor identities

def _cluster_disp(n, seed):
    cfg = synth.cluster(n + 1, seed)
    d = cfg.pos[1:] - cfg.pos[0]
    return d[np.linalg.norm(d, axis=1) < 5.0]


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 8, 11])
def test_fast_equals_naive_clusters(orc_full, n):
    d = _cluster_disp(n, 100 + n) if n else np.zeros((0, 3))
    Dn = orc_full.atom_descriptors(d, fast=False)
    Df = orc_full.atom_descriptors(d, fast=True)
    scale = np.maximum(np.abs(Dn), 1.0)
    assert np.all(np.abs(Dn - Df) <= 1e-13 * scale)
    if n == 0:
        assert Dn[0] == 1.0 and np.all(Dn[1:] == 0)


def test_fast_equals_naive_periodic(orc_small, orc_full):
    for o, cfg in [(orc_small, synth.config_small()), (orc_full, synth.config_train(3))]:
        lists = o.neighbor_lists(cfg, atoms=range(0, cfg.n, max(1, cfg.n // 6)))
        for js, sh, d in lists:
            Dn = o.atom_descriptors(d, fast=False)
            Df = o.atom_descriptors(d, fast=True)
            assert np.allclose(Dn, Df, rtol=1e-12, atol=1e-12 * np.abs(Dn).max())


def test_dimer_closed_form(orc_full):
    p = orc_full.params
    for r in [1.7, 2.9, 4.2]:
        u = synth.rng(3).normal(size=3)
        d = (r * u / np.linalg.norm(u))[None, :]
        D = orc_full.atom_descriptors(d)
        R, _ = orc_full.radial(np.array([r]))
        R = R[0]
        Ka = oracle.num_fourbody(p.P4)
        exp = [1.0] + list(R[: p.K2])
        for m in range(p.K3):
            exp += [R[m] ** 2] * (p.P3 + 1)      # w = 1 for j = k
        for m in range(p.K4):
            exp += [R[m] ** 3] * Ka              # all w = 1
        assert np.allclose(D, exp, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("theta", [0.7, math.pi / 3, 2.0])
def test_trimer_closed_form(orc_full, theta):
    p = orc_full.params
    r1, r2 = 2.6, 3.4
    d = np.array([[r1, 0, 0], [r2 * math.cos(theta), r2 * math.sin(theta), 0]])
    D = orc_full.atom_descriptors(d)
    R, _ = orc_full.radial(np.array([r1, r2]))
    w = math.cos(theta)
    col = 1 + p.K2
    for m in range(p.K3):
        for n in range(p.P3 + 1):
            exp = R[0, m] ** 2 + R[1, m] ** 2 + 2 * R[0, m] * R[1, m] * w ** n
            assert D[col] == pytest.approx(exp, rel=1e-13, abs=1e-15)
            col += 1
    # equal legs: D4 = 2 R^3 [f(1,1,1) + f(1,w,w) + f(w,1,w) + f(w,w,1)]
    d = np.array([[r1, 0, 0], [r1 * math.cos(theta), r1 * math.sin(theta), 0]])
    D = orc_full.atom_descriptors(d)
    R, _ = orc_full.radial(np.array([r1]))
    tab = oracle.fourbody_table(p.P4)
    col = 1 + p.K2 + p.K3 * (p.P3 + 1)
    for m in range(p.K4):
        for a, b, c in tab:
            f = lambda x, y, z: x ** a * y ** b * z ** c
            exp = 2 * R[0, m] ** 3 * (f(1, 1, 1) + f(1, w, w) + f(w, 1, w) + f(w, w, 1))
            assert D[col] == pytest.approx(exp, rel=1e-13, abs=1e-15)
            col += 1


def test_eq15c_inclusive_vs_exclusive(orc_full):
    for n, seed in [(4, 1), (9, 2)]:
        d = _cluster_disp(n, seed)
        D = orc_full.atom_descriptors(d)
        p = orc_full.params
        Dex = orc_full.atom_d3_exclusive(d)
        R, _ = orc_full.radial(np.linalg.norm(d, axis=1))
        D3 = D[1 + p.K2: 1 + p.K2 + p.K3 * (p.P3 + 1)].reshape(p.K3, p.P3 + 1)
        exp = 2 * Dex + np.sum(R[:, : p.K3] ** 2, axis=0)[:, None]
        assert np.allclose(D3, exp, rtol=1e-13, atol=1e-14)
        assert np.all(D3 >= -1e-15)


def test_eq27a_and_table2_sums(orc_full):
    p = orc_full.params
    tab = oracle.fourbody_table(p.P4)
    Ka = len(tab)
    for n, seed in [(5, 11), (10, 12)]:
        d = _cluster_disp(n, seed)
        D = orc_full.atom_descriptors(d)
        D2 = D[1: 1 + p.K2]
        D3 = D[1 + p.K2: 1 + p.K2 + p.K3 * (p.P3 + 1)].reshape(p.K3, p.P3 + 1)
        D4 = D[1 + p.K2 + p.K3 * (p.P3 + 1):].reshape(p.K4, Ka)
        for q, (a, b, c) in enumerate(tab):
            if b == 0 and c == 0:
                assert np.allclose(D4[:, q], D2[: p.K4] * D3[: p.K4, a], rtol=1e-13)
        G = orc_full.atom_g4_sums(d)
        assert np.allclose(G, 3 * D4, rtol=1e-12, atol=1e-13 * np.abs(D4).max())


# ------------------------------------------------------------ invariances

def test_invariance_cluster(orc_full):
    g = synth.rng(21)
    cfg = synth.cluster(9, 77)
    base = orc_full.descriptors(cfg)
    for trial in range(3):
        Qr = synth.random_rotation(g)
        if trial == 1:
            Qr = Qr @ np.diag([-1.0, 1.0, 1.0])  # reflection
        shift = g.normal(size=3)
        perm = g.permutation(cfg.n)
        c2 = synth.Config(pos=((cfg.pos - 10.0) @ Qr.T + 10.0 + shift)[perm], box=cfg.box, pbc=cfg.pbc)
        D = orc_full.descriptors(c2)
        assert np.allclose(D, base[perm], rtol=1e-12, atol=1e-12 * np.abs(base).max())


def test_invariance_periodic(orc_small):
    cfg = synth.config_small()
    base = orc_small.descriptors(cfg, atoms=range(0, cfg.n, 16))
    L = cfg.box[0]
    # 90 degree rotation about z: (x, y, z) -> (-y, x, z) + translate into the cell
    pos = np.stack([-cfg.pos[:, 1] + L, cfg.pos[:, 0], cfg.pos[:, 2]], axis=1) + 0.37
    D = orc_small.descriptors(synth.Config(pos=pos, box=cfg.box), atoms=range(0, cfg.n, 16))
    assert np.allclose(D, base, rtol=1e-12, atol=1e-12 * np.abs(base).max())
    pos = cfg.pos * np.array([1.0, -1.0, 1.0])  # reflection y -> -y
    D = orc_small.descriptors(synth.Config(pos=pos, box=cfg.box), atoms=range(0, cfg.n, 16))
    assert np.allclose(D, base, rtol=1e-12, atol=1e-12 * np.abs(base).max())


# --------------------------------------------------- derivatives and forces

@pytest.mark.parametrize("n", [1, 4, 9])
def test_dD_naive_equals_fast_and_fd(orc_full, n):
    d = _cluster_disp(n, 300 + n)
    dn = orc_full.atom_dD(d, fast=False)
    df = orc_full.atom_dD(d, fast=True)
    assert np.allclose(dn, df, rtol=1e-11, atol=1e-12 * np.abs(dn).max())
    h = 1e-5
    for j in range(len(d)):
        for t in range(3):
            dp = d.copy()
            dm = d.copy()
            dp[j, t] += h
            dm[j, t] -= h
            fd = (orc_full.atom_descriptors(dp) - orc_full.atom_descriptors(dm)) / (2 * h)
            assert np.allclose(dn[j, :, t], fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fd).max()))


def test_energy_adjoint_equals_explicit(orc_full):
    c = synth.coefficients(orc_full.M, 5)
    d = _cluster_disp(10, 9)
    E, g = orc_full.atom_energy_grad(d, c)
    D = orc_full.atom_descriptors(d)
    dD = orc_full.atom_dD(d)
    assert E == pytest.approx(D @ c, rel=1e-13)
    assert np.allclose(g, np.einsum("jmt,m->jt", dD, c), rtol=1e-11, atol=1e-13)


def _energy(o, cfg, c):
    Ei = [o.atom_energy_grad(d, c)[0] for _, _, d in o.neighbor_lists(cfg)]
    return math.fsum(Ei)


def test_forces_are_minus_energy_gradient():
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(4))  # 16 atoms, multi-image
    c = synth.coefficients(o.M, 8)
    _, E, F, W = o.energy_forces(cfg, c, fast=True)
    _, E2, F2, W2 = o.energy_forces(cfg, c, fast=False)
    assert E == pytest.approx(E2, rel=1e-12)
    assert np.allclose(F, F2, atol=1e-10)
    assert np.allclose(W, W2, atol=1e-10)
    h = 1e-5
    for k in [0, 5, 11]:
        for t in range(3):
            cp = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cm = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cp.pos[k, t] += h
            cm.pos[k, t] -= h
            fd = -(_energy(o, cp, c) - _energy(o, cm, c)) / (2 * h)
            assert F[k, t] == pytest.approx(fd, abs=1e-7)
    assert np.allclose(F.sum(0), 0.0, atol=1e-10)  # translation invariance


def test_virial_strain_derivative():
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(6))
    c = synth.coefficients(o.M, 9)
    _, _, _, W = o.energy_forces(cfg, c, fast=True)
    assert np.allclose(W, W.T, atol=1e-9)  # rotational invariance
    h = 1e-6
    for a, b in [(0, 0), (1, 2), (2, 1), (0, 1)]:
        def e_at(eps):
            S = np.eye(3)
            S[a, b] += eps
            # x -> (I + eps) x ; orthorhombic boxes stay orthorhombic only for diagonal strain,
            # so off-diagonal strain is applied to the displacements of a cluster-free copy
            return S
        if a == b:
            Sp, Sm = e_at(h), e_at(-h)
            cp = synth.Config(pos=cfg.pos @ Sp.T, box=cfg.box * np.diag(Sp))
            cm = synth.Config(pos=cfg.pos @ Sm.T, box=cfg.box * np.diag(Sm))
            fd = -(_energy(o, cp, c) - _energy(o, cm, c)) / (2 * h)
            assert W[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        else:
            # off-diagonal: use the per-pair displacement form directly
            tot_p = tot_m = 0.0
            Sp, Sm = e_at(h), e_at(-h)
            Ep, Em = [], []
            for _, _, d in o.neighbor_lists(cfg):
                Ep.append(o.atom_energy_grad(d @ Sp.T, c)[0])
                Em.append(o.atom_energy_grad(d @ Sm.T, c)[0])
            fd = -(math.fsum(Ep) - math.fsum(Em)) / (2 * h)
            assert W[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-8)


# -------------------------------------------------------------------- fit

def test_fit_recovers_teacher():
    params = synth.params_small()
    o = oracle.Oracle(params)
    g = synth.rng(31)
    cstar = synth.coefficients(o.M, 12)
    cfgs = []
    for k in range(12):
        base = synth.bcc(1) if k % 3 == 0 else synth.lattice(synth.FCC_BASIS, synth.A_FCC, 1, 1, 1)
        base = synth.strain_iso(base, g.uniform(-0.06, 0.06))
        cfgs.append(synth.jitter(base, 0.15, g))
    E_ref, F_ref = [], []
    for cfg in cfgs:
        _, E, F, _ = o.energy_forces(cfg, cstar, fast=True)
        E_ref.append(E)
        F_ref.append(F)
    c, A, b = o.fit(cfgs, E_ref, F_ref)
    assert np.linalg.norm(A @ cstar - b) <= 1e-10 * np.linalg.norm(b)
    assert np.allclose(c, cstar, rtol=1e-6, atol=1e-8)


# ----------------------------------------------------------- quadratic model

def _quad_beta(M, seed, scale=1e-5):
    b = synth.rng(seed).normal(0.0, scale, size=(M, M))
    return b


def test_quadratic_model_reduces_to_linear():
    """beta = 0: the quadratic model of Sec. 4 is the linear model (Eq. 57a)."""
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(71))
    c = synth.coefficients(o.M, 72)
    Ei, E, F, W = o.energy_forces(cfg, c, fast=True)
    Eq_i, Eq, Fq, Wq = o.energy_forces_quadratic(cfg, c, np.zeros((o.M, o.M)))
    assert np.allclose(Eq_i, Ei, rtol=1e-13, atol=1e-15)
    assert np.allclose(Fq, F, atol=1e-12) and np.allclose(Wq, W, atol=1e-12)


def test_quadratic_model_energy_and_forces():
    """Energy = c.D + D^T beta_upper D per atom (only the upper triangle of beta
    counts), forces = minus central differences of that energy, virial
    symmetric, net force zero."""
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(73))
    c = synth.coefficients(o.M, 74)
    beta = _quad_beta(o.M, 75)
    Ei, E, F, W = o.energy_forces_quadratic(cfg, c, beta)
    # the lower triangle is ignored
    Ei2, _, F2, _ = o.energy_forces_quadratic(cfg, c, np.triu(beta) + 7.0 * np.tril(np.ones_like(beta), -1))
    assert np.array_equal(Ei, Ei2) and np.array_equal(F, F2)

    def energy(cf):
        D = o.descriptors(cf, fast=False)  # naive sums, independent of the fast path
        return float(np.sum(D @ c) + sum(Di @ np.triu(beta) @ Di for Di in D))

    assert E == pytest.approx(energy(cfg), rel=1e-11)
    h = 1e-5
    for k in [0, 9]:
        for t in range(3):
            cp = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cm = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cp.pos[k, t] += h
            cm.pos[k, t] -= h
            fd = -(energy(cp) - energy(cm)) / (2 * h)
            assert F[k, t] == pytest.approx(fd, rel=1e-7, abs=1e-7)
    fs = np.max(np.abs(F))
    assert np.allclose(F.sum(0), 0.0, atol=1e-12 * max(fs, 1.0) * cfg.n)
    assert np.allclose(W, W.T, atol=1e-10 * max(np.max(np.abs(W)), 1.0))


# ----------------------------------------------------------- embedding model

def _emb_weights(o, seed):
    """Density weights on the two- and three-body columns (a MEAM-type density)
    and a cubic embedding polynomial."""
    g = synth.rng(seed)
    a = np.zeros(o.M)
    p = o.params
    col3 = 1 + p.K2
    a[1:col3 + p.K3 * (p.P3 + 1)] = g.normal(0.0, 1e-2, size=col3 + p.K3 * (p.P3 + 1) - 1)
    alpha = np.array([0.3, -0.2, 5e-3, -1e-4])
    return a, alpha


def test_embedding_model_reduces_to_linear():
    """alpha = 0: the embedding model of Sec. 3 is the linear model (Eq. 57a);
    alpha = (alpha_0, alpha_1): the linear model with c + alpha_1 a, plus alpha_0
    per atom."""
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(81))
    c = synth.coefficients(o.M, 82)
    a, _ = _emb_weights(o, 83)
    Ei, E, F, W = o.energy_forces(cfg, c, fast=True)
    Ee_i, _, Fe, We = o.energy_forces_embedding(cfg, c, a, np.zeros(3))
    assert np.allclose(Ee_i, Ei, rtol=1e-13, atol=1e-15)
    assert np.allclose(Fe, F, atol=1e-12) and np.allclose(We, W, atol=1e-12)
    Ei1, _, F1, W1 = o.energy_forces(cfg, c + 0.7 * a, fast=True)
    El_i, _, Fl, Wl = o.energy_forces_embedding(cfg, c, a, np.array([0.25, 0.7]))
    assert np.allclose(El_i, Ei1 + 0.25, rtol=1e-12, atol=1e-13)
    assert np.allclose(Fl, F1, atol=1e-12) and np.allclose(Wl, W1, atol=1e-12)


def test_embedding_degree_two_is_quadratic_model():
    """F(rho) = alpha_0 + alpha_1 rho + alpha_2 rho^2 with rho = a.D is the
    quadratic model (Sec. 4) with c + alpha_1 a + alpha_0 e_0 and beta = alpha_2 a a^T
    (upper triangle: a_m^2 on the diagonal, 2 a_m a_n above it) -- the paper's
    remark that polynomial embeddings are sums of products of descriptors."""
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(84))
    c = synth.coefficients(o.M, 85)
    a, _ = _emb_weights(o, 86)
    alpha = np.array([0.1, -0.3, 2e-2])
    Ee_i, Ee, Fe, We = o.energy_forces_embedding(cfg, c, a, alpha)
    beta = alpha[2] * (2.0 * np.triu(np.outer(a, a), 1) + np.diag(a * a))
    cq = c + alpha[1] * a
    cq[0] += alpha[0]
    Eq_i, Eq, Fq, Wq = o.energy_forces_quadratic(cfg, cq, beta)
    assert np.allclose(Ee_i, Eq_i, rtol=1e-12, atol=1e-13)
    assert np.allclose(Fe, Fq, rtol=1e-10, atol=1e-12) and np.allclose(We, Wq, rtol=1e-10, atol=1e-12)


def test_embedding_model_energy_and_forces():
    """Cubic embedding of a MEAM-type density: energy = c.D + F(a.D) from the
    naive descriptor sums, forces = minus central differences of that energy,
    net force zero, virial symmetric."""
    o = oracle.Oracle(synth.params_full())
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(87))
    c = synth.coefficients(o.M, 88)
    a, alpha = _emb_weights(o, 89)
    Ei, E, F, W = o.energy_forces_embedding(cfg, c, a, alpha)

    def energy(cf):
        D = o.descriptors(cf, fast=False)  # naive sums, independent of the fast path
        rho = D @ a
        return float(np.sum(D @ c) + np.sum(np.polyval(alpha[::-1], rho)))

    assert E == pytest.approx(energy(cfg), rel=1e-11)
    h = 1e-5
    for k in [0, 11]:
        for t in range(3):
            cp = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cm = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cp.pos[k, t] += h
            cm.pos[k, t] -= h
            fd = -(energy(cp) - energy(cm)) / (2 * h)
            assert F[k, t] == pytest.approx(fd, rel=1e-7, abs=1e-7)
    fs = np.max(np.abs(F))
    assert np.allclose(F.sum(0), 0.0, atol=1e-12 * max(fs, 1.0) * cfg.n)
    assert np.allclose(W, W.T, atol=1e-10 * max(np.max(np.abs(W)), 1.0))


# ------------------------------------------- exclusive three-body set (Eq. 15b)

def test_exclusive3_descriptors_are_the_pair_sums():
    """The exclusive three-body columns formed from the inclusive ones (Eq. 15c)
    equal the plain sums over pairs k > j of Eq. 15b written out in C; the two-,
    four-body and one-body columns are the inclusive ones."""
    o = oracle.Oracle(synth.params_full())
    p = o.params
    col3, n3 = 1 + p.K2, p.P3 + 1
    g = synth.rng(101)
    for n in (1, 2, 7, 19):
        d = g.normal(0.0, 1.0, size=(n, 3))
        d *= g.uniform(1.5, 4.8, size=n)[:, None] / np.linalg.norm(d, axis=1)[:, None]
        Dx = o.exclusive3_descriptors(d, fast=False)
        Dn = o.atom_descriptors(d, fast=False)
        ex = o.atom_d3_exclusive(d)
        assert np.allclose(Dx[col3:col3 + p.K3 * n3].reshape(p.K3, n3), ex, rtol=1e-12, atol=1e-13)
        assert np.array_equal(Dx[:col3], Dn[:col3]) and np.array_equal(Dx[col3 + p.K3 * n3:], Dn[col3 + p.K3 * n3:])


def test_exclusive3_energy_and_forces():
    """Linear model on the exclusive set: energy from the naive pair sums of
    Eq. 15b, forces = minus central differences of that energy, net force zero,
    virial symmetric."""
    o = oracle.Oracle(synth.params_full())
    p = o.params
    col3, n3 = 1 + p.K2, p.P3 + 1
    cfg = synth.jitter(synth.bcc(2), 0.1, synth.rng(102))
    c = synth.coefficients(o.M, 103)
    Ei, E, F, W = o.energy_forces_exclusive3(cfg, c)

    def energy(cf):
        sysd = o._system(cf)
        tot = 0.0
        for i in range(cf.n):
            _, _, d = o.neighbors(cf, i, sysd)
            D = np.array(o.atom_descriptors(d, fast=False))
            D[col3:col3 + p.K3 * n3] = o.atom_d3_exclusive(d).ravel()
            tot += float(D @ c)
        return tot

    assert E == pytest.approx(energy(cfg), rel=1e-11)
    h = 1e-5
    for k in [0, 13]:
        for t in range(3):
            cp = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cm = synth.Config(pos=cfg.pos.copy(), box=cfg.box)
            cp.pos[k, t] += h
            cm.pos[k, t] -= h
            fd = -(energy(cp) - energy(cm)) / (2 * h)
            assert F[k, t] == pytest.approx(fd, rel=1e-7, abs=1e-7)
    fs = np.max(np.abs(F))
    assert np.allclose(F.sum(0), 0.0, atol=1e-12 * max(fs, 1.0) * cfg.n)
    assert np.allclose(W, W.T, atol=1e-10 * max(np.max(np.abs(W)), 1.0))
