"""Batches of configurations and the ridge least-squares fit (Eq. 63a) on the GPU,
compared with the FP64 oracle (its own design matrix, solved with numpy's SVD
least squares).

Tolerances: per-configuration descriptors, energies and forces as in
test_gpu_parity.py; fitted coefficients: the GPU solves the normal equations
(condition number squared) while the oracle uses SVD, so c is compared through
the fitted energies and forces (relative 1e-8 of their scale) and directly with
a tolerance scaled by the conditioning; noise-free labels from a teacher c*
must give training errors at rounding level.
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


def training_configs(n, replica=0, max_atoms=40):
    out = []
    k = 0
    while len(out) < n:
        cfg = synth.config_train(k, replica)
        k += 1
        if cfg.n <= max_atoms:
            out.append(cfg)
    return out


def desc_err(D, Dref):
    den = np.max(np.abs(Dref), axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.max(np.abs(D - Dref), axis=0) / den))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_batch_descriptors(pkg, prec, tol):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = training_configs(10)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    D = pod.descriptors_batch(cfgs).cpu().numpy()
    Dref = np.concatenate([o.descriptors(c, fast=True) for c in cfgs], axis=0)
    assert desc_err(D, Dref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_energy_forces(pkg, prec):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = training_configs(8, replica=1)
    c = synth.coefficients(o.M, 77)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    out = pod.energy_forces_batch(cfgs, torch.tensor(c))
    E = out["E"].cpu().numpy()
    F = out["F"].cpu().numpy()
    offs = out["offs"]
    for k, cfg in enumerate(cfgs):
        _, Eo, Fo, _ = o.energy_forces(cfg, c, fast=True)
        scale = float(np.sum(np.abs(o.descriptors(cfg, fast=True) * c)))
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert abs(E[k] - Eo) <= tol * scale
        Fk = F[offs[k]:offs[k + 1]]
        if prec == "fp64":
            assert np.max(np.abs(Fk - Fo)) <= 1e-10 * max(1.0, np.max(np.abs(Fo)))
        else:
            assert np.max(np.abs(Fk - Fo)) <= 1e-4


def _labels(o, cfgs, c, noise=0.0, seed=0):
    g = synth.rng(seed)
    E_ref, F_ref = [], []
    for cfg in cfgs:
        _, E, F, _ = o.energy_forces(cfg, c, fast=True)
        E_ref.append(E + noise * 1e-3 * cfg.n * g.normal())
        F_ref.append(F + noise * 5e-2 * g.normal(size=F.shape))
    return np.array(E_ref), F_ref


def test_fit_recovers_teacher(pkg):
    p = synth.params_small()
    o = oracle.Oracle(p)
    cfgs = training_configs(16, replica=2)
    cstar = synth.coefficients(o.M, 12)
    E_ref, F_ref = _labels(o, cfgs, cstar)
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    c, maeE, maeF = pod.fit(cfgs, E_ref, F_ref)
    A, b = o.design_matrix(cfgs, E_ref, F_ref)
    # fitted values agree with the teacher's to rounding level
    assert np.max(np.abs(A @ c - b)) <= 1e-8 * np.max(np.abs(b))
    assert maeE <= 1e-9 and maeF <= 1e-8
    assert np.allclose(c, cstar, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fit_matches_oracle_with_noise(pkg, prec):
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = training_configs(24, replica=3, max_atoms=30)
    cstar = synth.coefficients(o.M, 13)
    E_ref, F_ref = _labels(o, cfgs, cstar, noise=1.0, seed=5)
    c_o, A, b = o.fit(cfgs, E_ref, F_ref)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    c, maeE, maeF = pod.fit(cfgs, E_ref, F_ref)
    # same fitted energies and forces (the predictions are what the fit fixes)
    pred, pred_o = A @ c, A @ c_o
    tol = 1e-7 if prec == "fp64" else 1e-3
    assert np.max(np.abs(pred - pred_o)) <= tol * np.max(np.abs(b))
    # training errors as the oracle computes them (its rows: per configuration
    # one energy row followed by 3 N_c force rows)
    e_rows, r = [], 0
    for cfg in cfgs:
        e_rows.append(r)
        r += 1 + 3 * cfg.n
    is_e = np.zeros(len(b), dtype=bool)
    is_e[e_rows] = True
    res = np.abs(pred_o - b)
    maeE_o = res[is_e].mean() / 100.0
    maeF_o = res[~is_e].mean()
    assert maeE == pytest.approx(maeE_o, rel=1e-3 if prec == "fp64" else 5e-2)
    assert maeF == pytest.approx(maeF_o, rel=1e-3 if prec == "fp64" else 5e-2)


def test_fit_singular_reports_error(pkg):
    """gamma = 0 with a single one-atom configuration: the normal equations are
    singular (only the one-body column is non-zero) and the call says so."""
    p = synth.params_small()
    pod = pkg.POD(p, precision="fp64")
    one = synth.Config(pos=np.array([[1.0, 1.0, 1.0]]), box=np.array([20.0, 20.0, 20.0]), pbc=(0, 0, 0))
    with pytest.raises(pkg.PodError) as ei:
        pod.fit([one], np.array([0.5]), [np.zeros((1, 3))], gamma=0.0)
    assert ei.value.code == pkg.POD_ESINGULAR


def test_batch_with_too_many_image_candidates_is_refused(pkg):
    """The batch neighbour search indexes an atom's (image, atom) candidates with
    32-bit integers; a configuration whose count can exceed that (1,300 atoms in a
    periodic box of 0.084 A: 121^3 images each) is refused while the batch is
    planned, before any kernel runs."""
    p = synth.params_full()
    pod = pkg.POD(p, precision="mixed")
    g = synth.rng(41)
    L = np.array([0.084, 0.084, 0.084])
    tiny = synth.Config(pos=g.uniform(0.0, 0.084, size=(1300, 3)), box=L, pbc=(1, 1, 1))
    ok = synth.config_train(0)
    with pytest.raises(pkg.PodError) as ei:
        pod.descriptors_batch([ok, tiny])
    assert ei.value.code == pkg.POD_EINVAL
    assert "candidates" in str(ei.value)
    D = pod.descriptors_batch([ok])  # the handle stays usable
    assert torch.isfinite(D).all()


def test_fit_stages_equal_single_call(pkg):
    """pod_fit_normal + pod_fit_solve + pod_fit_residual (the sharded-fit
    building blocks) reproduce pod_fit bit for bit on one GPU."""
    p = synth.params_small()
    o = oracle.Oracle(p)
    cfgs = training_configs(12, replica=4)
    cstar = synth.coefficients(o.M, 21)
    E_ref, F_ref = _labels(o, cfgs, cstar, noise=1.0, seed=8)
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    c, maeE, maeF = pod.fit(cfgs, E_ref, F_ref)
    G, r = pod.fit_normal(cfgs, E_ref, F_ref)
    assert np.allclose(G, G.T, rtol=0, atol=0)
    c2 = pod.fit_solve(G, r)
    se, sf, ne, nf = pod.fit_residual(c2)
    assert np.array_equal(c, c2)
    assert ne == len(cfgs) and nf == 3 * sum(cf.n for cf in cfgs)
    assert se / ne == pytest.approx(maeE, rel=1e-14) and sf / nf == pytest.approx(maeF, rel=1e-14)


def test_shards_one_after_another_equal_the_whole_fit(pkg):
    """The sharded fit (one configuration share per GPU, normal equations summed
    by an all-reduce) run as three shards one after another on this GPU: the
    summed G and r equal the unsharded ones to rounding, and the coefficients
    solved from them equal the one-call fit's."""
    from paper_2212_14446_gb300.parallel import shard_indices
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = training_configs(15, replica=6, max_atoms=30)
    cstar = synth.coefficients(o.M, 31)
    E_ref, F_ref = _labels(o, cfgs, cstar, noise=1.0, seed=9)
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    G_all, r_all = pod.fit_normal(cfgs, E_ref, F_ref)
    c_all, _, _ = pod.fit(cfgs, E_ref, F_ref)
    G = np.zeros_like(G_all)
    r = np.zeros_like(r_all)
    for rank in range(3):
        idx = shard_indices(len(cfgs), rank, 3)
        Gs, rs = pod.fit_normal([cfgs[i] for i in idx], E_ref[idx], [F_ref[i] for i in idx],
                                gamma=1e-12 if rank == 0 else 0.0)
        G += Gs
        r += rs
    scale = np.max(np.abs(G_all))
    assert np.max(np.abs(G - G_all)) <= 1e-12 * scale
    assert np.max(np.abs(r - r_all)) <= 1e-12 * np.max(np.abs(r_all))
    c = pod.fit_solve(G, r)
    A, b = o.design_matrix(cfgs, E_ref, F_ref)
    assert np.max(np.abs(A @ c - A @ c_all)) <= 1e-8 * np.max(np.abs(b))


@pytest.mark.parametrize("prec,ncfg,max_atoms", [("fp64", 15, 30), ("mixed", 15, 30), ("mixed", 150, 80)])
def test_tensor_core_gram_equals_fp64_syrk(pkg, prec, ncfg, max_atoms):
    """The normal-equation matrix from exact 8-bit slice products on the tensor
    cores -- tcgen05 (POD_OPT_GRAM = 0) and mma.sync (POD_OPT_GRAM = 2) -- equals
    the FP64 SYRK (POD_OPT_GRAM = 1) on the same design matrix to the SYRK's own
    rounding, is exactly symmetric, and gives the same fit; the two exact forms
    agree bit for bit (the same integer sums).  The larger case spans many
    256-row chunks and several row splits per slice pair."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = training_configs(ncfg, replica=7, max_atoms=max_atoms)
    cstar = synth.coefficients(o.M, 41)
    E_ref, F_ref = _labels(o, cfgs, cstar, noise=1.0, seed=12)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    pkg.pod_set_option(pod.h, pkg.POD_OPT_GRAM, 1)
    G64, r64 = pod.fit_normal(cfgs, E_ref, F_ref)
    c64, _, _ = pod.fit(cfgs, E_ref, F_ref)
    pkg.pod_set_option(pod.h, pkg.POD_OPT_GRAM, 2)
    Gmma, rmma = pod.fit_normal(cfgs, E_ref, F_ref)
    pkg.pod_set_option(pod.h, pkg.POD_OPT_GRAM, 0)
    with pytest.raises(pkg.PodError) as ei:  # only 0, 1 and 2 exist
        pkg.pod_set_option(pod.h, pkg.POD_OPT_GRAM, 3)
    assert ei.value.code == pkg.POD_EINVAL
    Gtc, rtc = pod.fit_normal(cfgs, E_ref, F_ref)
    ctc, _, _ = pod.fit(cfgs, E_ref, F_ref)
    assert np.array_equal(Gtc, Gmma)
    assert np.array_equal(Gtc, Gtc.T)
    d = np.sqrt(np.outer(np.diag(G64), np.diag(G64)))  # Cauchy-Schwarz scale of each entry
    assert np.max(np.abs(Gtc - G64) / d) <= 1e-13
    assert np.max(np.abs(rtc - r64)) <= 1e-13 * np.max(np.abs(r64))
    if ncfg <= 15:  # the oracle's design matrix (slow at the larger size)
        A, b = o.design_matrix(cfgs, E_ref, F_ref)
        assert np.max(np.abs(A @ ctc - A @ c64)) <= 1e-8 * np.max(np.abs(b))
    else:
        d = ctc - c64  # ||A d|| through the normal equations, against ||A c64||
        assert np.sqrt(abs(d @ G64 @ d)) <= 1e-8 * np.sqrt(c64 @ G64 @ c64)


def _dimer_set(n, seed):
    """Open dimers at random lengths and orientations: every three-body column of
    a mode equals every other of that mode (R_m^2) and every four-body column R_m^3,
    so A has rank 19 of 103 and A^T A + gamma I is positive definite only by
    gamma = 1e-12, far below the rounding of its entries."""
    g = synth.rng(seed)
    cfgs = []
    for _ in range(n):
        r = g.uniform(2.2, 4.8)
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0] + r * u])
        cfgs.append(synth.Config(pos=pos, box=np.array([30.0, 30.0, 30.0]), pbc=(0, 0, 0)))
    return cfgs


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_qr_fallback_on_singular_normal_equations(pkg, prec):
    """Cholesky of the normal equations fails (POD_ESINGULAR) on a rank-deficient
    design matrix with the paper's gamma = 1e-12; the QR solve of [A; sqrt(gamma) I]
    (the default fallback, or selected) matches the oracle's SVD least squares of
    the same augmented system through the fitted values A c."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = _dimer_set(40, 11)
    cstar = synth.coefficients(o.M, 14)
    E_ref, F_ref = _labels(o, cfgs, cstar, noise=1.0, seed=15)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    with pytest.raises(pkg.PodError) as ei:
        pod.fit(cfgs, E_ref, F_ref, solver="cholesky")
    assert ei.value.code == pkg.POD_ESINGULAR
    c_auto, maeE, maeF = pod.fit(cfgs, E_ref, F_ref)
    c_qr, _, _ = pod.fit(cfgs, E_ref, F_ref, solver="qr")
    assert np.array_equal(c_auto, c_qr)
    assert np.all(np.isfinite(c_qr))
    if prec == "mixed":
        # FP32 rounding breaks the exact collinearity of the mixed design matrix's
        # columns, so its regularised solution is not the FP64 one's; the solve path
        # is what is checked here
        return
    c_o, A, b = o.fit(cfgs, E_ref, F_ref)
    assert np.max(np.abs(A @ c_qr - A @ c_o)) <= 1e-8 * np.max(np.abs(b))
    res = np.abs(A @ c_o - b)
    assert maeF == pytest.approx(res[np.arange(len(b)) % 7 != 0].mean(), rel=1e-3)


@pytest.mark.parametrize("ncfg,max_atoms", [(12, 30), (150, 80)])
def test_qr_solve_equals_cholesky_when_well_posed(pkg, ncfg, max_atoms):
    """On well-conditioned training sets the QR solve (row blocks, merge levels,
    final block) and the Cholesky solve give the same fitted values; the larger
    set spans hundreds of row blocks and two merge levels."""
    p = synth.params_full()
    o = oracle.Oracle(p)
    cfgs = training_configs(ncfg, replica=9, max_atoms=max_atoms)
    cstar = synth.coefficients(o.M, 51)
    if ncfg <= 12:
        E_ref, F_ref = _labels(o, cfgs, cstar, noise=1.0, seed=16)
    else:
        pod64 = pkg.POD(p, precision="fp64", Q=o.Q)
        out = pod64.energy_forces_batch(cfgs, torch.tensor(cstar))
        E_ref = out["E"].cpu().numpy() + 1e-3 * synth.rng(17).normal(size=len(cfgs))
        Fall = out["F"].cpu().numpy()
        offs = out["offs"]
        F_ref = [Fall[offs[k]:offs[k + 1]] for k in range(len(cfgs))]
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    c_ch, mE_ch, mF_ch = pod.fit(cfgs, E_ref, F_ref, solver="cholesky")
    c_qr, mE_qr, mF_qr = pod.fit(cfgs, E_ref, F_ref, solver="qr")
    G, _ = pod.fit_normal(cfgs, E_ref, F_ref)
    d = c_qr - c_ch
    assert np.sqrt(abs(d @ G @ d)) <= 1e-8 * np.sqrt(c_ch @ G @ c_ch)
    assert mF_qr == pytest.approx(mF_ch, rel=1e-6)
    if ncfg <= 12:
        c_o, A, b = o.fit(cfgs, E_ref, F_ref)
        assert np.max(np.abs(A @ c_qr - A @ c_o)) <= 1e-8 * np.max(np.abs(b))
