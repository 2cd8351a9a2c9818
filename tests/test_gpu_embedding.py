"""Embedding model (Sec. 3: EAM and MEAM written with POD descriptors,
E_i = c.D_i + F(a.D_i) with a polynomial F) on the GPU against the FP64 oracle.
Tolerances as for the linear model: FP64 energy <= 1e-12 of sum_i |E_i|, forces
<= 1e-10 max|F|; mixed energy <= 1e-5 relative, forces <= 1e-4 of max|F|."""
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


def _weights(p, M, seed, three_body=True):
    """Density weights on the two-body columns (EAM-type) or on the two- and
    three-body columns (MEAM-type), and a cubic embedding polynomial."""
    g = synth.rng(seed)
    a = np.zeros(M)
    n = 1 + p.K2 + (p.K3 * (p.P3 + 1) if three_body else 0)
    a[1:n] = g.normal(0.0, 1e-2, size=n - 1)
    return a, np.array([0.3, -0.2, 5e-3, -1e-4])


def _dev(cfg):
    return torch.tensor(cfg.pos.T.copy(), device="cuda")


@pytest.mark.parametrize("which", ["full", "small"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("meam", [False, True])
def test_embedding_energy_forces(pkg, which, prec, meam):
    p = synth.params_full() if which == "full" else synth.params_small()
    o = oracle.Oracle(p)
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(91))
    c = synth.coefficients(o.M, 92)
    a, alpha = _weights(p, o.M, 93, three_body=meam)
    Ei_o, E_o, F_o, W_o = o.energy_forces_embedding(cfg, c, a, alpha)
    pod = pkg.POD(p, precision=prec, Q=o.Q)
    pod.set_embedding(a, alpha)
    out = pod.energy_forces(_dev(cfg), cfg.box, torch.tensor(c, device="cuda"))
    E = out["E"].item()
    F = out["F"].cpu().numpy()
    W = out["W"].cpu().numpy()
    Ei = out["Ei"].cpu().numpy()
    escale = float(np.sum(np.abs(Ei_o)))
    fmax = float(np.max(np.abs(F_o)))
    if prec == "fp64":
        assert abs(E - E_o) <= 1e-12 * escale
        assert np.max(np.abs(Ei - Ei_o)) <= 1e-12 * escale
        assert np.max(np.abs(F - F_o)) <= 1e-10 * fmax
        assert np.max(np.abs(W - W_o)) <= 1e-10 * max(np.max(np.abs(W_o)), escale)
    else:
        assert abs(E - E_o) <= 1e-5 * escale
        assert np.max(np.abs(F - F_o)) <= 1e-4 * max(fmax, 1.0)
        assert np.max(np.abs(W - W_o)) <= 1e-5 * max(np.max(np.abs(W_o)), escale)
    # back to the linear model
    pod.set_embedding(None)
    lin = pod.energy_forces(_dev(cfg), cfg.box, torch.tensor(c, device="cuda"))
    _, E_l, _, _ = o.energy_forces(cfg, c, fast=True)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(lin["E"].item() - E_l) <= tol * float(np.sum(np.abs(o.descriptors(cfg, fast=True) * c)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_embedding_degree_two_matches_quadratic(pkg, prec):
    """F(rho) = alpha_0 + alpha_1 rho + alpha_2 rho^2 on the GPU equals the GPU
    quadratic model with c + alpha_1 a + alpha_0 e_0 and beta = alpha_2 a a^T
    (two kernels, two arithmetic orders: within the path's tolerance)."""
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(4), 0.1, synth.rng(94))
    pod = pkg.POD(p, precision=prec)
    c = synth.coefficients(pod.M, 95)
    a, _ = _weights(p, pod.M, 96)
    alpha = np.array([0.1, -0.3, 2e-2])
    x = _dev(cfg)
    pod.set_embedding(a, alpha)
    e = pod.energy_forces(x, cfg.box, torch.tensor(c, device="cuda"))
    beta = alpha[2] * (2.0 * np.triu(np.outer(a, a), 1) + np.diag(a * a))
    cq = c + alpha[1] * a
    cq[0] += alpha[0]
    pod.set_quadratic(beta)
    q = pod.energy_forces(x, cfg.box, torch.tensor(cq, device="cuda"))
    tol_e, tol_f = (1e-12, 1e-10) if prec == "fp64" else (1e-5, 1e-4)
    escale = float(np.sum(np.abs(q["Ei"].cpu().numpy())))
    assert abs(e["E"].item() - q["E"].item()) <= tol_e * escale
    fq = q["F"].cpu().numpy()
    assert np.max(np.abs(e["F"].cpu().numpy() - fq)) <= tol_f * max(float(np.max(np.abs(fq))), 1.0)


def test_embedding_host_entry_and_errors(pkg):
    """The host-buffer entry evaluates the embedding model too, and bad
    embeddings are refused."""
    p = synth.params_full()
    cfg = synth.jitter(synth.bcc(3), 0.1, synth.rng(97))
    pod = pkg.POD(p, precision="mixed")
    c = synth.coefficients(pod.M, 98)
    a, alpha = _weights(p, pod.M, 99)
    pod.set_embedding(a, alpha)
    dev = pod.energy_forces(_dev(cfg), cfg.box, torch.tensor(c, device="cuda"))
    pos = torch.tensor(np.ascontiguousarray(cfg.pos.T)).pin_memory().numpy()
    for _ in range(2):
        host = pod.energy_forces_host(pos, cfg.box, c)
        assert host["E"][0] == dev["E"].item()
        assert np.array_equal(host["F"], dev["F"].cpu().numpy())
    with pytest.raises(pkg.PodError) as ei:
        pod.set_embedding(a, np.zeros(12))  # degree 11 > 8
    assert ei.value.code == pkg.POD_EINVAL
    with pytest.raises(pkg.PodError) as ei:
        pod.set_embedding(np.full(pod.M, np.nan), alpha)
    assert ei.value.code == pkg.POD_EINVAL
