"""Nonlinear training (Eq. 63b) of the quadratic and embedding models on the GPU.

* The loss and its parameter gradient (energies and forces of the batch,
  per-atom descriptors, their directional derivatives along F - F_ref and the
  gradient reduction, all through the library's FP64 path) against the FP64
  oracle: the loss from the oracle's own energies and forces of the quadratic
  and embedding models, the gradient against central differences of that loss.
* Training recovers a teacher: labels from a quadratic (embedding) teacher,
  L-BFGS from a perturbed start reduces the loss by eight orders of magnitude and
  recovers the identifiable parameters (quadratic: beta_mn for m, n >= 1 and c_n + beta_0n;
  the one-body descriptor is 1, so c_n and beta_0n enter only as their sum).
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


def _configs(n, replica, max_atoms):
    out, k = [], 0
    while len(out) < n:
        cfg = synth.config_train(k, replica)
        k += 1
        if cfg.n <= max_atoms:
            out.append(cfg)
    return out


def _oracle_loss(o, cfgs, E_ref, F_ref, model, parts, w_E=100.0, w_F=1.0):
    L = 0.0
    for cfg, e_ref, f_ref in zip(cfgs, E_ref, F_ref):
        if model == "quadratic":
            _, E, F, _ = o.energy_forces_quadratic(cfg, parts[0], parts[1])
        else:
            _, E, F, _ = o.energy_forces_embedding(cfg, parts[0], parts[1], parts[2])
        L += w_E ** 2 * ((E - e_ref) / cfg.n) ** 2 + w_F ** 2 * float(np.sum((F - f_ref) ** 2))
    return L


@pytest.mark.parametrize("model", ["quadratic", "embedding"])
def test_loss_gradient_against_oracle_differences(pkg, model):
    from paper_2212_14446_gb300.train import ForceMatchingLoss
    p = synth.params_small()
    o = oracle.Oracle(p)
    cfgs = _configs(5, 21, 30)
    g = synth.rng(22)
    ct = synth.coefficients(o.M, 23)
    E_ref, F_ref = [], []
    for cfg in cfgs:
        _, E, F, _ = o.energy_forces(cfg, ct)
        E_ref.append(E + 1e-3 * cfg.n * g.normal())
        F_ref.append(F + 5e-2 * g.normal(size=F.shape))
    pod = pkg.POD(p, precision="fp64", Q=o.Q)
    loss = ForceMatchingLoss(pod, cfgs, E_ref, F_ref, model)
    c = ct + 1e-3 * g.normal(size=o.M)
    if model == "quadratic":
        theta = loss.pack(c, 1e-3 * g.normal(size=(o.M, o.M)))
    else:
        a = np.zeros(o.M)
        a[1:] = 1e-2 * g.normal(size=o.M - 1)
        theta = loss.pack(c, a, np.array([0.3, -0.2, 5e-3, -1e-4]))
    L, grad = loss(theta)
    L_o = _oracle_loss(o, cfgs, E_ref, F_ref, model, loss.split(theta))
    assert L == pytest.approx(L_o, rel=1e-10)
    idx = sorted(set(synth.rng(24).choice(theta.size, size=12, replace=False).tolist()) | {0, o.M, theta.size - 1})
    for k in idx:
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (_oracle_loss(o, cfgs, E_ref, F_ref, model, loss.split(tp)) -
              _oracle_loss(o, cfgs, E_ref, F_ref, model, loss.split(tm))) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-5 * max(np.max(np.abs(grad)), 1e-12) + 1e-7 * abs(fd), (k, grad[k], fd)


def _teacher_labels(pkg, p, cfgs, model, parts):
    pod = pkg.POD(p, precision="fp64")
    if model == "quadratic":
        pod.set_quadratic(parts[1])
    else:
        pod.set_embedding(parts[1], parts[2])
    out = pod.energy_forces_batch(cfgs, torch.tensor(parts[0]))
    E = out["E"].cpu().numpy()
    Fall = out["F"].cpu().numpy()
    offs = out["offs"]
    return E, [Fall[offs[k]:offs[k + 1]] for k in range(len(cfgs))], pod.Q


def test_training_recovers_quadratic_teacher(pkg):
    from paper_2212_14446_gb300.train import train
    p = synth.params_small()
    M = oracle.Oracle(p).M
    cfgs = _configs(30, 25, 40)
    g = synth.rng(26)
    cstar = synth.coefficients(M, 27)
    bstar = np.triu(2e-3 * g.normal(size=(M, M)))
    E_ref, F_ref, Q = _teacher_labels(pkg, p, cfgs, "quadratic", (cstar, bstar))
    pod = pkg.POD(p, precision="fp64", Q=Q)
    theta0 = np.concatenate([cstar + 1e-3 * g.normal(size=M), np.zeros(M * (M + 1) // 2)])
    from paper_2212_14446_gb300.train import ForceMatchingLoss
    L0, _ = ForceMatchingLoss(pod, cfgs, E_ref, F_ref, "quadratic")(theta0)
    theta, L, hist = train(pod, cfgs, E_ref, F_ref, "quadratic", theta0, iters=400)
    assert L <= 1e-8 * L0, (L, L0, len(hist))
    c = theta[:M]
    beta = np.zeros((M, M))
    beta[np.triu_indices(M)] = theta[M:]
    assert np.max(np.abs(beta[1:, 1:] - bstar[1:, 1:])) <= 1e-3 * np.max(np.abs(bstar))
    assert np.max(np.abs((c[1:] + beta[0, 1:]) - (cstar[1:] + bstar[0, 1:]))) <= 1e-3 * np.max(np.abs(cstar))


def test_training_recovers_embedding_teacher(pkg):
    from paper_2212_14446_gb300.train import ForceMatchingLoss, train
    p = synth.params_small()
    M = oracle.Oracle(p).M
    cfgs = _configs(30, 28, 40)
    g = synth.rng(29)
    cstar = synth.coefficients(M, 30)
    astar = np.zeros(M)
    astar[1:] = 1e-2 * g.normal(size=M - 1)
    alstar = np.array([0.3, -0.2, 5e-3, -1e-4])
    E_ref, F_ref, Q = _teacher_labels(pkg, p, cfgs, "embedding", (cstar, astar, alstar))
    pod = pkg.POD(p, precision="fp64", Q=Q)
    theta0 = np.concatenate([cstar, astar * (1.0 + 0.05 * g.normal(size=M)), alstar * 1.05])
    loss = ForceMatchingLoss(pod, cfgs, E_ref, F_ref, "embedding")
    L0, _ = loss(theta0)
    theta, L, hist = train(pod, cfgs, E_ref, F_ref, "embedding", theta0, iters=400)
    assert L <= 1e-8 * L0, (L, L0, len(hist))
    # the trained model reproduces the teacher's energies and forces
    out = pod.energy_forces_batch(cfgs, torch.tensor(theta[:M]))
    E = out["E"].cpu().numpy()
    assert np.max(np.abs(E - E_ref) / np.array([cf.n for cf in cfgs])) <= 1e-6
