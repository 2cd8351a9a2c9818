"""The host side of the nonlinear training loop: L-BFGS with its diagonal
preconditioner on problems with known minimisers (no GPU)."""
import numpy as np

import synth
from paper_2212_14446_gb300.train import lbfgs, lbfgs_scaled


def _lsq(n=400, p=60, spread=8.0, seed=3):
    g = synth.rng(seed)
    A = g.normal(size=(n, p)) * np.logspace(-spread / 2, spread / 2, p)[None, :]  # column scales over 8 decades
    x_star = g.normal(size=p)
    b = A @ x_star

    def fun(x):
        r = A @ x - b
        return float(r @ r), 2.0 * A.T @ r
    return A, x_star, fun


def test_lbfgs_solves_a_well_scaled_quadratic():
    g = synth.rng(4)
    A = g.normal(size=(200, 30))
    x_star = g.normal(size=30)
    b = A @ x_star
    x, f, hist = lbfgs(lambda x: (float((A @ x - b) @ (A @ x - b)), 2 * A.T @ (A @ x - b)), np.zeros(30), iters=300)
    assert f <= 1e-20 * hist[0]
    assert np.allclose(x, x_star, rtol=1e-8, atol=1e-8)


def test_diagonal_preconditioner_recovers_badly_scaled_least_squares():
    """Columns over eight decades: scaling each variable by 1 / sqrt(diag(A^T A))
    lets L-BFGS reach the minimiser (the unscaled run stalls far above it)."""
    A, x_star, fun = _lsq()
    scale = 1.0 / np.sqrt(np.sum(A * A, axis=0))
    x, f, hist = lbfgs_scaled(fun, np.zeros(A.shape[1]), scale, iters=400)
    assert f <= 1e-20 * hist[0]
    assert np.max(np.abs(x - x_star) / np.maximum(np.abs(x_star), 1e-3)) <= 1e-6
    _, f_plain, _ = lbfgs(fun, np.zeros(A.shape[1]), iters=400)
    assert f_plain > 1e6 * f
