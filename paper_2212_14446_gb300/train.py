"""Nonlinear training of the quadratic and embedding POD models (Eq. 63b).

The linear model's loss is quadratic in c and its minimiser is the
least-squares fit of Eq. 63a (``POD.fit``).  The quadratic model (Sec. 4,
E_i = c . D_i + sum_{m <= n} beta_mn D_im D_in) and the embedding model (Sec. 3,
E_i = c . D_i + F(a . D_i), F(rho) = sum_k alpha_k rho^k) are trained here by
minimising the force-matching loss

    L(theta) = sum_c w_E^2 ((E_c - E_c^ref) / N_c)^2 + w_F^2 sum_k |F_k - F_k^ref|^2

with limited-memory BFGS.  Each loss evaluation runs on the GPU through the
library: energies and forces of the whole training batch with the current
parameters (pod_energy_forces), per-atom descriptors (pod_descriptors), their
directional derivatives along v = F - F^ref (pod_descriptors_tangent), and the
parameter gradient assembled from them (pod_model_gradients).  Only the
parameter vector and the L-BFGS two-loop recursion live on the host.
"""
from __future__ import annotations

import numpy as np


class ForceMatchingLoss:
    """L(theta) and dL/dtheta of one model on a training batch kept on the device.

    model: "quadratic" (theta = [c (M), beta_mn for m <= n, row-major]) or
    "embedding" (theta = [c (M), a (M), alpha_0..alpha_degree])."""

    def __init__(self, pod, configs, E_ref, F_ref, model, *, degree=3, w_E=100.0, w_F=1.0):
        import torch
        from . import POD, pod_energy_forces, pod_descriptors, pod_descriptors_tangent
        self._ef, self._desc, self._tan = pod_energy_forces, pod_descriptors, pod_descriptors_tangent
        if model not in ("quadratic", "embedding"):
            raise ValueError("model must be 'quadratic' or 'embedding'")
        self.pod, self.model, self.degree = pod, model, int(degree)
        self.w_E, self.w_F = float(w_E), float(w_F)
        M = pod.M
        self.M = M
        pos, offs, boxes, pbcs = POD.pack_batch(configs)
        self.offs = offs
        self.x = torch.tensor(pos, dtype=torch.float64, device="cuda")
        self.sysb = pod.batch_system(self.x, offs, boxes, pbcs)
        self.N = int(offs[-1])
        self.ncfg = len(configs)
        self.E_ref = torch.tensor(np.asarray(E_ref, dtype=np.float64), device="cuda")
        self.F_ref = torch.tensor(np.ascontiguousarray(np.concatenate([np.asarray(f) for f in F_ref], axis=0).T),
                                  dtype=torch.float64, device="cuda")
        n_c = np.diff(offs).astype(np.float64)
        self.n_cfg = torch.tensor(n_c, device="cuda")
        self.cfg_of = torch.tensor(np.repeat(np.arange(self.ncfg), np.diff(offs)), device="cuda")
        self.E = torch.empty(self.ncfg, dtype=torch.float64, device="cuda")
        self.F = torch.empty((3, self.N), dtype=torch.float64, device="cuda")
        self.D = torch.empty((self.N, M), dtype=torch.float64, device="cuda")
        self.Dd = torch.empty((self.N, M), dtype=torch.float64, device="cuda")
        self.nq = M * (M + 1) // 2
        self.n_params = M + (self.nq if model == "quadratic" else M + self.degree + 1)
        self.evals = 0

    # -- parameters
    def split(self, theta):
        M = self.M
        theta = np.asarray(theta, dtype=np.float64)
        c = theta[:M]
        if self.model == "quadratic":
            beta = np.zeros((M, M))
            beta[np.triu_indices(M)] = theta[M:]
            return c, beta
        return c, theta[M:2 * M], theta[2 * M:]

    def pack(self, c, *rest):
        M = self.M
        if self.model == "quadratic":
            return np.concatenate([np.asarray(c, dtype=np.float64), np.asarray(rest[0])[np.triu_indices(M)]])
        return np.concatenate([np.asarray(c, dtype=np.float64), np.asarray(rest[0], dtype=np.float64),
                               np.asarray(rest[1], dtype=np.float64)])

    def scales(self, theta, probes=16, seed=0):
        """Per-parameter scales for the optimiser: 1 / sqrt of the diagonal of the
        Gauss-Newton matrix J^T J of the loss's residuals (energy rows
        w_E E_c / N_c, force rows w_F F_k), estimated at theta from random sign
        probes z as the mean of (J^T z)^2 -- each J^T z one pass of the same
        kernels as the gradient (descriptor tangent along the force part of z,
        then the gradient reduction with the energy part as weights)."""
        import torch
        from . import pod_model_gradients
        self.set_model(theta)
        self._desc(self.pod.h, self.sysb, self.D)
        g = np.random.Generator(np.random.PCG64(seed))
        acc = np.zeros(self.n_params)
        n_c = self.n_cfg.cpu().numpy()
        cfg_of = self.cfg_of.cpu().numpy()
        for _ in range(probes):
            zE = g.choice([-1.0, 1.0], size=self.ncfg)
            zF = torch.tensor(g.choice([-1.0, 1.0], size=(3, self.N)), dtype=torch.float64, device="cuda")
            w = torch.tensor((self.w_E * zE / n_c)[cfg_of], dtype=torch.float64, device="cuda")
            self._tan(self.pod.h, self.sysb, zF, self.Dd)
            jz = pod_model_gradients(self.pod.h, self.D, self.Dd, w, -self.w_F, self.n_params)
            acc += jz * jz
        diag = acc / probes
        diag = np.where(diag > 0, diag, 1.0)
        return 1.0 / np.sqrt(diag)

    def set_model(self, theta):
        parts = self.split(theta)
        if self.model == "quadratic":
            self.pod.set_quadratic(parts[1])
        else:
            self.pod.set_embedding(parts[1], parts[2])
        return parts[0]

    # -- loss and gradient
    def __call__(self, theta):
        import torch
        from . import pod_model_gradients
        c = torch.tensor(self.set_model(theta), dtype=torch.float64, device="cuda")
        self._ef(self.pod.h, self.sysb, c, self.E, None, self.F, None)
        rE = (self.E - self.E_ref) / self.n_cfg
        v = (self.F - self.F_ref).contiguous()
        L = self.w_E ** 2 * float(torch.sum(rE * rE)) + self.w_F ** 2 * float(torch.sum(v * v))
        w = (2.0 * self.w_E ** 2 * rE / self.n_cfg)[self.cfg_of].contiguous()
        self._desc(self.pod.h, self.sysb, self.D)
        self._tan(self.pod.h, self.sysb, v, self.Dd)
        g = pod_model_gradients(self.pod.h, self.D, self.Dd, w, -2.0 * self.w_F ** 2, self.n_params)
        self.evals += 1
        return L, g


def lbfgs(fun, x0, iters=200, memory=30, gtol=1e-14, ftol=1e-15):
    """Limited-memory BFGS.  Line search: a trial step of length 1 along the
    L-BFGS direction d, then the minimiser of the quadratic through f(x), the
    slope g.d and f(x + d) (exact for a quadratic loss, so the iteration then
    behaves like conjugate gradients), kept if it decreases f, else the trial
    step, else backtracking.  fun(x) -> (f, g).  Stops after `iters` steps, when
    |g| falls below gtol |g_0|, when a step changes f by less than ftol |f|, or
    when no step decreases f.  Returns (x, f, history of f)."""
    x = np.array(x0, dtype=np.float64)
    f, g = fun(x)
    g0 = float(np.linalg.norm(g))
    hist = [f]
    S, Y = [], []
    for _ in range(iters):
        if not np.all(np.isfinite(g)) or f == 0.0 or np.linalg.norm(g) <= gtol * g0:
            break
        q = g.copy()
        alphas = []
        for s, y in reversed(list(zip(S, Y))):
            rho = 1.0 / float(y @ s)
            a = rho * float(s @ q)
            alphas.append((a, rho, s, y))
            q -= a * y
        if S:
            q *= float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
        for a, rho, s, y in reversed(alphas):
            b = rho * float(y @ q)
            q += (a - b) * s
        d = -q
        slope = float(g @ d)
        if slope >= 0:  # not a descent direction: restart along -g
            S, Y = [], []
            d = -g
            slope = -float(g @ g)
        f1, g1 = fun(x + d)
        best = (x + d, f1, g1)
        curv = 2.0 * (f1 - f - slope)
        if np.isfinite(f1) and curv > 0:
            xa = x + (-slope / curv) * d
            fa, ga = fun(xa)
            if np.isfinite(fa) and fa < f1:
                best = (xa, fa, ga)
        xn, fn, gn = best
        step = 1.0
        while not (np.isfinite(fn) and fn < f):  # backtracking
            step *= 0.5
            if step < 1e-20:
                return x, f, hist
            xn = x + step * d
            fn, gn = fun(xn)
        s, y = xn - x, gn - g
        if float(y @ s) > 1e-300:
            S.append(s)
            Y.append(y)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        done = abs(f - fn) <= ftol * abs(f)
        x, f, g = xn, fn, gn
        hist.append(f)
        if done:
            break
    return x, f, hist


def lbfgs_scaled(fun, x0, scale, **kw):
    """lbfgs in the variables y = x / scale (a diagonal preconditioner)."""
    scale = np.asarray(scale, dtype=np.float64)

    def fy(y):
        f, g = fun(y * scale)
        return f, g * scale

    y, f, hist = lbfgs(fy, np.asarray(x0, dtype=np.float64) / scale, **kw)
    return y * scale, f, hist


def train(pod, configs, E_ref, F_ref, model, theta0, *, degree=3, iters=200, w_E=100.0, w_F=1.0,
          precondition=False):
    """Minimise the force-matching loss of `model` from theta0 (see
    ForceMatchingLoss for the layout) with L-BFGS; with precondition=True each
    parameter is scaled by the Gauss-Newton diagonal at theta0 (random-probe
    estimate; it helps when parameter scales differ widely but the columns are
    not nearly collinear).  Leaves the trained model set on the handle and returns
    (theta, loss, history)."""
    loss = ForceMatchingLoss(pod, configs, E_ref, F_ref, model, degree=degree, w_E=w_E, w_F=w_F)
    if precondition:
        theta, f, hist = lbfgs_scaled(loss, theta0, loss.scales(theta0), iters=iters)
    else:
        theta, f, hist = lbfgs(loss, theta0, iters=iters)
    loss.set_model(theta)
    return theta, f, hist
