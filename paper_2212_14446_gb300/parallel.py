"""Fit sharded over ranks (one GPU per rank): configurations are independent,
so each rank builds the design matrix of its share and the normal equations
G = A^T A, r = A^T b (Eq. 63a) are summed with one all-reduce of M*M + M
doubles; every rank then solves the same system (Cholesky on its GPU) and the
training errors are summed with a second, 4-value all-reduce.

The three stages default to the library's pod_fit_normal / pod_fit_solve /
pod_fit_residual; they can be replaced (same signatures) to run the sharding
logic without a GPU.
"""
from __future__ import annotations

import numpy as np


def shard_indices(n_items: int, rank: int, world: int) -> list:
    """Round-robin share of rank `rank` (sizes differ by at most one)."""
    return list(range(rank, n_items, world))


def fit_sharded(pod, configs, E_ref, F_ref, *, w_E=100.0, w_F=1.0, gamma=1e-12, per_atom_energy=True, group=None,
                normal=None, solve=None, residual=None, device=None):
    """Returns (c, mae_E per atom, mae_F per component), identical on every rank."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    M = pod.M
    if normal is None:
        def normal(cfgs, E, F, g):
            return pod.fit_normal(cfgs, E, F, w_E=w_E, w_F=w_F, gamma=g, per_atom_energy=per_atom_energy)
    if solve is None:
        solve = pod.fit_solve
    if residual is None:
        residual = pod.fit_residual
    idx = shard_indices(len(configs), rank, world)
    E_ref = np.asarray(E_ref, dtype=np.float64)
    if idx:
        G, r = normal([configs[i] for i in idx], E_ref[idx], [F_ref[i] for i in idx], gamma if rank == 0 else 0.0)
    else:
        G, r = np.zeros((M, M)), np.zeros(M)
        if rank == 0:
            G = G + gamma * np.eye(M)
    buf = torch.tensor(np.concatenate([np.asarray(G).ravel(), np.asarray(r)]), dtype=torch.float64, device=device)
    dist.all_reduce(buf, group=group)
    buf = buf.cpu().numpy()
    c = solve(buf[: M * M].reshape(M, M), buf[M * M:])
    if idx:
        se, sf, ne, nf = residual(c)
    else:
        se, sf, ne, nf = 0.0, 0.0, 0, 0
    sums = torch.tensor([se, sf, float(ne), float(nf)], dtype=torch.float64, device=device)
    dist.all_reduce(sums, group=group)
    se, sf, ne, nf = sums.cpu().numpy()
    return c, se / max(ne, 1.0), sf / max(nf, 1.0)
