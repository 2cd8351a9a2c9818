"""Work split over ranks (one GPU per rank).

Fit: configurations are independent, so each rank builds the design matrix of
its share and the normal equations G = A^T A, r = A^T b (Eq. 63a) are summed
with one all-reduce of M*M + M doubles; every rank then solves the same system
(Cholesky on its GPU) and the training errors are summed with a second, 4-value
all-reduce.  The three stages default to the library's pod_fit_normal /
pod_fit_solve / pod_fit_residual; they can be replaced (same signatures) to run
the sharding logic without a GPU.

Energy and forces of one large periodic system: spatial decomposition into
slabs.  Each domain is evaluated as its local atoms plus ghost copies of every
atom within the cut-off of the slab (``n_local`` of pod_system), and the
domains' forces are summed onto the owning atoms.  Here the reverse exchange is
one all-reduce of the stitched force array (correct by construction, not the
point-to-point halo exchange a production MD code would use).
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


def slab_domains(pos, box, r_cut, n_slabs, axis=0):
    """Slabs along `axis` of a periodic box.  Returns one (idx, sub_pos, sub_box,
    sub_pbc, n_local) per slab: `sub_pos` ((n, 3)) holds the slab's local atoms
    (wrapped coordinate along `axis` in [s L / n_slabs, (s + 1) L / n_slabs)) first,
    then ghosts -- every periodic image along `axis` of any atom within `r_cut` of
    the slab -- and idx[k] is the original index of sub-system atom k.  The
    sub-box is open along `axis` (extent: the slab and both ghost layers, the
    coordinates shifted to start at 0) and keeps the periodic box along the
    other axes."""
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    L = float(box[axis])
    x = np.mod(pos[:, axis], L)
    width = L / n_slabs
    kmax = int(np.ceil(r_cut / L)) + 1
    out = []
    for s_ in range(n_slabs):
        lo, hi = s_ * width, (s_ + 1) * width
        local = np.nonzero((x >= lo) & (x < hi))[0] if s_ < n_slabs - 1 else np.nonzero(x >= lo)[0]
        gidx, gx = [], []
        for k in range(-kmax, kmax + 1):
            xs = x + k * L
            sel = (xs >= lo - r_cut) & (xs < hi + r_cut)
            if k == 0:
                sel &= ~((x >= lo) & ((x < hi) if s_ < n_slabs - 1 else True))
            gidx.append(np.nonzero(sel)[0])
            gx.append(xs[sel])
        gidx = np.concatenate(gidx)
        gx = np.concatenate(gx)
        idx = np.concatenate([local, gidx])
        sub = pos[idx].copy()
        sub[:, axis] = np.concatenate([x[local], gx]) - (lo - r_cut)
        sub_box = box.copy()
        sub_box[axis] = width + 2.0 * r_cut + 1e-9 * L
        pbc = [1, 1, 1]
        pbc[axis] = 0
        out.append((idx, sub, sub_box, tuple(pbc), len(local)))
    return out


def energy_forces_domains(evaluate, pos, box, r_cut, n_slabs, *, axis=0, group=None):
    """Energy, atom energies, forces and virial of a periodic system from its slab
    domains.  `evaluate(sub_pos, sub_box, sub_pbc, n_local)` returns (E, Ei, F, W)
    of one domain with forces on all of its atoms (local and ghost) -- e.g. the
    library's energy_forces with ``n_local``.  Without a process group every slab
    is evaluated here; with one, rank r evaluates slabs r, r + world, ... and one
    all-reduce of N * 3 + N + 10 doubles stitches the result on every rank."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    rank, world = 0, 1
    if group is not None:
        import torch.distributed as dist
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    F = np.zeros((N, 3))
    Ei = np.zeros(N)
    E = 0.0
    W = np.zeros((3, 3))
    for s_, (idx, sub, sub_box, pbc, n_local) in enumerate(slab_domains(pos, box, r_cut, n_slabs, axis)):
        if s_ % world != rank:
            continue
        e, ei, f, w = evaluate(sub, sub_box, pbc, n_local)
        E += float(e)
        np.add.at(F, idx, np.asarray(f, dtype=np.float64))
        Ei[idx[:n_local]] += np.asarray(ei, dtype=np.float64)[:n_local]
        W += np.asarray(w, dtype=np.float64).reshape(3, 3)
    if group is not None:
        import torch
        import torch.distributed as dist
        buf = torch.tensor(np.concatenate([F.ravel(), Ei, [E], W.ravel()]), dtype=torch.float64)
        dist.all_reduce(buf, group=group)
        b = buf.numpy()
        F = b[: 3 * N].reshape(N, 3)
        Ei = b[3 * N: 4 * N]
        E = float(b[4 * N])
        W = b[4 * N + 1:].reshape(3, 3)
    return E, Ei, F, W
