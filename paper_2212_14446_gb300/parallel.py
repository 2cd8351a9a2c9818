"""Work split over ranks (one GPU per rank).

Fit: configurations are independent, so each rank builds the design matrix of
its share and the normal equations G = A^T A, r = A^T b (Eq. 63a) are summed
with one all-reduce of M*M + M doubles; every rank then solves the same system
(Cholesky on its GPU) and the training errors are summed with a second, 4-value
all-reduce.  The three stages default to the library's pod_fit_normal /
pod_fit_solve / pod_fit_residual; they can be replaced (same signatures) to run
the sharding logic without a GPU.

Energy and forces of one large periodic system: spatial decomposition into
slabs along one axis, one slab per rank (``SlabDomain``).  Each rank owns the
atoms of its slab and keeps their positions and forces on its GPU.  Per
evaluation it
  1. selects on the device (pod_halo_select) its atoms within the list radius of
     its lower and upper slab faces, with their positions as the neighbouring
     domain lays them out (periodic image shift, domain origin);
  2. sends them to the neighbouring ranks and receives theirs (point to point:
     O(surface) data, not O(N));
  3. evaluates its domain -- own atoms first, ghosts after them (n_local), the
     axis open -- with forces on every atom of the domain;
  4. returns the forces on the ghosts to the ranks that own them and adds the
     forces returned to it onto its own halo atoms (pod_halo_add);
  5. sums E and the virial over ranks (one all-reduce of 10 doubles).
The exchange is torch.distributed point-to-point (NCCL between GPUs, gloo on the
host); the device steps are replaceable (``HostOps``) so the exchange logic runs
without a GPU.  ``slab_domains`` / ``energy_forces_domains`` are the earlier
host-side form (ghost selection in numpy, one all-reduce of the stitched force
array), kept as a reference.
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


# ---------------------------------------------------------------- slab halo exchange

class SlabDomain:
    """Slab `rank` of `world` along `axis` of a periodic orthorhombic box: owned
    atoms have the wrapped axis coordinate in [lo, hi); the domain evaluated on
    this rank spans [lo - r_list, hi + r_list) along the axis, laid out from 0
    (open boundary there), periodic along the other axes.  Needs slabs at least
    r_list wide, so that ghosts come from the two neighbouring slabs only."""

    def __init__(self, box, r_list, axis=0, rank=0, world=1):
        self.box = np.asarray(box, dtype=np.float64)
        self.r = float(r_list)
        self.axis = int(axis)
        self.rank, self.world = int(rank), int(world)
        self.L = float(self.box[self.axis])
        self.lo, self.hi = self.bounds(self.rank)
        if min(self.hi - self.lo, self.L / self.world) < self.r:
            raise ValueError("slabs must be at least the list radius wide")
        self.origin = self.lo - self.r
        self.sub_box = self.box.copy()
        self.sub_box[self.axis] = (self.hi - self.lo) + 2.0 * self.r + 1e-9 * self.L
        pbc = [1, 1, 1]
        pbc[self.axis] = 0
        self.sub_pbc = tuple(pbc)

    def bounds(self, rank):
        w = self.L / self.world
        return rank * w, (self.L if rank == self.world - 1 else (rank + 1) * w)

    def lower_rank(self):
        return (self.rank - 1) % self.world

    def upper_rank(self):
        return (self.rank + 1) % self.world

    def own(self):
        """(x0, x1, shift, offset) selecting the owned atoms in this domain's layout."""
        return self.lo, self.hi, 0.0, self.origin

    def lower_halo(self):
        """Owned atoms within r of the lower face, laid out for the lower neighbour
        (they become its upper ghosts; across the periodic boundary: +L)."""
        lo_n, _ = self.bounds(self.lower_rank())
        return self.lo, self.lo + self.r, (self.L if self.rank == 0 else 0.0), lo_n - self.r

    def upper_halo(self):
        """Owned atoms within r of the upper face, laid out for the upper neighbour
        (they become its lower ghosts; across the periodic boundary: -L)."""
        lo_n, _ = self.bounds(self.upper_rank())
        return self.hi - self.r, self.hi, (-self.L if self.rank == self.world - 1 else 0.0), lo_n - self.r


class DeviceOps:
    """The device steps of the exchange through the library (CUDA tensors)."""

    def __init__(self, pod, stream=None):
        self.pod = pod
        self.stream = stream

    def select(self, x, x0, x1, shift, offset, axis, L):
        import torch
        from . import pod_halo_select
        n = x.shape[1]
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
        out = torch.empty((3, max(n, 1)), dtype=torch.float64, device=x.device)
        k = pod_halo_select(self.pod.h, x, axis, L, x0, x1, shift, offset, max(n, 1), idx, out, self.stream)
        return idx[:k].contiguous(), out[:, :k].contiguous()

    def evaluate(self, sub, sub_box, sub_pbc, n_local, c):
        out = self.pod.energy_forces(sub, sub_box, c, pbc=sub_pbc, n_local=n_local, stream=self.stream)
        return out["E"].reshape(1), out["Ei"], out["F"].t().contiguous(), out["W"].reshape(9)

    def add(self, F, G, idx):
        from . import pod_halo_add
        if idx.numel():
            pod_halo_add(self.pod.h, G.contiguous(), idx, idx.numel(), F, self.stream)

    def cat(self, parts):
        import torch
        return torch.cat(parts, dim=1).contiguous()


class HostOps:
    """The same steps on the host (numpy arrays wrapped as CPU tensors), with
    `evaluate(sub (3, n), sub_box, sub_pbc, n_local, c) -> (E, Ei, F (3, n), W (9,))`
    supplied by the caller (e.g. the FP64 oracle)."""

    def __init__(self, evaluate):
        self._evaluate = evaluate

    def select(self, x, x0, x1, shift, offset, axis, L):
        import torch
        xa = x.numpy()
        v = xa[axis]
        xw = np.where((v >= 0.0) & (v < L), v, v - L * np.floor(v / L))
        idx = np.nonzero((xw >= x0) & (xw < x1))[0]
        out = xa[:, idx].copy()
        out[axis] = (xw[idx] + shift) - offset
        return torch.tensor(idx, dtype=torch.int32), torch.tensor(out)

    def evaluate(self, sub, sub_box, sub_pbc, n_local, c):
        import torch
        E, Ei, F, W = self._evaluate(sub.numpy(), sub_box, sub_pbc, n_local, c)
        return (torch.tensor([float(E)], dtype=torch.float64), torch.tensor(np.asarray(Ei)), torch.tensor(np.asarray(F)),
                torch.tensor(np.asarray(W).reshape(9)))

    def add(self, F, G, idx):
        if idx.numel():
            F[:, idx.long()] += G

    def cat(self, parts):
        import torch
        return torch.cat(parts, dim=1).contiguous()


class DistComm:
    """Neighbour exchange and sums over a torch.distributed process group
    (NCCL between GPUs, gloo on the host): point-to-point messages, posted in a
    fixed order so that two messages between the same pair of ranks (two slabs
    per ring) match in order."""

    def __init__(self, dom, group=None):
        self.dom = dom
        self.group = group

    def _p2p(self, sends, recvs):
        import torch.distributed as dist
        ops = [dist.P2POp(dist.isend, t, dst, self.group) for t, dst in sends]
        ops += [dist.P2POp(dist.irecv, t, src, self.group) for t, src in recvs]
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def swap(self, to_lower, to_upper):
        """Send (3, n) tensors to the lower and upper neighbours; returns what
        they sent here: (from_upper, from_lower)."""
        import torch
        lo, up = self.dom.lower_rank(), self.dom.upper_rank()
        dev = to_lower.device
        cnt = torch.tensor([to_lower.shape[1], to_upper.shape[1]], dtype=torch.int64, device=dev)
        cu = torch.zeros(2, dtype=torch.int64, device=dev)
        cl = torch.zeros(2, dtype=torch.int64, device=dev)
        self._p2p([(cnt, lo), (cnt.clone(), up)], [(cu, up), (cl, lo)])
        from_upper = torch.empty((3, int(cu[0])), dtype=to_lower.dtype, device=dev)
        from_lower = torch.empty((3, int(cl[1])), dtype=to_lower.dtype, device=dev)
        self._p2p([(to_lower.contiguous(), lo), (to_upper.contiguous(), up)], [(from_upper, up), (from_lower, lo)])
        return from_upper, from_lower

    def allreduce(self, t):
        import torch.distributed as dist
        dist.all_reduce(t, group=self.group)
        return t


class LoopComm:
    """One rank: the slab's two neighbours are the slab itself."""

    def swap(self, to_lower, to_upper):
        return to_lower, to_upper

    def allreduce(self, t):
        return t


class ThreadComm:
    """The exchange between ranks run as threads of one process (each thread one
    slab, with its own library handle): mailboxes keyed by sender, receiver and
    round, sums taken in rank order.  A thread hands over tensors only after its
    stream has finished them (the library's calls wait for their stream)."""

    def __init__(self, world):
        import threading
        self.world = world
        self.cv = threading.Condition()
        self.box = {}
        self.round = [0] * world
        self.sums = {}

    def rank(self, dom):
        comm = self

        class _R:
            def swap(self, to_lower, to_upper):
                return comm._swap(dom, to_lower, to_upper)

            def allreduce(self, t):
                return comm._allreduce(dom.rank, t)
        return _R()

    def _swap(self, dom, to_lower, to_upper):
        r = dom.rank
        with self.cv:
            k = self.round[r]
            self.round[r] += 1
            self.box[(r, dom.lower_rank(), "down", k)] = to_lower
            self.box[(r, dom.upper_rank(), "up", k)] = to_upper
            self.cv.notify_all()
            key_u = (dom.upper_rank(), r, "down", k)
            key_l = (dom.lower_rank(), r, "up", k)
            self.cv.wait_for(lambda: key_u in self.box and key_l in self.box, timeout=120)
            if key_u not in self.box or key_l not in self.box:
                raise TimeoutError("a rank did not reach the exchange")
            return self.box.pop(key_u), self.box.pop(key_l)

    def _allreduce(self, r, t):
        with self.cv:
            k = self.round[r]
            self.round[r] += 1
            self.sums.setdefault(k, {})[r] = t.clone()
            self.cv.notify_all()
            self.cv.wait_for(lambda: len(self.sums[k]) == self.world, timeout=120)
            if len(self.sums[k]) != self.world:
                raise TimeoutError("a rank did not reach the sum")
            tot = self.sums[k][0].clone()
            for q in range(1, self.world):
                tot += self.sums[k][q]
            return tot


def slab_energy_forces(dom, ops, x_own, c, comm=None):
    """One evaluation of a slab-decomposed system on this rank.  x_own (3, n):
    the positions of the atoms this rank owns (all inside its slab); comm:
    DistComm (a process group), ThreadComm.rank (ranks as threads) or LoopComm
    (one rank, the default).  Returns (E, Ei_own (n,), F_own (3, n), W (9,)),
    E and W summed over every rank."""
    import torch
    comm = comm if comm is not None else LoopComm()
    axis, L = dom.axis, dom.L
    n = x_own.shape[1]
    idx_own, local = ops.select(x_own, *dom.own(), axis, L)
    if idx_own.numel() != n:
        raise ValueError("every owned atom must lie inside its slab")
    idx_lo, halo_lo = ops.select(x_own, *dom.lower_halo(), axis, L)
    idx_hi, halo_hi = ops.select(x_own, *dom.upper_halo(), axis, L)
    # the lower halo becomes the lower neighbour's upper ghosts and vice versa
    ghost_upper, ghost_lower = comm.swap(halo_lo, halo_hi)
    ngl, ngu = ghost_lower.shape[1], ghost_upper.shape[1]
    sub = ops.cat([local, ghost_lower, ghost_upper])
    E, Ei, F, W = ops.evaluate(sub, dom.sub_box, dom.sub_pbc, n, c)
    F_own = F[:, :n].contiguous()
    f_lower = F[:, n:n + ngl].contiguous()              # forces on the lower neighbour's atoms
    f_upper = F[:, n + ngl:n + ngl + ngu].contiguous()  # forces on the upper neighbour's atoms
    back_hi, back_lo = comm.swap(f_lower, f_upper)
    if back_lo.shape[1] != idx_lo.numel() or back_hi.shape[1] != idx_hi.numel():
        raise RuntimeError("halo exchange: returned forces do not match the halo")
    # the owned atoms' share of the neighbours' pair terms, in a fixed order
    ops.add(F_own, back_lo, idx_lo)
    ops.add(F_own, back_hi, idx_hi)
    tot = torch.cat([E.reshape(1).to(torch.float64), W.reshape(9).to(torch.float64)])
    tot = comm.allreduce(tot)
    return tot[0], Ei[:n], F_own, tot[1:]


def owned_atoms(dom, pos):
    """Indices (ascending) of the atoms of pos ((N, 3) host array) that slab
    `dom` owns: wrapped axis coordinate in [lo, hi)."""
    v = np.asarray(pos, dtype=np.float64)[:, dom.axis]
    L = dom.L
    x = np.where((v >= 0.0) & (v < L), v, v - L * np.floor(v / L))
    return np.nonzero((x >= dom.lo) & (x < dom.hi))[0]
