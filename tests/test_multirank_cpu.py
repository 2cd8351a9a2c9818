"""The sharded fit on two CPU ranks (gloo): each rank forms the normal equations
of its round-robin share of configurations from the oracle's design matrix, one
all-reduce sums them, every rank solves; the result must equal the oracle's
single-process fit.  Exercises the sharding and reduction logic of
paper_2212_14446_gb300.parallel without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _configs():
    out, k = [], 0
    while len(out) < 9:
        cfg = synth.config_train(k, 7)
        k += 1
        if cfg.n <= 24:
            out.append(cfg)
    return out


class _OraclePod:
    """Stands in for the GPU handle: normal equations, solve and residuals from
    the oracle's design matrix."""

    def __init__(self, o):
        self.o = o
        self.M = o.M
        self.A = self.b = None
        self.n_e = 0

    def normal(self, cfgs, E, F, gamma):
        A, b = self.o.design_matrix(cfgs, E, F)
        self.A, self.b = A, b
        e_rows, r = [], 0
        for cfg in cfgs:
            e_rows.append(r)
            r += 1 + 3 * cfg.n
        self.is_e = np.zeros(len(b), dtype=bool)
        self.is_e[e_rows] = True
        return A.T @ A + gamma * np.eye(self.M), A.T @ b

    def solve(self, G, r):
        L = np.linalg.cholesky(G)
        return np.linalg.solve(L.T, np.linalg.solve(L, r))

    def residual(self, c):
        res = np.abs(self.A @ c - self.b)
        return res[self.is_e].sum() / 100.0, res[~self.is_e].sum(), int(self.is_e.sum()), int((~self.is_e).sum())


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2212_14446_gb300 import parallel
        p = synth.params_small()
        o = oracle.Oracle(p)
        cfgs = _configs()
        cstar = synth.coefficients(o.M, 3)
        g = synth.rng(11)
        E_ref, F_ref = [], []
        for cfg in cfgs:
            _, E, F, _ = o.energy_forces(cfg, cstar, fast=True)
            E_ref.append(E + 1e-3 * cfg.n * g.normal())
            F_ref.append(F + 5e-2 * g.normal(size=F.shape))
        fake = _OraclePod(o)
        c, maeE, maeF = parallel.fit_sharded(fake, cfgs, np.array(E_ref), F_ref, normal=fake.normal,
                                             solve=fake.solve, residual=fake.residual)
        q.put((rank, c, maeE, maeF))
    finally:
        dist.destroy_process_group()


def test_sharded_fit_two_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    res.sort(key=lambda t: t[0])
    (_, c0, e0, f0), (_, c1, e1, f1) = res
    assert np.array_equal(c0, c1) and e0 == e1 and f0 == f1  # every rank holds the same solution
    # the single-process oracle fit
    p = synth.params_small()
    o = oracle.Oracle(p)
    cfgs = _configs()
    cstar = synth.coefficients(o.M, 3)
    g = synth.rng(11)
    E_ref, F_ref = [], []
    for cfg in cfgs:
        _, E, F, _ = o.energy_forces(cfg, cstar, fast=True)
        E_ref.append(E + 1e-3 * cfg.n * g.normal())
        F_ref.append(F + 5e-2 * g.normal(size=F.shape))
    c_ref, A, b = o.fit(cfgs, E_ref, F_ref)
    assert np.max(np.abs(A @ c0 - A @ c_ref)) <= 1e-8 * np.max(np.abs(b))


def test_shard_indices_cover_everything():
    from paper_2212_14446_gb300 import parallel
    for n in (0, 1, 5, 9, 2000):
        for w in (1, 2, 3, 8):
            got = sorted(i for r in range(w) for i in parallel.shard_indices(n, r, w))
            assert got == list(range(n))
            sizes = [len(parallel.shard_indices(n, r, w)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1


# ------------------------------------------------- spatial decomposition (slabs)

def _slab_system():
    p = synth.params_small()
    cfg = synth.jitter(synth.bcc(4), 0.1, synth.rng(121))   # 128 atoms, box 13.3 A > 2 r_cut
    return p, cfg, synth.coefficients(oracle.Oracle(p).M, 122)


def _oracle_evaluator(o, c):
    def evaluate(sub, sub_box, pbc, n_local):
        cfg = synth.Config(pos=sub, box=sub_box, pbc=pbc)
        Ei, E, F, W = o.energy_forces_local(cfg, c, n_local)
        return E, Ei, F, W
    return evaluate


def test_slab_domains_cover_every_atom_once():
    """Every atom is local in exactly one slab; every ghost lies within r_cut of
    its slab (along the split axis) and is a periodic image of an atom."""
    from paper_2212_14446_gb300 import parallel
    p, cfg, _ = _slab_system()
    for n_slabs in (2, 3):
        owners = np.zeros(cfg.n, dtype=int)
        for idx, sub, sub_box, pbc, n_local in parallel.slab_domains(cfg.pos, cfg.box, p.r_cut, n_slabs):
            owners[idx[:n_local]] += 1
            assert pbc == (0, 1, 1)
            x = sub[:, 0]
            assert np.all(x >= 0.0) and np.all(x < sub_box[0])
            width = cfg.box[0] / n_slabs
            assert np.all((x[:n_local] >= p.r_cut) & (x[:n_local] < p.r_cut + width + 1e-9))
            # ghosts within r_cut of the slab, images of their atoms by whole boxes
            xg = x[n_local:]
            assert np.all((xg < p.r_cut) | (xg >= p.r_cut + width))
            s_ = int(round(np.min(np.mod(cfg.pos[idx[:n_local], 0], cfg.box[0])) // width)) if n_local else 0
            k = (sub[:, 0] + (s_ * width - p.r_cut) - cfg.pos[idx, 0]) / cfg.box[0]
            assert np.allclose(k, np.round(k), atol=1e-9)
            assert np.array_equal(sub[:, 1:], cfg.pos[idx, 1:])
        assert np.all(owners == 1)


def test_slab_decomposition_equals_whole_system():
    """The oracle on 2 and 3 slab domains (local atoms + ghosts within r_cut),
    forces summed onto the owners, equals the oracle on the whole periodic
    system: the decomposition loses and double-counts no pair term."""
    from paper_2212_14446_gb300 import parallel
    p, cfg, c = _slab_system()
    o = oracle.Oracle(p)
    Ei, E, F, W = o.energy_forces(cfg, c, fast=True)
    for n_slabs in (2, 3):
        Ed, Eid, Fd, Wd = parallel.energy_forces_domains(_oracle_evaluator(o, c), cfg.pos, cfg.box, p.r_cut, n_slabs)
        assert Ed == pytest.approx(E, rel=1e-12)
        assert np.allclose(Eid, Ei, rtol=1e-12, atol=1e-14)
        assert np.max(np.abs(Fd - F)) <= 1e-11 * np.max(np.abs(F))
        assert np.max(np.abs(Wd - W)) <= 1e-11 * np.max(np.abs(W))


def _slab_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2212_14446_gb300 import parallel
        p, cfg, c = _slab_system()
        o = oracle.Oracle(p)
        res = parallel.energy_forces_domains(_oracle_evaluator(o, c), cfg.pos, cfg.box, p.r_cut, 3,
                                             group=dist.group.WORLD)
        q.put((rank,) + tuple(res))
    finally:
        dist.destroy_process_group()


def test_slab_decomposition_two_ranks():
    """Three slabs on two CPU ranks (gloo): each rank evaluates its slabs, one
    all-reduce stitches forces, atom energies, E and W; every rank holds the
    single-process result."""
    from paper_2212_14446_gb300 import parallel
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, cfg, c = _slab_system()
    o = oracle.Oracle(p)
    E1, Ei1, F1, W1 = parallel.energy_forces_domains(_oracle_evaluator(o, c), cfg.pos, cfg.box, p.r_cut, 3)
    for _, E, Ei, F, W in res:
        assert E == pytest.approx(E1, rel=1e-14)
        assert np.allclose(F, F1, rtol=0, atol=1e-13 * np.max(np.abs(F1)))
        assert np.allclose(Ei, Ei1, rtol=1e-14, atol=0) and np.allclose(W, W1, rtol=1e-13, atol=1e-15)


# ------------------------------------- slab halo exchange (point to point, O(surface))

def _halo_system():
    p = synth.params_small()
    cfg = synth.jitter(synth.bcc(6), 0.1, synth.rng(131))   # 432 atoms, box 19.9 A: slabs of >= r_cut
    return p, cfg, synth.coefficients(oracle.Oracle(p).M, 132)


def _host_ops(o, c):
    from paper_2212_14446_gb300 import parallel

    def evaluate(sub, sub_box, pbc, n_local, c_):
        cfg = synth.Config(pos=np.ascontiguousarray(sub.T), box=sub_box, pbc=pbc)
        Ei, E, F, W = o.energy_forces_local(cfg, c, n_local)
        return E, Ei, F.T, W
    return parallel.HostOps(evaluate)


def _halo_rank(rank, world, p, cfg, c, comm_for):
    from paper_2212_14446_gb300 import parallel
    o = oracle.Oracle(p)
    dom = parallel.SlabDomain(cfg.box, p.r_cut, axis=0, rank=rank, world=world)
    own = parallel.owned_atoms(dom, cfg.pos)
    x = torch.tensor(np.ascontiguousarray(cfg.pos[own].T))
    E, Ei, F, W = parallel.slab_energy_forces(dom, _host_ops(o, c), x, c, comm_for(dom))
    return own, float(E), Ei.numpy(), F.numpy(), W.numpy()


def _assemble(n, parts):
    F = np.zeros((n, 3))
    Ei = np.zeros(n)
    seen = np.zeros(n, dtype=int)
    for own, _, ei, f, _ in parts:
        F[own] = f.T
        Ei[own] = ei
        seen[own] += 1
    assert np.all(seen == 1)  # every atom owned by exactly one slab
    return Ei, F


def _check_whole(p, cfg, c, parts):
    o = oracle.Oracle(p)
    Ei0, E0, F0, W0 = o.energy_forces(cfg, c, fast=True)
    Ei, F = _assemble(cfg.n, parts)
    for _, E, _, _, W in parts:  # E and W summed over ranks: the same on every rank
        assert E == pytest.approx(E0, rel=1e-12)
        assert np.max(np.abs(W.reshape(3, 3) - W0)) <= 1e-11 * np.max(np.abs(W0))
    assert np.allclose(Ei, Ei0, rtol=1e-12, atol=1e-14)
    assert np.max(np.abs(F - F0)) <= 1e-11 * np.max(np.abs(F0))


def test_halo_exchange_one_rank_is_the_periodic_system():
    """One slab: its halo layers come back to it as its own ghosts (the periodic
    images across the split axis), so the domain equals the whole system."""
    from paper_2212_14446_gb300 import parallel
    p, cfg, c = _halo_system()
    _check_whole(p, cfg, c, [_halo_rank(0, 1, p, cfg, c, lambda dom: parallel.LoopComm())])


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_ranks_as_threads(world):
    """Two and three slabs run as threads exchanging halos and ghost forces
    through mailboxes: owned forces, atom energies, E and W equal the whole
    system's (two slabs: both neighbours of a slab are the same rank)."""
    import threading
    from paper_2212_14446_gb300 import parallel
    p, cfg, c = _halo_system()
    tc = parallel.ThreadComm(world)
    out, errs = [None] * world, []

    def run(r):
        try:
            out[r] = _halo_rank(r, world, p, cfg, c, tc.rank)
        except Exception as ex:  # surfaced below
            errs.append(ex)

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    _check_whole(p, cfg, c, out)


def _halo_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2212_14446_gb300 import parallel
        p, cfg, c = _halo_system()
        q.put(_halo_rank(rank, world, p, cfg, c, lambda dom: parallel.DistComm(dom, dist.group.WORLD)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_halo_exchange_gloo_ranks(world):
    """Two CPU ranks (gloo, point-to-point messages; both neighbours of a slab
    are the other rank, so message order matters): each rank sends
    only the atoms within r_cut of its slab faces and receives only its ghosts'
    forces; the stitched result equals the single-process whole system."""
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_halo_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, cfg, c = _halo_system()
    _check_whole(p, cfg, c, res)
