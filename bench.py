#!/usr/bin/env python3
"""Benchmark: energy + forces (+ virial) of the linear fast-POD potential.

Workload (default): 8,192-atom BCC Ta (16^3 cubic cells, a = 3.316 A, +-3 %
isotropic strain, jitter N(0, 0.1 A)), r_in = 1, r_cut = 5 A, Ns = 8 snapshots
-> K = 6 radial modes, angular degree 4, 2/3/4-body descriptors (M = 103),
coefficients c ~ N(0, 0.01^2).  Synthetic inputs stand in for the tantalum
training data of the paper.

A step is one full evaluation: neighbour list (cell binning, search, sort,
reverse index), fused atom kernel (radial basis, atomic basis, contraction,
energy, adjoint, pair gradients), force gather + per-atom virial, FP64 energy
and virial reductions.  Metric: atom-steps/s (atoms x steps / device seconds).

Timing: W warm-up steps; the step is captured once in a CUDA graph; each of the
K timed steps is preceded by an L2 flush (a 512 MB write) outside its CUDA-event
pair; value = atoms * K / sum of the K step times, max over ranks.  The fused
atom kernel is timed separately with CUDA events recorded by the library on the
launching stream around that kernel (roofline).  ``e2e`` goes through the
host-buffer entry point with pinned host memory (positions and coefficients in,
energy, atom energies, forces and virial out, the transfers inside the timed
region; the host rewrites the inputs before each call, outside it).

Multi-GPU (torchrun): every rank evaluates its own independent configuration
(weak scaling, no collective on the data path); rank 0 prints the JSON line.

``--impl reference`` times the FP64 CPU oracle (the only reference this method
has: the paper publishes no code) on the same workload, through its fast route
(cell list + atom-density energy and pair gradients) on every host core.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0


# ------------------------------------------------------------ flop model
def monomials(P):
    out = []
    for n in range(P + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                out.append((a, b, n - a - b))
    return out


def algorithmic_flops_per_atom(params, n_pairs_per_atom):
    """Algorithmic arithmetic of one energy + force evaluation per atom, the
    per-unit figures of the method's operation count (independent of how the
    kernel schedules it):
      per pair  forward: snapshots (~12 Ns), projection R and R' (4 Ns K),
                monomials (N_a - 4), B += R A (2 K N_a)             ~0.7 kflop
                adjoint: e = a^T R and R' (a . A) (4 K N_a), grad of
                the angular polynomial and tangential output          ~1.15 kflop
                -> 1.9 kflop per pair at K = 6, N_a = 35 (Ns = 8)
      per atom  three- and four-body contraction and its adjoint over the
                K C_a triple terms of Eq. 30a (C_a of Table 5)        ~13 kflop
                at K = 6, C_a = 209
    For other parameters the per-pair figure scales with K N_a and the per-atom
    one with K C_a (K N_a for a three-body-only model)."""
    K, Pa = params.Kr, params.Pa
    NA = len(monomials(Pa))
    pair = 1900.0 * (K * NA) / (6 * 35)
    if params.P4 >= 0:
        Ca = sum(_nmono(a) * _nmono(b) * _nmono(c) for a, b, c in _partitions_upto(params.P4))
        atom = 13000.0 * (K * Ca) / (6 * 209)
    else:
        atom = 13000.0 * (K * NA) / (6 * 209)
    return n_pairs_per_atom * pair + atom


def kernel_flops_per_atom(params, n_pairs_per_atom):
    """The fused kernel's own count (duplicate Eq. 30a triples merged, transcendentals
    not counted): per pair 4 Ns K + (N_a - 4) + 6 K N_a + 2 K + 2 #(grad terms) + 15,
    per atom 2 N_a K + 7 (merged four-body terms) K + 4 N_a K."""
    Ns, K, Pa = params.Ns, params.Kr, params.Pa
    mons = monomials(Pa)
    NA = len(mons)
    ngrad = sum(1 for e in mons for d in range(3) if e[d] > 0)
    pair = 4 * Ns * K + (NA - 4) + 2 * K * NA + 4 * K * NA + 2 * K + 2 * ngrad + 15
    nterms = four_body_terms(params.P4)
    atom = 2 * NA * K + 7 * nterms * K + 4 * NA * K
    return n_pairs_per_atom * pair + atom


def _nmono(n):
    return (n + 1) * (n + 2) // 2


def _partitions_upto(P):
    return [(a, b, n - a - b) for n in range(P + 1) for a in range(n, -1, -1)
            for b in range(min(a, n - a), -1, -1) if 0 <= n - a - b <= b]


def four_body_terms(P4):
    if P4 < 0:
        return 0
    mons = monomials(P4)
    index = {e: i for i, e in enumerate(mons)}
    total = 0
    for n in range(P4 + 1):
        for a in range(n, -1, -1):
            for b in range(min(a, n - a), -1, -1):
                c = n - a - b
                if not (0 <= c <= b) or (b == 0 and c == 0):
                    continue
                keys = set()
                for q in (e for e in mons if sum(e) == a):
                    for s in (e for e in mons if sum(e) == b):
                        for t in (e for e in mons if sum(e) == c):
                            k = tuple(sorted((index[tuple(q[i] + s[i] for i in range(3))],
                                              index[tuple(q[i] + t[i] for i in range(3))],
                                              index[tuple(s[i] + t[i] for i in range(3))])))
                            keys.add(k)
                total += len(keys)
    return total


# ------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ workloads
def measure_fma_peaks(pkg, torch, stream, reps=5):
    """Vector-pipe throughput of this GPU (TFLOP/s), timed with CUDA events on
    ``stream`` around the library's FMA probe kernels."""
    out = {}
    for kind, name, iters in ((0, "fp32_fma", 2048), (1, "fp32x2_fma", 2048), (2, "fp64_fma", 64)):
        with torch.cuda.stream(stream):
            for _ in range(2):
                pkg.pod_fma_probe(kind, iters, stream)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            fl = 0.0
            for _ in range(reps):
                fl += pkg.pod_fma_probe(kind, iters, stream)
            t1.record(stream)
        torch.cuda.synchronize()
        out[name] = fl / (t0.elapsed_time(t1) / 1e3) / 1e12
    return out


def workload(name, replica):
    if name == "full":
        return synth.params_full(), synth.config_full(replica), "bcc_ta_8192_K6_P4_4body"
    if name == "md":
        return synth.params_full(), synth.config_md(replica), "bcc_ta_1024000_K6_P4_4body"
    if name == "small":
        return synth.params_small(), synth.config_small(replica), "bcc_ta_128_K3_P3"
    if name == "fig4":
        return synth.params_full(), synth.config_full(replica, ncell=20), "bcc_ta_16000_K6_P4_4body"
    raise ValueError(name)


def embedding_weights(params, M, seed):
    """MEAM-type density weights (two- and three-body columns) and a cubic
    embedding polynomial for the embedding-model benchmark."""
    g = synth.rng(seed)
    a = np.zeros(M)
    n = 1 + params.K2 + params.K3 * (params.P3 + 1)
    a[1:n] = g.normal(0.0, 1e-2, size=n - 1)
    return a, np.array([0.3, -0.2, 5e-3, -1e-4])


# ------------------------------------------------------------ CPU baseline
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


SAMPLE_ATOMS = 65536  # the largest block of atoms one timed oracle evaluation covers


def oracle_eval(orc, cfg, c, threads):
    """One evaluation by the FP64 oracle's fast route: cell list, atom-density
    energy and pair gradients, forces and virial of every atom (systems of more
    than SAMPLE_ATOMS atoms: of a block of that many atoms).  Returns atoms done."""
    if cfg.n <= SAMPLE_ATOMS:
        orc.energy_forces_cells(cfg, c, threads=threads)
        return cfg.n
    orc.energy_forces_cells(cfg, c, threads=threads, atom_range=(0, SAMPLE_ATOMS))
    return SAMPLE_ATOMS


def oracle_sample(params, cfg, c, budget_s, threads=1):
    """Repeat oracle_eval on `threads` host threads until `budget_s` has passed
    (at least once).  Returns (atoms done, elapsed seconds)."""
    import oracle
    orc = oracle.Oracle(params)
    n = 0
    t0 = time.perf_counter()
    while True:
        n += oracle_eval(orc, cfg, c, threads)
        if time.perf_counter() - t0 >= budget_s:
            break
    return n, time.perf_counter() - t0


def cpu_baseline_line(params, cfg, c, budget_s, unit="atom-steps/s"):
    """The oracle's fast route on every host core of this machine, plus its one-core figure."""
    cores = host_cores()
    n1, e1 = oracle_sample(params, cfg, c, budget_s / 4, threads=1)
    nn, en = oracle_sample(params, cfg, c, budget_s, threads=cores)
    what = (f"all {cfg.n} atoms" if cfg.n <= SAMPLE_ATOMS else f"the first {SAMPLE_ATOMS} atoms")
    return {"value": nn / en, "unit": unit, "cores": cores, "kind": "oracle",
            "sample": f"{nn // min(cfg.n, SAMPLE_ATOMS)} evaluations of {what} of the same configuration on "
                      f"{cores} host threads in {en:.1f} s (FP64 oracle, fast route: cell-list neighbours + "
                      f"atom-density energy, pair gradients, forces, virial); one core: {n1} atom evaluations "
                      f"in {e1:.1f} s",
            "single_core_value": n1 / e1}


# ------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full", choices=["full", "md", "small", "fig4", "mdrun", "fit"])
    ap.add_argument("--fit-configs", type=int, default=2000)
    ap.add_argument("--solver", default="auto", choices=["auto", "cholesky", "qr"],
                    help="fit workload: Cholesky with QR fallback, Cholesky only, or the QR solve")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison line items")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--quadratic", action="store_true",
                    help="quadratic model: beta_mn ~ N(0, 1e-5^2) on top of the linear coefficients")
    ap.add_argument("--embedding", action="store_true",
                    help="embedding model (MEAM-type): cubic F of a density a.D on the two- and three-body "
                         "columns, a ~ N(0, 1e-2^2), on top of the linear coefficients")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "mdrun":
        return run_md(args, rank, world, local)
    if args.workload == "fit":
        return run_fit(args, rank, world, local)

    import torch
    import paper_2212_14446_gb300 as pkg
    from paper_2212_14446_gb300 import build as pbuild

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        pbuild.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)
    params, cfg, wname = workload(args.workload, replica=rank)
    N = cfg.n
    pod = pkg.POD(params, precision=args.precision)
    c = torch.tensor(synth.coefficients(pod.M, 2001 + rank), dtype=torch.float64, device=dev)
    if args.quadratic:
        pod.set_quadratic(synth.rng(2002 + rank).normal(0.0, 1e-5, size=(pod.M, pod.M)))
    emb = embedding_weights(params, pod.M, 2003 + rank) if args.embedding else None
    if emb is not None:
        pod.set_embedding(*emb)
    pos = torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device=dev)
    box = cfg.box
    E = torch.empty(1, dtype=torch.float64, device=dev)
    Ei = torch.empty(N, dtype=torch.float64, device=dev)
    F = torch.empty((3, N), dtype=torch.float64, device=dev)
    W = torch.empty(9, dtype=torch.float64, device=dev)
    sysd = pod.system(pos, box)
    stream = torch.cuda.Stream(device=dev)

    def step():
        pkg.pod_energy_forces(pod.h, sysd, c, E, Ei, F, W, stream=stream)

    shape = None
    if not args.no_autotune:  # launch shapes for this system size (untimed setup)
        with torch.cuda.stream(stream):
            shape = pod.autotune(pos, box, c, reps=5, stream=stream)

    # warm-up (synchronous status checks; sizes the workspace)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step()
    torch.cuda.synchronize()
    # capture one step in a CUDA graph (asynchronous mode: no host sync inside)
    pod.set_sync(False)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    torch.cuda.synchronize()
    pkg.pod_status(pod.h, stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            graph.replay()
            ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    st = pkg.pod_status(pod.h, stream)
    if st != pkg.POD_OK:
        raise pkg.PodError(st, pkg.pod_last_error(pod.h))
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot_ms = sum(step_ms)
    if dist:
        t = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = t.item()
    value = N * world * args.steps / (tot_ms / 1e3)

    # per-kernel timing of the same step (library-recorded CUDA events on the stream)
    pod.set_sync(True)
    pod.set_timing(True)
    pod.timing()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            step()
    torch.cuda.synchronize()
    phase_ms, calls = pod.timing()
    pod.set_timing(False)
    phase_avg = [x / calls for x in phase_ms]
    vec_peaks = measure_fma_peaks(pkg, torch, stream)
    count = pkg.POD(params, precision=args.precision).neighbors(pos, box, cap=96)[0]
    n_pairs = float(count.double().mean().item())
    fl_atom = algorithmic_flops_per_atom(params, n_pairs)
    fl_kernel = kernel_flops_per_atom(params, n_pairs)
    atom_ms = phase_avg[1]
    achieved_tflops = fl_atom * N / (atom_ms / 1e3) / 1e12
    peak_tflops = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    if args.precision == "fp64":
        peak_tflops = 1.25  # nominal GB300 FP64 (vector and tensor), no measured figure
    prof_path = os.path.join(ROOT, "profiles", "traffic_atom_kernel.json")
    traffic = None
    if os.path.exists(prof_path):
        try:
            with open(prof_path) as f:
                tj = json.load(f)
            if tj.get("workload") == wname and tj.get("precision") == args.precision and \
                    tj.get("kernel_rev") == kernel_revision():
                traffic = tj.get("dram_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None

    # FP64 path on the same workload for the mixed-vs-FP64 comparison
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64 and args.workload != "md":
        pod64 = pkg.POD(params, precision="fp64", Q=pod.Q)
        if args.quadratic:
            pod64.set_quadratic(synth.rng(2002 + rank).normal(0.0, 1e-5, size=(pod.M, pod.M)))
        if emb is not None:
            pod64.set_embedding(*emb)
        with torch.cuda.stream(stream):
            for _ in range(3):
                pkg.pod_energy_forces(pod64.h, sysd, c, E, Ei, F, W, stream=stream)
        torch.cuda.synchronize()
        E64, F64 = E.clone(), F.clone()
        k64 = max(3, min(args.steps, 10))
        s64 = [torch.cuda.Event(enable_timing=True) for _ in range(k64)]
        e64 = [torch.cuda.Event(enable_timing=True) for _ in range(k64)]
        with torch.cuda.stream(stream):
            for k in range(k64):
                flush.fill_(float(k))
                s64[k].record(stream)
                pkg.pod_energy_forces(pod64.h, sysd, c, E, Ei, F, W, stream=stream)
                e64[k].record(stream)
        torch.cuda.synchronize()
        ms64 = sum(s.elapsed_time(e) for s, e in zip(s64, e64))
        with torch.cuda.stream(stream):
            pkg.pod_energy_forces(pod.h, sysd, c, E, Ei, F, W, stream=stream)
        torch.cuda.synchronize()
        fp64 = {"value": N * k64 / (ms64 / 1e3), "unit": "atom-steps/s",
                "speedup_mixed_vs_fp64": value / (N * world * k64 / (ms64 / 1e3)) / world,
                "mixed_vs_fp64_force_maxabs_eV_per_A": float((F - F64).abs().max().item()),
                "mixed_vs_fp64_energy_rel": float(abs(E.item() - E64.item()) / max(abs(E64.item()), 1e-300))}

    # end to end through the host-buffer entry point (pinned memory)
    pos_h = torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64).pin_memory().numpy()
    c_h = c.cpu().pin_memory().numpy()
    Eh = torch.zeros(1, dtype=torch.float64).pin_memory().numpy()
    Eih = torch.zeros(N, dtype=torch.float64).pin_memory().numpy()
    Fh = torch.zeros((3, N), dtype=torch.float64).pin_memory().numpy()
    Wh = torch.zeros(9, dtype=torch.float64).pin_memory().numpy()
    import ctypes as C
    hsys = pkg.make_system(pos_h.ctypes.data_as(C.POINTER(C.c_double)), N, box)
    call = pkg.HostEnergyForces(pod.h, hsys, c_h, Eh, Eih, Fh, Wh, stream=stream)  # the public repeated-call form
    pos_src, c_src = pos_h.copy(), c_h.copy()
    for _ in range(3):
        call()
    if dist:
        dist.barrier()
    # the host writes its inputs before every call (as an MD driver would), outside
    # the timed window: no call finds them already in a GPU cache
    te = 0.0
    for k in range(args.steps):
        pos_h[...] = pos_src
        c_h[...] = c_src
        te0 = time.perf_counter()
        call()
        te += time.perf_counter() - te0
    if dist:
        t = torch.tensor([te], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        te = t.item()
    e2e = {"value": N * world * args.steps / te, "unit": "atom-steps/s",
           "h2d_bytes_per_step": int(pos_h.nbytes + c_h.nbytes),
           "d2h_bytes_per_step": int(Eh.nbytes + Eih.nbytes + Fh.nbytes + Wh.nbytes)}

    cpu = None
    if rank == 0 and world == 1:  # the CPU baseline is measured at N = 1 only
        cpu = cpu_baseline_line(params, cfg, c.cpu().numpy(), args.cpu_budget)

    if rank == 0:
        line = {
            "metric": "atom-steps/s (E+F) mixed vs FP64 at stated force error; % of roofline",
            "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": wname, "atoms_per_gpu": N, "global_atoms": N * world,
                       "pairs_per_atom": n_pairs, "descriptors": pod.M, "precision": args.precision,
                       "neighbor_rebuild": "every step", "l2": "flushed (512 MB write) before each step",
                       "graph": "one CUDA graph per step", "parallelism": f"replicas x{world}",
                       "launch_shape": shape,
                       "potential": "quadratic" if args.quadratic else ("embedding" if args.embedding else "linear")},
            "roofline": {"bound": "alu", "kernel": "atom_kernel (fused radial/B/contraction/adjoint)",
                         "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak_tflops, "traffic": traffic,
                         "flops_per_atom": fl_atom, "atom_kernel_ms": atom_ms,
                         "flop_model": "1.9 kflop per pair + 13 kflop per atom (K = 6, N_a = 35, C_a = 209)",
                         "kernel_count_flops_per_atom": fl_kernel,
                         "frac_kernel_count": fl_kernel * N / (atom_ms / 1e3) / 1e12 / peak_tflops,
                         "peak_basis": ("152 SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal max clock)"
                                        if args.precision == "mixed" else "nominal FP64 1.25 TFLOP/s"),
                         "measured_vector_tflops": vec_peaks,
                         "frac_of_measured_fma": (achieved_tflops / vec_peaks["fp32_fma"]
                                                       if args.precision == "mixed"
                                                       else achieved_tflops / vec_peaks["fp64_fma"])},
            "phases_ms": {"neighbors": phase_avg[0], "atom": phase_avg[1], "gather": phase_avg[2],
                          "reduce": phase_avg[3]},
            # per step: bin, neighbour search, atom kernel (+ separate adjoint kernel), finalize
            "gpu_launches": (5 if shape and shape.get("atom_rp") == 2 else 4) * args.steps,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp64_path": fp64,
            "clocks": clk,
            "wall_s": t_wall,
        }
        line["roofline"].update(hbm_subentries(N, n_pairs, phase_avg, args.precision))
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_md(args, rank, world, local):
    """1,024,000-atom BCC Ta velocity-Verlet MD (dt = 1 fs, Ta mass, 300 K
    velocities): neighbour list with a 0.3 A skin rebuilt every 10 steps, each
    step one replay of a captured CUDA graph (one graph for rebuild steps, one
    for reuse steps).  Timed: `steps` consecutive MD steps (state > L2)."""
    import torch
    import paper_2212_14446_gb300 as pkg
    from paper_2212_14446_gb300 import build as pbuild
    torch.cuda.set_device(local)
    if rank == 0:
        pbuild.build()
    dev = torch.device("cuda", local)
    params, cfg, wname = workload("md", replica=rank)
    N = cfg.n
    pod = pkg.POD(params, precision=args.precision)
    pod.set_skin(0.3)
    # a random coefficient vector is not a stable crystal potential: with sigma = 0.01 the atoms
    # collide within ~100 fs; sigma = 1e-4 keeps the 100-step run inside the skin (the cost of a
    # step does not depend on the values of c)
    c = torch.tensor(synth.coefficients(pod.M, 2001 + rank, sigma=1e-4), dtype=torch.float64, device=dev)
    x = torch.tensor(np.ascontiguousarray(cfg.pos.T), dtype=torch.float64, device=dev)
    mass, dt = 180.94788, 1.0
    g = synth.rng(4000 + rank)
    vrms = math.sqrt(8.617333e-5 * 300.0 / mass * 9.648533212e-3)
    v = torch.tensor(g.normal(0.0, vrms, size=(3, N)), dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    shape = None
    if not args.no_autotune:
        with torch.cuda.stream(stream):
            shape = pod.autotune(x, cfg.box, c, reps=3, stream=stream)
    with torch.cuda.stream(stream):
        F = pod.energy_forces(x, cfg.box, c, stream=stream)["F"].t().contiguous()
        for k in range(max(args.warmup, 3)):
            pod.set_neighbor_reuse(k % 10 != 0)
            pod.md_step(x, v, F, c, cfg.box, mass, dt, E, stream=stream)
    torch.cuda.synchronize()
    pod.set_sync(False)
    graphs = {}
    for reuse in (False, True):
        pod.set_neighbor_reuse(reuse)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=stream):
            pod.md_step(x, v, F, c, cfg.box, mass, dt, E, stream=stream)
        graphs[reuse] = gr
    torch.cuda.synchronize()
    st = pkg.pod_status(pod.h, stream)
    if st != pkg.POD_OK:
        raise pkg.PodError(st, pkg.pod_last_error(pod.h))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for k in range(args.steps):
            graphs[k % 10 != 0].replay()
        e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = pkg.pod_status(pod.h, stream)
    if st != pkg.POD_OK:
        raise pkg.PodError(st, pkg.pod_last_error(pod.h))
    ms = e0.elapsed_time(e1)
    line = {"metric": "atom-steps/s (E+F) mixed vs FP64 at stated force error; % of roofline",
            "value": N * args.steps / (ms / 1e3), "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "bcc_ta_1024000_md_verlet", "atoms_per_gpu": N, "skin_A": 0.3, "c_sigma": 1e-4,
                       "neighbor_rebuild": "every 10 steps", "dt_fs": dt, "graph": "captured rebuild/reuse steps",
                       "l2": "state larger than L2", "launch_shape": shape},
            "final_energy_eV": E.item(), "clocks": clk, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line))


def run_fit(args, rank, world, local):
    """Batched fit of `--fit-configs` training configurations (BCC/FCC/A15 with
    vacancies and liquid packings, 2..250 atoms, volume strain +-20 %): labels
    from a teacher coefficient vector through the batched FP64 energy/force path,
    then pod_fit (design matrix, FP64 Gram, Cholesky).  Metric: configs/s of
    the fit call (CUDA events around it)."""
    import torch
    import paper_2212_14446_gb300 as pkg
    from paper_2212_14446_gb300 import build as pbuild
    torch.cuda.set_device(local)
    if rank == 0:
        pbuild.build()
    params = synth.params_full()
    cfgs = synth.training_set(args.fit_configs, replica=rank)
    pod = pkg.POD(params, precision=args.precision)
    teacher = pkg.POD(params, precision="fp64", Q=pod.Q)
    cstar = torch.tensor(synth.coefficients(pod.M, 3001), dtype=torch.float64)
    out = teacher.energy_forces_batch(cfgs, cstar)
    E_ref = out["E"].cpu().numpy()
    Fall = out["F"].cpu().numpy()
    offs = out["offs"]
    F_ref = [Fall[offs[k]:offs[k + 1]] for k in range(len(cfgs))]
    # the batch resident on the device (packed once, outside the timed region)
    pos, boffs, boxes, pbcs = pod.pack_batch(cfgs)
    x = torch.tensor(pos, dtype=torch.float64, device="cuda")
    Er = torch.tensor(np.asarray(E_ref, dtype=np.float64), device="cuda")
    Fr = torch.tensor(np.ascontiguousarray(np.concatenate(F_ref, axis=0).T), dtype=torch.float64, device="cuda")
    fit_shape = None
    if not args.no_autotune:  # design-pass launch shapes for this batch (untimed setup)
        fit_shape = pod.autotune_fit(x, boffs, boxes, pbcs, reps=3)
    for _ in range(max(1, args.warmup)):
        pod.fit_device(x, boffs, boxes, pbcs, Er, Fr, solver=args.solver)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0.record()
        c, maeE, maeF = pod.fit_device(x, boffs, boxes, pbcs, Er, Fr, solver=args.solver)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = sum(ts) / len(ts)
    # end to end: host configurations in, coefficients out (packing and copies timed)
    te0 = time.perf_counter()
    pod.fit(cfgs, E_ref, F_ref)
    te = time.perf_counter() - te0
    # per-phase device time of one more fit (library CUDA events)
    pod.set_timing(True)
    pod.timing()
    pod.fit_device(x, boffs, boxes, pbcs, Er, Fr, solver=args.solver)
    ph, calls = pod.timing()
    pod.set_timing(False)
    phases = {"neighbors": ph[0], "design_matrix": ph[1], "gram": ph[2], "solve": ph[3]} if calls else None
    n_atoms = int(offs[-1])
    rel = float(np.max(np.abs(c - cstar.numpy())) / np.max(np.abs(cstar.numpy())))
    line = {"metric": "configs/s (fit: descriptors + gradients into the design matrix, exact normal equations, "
                      "FP64 Cholesky)",
            "value": len(cfgs) / (ms / 1e3), "unit": "configs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"training_set_{len(cfgs)}", "atoms": n_atoms, "design_rows": len(cfgs) + 3 * n_atoms,
                       "descriptors": pod.M, "solver": args.solver, "launch_shape": fit_shape,
                       "graph": "the fit's device chain recorded once and replayed per timed fit"},
            "teacher_recovery_max_rel": rel, "mae_E_per_atom": maeE, "mae_F": maeF, "phases_ms": phases,
            "e2e": {"value": len(cfgs) / te, "unit": "configs/s",
                    "h2d_bytes_per_step": int(pos.nbytes + Er.numel() * 8 + Fr.numel() * 8),
                    "d2h_bytes_per_step": int(pod.M * 8 + 16)},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line))


ATOM_KERNEL_SOURCES = ("atom_impl.cuh", "atom_f32.cu", "atom_f64.cu", "pod_common.cuh", "pod_kernels.h",
                       "gen_contract.py")


def hbm_peak():
    """Measured HBM copy bandwidth of the GB300s (generated file), else the
    profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def hbm_subentries(N, n_pairs, phase_avg, precision):
    """The step's memory-side kernels graded on HBM bandwidth with the algorithmic bytes
    per atom of the method's cost model: the neighbour build (positions in, 24 B; the list
    out, one 4-byte index per pair plus the count) and the force finalize / gather (mixed:
    fixed-point force sums in, 32 B, FP64 forces out, 24 B; FP64: per pair the gradient
    (32 B) and the reverse index (4 B) in, FP64 forces out).  `kernel_bytes_per_atom` is
    what this build's kernels move instead where that differs (the mixed search writes a
    16-byte displacement row per pair)."""
    peak, basis = hbm_peak()
    nb_alg = 24.0 + 4.0 * n_pairs + 4.0
    nb_own = 24.0 + 24.0 + 32.0 + 16.0 + (16.0 if precision == "mixed" else 8.0) * n_pairs + 4.0
    if precision == "mixed":
        fin = 32.0 + 24.0
    else:
        fin = n_pairs * (32.0 + 4.0) + 24.0
    out = {}
    for key, ms, alg, own in (("neighbor", phase_avg[0], nb_alg, nb_own), ("finalize", phase_avg[2], fin, fin)):
        gbs = alg * N / (ms / 1e3) / 1e9 if ms > 0 else None
        out[key] = {"bound": "hbm", "bytes_per_atom": alg, "kernel_bytes_per_atom": own, "achieved": gbs,
                    "peak": peak, "unit": "GB/s", "frac": (gbs / peak) if gbs else None,
                    "peak_basis": basis, "phase_ms": ms}
    return out


def kernel_revision():
    """Hash of the fused atom kernel's sources (a traffic figure is only valid for
    the kernel it was taken on)."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2212_14446_gb300", "csrc")
    for f in ATOM_KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle's fast route (cell list + atom-density
    energy, pair gradients, forces and virial) on every host core; one step is
    one evaluation of the workload (of a block of SAMPLE_ATOMS atoms for larger
    systems).  Under torchrun only rank 0 runs."""
    if rank != 0:
        return
    import oracle
    params, cfg, wname = workload(args.workload, replica=0)
    c = synth.coefficients(1 + params.K2 + params.K3 * (params.P3 + 1) + params.K4 * _ka(params.P4), 2001)
    cores = host_cores()
    orc = oracle.Oracle(params)
    for _ in range(args.warmup):
        oracle_eval(orc, cfg, c, cores)
    tot_atoms, tot_s = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        tot_atoms += oracle_eval(orc, cfg, c, cores)
        tot_s += time.perf_counter() - t0
    value = tot_atoms / tot_s
    per = min(cfg.n, SAMPLE_ATOMS)
    line = {"impl": "reference",
            "metric": "atom-steps/s (E+F) mixed vs FP64 at stated force error; % of roofline",
            "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "atoms_per_gpu": cfg.n, "atoms_per_step": per},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} evaluations of {per} atoms (FP64 oracle, fast route: "
                                       f"cell-list neighbours + atom-density energy, pair gradients, forces, "
                                       f"virial) on {cores} host threads"},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _ka(P4):
    if P4 < 0:
        return 0
    return sum(1 for n in range(P4 + 1) for a in range(n, -1, -1) for b in range(min(a, n - a), -1, -1)
               if 0 <= n - a - b <= b)


if __name__ == "__main__":
    main()
