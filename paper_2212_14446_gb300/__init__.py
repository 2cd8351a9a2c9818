"""Python binding of the fastpod C ABI (``include/pod.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``_lib/libfastpod.so``; PyTorch provides device memory and streams.
The module fails loudly when the library has not been built -- there is no CPU
fallback.

Low-level functions carry the C names (``pod_create``, ``pod_descriptors``,
``pod_energy_forces``, ``pod_energy_forces_host``, ``pod_neighbors``,
``pod_fit``, ...).  :class:`POD` wraps a handle for convenience.

Layouts: positions and forces are structure-of-arrays ``(3, N)`` float64 on
the device; descriptors are ``(N, M)`` float64 (order in ``include/pod.h``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfastpod.so")

POD_OK, POD_EINVAL, POD_ENOMEM, POD_ECUDA, POD_ERANGE, POD_ENONFINITE, POD_ESINGULAR, POD_ENEIGH = (
    0, -1, -2, -3, -4, -5, -6, -7)
POD_EIO = -8
POD_FP64, POD_MIXED = 0, 1
POD_OPT_SYNC, POD_OPT_PRECISION, POD_OPT_TIMING, POD_OPT_RADIAL, POD_OPT_NEIGHBOR_REUSE = 1, 2, 3, 4, 5
POD_OPT_DESCRIPTORS = 6
POD_OPT_GRAM = 7
POD_OPT_ADJOINT = 8
POD_OPT_NEIGHBOR_TESTS = 9
POD_OPT_FIT_GRAPH = 10
POD_OPT_HOST_MAPPED = 11
POD_OPT_WORKSPACE_LIMIT_MB = 12
POD_EMB_MAX_DEGREE = 8
ERROR_NAMES = {0: "POD_OK", -1: "POD_EINVAL", -2: "POD_ENOMEM", -3: "POD_ECUDA", -4: "POD_ERANGE",
               -5: "POD_ENONFINITE", -6: "POD_ESINGULAR", -7: "POD_ENEIGH", -8: "POD_EIO"}


class PodError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class pod_params(C.Structure):
    _fields_ = [("r_in", C.c_double), ("r_cut", C.c_double),
                ("n_alpha", C.c_int), ("alpha", C.POINTER(C.c_double)),
                ("n_beta", C.c_int), ("beta", C.POINTER(C.c_double)),
                ("n_gamma", C.c_int), ("gamma", C.POINTER(C.c_double)),
                ("K2", C.c_int), ("K3", C.c_int), ("K4", C.c_int), ("P3", C.c_int), ("P4", C.c_int),
                ("n_grid", C.c_int), ("precision", C.c_int), ("Q", C.POINTER(C.c_double))]


class pod_system(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("pos", C.POINTER(C.c_double)),
                ("box", C.c_double * 3), ("pbc", C.c_int * 3),
                ("n_configs", C.c_int), ("atom_offs", C.POINTER(C.c_int)),
                ("boxes", C.POINTER(C.c_double)), ("pbcs", C.POINTER(C.c_int)), ("n_local", C.c_int)]


_SOLVERS = {"auto": 0, "cholesky": 1, "qr": 2}


class pod_fit_opts(C.Structure):
    _fields_ = [("w_E", C.c_double), ("w_F", C.c_double), ("gamma_reg", C.c_double),
                ("per_atom_energy", C.c_int), ("solver", C.c_int)]


EXPORTS = ["pod_create", "pod_destroy", "pod_info", "pod_set_option", "pod_status", "pod_timing",
           "pod_neighbors", "pod_descriptors", "pod_energy_forces", "pod_energy_forces_host", "pod_fit",
           "pod_fit_normal", "pod_fit_solve", "pod_fit_residual", "pod_fit_replays", "pod_descriptors_static",
           "pod_global_descriptors", "pod_descriptors_jvp", "pod_set_skin", "pod_md_step", "pod_fma_probe", "pod_autotune", "pod_set_quadratic",
           "pod_set_embedding", "pod_save", "pod_load", "pod_selftest_wait", "pod_halo_select", "pod_halo_add",
           "pod_descriptors_tangent", "pod_model_gradients", "pod_last_error"]

_lib = None
_lock = threading.Lock()


def lib():
    """Load ``libfastpod.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"fastpod CUDA library not built ({LIB_PATH}); run "
                                   "paper_2212_14446_gb300.build.build() first")
            L = C.CDLL(LIB_PATH)
            H = C.c_void_p
            dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
            S = C.POINTER(pod_system)
            sig = {
                "pod_create": (C.c_int, [C.POINTER(pod_params), C.POINTER(H)]),
                "pod_destroy": (C.c_int, [H]),
                "pod_info": (C.c_int, [H, ip, ip, ip, dp, dp]),
                "pod_set_option": (C.c_int, [H, C.c_int, C.c_int]),
                "pod_status": (C.c_int, [H, vp]),
                "pod_timing": (C.c_int, [H, dp, ip]),
                "pod_neighbors": (C.c_int, [H, S, C.c_int, ip, ip, ip, vp]),
                "pod_descriptors": (C.c_int, [H, S, dp, vp]),
                "pod_descriptors_static": (C.c_int, [H, S, dp, vp]),
                "pod_global_descriptors": (C.c_int, [H, S, dp, vp]),
                "pod_descriptors_jvp": (C.c_int, [H, S, dp, dp, vp]),
                "pod_set_skin": (C.c_int, [H, C.c_double]),
                "pod_md_step": (C.c_int, [H, S, dp, dp, dp, dp, C.c_double, C.c_double, dp, vp]),
                "pod_energy_forces": (C.c_int, [H, S, dp, dp, dp, dp, dp, vp]),
                "pod_energy_forces_host": (C.c_int, [H, S, vp, vp, vp, vp, vp, vp]),
                "pod_fit": (C.c_int, [H, S, dp, dp, C.POINTER(pod_fit_opts), dp, dp, dp]),
                "pod_fit_normal": (C.c_int, [H, S, dp, dp, C.POINTER(pod_fit_opts), dp, dp]),
                "pod_fit_solve": (C.c_int, [H, dp, dp, dp]),
                "pod_fit_residual": (C.c_int, [H, dp, dp, dp, ip, ip]),
                "pod_fma_probe": (C.c_int, [C.c_int, C.c_int, dp, vp]),
                "pod_selftest_wait": (C.c_int, [C.c_longlong, C.POINTER(C.c_int)]),
                "pod_autotune": (C.c_int, [H, S, dp, C.c_int, ip, dp, vp]),
                "pod_set_quadratic": (C.c_int, [H, dp]),
                "pod_set_embedding": (C.c_int, [H, dp, C.c_int, dp]),
                "pod_save": (C.c_int, [H, C.c_char_p, dp]),
                "pod_load": (C.c_int, [C.c_char_p, C.c_int, C.POINTER(H), dp, C.c_int, ip]),
                "pod_halo_select": (C.c_int, [H, dp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_int, ip, dp, ip, vp]),
                "pod_halo_add": (C.c_int, [H, dp, ip, C.c_int, dp, C.c_int, vp]),
                "pod_descriptors_tangent": (C.c_int, [H, S, dp, dp, vp]),
                "pod_model_gradients": (C.c_int, [H, C.c_int, dp, dp, dp, C.c_double, dp, vp]),
                "pod_fit_replays": (C.c_int, [H, ip]),
                "pod_last_error": (C.c_char_p, [H]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


# ------------------------------------------------------------- thin C names

def pod_create(params: pod_params):
    h = C.c_void_p()
    rc = lib().pod_create(C.byref(params), C.byref(h))
    if rc != POD_OK:
        msg = lib().pod_last_error(h).decode() if h.value else ""
        if h.value:
            lib().pod_destroy(h)
        raise PodError(rc, msg or "pod_create failed")
    return h


def pod_destroy(h):
    return lib().pod_destroy(h)


def pod_last_error(h) -> str:
    return lib().pod_last_error(h).decode()


def pod_selftest_wait(limit_ns: int) -> int:
    """Run the bounded-wait self-test (a wait on a barrier nothing arrives at,
    limit ``limit_ns`` ns); returns the status bits it reported (64 = ST_TIMEOUT)."""
    st = C.c_int(0)
    rc = lib().pod_selftest_wait(int(limit_ns), C.byref(st))
    if rc != POD_OK:
        raise PodError(rc, "pod_selftest_wait failed")
    return st.value


def pod_fma_probe(kind: int, iters: int, stream=None) -> float:
    """Launch the vector-pipe throughput probe on ``stream`` (kind 0 FP32 FMA,
    1 FP32 paired FMA, 2 FP64 FMA); returns the launch's flop count."""
    fl = C.c_double(0.0)
    rc = lib().pod_fma_probe(int(kind), int(iters), C.byref(fl), _stream(stream))
    if rc != POD_OK:
        raise PodError(rc, "pod_fma_probe failed")
    return fl.value


def _check(h, rc):
    if rc != POD_OK:
        raise PodError(rc, pod_last_error(h))


def _dptr(t):
    if t is None:
        return None
    return C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double))


def _iptr(t):
    if t is None:
        return None
    return C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_int))


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_system(pos_ptr, n_atoms, box, pbc=(1, 1, 1), batch=None, n_local=0):
    s = pod_system()
    s.n_atoms = int(n_atoms)
    s.n_local = int(n_local)
    s.pos = pos_ptr
    s.box = (C.c_double * 3)(*[float(b) for b in box])
    s.pbc = (C.c_int * 3)(*[int(p) for p in pbc])
    s.n_configs = 0
    keep = []
    if batch is not None:
        offs, boxes, pbcs = batch
        offs = np.ascontiguousarray(offs, dtype=np.int32)
        boxes = np.ascontiguousarray(boxes, dtype=np.float64)
        s.n_configs = len(offs) - 1
        s.atom_offs = offs.ctypes.data_as(C.POINTER(C.c_int))
        s.boxes = boxes.ctypes.data_as(C.POINTER(C.c_double))
        keep += [offs, boxes]
        if pbcs is not None:
            pbcs = np.ascontiguousarray(pbcs, dtype=np.int32)
            s.pbcs = pbcs.ctypes.data_as(C.POINTER(C.c_int))
            keep.append(pbcs)
    s._keep = keep
    return s


def pod_descriptors(h, sys, D, stream=None):
    _check(h, lib().pod_descriptors(h, C.byref(sys), _dptr(D), _stream(stream)))


def pod_descriptors_static(h, sys, D, stream=None):
    """Descriptors of one configuration (<= 4096 atoms) without any allocation."""
    _check(h, lib().pod_descriptors_static(h, C.byref(sys), _dptr(D), _stream(stream)))


def pod_halo_select(h, pos, axis, L, x0, x1, shift, offset, cap, idx, out, stream=None):
    """Atoms of pos (device (3, N)) whose wrapped coordinate along `axis` lies in
    [x0, x1), ascending: idx (device int32 [cap]) and out (device (3, cap)) the
    positions with that coordinate moved to x + shift - offset.  Returns the count."""
    n = C.c_int(0)
    _check(h, lib().pod_halo_select(h, _dptr(pos), int(pos.shape[1]), int(axis), float(L), float(x0), float(x1),
                                    float(shift), float(offset), int(cap), _iptr(idx), _dptr(out), C.byref(n),
                                    _stream(stream)))
    return n.value


def pod_halo_add(h, G, idx, n, F, stream=None):
    """F[:, idx[k]] += G[:, k] for k < n (device tensors; F (3, N), G (3, n))."""
    _check(h, lib().pod_halo_add(h, _dptr(G), _iptr(idx), int(n), _dptr(F), int(F.shape[1]), _stream(stream)))


def pod_descriptors_tangent(h, sys, v, Ddot, stream=None):
    """Per-atom Ddot[i] = sum_k (dD_i/dr_k) . v_k (v device (3, N), Ddot device (N, M))."""
    _check(h, lib().pod_descriptors_tangent(h, C.byref(sys), _dptr(v), _dptr(Ddot), _stream(stream)))


def pod_model_gradients(h, D, Ddot, w, t, n_out, stream=None):
    """Loss gradient of the handle's current model (see include/pod.h); returns a
    numpy array of n_out values."""
    g = np.zeros(n_out)
    _check(h, lib().pod_model_gradients(h, int(D.shape[0]), _dptr(D), _dptr(Ddot), _dptr(w), float(t),
                                        g.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
    return g


def pod_energy_forces(h, sys, c, E, Ei=None, F=None, W=None, stream=None):
    _check(h, lib().pod_energy_forces(h, C.byref(sys), _dptr(c), _dptr(E), _dptr(Ei), _dptr(F), _dptr(W),
                                      _stream(stream)))


def pod_autotune(h, sys, c, reps=5, stream=None):
    """Returns ([neigh wpb, atom wpb, gather wpb, gather blocks per SM, adjoint form
    (0 fused, 1 fused with R' staged, 2 separate kernel), neighbour tests (1
    block-wide, 0 warp per atom)], [ms neigh, atom, gather])."""
    shape = (C.c_int * 6)()
    ms = (C.c_double * 3)()
    _check(h, lib().pod_autotune(h, C.byref(sys), _dptr(c), int(reps), shape, ms, _stream(stream)))
    return list(shape), list(ms)


def pod_energy_forces_host(h, sys, c, E, Ei=None, F=None, W=None, stream=None):
    """Host float64 arrays (C-contiguous) in and out; the addresses are passed as is."""
    def hp(a):
        return None if a is None else a.ctypes.data
    _check(h, lib().pod_energy_forces_host(h, C.byref(sys), hp(c), hp(E), hp(Ei), hp(F), hp(W),
                                           _stream(stream)))


class HostEnergyForces:
    """pod_energy_forces_host on fixed host arrays, called repeatedly (an MD driver,
    a benchmark): the pointers and the stream are marshalled once, so each call
    costs one foreign call.  The arrays and `sys` must stay alive and in place."""

    def __init__(self, h, sys, c, E, Ei=None, F=None, W=None, stream=None):
        def hp(a):
            return C.c_void_p(None if a is None else a.ctypes.data)
        self.h = h
        self._keep = (sys, c, E, Ei, F, W, stream)
        self._fn = lib().pod_energy_forces_host
        self._args = (h, C.byref(sys), hp(c), hp(E), hp(Ei), hp(F), hp(W), _stream(stream))

    def __call__(self):
        rc = self._fn(*self._args)
        if rc != POD_OK:
            raise PodError(rc, pod_last_error(self.h))


def pod_neighbors(h, sys, cap, count, nbr, shift, stream=None):
    _check(h, lib().pod_neighbors(h, C.byref(sys), int(cap), _iptr(count), _iptr(nbr), _iptr(shift),
                                  _stream(stream)))


def pod_status(h, stream=None):
    return lib().pod_status(h, _stream(stream))


def pod_set_option(h, option, value):
    _check(h, lib().pod_set_option(h, int(option), int(value)))


def pod_timing(h):
    """(per-phase totals in ms [neighbours, atom kernel, gather, reduce], calls); resets."""
    ms = np.zeros(4)
    calls = C.c_int()
    _check(h, lib().pod_timing(h, ms.ctypes.data_as(C.POINTER(C.c_double)), C.byref(calls)))
    return ms, calls.value


# ----------------------------------------------------------------- wrapper

def _param_struct(params, precision, Q=None, n_grid=None):
    alpha = np.ascontiguousarray(params.alpha, dtype=np.float64)
    beta = np.ascontiguousarray(params.beta, dtype=np.float64)
    gamma = np.ascontiguousarray(params.gamma, dtype=np.float64)
    p = pod_params()
    p.r_in, p.r_cut = float(params.r_in), float(params.r_cut)
    p.n_alpha, p.alpha = len(alpha), alpha.ctypes.data_as(C.POINTER(C.c_double))
    p.n_beta, p.beta = len(beta), beta.ctypes.data_as(C.POINTER(C.c_double))
    p.n_gamma, p.gamma = len(gamma), gamma.ctypes.data_as(C.POINTER(C.c_double))
    p.K2, p.K3, p.K4, p.P3, p.P4 = (int(params.K2), int(params.K3), int(params.K4), int(params.P3),
                                    int(params.P4))
    p.n_grid = int(n_grid if n_grid is not None else getattr(params, "n_grid", 2000))
    p.precision = POD_MIXED if precision in ("mixed", POD_MIXED) else POD_FP64
    keep = [alpha, beta, gamma]
    if Q is not None:
        Qa = np.ascontiguousarray(Q, dtype=np.float64)
        p.Q = Qa.ctypes.data_as(C.POINTER(C.c_double))
        keep.append(Qa)
    p._keep = keep
    return p


def _soa(pos):
    """(N, 3) or (3, N) float64 CUDA tensor -> contiguous (3, N)."""
    import torch
    if pos.dim() != 2:
        raise ValueError("positions must be 2-D")
    if pos.shape[0] == 3 and pos.shape[1] != 3:
        t = pos
    elif pos.shape[1] == 3:
        t = pos.t()
    else:
        t = pos
    return t.to(dtype=torch.float64).contiguous()


class POD:
    """A fastpod handle bound to one parameter set.

    ``params`` is any object with attributes r_in, r_cut, alpha, beta, gamma,
    K2, K3, K4, P3, P4 (and optionally n_grid)."""

    def __init__(self, params, precision="fp64", Q=None, n_grid=None):
        self._p = _param_struct(params, precision, Q, n_grid)
        self.h = pod_create(self._p)
        self._read_info(precision)

    def _read_info(self, precision):
        M, Ns, K = C.c_int(), C.c_int(), C.c_int()
        _check(self.h, lib().pod_info(self.h, C.byref(M), C.byref(Ns), C.byref(K), None, None))
        self.M, self.Ns, self.K = M.value, Ns.value, K.value
        Qo = np.zeros((self.Ns, self.K))
        eig = np.zeros(self.Ns)
        _check(self.h, lib().pod_info(self.h, None, None, None, Qo.ctypes.data_as(C.POINTER(C.c_double)),
                                      eig.ctypes.data_as(C.POINTER(C.c_double))))
        self.Q, self.eig = Qo, eig
        self.precision = precision

    def save(self, path, c=None):
        """Model file: parameters, Q and (optionally) the coefficients c (M,)."""
        cp = None
        if c is not None:
            cv = np.ascontiguousarray(np.asarray(c.cpu() if hasattr(c, "cpu") else c, dtype=np.float64))
            if cv.shape != (self.M,):
                raise ValueError(f"c must be ({self.M},)")
            cp = cv.ctypes.data_as(C.POINTER(C.c_double))
        _check(self.h, lib().pod_save(self.h, os.fsencode(path), cp))

    @classmethod
    def load(cls, path, precision="fp64"):
        """Handle from a model file; returns (pod, c or None)."""
        h = C.c_void_p()
        c = np.zeros(4096)
        n = C.c_int(0)
        prec = POD_MIXED if precision in ("mixed", POD_MIXED) else POD_FP64
        rc = lib().pod_load(os.fsencode(path), prec, C.byref(h), c.ctypes.data_as(C.POINTER(C.c_double)), c.size,
                            C.byref(n))
        if rc != POD_OK:
            msg = pod_last_error(h.value) if h.value else f"cannot load {path}"
            if h.value:
                pod_destroy(h.value)
            raise PodError(rc, msg)
        obj = cls.__new__(cls)
        obj._p = None
        obj.h = h.value
        obj._read_info(precision)
        return obj, (c[: n.value].copy() if n.value else None)

    def close(self):
        if getattr(self, "h", None):
            pod_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision):
        pod_set_option(self.h, POD_OPT_PRECISION, POD_MIXED if precision in ("mixed", POD_MIXED) else POD_FP64)
        self.precision = precision

    def set_sync(self, on: bool):
        pod_set_option(self.h, POD_OPT_SYNC, 1 if on else 0)

    def set_radial(self, mode: str):
        """Mixed path: 'table' (default) or 'direct' radial evaluation."""
        pod_set_option(self.h, POD_OPT_RADIAL, 0 if mode == "table" else 1)

    def set_skin(self, skin: float):
        _check(self.h, lib().pod_set_skin(self.h, float(skin)))

    def set_neighbor_reuse(self, on: bool):
        pod_set_option(self.h, POD_OPT_NEIGHBOR_REUSE, 1 if on else 0)

    def set_descriptor_set(self, which: str):
        """Three-body columns: 'fast' (default, the fast POD sums of Eq. 26a) or
        'exclusive' (the original POD sums over pairs k > j, Eq. 15b)."""
        if which not in ("fast", "exclusive"):
            raise ValueError("descriptor set must be 'fast' or 'exclusive'")
        pod_set_option(self.h, POD_OPT_DESCRIPTORS, 1 if which == "exclusive" else 0)

    def md_step(self, pos_soa, v, F, c, box, mass, dt, E, pbc=(1, 1, 1), stream=None):
        """One velocity-Verlet step; pos_soa, v, F: (3, N) float64 CUDA tensors updated in place."""
        sysd = self.system(pos_soa, box, pbc)
        _check(self.h, lib().pod_md_step(self.h, C.byref(sysd), _dptr(pos_soa), _dptr(v), _dptr(F), _dptr(c),
                                         float(mass), float(dt), _dptr(E), _stream(stream)))

    def set_timing(self, on: bool):
        pod_set_option(self.h, POD_OPT_TIMING, 1 if on else 0)

    def set_adjoint_kernel(self, which: str):
        """Mixed linear path: "auto" (launch shape / size), "fused" or "separate"."""
        pod_set_option(self.h, POD_OPT_ADJOINT, {"auto": -1, "fused": 0, "separate": 1}[which])

    def set_neighbor_tests(self, which: str):
        """Neighbour search candidate tests: "auto" (launch shape / size),
        "blockwide" or "warp"."""
        pod_set_option(self.h, POD_OPT_NEIGHBOR_TESTS, {"auto": -1, "warp": 0, "blockwide": 1}[which])

    def autotune_fit(self, pos_soa, offs, boxes, pbcs, reps=3, stream=None):
        """Tune the fit's design pass on a device batch (pod_autotune with a batch);
        returns {"atom_wpb", "design_wpb", "ms"}."""
        shape, ms = pod_autotune(self.h, self.batch_system(pos_soa, offs, boxes, pbcs), None, reps, stream)
        return {"atom_wpb": shape[1], "design_wpb": shape[2], "ms": ms[1]}

    def set_workspace_limit_mb(self, mb: int):
        """Cap the handle's device workspace at mb MiB (0: no cap); growth past it
        raises PodError(POD_ENOMEM)."""
        pod_set_option(self.h, POD_OPT_WORKSPACE_LIMIT_MB, int(mb))

    def set_host_mapped(self, on: bool):
        """pod_energy_forces_host graph replays: kernels read and write mapped pinned
        host buffers directly (default on) or through copies."""
        pod_set_option(self.h, POD_OPT_HOST_MAPPED, 1 if on else 0)

    def set_fit_graph(self, on: bool):
        """pod_fit: record the fit's device chain and replay it on repeated calls (default on)."""
        pod_set_option(self.h, POD_OPT_FIT_GRAPH, 1 if on else 0)

    def fit_replays(self):
        """Number of pod_fit calls on this handle served by a recorded fit."""
        n = C.c_int(0)
        _check(self.h, lib().pod_fit_replays(self.h, C.byref(n)))
        return n.value

    def timing(self):
        return pod_timing(self.h)

    def system(self, pos_soa, box, pbc=(1, 1, 1), n_local=0):
        return make_system(_dptr(pos_soa), pos_soa.shape[1], box, pbc, n_local=n_local)

    def neighbors(self, pos, box, pbc=(1, 1, 1), cap=64, stream=None):
        import torch
        x = _soa(pos)
        n = x.shape[1]
        count = torch.zeros(n, dtype=torch.int32, device=x.device)
        nbr = torch.full((n, cap), -1, dtype=torch.int32, device=x.device)
        shift = torch.zeros((n, cap, 3), dtype=torch.int32, device=x.device)
        pod_neighbors(self.h, self.system(x, box, pbc), cap, count, nbr, shift, stream)
        return count, nbr, shift

    def descriptors(self, pos, box, pbc=(1, 1, 1), stream=None):
        import torch
        x = _soa(pos)
        D = torch.empty((x.shape[1], self.M), dtype=torch.float64, device=x.device)
        pod_descriptors(self.h, self.system(x, box, pbc), D, stream)
        return D

    def global_descriptors(self, pos, box, pbc=(1, 1, 1), stream=None):
        """G_m = sum_i D_im (Eq. 58a): (1, M) float64."""
        import torch
        x = _soa(pos)
        G = torch.empty((1, self.M), dtype=torch.float64, device=x.device)
        _check(self.h, lib().pod_global_descriptors(self.h, C.byref(self.system(x, box, pbc)), _dptr(G),
                                                    _stream(stream)))
        return G

    def descriptors_jvp(self, pos, box, v, pbc=(1, 1, 1), stream=None):
        """sum_k dG_m/dr_k . v_k for per-atom directions v ((N, 3) or (3, N)): (1, M)."""
        import torch
        x = _soa(pos)
        vv = _soa(v)
        Gd = torch.empty((1, self.M), dtype=torch.float64, device=x.device)
        _check(self.h, lib().pod_descriptors_jvp(self.h, C.byref(self.system(x, box, pbc)), _dptr(vv), _dptr(Gd),
                                                 _stream(stream)))
        return Gd

    def energy_forces(self, pos, box, c, pbc=(1, 1, 1), atom_energies=True, forces=True, virial=True,
                      stream=None, n_local=0):
        """E, E_i, F, W.  n_local > 0: atoms [0, n_local) are local and the rest
        ghosts (forces on all atoms, energies and virial of the local terms)."""
        import torch
        x = _soa(pos)
        n = x.shape[1]
        dev = x.device
        c = c.to(device=dev, dtype=torch.float64).contiguous()
        E = torch.empty(1, dtype=torch.float64, device=dev)
        Ei = torch.empty(n, dtype=torch.float64, device=dev) if atom_energies else None
        F = torch.empty((3, n), dtype=torch.float64, device=dev) if forces else None
        W = torch.empty(9, dtype=torch.float64, device=dev) if virial else None
        pod_energy_forces(self.h, self.system(x, box, pbc, n_local), c, E, Ei, F, W, stream)
        return {"E": E, "Ei": Ei, "F": None if F is None else F.t(), "W": None if W is None else W.view(3, 3)}

    def set_quadratic(self, beta=None):
        """Quadratic model E_i = c.D_i + sum_{m<=n} beta_mn D_im D_in (beta: (M, M), upper
        triangle read), or None for the linear model."""
        if beta is None:
            _check(self.h, lib().pod_set_quadratic(self.h, None))
            return
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
        if b.shape != (self.M, self.M):
            raise ValueError(f"beta must be ({self.M}, {self.M})")
        _check(self.h, lib().pod_set_quadratic(self.h, b.ctypes.data_as(C.POINTER(C.c_double))))

    def set_embedding(self, a=None, alpha=None):
        """Embedding model E_i = c.D_i + F(a.D_i), F(rho) = sum_k alpha[k] rho^k (a: (M,),
        alpha: (degree + 1,), 1 <= degree <= 8), or a=None for the linear model."""
        if a is None:
            _check(self.h, lib().pod_set_embedding(self.h, None, 0, None))
            return
        av = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
        if av.shape != (self.M,):
            raise ValueError(f"a must be ({self.M},)")
        if al.ndim != 1 or al.size < 2:
            raise ValueError("alpha must hold degree + 1 >= 2 coefficients")
        _check(self.h, lib().pod_set_embedding(self.h, av.ctypes.data_as(C.POINTER(C.c_double)), al.size - 1,
                                               al.ctypes.data_as(C.POINTER(C.c_double))))

    def autotune(self, pos, box, c, pbc=(1, 1, 1), reps=5, stream=None):
        """Pick the launch shape for this system size (pod_autotune); returns
        {"neigh_wpb", "atom_wpb", "gather_wpb", "gather_bps", "atom_rp", "neigh_blockwide",
        "ms": [neigh, atom, gather]}."""
        import torch
        x = _soa(pos)
        c = c.to(device=x.device, dtype=torch.float64).contiguous()
        shape, ms = pod_autotune(self.h, self.system(x, box, pbc), c, reps, stream)
        return {"neigh_wpb": shape[0], "atom_wpb": shape[1], "gather_wpb": shape[2], "gather_bps": shape[3],
                "atom_rp": shape[4], "neigh_blockwide": shape[5], "ms": ms}

    # -- batches of configurations --------------------------------------
    @staticmethod
    def pack_batch(configs):
        """Concatenate configurations: (pos SoA (3, N), atom_offs, boxes, pbcs)."""
        offs = np.zeros(len(configs) + 1, dtype=np.int32)
        for k, cf in enumerate(configs):
            offs[k + 1] = offs[k] + cf.pos.shape[0]
        pos = np.ascontiguousarray(np.concatenate([cf.pos for cf in configs], axis=0).T)
        boxes = np.array([cf.box for cf in configs], dtype=np.float64)
        pbcs = np.array([cf.pbc for cf in configs], dtype=np.int32)
        return pos, offs, boxes, pbcs

    def batch_system(self, pos_soa, offs, boxes, pbcs):
        return make_system(_dptr(pos_soa), pos_soa.shape[1], boxes[0], (1, 1, 1), batch=(offs, boxes, pbcs))

    def descriptors_batch(self, configs, stream=None):
        import torch
        pos, offs, boxes, pbcs = self.pack_batch(configs)
        x = torch.tensor(pos, dtype=torch.float64, device="cuda")
        D = torch.empty((x.shape[1], self.M), dtype=torch.float64, device=x.device)
        pod_descriptors(self.h, self.batch_system(x, offs, boxes, pbcs), D, stream)
        return D

    def energy_forces_batch(self, configs, c, stream=None):
        import torch
        pos, offs, boxes, pbcs = self.pack_batch(configs)
        x = torch.tensor(pos, dtype=torch.float64, device="cuda")
        n = x.shape[1]
        c = c.to(device=x.device, dtype=torch.float64).contiguous()
        E = torch.empty(len(configs), dtype=torch.float64, device=x.device)
        Ei = torch.empty(n, dtype=torch.float64, device=x.device)
        F = torch.empty((3, n), dtype=torch.float64, device=x.device)
        pod_energy_forces(self.h, self.batch_system(x, offs, boxes, pbcs), c, E, Ei, F, None, stream)
        return {"E": E, "Ei": Ei, "F": F.t(), "offs": offs}

    def fit(self, configs, E_ref, F_ref, w_E=100.0, w_F=1.0, gamma=1e-12, per_atom_energy=True, solver="auto"):
        """Ridge least-squares fit (Eq. 63a) on the GPU.  E_ref: (n_cfg,), F_ref: list of
        (N_c, 3) arrays; solver: "auto" (Cholesky, QR when a pivot is not positive),
        "cholesky" or "qr".  Returns (c, mae_E per atom, mae_F per component)."""
        import torch
        pos, offs, boxes, pbcs = self.pack_batch(configs)
        x = torch.tensor(pos, dtype=torch.float64, device="cuda")
        Er = torch.tensor(np.asarray(E_ref, dtype=np.float64), device=x.device)
        Fr = torch.tensor(np.ascontiguousarray(np.concatenate([np.asarray(f) for f in F_ref], axis=0).T),
                          dtype=torch.float64, device=x.device)
        o = pod_fit_opts(float(w_E), float(w_F), float(gamma), 1 if per_atom_energy else 0, _SOLVERS[solver])
        c = np.zeros(self.M)
        mE, mF = C.c_double(), C.c_double()
        sysb = self.batch_system(x, offs, boxes, pbcs)
        _check(self.h, lib().pod_fit(self.h, C.byref(sysb), _dptr(Er), _dptr(Fr), C.byref(o),
                                     c.ctypes.data_as(C.POINTER(C.c_double)), C.byref(mE), C.byref(mF)))
        return c, mE.value, mF.value

    def fit_device(self, pos_soa, offs, boxes, pbcs, E_ref, F_ref, w_E=100.0, w_F=1.0, gamma=1e-12,
                   per_atom_energy=True, solver="auto"):
        """pod_fit on a batch already on the device (pos_soa (3, N), E_ref (n_cfg,), F_ref (3, N)
        CUDA float64 tensors; offs/boxes/pbcs host arrays from pack_batch)."""
        o = pod_fit_opts(float(w_E), float(w_F), float(gamma), 1 if per_atom_energy else 0, _SOLVERS[solver])
        c = np.zeros(self.M)
        mE, mF = C.c_double(), C.c_double()
        sysb = self.batch_system(pos_soa, offs, boxes, pbcs)
        _check(self.h, lib().pod_fit(self.h, C.byref(sysb), _dptr(E_ref), _dptr(F_ref), C.byref(o),
                                     c.ctypes.data_as(C.POINTER(C.c_double)), C.byref(mE), C.byref(mF)))
        return c, mE.value, mF.value

    def fit_normal(self, configs, E_ref, F_ref, w_E=100.0, w_F=1.0, gamma=1e-12, per_atom_energy=True):
        """Normal equations (G = A^T A + gamma I, r = A^T b) of this batch; A stays
        on the device for fit_residual."""
        import torch
        pos, offs, boxes, pbcs = self.pack_batch(configs)
        x = torch.tensor(pos, dtype=torch.float64, device="cuda")
        Er = torch.tensor(np.asarray(E_ref, dtype=np.float64), device=x.device)
        Fr = torch.tensor(np.ascontiguousarray(np.concatenate([np.asarray(f) for f in F_ref], axis=0).T),
                          dtype=torch.float64, device=x.device)
        o = pod_fit_opts(float(w_E), float(w_F), float(gamma), 1 if per_atom_energy else 0, 0)
        G = np.zeros((self.M, self.M))
        r = np.zeros(self.M)
        sysb = self.batch_system(x, offs, boxes, pbcs)
        _check(self.h, lib().pod_fit_normal(self.h, C.byref(sysb), _dptr(Er), _dptr(Fr), C.byref(o),
                                            G.ctypes.data_as(C.POINTER(C.c_double)),
                                            r.ctypes.data_as(C.POINTER(C.c_double))))
        return G, r

    def fit_solve(self, G, r):
        G = np.ascontiguousarray(G, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        c = np.zeros(self.M)
        _check(self.h, lib().pod_fit_solve(self.h, G.ctypes.data_as(C.POINTER(C.c_double)),
                                           r.ctypes.data_as(C.POINTER(C.c_double)),
                                           c.ctypes.data_as(C.POINTER(C.c_double))))
        return c

    def fit_residual(self, c):
        """(sum |dE| per atom over energy rows, sum |dF| over force rows, n_E, n_F) of the last batch."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        se, sf = C.c_double(), C.c_double()
        ne, nf = C.c_int(), C.c_int()
        _check(self.h, lib().pod_fit_residual(self.h, c.ctypes.data_as(C.POINTER(C.c_double)), C.byref(se),
                                              C.byref(sf), C.byref(ne), C.byref(nf)))
        return se.value, sf.value, ne.value, nf.value

    def energy_forces_host(self, pos_soa: np.ndarray, box, c: np.ndarray, pbc=(1, 1, 1), stream=None):
        """Host-buffer entry point: numpy in, numpy out (copies inside the call)."""
        pos_soa = np.ascontiguousarray(pos_soa, dtype=np.float64)
        n = pos_soa.shape[1]
        E = np.zeros(1)
        F = np.zeros((3, n))
        W = np.zeros(9)
        Ei = np.zeros(n)
        sys = make_system(pos_soa.ctypes.data_as(C.POINTER(C.c_double)), n, box, pbc)
        pod_energy_forces_host(self.h, sys, np.ascontiguousarray(c, dtype=np.float64), E, Ei, F, W, stream)
        return {"E": E, "Ei": Ei, "F": F.T, "W": W.reshape(3, 3)}
