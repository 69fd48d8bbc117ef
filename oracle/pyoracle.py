"""ctypes wrapper of the CPU oracle (aw_oracle.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It builds the
oracle with gcc on first use (``-ffp-contract=off`` so that x86 and Arm hosts
round identically) into ``oracle/_build``, together with its two C++ builds
over the same source (``oc_scalar.hpp``): the tangent-linear one
(``TangentOracle``: every double a (value, tangent) pair) and the
operation-counting one (``Oracle(kind="count")``, ``flop_counts``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libaw_oracle.so")
_SRC = os.path.join(_HERE, "aw_oracle.c")
_VARIANTS = {"tlm": ("aw_oracle_tlm.cpp", "libaw_oracle_tlm.so"),
             "count": ("aw_oracle_count.cpp", "libaw_oracle_count.so")}
_lock = threading.Lock()
_lib = None
_libs = {}

# phases of the operation counts (oc_scalar.hpp)
PHASES = ("other", "nodes", "flux", "update", "recon", "dt", "predictor")

ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "BAD_MESH", -3: "NONPHYSICAL", -4: "DEADLOCK", -7: "STATE"}


class _Dual(C.Structure):
    _fields_ = [("v", C.c_double), ("d", C.c_double)]


class _ConfigDual(C.Structure):
    """oc_config of the tangent-linear build: every double a (value, tangent)."""
    _fields_ = [("order_M", C.c_int), ("gamma", _Dual), ("cfl", _Dual), ("time_quantum_log2", C.c_int),
                ("t_end", _Dual), ("gts", C.c_int), ("predictor_iters", C.c_int), ("mesh_velocity", C.c_int),
                ("flux", C.c_int), ("wall_u", _Dual), ("wall_v", _Dual), ("t_switch", _Dual),
                ("cfl_start", _Dual), ("kidder", _Dual * 5)]


def _stale(lib, srcs):
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(p) for p in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, gcc) and its two C++
    builds (tangent-linear, operation counting); return the plain one."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "aw_oracle.h")
    jobs = []
    if force or _stale(_LIB, [_SRC, hdr]):
        jobs.append((_LIB, ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
                            "-o", None, _SRC, "-lm"]))
    for src, lib in _VARIANTS.values():
        lib, src = os.path.join(_BUILD, lib), os.path.join(_HERE, src)
        if force or _stale(lib, [src, _SRC, hdr, os.path.join(_HERE, "oc_scalar.hpp")]):
            jobs.append((lib, ["g++", "-O2", "-std=c++17", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-w", "-o", None, src, "-lm"]))
    procs = []
    for lib, cmd in jobs:
        tmp = lib + f".{os.getpid()}.tmp"
        cmd[cmd.index(None)] = tmp
        procs.append((subprocess.Popen(cmd), tmp, lib))
    for p, tmp, lib in procs:
        if p.wait() != 0:
            raise RuntimeError(f"building {lib} failed")
        os.replace(tmp, lib)
    return _LIB


class _Config(C.Structure):
    _fields_ = [("order_M", C.c_int), ("gamma", C.c_double), ("cfl", C.c_double),
                ("time_quantum_log2", C.c_int), ("t_end", C.c_double), ("gts", C.c_int),
                ("predictor_iters", C.c_int), ("mesh_velocity", C.c_int), ("flux", C.c_int),
                ("wall_u", C.c_double), ("wall_v", C.c_double), ("t_switch", C.c_double),
                ("cfl_start", C.c_double), ("kidder", C.c_double * 5)]


def _load(kind="plain"):
    global _lib
    with _lock:
        if kind in _libs:
            return _libs[kind]
        if kind == "plain" or kind not in _VARIANTS:
            lib = C.CDLL(build())
        else:
            build()
            lib = C.CDLL(os.path.join(_BUILD, _VARIANTS[kind][1]))
        if True:
            P = C.c_void_p
            lib.oc_create.argtypes = [C.POINTER(_Config), C.POINTER(P)]
            lib.oc_destroy.argtypes = [P]
            lib.oc_last_error.argtypes = [P]
            lib.oc_last_error.restype = C.c_char_p
            lib.oc_load_mesh.argtypes = [P, C.c_int64, P, C.c_int64, P, P, P, P]
            lib.oc_load_state.argtypes = [P, P]
            lib.oc_load_state_xy.argtypes = [P, P, P]
            lib.oc_schedule.argtypes = [P, C.c_int, C.c_int64]
            lib.oc_get_schedule.argtypes = [P, P]
            lib.oc_set_schedule.argtypes = [P, C.c_int64, P]
            lib.oc_sweep.argtypes = [P, C.POINTER(C.c_int64)]
            lib.oc_advance_to.argtypes = [P, C.c_double, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            lib.oc_get_elem.argtypes = [P] + [P] * 8
            lib.oc_set_elem.argtypes = [P] + [P] * 8
            lib.oc_get_nodes.argtypes = [P, P, P]
            lib.oc_set_nodes.argtypes = [P, P, P]
            lib.oc_n_st.argtypes = [P]
            lib.oc_n_st.restype = C.c_int64
            lib.oc_n_edges.argtypes = [P]
            lib.oc_n_edges.restype = C.c_int64
            lib.oc_diag.argtypes = [P, P]
            lib.oc_get_stencils.argtypes = [P, C.c_int64, P, P, C.c_int]
            lib.oc_reconstruct_eval.argtypes = [P, C.c_int64, C.c_int64, P, P]
            lib.oc_predict_debug.argtypes = [P, P, C.c_double, P, P]
            lib.oc_flux_debug.argtypes = [P, P, P, P, C.c_int, P]
            lib.oc_eval_qh.argtypes = [P, P, C.c_int64, P, P]
            lib.oc_table.argtypes = [P, C.c_int, C.c_int64, P, P]
            if kind == "count":
                lib.oc_count_read.argtypes = [P]
                lib.oc_count_reset.argtypes = []
            if kind == "tlm":
                lib.oc_create.argtypes = [C.POINTER(_ConfigDual), C.POINTER(P)]
                lib.oc_advance_to.argtypes = [P, _Dual, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
                lib.oc_predict_debug.argtypes = [P, P, _Dual, P, P]
            if kind == "plain":
                _lib = lib
            _libs[kind] = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Oracle:
    """One oracle context (a mesh, a state and a configuration)."""

    def __init__(self, order_M=1, gamma=1.4, cfl=0.5, t_end=0.2, time_quantum_log2=20, gts=False,
                 predictor_iters=0, eulerian=False, flux="rusanov", wall_velocity=(0.0, 0.0), t_switch=0.0,
                 cfl_start=0.0, kidder=(0.9, 1.0, 1.0, 2.0, 1.0), kind="plain"):
        """kind: "plain" (the C build) or "count" (the operation-counting
        build, same arrays; see flop_counts)."""
        self.lib = _load(kind)
        self.kind = kind
        args = (order_M, gamma, cfl, time_quantum_log2, t_end, int(gts), predictor_iters, int(eulerian),
                {"rusanov": 0, "osher": 1}[flux], float(wall_velocity[0]), float(wall_velocity[1]),
                float(t_switch), float(cfl_start))
        if kind == "tlm":
            d = lambda x: _Dual(float(x), 0.0)  # noqa: E731
            a = list(args)
            for k in (1, 2, 4, 9, 10, 11, 12):
                a[k] = d(a[k])
            cfg = _ConfigDual(*a, (_Dual * 5)(*[d(v) for v in kidder]))
        else:
            cfg = _Config(*args, (C.c_double * 5)(*[float(v) for v in kidder]))
        h = C.c_void_p()
        rc = self.lib.oc_create(C.byref(cfg), C.byref(h))
        if rc:
            raise OracleError(rc, "oc_create")
        self.h = h
        self.M = order_M
        self.Mc = (order_M + 1) * (order_M + 2) // 2
        self.Nt = order_M + 1
        self.Nst = self.Mc * self.Nt
        self.gamma = gamma
        self.t_end = t_end
        self.K = time_quantum_log2
        self.tick = t_end / 2.0 ** time_quantum_log2
        self.n_tris = 0
        self.n_nodes = 0

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.oc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise OracleError(rc, self.lib.oc_last_error(self.h).decode())

    def load_mesh(self, mesh):
        xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        bc = np.ascontiguousarray(mesh["bc"], dtype=np.int8)
        shift = None if mesh.get("shift") is None else np.ascontiguousarray(mesh["shift"], dtype=np.int8)
        period = None if mesh.get("period") is None else np.ascontiguousarray(mesh["period"], dtype=np.float64)
        self._keep = (xy, tri, bc, shift, period)
        self._check(self.lib.oc_load_mesh(self.h, xy.shape[0], _ptr(xy), tri.shape[0], _ptr(tri), _ptr(bc),
                                          _ptr(shift), _ptr(period)))
        self.n_tris = tri.shape[0]
        self.n_nodes = xy.shape[0]

    def load_state(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        self._check(self.lib.oc_load_state(self.h, _ptr(Q)))

    def load_state_xy(self, Q, xy):
        """Initial state on moved node positions; the mesh pre-processing
        (stencils, total stencils, wall normals) stays that of load_mesh."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._check(self.lib.oc_load_state_xy(self.h, _ptr(Q), _ptr(xy)))

    def schedule(self, mode, k=0):
        """Frozen schedule: mode "record" logs the dt ticks of each element's
        first k updates, "replay" reuses them, "free" returns to CFL steps."""
        m = {"free": 0, "record": 1, "replay": 2}[mode]
        self._check(self.lib.oc_schedule(self.h, m, k))
        if m == 1:
            self._sched_k = k

    def get_schedule(self):
        out = np.empty((self.n_tris, self._sched_k), np.int64)
        self._check(self.lib.oc_get_schedule(self.h, _ptr(out)))
        return out

    def set_schedule(self, log):
        """Load a schedule log [n_tris][k]; schedule(2) then replays it."""
        log = np.ascontiguousarray(log, dtype=np.int64)
        self._check(self.lib.oc_set_schedule(self.h, log.shape[1], _ptr(log)))
        self._sched_k = log.shape[1]

    def sweep(self):
        n = C.c_int64(0)
        self._check(self.lib.oc_sweep(self.h, C.byref(n)))
        return n.value

    def advance(self, max_sweeps=10 ** 9):
        total, sweeps = 0, 0
        while sweeps < max_sweeps:
            n = self.sweep()
            if n == 0:
                break
            total += n
            sweeps += 1
        return sweeps, total

    def advance_to(self, t, max_sweeps=10 ** 9):
        """Sweeps until every element reached the sync time t (t_end or a
        whole number of ticks; reading R18); returns (sweeps, updates)."""
        ns, nu = C.c_int64(0), C.c_int64(0)
        self._check(self.lib.oc_advance_to(self.h, float(t), int(max_sweeps), C.byref(ns), C.byref(nu)))
        return ns.value, nu.value

    def get_elem(self):
        n, Nst = self.n_tris, self.Nst
        out = dict(Q=np.empty((n, 4)), QM=np.empty((n, 4)), HM=np.empty((n, 3)), t=np.empty(n, np.int64),
                   dt=np.empty(n, np.int64), X=np.empty((n, 6)), count=np.empty(n, np.int64),
                   qhat=np.empty((n, Nst, 4)))
        self._check(self.lib.oc_get_elem(self.h, *[_ptr(out[k]) for k in
                                                    ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")]))
        return out

    def set_elem(self, st):
        arrs = [np.ascontiguousarray(st[k], dtype=np.int64 if k in ("t", "dt", "count") else np.float64)
                for k in ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")]
        self._check(self.lib.oc_set_elem(self.h, *[_ptr(a) for a in arrs]))

    def get_nodes(self):
        X = np.empty((self.n_nodes, 2))
        t = np.empty(self.n_nodes, np.int64)
        self._check(self.lib.oc_get_nodes(self.h, _ptr(X), _ptr(t)))
        return X, t

    def set_nodes(self, X, t):
        X = np.ascontiguousarray(X, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.int64)
        self._check(self.lib.oc_set_nodes(self.h, _ptr(X), _ptr(t)))

    def diag(self):
        out = np.zeros(2)
        self._check(self.lib.oc_diag(self.h, _ptr(out)))
        return dict(gcl_max=out[0], gcl_checked=out[1])

    def n_edges(self):
        return self.lib.oc_n_edges(self.h)

    def stencils(self, i):
        mem = np.empty((7, 2 * self.Mc), np.int32)
        sw = np.empty(4096, np.int32)
        n = self.lib.oc_get_stencils(self.h, i, _ptr(mem), _ptr(sw), 4096)
        if n < 0:
            self._check(n)
        return mem, sw[:n].copy()

    def reconstruct_eval(self, i, xy):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        out = np.empty((xy.shape[0], 4))
        self._check(self.lib.oc_reconstruct_eval(self.h, i, xy.shape[0], _ptr(xy), _ptr(out)))
        return out

    def predict(self, X6, dt_sec, w_nodal):
        X6 = np.ascontiguousarray(X6, dtype=np.float64)
        w = np.ascontiguousarray(w_nodal, dtype=np.float64)
        out = np.empty((self.Nst, 4))
        self._check(self.lib.oc_predict_debug(self.h, _ptr(X6), float(dt_sec), _ptr(w), _ptr(out)))
        return out

    def flux(self, qL, qR, n3, bc=-1):
        qL = np.ascontiguousarray(qL, dtype=np.float64)
        qR = None if qR is None else np.ascontiguousarray(qR, dtype=np.float64)
        n3 = np.ascontiguousarray(n3, dtype=np.float64)
        out = np.empty(4)
        self._check(self.lib.oc_flux_debug(self.h, _ptr(qL), _ptr(qR), _ptr(n3), bc, _ptr(out)))
        return out

    def eval_qh(self, qhat, pts):
        qhat = np.ascontiguousarray(qhat, dtype=np.float64)
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        out = np.empty((pts.shape[0], 4))
        self._check(self.lib.oc_eval_qh(self.h, _ptr(qhat), pts.shape[0], _ptr(pts), _ptr(out)))
        return out

    def table(self, what, pts=None, npts=0):
        Mc, Nt = self.Mc, self.Nt
        if pts is not None:
            pts = np.ascontiguousarray(pts, dtype=np.float64)
            npts = pts.shape[0]
        shape = {0: (npts, Mc), 1: (Mc, Mc), 2: (Nt,), 3: (Nt, Nt), 4: (Nt, Nt), 5: (Mc, 2), 6: (2, npts),
                 7: (npts, Mc)}[what]
        out = np.empty(shape)
        self._check(self.lib.oc_table(self.h, what, npts, _ptr(pts), _ptr(out)))
        return out


def _pair(value, tangent=None):
    """[..., 2] array of (value, tangent) pairs: the dual layout."""
    v = np.asarray(value, dtype=np.float64)
    out = np.zeros(v.shape + (2,))
    out[..., 0] = v
    if tangent is not None:
        out[..., 1] = tangent
    return out


class TangentOracle(Oracle):
    """The tangent-linear build: the oracle's arithmetic on (value, tangent)
    pairs.  load_state_xy with seeded tangents, then sweeps, give the
    directional derivative of every output; values equal the plain build's
    bit for bit."""

    def __init__(self, **cfg):
        super().__init__(kind="tlm", **cfg)

    def load_mesh(self, mesh):
        xy = _pair(mesh["xy"])
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        bc = np.ascontiguousarray(mesh["bc"], dtype=np.int8)
        shift = None if mesh.get("shift") is None else np.ascontiguousarray(mesh["shift"], dtype=np.int8)
        period = None if mesh.get("period") is None else _pair(mesh["period"])
        self._keep = (xy, tri, bc, shift, period)
        self._check(self.lib.oc_load_mesh(self.h, tri.max() + 1 if False else mesh["xy"].shape[0], _ptr(xy),
                                          tri.shape[0], _ptr(tri), _ptr(bc), _ptr(shift), _ptr(period)))
        self.n_tris = tri.shape[0]
        self.n_nodes = mesh["xy"].shape[0]

    def load_state_xy(self, Q, xy, dQ=None, dxy=None):
        """Averages Q [n][4] and node positions xy [n_nodes][2] with the
        tangents dQ, dxy (zero if None)."""
        q, x = _pair(Q, dQ), _pair(xy, dxy)
        self._check(self.lib.oc_load_state_xy(self.h, _ptr(q), _ptr(x)))

    def load_state(self, Q, dQ=None):
        q = _pair(Q, dQ)
        self._check(self.lib.oc_load_state(self.h, _ptr(q)))

    def advance_to(self, t, max_sweeps=10 ** 9):
        ns, nu = C.c_int64(0), C.c_int64(0)
        self._check(self.lib.oc_advance_to(self.h, _Dual(float(t), 0.0), int(max_sweeps), C.byref(ns), C.byref(nu)))
        return ns.value, nu.value

    def get_elem(self):
        """(values, tangents): two dicts of the element arrays (integer
        arrays only in the first)."""
        n, Nst = self.n_tris, self.Nst
        out = dict(Q=np.empty((n, 4, 2)), QM=np.empty((n, 4, 2)), HM=np.empty((n, 3, 2)), t=np.empty(n, np.int64),
                   dt=np.empty(n, np.int64), X=np.empty((n, 6, 2)), count=np.empty(n, np.int64),
                   qhat=np.empty((n, Nst, 4, 2)))
        self._check(self.lib.oc_get_elem(self.h, *[_ptr(out[k]) for k in
                                                    ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")]))
        val = {k: (v[..., 0] if v.dtype == np.float64 else v) for k, v in out.items()}
        tan = {k: v[..., 1] for k, v in out.items() if v.dtype == np.float64}
        return val, tan

    def get_nodes(self):
        X = np.empty((self.n_nodes, 2, 2))
        t = np.empty(self.n_nodes, np.int64)
        self._check(self.lib.oc_get_nodes(self.h, _ptr(X), _ptr(t)))
        return X[..., 0], X[..., 1], t

    def set_elem(self, st):
        raise NotImplementedError("the tangent-linear build starts from load_state / load_state_xy")


def flop_counts(oracle):
    """Floating-point operations counted so far by an Oracle(kind="count"),
    by phase (PHASES)."""
    out = np.zeros(len(PHASES), np.int64)
    oracle.lib.oc_count_read(out.ctypes.data_as(C.c_void_p))
    return dict(zip(PHASES, out.tolist()))


def flop_reset(oracle):
    oracle.lib.oc_count_reset()
