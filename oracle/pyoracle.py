"""ctypes wrapper of the CPU oracle (aw_oracle.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It builds the
oracle with gcc on first use (``-ffp-contract=off`` so that x86 and Arm hosts
round identically) into ``oracle/_build``.
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
_lock = threading.Lock()
_lib = None

ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "BAD_MESH", -3: "NONPHYSICAL", -4: "DEADLOCK", -7: "STATE"}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "aw_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [("order_M", C.c_int), ("gamma", C.c_double), ("cfl", C.c_double),
                ("time_quantum_log2", C.c_int), ("t_end", C.c_double), ("gts", C.c_int),
                ("predictor_iters", C.c_int), ("mesh_velocity", C.c_int), ("flux", C.c_int),
                ("wall_u", C.c_double), ("wall_v", C.c_double), ("t_switch", C.c_double),
                ("cfl_start", C.c_double), ("kidder", C.c_double * 5)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
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
            _lib = lib
    return _lib


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
                 cfl_start=0.0, kidder=(0.9, 1.0, 1.0, 2.0, 1.0)):
        self.lib = _load()
        cfg = _Config(order_M, gamma, cfl, time_quantum_log2, t_end, int(gts), predictor_iters, int(eulerian),
                      {"rusanov": 0, "osher": 1}[flux], float(wall_velocity[0]), float(wall_velocity[1]),
                      float(t_switch), float(cfl_start), (C.c_double * 5)(*[float(v) for v in kidder]))
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
