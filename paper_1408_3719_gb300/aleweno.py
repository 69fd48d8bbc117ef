"""ctypes binding of the C ABI in ``include/aleweno.h`` (argument marshalling
only: every step of the scheme runs in the CUDA library).

``load()`` opens ``_build/libaleweno.so`` and raises if it is missing; there
is no CPU fallback.  ``Solver`` mirrors the C entry points.  Arrays may be
numpy arrays (host) or CUDA torch tensors (device); the library copies with
unified addressing, so both work.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libaleweno.so")

AW_ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "BAD_MESH", -3: "NONPHYSICAL", -4: "DEADLOCK", -5: "TIMEOUT",
             -6: "CUDA", -7: "STATE"}

EXPORTED = ["aw_create", "aw_destroy", "aw_last_error", "aw_load_mesh", "aw_load_batch", "aw_load_state",
            "aw_lts_sweep",
            "aw_gts_step", "aw_advance_to", "aw_enqueue_sweeps", "aw_sync", "aw_get_state", "aw_get_nodes",
            "aw_get_update_counts", "aw_get_elem_arrays", "aw_set_elem_arrays", "aw_get_node_arrays",
            "aw_set_node_arrays", "aw_diagnostics", "aw_sizes", "aw_profile_enable", "aw_profile_read",
            "aw_kernel_name", "aw_ready_set_noalloc", "aw_measure_fp64_peak", "aw_load_state_xy", "aw_schedule",
            "aw_get_schedule", "aw_adjoint_forward", "aw_adjoint", "aw_adjoint_selftest", "aw_set_tiles",
            "aw_get_tiles", "aw_autotune"]

_lock = threading.Lock()
_lib = None


class AwConfig(C.Structure):
    _fields_ = [("order_M", C.c_int), ("gamma", C.c_double), ("cfl", C.c_double),
                ("time_quantum_log2", C.c_int), ("t_end", C.c_double), ("gts", C.c_int),
                ("predictor_iters", C.c_int), ("mesh_velocity", C.c_int), ("cuda_stream", C.c_void_p),
                ("flux", C.c_int), ("wall_u", C.c_double), ("wall_v", C.c_double),
                ("t_switch", C.c_double), ("cfl_start", C.c_double), ("kidder", C.c_double * 5)]


class AwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{AW_ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Open the CUDA library (build it first with paper_1408_3719_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
            lib = C.CDLL(p)
            P = C.c_void_p
            i64 = C.c_int64
            lib.aw_create.argtypes = [C.POINTER(AwConfig), C.POINTER(P)]
            lib.aw_destroy.argtypes = [P]
            lib.aw_destroy.restype = None
            lib.aw_last_error.argtypes = [P]
            lib.aw_last_error.restype = C.c_char_p
            lib.aw_load_mesh.argtypes = [P, i64, P, i64, P, P, P, P]
            lib.aw_load_batch.argtypes = [P, C.c_int, P, P, P, P, P, P]
            lib.aw_load_state.argtypes = [P, P]
            lib.aw_lts_sweep.argtypes = [P, C.POINTER(i64)]
            lib.aw_gts_step.argtypes = [P, C.POINTER(i64)]
            lib.aw_advance_to.argtypes = [P, C.c_double, i64, C.POINTER(i64), C.POINTER(i64)]
            lib.aw_enqueue_sweeps.argtypes = [P, i64]
            lib.aw_sync.argtypes = [P, C.POINTER(i64)]
            lib.aw_get_state.argtypes = [P, P, P]
            lib.aw_get_nodes.argtypes = [P, P, P]
            lib.aw_get_update_counts.argtypes = [P, P, C.POINTER(i64)]
            lib.aw_get_elem_arrays.argtypes = [P] + [P] * 8
            lib.aw_set_elem_arrays.argtypes = [P] + [P] * 8
            lib.aw_get_node_arrays.argtypes = [P, P, P]
            lib.aw_set_node_arrays.argtypes = [P, P, P]
            lib.aw_diagnostics.argtypes = [P, P]
            lib.aw_sizes.argtypes = [P, P]
            lib.aw_profile_enable.argtypes = [P, C.c_int]
            lib.aw_profile_read.argtypes = [P, P, C.POINTER(i64)]
            lib.aw_kernel_name.argtypes = [C.c_int]
            lib.aw_kernel_name.restype = C.c_char_p
            lib.aw_ready_set_noalloc.argtypes = [P, P, P]
            lib.aw_measure_fp64_peak.argtypes = [C.POINTER(C.c_double)]
            lib.aw_load_state_xy.argtypes = [P, P, P]
            lib.aw_schedule.argtypes = [P, C.c_int, i64]
            lib.aw_get_schedule.argtypes = [P, P]
            lib.aw_adjoint_forward.argtypes = [P, i64, i64]
            lib.aw_adjoint.argtypes = [P, P, P, P, P, P]
            lib.aw_adjoint_selftest.argtypes = [C.c_int, C.c_uint64, P]
            lib.aw_set_tiles.argtypes = [P, P]
            lib.aw_get_tiles.argtypes = [P, P]
            lib.aw_autotune.argtypes = [P, i64, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor (host or device)
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def fp64_peak_gflops() -> float:
    v = C.c_double(0.0)
    rc = load().aw_measure_fp64_peak(C.byref(v))
    if rc:
        raise AwError(rc, "aw_measure_fp64_peak")
    return v.value


def adjoint_selftest(order_M: int, seed: int = 1):
    """Largest relative mismatch of each element-level reverse (reconstruction,
    predictor, edge flux, node solver) against central differences of its
    forward, computed on the host (no GPU needed)."""
    r = np.zeros(4)
    rc = load().aw_adjoint_selftest(order_M, seed, _ptr(r))
    if rc:
        raise AwError(rc, "aw_adjoint_selftest")
    return dict(recon=r[0], predictor=r[1], edge=r[2], node=r[3])


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _arr(a, dtype):
    """numpy arrays are made contiguous in dtype; torch tensors (host,
    pinned or device) pass as they are (the caller gives the layout)."""
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


class Solver:
    """One GPU context: mesh, LTS state and configuration."""

    def __init__(self, order_M=1, gamma=1.4, cfl=0.5, t_end=0.2, time_quantum_log2=20, gts=False,
                 predictor_iters=0, eulerian=False, stream=None, flux="rusanov", wall_velocity=(0.0, 0.0),
                 t_switch=0.0, cfl_start=0.0, kidder=(0.9, 1.0, 1.0, 2.0, 1.0)):
        self.lib = load()
        cfg = AwConfig(order_M, gamma, cfl, time_quantum_log2, t_end, int(gts), predictor_iters, int(eulerian),
                       stream, {"rusanov": 0, "osher": 1}[flux], float(wall_velocity[0]), float(wall_velocity[1]),
                       float(t_switch), float(cfl_start), (C.c_double * 5)(*[float(v) for v in kidder]))
        h = C.c_void_p()
        rc = self.lib.aw_create(C.byref(cfg), C.byref(h))
        if rc:
            raise AwError(rc, "aw_create")
        self.h = h
        self.M = order_M
        self.Mc = (order_M + 1) * (order_M + 2) // 2
        self.Nt = order_M + 1
        self.Nst = self.Mc * self.Nt
        self.t_end = t_end
        self.tick = t_end / 2.0 ** time_quantum_log2
        self.n_tris = 0
        self.n_nodes = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.aw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise AwError(rc, self.lib.aw_last_error(self.h).decode())

    def load_mesh(self, mesh):
        xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
        bc = np.ascontiguousarray(mesh["bc"], dtype=np.int8)
        shift = None if mesh.get("shift") is None else np.ascontiguousarray(mesh["shift"], dtype=np.int8)
        period = None if mesh.get("period") is None else np.ascontiguousarray(mesh["period"], dtype=np.float64)
        self._check(self.lib.aw_load_mesh(self.h, xy.shape[0], _ptr(xy), tri.shape[0], _ptr(tri), _ptr(bc),
                                          _ptr(shift), _ptr(period)))
        self.n_tris = tri.shape[0]
        self.n_nodes = xy.shape[0]

    def load_batch(self, meshes, t_ends):
        """Independent non-periodic meshes advanced together (see aw_load_batch)."""
        node_off = np.zeros(len(meshes) + 1, np.int64)
        tri_off = np.zeros(len(meshes) + 1, np.int64)
        for k, m in enumerate(meshes):
            if m.get("period") is not None:
                raise ValueError("batched meshes must not be periodic")
            node_off[k + 1] = node_off[k] + m["xy"].shape[0]
            tri_off[k + 1] = tri_off[k] + m["tri"].shape[0]
        xy = np.ascontiguousarray(np.concatenate([m["xy"] for m in meshes]), dtype=np.float64)
        tri = np.ascontiguousarray(np.concatenate([m["tri"] for m in meshes]), dtype=np.int32)
        bc = np.ascontiguousarray(np.concatenate([m["bc"] for m in meshes]), dtype=np.int8)
        te = np.ascontiguousarray(t_ends, dtype=np.float64)
        self._check(self.lib.aw_load_batch(self.h, len(meshes), _ptr(node_off), _ptr(tri_off), _ptr(te), _ptr(xy),
                                           _ptr(tri), _ptr(bc)))
        self.n_tris = int(tri_off[-1])
        self.n_nodes = int(node_off[-1])
        self.node_offsets, self.tri_offsets = node_off, tri_off

    def load_state(self, Q):
        if not hasattr(Q, "data_ptr"):
            Q = np.ascontiguousarray(Q, dtype=np.float64)
        self._check(self.lib.aw_load_state(self.h, _ptr(Q)))

    def load_state_xy(self, Q, xy):
        """Initial state on node positions xy; the mesh pre-processing stays."""
        Q, xy = _f64(Q), _f64(xy)
        self._check(self.lib.aw_load_state_xy(self.h, _ptr(Q), _ptr(xy)))

    def schedule(self, mode, k=0):
        """Frozen schedule: "record" the dt ticks of each element's first k
        updates, "replay" them, or "free" (CFL steps)."""
        self._check(self.lib.aw_schedule(self.h, {"free": 0, "record": 1, "replay": 2}[mode], k))
        if mode == "record":
            self._sched_k = k

    def get_schedule(self):
        out = np.empty((self.n_tris, self._sched_k), np.int64)
        self._check(self.lib.aw_get_schedule(self.h, _ptr(out)))
        return out

    def adjoint_forward(self, n_sweeps, ckpt_every=10):
        """n_sweeps sweeps from the state just loaded, keeping checkpoints."""
        self._check(self.lib.aw_adjoint_forward(self.h, n_sweeps, ckpt_every))

    def adjoint(self, dJdQ=None, dJdX=None, dJdxy=None, out_Q=None, out_xy=None):
        """dJ/dQ0 [n_tris,4] and dJ/dxy0 [n_nodes,2] of the recorded run from
        dJ/d(final Q [n_tris,4], element corners [n_tris,6], nodes [n_nodes,2])."""
        gQ = np.empty((self.n_tris, 4)) if out_Q is None else out_Q
        gxy = np.empty((self.n_nodes, 2)) if out_xy is None else out_xy
        self._check(self.lib.aw_adjoint(self.h, _ptr(_f64(dJdQ)), _ptr(_f64(dJdX)), _ptr(_f64(dJdxy)), _ptr(gQ),
                                        _ptr(gxy)))
        return gQ, gxy

    def set_tiles(self, recon_half=0, pred_wide=0, bpsm=8):
        t = np.array([recon_half, pred_wide, bpsm], np.int32)
        self._check(self.lib.aw_set_tiles(self.h, _ptr(t)))

    def get_tiles(self):
        t = np.zeros(3, np.int32)
        self._check(self.lib.aw_get_tiles(self.h, _ptr(t)))
        return dict(recon_half=int(t[0]), pred_wide=int(t[1]), bpsm=int(t[2]))

    def autotune(self, n_sweeps=20):
        """Time the 12 tile shapes on the loaded state, keep the fastest;
        returns (chosen tiles, {(recon_half, pred_wide, bpsm): ms})."""
        ms = np.zeros(12)
        best = np.zeros(3, np.int32)
        self._check(self.lib.aw_autotune(self.h, n_sweeps, _ptr(ms), _ptr(best)))
        table = {(k // 6, (k // 3) % 2, (4, 8, 16)[k % 3]): float(ms[k]) for k in range(12)}
        return dict(recon_half=int(best[0]), pred_wide=int(best[1]), bpsm=int(best[2])), table

    def sweep(self):
        n = C.c_int64(0)
        self._check(self.lib.aw_lts_sweep(self.h, C.byref(n)))
        return n.value

    def gts_step(self):
        n = C.c_int64(0)
        self._check(self.lib.aw_gts_step(self.h, C.byref(n)))
        return n.value

    def advance(self, max_sweeps=10 ** 12):
        return self.advance_to(self.t_end, max_sweeps)

    def advance_to(self, t, max_sweeps=10 ** 12):
        """Sweeps until every element reached the sync time t (t_end, or a
        whole number of ticks not behind any element); (sweeps, updates)."""
        s, u = C.c_int64(0), C.c_int64(0)
        self._check(self.lib.aw_advance_to(self.h, float(t), int(max_sweeps), C.byref(s), C.byref(u)))
        return s.value, u.value

    def enqueue(self, n):
        self._check(self.lib.aw_enqueue_sweeps(self.h, n))

    def sync(self):
        n = C.c_int64(0)
        self._check(self.lib.aw_sync(self.h, C.byref(n)))
        return n.value

    def get_state(self, Q=None, t=None):
        Q = np.empty((self.n_tris, 4)) if Q is None else Q
        self._check(self.lib.aw_get_state(self.h, _ptr(Q), _ptr(t)))
        return Q

    def get_elem(self):
        n, Nst = self.n_tris, self.Nst
        out = dict(Q=np.empty((n, 4)), QM=np.empty((n, 4)), HM=np.empty((n, 3)), t=np.empty(n, np.int64),
                   dt=np.empty(n, np.int64), X=np.empty((n, 6)), count=np.empty(n, np.int64),
                   qhat=np.empty((n, Nst, 4)))
        self._check(self.lib.aw_get_elem_arrays(self.h, *[_ptr(out[k]) for k in
                                                           ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")]))
        return out

    def get_elem_into(self, **out):
        """Copy the named element arrays (Q, QM, HM, t, dt, X, count, qhat)
        into the given buffers: numpy arrays or torch tensors (host or
        device, contiguous, of the layout of include/aleweno.h)."""
        keys = ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")
        bad = set(out) - set(keys)
        if bad:
            raise ValueError(f"unknown element arrays {sorted(bad)}")
        self._check(self.lib.aw_get_elem_arrays(self.h, *[_ptr(out.get(k)) for k in keys]))

    def set_elem(self, st):
        arrs = [_arr(st[k], np.int64 if k in ("t", "dt", "count") else np.float64)
                for k in ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")]
        self._check(self.lib.aw_set_elem_arrays(self.h, *[_ptr(a) for a in arrs]))

    def get_nodes(self):
        X = np.empty((self.n_nodes, 2))
        t = np.empty(self.n_nodes, np.int64)
        self._check(self.lib.aw_get_node_arrays(self.h, _ptr(X), _ptr(t)))
        return X, t

    def set_nodes(self, X, t):
        X = _arr(X, np.float64)
        t = _arr(t, np.int64)
        self._check(self.lib.aw_set_node_arrays(self.h, _ptr(X), _ptr(t)))

    def update_counts(self):
        per = np.empty(self.n_tris, np.int64)
        tot = C.c_int64(0)
        self._check(self.lib.aw_get_update_counts(self.h, _ptr(per), C.byref(tot)))
        return per, tot.value

    def diag(self):
        out = np.zeros(4)
        self._check(self.lib.aw_diagnostics(self.h, _ptr(out)))
        return dict(gcl_max=out[0], updates=out[1], sweeps=out[2], surfaces=out[3])

    def profile(self, on=True):
        self._check(self.lib.aw_profile_enable(self.h, int(on)))

    def profile_read(self):
        ms = np.zeros(32)
        sw = C.c_int64(0)
        n = self.lib.aw_profile_read(self.h, _ptr(ms), C.byref(sw))
        if n < 0:
            self._check(n)
        names = [self.lib.aw_kernel_name(k).decode() for k in range(n)]
        return dict(zip(names, ms[:n].tolist())), sw.value

    def sizes(self):
        out = np.zeros(6, np.int64)
        self._check(self.lib.aw_sizes(self.h, _ptr(out)))
        return dict(n_tris=int(out[0]), n_nodes=int(out[1]), n_edges=int(out[2]), n_st=int(out[3]),
                    sw_entries=int(out[4]), u_entries=int(out[5]))
