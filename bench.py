"""Benchmark: FP64 element updates per second of the LTS ALE ADER-WENO sweep.

One step = one LTS sweep (update criterion, node motion, space-time fluxes,
FV update, projection + WENO + time step, predictor) over the resident
state.  Default workload: the cylindrical explosion (EP1 data: rho, p = 1, 1
inside r < 0.5, 0.125, 0.1 outside) on a ~500k-triangle disc graded 10x from
centre to rim, P3 scheme (fourth order), local time stepping.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--order 3] [--hc 0.00114]

Under torchrun (N > 1) every rank runs its own replica of the workload on its
GPU (the mesh is not partitioned); rank 0 prints one JSON line with the
aggregate rate over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 element-updates/s, LTS P3: plain vs batched vs adjoint; % HBM roofline"
UNIT = "element-updates/s"


# ---------------------------------------------------------------------------
# algorithmic FP64 operation counts per element update (one flop per add,
# multiply, divide or square root; an FMA counts two), from the operation
# counts of the predictor (Sec. 2.3) and the reconstruction (Sec. 2.2)
# ---------------------------------------------------------------------------

def predictor_flops(M: int) -> float:
    Mc, Nt = (M + 1) * (M + 2) // 2, M + 1
    nit = M + 1
    per_node = (2 * 2 * Mc * 14      # d/dxi, d/deta of q (4), f (4), g (4), x (2)
                + 2 * 2 * Nt         # d/dtau of the two coordinates
                + 2 + 18             # 1/rho, velocity, pressure, fluxes f and g
                + 16                 # inverse metric (one division) and xi_t, eta_t
                + 4 * 6 * 2          # P = -(Q_xi xi_t + ... + g_eta eta_y)
                + 6 * Nt * 2 * M / Nt)  # Picard update of q (4) and x (2) on the tau > 0 slices
    products = 3 * Nt * Nt * 4 * 2 * (Mc + Nt) + Nt * 4 * 2 * (Mc + Nt) + 3 * Nt * (1 + 2 * 2 * Nt)
    return per_node * Mc * Nt * nit + products


def recon_flops(M: int, members: float) -> float:
    Mc, Nt = (M + 1) * (M + 2) // 2, M + 1
    NU, NE = Mc - 1, 2 * Mc
    # monomial averages over the member from its centroid and central moments
    moments = {1: 6, 2: 36, 3: 90}[M]
    per_member = (6 * 2 * Nt + 4 * 2 * (Nt - 1) + 4   # virtual vertices and average (Horner)
                  + 3 * 8                              # map to the reference frame of T_i
                  + moments + NU + 4)
    per_stencil = ((NE - 1) * (NU * (NU + 1) + 8 * NU)  # normal equations
                   + NU ** 3 / 3 + 2 * NU               # Cholesky
                   + 4 * 2 * NU * NU                    # two triangular solves, 4 right-hand sides
                   + 4 * (4 * (NE - 1) * NU + 2 * NU * NU)  # one refinement: r = b - A y, A^T r, two solves
                   + NU * 32                            # characteristic projection
                   + 4 * (NU * (NU + 1) + NU))          # smoothness indicators
    weights = 4 * (7 * 8 + NU * 7 * 2) + NU * 32 + Mc * 4 * NU * 2
    dt = 4 * 60
    return members * per_member + 7 * per_stencil + weights + dt


def hbm_bytes_per_update(M: int, sw_per_elem: float, members_per_elem: float = 0.0) -> float:
    """Compulsory DRAM bytes of one element update with perfect on-chip reuse
    in a sweep: read its state, ticks, corners and node data (~28 words) and
    its predictor tables (4 N_st words), write the new predictor and tables
    (4 N_st words), state and nodes (~30 words); read its stencil and total
    stencil index lists (7 n_e + |S^W| int32); and, under local time
    stepping (the ready elements of a sweep are sparse, so their stencils
    barely overlap), gather for each distinct stencil member the data of its
    virtual projection: ticks (2), corners (6), average and its tau
    polynomial (4 (M+1)), vertex displacement polynomials (6 (M+1)) and
    periodic offset (2) words."""
    Mc = (M + 1) * (M + 2) // 2
    Nst = Mc * (M + 1)
    member = 8.0 * (2 + 6 + 4 * (M + 1) + 6 * (M + 1) + 2)
    return 8.0 * (28 + 4 * Nst + 4 * Nst + 30) + 4.0 * (7 * 2 * Mc + sw_per_elem) + members_per_elem * member


def host_info():
    """CPU model and core count of the host running the oracle."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu": model, "machine": platform.machine(), "cores_available": os.cpu_count()}


def flux_flops(M: int) -> float:
    """FP64 operations of one space-time edge surface (Rusanov-type flux,
    (M+1)^2 Gauss points)."""
    Nt = M + 1
    per_point = (4                      # corner times (ticks x tick length)
                 + 33 + 9               # bilinear surface derivatives, normal = cross product
                 + 11                   # time of the point
                 + 2 * (2 + 8 * (Nt - 1))  # each side's local tau and trace (4 variables, Horner)
                 + 2 * 53               # each side's velocity, pressure, sound speed, f, g and F.n
                 + 15 + 16              # |n_xy|, mesh normal speed, s_max; the Rusanov combination
                 + 8 + 7)               # weights of the flux and GCL vector; sum over the points
    return Nt * Nt * per_point


# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(ms: float, updates: int, dist=None, device="cpu"):
    """Whole-job figures over ranks: the slowest rank's time and the sum of
    all ranks' element updates (each rank runs its own replica)."""
    if dist is None:
        return ms, float(updates)
    import torch
    t = torch.tensor([ms, float(updates)], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def workload(order: int, hc: float, flux: str = "rusanov", t_switch: float = 0.01):
    """The explosion EP1 on the graded disc; with t_switch > 0 the run takes
    global steps (CFL 0.5) until t_switch and local steps after, the start-up
    of Sec. 3.5 with which the fourth-order run reaches t_end (without it the
    first local step of an element on the initial jump overshoots)."""
    from paper_1408_3719_gb300 import workloads as W
    mesh, Q = W.explosion(hc)
    cfg = dict(order_M=order, t_end=0.25, time_quantum_log2=20, flux=flux)
    if t_switch > 0:
        cfg.update(t_switch=t_switch, cfl_start=0.5)
    return mesh, Q, cfg


def oracle_counts(order: int, flux: str = "rusanov", sweeps: int = 3):
    """FP64 operations per element update (reconstruction with its virtual
    projection, local step, predictor, whole update) and per space-time
    surface (fluxes) counted by the oracle's counting build on the bounded
    sample disc: the plain oracle's own arithmetic, an upper bound of the
    method as the kernels formulate it."""
    from oracle.pyoracle import Oracle, flop_counts, flop_reset
    from paper_1408_3719_gb300 import workloads as W
    mesh, Q = W.explosion(0.005)
    o = Oracle(order_M=order, t_end=0.25, flux=flux, kind="count")
    o.load_mesh(mesh)
    o.load_state(Q)
    tri = np.asarray(mesh["tri"])
    edges = {tuple(sorted((int(t[k]), int(t[(k + 1) % 3])))) for t in tri for k in range(3)}
    ea = np.array(sorted(edges))
    flop_reset(o)
    ups = surf = 0
    for _ in range(sweeps):
        _, nt0 = o.get_nodes()
        ups += o.sweep()
        _, nt1 = o.get_nodes()
        moved = nt1 != nt0
        surf += int(np.count_nonzero(moved[ea[:, 0]] | moved[ea[:, 1]]))
    f = flop_counts(o)
    return {"per_update": {k: f[k] / ups for k in ("recon", "dt", "predictor", "nodes", "update")},
            "per_update_total": sum(f.values()) / ups, "flux_per_surface": f["flux"] / max(surf, 1),
            "sample": f"{sweeps} sweeps ({ups} updates, {surf} surfaces) of the {tri.shape[0]}-triangle disc"}


def read_ncu_counters(path):
    """key = value lines of a committed ncu summary (profiles/); {} if absent."""
    out = {}
    try:
        with open(path) as f:
            for line in f:
                line = line.split("#", 1)[0].strip()
                if "=" in line:
                    k, v = (x.strip() for x in line.split("=", 1))
                    try:
                        out[k] = v if k == "source_sha" else float(v)
                    except ValueError:
                        out[k] = v
    except OSError:
        pass
    return out


def kernel_source_digest():
    import hashlib
    with open(os.path.join(ROOT, "paper_1408_3719_gb300", "csrc", "aw_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def cpu_sample(order: int, seconds: float, warmup: int = 0, steps: int | None = None, flux: str = "rusanov",
               t_switch: float = 0.01):
    """The oracle on a bounded sample: the same generator and scheme on a
    ~26k-triangle disc; setup untimed; sweeps timed until `seconds` elapse
    (or `steps` sweeps)."""
    from oracle.pyoracle import Oracle
    from paper_1408_3719_gb300 import workloads as W
    mesh, Q = W.explosion(0.005)
    extra = dict(t_switch=t_switch, cfl_start=0.5) if t_switch > 0 else {}
    o = Oracle(order_M=order, t_end=0.25, flux=flux, **extra)
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(warmup):
        o.sweep()
    ups, sweeps = 0, 0
    t0 = time.perf_counter()
    while True:
        ups += o.sweep()
        sweeps += 1
        el = time.perf_counter() - t0
        if (steps is not None and sweeps >= steps) or (steps is None and el >= seconds):
            break
    return ups / el, dict(sweeps=sweeps, updates=ups, seconds=el, n_tris=int(mesh["tri"].shape[0]))


def _flux_tag(args):
    return "" if args.flux == "rusanov" else f", {args.flux} flux"


def explosion_config(args, n_tris: int, world: int) -> dict:
    """The workload keys of the explosion bench line, shared by both arms."""
    start = (f"global steps (CFL 0.5) until t = {args.t_switch:g}, then local steps" if args.t_switch > 0
             else "local steps from t = 0")
    return {"workload": f"cylindrical explosion EP1 on a graded disc, {n_tris} triangles, "
                        f"P{args.order} LTS, CFL 0.5, t_end 0.25, {start}{_flux_tag(args)}",
            "n_tris": n_tris, "order_M": args.order, "t_switch": args.t_switch,
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank):
    if rank != 0:
        return
    # the line names the workload of the GPU arm; the oracle runs a bounded
    # sample of it (the same generator and scheme on a smaller disc)
    mesh, _, _ = workload(args.order, args.hc, args.flux)
    full_tris = int(mesh["tri"].shape[0])
    del mesh
    rate, info = cpu_sample(args.order, 0, warmup=args.warmup, steps=args.steps, flux=args.flux,
                            t_switch=args.t_switch)
    sample = (f"oracle (plain serial C, FP64) on a {info['n_tris']}-triangle graded disc, same EP1 data and "
              f"P{args.order} LTS scheme, {args.flux} flux; {info['sweeps']} timed sweeps ({info['updates']} updates) after "
              f"{args.warmup} warm-up sweeps; pre-processing untimed")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * info["seconds"] / info["sweeps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": explosion_config(args, full_tris, 1),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_info()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def warm_into_run(s, t_warm, chunk=200, max_sweeps=200000):
    """Sweeps until every element is past t_warm (no sync point: the elements
    keep their own times, as in the middle of a run); returns the sweeps."""
    n = 0
    t = np.empty(s.n_tris)
    while n < max_sweeps:
        s.enqueue(chunk)
        s.sync()
        n += chunk
        s.get_state(t=t)
        if t.min() >= t_warm:
            break
    return n, t


def run_ours(args, rank, world):
    import torch
    from paper_1408_3719_gb300 import aleweno

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    aleweno.load()
    mesh, Q, cfg = workload(args.order, args.hc, args.flux, args.t_switch)
    n_tris = int(mesh["tri"].shape[0])
    # a dedicated (non-default) stream: the library launches on it and the
    # CUDA events below are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = aleweno.Solver(**cfg, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    s.load_mesh(mesh)
    t_mesh = time.perf_counter() - t0
    s.load_state(Q)
    sizes = s.sizes()
    peak_gflops = aleweno.fp64_peak_gflops()
    # into the run: through the start-up's global steps until every element
    # is past t_warm (untimed), so that the timed sweeps are local-time-step
    # sweeps from the middle of the run the line names; --save-state keeps
    # that state in a file and --load-state starts from such a file (short
    # profiling runs: a few launches instead of thousands)
    t0 = time.perf_counter()
    if args.load_state:
        z = np.load(args.load_state)
        s.set_elem({k: z[k] for k in ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")})
        s.set_nodes(z["nX"], z["nt"])
        warm_sweeps, t_el = int(z["sweeps"]), np.empty(n_tris)
    else:
        warm_sweeps, t_el = warm_into_run(s, args.t_warm)
    if args.save_state:
        e, (nX, nt) = s.get_elem(), s.get_nodes()
        np.savez(args.save_state, nX=nX, nt=nt, sweeps=warm_sweeps, **e)
    t_warm_s = time.perf_counter() - t0
    # the mid-run state for the end-to-end measurement below (the autotuner
    # restores the state it starts from)
    snap, snap_nodes = (s.get_elem(), s.get_nodes()) if args.e2e else (None, None)
    # clocks and throttle reasons sampled from the autotuner's sweeps through
    # the timed region (which alone lasts ~10 ms, shorter than nvidia-smi's
    # 20 ms sampling period): the same kernels at the same load
    clocks = ClockSampler(local)
    clocks.start()
    # tile shapes picked by the library's autotuner on this state (it times
    # the same sweeps for every shape and restores the state)
    if args.tiles:
        s.set_tiles(*[int(v) for v in args.tiles.split(",")])
        tiles, tune_ms = s.get_tiles(), {}
    else:
        tiles, tune_ms = s.autotune(args.tune_sweeps) if args.tune_sweeps > 0 else (s.get_tiles(), {})
    for _ in range(args.warmup):
        s.sweep()
    s.get_state(t=t_el)
    t_range = [float(t_el.min()), float(np.median(t_el)), float(t_el.max())]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > 129 MB L2
    s.sync()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        s.enqueue(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    clk["window"] = "the autotuner's sweeps, the warm-up sweeps and the timed region (same kernels, same load)"
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    updates = s.sync()
    # per-kernel CUDA-event times: a second pass of the same number of sweeps
    # with events between the launches (the timed pass above runs each sweep
    # as one captured CUDA graph)
    s.profile(True)
    surf0 = s.diag()["surfaces"]
    for k in range(args.steps):
        flush.fill_(float(k))
        s.enqueue(1)
    prof_updates = s.sync()
    prof_surfaces = s.diag()["surfaces"] - surf0
    kms, ksweeps = s.profile_read()
    s.profile(False)
    ms_max, updates_all = aggregate(ms, updates, dist, "cuda")
    value = updates_all / (ms_max * 1e-3)

    # dominant kernel and its roofline (FP64 pipe: this path is ALU-bound)
    dom = max(kms, key=kms.get)
    members = sizes["u_entries"] / max(sizes["n_tris"], 1)
    # FP64 operations of the profiled pass: per update (predictor,
    # reconstruction) or per space-time edge surface (fluxes)
    model = {"k_predict": (predictor_flops(args.order), prof_updates, "update"),
             "k_recon": (recon_flops(args.order, members), prof_updates, "update"),
             "k_flux": (flux_flops(args.order), prof_surfaces, "surface")}
    # per-launch DRAM bytes and executed FP64 operations of the same kernels
    # from the committed ncu capture, used only while the kernel source is
    # the one that capture measured
    ncu = read_ncu_counters(os.path.join(ROOT, "profiles", f"ncu_counters_explosion_p{args.order}.txt"))
    ncu_valid = ncu.get("source_sha") == kernel_source_digest() and args.flux == "rusanov"
    roof = None
    if dom in model and kms[dom] > 0:
        per_unit, units, unit_name = model[dom]
        achieved = per_unit * units / (kms[dom] * 1e-3) / 1e12
        peak = peak_gflops / 1e3
        launches = ksweeps
        traffic = executed = None
        if ncu_valid and f"{dom}.units" in ncu:
            per_unit_bytes = ncu[f"{dom}.dram_bytes"] / ncu[f"{dom}.units"]
            traffic = per_unit_bytes * units / launches
            exec_per_unit = ncu[f"{dom}.fp64_ops"] / ncu[f"{dom}.units"]
            executed = {"flops_per_unit": exec_per_unit,
                        "achieved": exec_per_unit * units / (kms[dom] * 1e-3) / 1e12,
                        "frac": exec_per_unit * units / (kms[dom] * 1e-3) / 1e12 / peak,
                        "note": "FP64 operations the kernel executes (2 per DFMA, 1 per DADD/DMUL), ncu counters "
                                "per unit from the committed capture"}
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_note": ("DRAM bytes per launch: ncu dram__bytes_read + write per unit of the committed "
                                 "capture x the units of an average timed launch" if traffic is not None else
                                 "null: no ncu capture of the current kernel source"),
                "peak_source": "measured FP64 DFMA throughput (aw_measure_fp64_peak, this run); "
                               "MEASURED_PEAKS.json has no FP64 figure",
                f"flops_per_{unit_name}": per_unit, f"{unit_name}s_profiled": units,
                "flops_note": "operation count of the method's steps as the kernel formulates them (bench.py: "
                              "predictor_flops, recon_flops, flux_flops)",
                "executed": executed}
    # the HBM roofline this FP64-bound path is far from: compulsory bytes per
    # update x update rate, against the measured copy bandwidth
    bpu = hbm_bytes_per_update(args.order, sizes["sw_entries"] / n_tris, members)
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    hbm = {"bytes_per_update": bpu, "achieved_GBs": value * bpu / 1e9, "peak_GBs": hbm_peak,
           "frac": (value * bpu / 1e9 / hbm_peak) if hbm_peak else None,
           "note": "algorithmic (compulsory) bytes, with the gathers of the stencil members' virtual data; the "
                   "path is bound by the FP64 pipe, see roofline"}

    # end to end through the C ABI with host buffers: the mid-run state
    # (taken just before the driver's warm-up sweeps) uploaded from pinned host
    # memory, e2e_sweeps sweeps, the averages read back to pinned host memory
    e2e = None
    if args.e2e:
        s2 = aleweno.Solver(**cfg, stream=stream.cuda_stream)
        s2.load_mesh(mesh)
        s2.set_tiles(tiles["recon_half"], tiles["pred_wide"], tiles["bpsm"])  # the shape picked above
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in snap.items()}
        pnX, pnt = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in snap_nodes)
        out = torch.empty((n_tris, 4), dtype=torch.float64).pin_memory()
        nst = args.e2e_sweeps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.set_elem(pin)
        s2.set_nodes(pnX, pnt)
        s2.enqueue(nst)
        ups = s2.sync()
        s2.get_state(out)
        el = time.perf_counter() - t0
        h2d = sum(v.numel() * v.element_size() for v in pin.values()) + pnX.numel() * 8 + pnt.numel() * 8
        e2e = {"value": ups / el, "unit": UNIT, "h2d_bytes_per_step": h2d / nst,
               "d2h_bytes_per_step": (out.numel() * 8 + 16) / nst,
               "note": "aw_set_elem_arrays + aw_set_node_arrays (the mid-run state before the driver's warm-up sweeps, "
                       "pinned host memory) + aw_enqueue_sweeps + aw_sync (update count) + aw_get_state (averages "
                       "to pinned host memory), host wall time, the tile shapes of the device-timed run"}
        s2.close()
        del pin

    # the whole run the line names, from the loaded state to t_end
    full = None
    if args.full_run and rank == 0:
        s3 = aleweno.Solver(**cfg, stream=stream.cuda_stream)
        s3.load_mesh(mesh)
        s3.set_tiles(tiles["recon_half"], tiles["pred_wide"], tiles["bpsm"])
        s3.load_state(Q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sweeps_f, ups_f = s3.advance()
        el = time.perf_counter() - t0
        full = {"value": ups_f / el, "unit": UNIT, "seconds": el, "updates": ups_f, "sweeps": sweeps_f,
                "note": "aw_advance_to(t_end) from the loaded state (start-up and all local steps), host wall "
                        "time, device-resident state"}
        s3.close()

    cpu = None
    if rank == 0 and world == 1 and args.cpu_baseline:
        rate, info = cpu_sample(args.order, args.cpu_seconds, flux=args.flux, t_switch=args.t_switch)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": f"oracle (serial C, FP64) on a {info['n_tris']}-triangle graded disc with the same EP1 "
                         f"data and P{args.order} LTS scheme with its start-up, {info['sweeps']} sweeps from t=0 "
                         f"({info['updates']} updates, {info['seconds']:.1f} s), pre-processing untimed"}
        try:
            cpu["oracle_flops"] = oracle_counts(args.order, args.flux)
        except Exception as exc:  # the counting build is context, not the baseline
            cpu["oracle_flops"] = {"unavailable": str(exc)[:200]}
    if rank == 0:
        share_tot = sum(kms.values()) or 1.0
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {**explosion_config(args, n_tris, world),
                           "timed_from": f"{warm_sweeps + args.warmup} sweeps into the run, element times "
                                         f"min/median/max {t_range[0]:.4f}/{t_range[1]:.4f}/{t_range[2]:.4f}",
                           "l2": "256 MiB write between timed sweeps (L2 is 129 MB)",
                           "updates_timed": int(updates_all), "sw_entries_per_elem": sizes["sw_entries"] / n_tris,
                           "stencil_members_per_elem": members},
                "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e, "full_run": full,
                "gpu_launches": len(kms) * args.steps,
                "clocks": clk,
                "kernels": {k: {"ms": v, "share": v / share_tot} for k, v in kms.items()},
                "kernels_note": f"CUDA-event times over a second pass of {ksweeps} sweeps ({prof_updates} updates)",
                "tiles": tiles,
                "autotune_ms": {f"recon_half={k[0]},pred_wide={k[1]},bpsm={k[2]}": v for k, v in tune_ms.items()},
                "fp64_peak_gflops": peak_gflops, "warm_s": t_warm_s}
        s.close()
        if args.extras and world == 1:
            line.update(run_extras(args))
        print(json.dumps(line), flush=True)
    else:
        s.close()
    if dist:
        dist.destroy_process_group()


def run_extras(args):
    """The batched and adjoint figures of the metric, measured after the main
    line (each with its own short step count): the batched sweep over the
    config's 256 instances against a per-instance loop, and the adjoint of
    the 50-sweep vortex run against its forward, for the objective on the
    disc r < 1 and for one over every element (no zero adjoints to skip)."""
    out = {}
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = args.extra_steps, 3
    try:
        sub.order = 2
        out["batched"] = run_batched(sub, 0, 1, emit=False)
        out["batched_over_loop"] = out["batched"]["batched_over_loop"]
    except Exception as exc:
        out["batched"] = {"unavailable": str(exc)[:200]}
    for objective, key in (("disc", "adjoint"), ("global", "adjoint_global")):
        try:
            sub.order, sub.objective = 2, objective
            out[key] = run_adjoint(sub, emit=False)
            out[key + "_over_forward"] = out[key]["adjoint_over_forward"]
        except Exception as exc:
            out[key] = {"unavailable": str(exc)[:200]}
    return out


def shard_instances(sizes, world):
    """Independent instances over ranks, largest first to the least-loaded
    rank (deterministic); returns the instance indices of every rank."""
    parts = [[] for _ in range(world)]
    load = [0] * world
    for k in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(k)
        load[r] += sizes[k]
    return [sorted(p) for p in parts]


def run_batched(args, rank=0, world=1, emit=True):
    """Config 4: many independent explosion / shock-tube instances advanced by
    one sweep over the batch, against a loop that runs the same instances one
    context at a time on the same GPU.  With N ranks the instances are
    sharded (no collective on the data path: each rank advances its own
    batch; only the timings are reduced)."""
    import torch
    from paper_1408_3719_gb300 import aleweno
    from paper_1408_3719_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    aleweno.load()
    inst_all = W.batched_instances(args.instances, lo=args.min_tris, hi=args.max_tris)
    part = shard_instances([int(d["mesh"]["tri"].shape[0]) for d in inst_all], world)[rank]
    inst = [inst_all[k] for k in part]
    meshes, qs, t_ends = [d["mesh"] for d in inst], [d["q"] for d in inst], [d["t_end"] for d in inst]
    n_tris = sum(int(m["tri"].shape[0]) for m in meshes)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(solvers, steps):
        for s in solvers:
            s.sync()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            e0.record(stream)
            for s in solvers:
                s.enqueue(1)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        return sum(s.sync() for s in solvers), ms

    cfg = dict(order_M=args.order, t_end=max(t_ends), time_quantum_log2=20)
    b = aleweno.Solver(**cfg, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    b.load_batch(meshes, t_ends)
    t_pre = time.perf_counter() - t0
    b.load_state(np.concatenate(qs))
    if args.tiles:
        b.set_tiles(*[int(v) for v in args.tiles.split(",")])
        tiles, tune_ms = b.get_tiles(), {}
    else:
        tiles, tune_ms = b.autotune(args.tune_sweeps) if args.tune_sweeps > 0 else (b.get_tiles(), {})
    for _ in range(args.warmup):
        b.enqueue(1)
    ub, msb = timed([b], args.steps)
    b.close()
    loop = []
    for m, q, te in zip(meshes, qs, t_ends):
        s = aleweno.Solver(order_M=args.order, t_end=te, time_quantum_log2=20, stream=stream.cuda_stream)
        s.load_mesh(m)
        s.load_state(q)
        for _ in range(args.warmup):
            s.enqueue(1)
        loop.append(s)
    ul, msl = timed(loop, args.steps)
    for s in loop:
        s.close()
    msb, ub = aggregate(msb, ub, dist, "cuda")
    msl, ul = aggregate(msl, ul, dist, "cuda")
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    n_tris = sum(int(d["mesh"]["tri"].shape[0]) for d in inst_all)
    vb, vl = ub / (msb * 1e-3), ul / (msl * 1e-3)
    line = {"metric": METRIC, "value": vb, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": msb / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched: {len(inst_all)} explosion/shock-tube instances, {n_tris} triangles, "
                                   f"P{args.order} LTS, one sweep over the batch per step",
                       "n_tris": n_tris, "instances": len(inst_all), "preprocessing_s": t_pre,
                       "parallelism": f"instances sharded over {world} rank(s), largest first",
                       "l2": "256 MiB write between timed sweeps"},
            "tiles": tiles, "autotune_ms": {f"recon_half={k[0]},pred_wide={k[1]},bpsm={k[2]}": v
                                             for k, v in tune_ms.items()},
            "per_instance_loop": {"value": vl, "unit": UNIT, "ms_per_step": msl / args.steps,
                                  "note": "same instances, one context per instance (default tiles), one sweep "
                                          "of each per step"},
            "batched_over_loop": vb / vl}
    if emit:
        print(json.dumps(line), flush=True)
    return {"value": vb, "unit": UNIT, "ms_per_step": msb / args.steps, "steps": args.steps,
            "workload": line["config"]["workload"], "per_instance_loop": line["per_instance_loop"],
            "batched_over_loop": vb / vl, "tiles": tiles}


def run_adjoint(args, emit=True):
    """Config 5: gradient of the kinetic energy in the disc r < 1 about the
    vortex centre after 50 LTS sweeps of P2 on the ~50k-triangle isentropic
    vortex, with respect to the initial averages and node positions
    (checkpoints every 10 sweeps).  One step = load, checkpointed forward run,
    reverse pass.  value = element updates of the forward run differentiated
    per second of the reverse pass."""
    import torch
    from paper_1408_3719_gb300 import aleweno
    from paper_1408_3719_gb300 import workloads as W

    torch.cuda.set_device(0)
    aleweno.load()
    mesh, Q0 = W.vortex(args.vortex_n)
    n_sw, ck = args.adj_sweeps, args.ckpt
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    s = aleweno.Solver(order_M=args.order, t_end=1.0, stream=stream.cuda_stream)
    s.load_mesh(mesh)
    corners = W._corner_coords(mesh).mean(1) - 5.0
    if args.objective == "global":  # every element: no zero adjoints to skip
        mask = np.ones(Q0.shape[0])
    else:
        mask = (np.hypot(corners[:, 0], corners[:, 1]) < 1.0).astype(np.float64)

    def dJ(e):
        Q, X = e["Q"], e["X"]
        A = 0.5 * ((X[:, 2] - X[:, 0]) * (X[:, 5] - X[:, 1]) - (X[:, 3] - X[:, 1]) * (X[:, 4] - X[:, 0]))
        ke = 0.5 * (Q[:, 1] ** 2 + Q[:, 2] ** 2) / Q[:, 0]
        gQ = np.zeros_like(Q)
        gQ[:, 0] = -mask * A * ke / Q[:, 0]
        gQ[:, 1] = mask * A * Q[:, 1] / Q[:, 0]
        gQ[:, 2] = mask * A * Q[:, 2] / Q[:, 0]
        sk = 0.5 * mask * ke
        gX = np.stack([sk * (X[:, 3] - X[:, 5]), sk * (X[:, 4] - X[:, 2]), sk * (X[:, 5] - X[:, 1]),
                       sk * (X[:, 0] - X[:, 4]), sk * (X[:, 1] - X[:, 3]), sk * (X[:, 2] - X[:, 0])], axis=1)
        return gQ, gX

    def ev():
        return torch.cuda.Event(enable_timing=True)

    t_load, t_plain, t_fwd, t_adj, updates = [], [], [], [], 0
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        el0, e0, e1 = ev(), ev(), ev()
        el0.record(stream)
        s.load_state(Q0)
        e0.record(stream)
        s.enqueue(n_sw)
        e1.record(stream)
        updates = s.sync()
        e1.synchronize()
        flush.fill_(float(k))
        s.load_state(Q0)
        e2, e3, e4 = ev(), ev(), ev()
        e2.record(stream)
        s.adjoint_forward(n_sw, ck)
        e3.record(stream)
        gQ, gX = (torch.from_numpy(g).to("cuda") for g in dJ(s.get_elem()))
        oQ = torch.empty(Q0.shape, dtype=torch.float64, device="cuda")
        oxy = torch.empty((s.n_nodes, 2), dtype=torch.float64, device="cuda")
        flush.fill_(float(k))
        e4.record(stream)
        s.adjoint(gQ, gX, None, out_Q=oQ, out_xy=oxy)
        e5 = ev()
        e5.record(stream)
        e5.synchronize()
        if k >= args.warmup:
            t_load.append(el0.elapsed_time(e0))
            t_plain.append(e0.elapsed_time(e1))
            t_fwd.append(e2.elapsed_time(e3))
            t_adj.append(e4.elapsed_time(e5))
    ml, mp, mf, ma = (float(np.median(t)) for t in (t_load, t_plain, t_fwd, t_adj))
    line = {"metric": METRIC, "value": updates / (ma * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ma, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"adjoint: isentropic vortex, {Q0.shape[0]} triangles, P{args.order} LTS, "
                                   f"{n_sw} sweeps, checkpoints every {ck}; objective: kinetic energy "
                                   + ("of every element" if args.objective == "global" else "in the disc r < 1")
                                   + "; value = forward element updates differentiated per second of the "
                                     "reverse pass",
                       "objective": args.objective,
                       "n_tris": int(Q0.shape[0]), "sweeps": n_sw, "ckpt_every": ck, "forward_updates": int(updates),
                       "l2": "256 MiB write before each timed pass",
                       "adjoint_io": "seed dJ/d(final state) and gradients in device memory"},
            "load_state_ms": ml, "sweeps_ms": mp, "forward_ms": ml + mp,
            "forward_with_checkpoints_ms": mf, "adjoint_ms": ma,
            "adjoint_over_forward": ma / (ml + mp), "adjoint_over_sweeps": ma / mp,
            "note": "forward = aw_load_state (pre-processing phase over every element) + the sweeps: the map "
                    "the gradient differentiates"}
    if emit:
        print(json.dumps(line), flush=True)
    return {"value": line["value"], "unit": UNIT, "steps": args.steps, "workload": line["config"]["workload"],
            "forward_ms": ml + mp, "adjoint_ms": ma, "adjoint_over_forward": ma / (ml + mp),
            "adjoint_over_sweeps": ma / mp}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--hc", type=float, default=0.00114)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--e2e-sweeps", type=int, default=500)
    ap.add_argument("--workload", default="explosion", choices=["explosion", "batched", "adjoint"])
    ap.add_argument("--vortex-n", type=int, default=158)
    ap.add_argument("--tune-sweeps", type=int, default=20)
    ap.add_argument("--tiles", default=None,
                    help="recon_half,pred_wide,bpsm: fixed tile shapes instead of the autotuner")
    ap.add_argument("--adj-sweeps", type=int, default=50)
    ap.add_argument("--ckpt", type=int, default=10)
    ap.add_argument("--flux", default="rusanov", choices=["rusanov", "osher"],
                    help="numerical flux of the explosion workload and its oracle sample")
    ap.add_argument("--objective", default="disc", choices=["disc", "global"])
    ap.add_argument("--t-switch", type=float, default=0.01,
                    help="global steps until this time, local steps after (0: local steps from t = 0)")
    ap.add_argument("--t-warm", type=float, default=0.02,
                    help="untimed sweeps until every element is past this time before the timed sweeps")
    ap.add_argument("--no-full-run", dest="full_run", action="store_false",
                    help="skip the run from the loaded state to t_end")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the batched and adjoint figures after the main line")
    ap.add_argument("--extra-steps", type=int, default=10)
    ap.add_argument("--save-state", default=None, help="write the warmed-up state to this .npz file")
    ap.add_argument("--load-state", default=None, help="start from a state written by --save-state")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--min-tris", type=int, default=2000)
    ap.add_argument("--max-tris", type=int, default=60000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "adjoint":
        if args.order == 3 and "--order" not in sys.argv:
            args.order = 2
        if rank == 0:
            run_adjoint(args)
        return
    if args.workload == "batched":
        if args.order == 3 and "--order" not in sys.argv:
            args.order = 2
        run_batched(args, rank, world)
        return
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
