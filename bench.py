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
    nq = {1: 1, 2: 3, 3: 4}[M]
    per_member = (6 * 2 * Nt + 4 * 2 * (Nt - 1) + 4   # virtual vertices and average (Horner)
                  + 3 * 8                              # map to the reference frame of T_i
                  + nq * (4 + max(NU - 2, 0) + 2 * NU) + NU + 4)
    per_stencil = ((NE - 1) * (NU * (NU + 1) + 8 * NU)  # normal equations
                   + NU ** 3 / 3 + 2 * NU               # Cholesky
                   + 4 * 2 * NU * NU                    # two triangular solves, 4 right-hand sides
                   + NU * 32                            # characteristic projection
                   + 4 * (NU * (NU + 1) + NU))          # smoothness indicators
    weights = 4 * (7 * 8 + NU * 7 * 2) + NU * 32 + Mc * 4 * NU * 2
    dt = 4 * 60
    return members * per_member + 7 * per_stencil + weights + dt


def hbm_bytes_per_update(M: int, sw_per_elem: float) -> float:
    """Compulsory DRAM bytes of one element update with perfect on-chip reuse
    in a sweep: read its state, ticks, corners and node data (~28 words) and
    its predictor tables (4 N_st words), write the new predictor and tables
    (4 N_st words), state and nodes (~30 words); read its stencil and total
    stencil index lists (7 n_e + |S^W| int32)."""
    Mc = (M + 1) * (M + 2) // 2
    Nst = Mc * (M + 1)
    return 8.0 * (28 + 4 * Nst + 4 * Nst + 30) + 4.0 * (7 * 2 * Mc + sw_per_elem)


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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


def workload(order: int, hc: float, flux: str = "rusanov"):
    from paper_1408_3719_gb300 import workloads as W
    mesh, Q = W.explosion(hc)
    return mesh, Q, dict(order_M=order, t_end=0.25, time_quantum_log2=20, flux=flux)


def cpu_sample(order: int, seconds: float, warmup: int = 0, steps: int | None = None, flux: str = "rusanov"):
    """The oracle on a bounded sample: the same generator and scheme on a
    ~26k-triangle disc; setup untimed; sweeps timed until `seconds` elapse
    (or `steps` sweeps)."""
    from oracle.pyoracle import Oracle
    from paper_1408_3719_gb300 import workloads as W
    mesh, Q = W.explosion(0.005)
    o = Oracle(order_M=order, t_end=0.25, flux=flux)
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
    return {"workload": f"cylindrical explosion EP1 on a graded disc, {n_tris} triangles, "
                        f"P{args.order} LTS, CFL 0.5, t_end 0.25{_flux_tag(args)}",
            "n_tris": n_tris, "order_M": args.order, "parallelism": f"replicas x{world}"}


def run_reference(args, rank):
    if rank != 0:
        return
    # the line names the workload of the GPU arm; the oracle runs a bounded
    # sample of it (the same generator and scheme on a smaller disc)
    mesh, _, _ = workload(args.order, args.hc, args.flux)
    full_tris = int(mesh["tri"].shape[0])
    del mesh
    rate, info = cpu_sample(args.order, 0, warmup=args.warmup, steps=args.steps, flux=args.flux)
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
    mesh, Q, cfg = workload(args.order, args.hc, args.flux)
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
    # tile shapes picked by the library's autotuner on this state (it times
    # the same sweeps for every shape and restores the state)
    if args.tiles:
        s.set_tiles(*[int(v) for v in args.tiles.split(",")])
        tiles, tune_ms = s.get_tiles(), {}
    else:
        tiles, tune_ms = s.autotune(args.tune_sweeps) if args.tune_sweeps > 0 else (s.get_tiles(), {})
    for _ in range(args.warmup):
        s.sweep()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > 129 MB L2
    s.sync()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks.start()
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
    roof = None
    if dom in model and kms[dom] > 0:
        per_unit, units, unit_name = model[dom]
        achieved = per_unit * units / (kms[dom] * 1e-3) / 1e12
        peak = peak_gflops / 1e3
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "measured FP64 DFMA throughput (aw_measure_fp64_peak, this run)",
                f"flops_per_{unit_name}": per_unit, f"{unit_name}s_profiled": units}
    # the HBM roofline this FP64-bound path is far from: compulsory bytes per
    # update x update rate, against the measured copy bandwidth
    bpu = hbm_bytes_per_update(args.order, sizes["sw_entries"] / n_tris)
    hbm_peak = None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    hbm = {"bytes_per_update": bpu, "achieved_GBs": value * bpu / 1e9, "peak_GBs": hbm_peak,
           "frac": (value * bpu / 1e9 / hbm_peak) if hbm_peak else None,
           "note": "algorithmic (compulsory) bytes; the path is bound by the FP64 pipe, see roofline"}

    # end to end through the C ABI with host buffers: state upload + initial
    # phase, the same number of sweeps, state download
    e2e = None
    if args.e2e:
        s2 = aleweno.Solver(**cfg)
        s2.load_mesh(mesh)
        s2.set_tiles(tiles["recon_half"], tiles["pred_wide"], tiles["bpsm"])  # the shape picked above
        Qh = np.ascontiguousarray(Q)
        out = np.empty_like(Qh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.load_state(Qh)
        s2.sync()
        s2.enqueue(args.e2e_sweeps)
        ups = s2.sync()
        s2.get_state(out)
        el = time.perf_counter() - t0
        nst = args.e2e_sweeps
        e2e = {"value": ups / el, "unit": UNIT, "h2d_bytes_per_step": Qh.nbytes / nst,
               "d2h_bytes_per_step": (out.nbytes + 16) / nst,
               "note": "aw_load_state(host Q, with the pre-processing phase of the state) + aw_enqueue_sweeps + "
                       "aw_sync (update count) + aw_get_state(host Q), with the tile shapes of the device-timed "
                       f"run; mesh pre-processing ({t_mesh:.1f} s, once per mesh) excluded"}
        s2.close()

    cpu = None
    if rank == 0 and world == 1 and args.cpu_baseline:
        rate, info = cpu_sample(args.order, args.cpu_seconds, flux=args.flux)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": f"oracle (serial C, FP64) on a {info['n_tris']}-triangle graded disc with the same EP1 "
                         f"data and P{args.order} LTS scheme, {info['sweeps']} sweeps from t=0 "
                         f"({info['updates']} updates, {info['seconds']:.1f} s), pre-processing untimed"}
    if rank == 0:
        share_tot = sum(kms.values()) or 1.0
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {**explosion_config(args, n_tris, world),
                           "l2": "256 MiB write between timed sweeps (L2 is 129 MB)",
                           "updates_timed": int(updates_all), "sw_entries_per_elem": sizes["sw_entries"] / n_tris},
                "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": len(kms) * args.steps,
                "clocks": clk,
                "kernels": {k: {"ms": v, "share": v / share_tot} for k, v in kms.items()},
                "kernels_note": f"CUDA-event times over a second pass of {ksweeps} sweeps ({prof_updates} updates)",
                "tiles": tiles,
                "autotune_ms": {f"recon_half={k[0]},pred_wide={k[1]},bpsm={k[2]}": v for k, v in tune_ms.items()},
                "fp64_peak_gflops": peak_gflops}
        print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


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


def run_batched(args, rank=0, world=1):
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
    print(json.dumps(line), flush=True)


def run_adjoint(args):
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
        gQ, gX = dJ(s.get_elem())
        flush.fill_(float(k))
        e4.record(stream)
        s.adjoint(gQ, gX, None)
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
                       "l2": "256 MiB write before each timed pass"},
            "load_state_ms": ml, "sweeps_ms": mp, "forward_ms": ml + mp,
            "forward_with_checkpoints_ms": mf, "adjoint_ms": ma,
            "adjoint_over_forward": ma / (ml + mp), "adjoint_over_sweeps": ma / mp,
            "note": "forward = aw_load_state (pre-processing phase over every element) + the sweeps: the map "
                    "the gradient differentiates"}
    print(json.dumps(line), flush=True)


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
