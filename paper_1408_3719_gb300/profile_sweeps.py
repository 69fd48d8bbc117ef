"""A few sweeps of the explosion workload from a saved mid-run state, for
profiling the sweep kernels with few launches (a profiler replays every
captured launch; thousands of warm-up launches before it are costly).

    # the mid-run state: global steps until t_switch, local steps until every
    # element is past t_warm, saved with its tile shapes
    python -m paper_1408_3719_gb300.profile_sweeps --order 3 --hc 0.00114 --save /tmp/mid.npz
    # a profiled run: load it, run the sweeps, print each sweep's units
    python -m paper_1408_3719_gb300.profile_sweeps --order 3 --hc 0.00114 --load /tmp/mid.npz --sweeps 3

Each sweep prints one JSON line: its element updates and the space-time edge
surfaces it integrated (the units of the reconstruction / predictor and of
the flux kernel).  Every sweep is one launch of each of the eight sweep
kernels; loading the state launches k_products once.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1408_3719_gb300 import aleweno  # noqa: E402
from paper_1408_3719_gb300 import workloads as W  # noqa: E402

KEYS = ("Q", "QM", "HM", "t", "dt", "X", "count", "qhat")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--hc", type=float, default=0.00114)
    ap.add_argument("--t-switch", type=float, default=0.01)
    ap.add_argument("--t-warm", type=float, default=0.02)
    ap.add_argument("--tiles", default="1,1,4", help="recon_half,pred_wide,bpsm")
    ap.add_argument("--save", default=None)
    ap.add_argument("--load", default=None)
    ap.add_argument("--sweeps", type=int, default=3)
    a = ap.parse_args()
    mesh, Q = W.explosion(a.hc)
    cfg = dict(order_M=a.order, t_end=0.25, time_quantum_log2=20)
    if a.t_switch > 0:
        cfg.update(t_switch=a.t_switch, cfl_start=0.5)
    s = aleweno.Solver(**cfg)
    s.load_mesh(mesh)
    s.set_tiles(*[int(v) for v in a.tiles.split(",")])
    if a.load:
        z = np.load(a.load)
        s.set_elem({k: z[k] for k in KEYS})
        s.set_nodes(z["nX"], z["nt"])
    else:
        s.load_state(Q)
        t = np.empty(s.n_tris)
        while True:
            s.enqueue(200)
            s.sync()
            s.get_state(t=t)
            if t.min() >= a.t_warm:
                break
    if a.save:
        e, (nX, nt) = s.get_elem(), s.get_nodes()
        np.savez(a.save, nX=nX, nt=nt, **e)
    print(json.dumps({"n_tris": s.n_tris, "order": a.order}), flush=True)
    for k in range(a.sweeps):
        f0 = s.diag()["surfaces"]
        n = s.sweep()
        print(json.dumps({"sweep": k, "updates": n, "surfaces": s.diag()["surfaces"] - f0}), flush=True)
    s.close()


if __name__ == "__main__":
    main()
