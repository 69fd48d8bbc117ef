"""Full runs of the paper's test configurations on the GPU library.

    python -m paper_1408_3719_gb300.runs sod [--gts] [--order 1]
    python -m paper_1408_3719_gb300.runs vortex --n 45 90 179 [--order 3]
    python -m paper_1408_3719_gb300.runs explosion [--order 2] [--hc 0.00114] [--gts]
                                                   [--cfl 0.5] [--t-switch T --cfl-start C]

``--flux osher`` selects the Osher-type ALE flux instead of the Rusanov-type
one for any case.

The paper's own set-ups (third order = P2, Osher-type flux, LTS and GTS):

    python -m paper_1408_3719_gb300.runs rp --problem RP1|RP2 [--gts]
    python -m paper_1408_3719_gb300.runs ep --problem EP1|EP2 [--gts] [--t-end 0.2]
    python -m paper_1408_3719_gb300.runs table
    python -m paper_1408_3719_gb300.runs saltzman [--gts]   (Rusanov-type flux, Sec. 3.5)
    python -m paper_1408_3719_gb300.runs kidder [--gts]     (fourth order, Sec. 3.4)

``table`` runs RP1, RP2, EP1 and EP2 with both time-stepping modes and prints
the update counts beside those of Tables tab.RPdata and tab.EPdata.

Each prints one JSON line per run: element updates, productive sweeps, wall
time, updates/s, and the accuracy measure of the configuration (density L1
error against the exact Riemann solution for the shock tube, Sec. 3.2; L2
error of the density cell averages against the exact stationary vortex,
Sec. 3.1).  The inputs are the seeded synthetic workloads of
``paper_1408_3719_gb300.workloads``.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import aleweno
from . import exact
from . import radial
from . import workloads as W

# element updates to the final time printed in Tables tab.RPdata and tab.EPdata
# (third-order scheme, Osher-type flux): (GTS, LTS)
PAPER_UPDATES = {"RP1": (10.120404e6, 3.257847e6), "RP2": (23.349964e6, 5.020780e6),
                 "EP1": (30.804224e6, 12.206887e6), "EP2": (181.412376e6, 38.274477e6)}


def _areas(X):
    return 0.5 * ((X[:, 2] - X[:, 0]) * (X[:, 5] - X[:, 1]) - (X[:, 3] - X[:, 1]) * (X[:, 4] - X[:, 0]))


def _run(mesh, Q, **cfg):
    s = aleweno.Solver(**cfg)
    t0 = time.perf_counter()
    s.load_mesh(mesh)
    t1 = time.perf_counter()
    s.load_state(Q)
    try:
        sweeps, updates = s.advance()
    except aleweno.AwError as err:
        e = s.get_elem()
        fail = dict(error=str(err), t_min=float(e["t"].min() * s.tick), t_max=float(e["t"].max() * s.tick),
                    updates=int(e["count"].sum()))
        if "element" in str(err):
            i = int(str(err).split("element ")[1].split()[0])
            X = e["X"][i]
            fail.update(elem=i, t_elem=float(e["t"][i] * s.tick), Q=e["Q"][i].tolist(), X=X.tolist(),
                        area=float(_areas(X[None])[0]), r=float(np.linalg.norm(X.reshape(3, 2).mean(0))))
        s.close()
        raise RuntimeError(json.dumps(fail)) from err
    t2 = time.perf_counter()
    e = s.get_elem()
    info = dict(n_tris=int(mesh["tri"].shape[0]), order_M=cfg.get("order_M"), gts=bool(cfg.get("gts", False)),
                flux=cfg.get("flux", "rusanov"),
                sweeps=sweeps, updates=updates, setup_s=t1 - t0, run_s=t2 - t1,
                updates_per_s=updates / max(t2 - t1, 1e-12), gcl_max=s.diag()["gcl_max"])
    s.close()
    return e, info


def sod(order=1, gts=True, nx=100, ny=10, flux="rusanov"):
    mesh, Q = W.sod_tube(nx, ny)
    e, info = _run(mesh, Q, order_M=order, t_end=0.2, gts=gts, flux=flux)
    A = _areas(e["X"])
    cx = e["X"].reshape(-1, 3, 2).mean(1)[:, 0]
    ex = exact.sample(cx, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1))
    info.update(config="Sod tube", l1_rho=float(np.sum(np.abs(e["Q"][:, 0] - ex[:, 0]) * A) / A.sum()))
    return info


def vortex(n, order=3, gts=False, flux="rusanov"):
    mesh, Q = W.vortex(n)
    e, info = _run(mesh, Q, order_M=order, t_end=1.0, gts=gts, flux=flux)
    x, w = np.polynomial.legendre.leggauss(6)
    x, w = 0.5 * (x + 1), 0.5 * w
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    s_, t_, w_ = (u * (1 - v)).ravel(), v.ravel(), (2 * wu * wv * (1 - v)).ravel()
    P = e["X"].reshape(-1, 3, 2)
    pts = P[:, 0][:, None] + s_[None, :, None] * (P[:, 1] - P[:, 0])[:, None] + t_[None, :, None] * (P[:, 2] - P[:, 0])[:, None]
    ex = np.einsum("nqv,q->nv", W.vortex_state(pts[..., 0], pts[..., 1], 1.4, mesh["period"]), w_)
    A = _areas(e["X"])
    Pd = P[:, [0, 1, 2, 0]]
    d = np.linalg.norm(np.diff(Pd, axis=1), axis=2)
    circ = d.prod(1) / (2.0 * A)  # circumcircle diameter a b c / (2 |T|)
    info.update(config="isentropic vortex", n=n, l2_rho=float(math.sqrt(np.sum(A * (e["Q"][:, 0] - ex[:, 0]) ** 2))),
                h_max_circumdiameter=float(circ.max()))
    return info


def explosion(order=2, hc=0.00114, gts=False, flux="rusanov", cfl=0.5, t_switch=0.0, cfl_start=0.0):
    """The cylindrical explosion on the graded disc.  ``t_switch`` > 0 starts
    the run with global steps of CFL ``cfl_start`` up to that time, then local
    steps (the start-up the paper gives its piston problem, Sec. 3.5)."""
    mesh, Q = W.explosion(hc)
    e, info = _run(mesh, Q, order_M=order, t_end=0.25, gts=gts, flux=flux, cfl=cfl,
                   t_switch=t_switch, cfl_start=cfl_start)
    r = np.linalg.norm(e["X"].reshape(-1, 3, 2).mean(1), axis=1)
    info.update(config="explosion EP1", cfl=cfl, t_switch=t_switch, cfl_start=cfl_start,
                rho_max=float(e["Q"][:, 0].max()), r_max=float(r.max()))
    return info


def riemann(case="RP1", order=2, gts=False, flux="osher", jitter=0.0, cfl=0.5):
    """A shock tube of Sec. 3.2 as the paper sets it up; density L1 error of
    the averages against the exact solution, weighted by area."""
    mesh, Q, t_end = W.riemann_problem(case, jitter=jitter)
    e, info = _run(mesh, Q, order_M=order, t_end=t_end, gts=gts, flux=flux, cfl=cfl)
    A = _areas(e["X"])
    cx = e["X"].reshape(-1, 3, 2).mean(1)[:, 0]
    left, right, _ = W.RIEMANN_PROBLEMS[case]
    ex = exact.sample(cx, t_end, 0.0, (left[0], left[1], left[3]), (right[0], right[1], right[3]))
    info.update(config=case, t_end=t_end, jitter=jitter,
                l1_rho=float(np.sum(np.abs(e["Q"][:, 0] - ex[:, 0]) * A) / A.sum()),
                paper_updates=PAPER_UPDATES[case][0 if gts else 1])
    return info


_REFERENCE = {}


def _radial_reference(case, t_end, n):
    key = (case, t_end, n)
    if key not in _REFERENCE:
        inner, outer, _ = W.EXPLOSION_PROBLEMS[case]
        _REFERENCE[key] = radial.solve((inner[0], inner[1], inner[3]), (outer[0], outer[1], outer[3]),
                                       r_d=0.5, t_end=t_end, n=n)
    return _REFERENCE[key]


def explosion_paper(case="EP1", order=2, gts=False, flux="osher", t_end=None, n_ref=15000, cfl=0.5,
                    t_switch=0.0, cfl_start=0.0):
    """An explosion of Sec. 3.3 on the stand-in for mesh m1; density and
    pressure L1 differences (area-weighted) against the 1D radial reference
    solution of eqs. inhomEuler on n_ref points, sampled at the centroids.
    ``t_switch`` > 0: global steps of CFL ``cfl_start`` until then."""
    mesh, Q, t_def = W.explosion_problem(case)
    t_end = t_def if t_end is None else t_end
    e, info = _run(mesh, Q, order_M=order, t_end=t_end, gts=gts, flux=flux, cfl=cfl, t_switch=t_switch,
                   cfl_start=cfl_start)
    A = _areas(e["X"])
    rc = np.linalg.norm(e["X"].reshape(-1, 3, 2).mean(1), axis=1)
    r, rho, u, p = _radial_reference(case, t_end, n_ref)
    g = 1.4
    q = e["Q"]
    pr = (g - 1) * (q[:, 3] - 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2) / q[:, 0])
    d_rho = np.abs(q[:, 0] - radial.sample(rc, r, rho))
    d_p = np.abs(pr - radial.sample(rc, r, p))
    info.update(config=case, t_end=t_end, l1_rho_vs_radial=float(np.sum(d_rho * A) / A.sum()),
                l1_p_vs_radial=float(np.sum(d_p * A) / A.sum()), rho_max=float(q[:, 0].max()),
                rho_max_radial=float(rho.max()), r_max=float(rc.max()),
                paper_updates=PAPER_UPDATES[case][0 if gts else 1])
    return info


def saltzman(order=2, gts=False, flux="rusanov", t_end=0.6, cfl=0.5):
    """The Saltzman piston of Sec. 3.5: third order, Rusanov-type flux, global
    steps with CFL 0.1 until t = 0.01, then local (or global) steps with CFL
    ``cfl``; density and velocity L1 errors against the exact piston shock."""
    mesh, Q = W.saltzman()
    g = 5.0 / 3.0
    e, info = _run(mesh, Q, order_M=order, gamma=g, t_end=t_end, gts=gts, flux=flux, wall_velocity=(1.0, 0.0),
                   t_switch=0.01, cfl_start=0.1, cfl=cfl)
    A = _areas(e["X"])
    cx = e["X"].reshape(-1, 3, 2).mean(1)[:, 0]
    s, rho1, _ = W.piston_shock()
    behind = cx < s * t_end
    rho_ex = np.where(behind, rho1, 1.0)
    u_ex = np.where(behind, 1.0, 0.0)
    q = e["Q"]
    info.update(config="Saltzman", t_end=t_end, l1_rho=float(np.sum(np.abs(q[:, 0] - rho_ex) * A) / A.sum()),
                l1_u=float(np.sum(np.abs(q[:, 1] / q[:, 0] - u_ex) * A) / A.sum()), shock_x=float(s * t_end))
    return info


# Table tab.Kidder: frontier radii at t_f (fourth order, Osher-type flux)
PAPER_KIDDER = {"inner": (0.45, 0.44996063, 3.94e-05), "outer": (0.5, 0.49930053, 6.99e-04)}


def kidder(order=3, gts=False, flux="osher", nr=10, nth=120):
    """The Kidder compression of Sec. 3.4 to t_f = sqrt(3)/2 tau: the radii of
    the inner and outer frontier (mean over their nodes) against the exact
    0.45 and 0.5, and the density's L1 error against the exact solution."""
    mesh, Q, tf = W.kidder(nr, nth)
    s = aleweno.Solver(order_M=order, gamma=2.0, t_end=tf, gts=gts, flux=flux)
    s.load_mesh(mesh)
    s.load_state(Q)
    t0 = time.perf_counter()
    sweeps, updates = s.advance()
    run_s = time.perf_counter() - t0
    X, _ = s.get_nodes()
    e = s.get_elem()
    s.close()
    r0 = np.hypot(*mesh["xy"].T)
    rn = np.hypot(*X.T)
    r_in, r_out = float(rn[np.abs(r0 - 0.9) < 1e-12].mean()), float(rn[np.abs(r0 - 1.0) < 1e-12].mean())
    A = _areas(e["X"])
    c = e["X"].reshape(-1, 3, 2).mean(1)
    rho_ex = W.kidder_prim(c[:, 0], c[:, 1], tf)[0]
    return dict(config="Kidder", n_tris=int(mesh["tri"].shape[0]), order_M=order, gts=gts, flux=flux, t_end=tf,
                sweeps=sweeps, updates=updates, run_s=run_s, r_inner=r_in, r_outer=r_out,
                err_inner=abs(r_in - 0.45), err_outer=abs(r_out - 0.5),
                l1_rho_rel=float(np.sum(np.abs(e["Q"][:, 0] - rho_ex) * A) / np.sum(rho_ex * A)),
                paper=PAPER_KIDDER)


def table(order=2, flux="osher"):
    """GTS and LTS update counts of RP1, RP2, EP1, EP2 beside the paper's."""
    out = []
    # EP1 twice: its final time is 0.2 in Table tab.iniEP2D, 0.25 in its figure
    for case, t_end in (("RP1", None), ("RP2", None), ("EP1", 0.2), ("EP1", 0.25), ("EP2", None)):
        runs = {}
        for gts in (True, False):
            try:
                runs[gts] = riemann(case, order, gts, flux) if case.startswith("RP") else \
                    explosion_paper(case, order, gts, flux, t_end)
            except RuntimeError as err:
                runs[gts] = dict(config=case, gts=gts, failed=str(err)[:400])
            print(json.dumps(runs[gts]), flush=True)
        if "updates" in runs[True] and "updates" in runs[False]:
            pg, pl = PAPER_UPDATES[case]
            row = dict(config=case, t_end=runs[False]["t_end"], gts_updates=runs[True]["updates"],
                       lts_updates=runs[False]["updates"],
                       ratio=runs[True]["updates"] / runs[False]["updates"], paper_gts=pg, paper_lts=pl,
                       paper_ratio=pg / pl, n_tris=runs[False]["n_tris"])
            print(json.dumps(row), flush=True)
            out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["sod", "vortex", "explosion", "rp", "ep", "table", "saltzman", "kidder"])
    ap.add_argument("--problem", default=None, help="RP1 | RP2 (rp), EP1 | EP2 (ep)")
    ap.add_argument("--t-end", type=float, default=None)
    ap.add_argument("--order", type=int, default=None)
    ap.add_argument("--gts", action="store_true")
    ap.add_argument("--n", type=int, nargs="+", default=[45, 90, 179])
    ap.add_argument("--hc", type=float, default=0.00114)
    ap.add_argument("--cfl", type=float, default=0.5,
                    help="explosion, rp, ep, saltzman: CFL number of eq. timestep (saltzman: after its start-up)")
    ap.add_argument("--t-switch", type=float, default=0.0,
                    help="explosion, ep: global steps until this time, then local steps")
    ap.add_argument("--cfl-start", type=float, default=0.0, help="explosion, ep: CFL of the start-up steps")
    ap.add_argument("--flux", default=None, choices=["rusanov", "osher"],
                    help="default: rusanov for sod/vortex/explosion, osher (the paper's) for rp/ep/table")
    a = ap.parse_args()
    aleweno.load()
    paper = a.case in ("rp", "ep", "table")
    flux = a.flux or ("osher" if paper else "rusanov")
    if a.case == "kidder":
        print(json.dumps(kidder(a.order or 3, a.gts, a.flux or "osher")), flush=True)
    elif a.case == "saltzman":
        try:
            print(json.dumps(saltzman(a.order or 2, a.gts, a.flux or "rusanov", a.t_end or 0.6, a.cfl)), flush=True)
        except RuntimeError as err:
            print(json.dumps(dict(config="Saltzman", gts=a.gts, failed=str(err)[:600])), flush=True)
    elif a.case == "rp":
        print(json.dumps(riemann(a.problem or "RP1", a.order or 2, a.gts, flux, cfl=a.cfl)), flush=True)
    elif a.case == "ep":
        print(json.dumps(explosion_paper(a.problem or "EP1", a.order or 2, a.gts, flux, a.t_end, cfl=a.cfl,
                                         t_switch=a.t_switch, cfl_start=a.cfl_start or a.cfl)), flush=True)
    elif a.case == "table":
        table(a.order or 2, flux)
    elif a.case == "sod":
        print(json.dumps(sod(a.order or 1, a.gts, flux=flux)), flush=True)
    elif a.case == "vortex":
        prev = None
        for n in a.n:
            r = vortex(n, a.order or 3, a.gts, flux)
            if prev:
                r["order_vs_previous"] = math.log(prev["l2_rho"] / r["l2_rho"]) / math.log(
                    r["h_max_circumdiameter"] / prev["h_max_circumdiameter"]) * -1
            print(json.dumps(r), flush=True)
            prev = r
    else:
        print(json.dumps(explosion(a.order or 2, a.hc, a.gts, flux, a.cfl, a.t_switch, a.cfl_start or a.cfl)),
              flush=True)


if __name__ == "__main__":
    main()
