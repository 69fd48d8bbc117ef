"""Seeded synthetic inputs: meshes and initial cell averages.

This module is the one piece of code that both the CUDA path and the CPU
oracle consume.  It holds no step of the ALE ADER-WENO scheme itself: it builds
triangulations (node coordinates, CCW connectivity, boundary tags, periodic
image shifts) and the initial cell averages Q_i^0 (the input of the
pre-processing phase, Sec. 2.6) by plain quadrature of a closed-form initial
condition.

The paper's meshes are not available, so each generator stands in for one of
the paper's workloads:

* ``shock_tube``   -- the Riemann problems of Sec. 3.2 (Sod, Table tab.iniRP2D)
                      on a jittered, randomly split 100x10 grid.
* ``vortex_grid``  -- the isentropic vortex of Sec. 3.1 (eqs. ShuVortIC,
                      ShuVortDelta, rhopressDelta) on a periodic jittered torus.
* ``disc``         -- the cylindrical explosions of Sec. 3.3 (Table
                      tab.iniEP2D) on a radially graded disc.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014), written out
below from its published definition.

Mesh dictionary keys (the layout the C ABI ``aw_load_mesh`` takes):
  xy     float64 [n_nodes, 2]
  tri    int32   [n_tris, 3]   counter-clockwise
  bc     int8    [n_tris, 3]   per local edge e = (v_e -> v_{e+1 mod 3}):
                               -1 interior, 0 slip wall, 1 transmissive
  shift  int8    [n_tris, 3, 2] periodic image of each corner (or None):
                               corner = xy[node] + shift * period
  period float64 [2] or None
"""
from __future__ import annotations

import math
import numpy as np

BC_INTERIOR = -1
BC_WALL = 0
BC_TRANSMISSIVE = 1

SEED_BASE = 1408371900

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


class SplitMix64:
    """splitmix64: state += golden gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + k * np.uint64(0x9E3779B97F4A7C15)
            self.state = self.state + np.uint64(n) * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


# ---------------------------------------------------------------------------
# topology helpers (boundary detection only; no scheme arithmetic)
# ---------------------------------------------------------------------------

def _boundary_edges(tri: np.ndarray) -> np.ndarray:
    """Boolean [n_tris, 3]: True where local edge e has no twin."""
    n = tri.shape[0]
    a = tri.reshape(-1)
    b = np.roll(tri, -1, axis=1).reshape(-1)
    key_fwd = a.astype(np.int64) * (1 << 32) + b.astype(np.int64)
    key_rev = b.astype(np.int64) * (1 << 32) + a.astype(np.int64)
    has_twin = np.isin(key_fwd, key_rev)
    return (~has_twin).reshape(n, 3)


def _signed_areas(xy, tri, shift=None, period=None):
    p = xy[tri]
    if shift is not None:
        p = p + shift.astype(np.float64) * np.asarray(period)[None, None, :]
    d1 = p[:, 1] - p[:, 0]
    d2 = p[:, 2] - p[:, 0]
    return 0.5 * (d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])


# ---------------------------------------------------------------------------
# generators
# ---------------------------------------------------------------------------

def shock_tube_mesh(nx: int = 100, ny: int = 10, lx: float = 1.0, ly: float = 0.1,
                    jitter: float = 0.2, seed: int = SEED_BASE + 0, diagonal: str = "short") -> dict:
    """Jittered structured grid on [0,lx]x[0,ly], slip walls on all four
    sides.  Each quad is split along its shorter diagonal (``diagonal="short"``,
    the Delaunay choice for these nearly square quads) or along a random one
    (``diagonal="random"``).  Random diagonals on the jittered grid produce
    occasional triangles with an angle near 140 degrees, which purely
    Lagrangian motion across a shock can invert."""
    rng = SplitMix64(seed)
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    xy = np.stack([ii * hx, jj * hy], axis=-1).reshape(-1, 2).astype(np.float64)
    interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).reshape(-1)
    nint = int(interior.sum())
    jx = rng.uniform(nint, -jitter * hx, jitter * hx)
    jy = rng.uniform(nint, -jitter * hy, jitter * hy)
    xy[interior, 0] += jx
    xy[interior, 1] += jy
    node = lambda i, j: i * (ny + 1) + j
    diag = rng.uniform(nx * ny) < 0.5
    tris = []
    q = 0
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = node(i, j), node(i + 1, j), node(i + 1, j + 1), node(i, j + 1)
            if diagonal == "short":
                use_ac = np.sum((xy[a] - xy[c]) ** 2) <= np.sum((xy[b] - xy[d]) ** 2)
            else:
                use_ac = diag[q]
            if use_ac:
                tris.append((a, b, c)); tris.append((a, c, d))
            else:
                tris.append((a, b, d)); tris.append((b, c, d))
            q += 1
    tri = np.asarray(tris, dtype=np.int32)
    bnd = _boundary_edges(tri)
    bc = np.where(bnd, BC_WALL, BC_INTERIOR).astype(np.int8)
    assert np.all(_signed_areas(xy, tri) > 0)
    return dict(xy=xy, tri=tri, bc=bc, shift=None, period=None,
                name=f"shock_tube_{nx}x{ny}")


def tube_mesh_periodic_y(nx: int = 211, ny: int = 21, x0: float = -0.5, lx: float = 1.0,
                         y0: float = -0.05, ly: float = 0.1, jitter: float = 0.1,
                         seed: int = SEED_BASE + 4) -> dict:
    """Jittered grid on [x0, x0+lx] x [y0, y0+ly], periodic in y and
    transmissive at both x ends (the set-up of the shock tubes of Sec. 3.2);
    every quad split along its shorter diagonal.  2 nx ny triangles; the
    default 211 x 21 gives the paper's N_E = 8862 at h ~ 1/200.  The default
    jitter (0.1 h: smallest angle 34 degrees) stands in for a generator's
    mesh for the tests."""
    rng = SplitMix64(seed)
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny), indexing="ij")
    xy = np.stack([x0 + ii * hx, y0 + jj * hy], axis=-1).reshape(-1, 2).astype(np.float64)
    inner_x = ((ii > 0) & (ii < nx)).reshape(-1)
    jx = rng.uniform(xy.shape[0], -jitter * hx, jitter * hx)
    jy = rng.uniform(xy.shape[0], -jitter * hy, jitter * hy)
    xy[inner_x, 0] += jx[inner_x]
    xy[:, 1] += jy
    period = np.array([0.0, ly])
    tris, shifts = [], []
    for i in range(nx):
        for j in range(ny):
            corners = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            ids = [ci * ny + (cj % ny) for ci, cj in corners]
            sh = [(0, cj // ny) for ci, cj in corners]
            P = [xy[k] + np.array(s_) * period for k, s_ in zip(ids, sh)]
            a, b, c, d = range(4)
            use_ac = np.sum((P[a] - P[c]) ** 2) <= np.sum((P[b] - P[d]) ** 2)
            pick = [(a, b, c), (a, c, d)] if use_ac else [(a, b, d), (b, c, d)]
            for t in pick:
                tris.append([ids[k] for k in t])
                shifts.append([sh[k] for k in t])
    tri = np.asarray(tris, dtype=np.int32)
    shift = np.asarray(shifts, dtype=np.int8)
    bnd = _boundary_edges(tri)
    bc = np.where(bnd, BC_TRANSMISSIVE, BC_INTERIOR).astype(np.int8)
    assert np.all(_signed_areas(xy, tri, shift, period) > 0)
    return dict(xy=xy, tri=tri, bc=bc, shift=shift, period=period,
                name=f"tube_periodic_y_{nx}x{ny}")


def vortex_grid_mesh(n: int, length: float = 10.0, jitter: float = 0.2,
                     seed: int = SEED_BASE + 1) -> dict:
    """Periodic n x n torus grid on [0,length]^2, every node jittered,
    random diagonals; 2 n^2 triangles."""
    rng = SplitMix64(seed)
    h = length / n
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xy = np.stack([ii * h, jj * h], axis=-1).reshape(-1, 2).astype(np.float64)
    xy[:, 0] += rng.uniform(n * n, -jitter * h, jitter * h)
    xy[:, 1] += rng.uniform(n * n, -jitter * h, jitter * h)
    diag = rng.uniform(n * n) < 0.5
    tris, shifts = [], []
    q = 0
    for i in range(n):
        for j in range(n):
            corners = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            ids = [(ci % n) * n + (cj % n) for ci, cj in corners]
            sh = [(ci // n, cj // n) for ci, cj in corners]
            a, b, c, d = range(4)
            pick = [(a, b, c), (a, c, d)] if diag[q] else [(a, b, d), (b, c, d)]
            for t in pick:
                tris.append([ids[k] for k in t])
                shifts.append([sh[k] for k in t])
            q += 1
    tri = np.asarray(tris, dtype=np.int32)
    shift = np.asarray(shifts, dtype=np.int8)
    period = np.array([length, length])
    bc = np.full(tri.shape, BC_INTERIOR, dtype=np.int8)
    assert not _boundary_edges(tri).any()
    assert np.all(_signed_areas(xy, tri, shift, period) > 0)
    return dict(xy=xy, tri=tri, bc=bc, shift=shift, period=period,
                name=f"vortex_torus_{n}")


def disc_mesh(h_centre: float, grading: float = 10.0, radius: float = 1.0,
              seed: int = SEED_BASE + 2, layer: float = 0.866, hfun=None) -> dict:
    """Graded disc of the given radius: concentric rings with spacing
    h(r) = h_centre * grading**(r/radius) (or the given ``hfun(r)``),
    stitched by angular merge; a fan closes the centre.  Transmissive rim."""
    rng = SplitMix64(seed)
    if hfun is None:
        hfun = lambda r: h_centre * grading ** (r / radius)
    radii = [0.0]
    r = hfun(0.0)
    while r < radius:
        radii.append(r)
        r = r + layer * hfun(r)
    # stretch so the last ring sits on the rim
    radii = np.asarray(radii[1:] + [radius])
    if len(radii) > 1 and radii[-1] - radii[-2] < 0.5 * layer * hfun(radius):
        radii = np.delete(radii, -2)
    counts = [max(6, int(round(2 * math.pi * rk / hfun(rk)))) for rk in radii]
    phases = rng.uniform(len(radii))
    xy = [np.zeros((1, 2))]
    ring_start = []
    start = 1
    ring_angles = []
    for rk, nk, ph in zip(radii, counts, phases):
        ang = (ph + np.arange(nk)) * (2 * math.pi / nk)
        xy.append(np.stack([rk * np.cos(ang), rk * np.sin(ang)], axis=-1))
        ring_start.append(start)
        ring_angles.append(ang)
        start += nk
    xy = np.concatenate(xy, axis=0)
    tris = []
    # centre fan
    n0, s0 = counts[0], ring_start[0]
    for m in range(n0):
        tris.append((0, s0 + m, s0 + (m + 1) % n0))
    # ring stitching
    for k in range(len(radii) - 1):
        na, nb = counts[k], counts[k + 1]
        sa, sb = ring_start[k], ring_start[k + 1]
        a_ang = ring_angles[k]
        b_ang = ring_angles[k + 1]
        # outer start j0 with b(j0) <= a(0) < b(j0) + 2pi/nb
        db = 2 * math.pi / nb
        da = 2 * math.pi / na
        a0 = a_ang[0]
        jshift = int(math.floor((a0 - b_ang[0]) / db))
        bang = lambda j: b_ang[0] + (j + jshift) * db
        aang = lambda i: a0 + i * da
        i = j = 0
        while i < na or j < nb:
            adv_a = (j >= nb) or (i < na and aang(i + 1) <= bang(j + 1))
            A_i = sa + i % na
            B_j = sb + (j + jshift) % nb
            if adv_a:
                tris.append((A_i, B_j, sa + (i + 1) % na)); i += 1
            else:
                tris.append((A_i, B_j, sb + (j + 1 + jshift) % nb)); j += 1
    tri = np.asarray(tris, dtype=np.int32)
    bnd = _boundary_edges(tri)
    bc = np.where(bnd, BC_TRANSMISSIVE, BC_INTERIOR).astype(np.int8)
    assert np.all(_signed_areas(xy, tri) > 0)
    return dict(xy=xy, tri=tri, bc=bc, shift=None, period=None,
                name=f"disc_{tri.shape[0]}")


# ---------------------------------------------------------------------------
# initial conditions (closed forms) and their cell averages
# ---------------------------------------------------------------------------

def prim_to_cons(rho, u, v, p, gamma):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=-1)


def _corner_coords(mesh):
    p = mesh["xy"][mesh["tri"]]
    if mesh["shift"] is not None:
        p = p + mesh["shift"].astype(np.float64) * np.asarray(mesh["period"])[None, None, :]
    return p  # [n, 3, 2]


def _gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _duffy_rule(n):
    """Points (barycentric weights of vertices 1 and 2) and weights that sum
    to 1 for averaging over a triangle; exact for degree 2n-2."""
    x, w = _gauss_legendre01(n)
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    s = (u * (1 - v)).reshape(-1)
    t = v.reshape(-1)
    ww = (wu * wv * (1 - v)).reshape(-1) * 2.0
    return s, t, ww


def _subtriangle_rule(k):
    """Centroids of the k^2 congruent sub-triangles (midpoint rule),
    for piecewise-constant data; weights sum to 1."""
    pts = []
    for i in range(k):
        for j in range(k - i):
            pts.append(((i + 1 / 3) / k, (j + 1 / 3) / k))
            if i + j < k - 1:
                pts.append(((i + 2 / 3) / k, (j + 2 / 3) / k))
    pts = np.asarray(pts)
    return pts[:, 0], pts[:, 1], np.full(len(pts), 1.0 / len(pts))


def cell_average(mesh, fun, rule):
    """Average of fun(x, y) -> [.., 4] over each triangle with a barycentric rule."""
    s, t, w = rule
    p = _corner_coords(mesh)
    x0 = p[:, 0][:, None, :]
    d1 = (p[:, 1] - p[:, 0])[:, None, :]
    d2 = (p[:, 2] - p[:, 0])[:, None, :]
    pts = x0 + s[None, :, None] * d1 + t[None, :, None] * d2  # [n, q, 2]
    vals = fun(pts[..., 0], pts[..., 1])  # [n, q, 4]
    return np.einsum("nqv,q->nv", vals, w)


def riemann_state(x, y, left, right, x_d, gamma):
    """Primitive (rho,u,v,p) left of x_d and right of it, as conserved."""
    ql = prim_to_cons(*[np.float64(c) for c in left], gamma)
    qr = prim_to_cons(*[np.float64(c) for c in right], gamma)
    m = (x < x_d)[..., None]
    return np.where(m, ql, qr)


def explosion_state(x, y, inner, outer, radius, gamma):
    qi = prim_to_cons(*[np.float64(c) for c in inner], gamma)
    qo = prim_to_cons(*[np.float64(c) for c in outer], gamma)
    m = ((x * x + y * y) < radius * radius)[..., None]
    return np.where(m, qi, qo)


def vortex_prim(x, y, gamma=1.4, eps=5.0, centre=(5.0, 5.0), background=(1.0, 0.0, 0.0, 1.0)):
    """Isentropic vortex, eqs. ShuVortIC, ShuVortDelta, rhopressDelta."""
    dx, dy = x - centre[0], y - centre[1]
    r2 = dx * dx + dy * dy
    du = eps / (2 * math.pi) * np.exp(0.5 * (1 - r2)) * (-dy)
    dv = eps / (2 * math.pi) * np.exp(0.5 * (1 - r2)) * dx
    dT = -(gamma - 1) * eps * eps / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
    rho = background[0] * 0 + (1 + dT) ** (1 / (gamma - 1))
    p = (1 + dT) ** (gamma / (gamma - 1))
    return rho, background[1] + du, background[2] + dv, p


def vortex_state(x, y, gamma=1.4, period=None):
    if period is not None:
        # nearest periodic image of the centre
        x = np.mod(x - 5.0 + 0.5 * period[0], period[0]) + 5.0 - 0.5 * period[0]
        y = np.mod(y - 5.0 + 0.5 * period[1], period[1]) + 5.0 - 0.5 * period[1]
    return prim_to_cons(*vortex_prim(x, y, gamma), gamma)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def sod_tube(nx=100, ny=10, seed=SEED_BASE + 0, gamma=1.4):
    """Sod shock tube on [0,1]x[0,0.1]: left (1,0,0,1), right (0.125,0,0,0.1) at x=0.5."""
    mesh = shock_tube_mesh(nx, ny, 1.0, 0.1, seed=seed)
    q = cell_average(mesh, lambda x, y: riemann_state(x, y, (1, 0, 0, 1), (0.125, 0, 0, 0.1), 0.5, gamma),
                     _subtriangle_rule(16))
    return mesh, q


def vortex(n, seed=SEED_BASE + 1, gamma=1.4):
    mesh = vortex_grid_mesh(n, seed=seed)
    q = cell_average(mesh, lambda x, y: vortex_state(x, y, gamma, mesh["period"]), _duffy_rule(8))
    return mesh, q


def explosion(h_centre, seed=SEED_BASE + 2, gamma=1.4, inner=(1, 0, 0, 1), outer=(0.125, 0, 0, 0.1),
              radius=0.5, grading=10.0):
    mesh = disc_mesh(h_centre, grading=grading, seed=seed)
    q = cell_average(mesh, lambda x, y: explosion_state(x, y, inner, outer, radius, gamma),
                     _subtriangle_rule(16))
    return mesh, q


# Table tab.iniRP2D: primitive (rho, u, v, p) left and right of x_d = 0, final time
RIEMANN_PROBLEMS = {
    "RP1": ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 0.2),
    "RP2": ((0.445, 0.698, 0.0, 3.528), (0.5, 0.0, 0.0, 0.571), 0.1),
}

# Table tab.iniEP2D: primitive inner (r < 0.5) and outer states, final time
# (EP1's final time is 0.2 in the table and 0.25 in the caption of its figure)
EXPLOSION_PROBLEMS = {
    "EP1": ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 0.25),
    "EP2": ((1.0, 0.0, 0.0, 1000.0), (1.0, 0.0, 0.0, 0.01), 0.012),
}


def riemann_problem(case="RP1", nx=211, ny=21, seed=SEED_BASE + 4, gamma=1.4, jitter=0.0):
    """The shock tubes of Sec. 3.2 as the paper sets them up: [-0.5, 0.5] x
    [-0.05, 0.05], periodic in y, transmissive in x, discontinuity at x = 0;
    returns (mesh, Q, t_end).  The default grid is unjittered: under the
    Osher-type flux, RP2 at third order collapses single elements behind its
    shock on grids jittered by 0.05 h or more (RP1 by 0.2 h)."""
    left, right, t_end = RIEMANN_PROBLEMS[case]
    mesh = tube_mesh_periodic_y(nx, ny, seed=seed, jitter=jitter)
    q = cell_average(mesh, lambda x, y: riemann_state(x, y, left, right, 0.0, gamma), _subtriangle_rule(16))
    return mesh, q, t_end


def disc_m1_mesh(scale=0.86, seed=SEED_BASE + 5):
    """Stand-in for the paper's mesh m1 of Sec. 3.3: unit disc with size
    h = 1/100 for r <= 0.5 and 1/50 beyond r = 0.53 (linear in between, so
    that no triangle at the interface is worse than elsewhere: smallest angle
    28 degrees), both multiplied by ``scale``; the default gives 44,097
    triangles (the paper: N_E = 43756)."""
    return disc_mesh(0.0, seed=seed,
                     hfun=lambda r: scale * (0.01 if r <= 0.5 else 0.01 + 0.01 * min(1.0, (r - 0.5) / 0.03)))


def explosion_problem(case="EP1", scale=0.86, seed=SEED_BASE + 5, gamma=1.4):
    """The explosions of Sec. 3.3 on the m1 stand-in; returns (mesh, Q, t_end)."""
    inner, outer, t_end = EXPLOSION_PROBLEMS[case]
    mesh = disc_m1_mesh(scale, seed)
    q = cell_average(mesh, lambda x, y: explosion_state(x, y, inner, outer, 0.5, gamma), _subtriangle_rule(16))
    return mesh, q, t_end


BC_MOVING_WALL = 2


def saltzman(nx=100, ny=10, gamma=5.0 / 3.0, e0=1e-4):
    """The Saltzman piston problem of Sec. 3.5: 100 x 10 squares on
    [0, 1] x [0, 0.1], each split into two right triangles, skewed by
    x' = x + (0.1 - y) sin(pi x); gas at rest with rho = 1 and internal
    energy e0; the left side is a slip wall moving with velocity (1, 0)
    (tag 2), the other sides fixed slip walls.  Returns (mesh, Q)."""
    mesh = shock_tube_mesh(nx, ny, 1.0, 0.1, jitter=0.0, seed=SEED_BASE + 6)
    xy = mesh["xy"]
    xy[:, 0] = xy[:, 0] + (0.1 - xy[:, 1]) * np.sin(np.pi * xy[:, 0])
    P = _corner_coords(mesh)
    bc = mesh["bc"].copy()
    for i, e in zip(*np.nonzero(bc == BC_WALL)):
        a, b = P[i, e], P[i, (e + 1) % 3]
        if abs(a[0]) < 1e-12 and abs(b[0]) < 1e-12:
            bc[i, e] = BC_MOVING_WALL
    assert np.all(_signed_areas(xy, mesh["tri"]) > 0)
    mesh = dict(mesh, xy=xy, bc=bc, name=f"saltzman_{nx}x{ny}")
    q = np.tile(prim_to_cons(1.0, 0.0, 0.0, (gamma - 1.0) * e0, gamma), (mesh["tri"].shape[0], 1))
    return mesh, q


def piston_shock(u_p=1.0, rho0=1.0, p0=(5.0 / 3.0 - 1.0) * 1e-4, gamma=5.0 / 3.0):
    """Exact state behind the shock driven by a piston of speed u_p into gas
    at rest (Rankine-Hugoniot): returns (shock speed, rho1, p1)."""
    c0 = math.sqrt(gamma * p0 / rho0)
    a = 0.25 * (gamma + 1.0) * u_p
    s = a + math.sqrt(a * a + c0 * c0)
    rho1 = rho0 * s / (s - u_p)
    p1 = p0 + rho0 * s * u_p
    return s, rho1, p1


BC_KIDDER = 3
KIDDER = (0.9, 1.0, 1.0, 2.0, 1.0)  # r_i0, r_e0, rho_i0, rho_e0, s0 (Sec. 3.4), gamma = 2


def kidder_tau(kidder=KIDDER, gamma=2.0):
    """Focalisation time of the Kidder compression (Sec. 3.4)."""
    ri, re, rhoi, rhoe, s0 = kidder
    ci2, ce2 = gamma * s0 * rhoi ** (gamma - 1.0), gamma * s0 * rhoe ** (gamma - 1.0)
    return math.sqrt(0.5 * (gamma - 1.0) * (re * re - ri * ri) / (ce2 - ci2))


def kidder_prim(x, y, t, kidder=KIDDER, gamma=2.0):
    """Exact primitive state (rho, u, v, p) of the Kidder compression at
    (x, y, t) (eqs. KidderIC, KidderEx): homothety h(t) = sqrt(1 - t^2/tau^2),
    density rho0(R/h)/h^2, radial velocity h' R/h, pressure s0 rho^gamma."""
    ri, re, rhoi, rhoe, s0 = kidder
    tau = kidder_tau(kidder, gamma)
    h = math.sqrt(1.0 - t * t / (tau * tau))
    dh = -t / (tau * tau * h)
    r = np.hypot(x, y) / h
    w = (r * r - ri * ri) / (re * re - ri * ri)
    rho = ((1.0 - w) * rhoi ** (gamma - 1.0) + w * rhoe ** (gamma - 1.0)) ** (1.0 / (gamma - 1.0)) / (h * h)
    return rho, dh / h * x, dh / h * y, s0 * rho ** gamma


def kidder(nr=10, nth=120, kidder=KIDDER, gamma=2.0):
    """The Kidder problem of Sec. 3.4: the quarter shell r_i0 <= r <= r_e0,
    0 <= theta <= pi/2 on an nr x nth polar grid (each cell split along its
    shorter diagonal), slip walls on the two straight sides, the exact state
    (tag 3) on the two arcs; cell averages of the exact state at t = 0.
    Returns (mesh, Q, t_f) with t_f = sqrt(3)/2 tau, where h(t_f) = 1/2."""
    ri, re = kidder[0], kidder[1]
    rr = np.linspace(ri, re, nr + 1)
    th = np.linspace(0.0, 0.5 * math.pi, nth + 1)
    R, TH = np.meshgrid(rr, th, indexing="ij")
    xy = np.stack([R * np.cos(TH), R * np.sin(TH)], axis=-1).reshape(-1, 2)
    xy[np.abs(xy) < 1e-15] = 0.0
    node = lambda i, j: i * (nth + 1) + j
    tris = []
    for i in range(nr):
        for j in range(nth):
            a, b, c, d = node(i, j), node(i + 1, j), node(i + 1, j + 1), node(i, j + 1)
            if np.sum((xy[a] - xy[c]) ** 2) <= np.sum((xy[b] - xy[d]) ** 2):
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    tri = np.asarray(tris, dtype=np.int32)
    assert np.all(_signed_areas(xy, tri) > 0)
    bnd = _boundary_edges(tri)
    bc = np.full(tri.shape, BC_INTERIOR, dtype=np.int8)
    P = xy[tri]
    for i, e in zip(*np.nonzero(bnd)):
        a, b = P[i, e], P[i, (e + 1) % 3]
        ra, rb = np.hypot(*a), np.hypot(*b)
        arc = (abs(ra - ri) < 1e-12 and abs(rb - ri) < 1e-12) or (abs(ra - re) < 1e-12 and abs(rb - re) < 1e-12)
        bc[i, e] = BC_KIDDER if arc else BC_WALL
    mesh = dict(xy=xy, tri=tri, bc=bc, shift=None, period=None, name=f"kidder_{nr}x{nth}")
    q = cell_average(mesh, lambda x, y: prim_to_cons(*kidder_prim(x, y, 0.0, kidder, gamma), gamma), _duffy_rule(8))
    return mesh, q, 0.5 * math.sqrt(3.0) * kidder_tau(kidder, gamma)


def batched_instances(n_inst=256, lo=2000, hi=60000, seed=SEED_BASE + 3, gamma=1.4, size_scale=1.0):
    """Independent explosion / shock-tube instances with log-uniform sizes,
    density ratio U[2,10], pressure ratio U[2,20], interface U[0.3,0.6]."""
    rng = SplitMix64(seed)
    kinds = rng.uniform(n_inst) < 0.5
    sizes = np.exp(rng.uniform(n_inst, math.log(lo), math.log(hi))) * size_scale
    dr = rng.uniform(n_inst, 2.0, 10.0)
    pr = rng.uniform(n_inst, 2.0, 20.0)
    xd = rng.uniform(n_inst, 0.3, 0.6)
    out = []
    for k in range(n_inst):
        inner = (1.0, 0.0, 0.0, 1.0)
        outer = (1.0 / dr[k], 0.0, 0.0, 1.0 / pr[k])
        if kinds[k]:
            hc = math.sqrt(0.646 / sizes[k])
            mesh = disc_mesh(hc, seed=seed + 1000 + k)
            q = cell_average(mesh, lambda x, y: explosion_state(x, y, inner, outer, xd[k], gamma),
                             _subtriangle_rule(8))
            t_end = 0.25
        else:
            nx = max(10, int(round(sizes[k] / 20.0)))
            mesh = shock_tube_mesh(nx, 10, 1.0, 10.0 / nx, seed=seed + 1000 + k)
            q = cell_average(mesh, lambda x, y: riemann_state(x, y, inner, outer, xd[k], gamma),
                             _subtriangle_rule(8))
            t_end = 0.2
        out.append(dict(mesh=mesh, q=q, t_end=t_end, kind="explosion" if kinds[k] else "tube"))
    return out
