"""The hand-written adjoint of the LTS sweep map, for the schedule a run takes
(ready sets and integer time steps held fixed, stencils of the loaded mesh
kept), against central finite differences: of the GPU path itself with the
recorded schedule replayed, and of the oracle with its own recorded schedule
replayed.  Objective: kinetic energy of the elements whose initial centroid
lies in the disc r < 1 about the vortex centre (5, 5), evaluated on the final
averages and element corners.  The small cases start from the vortex with an
entropy wave (every characteristic field carries data, see
tests.adjoint_fd.wavy_vortex); the full-size case is the isentropic vortex."""
import multiprocessing as mp

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_3719_gb300 import workloads as W  # noqa: E402

from tests.adjoint_fd import H, _dJ, _direction, _J, _mask, _oracle_fd, agree, wavy_vortex  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno
    return aleweno


class GpuCase:
    """One GPU context with a recorded base run and its adjoint gradient."""

    def __init__(self, aleweno, mesh, Q0, order, n_sweeps, ckpt=10, mask=None):
        self.mesh, self.Q0, self.xy0, self.n = mesh, Q0, mesh["xy"].copy(), n_sweeps
        self.mask = _mask(mesh) if mask is None else mask
        s = aleweno.Solver(order_M=order, t_end=1.0)
        s.load_mesh(mesh)
        s.schedule("record", n_sweeps + 2)
        s.load_state_xy(Q0, self.xy0)
        s.adjoint_forward(n_sweeps, ckpt)
        e = s.get_elem()
        self.final = e
        self.J0 = _J(e["Q"], e["X"], self.mask)
        gQ, gX = _dJ(e["Q"], e["X"], self.mask)
        self.gQ0, self.gxy0 = s.adjoint(gQ, gX, None)
        self.log = s.get_schedule()
        s.schedule("replay")
        self.s = s

    def J(self, Q0, xy0):
        self.s.load_state_xy(Q0, xy0)
        if self.n:
            self.s.enqueue(self.n)
            self.s.sync()
        e = self.s.get_elem()
        return _J(e["Q"], e["X"], self.mask)

    def check(self, vQ, vxy):
        fd = (self.J(self.Q0 + H * vQ, self.xy0 + H * vxy) - self.J(self.Q0 - H * vQ, self.xy0 - H * vxy)) / (2 * H)
        ad = float(np.sum(self.gQ0 * vQ) + np.sum(self.gxy0 * vxy))
        return ad, fd


@pytest.mark.parametrize("order,n_sweeps,kind", [(2, 1, "Q"), (2, 1, "xy"), (2, 4, "Q"), (2, 4, "xy"),
                                                 (2, 20, "both"), (1, 12, "both"), (3, 12, "both")])
def test_adjoint_matches_gpu_central_differences(order, n_sweeps, kind):
    aleweno = _need_gpu()
    mesh, Q0 = wavy_vortex(14)
    run = GpuCase(aleweno, mesh, Q0, order, n_sweeps)
    rng = np.random.default_rng(100 + 10 * order + n_sweeps)
    for _ in range(3):
        vQ, vxy = _direction(rng, Q0, run.xy0, kind)
        ad, fd = run.check(vQ, vxy)
        assert agree(ad, fd, run.J0), (ad, fd)


def _wavy_tube(nx=30, ny=5, gamma=1.4):
    """Smooth flow through the tube that is periodic in y and transmissive in
    x (inflow on the left, outflow on the right), every characteristic field
    carrying data, resolved by 30 cells per wavelength (a wave along y would
    have 5 cells per wavelength on this mesh: its nonlinear weights would
    curve within the difference step)."""
    mesh = W.tube_mesh_periodic_y(nx, ny)

    def fun(x, y):
        k = 2 * np.pi
        rho = 1.0 + 0.2 * np.sin(k * x + 0.3)
        u = 0.3 + 0.1 * np.cos(k * x)
        v = 0.05 * np.sin(k * x + 0.5)
        p = 1.0 + 0.1 * np.sin(k * x + 1.0)
        return W.prim_to_cons(rho, u, v, p, gamma)

    return mesh, W.cell_average(mesh, fun, W._duffy_rule(8))


@pytest.mark.parametrize("order", [1, 2])
def test_adjoint_through_transmissive_boundaries(order):
    """The outer state of a transmissive edge is the boundary element's
    average: its adjoint goes to that average."""
    aleweno = _need_gpu()
    mesh, Q0 = _wavy_tube()
    run = GpuCase(aleweno, mesh, Q0, order, 12, 5, mask=np.ones(mesh["tri"].shape[0]))
    rng = np.random.default_rng(300 + order)
    for kind in ("Q", "xy", "both"):
        vQ, vxy = _direction(rng, Q0, run.xy0, kind)
        # fourth-order difference: at P1 this flow's third derivative along
        # the directions puts the central difference of step 1e-6 1.5e-5 off
        # (its error falls as H^2 towards the adjoint value)
        Jd = lambda e: run.J(Q0 + e * vQ, run.xy0 + e * vxy)
        fd = (8 * (Jd(H) - Jd(-H)) - (Jd(2 * H) - Jd(-2 * H))) / (12 * H)
        ad = float(np.sum(run.gQ0 * vQ) + np.sum(run.gxy0 * vxy))
        assert agree(ad, fd, run.J0), (kind, ad, fd)


def test_schedule_record_matches_oracle_and_replay_is_exact():
    aleweno = _need_gpu()
    from oracle.pyoracle import Oracle
    mesh, Q0 = W.vortex(12)
    n = 15
    s = aleweno.Solver(order_M=2, t_end=1.0)
    s.load_mesh(mesh)
    s.schedule("record", n + 2)
    s.load_state(Q0)
    for _ in range(n):
        s.sweep()
    e1 = s.get_elem()
    log = s.get_schedule()
    o = Oracle(order_M=2, t_end=1.0)
    o.load_mesh(mesh)
    o.schedule("record", n + 2)
    o.load_state(Q0)
    for _ in range(n):
        o.sweep()
    assert np.array_equal(log, o.get_schedule())
    s.schedule("replay")
    s.load_state(Q0)
    for _ in range(n):
        s.sweep()
    e2 = s.get_elem()
    for k in ("Q", "QM", "X", "t", "dt", "count"):
        assert np.array_equal(e1[k], e2[k]), k


def test_load_state_xy_matches_oracle():
    aleweno = _need_gpu()
    from oracle.pyoracle import Oracle
    mesh, Q0 = W.vortex(12)
    rng = np.random.default_rng(7)
    xy = mesh["xy"] + 2e-3 * rng.standard_normal(mesh["xy"].shape)
    s = aleweno.Solver(order_M=2, t_end=1.0)
    s.load_mesh(mesh)
    s.load_state_xy(Q0, xy)
    o = Oracle(order_M=2, t_end=1.0)
    o.load_mesh(mesh)
    o.load_state_xy(Q0, xy)
    for _ in range(4):
        assert s.sweep() == o.sweep()
    eg, eo = s.get_elem(), o.get_elem()
    for k in ("t", "dt", "count"):
        assert np.array_equal(eg[k], eo[k]), k
    assert np.abs(eg["Q"] - eo["Q"]).max() < 1e-12 * np.abs(eo["Q"]).max()
    assert np.abs(eg["X"] - eo["X"]).max() < 1e-12 * 10.0


def test_checkpoint_interval_does_not_change_the_gradient():
    aleweno = _need_gpu()
    mesh, Q0 = W.vortex(12)
    ref = None
    for ck in (1, 4, 25):
        run = GpuCase(aleweno, mesh, Q0, 2, 25, ck)
        g = np.concatenate([run.gQ0.ravel(), run.gxy0.ravel()])
        if ref is None:
            ref = g
        else:
            assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


def test_autograd_function_gives_the_adjoint_gradient():
    aleweno = _need_gpu()
    from paper_1408_3719_gb300.adjoint import LtsRun, kinetic_energy
    mesh, Q0 = W.vortex(12)
    s = aleweno.Solver(order_M=2, t_end=1.0)
    s.load_mesh(mesh)
    Qt = torch.tensor(Q0, dtype=torch.float64, device="cuda", requires_grad=True)
    xyt = torch.tensor(mesh["xy"], dtype=torch.float64, device="cuda", requires_grad=True)
    mask = torch.tensor(_mask(mesh), device="cuda")
    Q, X = LtsRun.apply(Qt, xyt, s, 10, 5)
    assert Q.is_cuda and X.is_cuda  # the run's outputs stay on the device
    J = kinetic_energy(Q, X, mask)
    J.backward()
    assert Qt.grad.is_cuda and xyt.grad.is_cuda
    run = GpuCase(aleweno, mesh, Q0, 2, 10, 5)
    assert abs(J.item() - run.J0) <= 1e-14 * abs(run.J0)
    assert np.abs(Qt.grad.cpu().numpy() - run.gQ0).max() <= 1e-12 * np.abs(run.gQ0).max()
    assert np.abs(xyt.grad.cpu().numpy() - run.gxy0).max() <= 1e-12 * np.abs(run.gxy0).max()


def _against_oracle(mesh, Q0, n_sweeps, n_dirs, workers):
    aleweno = _need_gpu()
    n_vortex = mesh["tri"].shape[0]
    run = GpuCase(aleweno, mesh, Q0, 2, n_sweeps, 10)
    rng = np.random.default_rng(2024 + n_vortex)
    dirs = [_direction(rng, Q0, run.xy0, ("Q", "xy", "both")[k % 3]) for k in range(n_dirs)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers, n_dirs)) as pool:
        res = pool.map(_oracle_fd, [(mesh, Q0, 2, n_sweeps, vQ, vxy) for vQ, vxy in dirs])
    for (vQ, vxy), (fd, log) in zip(dirs, res):
        assert np.array_equal(log, run.log)  # both sides took the same schedule
        ad = float(np.sum(run.gQ0 * vQ) + np.sum(run.gxy0 * vxy))
        assert agree(ad, fd, run.J0), (ad, fd)


def test_adjoint_matches_oracle_central_differences_small():
    _against_oracle(*wavy_vortex(16), 50, 20, 8)


def test_adjoint_matches_oracle_central_differences_full_size():
    """The adjoint workload: 50 sweeps of P2 on the ~50k-triangle isentropic
    vortex, checkpoints every 10 sweeps, 20 random directions."""
    _against_oracle(*W.vortex(158), 50, 20, 16)
