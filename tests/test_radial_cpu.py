"""Pins of the 1D radial reference solver (eqs. inhomEuler / matrixInhomEuler,
the reference solution of the explosions of Sec. 3.3) against what the
mathematics fixes: with alpha = 0 it is a shock-tube solver and converges to
the exact Riemann solution; with alpha = 1 the r-weighted balance laws of
mass, radial momentum (whose source is the pressure) and energy close to
O(dx), which a dropped, mis-signed or mis-weighted source term would break."""
import numpy as np
import pytest

from paper_1408_3719_gb300 import exact, radial


def test_planar_mode_converges_to_the_exact_sod_solution():
    err = []
    for n in (400, 1600):
        r, rho, u, p = radial.solve((1, 0, 1), (0.125, 0, 0.1), r_d=0.5, t_end=0.2, n=n, alpha=0)
        ex = exact.sample(r, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1))
        err.append(np.mean(np.abs(rho - ex[:, 0])))
        assert np.mean(np.abs(p - ex[:, 2])) < 5e-3
    assert err[0] < 2.5e-3
    assert err[1] < 0.5 * err[0]


def _residuals(inner, outer, t_end, n, g=1.4):
    b = {}
    r, rho, u, p = radial.solve(inner, outer, t_end=t_end, n=n, budget=b)
    dx = 1.0 / n
    inside = r < 0.5
    rho0 = np.where(inside, inner[0], outer[0])
    p0 = np.where(inside, inner[2], outer[2])
    M = lambda f: float(np.sum(r * f * dx))  # int r f dr
    mass = (M(rho) - M(rho0) + b["outflow"][0]) / M(rho0)
    mom = (M(rho * u) + b["outflow"][1] - b["pressure"]) / b["pressure"]
    ener = (M(p / (g - 1) + 0.5 * rho * u * u) - M(p0 / (g - 1)) + b["outflow"][2]) / M(p0 / (g - 1))
    return np.abs([mass, mom, ener])


@pytest.mark.parametrize("case", ["EP1", "EP2"])
def test_cylindrical_balance_laws_close_to_first_order(case):
    inner, outer, t_end = {"EP1": ((1, 0, 1), (0.125, 0, 0.1), 0.25),
                           "EP2": ((1, 0, 1000), (1, 0, 0.01), 0.012)}[case]
    r1 = _residuals(inner, outer, t_end, 750)
    r2 = _residuals(inner, outer, t_end, 1500)
    assert np.all(r1 < 2e-3), r1
    assert np.all(r2 < r1 / 1.6), (r1, r2)


def test_cylindrical_explosion_shape():
    """EP1 at t = 0.25: the centre is still at rest in the inner state (the
    inward rarefaction head, speed sqrt(1.4), reaches r = 0 at t = 0.42),
    the shock has left r = 0.5, and the outer rim is untouched."""
    r, rho, u, p = radial.solve((1, 0, 1), (0.125, 0, 0.1), t_end=0.25, n=1500)
    assert abs(rho[0] - 1.0) < 1e-12 and abs(u[0]) < 1e-12
    assert abs(rho[-1] - 0.125) < 1e-12
    shock = r[np.nonzero(np.abs(p - 0.1) > 1e-6)[0].max()]
    assert 0.8 < shock < 1.0
    assert np.all(u >= -1e-12)
