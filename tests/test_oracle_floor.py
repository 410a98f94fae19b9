"""Pins of the rounding-floor stop of the 2-D oracle: the floor norm against its
definition written out node by node, and the OK_FLOOR exit of Alg. 1
(damped_newton) on problems where the step at which it fires is known in
advance."""
import math

import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import discretization as fd
from oracle import pointwise as pw
from oracle import ras as oras
from oracle.newton import ENOCONV, OK, OK_FLOOR, U_ROUND, damped_newton


def _floor_by_loops(n, beta, nu, mu, eps, Y, P, f, yd, box, cubic=True):
    """sqrt(sum over the box nodes of My^2 + Mp^2), with My, Mp the sums of the
    absolute values of every term of F_y, F_p (Sec. 3.3) at that node; the
    smoothed projection from its definition as a difference of square roots."""
    x0, x1, y0, y1 = box

    def val(Z, i, j):
        return Z[j, i] if (0 <= i < n and 0 <= j < n) else 0.0

    total = 0.0
    for j in range(y0, y1):
        for i in range(x0, x1):
            yc, pc = Y[j, i], P[j, i]
            nb_y = sum(abs(val(Y, i + di, j + dj)) for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)))
            nb_p = sum(abs(val(P, i + di, j + dj)) for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)))
            phi = yc ** 3 if cubic else math.exp(yc)
            dphi = 3 * yc ** 2 if cubic else math.exp(yc)
            x = -pc / mu
            peps = 0.5 * (math.sqrt((x + 1) ** 2 + eps) - math.sqrt((x - 1) ** 2 + eps))
            My = (beta * (4 * abs(yc) + nb_y) + abs(phi) + abs(f[j, i])
                  + abs(pc) / nu + mu * abs(peps) / nu)
            Mp = beta * (4 * abs(pc) + nb_p) + abs(dphi * pc) + abs(yc) + abs(yd[j, i])
            total += My * My + Mp * Mp
    return math.sqrt(total)


@pytest.mark.parametrize("box", [None, (1, 5, 2, 6), (0, 3, 0, 7)])
@pytest.mark.parametrize("kind", [pw.PHI_CUBIC, pw.PHI_EXP])
def test_floor_norm_2d_is_the_sum_of_absolute_terms(box, kind):
    n, nu, mu, eps = 7, 1e-3, 0.4, 1e-3
    rng = np.random.default_rng(11)
    yd, f = rng.standard_normal((2, n, n))
    prob = fd.Problem(n, kind, nu, mu, yd, f)
    Y = 0.5 * rng.standard_normal((n, n))
    P = rng.standard_normal((n, n))
    b = fd.full_box(n) if box is None else box
    ref = _floor_by_loops(n, prob.beta, nu, mu, eps, Y, P, f, yd, b, cubic=(kind == pw.PHI_CUBIC))
    got = fd.residual_floor_norm(prob, Y, P, eps, box)
    assert abs(got - ref) <= 1e-13 * ref, (got, ref)


def _sqrt2_newton(x0, eps0, eps_min, tol, floor=True, kmax=50):
    """Alg. 1 on F(x) = x^2 - 2 (no eps dependence): M(x) = x^2 + 2 is the sum
    of |terms| of F."""
    return damped_newton(lambda x, e: np.array([x[0] * x[0] - 2.0]),
                         lambda x, e, F: -F / (2.0 * x[0]),
                         np.array([x0]), eps0, eps_min, 0.1, 1.1, tol, kmax,
                         floor=(lambda x, e: x[0] * x[0] + 2.0) if floor else None)


def test_floor_exit_fires_at_the_first_rounding_level_residual():
    """From x0 = 1 Newton's iterates for sqrt(2) are 3/2, 17/12, 577/408,
    665857/470832, then sqrt(2) to rounding. With tol = 0 only the floor test
    can stop the loop; it fires at the first iterate whose residual is below
    16 u (x^2 + 2) = 7.1e-15, i.e. at k = 5 (|F(x4)| = 4.5e-12)."""
    r = _sqrt2_newton(1.0, 1e-3, 1e-3, 0.0)
    assert r.status == OK_FLOOR and r.iterations == 5
    assert abs(r.x[0] - math.sqrt(2.0)) <= 2 * U_ROUND * math.sqrt(2.0)
    hist = [h[1] for h in r.history]
    assert abs(hist[4] - abs(665857.0 ** 2 / 470832.0 ** 2 - 2.0)) <= 1e-15
    assert hist[4] > 16 * U_ROUND * (hist[4] + 4.0)
    # the same run without the floor test exhausts kmax
    r2 = _sqrt2_newton(1.0, 1e-3, 1e-3, 0.0, floor=False, kmax=12)
    assert r2.status == ENOCONV and r2.iterations == 12
    # a reachable tolerance stops with OK before the floor is met
    r3 = _sqrt2_newton(1.0, 1e-3, 1e-3, 1e-5)
    assert r3.status == OK and r3.iterations == 3


def test_floor_exit_waits_for_eps_min():
    """Stop tests apply only at eps_min (reading C6): started at the root with
    eps_0 = 1e-1, gamma = 0.1, eps_min = 1e-4, the loop must take the three
    continuation steps (1e-1 -> 1e-2 -> 1e-3 -> 1e-4) before the floor exit."""
    r = _sqrt2_newton(math.sqrt(2.0), 1e-1, 1e-4, 0.0)
    assert r.status == OK_FLOOR and r.iterations == 3
    assert r.eps == 1e-4


def test_local_solve_below_rounding_ends_on_the_floor():
    """A local Newton solve (Alg. 1 on K_i) asked for inner_tol = 0 ends with
    OK_FLOOR at eps_min, well before kmax, with a residual at rounding level of
    its floor norm; without the floor factor it runs into kmax."""
    n = 12
    rng = np.random.default_rng(3)
    prob = fd.Problem(n, pw.PHI_CUBIC, 1e-2, 0.05, rng.standard_normal((n, n)))
    sub = dd.subdomains(n, 2, 2, 1)[3]
    Z = np.zeros((n, n))
    o = oras.Options(eps0=1e-2, gamma=0.1, eps_min=1e-4, inner_tol=0.0, kmax_inner=40)
    loc = oras.local_correction(prob, Z, Z, sub, o.eps0, o.eps_min, o, factor_at_solution=False)
    assert loc.newton.status == OK_FLOOR and loc.newton.iterations < 20
    assert loc.newton.eps == 1e-4
    Yi, Pi = loc.Yi, loc.Pi
    flr = fd.residual_floor_norm(prob, Yi, Pi, 1e-4, sub.box)
    assert loc.newton.norm <= 16 * U_ROUND * flr
    o2 = oras.Options(eps0=1e-2, gamma=0.1, eps_min=1e-4, inner_tol=0.0, kmax_inner=25, floor_factor=0.0)
    loc2 = oras.local_correction(prob, Z, Z, sub, o2.eps0, o2.eps_min, o2, factor_at_solution=False)
    assert loc2.newton.status == ENOCONV and loc2.newton.iterations == 25
