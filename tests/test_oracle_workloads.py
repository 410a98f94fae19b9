"""Pins of the manufactured model problem of Sec. 4 (oracle/workloads.py):
a brute-force dense Newton solve of the state equation on a tiny grid with its
own dense Laplacian, the closed form of the eps -> 0 control (soft threshold),
the construction's residual at rounding level, and convergence of the
eps-solutions towards the manufactured pair as eps shrinks."""
import numpy as np
import pytest

from oracle import discretization as fd
from oracle import pointwise as pw
from oracle import ras as oras
from oracle import solvers
from oracle import workloads as wl
from paper_2411_00546_gb300 import inputs


def _dense_laplacian(n):
    h = 1.0 / (n + 1)
    A = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            q = j * n + i
            A[q, q] = 4.0 / h ** 2
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    A[q, jj * n + ii] = -1.0 / h ** 2
    return A


def test_state_solve_matches_dense_brute_force():
    n, nu, mu, kappa, eps = 5, 1e-6, 1.0, 0.1, 1e-15
    pbar = inputs.yd_manufactured_paper(n, mu, 1)
    Y, yd = wl.manufactured(pbar, n, nu=nu, mu=mu, kappa=kappa, eps=eps)
    A = _dense_laplacian(n)
    p = pbar.ravel()
    # control at the adjoint, soft threshold plus smoothing: u = -(1/nu)(p + mu P_eps(-p/mu)),
    # evaluated in 50 digits (in FP64 the printed difference loses 2^-53/eps where |p| < mu)
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(50):
        def u_mp(pv):
            P, M, E = mpmath.mpf(float(pv)), mpmath.mpf(mu), mpmath.mpf(eps)
            x = -P / M
            Pe = (mpmath.sqrt((x + 1) ** 2 + E) - mpmath.sqrt((x - 1) ** 2 + E)) / 2
            return float(-(P + M * Pe) / mpmath.mpf(nu))
        rhs = np.array([u_mp(v) for v in p])
    y = np.zeros(n * n)
    for _ in range(200):
        g = A @ y + kappa * (y ** 3 + np.exp(kappa * y)) - rhs
        if np.linalg.norm(g) <= 1e-13 * np.linalg.norm(rhs):
            break
        J = A + np.diag(kappa * (3 * y ** 2 + kappa * np.exp(kappa * y)))
        y = y - np.linalg.solve(J, g)
    assert np.abs(Y.ravel() - y).max() <= 1e-10 * np.abs(y).max()
    yd_ref = -A @ p - kappa * (3 * y ** 2 + kappa * np.exp(kappa * y)) * p + y
    assert np.abs(yd.ravel() - yd_ref).max() <= 1e-10 * np.abs(yd_ref).max()


def test_control_at_tiny_eps_is_the_soft_threshold():
    n, nu, mu = 31, 1e-6, 1.0
    pbar = inputs.yd_manufactured_paper(n, mu, 5)
    u = pw.u_eps(pbar, 1e-15, nu, mu)
    soft = -(1.0 / nu) * np.sign(pbar) * np.maximum(np.abs(pbar) - mu, 0.0)
    assert np.abs(u - soft).max() <= 1e-6 * np.abs(soft).max()
    assert np.any(np.abs(pbar) > mu) and np.any(soft == 0.0)   # both regimes occur


def test_manufactured_pair_solves_the_system():
    n = 31
    pbar = inputs.yd_manufactured_paper(n, 1.0, 5)
    Y, yd = wl.manufactured(pbar, n)
    prob = fd.Problem(n, pw.PHI_KAPPA, 1e-6, 1.0, yd, kappa=0.1)
    Fy, Fp = fd.residual(prob, Y, pbar, 1e-15)
    flr = fd.residual_floor_norm(prob, Y, pbar, 1e-15)
    assert np.sqrt(np.sum(Fy ** 2) + np.sum(Fp ** 2)) <= 1e-13 * flr


def test_eps_solutions_approach_the_manufactured_pair():
    n = 31
    pbar = inputs.yd_manufactured_paper(n, 1.0, 5)
    Y, yd = wl.manufactured(pbar, n)
    prob = fd.Problem(n, pw.PHI_KAPPA, 1e-6, 1.0, yd, kappa=0.1)
    errs = []
    for eps_min in (1e-2, 1e-4, 1e-6):
        o = oras.Options(tol=1e-10, inner_tol=1e-8, sigma=1.1, eps0=max(0.1, eps_min), gamma=0.1, eps_min=eps_min)
        r = solvers.raspen(prob, 2, 2, 2, o)
        errs.append(np.abs(r.P - pbar).max() / np.abs(pbar).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3, errs


def test_raspen_reaches_the_manufactured_pair_at_the_paper_eps():
    """At eps_min = 1e-15 the manufactured (ybar, pbar) is the exact discrete
    solution: a full RASPEN solve from x0 = 0 (the paper's continuation
    eps0 = 1, gamma = 1/5) must reproduce it."""
    n = 31
    pbar = inputs.yd_manufactured_paper(n, 1.0, 5)
    Y, yd = wl.manufactured(pbar, n)
    prob = fd.Problem(n, pw.PHI_KAPPA, 1e-6, 1.0, yd, kappa=0.1)
    o = oras.Options(tol=1e-10, inner_tol=1e-8, sigma=1.1, eps0=1.0, gamma=0.2, eps_min=1e-15)
    r = solvers.raspen(prob, 2, 2, 2, o)
    assert r.status == 0
    assert np.abs(r.Y - Y).max() <= 1e-10 * np.abs(Y).max()
    assert np.abs(r.P - pbar).max() <= 1e-10 * np.abs(pbar).max()
