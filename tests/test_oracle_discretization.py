"""Pins of the oracle's discretisation: A_h against its eigenpairs, F' against
finite differences of F, box restriction against the global assembly, the band
storage against a dense solve, and F itself against the optimum of the discrete
optimal control problem (P), found by an independent method."""
import numpy as np
import pytest
from scipy import optimize
from scipy.linalg import lapack

from oracle import discretization as fd
from oracle import pointwise as pw
from oracle import ras, solvers


def _rand_problem(n, kind=pw.PHI_CUBIC, nu=1e-2, mu=5e-2, seed=0):
    rng = np.random.default_rng(seed)
    return fd.Problem(n, kind, nu, mu, rng.standard_normal((n, n)), 0.3 * rng.standard_normal((n, n)))


def test_A_h_eigenpairs():
    """5-point Dirichlet Laplacian: sin(k pi x1) sin(l pi x2) is an eigenvector
    with eigenvalue (4/h^2)(sin^2(k pi h/2) + sin^2(l pi h/2))."""
    n = 7
    prob = _rand_problem(n)
    h = prob.h
    x = (np.arange(n) + 1) * h
    for k, l in [(1, 1), (2, 5), (7, 3)]:
        v = np.outer(np.sin(l * np.pi * x), np.sin(k * np.pi * x))
        lam = 4 / h ** 2 * (np.sin(k * np.pi * h / 2) ** 2 + np.sin(l * np.pi * h / 2) ** 2)
        np.testing.assert_allclose(fd.apply_A(prob, v), lam * v, atol=1e-11 * lam)


@pytest.mark.parametrize("kind", [pw.PHI_CUBIC, pw.PHI_EXP, pw.PHI_KAPPA])
@pytest.mark.parametrize("eps", [1.0, 1e-3])
def test_jacobian_against_central_differences(kind, eps):
    n = 9
    prob = _rand_problem(n, kind)
    rng = np.random.default_rng(1)
    Y = 0.7 * rng.standard_normal((n, n))
    P = prob.mu * 2 * rng.standard_normal((n, n))   # straddles |p| = mu
    dY = rng.standard_normal((n, n))
    dP = prob.mu * rng.standard_normal((n, n))
    t = 1e-6
    Fp_ = fd.residual(prob, Y + t * dY, P + t * dP, eps)
    Fm_ = fd.residual(prob, Y - t * dY, P - t * dP, eps)
    Jy, Jp = fd.jacvec(prob, Y, P, eps, dY, dP)
    for fdv, jv in zip(((Fp_[0] - Fm_[0]) / (2 * t), (Fp_[1] - Fm_[1]) / (2 * t)), (Jy, Jp)):
        assert np.max(np.abs(fdv - jv)) <= 1e-6 * np.max(np.abs(jv))
    # the assembled sparse Jacobian, both orderings, matches the action
    Jpl = fd.jacobian_matrix(prob, Y, P, eps, interleaved=False)
    v = Jpl @ np.concatenate([dY.ravel(), dP.ravel()])
    np.testing.assert_allclose(v, np.concatenate([Jy.ravel(), Jp.ravel()]), rtol=1e-13, atol=1e-10)
    Jil = fd.jacobian_matrix(prob, Y, P, eps, interleaved=True)
    np.testing.assert_allclose(Jil @ fd.interleave(dY, dP), fd.interleave(Jy, Jp), rtol=1e-13, atol=1e-10)


def test_box_restriction_matches_global():
    """R F(z) and R F'(z) P on a box equal rows/columns of the global objects."""
    n = 11
    prob = _rand_problem(n, pw.PHI_EXP)
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((n, n))
    P = 0.1 * rng.standard_normal((n, n))
    box = (2, 8, 3, 11)
    x0, x1, y0, y1 = box
    Fy, Fp = fd.residual(prob, Y, P, 1e-2)
    by, bp = fd.residual(prob, Y, P, 1e-2, box)
    np.testing.assert_array_equal(by, Fy[y0:y1, x0:x1])
    np.testing.assert_array_equal(bp, Fp[y0:y1, x0:x1])
    Jg = fd.jacobian_matrix(prob, Y, P, 1e-2, interleaved=True).toarray()
    nodes = np.array([j * n + i for j in range(y0, y1) for i in range(x0, x1)])
    idx = np.empty(2 * nodes.size, dtype=int)
    idx[0::2] = 2 * nodes
    idx[1::2] = 2 * nodes + 1
    Jb = fd.jacobian_matrix(prob, Y, P, 1e-2, box, interleaved=True).toarray()
    np.testing.assert_array_equal(Jb, Jg[np.ix_(idx, idx)])


def test_band_storage_solve_matches_dense():
    n = 9
    prob = _rand_problem(n, pw.PHI_CUBIC, nu=1e-5, mu=1e-3)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, n))
    P = 1e-3 * rng.standard_normal((n, n))
    box = (1, 7, 0, 5)
    J = fd.jacobian_matrix(prob, Y, P, 1e-4, box)
    wx = box[1] - box[0]
    fac = ras.BandFactor(J, 2 * wx, 2 * wx)
    b = rng.standard_normal(J.shape[0])
    np.testing.assert_allclose(fac.solve(b), np.linalg.solve(J.toarray(), b), rtol=1e-10, atol=1e-14)


def _dense_laplacian(n):
    """5-point A_h written from its definition, independent of the oracle."""
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


@pytest.mark.parametrize("kind", [pw.PHI_CUBIC, pw.PHI_EXP])
def test_residual_reproduces_optimum_of_problem_P(kind):
    """The discrete problem (P): minimise 1/2|y - y_d|^2 + nu/2 |u|^2 + mu |u|_1
    subject to A_h y + phi(y) = f + u. Its minimiser is found here by proximal
    gradient on the reduced cost (state solved by scipy's fsolve, gradient by
    central differences of the cost), with no use of the optimality system.
    The oracle's F(x, eps) = 0 at eps -> 0 must give the same control, within
    the O(sqrt(eps)) of Lemma 5 / Thm 4."""
    n = 3
    nu, mu = 1e-2, 0.4
    rng = np.random.default_rng(7)
    yd = 20.0 * rng.standard_normal((n, n))
    f = 0.5 * rng.standard_normal((n, n))
    A = _dense_laplacian(n)
    ph = {pw.PHI_CUBIC: lambda y: y ** 3, pw.PHI_EXP: np.exp}[kind]

    def state(u):
        g = lambda y: A @ y + ph(y) - f.ravel() - u
        return optimize.fsolve(g, np.zeros(n * n), xtol=1e-14)

    def jsmooth(u):
        y = state(u)
        return 0.5 * np.sum((y - yd.ravel()) ** 2) + 0.5 * nu * np.sum(u ** 2)

    def grad(u, t=1e-5):
        g = np.zeros_like(u)
        for k in range(u.size):
            e = np.zeros_like(u)
            e[k] = t
            g[k] = (jsmooth(u + e) - jsmooth(u - e)) / (2 * t)
        return g

    L = 1.0 / np.linalg.eigvalsh(A).min() ** 2 + nu
    step = 1.0 / L
    u = np.zeros(n * n)
    for _ in range(200):
        v = u - step * grad(u)
        u_new = np.sign(v) * np.maximum(np.abs(v) - step * mu, 0.0)
        if np.max(np.abs(u_new - u)) < 1e-12 * max(1.0, np.max(np.abs(u))):
            u = u_new
            break
        u = u_new
    assert np.any(u == 0.0) and np.any(u != 0.0), "pin needs both zero and active controls"

    prob = fd.Problem(n, kind, nu, mu, yd, f)
    opts = ras.Options(eps0=1.0, gamma=0.1, eps_min=1e-13, tol=1e-13)
    res = solvers.newton_dense(prob, opts)
    assert res.status >= 0
    u_or = pw.u_eps(res.P, 1e-13, nu, mu).ravel()
    scale = np.max(np.abs(u))
    assert np.max(np.abs(u_or - u)) <= 1e-5 * scale, (u_or, u)
    np.testing.assert_allclose(res.Y.ravel(), state(u), atol=1e-6 * np.max(np.abs(state(u))))
