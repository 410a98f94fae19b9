"""Pins of the model problem on the unit cube (oracle/three_d.py): the 7-point
operator against its eigenpairs and its matrix form, the Jacobian against
central differences, the partition identities, a manufactured root built with
an independently assembled dense Laplacian and reached by RASPEN from x0 = 0,
one subdomain giving one Newton step, Alg. 4 against differences of the RASPEN
function, and the rounding-floor norm against its definition."""
import numpy as np

from oracle import pointwise as pw
from oracle import ras as oras
from oracle import three_d as t3


def _grid(n):
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    return np.meshgrid(x, x, x, indexing="ij")   # [k, j, i] -> (x3, x2, x1)


def test_operator_eigenpairs_and_matrix_form():
    n = 7
    prob = t3.Problem(n, pw.PHI_CUBIC, 1.0, 1.0, np.zeros((n, n, n)))
    X3, X2, X1 = _grid(n)
    h = prob.h
    for a, b, c in ((1, 1, 1), (2, 3, 1), (7, 1, 4)):
        v = np.sin(a * np.pi * X1) * np.sin(b * np.pi * X2) * np.sin(c * np.pi * X3)
        lam = prob.beta * (6.0 - 2 * np.cos(a * np.pi * h) - 2 * np.cos(b * np.pi * h) - 2 * np.cos(c * np.pi * h))
        assert np.abs(t3.apply_A(prob, v) - lam * v).max() <= 1e-9 * lam
    v = np.random.default_rng(1).standard_normal((n, n, n))
    L = t3.laplacian_matrix(prob.beta, n, n, n)
    assert np.abs(L @ v.ravel() - t3.apply_A(prob, v).ravel()).max() <= 1e-10 * prob.beta


def test_jacobian_against_central_differences():
    n, eps = 4, 1e-3
    rng = np.random.default_rng(2)
    for phi in (pw.PHI_CUBIC, pw.PHI_EXP, pw.PHI_KAPPA):
        prob = t3.Problem(n, phi, 1e-2, 0.3, rng.standard_normal((n, n, n)), rng.standard_normal((n, n, n)))
        Y, P = 0.5 * rng.standard_normal((n, n, n)), 0.5 * rng.standard_normal((n, n, n))
        dY, dP = rng.standard_normal((n, n, n)), rng.standard_normal((n, n, n))
        d = 1e-6
        Fp_y, Fp_p = t3.residual(prob, Y + d * dY, P + d * dP, eps)
        Fm_y, Fm_p = t3.residual(prob, Y - d * dY, P - d * dP, eps)
        jy, jp = t3.jacvec(prob, Y, P, eps, dY, dP)
        scale = np.abs(np.concatenate([jy.ravel(), jp.ravel()])).max()
        assert np.abs((Fp_y - Fm_y) / (2 * d) - jy).max() <= 1e-6 * scale
        assert np.abs((Fp_p - Fm_p) / (2 * d) - jp).max() <= 1e-6 * scale
        J = t3.jacobian_matrix(prob, Y, P, eps)
        assert np.abs(J @ t3.interleave(dY, dP) - t3.interleave(jy, jp)).max() <= 1e-9 * scale


def test_restricted_prolongations_partition_the_grid():
    n = 9
    subs = t3.subdomains(n, 2, 3, 2, 2)
    total = sum(t3.prolong_restricted(np.ones(s.shape, dtype=np.int64), s, n) for s in subs)
    assert np.array_equal(total, np.ones((n, n, n)))
    assert sorted(s.index for s in subs) == list(range(12))


def _dense_laplacian(n):
    h = 1.0 / (n + 1)
    A = np.zeros((n ** 3, n ** 3))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                q = (k * n + j) * n + i
                A[q, q] = 6.0 / h ** 2
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < n and 0 <= jj < n and 0 <= kk < n:
                        A[q, (kk * n + jj) * n + ii] = -1.0 / h ** 2
    return A


def _manufactured(n, nu, mu, eps):
    """(y*, p*) chosen, then f and y_d set so that F(y*, p*, eps) = 0, with a
    dense Laplacian of its own and the closed forms of phi and P_eps."""
    X3, X2, X1 = _grid(n)
    ys = 0.3 * np.sin(np.pi * X1) * np.sin(2 * np.pi * X2) * np.sin(np.pi * X3)
    ps = 2.0 * mu * np.sin(2 * np.pi * X1) * np.sin(np.pi * X2) * np.sin(np.pi * X3)
    A = _dense_laplacian(n)
    y, p = ys.ravel(), ps.ravel()
    x = -p / mu
    Peps = 2 * x / (np.sqrt((x + 1) ** 2 + eps) + np.sqrt((x - 1) ** 2 + eps))
    f = A @ y + y ** 3 + (1.0 / nu) * (p + mu * Peps)
    y_d = -(A @ p + 3 * y ** 2 * p - y)
    return ys, ps, f.reshape(n, n, n), y_d.reshape(n, n, n)


def test_raspen_reaches_a_manufactured_root():
    n, nu, mu, eps = 6, 1e-3, 1e-2, 1e-6
    ys, ps, f, y_d = _manufactured(n, nu, mu, eps)
    prob = t3.Problem(n, pw.PHI_CUBIC, nu, mu, y_d, f)
    o = oras.Options(tol=1e-12, inner_tol=1e-10, sigma=1.1, eps0=0.1, gamma=0.1, eps_min=eps)
    r = t3.raspen(prob, 2, 2, 2, 1, o)
    assert r.status == 0 and r.outer >= 1
    assert np.abs(r.Y - ys).max() <= 1e-9 * np.abs(ys).max()
    assert np.abs(r.P - ps).max() <= 1e-9 * np.abs(ps).max()


def test_one_subdomain_is_one_newton_step():
    n, nu, mu, eps = 4, 1e-3, 1e-2, 1e-6
    ys, ps, f, y_d = _manufactured(n, nu, mu, eps)
    prob = t3.Problem(n, pw.PHI_CUBIC, nu, mu, y_d, f)
    o = oras.Options(tol=1e-12, inner_tol=1e-11, sigma=1.1, eps0=eps, gamma=0.1, eps_min=eps)
    state = t3.ras_apply(prob, np.zeros((n, n, n)), np.zeros((n, n, n)), t3.subdomains(n, 1, 1, 1, 0), o, False)
    # the local problem is the whole system: C(0) = x* and the RASPEN Jacobian is -I
    assert np.abs(state.Fy - ys).max() <= 1e-9 * np.abs(ys).max()
    d = np.random.default_rng(3).standard_normal((2, n, n, n))
    jy, jp = t3.jvp(prob, state, d[0], d[1])
    assert np.abs(jy + d[0]).max() <= 1e-9 and np.abs(jp + d[1]).max() <= 1e-9
    r = t3.raspen(prob, 1, 1, 1, 0, o)
    assert r.outer == 1


def test_jvp_against_differences_of_the_ras_function():
    n, nu, mu, eps = 4, 1e-3, 1e-2, 1e-6
    ys, ps, f, y_d = _manufactured(n, nu, mu, eps)
    prob = t3.Problem(n, pw.PHI_CUBIC, nu, mu, y_d, f)
    o = oras.Options(tol=1e-12, inner_tol=1e-12, sigma=1.1, eps0=eps, gamma=0.1, eps_min=eps)
    subs = t3.subdomains(n, 2, 1, 2, 1)
    Y, P = 0.9 * ys, 0.9 * ps
    d = np.random.default_rng(4).standard_normal((2, n, n, n))
    state = t3.ras_apply(prob, Y, P, subs, o, False)
    jy, jp = t3.jvp(prob, state, d[0], d[1])
    scale = np.abs(np.concatenate([jy.ravel(), jp.ravel()])).max()
    errs = []
    for h in (1e-5, 1e-6):
        sp_ = t3.ras_apply(prob, Y + h * d[0], P + h * d[1], subs, o, False)
        sm_ = t3.ras_apply(prob, Y - h * d[0], P - h * d[1], subs, o, False)
        errs.append(max(np.abs((sp_.Fy - sm_.Fy) / (2 * h) - jy).max(),
                        np.abs((sp_.Fp - sm_.Fp) / (2 * h) - jp).max()) / scale)
    # central differences converge to the Jacobian action as h^2
    assert errs[1] <= 1e-4 and errs[0] / errs[1] > 50, errs


def test_floor_norm_is_the_sum_of_absolute_terms():
    n = 3
    rng = np.random.default_rng(5)
    prob = t3.Problem(n, pw.PHI_CUBIC, 1e-2, 0.5, rng.standard_normal((n, n, n)), rng.standard_normal((n, n, n)))
    Y, P = rng.standard_normal((n, n, n)), rng.standard_normal((n, n, n))
    A = _dense_laplacian(n)
    absA = np.abs(A)
    y, p = Y.ravel(), P.ravel()
    x = -p / 0.5
    Peps = 2 * x / (np.sqrt((x + 1) ** 2 + 1e-3) + np.sqrt((x - 1) ** 2 + 1e-3))
    My = absA @ np.abs(y) + np.abs(y ** 3) + np.abs(prob.f.ravel()) + (1 / 1e-2) * (np.abs(p) + 0.5 * np.abs(Peps))
    Mp = absA @ np.abs(p) + np.abs(3 * y ** 2 * p) + np.abs(y) + np.abs(prob.y_d.ravel())
    ref = np.sqrt(np.sum(My ** 2) + np.sum(Mp ** 2))
    assert abs(t3.residual_floor_norm(prob, Y, P, 1e-3) - ref) <= 1e-12 * ref
