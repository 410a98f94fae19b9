"""Pins of the oracle's decomposition, Alg. 1, GMRES, the RAS pieces and the
outer solvers against identities the paper states and against independent
solvers (dense LU Newton, scipy sparse direct)."""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import discretization as fd
from oracle import pointwise as pw
from oracle import ras, solvers
from oracle.gmres import gmres
from oracle.newton import damped_newton, OK, OK_FLOOR, ENOCONV


# ---------------------------------------------------------------- decomposition
@pytest.mark.parametrize("n,s", [(63, 4), (255, 8), (1023, 16), (10, 3), (7, 7), (5, 1)])
def test_blocks_are_balanced_partition(n, s):
    b = dd.blocks(n, s)
    sizes = [e - a for a, e in b]
    assert b[0][0] == 0 and b[-1][1] == n
    assert all(b[k][1] == b[k + 1][0] for k in range(s - 1))
    assert sorted(set(sizes)) in ([n // s], [n // s, n // s + 1])
    assert sizes == sorted(sizes, reverse=True)   # larger blocks first


@pytest.mark.parametrize("n,sx,sy,ov", [(63, 4, 4, 2), (20, 3, 2, 1), (9, 2, 3, 0), (16, 4, 4, 5)])
def test_restriction_prolongation_identities(n, sx, sy, ov):
    """R_i P_i = I and sum_i tilde P_i R_i = I (Sec. 4.2), as exact integer identities."""
    subs = dd.subdomains(n, sx, sy, ov)
    Z = np.arange(n * n, dtype=np.float64).reshape(n, n) + 1.0
    acc = np.zeros((n, n))
    for s in subs:
        z = np.arange(s.wx * s.wy, dtype=np.float64).reshape(s.wy, s.wx) + 7.0
        np.testing.assert_array_equal(dd.restrict(dd.prolong(z, s.box, n), s.box), z)
        acc += dd.prolong_restricted(dd.restrict(Z, s.box), s, n)
        ox0, ox1, oy0, oy1 = s.owned
        assert s.box == (max(0, ox0 - ov), min(n, ox1 + ov), max(0, oy0 - ov), min(n, oy1 + ov))
    np.testing.assert_array_equal(acc, Z)


def test_paper_sizes_for_1023():
    subs = dd.subdomains(1023, 16, 16, 8)
    assert max(s.wx for s in subs) == 80 and min(s.wx for s in subs) == 71
    assert sum(2 * s.wx * s.wy for s in subs) == 3190338


# ---------------------------------------------------------------- Alg. 1
def test_newton_quadratic_convergence_scalar():
    res = damped_newton(lambda x, e: x ** 3 - 2.0, lambda x, e, F: -F / (3 * x ** 2),
                        np.array([1.0]), 1.0, 1.0, 0.5, 1.1, 1e-15, 50)
    assert res.status == OK
    assert abs(res.x[0] - 2 ** (1 / 3)) < 1e-15
    assert res.iterations <= 6


def test_newton_trivial_case_counts_continuation_steps():
    """F == 0: d = 0 every step; with the stop test applied at eps_min only,
    the iteration count is the number of continuation steps."""
    res = damped_newton(lambda x, e: np.zeros(3), lambda x, e, F: np.zeros(3), np.zeros(3),
                        1e-1, 1e-6, 0.1, 1.1, 1e-10, 50)
    assert res.status == OK and res.iterations == 5 and res.eps == 1e-6


def test_newton_backtracking_relaxed():
    """arctan from x0 = 3: the full Newton step overshoots and grows |F|; the
    relaxed test with sigma halves alpha until |F(x + alpha d)| <= sigma |F(x)|."""
    F = lambda x, e: np.arctan(x)
    S = lambda x, e, f: -f * (1 + x ** 2)
    res = damped_newton(F, S, np.array([3.0]), 1.0, 1.0, 0.5, 1.0, 1e-14, 50)
    assert res.status == OK and abs(res.x[0]) < 1e-14
    assert res.halvings >= 1
    for eps, nrm, alpha in res.history:
        assert alpha in [2.0 ** -k for k in range(21)]


def test_newton_kmax():
    res = damped_newton(lambda x, e: x ** 3 - 2.0, lambda x, e, F: -F / (3 * x ** 2),
                        np.array([1.0]), 1.0, 1.0, 0.5, 1.1, 1e-15, 2)
    assert res.status == ENOCONV and res.iterations == 2


# ---------------------------------------------------------------- GMRES
def test_gmres_against_direct_solve():
    rng = np.random.default_rng(0)
    N = 60
    A = np.eye(N) * 4 + rng.standard_normal((N, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    ref = np.linalg.solve(A, b)
    for m in (5, 30, 80):
        g = gmres(lambda v: A @ v, b, m=m, rtol=1e-12, maxit=2000)
        assert g.converged
        np.testing.assert_allclose(g.x, ref, rtol=1e-9, atol=1e-11)
    # right preconditioning with the exact inverse converges in one step
    Ainv = np.linalg.inv(A)
    g = gmres(lambda v: A @ v, b, m=30, rtol=1e-10, M=lambda v: Ainv @ v)
    assert g.iterations == 1
    np.testing.assert_allclose(g.x, ref, rtol=1e-10)


def test_gmres_exact_in_N_steps():
    rng = np.random.default_rng(1)
    N = 12
    A = rng.standard_normal((N, N)) + 3 * np.eye(N)
    b = rng.standard_normal(N)
    g = gmres(lambda v: A @ v, b, m=N, rtol=1e-14, maxit=N)
    np.testing.assert_allclose(g.x, np.linalg.solve(A, b), rtol=1e-8)


# ---------------------------------------------------------------- RAS pieces
def _small_problem(n=12, kind=pw.PHI_CUBIC, nu=1e-3, mu=2e-2, seed=3):
    x = (np.arange(n) + 1) / (n + 1)
    yd = 3.0 * np.outer(np.sin(2 * np.pi * x), np.sin(np.pi * x))
    return fd.Problem(n, kind, nu, mu, yd)


def test_F_vanishes_at_root_with_no_inner_iterations():
    """F_eps(x*) = 0 at a root of F (RASPEN function definition, Sec. 4.2): the
    local residual K_i(0) = R_i F(x*) is already below tolerance."""
    prob = _small_problem()
    opts = ras.Options(eps0=1e-4, gamma=0.1, eps_min=1e-4, tol=1e-13, inner_tol=1e-8)
    root = solvers.newton_sparse(prob, opts)
    subs = dd.subdomains(prob.n, 3, 2, 2)
    st = ras.ras_apply(prob, root.Y, root.P, subs, opts, continuation=False)
    assert st.iterations == [0] * len(subs)
    assert np.max(np.abs(st.Fy)) == 0.0 and np.max(np.abs(st.Fp)) == 0.0


def test_single_subdomain_gives_exact_correction_and_one_step():
    """s = 1: C(x) = x* - x, F' = -I, RASPEN converges in one outer step."""
    prob = _small_problem(10)
    opts = ras.Options(eps0=1e-3, gamma=0.1, eps_min=1e-3, tol=1e-10, inner_tol=1e-12)
    root = solvers.newton_sparse(prob, ras.Options(eps0=1e-3, gamma=0.1, eps_min=1e-3, tol=1e-14))
    subs = dd.subdomains(prob.n, 1, 1, 0)
    Y = 0.1 * root.Y
    P = 0.5 * root.P
    st = ras.ras_apply(prob, Y, P, subs, opts, continuation=False)
    np.testing.assert_allclose(st.Fy, root.Y - Y, atol=1e-10 * np.abs(root.Y).max())
    np.testing.assert_allclose(st.Fp, root.P - P, atol=1e-10 * np.abs(root.P).max())
    d = np.random.default_rng(0).standard_normal((2, prob.n, prob.n))
    jy, jp = ras.jvp(prob, st, d[0], d[1])
    np.testing.assert_allclose(jy, -d[0], atol=1e-9)
    np.testing.assert_allclose(jp, -d[1], atol=1e-9)
    r = solvers.raspen(prob, 1, 1, 0, ras.Options(eps0=1e-3, gamma=0.1, eps_min=1e-3, tol=1e-8,
                                                   inner_tol=1e-12))
    assert r.outer <= 1


def test_ras_fixed_point_converges_to_monolithic_root():
    """x <- x + F_eps(x) (the nonlinear RAS iteration, Sec. 4.2) reaches the
    root found by the monolithic sparse-direct Newton."""
    prob = _small_problem(14)
    opts = ras.Options(eps0=1e-2, gamma=0.1, eps_min=1e-2, tol=1e-14, inner_tol=1e-12)
    root = solvers.newton_sparse(prob, opts)
    subs = dd.subdomains(prob.n, 3, 3, 2)
    Y = np.zeros_like(root.Y)
    P = np.zeros_like(root.P)
    for _ in range(60):
        st = ras.ras_apply(prob, Y, P, subs, opts, continuation=False, factor_at_solution=False)
        Y = Y + st.Fy
        P = P + st.Fp
    assert np.max(np.abs(Y - root.Y)) <= 1e-8 * np.abs(root.Y).max()
    assert np.max(np.abs(P - root.P)) <= 1e-8 * np.abs(root.P).max()


def test_jvp_against_central_differences_of_F():
    """Alg. 4 (with the derivative of C_i) against finite differences of the
    RASPEN function itself."""
    prob = _small_problem(10)
    opts = ras.Options(eps0=1e-2, gamma=0.1, eps_min=1e-2, tol=1e-12, inner_tol=1e-13,
                       floor_factor=0.0)
    subs = dd.subdomains(prob.n, 2, 2, 1)
    rng = np.random.default_rng(5)
    Y = 0.5 * rng.standard_normal((prob.n, prob.n))
    P = 0.02 * rng.standard_normal((prob.n, prob.n))
    dY = rng.standard_normal((prob.n, prob.n))
    dP = 0.02 * rng.standard_normal((prob.n, prob.n))
    st = ras.ras_apply(prob, Y, P, subs, opts, continuation=False)
    jy, jp = ras.jvp(prob, st, dY, dP)
    t = 1e-5
    a = ras.ras_apply(prob, Y + t * dY, P + t * dP, subs, opts, False, False)
    b = ras.ras_apply(prob, Y - t * dY, P - t * dP, subs, opts, False, False)
    fy = (a.Fy - b.Fy) / (2 * t)
    fp = (a.Fp - b.Fp) / (2 * t)
    assert np.max(np.abs(fy - jy)) <= 1e-6 * np.max(np.abs(jy))
    assert np.max(np.abs(fp - jp)) <= 1e-6 * np.max(np.abs(jp))


def test_linear_ras_single_subdomain_is_exact_inverse():
    prob = _small_problem(8)
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((8, 8))
    P = 0.01 * rng.standard_normal((8, 8))
    pre = ras.LinearRas(prob, Y, P, dd.subdomains(8, 1, 1, 0), 1e-3)
    rY, rP = rng.standard_normal((2, 8, 8))
    zy, zp = pre.apply(rY, rP)
    jy, jp = fd.jacvec(prob, Y, P, 1e-3, zy, zp)
    np.testing.assert_allclose(jy, rY, atol=1e-9)
    np.testing.assert_allclose(jp, rP, atol=1e-9)


# ---------------------------------------------------------------- outer solvers
@pytest.mark.parametrize("n,s", [(4, 2), (8, 2)])
@pytest.mark.parametrize("kind", [pw.PHI_CUBIC, pw.PHI_EXP])
def test_all_solvers_reach_the_dense_newton_root(n, s, kind):
    x = (np.arange(n) + 1) / (n + 1)
    yd = 40.0 * np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x))
    prob = fd.Problem(n, kind, 1e-3, 5e-2, yd)
    opts = ras.Options(eps0=0.1, gamma=0.1, eps_min=1e-6, tol=1e-12, inner_tol=1e-10)
    dense = solvers.newton_dense(prob, opts)
    assert dense.status >= 0
    scale_y = np.abs(dense.Y).max()
    scale_p = np.abs(dense.P).max()
    for res in (solvers.raspen(prob, s, s, 1, opts), solvers.newton_ras(prob, s, s, 1, opts),
                solvers.newton_sparse(prob, opts), solvers.newton_gmres(prob, opts)):
        assert res.status >= 0
        assert np.max(np.abs(res.Y - dense.Y)) <= 1e-12 * scale_y
        assert np.max(np.abs(res.P - dense.P)) <= 1e-12 * scale_p


@pytest.mark.parametrize("eps0", [1e-6, 0.1])
def test_newton_gmres_follows_the_direct_newton_steps(eps0):
    """Unpreconditioned GMRES solved to a tight tolerance reproduces the Newton
    steps of the sparse direct solver: same iterate sequence (to the GMRES
    accuracy), same iteration and halving counts, with (Newton_eps) and
    without (Newton) continuation."""
    n = 12
    x = (np.arange(n) + 1) / (n + 1)
    yd = 30.0 * np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x))
    prob = fd.Problem(n, pw.PHI_CUBIC, 1e-3, 5e-2, yd)
    opts = ras.Options(eps0=eps0, gamma=0.1, eps_min=1e-6, tol=1e-12, gmres_rtol=1e-13, gmres_maxit=4000)
    a = solvers.newton_sparse(prob, opts)
    b = solvers.newton_gmres(prob, opts)
    assert a.status >= 0 and b.status >= 0
    assert a.outer == b.outer
    assert a.newton.halvings == b.newton.halvings
    assert np.max(np.abs(b.Y - a.Y)) <= 1e-10 * np.abs(a.Y).max()
    assert np.max(np.abs(b.P - a.P)) <= 1e-10 * np.abs(a.P).max()
    assert len(b.gmres_its) == b.outer and all(k > 0 for k in b.gmres_its)


def test_eps_solutions_converge():
    """x(eps) -> x as eps -> 0 (Thm 3), at a rate no worse than O(sqrt(eps)) (Thm 4):
    the successive differences of x(eps) for eps = 10^-k decrease."""
    n = 15
    x = (np.arange(n) + 1) / (n + 1)
    yd = 30.0 * np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x))
    prob = fd.Problem(n, pw.PHI_CUBIC, 1e-3, 5e-2, yd)
    sols = []
    for k in range(1, 9):
        e = 10.0 ** -k
        r = solvers.newton_sparse(prob, ras.Options(eps0=1.0, gamma=0.1, eps_min=e, tol=1e-13))
        sols.append(np.concatenate([r.Y.ravel(), r.P.ravel()]))
    diffs = [np.linalg.norm(sols[k + 1] - sols[k]) for k in range(len(sols) - 1)]
    assert all(diffs[k + 1] < diffs[k] for k in range(len(diffs) - 1)), diffs
    # no slower than sqrt(eps): each tenfold eps reduction shrinks by >= sqrt(10)/1.5
    assert all(diffs[k + 1] <= diffs[k] / (np.sqrt(10) / 1.5) for k in range(len(diffs) - 1)), diffs
