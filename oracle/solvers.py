"""Outer solvers. Test infrastructure.

* raspen: Alg. 2, one-level RASPEN. Newton on F_eps(x) = 0 (the RASPEN function
  of Alg. 3), undamped (x <- x + d), the Newton system solved by GMRES with the
  Jacobian action of Alg. 4. eps-continuation runs only inside the local
  solves of the first evaluation F_eps(x^0); every later evaluation starts the
  local solves at eps_min.
* newton_ras: Alg. 1 on the global system F_eps(x) = 0 whose Newton systems
  are solved by GMRES right-preconditioned with the linear RAS preconditioner
  (the paper's Newton_RAS, Sec. 4.1 and 5.1). With eps_0 > eps_min it is
  Newton_RAS,eps.
* newton_gmres: Alg. 1 on the global system whose Newton systems are solved by
  unpreconditioned GMRES (the paper's Newton and, with eps_0 > eps_min,
  Newton_eps baselines, Sec. 4.1 and 5.1).
* newton_dense: Alg. 1 with a dense LU solve of the full Jacobian (brute force,
  small grids only).
* newton_sparse: Alg. 1 with a sparse direct solve of the full Jacobian.

Global vectors are planar: [y.ravel(), p.ravel()].
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import discretization as fd
from . import decomposition as dd
from . import ras
from .gmres import gmres
from .newton import damped_newton, OK, ENOCONV


def _split(v, n):
    return v[:n * n].reshape(n, n), v[n * n:].reshape(n, n)


def _join(a, b):
    return np.concatenate([a.ravel(), b.ravel()])


class SolveResult:
    def __init__(self):
        self.Y = None
        self.P = None
        self.outer = 0
        self.gmres_its = []
        self.inner_its = []      # per outer evaluation: list of per-subdomain counts
        self.norms = []
        self.status = OK


def raspen(prob, sx, sy, overlap, opts, Y0=None, P0=None, engine=None):
    """Alg. 2. `engine` evaluates Alg. 3 (apply) and Alg. 4 (jvp); the default
    runs the subdomains one after another, oracle.parallel.ParallelEngine
    spreads them over processes with identical results."""
    n = prob.n
    subs = dd.subdomains(n, sx, sy, overlap)
    if engine is None:
        engine = ras.SerialEngine(prob, subs, opts)
    Y = np.zeros((n, n)) if Y0 is None else Y0.copy()
    P = np.zeros((n, n)) if P0 is None else P0.copy()
    out = SolveResult()
    state = engine.apply(Y, P, True)
    out.inner_its.append(state.iterations)
    Fn = float(np.linalg.norm(_join(state.Fy, state.Fp)))
    out.norms.append(Fn)
    stop = max(opts.tol, opts.tol * Fn)
    k = 0
    while Fn > stop and k < opts.kmax_outer_raspen:
        def A(v):
            dY, dP = _split(v, n)
            jy, jp = engine.jvp(state, dY, dP)
            return _join(jy, jp)
        g = gmres(A, -_join(state.Fy, state.Fp), opts.gmres_restart, opts.gmres_rtol, opts.gmres_maxit)
        out.gmres_its.append(g.iterations)
        dY, dP = _split(g.x, n)
        Y = Y + dY
        P = P + dP
        k += 1
        state = engine.apply(Y, P, False)
        out.inner_its.append(state.iterations)
        Fn = float(np.linalg.norm(_join(state.Fy, state.Fp)))
        out.norms.append(Fn)
    out.status = OK if Fn <= stop else ENOCONV
    out.Y, out.P, out.outer = Y, P, k
    return out


def _global_residual(prob):
    n = prob.n

    def residual(v, eps):
        Y, P = _split(v, n)
        return _join(*fd.residual(prob, Y, P, eps))

    def floor(v, eps):
        Y, P = _split(v, n)
        return fd.residual_floor_norm(prob, Y, P, eps)
    return residual, floor


def newton_ras(prob, sx, sy, overlap, opts, Y0=None, P0=None):
    n = prob.n
    subs = dd.subdomains(n, sx, sy, overlap)
    residual, floor = _global_residual(prob)
    gm = []

    def solve(v, eps, F):
        Y, P = _split(v, n)
        pre = ras.LinearRas(prob, Y, P, subs, eps)

        def A(w):
            wY, wP = _split(w, n)
            return _join(*fd.jacvec(prob, Y, P, eps, wY, wP))

        def M(w):
            wY, wP = _split(w, n)
            return _join(*pre.apply(wY, wP))
        g = gmres(A, -F, opts.gmres_restart, opts.gmres_rtol, opts.gmres_maxit, M)
        gm.append(g.iterations)
        return g.x

    x0 = np.zeros(2 * n * n) if Y0 is None else _join(Y0, P0)
    res = damped_newton(residual, solve, x0, opts.eps0, opts.eps_min, opts.gamma, opts.sigma,
                        opts.tol, opts.kmax_outer_newton, opts.max_halvings, floor, opts.floor_factor)
    out = SolveResult()
    out.Y, out.P = _split(res.x, n)
    out.outer = res.iterations
    out.gmres_its = gm
    out.status = res.status
    out.newton = res
    return out


def newton_gmres(prob, opts, Y0=None, P0=None):
    """Alg. 1 with GMRES(m) on the full Jacobian F'_eps(x), no preconditioner."""
    n = prob.n
    residual, floor = _global_residual(prob)
    gm = []

    def solve(v, eps, F):
        Y, P = _split(v, n)

        def A(w):
            wY, wP = _split(w, n)
            return _join(*fd.jacvec(prob, Y, P, eps, wY, wP))
        g = gmres(A, -F, opts.gmres_restart, opts.gmres_rtol, opts.gmres_maxit)
        gm.append(g.iterations)
        return g.x

    x0 = np.zeros(2 * n * n) if Y0 is None else _join(Y0, P0)
    res = damped_newton(residual, solve, x0, opts.eps0, opts.eps_min, opts.gamma, opts.sigma,
                        opts.tol, opts.kmax_outer_newton, opts.max_halvings, floor, opts.floor_factor)
    out = SolveResult()
    out.Y, out.P = _split(res.x, n)
    out.outer = res.iterations
    out.gmres_its = gm
    out.status = res.status
    out.newton = res
    return out


def _newton_direct(prob, opts, x0, dense):
    n = prob.n
    residual, floor = _global_residual(prob)

    def solve(v, eps, F):
        Y, P = _split(v, n)
        J = fd.jacobian_matrix(prob, Y, P, eps, interleaved=False)
        if dense:
            return np.linalg.solve(J.toarray(), -F)
        return spla.spsolve(J.tocsc(), -F)

    x0 = np.zeros(2 * n * n) if x0 is None else x0
    res = damped_newton(residual, solve, x0, opts.eps0, opts.eps_min, opts.gamma, opts.sigma,
                        opts.tol, opts.kmax_outer_newton, opts.max_halvings, floor, opts.floor_factor)
    out = SolveResult()
    out.Y, out.P = _split(res.x, n)
    out.outer = res.iterations
    out.status = res.status
    out.newton = res
    return out


def newton_dense(prob, opts, x0=None):
    """Brute force: Alg. 1 with dense LU of the full Jacobian (n <= 8)."""
    if prob.n > 16:
        raise ValueError("dense brute force is meant for tiny grids")
    return _newton_direct(prob, opts, x0, dense=True)


def newton_sparse(prob, opts, x0=None):
    """Alg. 1 with a sparse direct solve of the full Jacobian."""
    return _newton_direct(prob, opts, x0, dense=False)
