"""Damped Newton with eps-continuation and relaxed backtracking (Alg. 1, Sec. 4.1).
Test infrastructure.

Readings taken where the paper leaves a choice:

* Norm: the Euclidean norm of the residual vector, both fields together.
* Stop test: ||F_{eps_k}(x^k)|| <= max(tol, tol ||F_{eps_0}(x^0)||) ends the
  loop only once eps_k has reached eps_min (the printed test alone could stop
  on a residual of a more strongly smoothed system).
* Rounding floor: when that tolerance lies below the rounding error of an FP64
  evaluation of F, the loop also stops (at eps_min) once
  ||F|| <= floor_factor * 2^-53 * ||M|| with M the nodewise sums of |terms| of F.
* Iteration limit: at most kmax Newton steps, then status ENOCONV.
* Backtracking: alpha = 1, 1/2, 1/4, ... at most max_halvings times; if the
  relaxed test ||F(x + alpha d)|| <= sigma ||F(x)|| still fails, the last
  (smallest) step is taken and counted in `exhausted`.
* After the step, eps_{k+1} = max(gamma eps_k, eps_min), where a product
  gamma eps_k within a relative 1e-9 of eps_min counts as eps_min (the exact
  geometric sequence 0.1 * 0.1^5 reaches 1e-6, its FP64 rounding lands one ulp
  above it). When eps is unchanged the residual of the accepted trial point is
  reused (same value).
"""
import numpy as np

U_ROUND = 2.0 ** -53

OK = 0
OK_FLOOR = 1
ENOCONV = -3
ENONFINITE = -6


class NewtonResult:
    def __init__(self):
        self.x = None
        self.iterations = 0
        self.status = OK
        self.eps = None
        self.norm = None
        self.norm0 = None
        self.halvings = 0
        self.exhausted = 0
        self.history = []   # (eps_k, ||F||, alpha) per iteration


def next_eps(eps, gamma, eps_min):
    """eps_{k+1} = max(gamma eps_k, eps_min) with the 1e-9 snap to eps_min."""
    e = gamma * eps
    if e <= eps_min * (1.0 + 1e-9):
        return eps_min
    return e


def damped_newton(residual, solve, x0, eps0, eps_min, gamma, sigma, tol, kmax,
                  max_halvings=20, floor=None, floor_factor=16.0, norm=None):
    """Alg. 1.

    residual(x, eps) -> F_eps(x) (1-D array)
    solve(x, eps, F) -> d with F'_eps(x) d = -F
    floor(x, eps)    -> ||M|| for the rounding-floor test (or None)
    """
    norm = np.linalg.norm if norm is None else norm
    out = NewtonResult()
    x = np.array(x0, dtype=np.float64, copy=True)
    eps = float(eps0)
    F = residual(x, eps)
    nrm = float(norm(F))
    out.norm0 = nrm
    stop = max(tol, tol * nrm)
    k = 0
    while True:
        if not np.isfinite(nrm):
            out.status = ENONFINITE
            break
        if eps == eps_min:
            if nrm <= stop:
                out.status = OK
                break
            if floor is not None and nrm <= floor_factor * U_ROUND * floor(x, eps):
                out.status = OK_FLOOR
                break
        if k >= kmax:
            out.status = ENOCONV
            break
        d = solve(x, eps, F)
        alpha = 1.0
        h = 0
        while True:
            xt = x + alpha * d
            Ft = residual(xt, eps)
            nt = float(norm(Ft))
            if nt <= sigma * nrm or h == max_halvings:
                break
            alpha *= 0.5
            h += 1
        if not nt <= sigma * nrm:
            out.exhausted += 1
        out.halvings += h
        out.history.append((eps, nrm, alpha))
        x = xt
        eps_next = next_eps(eps, gamma, eps_min)
        if eps_next == eps:
            F, nrm = Ft, nt
        else:
            F = residual(x, eps_next)
            nrm = float(norm(F))
        eps = eps_next
        k += 1
    out.x = x
    out.iterations = k
    out.eps = eps
    out.norm = nrm
    return out
