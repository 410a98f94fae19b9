"""Nonlinear RAS pieces of Sec. 4.2. Test infrastructure.

* local_correction: C_i(x), the solution of the local problem
      K_i(c) = R_i F_eps(x + P_i c) = 0
  (reading of the local-correction equation: C_i is a correction added to x on
  Omega_i, with Dirichlet data x on the ring around Omega_i and 0 on the
  boundary of Omega), computed by Alg. 1 from c = 0 with a direct band solve of
  the local Jacobian J_i = R_i F'_eps(x + P_i c) P_i (LAPACK dgbtrf/dgbtrs,
  partial pivoting).
* ras_apply: Alg. 3, F_eps(x) = sum_i tilde P_i C_i(x) (the RASPEN function),
  keeping every C_i and a factorisation of J_i at x^(i) = x + P_i C_i(x).
* jvp: Alg. 4, F_eps'(x) d = sum_i tilde P_i C_i'(x) d with
      C_i'(x) d = -(R_i F'_eps(x^(i)) P_i)^-1 R_i F'_eps(x^(i)) d,
  written literally: the full product R_i F'(x^(i)) d, then the local solve.
* ras_precondition: the linear RAS preconditioner
      M^-1 r = sum_i tilde P_i (R_i F'_eps(x) P_i)^-1 R_i r.
"""
import numpy as np
from scipy.linalg import lapack

from . import discretization as fd
from . import decomposition as dd
from .newton import damped_newton


class Options:
    """Solver parameters. Defaults are the paper's settings (Sec. 5): outer tol
    1e-10, inner tol 1e-8, eps_0 = 1, gamma = 1/5, sigma = 1.1."""

    def __init__(self, **kw):
        self.tol = 1e-10
        self.inner_tol = 1e-8
        self.sigma = 1.1
        self.eps0 = 1.0
        self.gamma = 0.2
        self.eps_min = 1e-6
        self.kmax_outer_raspen = 50
        self.kmax_outer_newton = 200
        self.kmax_inner = 100
        self.max_halvings = 20
        self.gmres_restart = 30
        self.gmres_rtol = 1e-8
        self.gmres_maxit = 1000
        self.floor_factor = 16.0
        for k, v in kw.items():
            if not hasattr(self, k):
                raise KeyError(k)
            setattr(self, k, v)


class SingularJacobian(RuntimeError):
    pass


class BandFactor:
    """LU with partial pivoting of a local Jacobian in band storage (LAPACK)."""

    def __init__(self, J, kl, ku):
        self.kl, self.ku = kl, ku
        ab = fd.to_band(J, kl, ku)
        self.lu, self.piv, info = lapack.dgbtrf(ab, kl, ku)
        if info != 0:
            raise SingularJacobian("dgbtrf info=%d" % info)

    def solve(self, rhs):
        x, info = lapack.dgbtrs(self.lu, self.kl, self.ku, np.asarray(rhs, dtype=np.float64), self.piv)
        if info != 0:
            raise RuntimeError("dgbtrs info=%d" % info)
        return x


def _shifted_state(Y, P, sub, c):
    """x + P_i c as full grid functions."""
    x0, x1, y0, y1 = sub.box
    cy, cp = fd.deinterleave(c, sub.wx, sub.wy)
    Yi = Y.copy()
    Pi = P.copy()
    Yi[y0:y1, x0:x1] += cy
    Pi[y0:y1, x0:x1] += cp
    return Yi, Pi


def local_jacobian_factor(prob, Yi, Pi, eps, sub):
    J = fd.jacobian_matrix(prob, Yi, Pi, eps, sub.box, interleaved=True)
    return BandFactor(J, 2 * sub.wx, 2 * sub.wx)


class LocalResult:
    def __init__(self, sub, newton, Yi, Pi):
        self.sub = sub
        self.newton = newton
        self.C = newton.x          # C_i(x), interleaved local vector
        self.Yi, self.Pi = Yi, Pi  # x^(i) = x + P_i C_i(x)
        self.factor = None         # factorisation of J_i at x^(i), eps_min


def local_correction(prob, Y, P, sub, eps0, eps_min, opts, factor_at_solution=True):
    """C_i(x) by Alg. 1 on K_i, from c = 0 (Sec. 4.2, Alg. 3)."""
    box = sub.box

    def residual(c, eps):
        Yi, Pi = _shifted_state(Y, P, sub, c)
        return fd.interleave(*fd.residual(prob, Yi, Pi, eps, box))

    def solve(c, eps, F):
        Yi, Pi = _shifted_state(Y, P, sub, c)
        return -local_jacobian_factor(prob, Yi, Pi, eps, sub).solve(F)

    def floor(c, eps):
        Yi, Pi = _shifted_state(Y, P, sub, c)
        return fd.residual_floor_norm(prob, Yi, Pi, eps, box)

    res = damped_newton(residual, solve, np.zeros(2 * sub.wx * sub.wy), eps0, eps_min,
                        opts.gamma, opts.sigma, opts.inner_tol, opts.kmax_inner,
                        opts.max_halvings, floor, opts.floor_factor)
    Yi, Pi = _shifted_state(Y, P, sub, res.x)
    out = LocalResult(sub, res, Yi, Pi)
    if factor_at_solution:
        out.factor = local_jacobian_factor(prob, Yi, Pi, eps_min, sub)
    return out


class RasState:
    """Output of Alg. 3: F_eps(x) and the stored local results."""

    def __init__(self, Fy, Fp, locals_, eps_min):
        self.Fy, self.Fp = Fy, Fp
        self.locals = locals_
        self.eps_min = eps_min

    @property
    def iterations(self):
        return [l.newton.iterations for l in self.locals]

    @property
    def statuses(self):
        return [l.newton.status for l in self.locals]


def ras_apply(prob, Y, P, subs, opts, continuation, factor_at_solution=True, only=None):
    """Alg. 3: local corrections for every subdomain, then
    F_eps(x) = sum_i tilde P_i C_i(x). With continuation the local Newton
    solves start at eps_0, otherwise at eps_min. `only` restricts the work to a
    list of subdomain indices (used for sampled checks)."""
    n = prob.n
    eps0 = opts.eps0 if continuation else opts.eps_min
    Fy = np.zeros((n, n))
    Fp = np.zeros((n, n))
    locs = []
    for sub in subs:
        if only is not None and sub.index not in only:
            continue
        loc = local_correction(prob, Y, P, sub, eps0, opts.eps_min, opts, factor_at_solution)
        cy, cp = fd.deinterleave(loc.C, sub.wx, sub.wy)
        Fy += dd.prolong_restricted(cy, sub, n)
        Fp += dd.prolong_restricted(cp, sub, n)
        locs.append(loc)
    return RasState(Fy, Fp, locs, opts.eps_min)


def local_jvp(prob, loc, eps_min, dY, dP):
    """C_i'(x) d = -(R_i F'(x^(i)) P_i)^-1 R_i F'(x^(i)) d on the box of
    subdomain i (one term of Alg. 4), written literally: the full product
    R_i F'(x^(i)) d, then the local solve. Returns the two box fields."""
    sub = loc.sub
    vy, vp = fd.jacvec(prob, loc.Yi, loc.Pi, eps_min, dY, dP, sub.box)
    z = loc.factor.solve(fd.interleave(vy, vp))
    return fd.deinterleave(-z, sub.wx, sub.wy)


def jvp(prob, state, dY, dP):
    """Alg. 4: F_eps'(x) d = sum_i tilde P_i C_i'(x) d."""
    n = prob.n
    out_y = np.zeros((n, n))
    out_p = np.zeros((n, n))
    for loc in state.locals:
        zy, zp = local_jvp(prob, loc, state.eps_min, dY, dP)
        out_y += dd.prolong_restricted(zy, loc.sub, n)
        out_p += dd.prolong_restricted(zp, loc.sub, n)
    return out_y, out_p


class SerialEngine:
    """Alg. 3 and Alg. 4 over the subdomains one after another."""

    def __init__(self, prob, subs, opts):
        self.prob, self.subs, self.opts = prob, subs, opts

    def apply(self, Y, P, continuation):
        return ras_apply(self.prob, Y, P, self.subs, self.opts, continuation)

    def jvp(self, state, dY, dP):
        return jvp(self.prob, state, dY, dP)


class LinearRas:
    """Linear RAS preconditioner with the local Jacobians at x (c = 0)."""

    def __init__(self, prob, Y, P, subs, eps):
        self.prob = prob
        self.subs = subs
        self.factors = [local_jacobian_factor(prob, Y, P, eps, s) for s in subs]

    def apply(self, rY, rP):
        n = self.prob.n
        oy = np.zeros((n, n))
        op = np.zeros((n, n))
        for sub, fac in zip(self.subs, self.factors):
            r = fd.interleave(dd.restrict(rY, sub.box), dd.restrict(rP, sub.box))
            z = fac.solve(r)
            zy, zp = fd.deinterleave(z, sub.wx, sub.wy)
            oy += dd.prolong_restricted(zy, sub, n)
            op += dd.prolong_restricted(zp, sub, n)
        return oy, op
