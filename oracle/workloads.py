"""The paper's model problem with a manufactured solution (Sec. 4). Test infrastructure.

Sec. 4 fixes Omega = (0,1)^2, A = -Laplace, phi(y) = kappa (y^3 + exp(kappa y))
with kappa = 0.1, nu = 1e-6, mu = 1, f = 0, the adjoint

    pbar = 1.3 mu sin(2 pi k x1) sin(2 pi k x2),   k = 5,

the state ybar as the solution of the state equation at eps = 1e-15, and

    y_d = -A pbar - phi'(ybar) pbar + ybar,

so that (ybar, pbar) solves the optimality system at that eps.

Reading (the paper prints the state equation with -(1/nu)(pbar + mu P_eps(-pbar/mu))):
with the sign of the system of Sec. 3.3 (the F_y of discretization.py) only
+(1/nu)(...) makes (ybar, pbar) a solution, so ybar solves F_y(ybar, pbar) = 0:
A y + phi(y) - f + (1/nu)(pbar + mu P_eps(-pbar/mu)) = 0.

The state equation is solved by damped Newton with sparse direct solves of
A + diag(phi'(y)) (symmetric positive definite: phi' > 0).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretization as fd
from . import pointwise as pw


def state_solve(prob, P, eps, rtol=1e-14, kmax=100):
    """ybar with F_y(ybar, P) = 0 (Sec. 3.3 F_y at fixed adjoint P), from y = 0.
    Backtracking halves the step until ||F_y|| decreases by the factor
    1 - 1e-4 alpha. Stops at ||F_y|| <= rtol ||F_y(0)||, or when no step
    decreases ||F_y|| any more (rounding level); raises if neither happens."""
    n = prob.n
    L = fd.laplacian_matrix(prob.beta, n, n)
    Y = np.zeros((n, n))

    def fy(Yv):
        return fd.residual(prob, Yv, P, eps)[0]

    F = fy(Y)
    nrm0 = nrm = float(np.linalg.norm(F))
    for _ in range(kmax):
        if nrm <= rtol * nrm0:
            return Y
        _, dph, _ = prob.phi(Y)
        J = (L + sp.diags(dph.ravel())).tocsc()
        d = spla.spsolve(J, -F.ravel()).reshape(n, n)
        alpha, moved = 1.0, False
        for _h in range(40):
            Ft = fy(Y + alpha * d)
            nt = float(np.linalg.norm(Ft))
            if nt <= (1.0 - 1e-4 * alpha) * nrm:
                Y, F, nrm, moved = Y + alpha * d, Ft, nt, True
                break
            alpha *= 0.5
        if not moved:
            if nrm <= 1e-9 * nrm0:
                return Y
            raise RuntimeError("state solve stalled at ||F_y|| = %g (initial %g)" % (nrm, nrm0))
    raise RuntimeError("state solve did not converge in %d steps" % kmax)


def manufactured(pbar, n, nu=1e-6, mu=1.0, kappa=0.1, eps=1e-15, f=None):
    """(ybar, y_d) of Sec. 4 for the adjoint pbar ((n, n) array) with phi =
    kappa (y^3 + exp(kappa y)): ybar from the state equation at eps, then
    y_d = -A pbar - phi'(ybar) pbar + ybar, so that F(ybar, pbar, eps) = 0."""
    prob = fd.Problem(n, pw.PHI_KAPPA, nu, mu, np.zeros((n, n)), f, kappa=kappa)
    Y = state_solve(prob, pbar, eps)
    _, dph, _ = prob.phi(Y)
    y_d = -fd.apply_A(prob, pbar) - dph * pbar + Y
    return Y, y_d
