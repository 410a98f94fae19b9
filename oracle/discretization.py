"""Finite-difference discretisation of the reduced smoothed system. Test infrastructure.

The model problem of Sec. 4: Omega = (0,1)^2, A = -Laplace with homogeneous
Dirichlet conditions, discretised by the 5-point finite-difference stencil on a
uniform grid of n x n interior nodes, h = 1/(n+1). Nonlinearities act nodewise.

Grid functions are (n, n) float64 arrays indexed [j, i]: i is the x1 index
(fastest), j the x2 index; node (i, j) sits at (x1, x2) = ((i+1)h, (j+1)h).

The residual is the map F(x, eps) of Sec. 3.3 with x = (y, p):

    F_y = A y + phi(y) - f + (1/nu) (p + mu P_eps(-p/mu))   (= A y + phi(y) - f - u_eps(p))
    F_p = A p + phi'(y) p - y + y_d

and its Jacobian (Sec. 3.3)

    [[A + phi'(y),      (1/nu)(I - P_eps'(-p/mu))],
     [phi''(y) p - I,    A + phi'(y)             ]].

A "box" is (x0, x1, y0, y1), half-open node-index ranges in i and j. Evaluating
F on a box uses the values of (y, p) on the box and on the ring of nodes around
it (zero outside the grid), which is all the 5-point stencil reads.
"""
import numpy as np
import scipy.sparse as sp

from . import pointwise as pw


class Problem:
    """Data of one discrete control problem (P): grid, phi, nu, mu, y_d, f."""

    def __init__(self, n, phi_kind, nu, mu, y_d, f=None, kappa=0.1):
        self.n = int(n)
        self.h = 1.0 / (n + 1)
        self.beta = 1.0 / (self.h * self.h)
        self.phi_kind = phi_kind
        self.kappa = kappa
        self.nu = float(nu)
        self.mu = float(mu)
        self.y_d = np.ascontiguousarray(y_d, dtype=np.float64).reshape(n, n)
        self.f = (np.zeros((n, n)) if f is None
                  else np.ascontiguousarray(f, dtype=np.float64).reshape(n, n))

    def phi(self, y):
        return pw.phi(self.phi_kind, y, self.kappa)


def full_box(n):
    return (0, n, 0, n)


def _stencil_parts(Z, box):
    """Centre values and the four neighbours of every box node (zero Dirichlet)."""
    x0, x1, y0, y1 = box
    Zp = np.pad(Z, 1)
    c = Zp[y0 + 1:y1 + 1, x0 + 1:x1 + 1]
    w = Zp[y0 + 1:y1 + 1, x0:x1]
    e = Zp[y0 + 1:y1 + 1, x0 + 2:x1 + 2]
    s = Zp[y0:y1, x0 + 1:x1 + 1]
    nn = Zp[y0 + 2:y1 + 2, x0 + 1:x1 + 1]
    return c, w, e, s, nn


def apply_A(prob, Z, box=None):
    """(A_h Z) on the box: beta (4 z - sum of the four neighbours)."""
    box = full_box(prob.n) if box is None else box
    c, w, e, s, nn = _stencil_parts(Z, box)
    return prob.beta * (4.0 * c - w - e - s - nn)


def residual(prob, Y, P, eps, box=None):
    """F(x, eps) of Sec. 3.3 evaluated at the nodes of `box`; returns (F_y, F_p)."""
    box = full_box(prob.n) if box is None else box
    x0, x1, y0, y1 = box
    y = Y[y0:y1, x0:x1]
    p = P[y0:y1, x0:x1]
    ph, dph, _ = prob.phi(y)
    Fy = (apply_A(prob, Y, box) + ph - prob.f[y0:y1, x0:x1]
          - pw.u_eps(p, eps, prob.nu, prob.mu))
    Fp = apply_A(prob, P, box) + dph * p - y + prob.y_d[y0:y1, x0:x1]
    return Fy, Fp


def residual_floor_norm(prob, Y, P, eps, box=None):
    """2-norm of the nodewise sums of |terms| of F on the box.

    u_round times this number is the size of the rounding error of an FP64
    evaluation of F. The stop tests use it to recognise a residual that has
    reached rounding level when the requested tolerance lies below that level.
    """
    box = full_box(prob.n) if box is None else box
    x0, x1, y0, y1 = box
    cy, wy, ey, sy, ny = _stencil_parts(Y, box)
    cp, wp, ep, spp, npp = _stencil_parts(P, box)
    ph, dph, _ = prob.phi(cy)
    My = (prob.beta * (4.0 * np.abs(cy) + np.abs(wy) + np.abs(ey) + np.abs(sy) + np.abs(ny))
          + np.abs(ph) + np.abs(prob.f[y0:y1, x0:x1])
          + (1.0 / prob.nu) * (np.abs(cp) + prob.mu * np.abs(pw.P_eps(-cp / prob.mu, eps))))
    Mp = (prob.beta * (4.0 * np.abs(cp) + np.abs(wp) + np.abs(ep) + np.abs(spp) + np.abs(npp))
          + np.abs(dph * cp) + np.abs(cy) + np.abs(prob.y_d[y0:y1, x0:x1]))
    return float(np.sqrt(np.sum(My * My) + np.sum(Mp * Mp)))


def jacobian_coefficients(prob, y, p, eps):
    """Nodewise entries of the Jacobian (Sec. 3.3): diagonal addend phi'(y),
    (1,2) block (1/nu)(1 - P_eps'(-p/mu)), (2,1) block phi''(y) p - 1."""
    _, dph, d2ph = prob.phi(y)
    b = (1.0 / prob.nu) * pw.one_minus_dP_eps(-p / prob.mu, eps)
    c = d2ph * p - 1.0
    return dph, b, c


def jacvec(prob, Y, P, eps, dY, dP, box=None):
    """F'(x, eps) d evaluated at the nodes of `box` (d given on the whole grid)."""
    box = full_box(prob.n) if box is None else box
    x0, x1, y0, y1 = box
    dph, b, c = jacobian_coefficients(prob, Y[y0:y1, x0:x1], P[y0:y1, x0:x1], eps)
    dy = dY[y0:y1, x0:x1]
    dp = dP[y0:y1, x0:x1]
    Jy = apply_A(prob, dY, box) + dph * dy + b * dp
    Jp = apply_A(prob, dP, box) + c * dy + dph * dp
    return Jy, Jp


def laplacian_matrix(beta, wx, wy):
    """Sparse 5-point matrix beta (4 I - neighbours) on a wx-by-wy node block,
    node index q = jj*wx + ii; neighbours outside the block are dropped."""
    tx = sp.diags([-np.ones(wx - 1), 2.0 * np.ones(wx), -np.ones(wx - 1)], [-1, 0, 1])
    ty = sp.diags([-np.ones(wy - 1), 2.0 * np.ones(wy), -np.ones(wy - 1)], [-1, 0, 1])
    return (beta * (sp.kron(sp.identity(wy), tx) + sp.kron(ty, sp.identity(wx)))).tocsr()


def jacobian_matrix(prob, Y, P, eps, box=None, interleaved=True):
    """Sparse Jacobian block R F'(x) P of the box nodes (whole grid by default).

    Restricting F' to the rows and columns of a box keeps the box's own 5-point
    couplings; couplings to nodes outside the box belong to the dropped columns.
    Ordering: interleaved (unknown 2q + field, field 0 = y, 1 = p) or planar
    ([all y; all p]).
    """
    box = full_box(prob.n) if box is None else box
    x0, x1, y0, y1 = box
    wx, wy = x1 - x0, y1 - y0
    dph, b, c = jacobian_coefficients(prob, Y[y0:y1, x0:x1], P[y0:y1, x0:x1], eps)
    L = laplacian_matrix(prob.beta, wx, wy)
    Dd = sp.diags(dph.ravel())
    J = sp.bmat([[L + Dd, sp.diags(b.ravel())],
                 [sp.diags(c.ravel()), L + Dd]]).tocsr()
    if not interleaved:
        return J
    m = wx * wy
    perm = np.empty(2 * m, dtype=np.int64)
    perm[0::2] = np.arange(m)
    perm[1::2] = m + np.arange(m)
    return J[perm][:, perm].tocsr()


def to_band(J, kl, ku):
    """LAPACK general-band storage with kl extra rows for pivot fill:
    ab[kl + ku + r - col, col] = J[r, col]."""
    J = J.tocoo()
    N = J.shape[0]
    ab = np.zeros((2 * kl + ku + 1, N))
    if np.any(J.row - J.col > kl) or np.any(J.col - J.row > ku):
        raise ValueError("matrix exceeds the stated band")
    ab[kl + ku + J.row - J.col, J.col] = J.data
    return ab


def interleave(Fy, Fp):
    """Planar (wy, wx) pair -> interleaved local vector of length 2*wx*wy."""
    v = np.empty(2 * Fy.size)
    v[0::2] = Fy.ravel()
    v[1::2] = Fp.ravel()
    return v


def deinterleave(v, wx, wy):
    return v[0::2].reshape(wy, wx), v[1::2].reshape(wy, wx)
