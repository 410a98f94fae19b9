"""The model problem on the unit cube (Omega = (0,1)^3, Assumption 1 allows
n = 2, 3), with the RASPEN pieces of Sec. 4. Test infrastructure.

Discretisation: A = -Laplace by the 7-point finite-difference stencil on an
n x n x n grid of interior nodes, h = 1/(n+1), zero Dirichlet data. Grid
functions are (n, n, n) float64 arrays indexed [k, j, i] (x1 index i fastest,
then x2, then x3). The residual is F(x, eps) of Sec. 3.3 with x = (y, p):

    F_y = A y + phi(y) - f + (1/nu) (p + mu P_eps(-p/mu))
    F_p = A p + phi'(y) p - y + y_d,

the same nodewise terms as the 2-D discretisation (discretization.py), only
the stencil differs.

A box is (x0, x1, y0, y1, z0, z1), half-open node-index ranges. Local vectors
on a box interleave (y, p) per node, nodes with x1 fastest, then x2, then x3.
The decomposition, the local problems (reading C5: C_i is a correction), Alg. 1
for them, Alg. 3, Alg. 4 and Alg. 2 follow ras.py and solvers.py; the local
Jacobians are factorised by a sparse LU (SuperLU with partial pivoting) as the
library step, since the 3-D band is too wide for a band solver.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import decomposition as dd
from . import pointwise as pw
from .gmres import gmres
from .newton import damped_newton, OK, ENOCONV


class Problem:
    """Data of one discrete control problem (P) on the cube."""

    def __init__(self, n, phi_kind, nu, mu, y_d, f=None, kappa=0.1):
        self.n = int(n)
        self.h = 1.0 / (n + 1)
        self.beta = 1.0 / (self.h * self.h)
        self.phi_kind = phi_kind
        self.kappa = kappa
        self.nu = float(nu)
        self.mu = float(mu)
        self.y_d = np.ascontiguousarray(y_d, dtype=np.float64).reshape(n, n, n)
        self.f = (np.zeros((n, n, n)) if f is None
                  else np.ascontiguousarray(f, dtype=np.float64).reshape(n, n, n))

    def phi(self, y):
        return pw.phi(self.phi_kind, y, self.kappa)


def full_box(n):
    return (0, n, 0, n, 0, n)


def box_shape(box):
    x0, x1, y0, y1, z0, z1 = box
    return (z1 - z0, y1 - y0, x1 - x0)


def _cut(Z, box):
    x0, x1, y0, y1, z0, z1 = box
    return Z[z0:z1, y0:y1, x0:x1]


def apply_A(prob, Z, box=None):
    """(A_h Z) on the box: beta (6 z - sum of the six neighbours), zero outside the grid."""
    box = full_box(prob.n) if box is None else box
    x0, x1, y0, y1, z0, z1 = box
    Zp = np.pad(Z, 1)
    c = Zp[z0 + 1:z1 + 1, y0 + 1:y1 + 1, x0 + 1:x1 + 1]
    nb = (Zp[z0 + 1:z1 + 1, y0 + 1:y1 + 1, x0:x1] + Zp[z0 + 1:z1 + 1, y0 + 1:y1 + 1, x0 + 2:x1 + 2]
          + Zp[z0 + 1:z1 + 1, y0:y1, x0 + 1:x1 + 1] + Zp[z0 + 1:z1 + 1, y0 + 2:y1 + 2, x0 + 1:x1 + 1]
          + Zp[z0:z1, y0 + 1:y1 + 1, x0 + 1:x1 + 1] + Zp[z0 + 2:z1 + 2, y0 + 1:y1 + 1, x0 + 1:x1 + 1])
    return prob.beta * (6.0 * c - nb)


def residual(prob, Y, P, eps, box=None):
    """F(x, eps) of Sec. 3.3 at the nodes of `box`; returns (F_y, F_p)."""
    box = full_box(prob.n) if box is None else box
    y = _cut(Y, box)
    p = _cut(P, box)
    ph, dph, _ = prob.phi(y)
    Fy = (apply_A(prob, Y, box) + ph - _cut(prob.f, box)
          - pw.u_eps(p, eps, prob.nu, prob.mu))
    Fp = apply_A(prob, P, box) + dph * p - y + _cut(prob.y_d, box)
    return Fy, Fp


def residual_floor_norm(prob, Y, P, eps, box=None):
    """2-norm of the nodewise sums of |terms| of F on the box (the size of the
    rounding error of an FP64 evaluation of F, divided by u_round)."""
    box = full_box(prob.n) if box is None else box
    # beta (6 |z| + sum of the six |neighbours|) = -A|Z| + 12 beta |z|
    absA = lambda Z: 12.0 * prob.beta * np.abs(_cut(Z, box)) - apply_A(prob, np.abs(Z), box)
    y, p = _cut(Y, box), _cut(P, box)
    ph, dph, _ = prob.phi(y)
    My = (absA(Y) + np.abs(ph) + np.abs(_cut(prob.f, box))
          + (1.0 / prob.nu) * (np.abs(p) + prob.mu * np.abs(pw.P_eps(-p / prob.mu, eps))))
    Mp = absA(P) + np.abs(dph * p) + np.abs(y) + np.abs(_cut(prob.y_d, box))
    return float(np.sqrt(np.sum(My * My) + np.sum(Mp * Mp)))


def jacvec(prob, Y, P, eps, dY, dP, box=None):
    """F'(x, eps) d at the nodes of `box` (d given on the whole grid)."""
    box = full_box(prob.n) if box is None else box
    y = _cut(Y, box)
    p = _cut(P, box)
    _, dph, d2ph = prob.phi(y)
    b = (1.0 / prob.nu) * pw.one_minus_dP_eps(-p / prob.mu, eps)
    c = d2ph * p - 1.0
    dy = _cut(dY, box)
    dp = _cut(dP, box)
    return apply_A(prob, dY, box) + dph * dy + b * dp, apply_A(prob, dP, box) + c * dy + dph * dp


def laplacian_matrix(beta, wx, wy, wz):
    """Sparse 7-point matrix beta (6 I - neighbours) on a wx x wy x wz node
    block, node q = (kk*wy + jj)*wx + ii; neighbours outside the block dropped."""
    def t(w):
        return sp.diags([-np.ones(w - 1), 2.0 * np.ones(w), -np.ones(w - 1)], [-1, 0, 1])
    Ix, Iy, Iz = sp.identity(wx), sp.identity(wy), sp.identity(wz)
    return (beta * (sp.kron(Iz, sp.kron(Iy, t(wx))) + sp.kron(Iz, sp.kron(t(wy), Ix))
                    + sp.kron(t(wz), sp.kron(Iy, Ix)))).tocsr()


def jacobian_matrix(prob, Y, P, eps, box=None):
    """Sparse Jacobian R F'(x) P of the box nodes, (y, p) interleaved per node."""
    box = full_box(prob.n) if box is None else box
    wz, wy, wx = box_shape(box)
    N = wx * wy * wz
    y = _cut(Y, box).ravel()
    p = _cut(P, box).ravel()
    _, dph, d2ph = prob.phi(y)
    b = (1.0 / prob.nu) * pw.one_minus_dP_eps(-p / prob.mu, eps)
    c = d2ph * p - 1.0
    L = laplacian_matrix(prob.beta, wx, wy, wz)
    planar = sp.bmat([[L + sp.diags(dph), sp.diags(b)], [sp.diags(c), L + sp.diags(dph)]]).tocsr()
    perm = np.empty(2 * N, dtype=np.int64)   # interleaved index -> planar index
    perm[0::2] = np.arange(N)
    perm[1::2] = N + np.arange(N)
    return planar[perm][:, perm].tocsc()


def interleave(Fy, Fp):
    out = np.empty(2 * Fy.size)
    out[0::2] = Fy.ravel()
    out[1::2] = Fp.ravel()
    return out


def deinterleave(v, shape):
    return v[0::2].reshape(shape), v[1::2].reshape(shape)


# ----------------------------------------------------------- decomposition
class Subdomain:
    def __init__(self, index, owned, box):
        self.index = index
        self.owned = owned     # (x0, x1, y0, y1, z0, z1) of tilde Omega_i
        self.box = box         # the same of Omega_i

    @property
    def shape(self):
        return box_shape(self.box)


def subdomains(n, sx, sy, sz, overlap):
    """Balanced blocks in every direction grown by `overlap` layers (clipped);
    index i = (bz * sy + by) * sx + bx."""
    if overlap < 0:
        raise ValueError("overlap must be >= 0")
    out = []
    for bz, (oz0, oz1) in enumerate(dd.blocks(n, sz)):
        for by, (oy0, oy1) in enumerate(dd.blocks(n, sy)):
            for bx, (ox0, ox1) in enumerate(dd.blocks(n, sx)):
                box = (max(0, ox0 - overlap), min(n, ox1 + overlap), max(0, oy0 - overlap),
                       min(n, oy1 + overlap), max(0, oz0 - overlap), min(n, oz1 + overlap))
                out.append(Subdomain((bz * sy + by) * sx + bx, (ox0, ox1, oy0, oy1, oz0, oz1), box))
    return out


def prolong_restricted(z, sub, n):
    """tilde P_i: box values -> grid function keeping only the owned nodes."""
    x0, x1, y0, y1, z0, z1 = sub.box
    ox0, ox1, oy0, oy1, oz0, oz1 = sub.owned
    Z = np.zeros((n, n, n))
    Z[oz0:oz1, oy0:oy1, ox0:ox1] = z[oz0 - z0:oz1 - z0, oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0]
    return Z


# ------------------------------------------------------- local problems
class LocalResult:
    def __init__(self, sub, newton, Yi, Pi):
        self.sub = sub
        self.newton = newton
        self.C = newton.x
        self.Yi, self.Pi = Yi, Pi   # x^(i) = x + P_i C_i(x)
        self.factor = None


def _shifted_state(Y, P, sub, c):
    cy, cp = deinterleave(c, sub.shape)
    Yi, Pi = Y.copy(), P.copy()
    x0, x1, y0, y1, z0, z1 = sub.box
    Yi[z0:z1, y0:y1, x0:x1] += cy
    Pi[z0:z1, y0:y1, x0:x1] += cp
    return Yi, Pi


def local_factor(prob, Yi, Pi, eps, sub):
    return spla.splu(jacobian_matrix(prob, Yi, Pi, eps, sub.box))


def local_correction(prob, Y, P, sub, eps0, eps_min, opts):
    """C_i(x): Alg. 1 on K_i(c) = R_i F_eps(x + P_i c) from c = 0 (Sec. 4.2)."""
    def res(c, eps):
        Yi, Pi = _shifted_state(Y, P, sub, c)
        return interleave(*residual(prob, Yi, Pi, eps, sub.box))

    def solve(c, eps, F):
        Yi, Pi = _shifted_state(Y, P, sub, c)
        return -local_factor(prob, Yi, Pi, eps, sub).solve(F)

    def floor(c, eps):
        Yi, Pi = _shifted_state(Y, P, sub, c)
        return residual_floor_norm(prob, Yi, Pi, eps, sub.box)

    wz, wy, wx = sub.shape
    r = damped_newton(res, solve, np.zeros(2 * wx * wy * wz), eps0, eps_min, opts.gamma, opts.sigma,
                      opts.inner_tol, opts.kmax_inner, opts.max_halvings, floor, opts.floor_factor)
    Yi, Pi = _shifted_state(Y, P, sub, r.x)
    out = LocalResult(sub, r, Yi, Pi)
    out.factor = local_factor(prob, Yi, Pi, eps_min, sub)
    return out


class RasState:
    def __init__(self, Fy, Fp, locals_, eps_min):
        self.Fy, self.Fp = Fy, Fp
        self.locals = locals_
        self.eps_min = eps_min

    @property
    def iterations(self):
        return [l.newton.iterations for l in self.locals]


def ras_apply(prob, Y, P, subs, opts, continuation):
    """Alg. 3: F_eps(x) = sum_i tilde P_i C_i(x)."""
    n = prob.n
    eps0 = opts.eps0 if continuation else opts.eps_min
    Fy = np.zeros((n, n, n))
    Fp = np.zeros((n, n, n))
    locs = []
    for sub in subs:
        loc = local_correction(prob, Y, P, sub, eps0, opts.eps_min, opts)
        cy, cp = deinterleave(loc.C, sub.shape)
        Fy += prolong_restricted(cy, sub, n)
        Fp += prolong_restricted(cp, sub, n)
        locs.append(loc)
    return RasState(Fy, Fp, locs, opts.eps_min)


def jvp(prob, state, dY, dP):
    """Alg. 4: sum_i tilde P_i C_i'(x) d, C_i'(x) d = -(R_i F' P_i)^-1 R_i F'(x^(i)) d."""
    n = prob.n
    oy = np.zeros((n, n, n))
    op = np.zeros((n, n, n))
    for loc in state.locals:
        vy, vp = jacvec(prob, loc.Yi, loc.Pi, state.eps_min, dY, dP, loc.sub.box)
        zy, zp = deinterleave(-loc.factor.solve(interleave(vy, vp)), loc.sub.shape)
        oy += prolong_restricted(zy, loc.sub, n)
        op += prolong_restricted(zp, loc.sub, n)
    return oy, op


class SolveResult:
    def __init__(self):
        self.Y = self.P = None
        self.outer = 0
        self.gmres_its = []
        self.inner_its = []
        self.status = OK


def _split(v, n):
    N = n ** 3
    return v[:N].reshape(n, n, n), v[N:].reshape(n, n, n)


def _join(a, b):
    return np.concatenate([a.ravel(), b.ravel()])


def raspen(prob, sx, sy, sz, overlap, opts):
    """Alg. 2: Newton on F_eps(x) = 0 from x = 0, undamped, GMRES with Alg. 4;
    continuation only in the first evaluation's local solves."""
    n = prob.n
    subs = subdomains(n, sx, sy, sz, overlap)
    Y = np.zeros((n, n, n))
    P = np.zeros((n, n, n))
    out = SolveResult()
    state = ras_apply(prob, Y, P, subs, opts, continuation=True)
    out.inner_its.append(state.iterations)
    Fn = float(np.linalg.norm(_join(state.Fy, state.Fp)))
    stop = max(opts.tol, opts.tol * Fn)
    k = 0
    while Fn > stop and k < opts.kmax_outer_raspen:
        def A(v):
            return _join(*jvp(prob, state, *_split(v, n)))
        g = gmres(A, -_join(state.Fy, state.Fp), opts.gmres_restart, opts.gmres_rtol, opts.gmres_maxit)
        out.gmres_its.append(g.iterations)
        dY, dP = _split(g.x, n)
        Y, P = Y + dY, P + dP
        k += 1
        state = ras_apply(prob, Y, P, subs, opts, continuation=False)
        out.inner_its.append(state.iterations)
        Fn = float(np.linalg.norm(_join(state.Fy, state.Fp)))
    out.status = OK if Fn <= stop else ENOCONV
    out.Y, out.P, out.outer = Y, P, k
    return out
