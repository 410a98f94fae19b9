"""Restarted GMRES(m), the matrix-free Krylov solver of Sec. 4 (Alg. 2, Newton_RAS).
Test infrastructure.

The paper does not give restart length, tolerance, orthogonalisation or the
side of preconditioning. Readings: x0 = 0; Arnoldi with classical Gram-Schmidt
applied twice (CGS2); Givens rotations on the Hessenberg matrix; stop when the
residual estimate is <= rtol ||b||; restart after m steps from the true
residual; at most maxit steps in total; optional right preconditioner M, so the
iterate is x = M(V y).
"""
import numpy as np
from scipy.linalg import solve_triangular


class GmresResult:
    def __init__(self, x, iterations, converged, resnorm):
        self.x = x
        self.iterations = iterations
        self.converged = converged
        self.resnorm = resnorm


def gmres(A, b, m=30, rtol=1e-8, maxit=1000, M=None):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return GmresResult(x, 0, True, 0.0)
    target = rtol * bnorm
    total = 0
    r = b.copy()
    while True:
        beta = float(np.linalg.norm(r))
        if beta <= target or total >= maxit:
            return GmresResult(x, total, beta <= target, beta)
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        steps = 0
        for j in range(m):
            z = M(V[j]) if M is not None else V[j]
            w = A(z)
            h1 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h1
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h1 + h2
            hn = float(np.linalg.norm(w))
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = float(np.hypot(H[j, j], H[j + 1, j]))
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            steps = j + 1
            if hn == 0.0 or abs(g[j + 1]) <= target or total >= maxit:
                break
            V[j + 1] = w / hn
        y = solve_triangular(H[:steps, :steps], g[:steps])
        upd = V[:steps].T @ y
        x = x + (M(upd) if M is not None else upd)
        r = b - A(x)
