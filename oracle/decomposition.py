"""Overlapping domain decomposition of Sec. 4.2. Test infrastructure.

* The non-overlapping subdomains (tilde Omega_i) split the n interior nodes of
  each direction into s balanced blocks: the first (n mod s) blocks have
  ceil(n/s) nodes, the rest floor(n/s).
* Each overlapping subdomain Omega_i is its block grown by `overlap` node
  layers on every side, clipped at the boundary of Omega.
* Subdomain index i = by * sx + bx (x1 direction fastest).
* R_i restricts a grid function to Omega_i, P_i extends by zero from Omega_i,
  and the restricted prolongation tilde P_i extends by zero from the
  non-overlapping part tilde Omega_i only. They satisfy R_i P_i = I and
  sum_i tilde P_i R_i = I (Sec. 4.2).
"""
import numpy as np


def blocks(n, s):
    """Start and end (half-open) of the s balanced blocks of range(n)."""
    if not (1 <= s <= n):
        raise ValueError("need 1 <= s <= n")
    sizes = [n // s + (1 if k < n % s else 0) for k in range(s)]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    return [(int(starts[k]), int(starts[k + 1])) for k in range(s)]


class Subdomain:
    def __init__(self, index, owned, box):
        self.index = index
        self.owned = owned     # (x0, x1, y0, y1) of tilde Omega_i
        self.box = box         # (x0, x1, y0, y1) of Omega_i

    @property
    def wx(self):
        return self.box[1] - self.box[0]

    @property
    def wy(self):
        return self.box[3] - self.box[2]


def subdomains(n, sx, sy, overlap):
    if overlap < 0:
        raise ValueError("overlap must be >= 0")
    bxs = blocks(n, sx)
    bys = blocks(n, sy)
    out = []
    for by, (oy0, oy1) in enumerate(bys):
        for bx, (ox0, ox1) in enumerate(bxs):
            box = (max(0, ox0 - overlap), min(n, ox1 + overlap),
                   max(0, oy0 - overlap), min(n, oy1 + overlap))
            out.append(Subdomain(by * sx + bx, (ox0, ox1, oy0, oy1), box))
    return out


def restrict(Z, box):
    """R_i: grid function -> its values on the box."""
    x0, x1, y0, y1 = box
    return Z[y0:y1, x0:x1].copy()


def prolong(z, box, n):
    """P_i: box values -> grid function, zero outside the box."""
    x0, x1, y0, y1 = box
    Z = np.zeros((n, n))
    Z[y0:y1, x0:x1] = z
    return Z


def prolong_restricted(z, sub, n):
    """tilde P_i: box values -> grid function keeping only the owned nodes."""
    x0, x1, y0, y1 = sub.box
    ox0, ox1, oy0, oy1 = sub.owned
    Z = np.zeros((n, n))
    Z[oy0:oy1, ox0:ox1] = z[oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0]
    return Z
