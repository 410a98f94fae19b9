"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module generates problem data only (desired states y_d, parameters,
batches, arrival streams). It holds none of the solver's arithmetic, imports
nothing from the solver, and is safe to import without a GPU.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the two xor-shift-multiply mixing rounds with 0xBF58476D1CE4E5B9 and
0x94D049BB133111EB; a double in [0, 1) is the top 53 bits times 2^-53.

Grid functions are (n, n) float64 arrays indexed [j, i] (i = x1 index,
fastest); node (i, j) sits at ((i+1)h, (j+1)h), h = 1/(n+1).
"""
import math

import numpy as np

_MASK = (1 << 64) - 1

PHI_CUBIC = 0
PHI_EXP = 1
PHI_KAPPA = 2


class SplitMix64:
    def __init__(self, seed):
        self.state = int(seed) & _MASK

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self):
        return (self.next_u64() >> 11) * (2.0 ** -53)

    def randint(self, lo, hi):
        """Integer uniform on [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def log_uniform(self, lo, hi):
        return math.exp(math.log(lo) + self.uniform() * (math.log(hi) - math.log(lo)))


def coords(n):
    h = 1.0 / (n + 1)
    return (np.arange(n) + 1.0) * h


def yd_sine(n):
    """y_d(x1, x2) = sin(2 pi x1) sin(2 pi x2)."""
    x = coords(n)
    return np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x))


def yd_fourier(n, seed, modes=8, fmax=6):
    """Sum of `modes` products sin(2 pi j x1) sin(2 pi l x2) with amplitude
    a ~ U(-1, 1) and frequencies j, l ~ U{1..fmax}, drawn in the order
    (a, j, l) per mode from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    x = coords(n)
    y = np.zeros((n, n))
    for _ in range(modes):
        a = 2.0 * rng.uniform() - 1.0
        j = rng.randint(1, fmax)
        l = rng.randint(1, fmax)
        y += a * np.outer(np.sin(2 * np.pi * l * x), np.sin(2 * np.pi * j * x))
    return y


def yd_manufactured_paper(n, mu=1.0, ktilde=5):
    """The adjoint pbar = 1.3 mu sin(2 pi k x1) sin(2 pi k x2) of the paper's
    model problem (Sec. 4); y_d is then derived from it by the solver side."""
    x = coords(n)
    return 1.3 * mu * np.outer(np.sin(2 * np.pi * ktilde * x), np.sin(2 * np.pi * ktilde * x))


def problem(name, **over):
    """Named workloads. Each entry: n, layout (sx, sy), overlap, phi, nu, mu,
    y_d, eps schedule (eps0, gamma, eps_min), tolerances."""
    base = dict(eps0=0.1, gamma=0.1, eps_min=1e-6, tol=1e-10, inner_tol=1e-8, sigma=1.1,
                kappa=0.1)
    if name == "n63":            # 63^2 grid, 4x4 subdomains, overlap 2
        cfg = dict(n=63, sx=4, sy=4, overlap=2, phi=PHI_CUBIC, nu=1e-4, mu=1e-3, yd=("sine",))
    elif name == "n255":         # 255^2 grid, 8x8 subdomains, overlap 4, GMRES(30)
        cfg = dict(n=255, sx=8, sy=8, overlap=4, phi=PHI_CUBIC, nu=1e-5, mu=1e-3, yd=("fourier", 1))
    elif name == "n1023":        # 1023^2 grid, 16x16 subdomains of 64^2, overlap 8
        cfg = dict(n=1023, sx=16, sy=16, overlap=8, phi=PHI_CUBIC, nu=1e-6, mu=1e-2, yd=("fourier", 1))
    elif name == "n511":         # same subdomain shape as n1023 on a 511^2 grid (8x8 subdomains)
        cfg = dict(n=511, sx=8, sy=8, overlap=8, phi=PHI_CUBIC, nu=1e-6, mu=1e-2, yd=("fourier", 1))
    elif name == "n1023_active":  # n1023 with mu = 1e-3: the L1 term is active (nonzero control)
        cfg = dict(n=1023, sx=16, sy=16, overlap=8, phi=PHI_CUBIC, nu=1e-6, mu=1e-3, yd=("fourier", 1))
    elif name.startswith("weak"):  # weak-scaling layout: s x s subdomains of 50^2 nodes, overlap 2
        s_ = int(name[4:])
        cfg = dict(n=50 * s_, sx=s_, sy=s_, overlap=2, phi=PHI_CUBIC, nu=1e-6, mu=1e-2, yd=("fourier", 1))
    else:
        raise KeyError(name)
    base.update(cfg)
    base.update(over)
    return base


def make_yd(cfg):
    kind = cfg["yd"]
    if kind[0] == "sine":
        return yd_sine(cfg["n"])
    if kind[0] == "fourier":
        return yd_fourier(cfg["n"], kind[1])
    raise KeyError(kind)


def yd_sine3(n):
    """The cube: y_d(x1, x2, x3) = sin(2 pi x1) sin(2 pi x2) sin(2 pi x3), an
    (n, n, n) array indexed [k, j, i] (x1 fastest)."""
    s = np.sin(2 * np.pi * coords(n))
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


def yd_fourier3(n, seed, modes=8, fmax=4):
    """The cube: sum of `modes` products sin(2 pi a x1) sin(2 pi b x2)
    sin(2 pi c x3), amplitude ~ U(-1, 1), frequencies ~ U{1..fmax}, drawn in the
    order (amplitude, a, b, c) per mode from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    x = coords(n)
    y = np.zeros((n, n, n))
    for _ in range(modes):
        amp = 2.0 * rng.uniform() - 1.0
        a, b, c = rng.randint(1, fmax), rng.randint(1, fmax), rng.randint(1, fmax)
        sa, sb, sc = np.sin(2 * np.pi * a * x), np.sin(2 * np.pi * b * x), np.sin(2 * np.pi * c * x)
        y += amp * sc[:, None, None] * sb[None, :, None] * sa[None, None, :]
    return y


def problem3(name, **over):
    """Named workloads on the unit cube (7-point stencil): n, layout
    (sx, sy, sz), overlap, phi, nu, mu, y_d and the eps schedule. Every box
    plane has at most 80 nodes."""
    base = dict(eps0=0.1, gamma=0.1, eps_min=1e-6, tol=1e-10, inner_tol=1e-8, sigma=1.1, kappa=0.1)
    if name == "c15":            # 15^3 grid, 3x3x3 boxes, overlap 1
        cfg = dict(n=15, sx=3, sy=3, sz=3, overlap=1, phi=PHI_CUBIC, nu=1e-4, mu=1e-3, yd=("sine3",))
    elif name == "c23":          # 23^3 grid, 4x4x4 boxes, overlap 1, Fourier data
        cfg = dict(n=23, sx=4, sy=4, sz=4, overlap=1, phi=PHI_CUBIC, nu=1e-5, mu=1e-3, yd=("fourier3", 3))
    elif name == "c63":          # 63^3 grid, 11x11x8 boxes of about 6 x 6 x 8 nodes, overlap 1
        cfg = dict(n=63, sx=11, sy=11, sz=8, overlap=1, phi=PHI_CUBIC, nu=1e-5, mu=1e-3, yd=("fourier3", 3))
    else:
        raise KeyError(name)
    base.update(cfg)
    base.update(over)
    return base


def make_yd3(cfg):
    kind = cfg["yd"]
    if kind[0] == "sine3":
        return yd_sine3(cfg["n"])
    if kind[0] == "fourier3":
        return yd_fourier3(cfg["n"], kind[1])
    raise KeyError(kind)


def uneven_batch(seed=4, count=64):
    """64 independent problems of uneven size: n ~ U{63,127,255,511},
    mu ~ logU[1e-4,1e-2], nu ~ logU[1e-6,1e-3], phi ~ U{y^3, exp}, block size
    b ~ U{32..64} (s = ceil(n/b)), overlap ~ U{2..8}, Fourier y_d with seed
    1000 + k."""
    rng = SplitMix64(seed)
    out = []
    for k in range(count):
        n = (63, 127, 255, 511)[rng.randint(0, 3)]
        mu = rng.log_uniform(1e-4, 1e-2)
        nu = rng.log_uniform(1e-6, 1e-3)
        phi = (PHI_CUBIC, PHI_EXP)[rng.randint(0, 1)]
        b = rng.randint(32, 64)
        overlap = rng.randint(2, 8)
        s = -(-n // b)
        out.append(dict(n=n, sx=s, sy=s, overlap=overlap, phi=phi, nu=nu, mu=mu,
                        yd=("fourier", 1000 + k), eps0=0.1, gamma=0.1, eps_min=1e-6,
                        tol=1e-10, inner_tol=1e-8, sigma=1.1, kappa=0.1))
    return out


def arrival_stream(seed=5, rate=200.0, count=2000, sizes=(127, 255, 511, 1023)):
    """Poisson arrivals (exponential gaps) of problems shaped like the uneven
    batch, with n drawn from `sizes`. Returns a list of (t_arrival_s, cfg)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        n = sizes[rng.randint(0, len(sizes) - 1)]
        mu = rng.log_uniform(1e-4, 1e-2)
        nu = rng.log_uniform(1e-6, 1e-3)
        phi = (PHI_CUBIC, PHI_EXP)[rng.randint(0, 1)]
        b = rng.randint(32, 64)
        overlap = rng.randint(2, 8)
        s = -(-n // b)
        out.append((t, dict(n=n, sx=s, sy=s, overlap=overlap, phi=phi, nu=nu, mu=mu,
                            yd=("fourier", 5000 + k), eps0=0.1, gamma=0.1, eps_min=1e-6,
                            tol=1e-10, inner_tol=1e-8, sigma=1.1, kappa=0.1)))
    return out
