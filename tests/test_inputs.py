"""The seeded input generators (paper_2411_00546_gb300/inputs.py) on CPU: the
published SplitMix64 stream, the grid layout of the square's and the cube's
desired states (x1 fastest, node (i, j, k) at ((i+1)h, (j+1)h, (k+1)h)),
their determinism, and that the named cube workloads keep every box plane
within the register-tile limit of 80 nodes."""
import math

import numpy as np

from paper_2411_00546_gb300 import inputs


def test_splitmix64_matches_its_published_first_outputs():
    # SplitMix64 with seed 0: the first outputs of the reference generator
    # (Steele, Lea & Flood), as tabulated with the algorithm's description
    g = inputs.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_square_sine_layout():
    n = 7
    h = 1.0 / (n + 1)
    y = inputs.yd_sine(n)
    for j, i in ((0, 0), (2, 5), (6, 3)):
        assert y[j, i] == math.sin(2 * math.pi * (i + 1) * h) * math.sin(2 * math.pi * (j + 1) * h)


def test_cube_sine_layout():
    n = 6
    h = 1.0 / (n + 1)
    y = inputs.yd_sine3(n)
    assert y.shape == (n, n, n)
    for k, j, i in ((0, 0, 0), (1, 4, 2), (5, 3, 1)):
        ref = (math.sin(2 * math.pi * (i + 1) * h) * math.sin(2 * math.pi * (j + 1) * h)
               * math.sin(2 * math.pi * (k + 1) * h))
        assert abs(y[k, j, i] - ref) <= 1e-15


def test_cube_fourier_draws_and_layout():
    """yd_fourier3 against a node-by-node sum with the same draws (amplitude,
    then the x1, x2, x3 frequencies of each mode), and the same seed twice."""
    n, seed = 5, 7
    y = inputs.yd_fourier3(n, seed)
    np.testing.assert_array_equal(y, inputs.yd_fourier3(n, seed))
    g = inputs.SplitMix64(seed)
    modes = []
    for _ in range(8):
        amp = 2.0 * g.uniform() - 1.0
        modes.append((amp, g.randint(1, 4), g.randint(1, 4), g.randint(1, 4)))
    h = 1.0 / (n + 1)
    for k, j, i in ((0, 0, 0), (4, 1, 3), (2, 2, 2)):
        ref = sum(amp * math.sin(2 * math.pi * a * (i + 1) * h) * math.sin(2 * math.pi * b * (j + 1) * h)
                  * math.sin(2 * math.pi * c * (k + 1) * h) for amp, a, b, c in modes)
        assert abs(y[k, j, i] - ref) <= 1e-13


def _blocks(n, s):
    base, extra = divmod(n, s)
    out, x = [], 0
    for k in range(s):
        w = base + (1 if k < extra else 0)
        out.append((x, x + w))
        x += w
    return out


def test_named_cube_workloads_fit_the_register_tiles():
    for name in ("c15", "c23", "c63"):
        cfg = inputs.problem3(name)
        n, ov = cfg["n"], cfg["overlap"]
        widest = 0
        for a0, a1 in _blocks(n, cfg["sx"]):
            for b0, b1 in _blocks(n, cfg["sy"]):
                wx = min(n, a1 + ov) - max(0, a0 - ov)
                wy = min(n, b1 + ov) - max(0, b0 - ov)
                widest = max(widest, wx * wy)
        assert widest <= 80, (name, widest)
