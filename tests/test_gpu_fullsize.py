"""Parity at the benchmark's sizes (n = 255 and the n = 1023 bench workload),
through the C ABI, in the launch configuration bench.py times.

* n = 255 (8 x 8 subdomains): full RASPEN solves against the oracle's.
* n = 1023 (16 x 16 subdomains of 64^2, overlap 8): the oracle cannot run the
  whole solve in a test, but every local correction C_i(x) of the RASPEN
  function is an independent local Newton solve (Alg. 3). The GPU's first
  evaluation F(x0) (with continuation) is checked against the oracle's
  corrections on sampled subdomains (corner, edges, interior): same values on
  the owned nodes and the same local iteration counts. The full solves are
  checked by properties that hold at any size: the oracle's residual F at the
  GPU solution is at the solver's tolerance, and the mixed-precision solution
  matches the FP64 one.
"""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import discretization as fd
from oracle import ras as oras
from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_problem, oracle_opts, oracle_problem, rel_inf, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)]


@pytest.fixture(scope="module")
def n255_solve():
    cfg = inputs.problem("n255")
    prob = oracle_problem(cfg)
    return cfg, solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], oracle_opts(cfg))


@pytest.mark.parametrize("prec,tol", PRECS)
def test_n255_raspen_solve(n255_solve, prec, tol):
    cfg, ref = n255_solve
    n = cfg["n"]
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
    finally:
        ras.ras_destroy(h)


def _sample(subs, sx, sy):
    """Corner, two edges and two interior subdomains."""
    picks = [0, sx - 1, (sy - 1) * sx, sx // 2, (sy // 2) * sx + sx // 2, (sy // 2) * sx + 1]
    return [subs[k] for k in sorted(set(picks))]


@pytest.fixture(scope="module")
def n1023():
    cfg = inputs.problem("n1023")
    prob = oracle_problem(cfg)
    subs = dd.subdomains(cfg["n"], cfg["sx"], cfg["sy"], cfg["overlap"])
    return cfg, prob, subs


@pytest.mark.parametrize("prec,tol", PRECS)
def test_n1023_first_evaluation_sampled(n1023, prec, tol):
    cfg, prob, subs = n1023
    n = cfg["n"]
    opts = oracle_opts(cfg)
    h = gpu_problem(cfg, prec)
    try:
        Fy, Fp = zeros(n), zeros(n)
        ras.ras_apply(h, zeros(n), zeros(n), 1, Fy, Fp)
        its = ras.ras_local_iterations(h)
        Fy, Fp = Fy.cpu().numpy(), Fp.cpu().numpy()
    finally:
        ras.ras_destroy(h)
    Z = np.zeros((n, n))
    for sub in _sample(subs, cfg["sx"], cfg["sy"]):
        loc = oras.local_correction(prob, Z, Z, sub, opts.eps0, opts.eps_min, opts, factor_at_solution=False)
        cy, cp = fd.deinterleave(loc.C, sub.wx, sub.wy)
        ox0, ox1, oy0, oy1 = sub.owned
        x0, _, y0, _ = sub.box
        ry = cy[oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0]
        rp = cp[oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0]
        assert its[sub.index] == loc.newton.iterations, sub.index
        assert rel_inf(Fy[oy0:oy1, ox0:ox1], ry) <= tol, sub.index
        assert rel_inf(Fp[oy0:oy1, ox0:ox1], rp) <= tol, sub.index


@pytest.fixture(scope="module")
def n1023_solves(n1023):
    cfg, prob, subs = n1023
    n = cfg["n"]
    out = {}
    for prec in (ras.RAS_FP64, ras.RAS_MIXED):
        h = gpu_problem(cfg, prec)
        try:
            y, p = zeros(n), zeros(n)
            rc, st = ras.ras_raspen_solve(h, y, p)
            out[prec] = (y.cpu().numpy(), p.cpu().numpy(), st)
        finally:
            ras.ras_destroy(h)
    return out


def test_n1023_solution_properties(n1023, n1023_solves):
    """The oracle's F at the GPU solutions is at the solve's accuracy, and the
    mixed-precision solution equals the FP64 one within the mixed tolerance."""
    cfg, prob, subs = n1023
    F0 = np.sqrt(np.sum(prob.y_d ** 2))           # ||F(x0 = 0)|| (f = 0: only F_p = y_d)
    for prec, (Y, P, st) in n1023_solves.items():
        assert st.status == 0 and st.outer_its >= 1
        Fy, Fp = fd.residual(prob, Y, P, cfg["eps_min"])
        res = np.sqrt(np.sum(Fy ** 2) + np.sum(Fp ** 2))
        flr = fd.residual_floor_norm(prob, Y, P, cfg["eps_min"])
        # converged: at the requested relative tolerance or at FP64 rounding level
        assert res <= max(1e-8 * F0, 64 * 2.0 ** -53 * flr), (prec, res, F0, flr)
    Y64, P64, _ = n1023_solves[ras.RAS_FP64]
    Ym, Pm, _ = n1023_solves[ras.RAS_MIXED]
    assert rel_inf(Ym, Y64, P64) <= MIXED_TOL
    assert rel_inf(Pm, P64, Y64) <= MIXED_TOL


# The other members of the n = 255 family (phi in {exp, y^3}, mu in {1e-3,
# 5e-3}, Fourier seeds 1-3): one variant per changed factor, full RASPEN
# solves against the oracle in FP64 and mixed precision.
N255_VARIANTS = [(1, 1e-3, 2), (0, 5e-3, 3), (1, 5e-3, 1)]


@pytest.fixture(scope="module", params=N255_VARIANTS, ids=lambda v: "phi%d-mu%g-seed%d" % v)
def n255_variant(request):
    phi, mu, seed = request.param
    cfg = inputs.problem("n255", phi=phi, mu=mu, yd=("fourier", seed))
    prob = oracle_problem(cfg)
    return cfg, solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], oracle_opts(cfg))


@pytest.mark.parametrize("prec,tol", PRECS)
def test_n255_variant_raspen_solve(n255_variant, prec, tol):
    cfg, ref = n255_variant
    n = cfg["n"]
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y, ref.P) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P, ref.Y) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
    finally:
        ras.ras_destroy(h)
