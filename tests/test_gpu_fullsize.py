"""Parity at the benchmark's sizes (n = 255 and the n = 1023 bench workload),
through the C ABI, in the launch configuration bench.py times.

* n = 255 (8 x 8 subdomains): full RASPEN solves against the oracle's.
* n = 1023 (16 x 16 subdomains of 64^2, overlap 8), inactive (mu = 1e-2) and
  active (mu = 1e-3) L1 control: full RASPEN_eps solves in FP64 and in mixed
  precision against the oracle's own solve of the same seeded problem, stored
  in tests/golden/raspen_<name>.npz by tests/golden/make_raspen_golden.py
  (which calls only the oracle): every element of y and of p on its own
  scale, the outer and Krylov counts, and the local Newton counts of every
  subdomain in every evaluation of the RASPEN function.
* n = 1023 first evaluation: sampled subdomains against a live oracle run.
"""
import os

import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import discretization as fd
from oracle import ras as oras
from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_opts, gpu_problem, oracle_opts, oracle_problem, rel_inf, zeros

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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "raspen_%s.npz")


@pytest.fixture(scope="module", params=["n1023", "n1023_active"])
def stored_oracle_solve(request):
    g = np.load(GOLDEN % request.param)
    return request.param, {k: g[k] for k in g.files}


@pytest.mark.parametrize("prec,tol", PRECS)
def test_n1023_solve_matches_the_stored_oracle_solve(stored_oracle_solve, prec, tol):
    name, g = stored_oracle_solve
    cfg = inputs.problem(name)
    n = cfg["n"]
    outer = int(g["outer"])
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert int(g["status"]) == 0 and st.status == ras.RAS_OK
        ey = rel_inf(y.cpu().numpy(), g["Y"])
        ep = rel_inf(p.cpu().numpy(), g["P"])
        assert ey <= tol and ep <= tol, (ey, ep)
        assert st.outer_its == outer
        assert st.gmres_its == int(g["gmres_its"].sum())
        assert st.evaluations == g["inner_its"].shape[0] == outer + 1
        assert st.inner_its_sum == int(g["inner_its"].sum())
        assert ras.ras_local_iterations(h) == [int(v) for v in g["inner_its"][outer]]
        # the local counts of every earlier evaluation: the same solve stopped
        # after k outer iterations ends on evaluation k
        for k in range(outer):
            ras.ras_set_opts(h, gpu_opts(cfg, prec, kmax_outer_raspen=k))
            y.zero_()
            p.zero_()
            rc, st = ras.ras_raspen_solve(h, y, p, check=False)
            assert st.evaluations == k + 1
            assert ras.ras_local_iterations(h) == [int(v) for v in g["inner_its"][k]], (name, k)
    finally:
        ras.ras_destroy(h)


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
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
    finally:
        ras.ras_destroy(h)
