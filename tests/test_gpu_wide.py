"""Wide local blocks (160 < 2 wx <= 512 unknowns per block row: the paper's
2 x s and small s x s layouts) against the oracle: the RASPEN function with
per-subdomain local counts, its Jacobian action, the linear RAS
preconditioner, full RASPEN and Newton_RAS solves in FP64 and mixed precision
with equal outer and local counts, a case that needs row interchanges, a
batch mixing wide and narrow blocks, and the upper limit. Same bars as the
other parity tests."""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import ras as oras
from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import (FP64_TOL, MIXED_TOL, gpu_opts, gpu_problem, oracle_opts, oracle_problem, rel_inf,
                      to_dev, zeros)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)]
INEXACT_TOL = 1e-3
LAYOUTS = {"n100-1x2": dict(n=100, sx=1, sy=2, overlap=2),     # blocks of 100 x 52: 200 unknowns per row
           "n170-2x2": dict(n=170, sx=2, sy=2, overlap=2)}     # blocks of 87 x 87: 174 unknowns per row


def _cfg(name, **over):
    kw = dict(LAYOUTS[name])
    kw.update(over)
    return inputs.problem("n63", **kw)


def _state(n, seed, ys=0.3, ps=1e-3):
    rng = np.random.default_rng(seed)
    return ys * rng.standard_normal((n, n)), ps * rng.standard_normal((n, n))


@pytest.fixture(scope="module")
def wide_oracle():
    cfg = _cfg("n170-2x2")
    prob = oracle_problem(cfg)
    subs = dd.subdomains(cfg["n"], cfg["sx"], cfg["sy"], cfg["overlap"])
    opts = oracle_opts(cfg)
    Y, P = _state(cfg["n"], 8)
    out = {"cfg": cfg, "prob": prob, "subs": subs, "opts": opts, "Y": Y, "P": P}
    out["zero"] = oras.ras_apply(prob, np.zeros_like(Y), np.zeros_like(P), subs, opts, continuation=True)
    out["rand"] = oras.ras_apply(prob, Y, P, subs, opts, continuation=False)
    return out


@pytest.mark.parametrize("prec,tol", PRECS)
def test_wide_ras_apply(wide_oracle, prec, tol):
    o = wide_oracle
    n = o["cfg"]["n"]
    h = gpu_problem(o["cfg"], prec)
    try:
        for key, Y, P, cont in (("zero", np.zeros((n, n)), np.zeros((n, n)), 1), ("rand", o["Y"], o["P"], 0)):
            Fy, Fp = zeros(n), zeros(n)
            ras.ras_apply(h, to_dev(Y), to_dev(P), cont, Fy, Fp)
            ref = o[key]
            assert rel_inf(Fy.cpu().numpy(), ref.Fy) <= tol, key
            assert rel_inf(Fp.cpu().numpy(), ref.Fp) <= tol, key
            assert ras.ras_local_iterations(h) == ref.iterations, key
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_wide_jvp(wide_oracle, prec, tol):
    o = wide_oracle
    n = o["cfg"]["n"]
    h = gpu_problem(o["cfg"], prec)
    try:
        Fy, Fp = zeros(n), zeros(n)
        ras.ras_apply(h, to_dev(o["Y"]), to_dev(o["P"]), 0, Fy, Fp)
        rng = np.random.default_rng(29)
        dY, dP = rng.standard_normal((n, n)), 1e-3 * rng.standard_normal((n, n))
        oy, op = zeros(n), zeros(n)
        ras.ras_jvp(h, to_dev(dY), to_dev(dP), oy, op)
        ry, rp = oras.jvp(o["prob"], o["rand"], dY, dP)
        assert rel_inf(oy.cpu().numpy(), ry) <= tol
        assert rel_inf(op.cpu().numpy(), rp) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, INEXACT_TOL)])
def test_wide_linear_ras(wide_oracle, prec, tol):
    o = wide_oracle
    n, eps = o["cfg"]["n"], 1e-3
    h = gpu_problem(o["cfg"], prec)
    try:
        rng = np.random.default_rng(31)
        rY, rP = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        zy, zp = zeros(n), zeros(n)
        ras.ras_precondition(h, to_dev(o["Y"]), to_dev(o["P"]), eps, to_dev(rY), to_dev(rP), zy, zp)
        ref = oras.LinearRas(o["prob"], o["Y"], o["P"], o["subs"], eps).apply(rY, rP)
        assert rel_inf(zy.cpu().numpy(), ref[0]) <= tol
        assert rel_inf(zp.cpu().numpy(), ref[1]) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.fixture(scope="module", params=sorted(LAYOUTS))
def wide_solve(request):
    cfg = _cfg(request.param)
    prob = oracle_problem(cfg)
    return cfg, solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], oracle_opts(cfg))


@pytest.mark.parametrize("prec,tol", PRECS)
def test_wide_raspen_solve(wide_solve, prec, tol):
    cfg, ref = wide_solve
    n = cfg["n"]
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
        # Krylov counts within 15 %: on n170-2x2 the GMRES residuals flatten out
        # near the tolerance, so rounding moves the step that crosses it (the
        # oracle itself takes 9 steps in its last solve on one host's BLAS and
        # 10 on another's, and the mixed-precision solve up to 3 more in all)
        k = sum(ref.gmres_its)
        assert abs(st.gmres_its - k) <= max(2, int(0.15 * k))
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_wide_newton_ras_solve(prec, tol):
    cfg = _cfg("n100-1x2")
    n = cfg["n"]
    ref = solvers.newton_ras(oracle_problem(cfg), cfg["sx"], cfg["sy"], cfg["overlap"], oracle_opts(cfg))
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_newton_ras_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
    finally:
        ras.ras_destroy(h)


def test_wide_pivoting_fallback():
    """nu tiny on one 90 x 90 subdomain (180 unknowns per block row): the
    coupling (1/nu)(1 - P_eps') dwarfs the diagonal, so partial pivoting must
    interchange rows (the oracle's band LU does, and so does the wide-block
    kernel's blocked sweep)."""
    n, nu = 90, 1e-9
    cfg = inputs.problem("n63", n=n, sx=1, sy=1, overlap=0, nu=nu, mu=1e-3, eps0=1e-1, eps_min=1e-3)
    yd = 3.0 * inputs.yd_fourier(n, 11)
    prob = oracle_problem(cfg, yd=yd)
    subs = dd.subdomains(n, 1, 1, 0)
    ref = oras.ras_apply(prob, np.zeros((n, n)), np.zeros((n, n)), subs, oracle_opts(cfg), True)
    J = oras.local_jacobian_factor(prob, np.zeros((n, n)), 1e-4 * np.ones((n, n)), 1e-3, subs[0])
    assert np.any(J.piv != np.arange(1, J.piv.size + 1))
    for prec, tol in PRECS:
        h = gpu_problem(cfg, prec, yd=yd)
        try:
            Fy, Fp = zeros(n), zeros(n)
            ras.ras_apply(h, zeros(n), zeros(n), 1, Fy, Fp)
            assert rel_inf(Fy.cpu().numpy(), ref.Fy) <= tol
            assert rel_inf(Fp.cpu().numpy(), ref.Fp) <= tol
            assert ras.ras_local_iterations(h) == ref.iterations
        finally:
            ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_batch_mixing_wide_and_narrow_blocks(prec, tol):
    cfgs = [inputs.problem("n63"), _cfg("n100-1x2")]
    refs = [solvers.raspen(oracle_problem(c), c["sx"], c["sy"], c["overlap"], oracle_opts(c)) for c in cfgs]
    probs = [dict(n=c["n"], sx=c["sx"], sy=c["sy"], overlap=c["overlap"], phi=c["phi"], nu=c["nu"], mu=c["mu"],
                  y_d=to_dev(inputs.make_yd(c))) for c in cfgs]
    h = ras.ras_batch_create(probs, gpu_opts(cfgs[0], prec))
    try:
        ys = [zeros(c["n"]) for c in cfgs]
        ps = [zeros(c["n"]) for c in cfgs]
        rc, stats = ras.ras_batch_raspen_solve(h, ys, ps)
        for c, ref, st, y, p in zip(cfgs, refs, stats, ys, ps):
            assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
            assert rel_inf(p.cpu().numpy(), ref.P) <= tol
            assert st.outer_its == ref.outer
            assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
    finally:
        ras.ras_destroy(h)


def test_blocks_over_512_unknowns_are_refused():
    cfg = inputs.problem("n63", n=300, sx=1, sy=2, overlap=2)    # rows of 300 nodes
    with pytest.raises(ras.RasError):
        gpu_problem(cfg, ras.RAS_FP64)
