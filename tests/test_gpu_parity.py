"""GPU-vs-oracle parity through the C ABI (libras.so), on identical seeded inputs.

Bar: relative infinity-norm error per field <= 1e-10 in FP64 mode and <= 1e-8
in mixed mode for every result the method defines exactly (residual, RASPEN
function, its Jacobian action, solves), equal local Newton iteration counts per
subdomain, and for the mixed-precision operators run without FP64 refinement
(FP32 local solves: the linear RAS preconditioner, and the Jacobian action with
jvp_ir = 0) the bound cond(J_i) * 2^-24 with cond(J_i) <= 1e4, i.e. 1e-3.
"""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import discretization as fd
from oracle import ras as oras
from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import (FP64_TOL, MIXED_TOL, gpu_problem, oracle_opts, oracle_problem, rel_inf, to_dev,
                      zeros)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)]
INEXACT_TOL = 1e-3


def _cfg(name="n63", **over):
    return inputs.problem(name, **over)


def _state(n, seed, ys=0.3, ps=1e-3):
    rng = np.random.default_rng(seed)
    return ys * rng.standard_normal((n, n)), ps * rng.standard_normal((n, n))


@pytest.mark.parametrize("n", [63, 100])
@pytest.mark.parametrize("phi", [0, 1, 2])
def test_residual(n, phi):
    cfg = _cfg(n=n, phi=phi, sx=3, sy=3)
    rng = np.random.default_rng(n + phi)
    f = 0.5 * rng.standard_normal((n, n))
    prob = oracle_problem(cfg, f=f)
    h = gpu_problem(cfg, ras.RAS_FP64, f=f)
    try:
        Y, P = _state(n, 11)
        for eps in (1e-1, 1e-6):
            Fy, Fp = zeros(n), zeros(n)
            nrm = ras.ras_residual(h, to_dev(Y), to_dev(P), eps, Fy, Fp)
            oy, op = fd.residual(prob, Y, P, eps)
            scale = prob.beta * max(np.abs(Y).max(), np.abs(P).max())
            assert np.max(np.abs(Fy.cpu().numpy() - oy)) <= 1e-13 * scale + 1e-12 * np.abs(oy).max()
            assert np.max(np.abs(Fp.cpu().numpy() - op)) <= 1e-13 * scale + 1e-12 * np.abs(op).max()
            ref = np.sqrt(np.sum(oy ** 2) + np.sum(op ** 2))
            assert abs(nrm - ref) <= 1e-12 * ref
    finally:
        ras.ras_destroy(h)


@pytest.fixture(scope="module")
def n63_oracle():
    cfg = _cfg()
    prob = oracle_problem(cfg)
    subs = dd.subdomains(cfg["n"], cfg["sx"], cfg["sy"], cfg["overlap"])
    opts = oracle_opts(cfg)
    Y, P = _state(cfg["n"], 3)
    out = {"cfg": cfg, "prob": prob, "subs": subs, "opts": opts, "Y": Y, "P": P}
    out["zero"] = oras.ras_apply(prob, np.zeros_like(Y), np.zeros_like(P), subs, opts, continuation=True)
    out["rand"] = oras.ras_apply(prob, Y, P, subs, opts, continuation=False)
    return out


@pytest.mark.parametrize("prec,tol", PRECS)
def test_ras_apply_parity(n63_oracle, prec, tol):
    o = n63_oracle
    n = o["cfg"]["n"]
    h = gpu_problem(o["cfg"], prec)
    try:
        for key, Y, P, cont in (("zero", np.zeros((n, n)), np.zeros((n, n)), 1),
                                ("rand", o["Y"], o["P"], 0)):
            Fy, Fp = zeros(n), zeros(n)
            rc, st = ras.ras_apply(h, to_dev(Y), to_dev(P), cont, Fy, Fp)
            ref = o[key]
            assert rel_inf(Fy.cpu().numpy(), ref.Fy) <= tol, key
            assert rel_inf(Fp.cpu().numpy(), ref.Fp) <= tol, key
            assert ras.ras_local_iterations(h) == ref.iterations, key
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol,jvp_ir", [(ras.RAS_FP64, FP64_TOL, 1), (ras.RAS_MIXED, MIXED_TOL, 1),
                                             (ras.RAS_MIXED, INEXACT_TOL, 0)])
def test_jvp_parity(n63_oracle, prec, tol, jvp_ir):
    o = n63_oracle
    n = o["cfg"]["n"]
    h = gpu_problem(o["cfg"], prec, jvp_ir=jvp_ir)
    try:
        Fy, Fp = zeros(n), zeros(n)
        ras.ras_apply(h, to_dev(o["Y"]), to_dev(o["P"]), 0, Fy, Fp)
        rng = np.random.default_rng(9)
        dY, dP = rng.standard_normal((n, n)), 1e-3 * rng.standard_normal((n, n))
        oy, op = zeros(n), zeros(n)
        ras.ras_jvp(h, to_dev(dY), to_dev(dP), oy, op)
        ry, rp = oras.jvp(o["prob"], o["rand"], dY, dP)
        assert rel_inf(oy.cpu().numpy(), ry) <= tol
        assert rel_inf(op.cpu().numpy(), rp) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, INEXACT_TOL)])
def test_linear_ras_parity(n63_oracle, prec, tol):
    o = n63_oracle
    n = o["cfg"]["n"]
    eps = 1e-3
    h = gpu_problem(o["cfg"], prec)
    try:
        rng = np.random.default_rng(4)
        rY, rP = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        zy, zp = zeros(n), zeros(n)
        ras.ras_precondition(h, to_dev(o["Y"]), to_dev(o["P"]), eps, to_dev(rY), to_dev(rP), zy, zp)
        ref = oras.LinearRas(o["prob"], o["Y"], o["P"], o["subs"], eps).apply(rY, rP)
        assert rel_inf(zy.cpu().numpy(), ref[0]) <= tol
        assert rel_inf(zp.cpu().numpy(), ref[1]) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.fixture(scope="module")
def n63_solves():
    cfg = _cfg()
    prob = oracle_problem(cfg)
    opts = oracle_opts(cfg)
    r = solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], opts)
    q = solvers.newton_ras(prob, cfg["sx"], cfg["sy"], cfg["overlap"], opts)
    return cfg, r, q


@pytest.mark.parametrize("prec,tol", PRECS)
def test_raspen_solve_parity(n63_solves, prec, tol):
    cfg, ref, _ = n63_solves
    n = cfg["n"]
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
        assert st.inner_its_max == sum(max(i) for i in ref.inner_its)
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_newton_ras_solve_parity(n63_solves, prec, tol):
    cfg, _, ref = n63_solves
    n = cfg["n"]
    h = gpu_problem(cfg, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_newton_ras_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
    finally:
        ras.ras_destroy(h)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("n,sx,sy,ov,phi", [
    (20, 1, 1, 0, 0),      # single subdomain = whole grid
    (37, 3, 2, 0, 1),      # no overlap, non-square layout, ragged blocks, exp
    (50, 4, 3, 3, 2),      # kappa nonlinearity, ragged, wide overlap
    (9, 9, 9, 1, 0),       # one-node blocks
])
def test_ras_apply_layouts(n, sx, sy, ov, phi):
    cfg = _cfg(n=n, sx=sx, sy=sy, overlap=ov, phi=phi, nu=1e-3, mu=2e-2)
    rng = np.random.default_rng(n)
    yd = 5.0 * inputs.yd_fourier(n, 7)
    f = 0.3 * rng.standard_normal((n, n))
    prob = oracle_problem(cfg, yd=yd, f=f)
    subs = dd.subdomains(n, sx, sy, ov)
    ref = oras.ras_apply(prob, np.zeros((n, n)), np.zeros((n, n)), subs, oracle_opts(cfg), True)
    for prec, tol in PRECS:
        h = gpu_problem(cfg, prec, yd=yd, f=f)
        try:
            Fy, Fp = zeros(n), zeros(n)
            ras.ras_apply(h, zeros(n), zeros(n), 1, Fy, Fp)
            assert rel_inf(Fy.cpu().numpy(), ref.Fy) <= tol
            assert rel_inf(Fp.cpu().numpy(), ref.Fp) <= tol
            assert ras.ras_local_iterations(h) == ref.iterations
        finally:
            ras.ras_destroy(h)


def test_root_gives_zero_corrections():
    """At a root of F the RASPEN function vanishes with no local iterations."""
    cfg = _cfg(n=30, sx=3, sy=3, overlap=2, eps0=1e-4, eps_min=1e-4)
    prob = oracle_problem(cfg)
    root = solvers.newton_sparse(prob, oracle_opts(cfg, tol=1e-14))
    h = gpu_problem(cfg, ras.RAS_FP64)
    try:
        Fy, Fp = zeros(30), zeros(30)
        ras.ras_apply(h, to_dev(root.Y), to_dev(root.P), 0, Fy, Fp)
        assert ras.ras_local_iterations(h) == [0] * 9
        assert float(Fy.abs().max()) == 0.0 and float(Fp.abs().max()) == 0.0
    finally:
        ras.ras_destroy(h)


def test_invalid_arguments():
    n = 40
    yd = to_dev(inputs.yd_sine(n))
    with pytest.raises(ras.RasError):
        ras.ras_create(n, n + 1, 2, 1, 0, 1e-4, 1e-3, yd)          # sx > n
    with pytest.raises(ras.RasError):
        ras.ras_create(n, 2, 2, 1, 0, -1.0, 1e-3, yd)              # nu <= 0
    with pytest.raises(ras.RasError):
        ras.ras_create(300, 1, 1, 0, 0, 1e-4, 1e-3, to_dev(inputs.yd_sine(300)))  # 2*wx > 512
    with pytest.raises(ras.RasError):
        ras.ras_create(n, 2, 2, 1, 7, 1e-4, 1e-3, yd)              # unknown phi
    h = ras.ras_create(n, 2, 2, 1, 0, 1e-4, 1e-3, yd)
    try:
        with pytest.raises(ras.RasError) as e:
            ras.ras_jvp(h, zeros(n), zeros(n), zeros(n), zeros(n))
        assert e.value.code == ras.RAS_ESTATE
        with pytest.raises(ras.RasError):
            ras.ras_set_eps(h, 0.0)
    finally:
        ras.ras_destroy(h)


def test_nonfinite_input_is_reported():
    n = 30
    cfg = _cfg(n=n, sx=2, sy=2, overlap=1)
    yd = inputs.yd_sine(n)
    yd[5, 7] = np.nan
    h = gpu_problem(cfg, ras.RAS_FP64, yd=yd)
    try:
        Fy, Fp = zeros(n), zeros(n)
        rc, st = ras.ras_apply(h, zeros(n), zeros(n), 1, Fy, Fp, check=False)
        assert rc == ras.RAS_ENONFINITE
        assert st.local_failures >= 1
    finally:
        ras.ras_destroy(h)


def test_host_entry_point_matches_device_solve(n63_solves):
    cfg, ref, _ = n63_solves
    n = cfg["n"]
    h = gpu_problem(cfg, ras.RAS_FP64)
    try:
        yh = torch.zeros((n, n), dtype=torch.float64).pin_memory()
        ph = torch.zeros((n, n), dtype=torch.float64).pin_memory()
        ydh = torch.tensor(inputs.make_yd(cfg)).pin_memory()
        ras.ras_solve_host(h, ras.RAS_METHOD_RASPEN, ydh, yh, ph)
        assert rel_inf(yh.numpy(), ref.Y) <= FP64_TOL
        assert rel_inf(ph.numpy(), ref.P) <= FP64_TOL
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("n,s,nu", [(20, 2, 1e-9), (31, 3, 1e-10)])
def test_pivoting_cases(n, s, nu):
    """nu tiny: the (y, p) coupling (1/nu)(1 - P_eps') of the local Jacobian
    dwarfs its diagonal 4/h^2 + phi', so partial pivoting must interchange
    rows (the register factorisation's fallback path and the FP64 kernel's
    pivoting). Same bar as the other parity tests."""
    cfg = _cfg(n=n, sx=s, sy=s, overlap=2, nu=nu, mu=1e-3, eps0=1e-1, eps_min=1e-3)
    yd = 3.0 * inputs.yd_fourier(n, 11)
    prob = oracle_problem(cfg, yd=yd)
    subs = dd.subdomains(n, s, s, 2)
    ref = oras.ras_apply(prob, np.zeros((n, n)), np.zeros((n, n)), subs, oracle_opts(cfg), True)
    # the oracle's band LU does interchange rows here
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
