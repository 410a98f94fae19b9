"""The unit cube (Assumption 1, n = 3: the 7-point stencil) on the GPU against
the oracle's cube model (oracle/three_d.py), through ras_create3: the residual,
the RASPEN function with its local iteration counts per box, its Jacobian
action (Alg. 4), the linear RAS preconditioner, and full RASPEN solves in FP64
and mixed precision with equal outer, local and Krylov counts. Same bars as
the square's parity tests: 1e-10 (FP64) and 1e-8 (mixed) relative inf-norm
per field, 1e-3 for FP32 solves without refinement."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import ras as oras
from oracle import three_d as t3
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, rel_inf, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)]
INEXACT_TOL = 1e-3


def zeros3(n):
    return torch.zeros((n, n, n), dtype=torch.float64, device="cuda")


def oracle_problem3(cfg, yd=None, f=None):
    yd = inputs.make_yd3(cfg) if yd is None else yd
    return t3.Problem(cfg["n"], cfg["phi"], cfg["nu"], cfg["mu"], yd, f, kappa=cfg["kappa"])


def oracle_opts3(cfg):
    return oras.Options(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"], eps0=cfg["eps0"],
                        gamma=cfg["gamma"], eps_min=cfg["eps_min"])


def gpu_problem3(cfg, prec, yd=None, f=None, **over):
    yd = inputs.make_yd3(cfg) if yd is None else yd
    kw = dict(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"], eps0=cfg["eps0"],
              gamma=cfg["gamma"], eps_min=cfg["eps_min"], precision=prec, kappa=cfg["kappa"])
    kw.update(over)
    return ras.ras_create3(cfg["n"], cfg["sx"], cfg["sy"], cfg["sz"], cfg["overlap"], cfg["phi"], cfg["nu"],
                           cfg["mu"], to_dev(yd), None if f is None else to_dev(f), ras.make_opts(**kw))


def _state(n, seed, ys=0.3, ps=1e-3):
    rng = np.random.default_rng(seed)
    return ys * rng.standard_normal((n, n, n)), ps * rng.standard_normal((n, n, n))


@pytest.mark.parametrize("phi", [0, 1, 2])
def test_cube_residual(phi):
    n = 13
    cfg = inputs.problem3("c15", n=n, phi=phi, sx=2, sy=2, sz=2)
    rng = np.random.default_rng(40 + phi)
    f = 0.5 * rng.standard_normal((n, n, n))
    prob = oracle_problem3(cfg, f=f)
    h = gpu_problem3(cfg, ras.RAS_FP64, f=f)
    try:
        assert ras.ras_problem_dim(h) == 3
        Y, P = _state(n, 12)
        for eps in (1e-1, 1e-6):
            Fy, Fp = zeros3(n), zeros3(n)
            nrm = ras.ras_residual(h, to_dev(Y), to_dev(P), eps, Fy, Fp)
            oy, op = t3.residual(prob, Y, P, eps)
            scale = prob.beta * max(np.abs(Y).max(), np.abs(P).max())
            assert np.max(np.abs(Fy.cpu().numpy() - oy)) <= 1e-13 * scale + 1e-12 * np.abs(oy).max()
            assert np.max(np.abs(Fp.cpu().numpy() - op)) <= 1e-13 * scale + 1e-12 * np.abs(op).max()
            ref = np.sqrt(np.sum(oy ** 2) + np.sum(op ** 2))
            assert abs(nrm - ref) <= 1e-12 * ref
    finally:
        ras.ras_destroy(h)


@pytest.fixture(scope="module")
def c15_oracle():
    cfg = inputs.problem3("c15")
    prob = oracle_problem3(cfg)
    subs = t3.subdomains(cfg["n"], cfg["sx"], cfg["sy"], cfg["sz"], cfg["overlap"])
    opts = oracle_opts3(cfg)
    Y, P = _state(cfg["n"], 5)
    out = {"cfg": cfg, "prob": prob, "subs": subs, "opts": opts, "Y": Y, "P": P}
    out["zero"] = t3.ras_apply(prob, np.zeros_like(Y), np.zeros_like(P), subs, opts, continuation=True)
    out["rand"] = t3.ras_apply(prob, Y, P, subs, opts, continuation=False)
    return out


@pytest.mark.parametrize("prec,tol", PRECS)
def test_cube_ras_apply(c15_oracle, prec, tol):
    o = c15_oracle
    n = o["cfg"]["n"]
    h = gpu_problem3(o["cfg"], prec)
    try:
        assert ras.ras_subdomain_count(h) == len(o["subs"])
        for key, Y, P, cont in (("zero", np.zeros((n, n, n)), np.zeros((n, n, n)), 1),
                                ("rand", o["Y"], o["P"], 0)):
            Fy, Fp = zeros3(n), zeros3(n)
            ras.ras_apply(h, to_dev(Y), to_dev(P), cont, Fy, Fp)
            ref = o[key]
            assert rel_inf(Fy.cpu().numpy(), ref.Fy) <= tol, key
            assert rel_inf(Fp.cpu().numpy(), ref.Fp) <= tol, key
            assert ras.ras_local_iterations(h) == ref.iterations, key
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_cube_jvp(c15_oracle, prec, tol):
    o = c15_oracle
    n = o["cfg"]["n"]
    h = gpu_problem3(o["cfg"], prec)
    try:
        Fy, Fp = zeros3(n), zeros3(n)
        ras.ras_apply(h, to_dev(o["Y"]), to_dev(o["P"]), 0, Fy, Fp)
        rng = np.random.default_rng(19)
        dY, dP = rng.standard_normal((n, n, n)), 1e-3 * rng.standard_normal((n, n, n))
        oy, op = zeros3(n), zeros3(n)
        ras.ras_jvp(h, to_dev(dY), to_dev(dP), oy, op)
        ry, rp = t3.jvp(o["prob"], o["rand"], dY, dP)
        assert rel_inf(oy.cpu().numpy(), ry) <= tol
        assert rel_inf(op.cpu().numpy(), rp) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, INEXACT_TOL)])
def test_cube_linear_ras(c15_oracle, prec, tol):
    """Z = sum_i tilde P_i J_i^-1 R_i R (the linear RAS preconditioner), J_i the
    box Jacobians at (Y, P, eps), each applied by the oracle's sparse LU."""
    o = c15_oracle
    n, prob, eps = o["cfg"]["n"], o["prob"], 1e-3
    rng = np.random.default_rng(23)
    Ry, Rp = rng.standard_normal((n, n, n)), rng.standard_normal((n, n, n))
    zy_ref, zp_ref = np.zeros((n, n, n)), np.zeros((n, n, n))
    for sub in o["subs"]:
        J = t3.jacobian_matrix(prob, o["Y"], o["P"], eps, sub.box)
        x0, x1, y0, y1, z0, z1 = sub.box
        z = spla.splu(J).solve(t3.interleave(Ry[z0:z1, y0:y1, x0:x1], Rp[z0:z1, y0:y1, x0:x1]))
        cy, cp = t3.deinterleave(z, sub.shape)
        zy_ref += t3.prolong_restricted(cy, sub, n)
        zp_ref += t3.prolong_restricted(cp, sub, n)
    h = gpu_problem3(o["cfg"], prec)
    try:
        zy, zp = zeros3(n), zeros3(n)
        ras.ras_precondition(h, to_dev(o["Y"]), to_dev(o["P"]), eps, to_dev(Ry), to_dev(Rp), zy, zp)
        assert rel_inf(zy.cpu().numpy(), zy_ref) <= tol
        assert rel_inf(zp.cpu().numpy(), zp_ref) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.fixture(scope="module", params=["c15", "c23"])
def cube_solve(request):
    cfg = inputs.problem3(request.param)
    prob = oracle_problem3(cfg)
    return cfg, t3.raspen(prob, cfg["sx"], cfg["sy"], cfg["sz"], cfg["overlap"], oracle_opts3(cfg))


@pytest.mark.parametrize("prec,tol", PRECS)
def test_cube_raspen_solve(cube_solve, prec, tol):
    cfg, ref = cube_solve
    n = cfg["n"]
    h = gpu_problem3(cfg, prec)
    try:
        y, p = zeros3(n), zeros3(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
        assert st.gmres_its == sum(ref.gmres_its)
    finally:
        ras.ras_destroy(h)


def test_cube_newton_ras_reaches_the_oracle_root(cube_solve):
    """Newton_RAS on the cube (no oracle of its own there) reaches the root
    of F_eps the oracle's RASPEN found, to the accuracy the two stop tests
    leave (relative residual 1e-10 on both sides)."""
    cfg, ref = cube_solve
    n = cfg["n"]
    h = gpu_problem3(cfg, ras.RAS_FP64)
    try:
        y, p = zeros3(n), zeros3(n)
        rc, st = ras.ras_newton_ras_solve(h, y, p)
        assert rc in (ras.RAS_OK, ras.RAS_OK_FLOOR)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= 1e-6
        assert rel_inf(p.cpu().numpy(), ref.P) <= 1e-6
        Fy, Fp = t3.residual(oracle_problem3(cfg), y.cpu().numpy(), p.cpu().numpy(), cfg["eps_min"])
        F0y, F0p = t3.residual(oracle_problem3(cfg), np.zeros((n, n, n)), np.zeros((n, n, n)), cfg["eps_min"])
        assert np.sqrt(np.sum(Fy ** 2) + np.sum(Fp ** 2)) <= 1e-9 * np.sqrt(np.sum(F0y ** 2) + np.sum(F0p ** 2))
    finally:
        ras.ras_destroy(h)


def test_cube_manufactured_root():
    """ras_manufacture on the cube: F(ybar, pbar) at rounding level under the
    oracle's 7-point residual with the y_d it returns."""
    cfg = inputs.problem3("c15", phi=2, nu=1e-6, mu=1.0)
    n = cfg["n"]
    x = inputs.coords(n)
    s = np.sin(2 * np.pi * 2 * x)
    pbar = 1.3 * s[:, None, None] * s[None, :, None] * s[None, None, :]
    h = gpu_problem3(cfg, ras.RAS_FP64, yd=np.zeros((n, n, n)))
    try:
        yb, yd = zeros3(n), zeros3(n)
        ras.ras_manufacture(h, to_dev(pbar), 1e-15, yb, yd)
        prob = oracle_problem3(cfg, yd=yd.cpu().numpy())
        Fy, Fp = t3.residual(prob, yb.cpu().numpy(), pbar, 1e-15)
        flr = t3.residual_floor_norm(prob, yb.cpu().numpy(), pbar, 1e-15)
        assert np.sqrt(np.sum(Fy ** 2) + np.sum(Fp ** 2)) <= 1e-12 * flr
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_cube_wide_planes(prec, tol):
    """Box planes of 9 x 9 nodes (162 unknowns): the wide-block path on the
    cube, a full RASPEN solve against the oracle."""
    cfg = inputs.problem3("c15", sx=2, sy=2, sz=3)
    ref = t3.raspen(oracle_problem3(cfg), cfg["sx"], cfg["sy"], cfg["sz"], cfg["overlap"], oracle_opts3(cfg))
    n = cfg["n"]
    h = gpu_problem3(cfg, prec)
    try:
        y, p = zeros3(n), zeros3(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its)
    finally:
        ras.ras_destroy(h)


def test_cube_refuses_planes_over_256_nodes():
    cfg = inputs.problem3("c15", n=17, sx=1, sy=1, sz=3)   # planes of 17 x 17 nodes
    with pytest.raises(ras.RasError):
        gpu_problem3(cfg, ras.RAS_FP64)
    cfg = inputs.problem3("c15", sz=0)
    with pytest.raises(ras.RasError):
        gpu_problem3(cfg, ras.RAS_FP64)
