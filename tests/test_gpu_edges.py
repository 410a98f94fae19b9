"""Edge cases of the CUDA path against the oracle: the smallest grid, data
whose root is x = 0, the widest local block of the register-tile and
streaming kernels (2 wx = 160; wider blocks take the wide-block path),
an inactive control (mu large: u = 0 everywhere), and empty batches."""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import ras as oras
from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_problem, oracle_opts, oracle_problem, rel_inf, to_dev, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)]


def _cfg(**kw):
    c = dict(inputs.problem("n63"))
    c.update(kw)
    return c


@pytest.mark.parametrize("prec,tol", PRECS)
@pytest.mark.parametrize("n,s,ov", [(2, 1, 0), (2, 2, 1), (3, 3, 1)])
def test_smallest_grids_reach_the_dense_newton_root(n, s, ov, prec, tol):
    c = _cfg(n=n, sx=s, sy=s, overlap=ov, nu=1e-3, mu=5e-2)
    yd = 40.0 * np.ones((n, n))
    prob = oracle_problem(c, yd=yd)
    ref = solvers.newton_dense(prob, oracle_opts(c, tol=1e-13))
    assert ref.status >= 0
    h = gpu_problem(c, prec, yd=yd)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rc in (ras.RAS_OK, ras.RAS_OK_FLOOR)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("solve", ["raspen", "newton_ras", "newton"])
def test_zero_data_root_is_zero(solve):
    """f = 0, y_d = 0: x = 0 solves the system for every eps. RASPEN stops at
    once (its first evaluation already holds the continuation); Alg. 1 applies
    its stop test only at eps_min, so Newton_RAS and Newton take the
    continuation steps with zero Newton steps, as the oracle does."""
    n = 31
    c = _cfg(n=n, sx=2, sy=2, overlap=2)
    zero = np.zeros((n, n))
    prob = oracle_problem(c, yd=zero)
    ref = {"raspen": lambda: solvers.raspen(prob, 2, 2, 2, oracle_opts(c)),
           "newton_ras": lambda: solvers.newton_ras(prob, 2, 2, 2, oracle_opts(c)),
           "newton": lambda: solvers.newton_gmres(prob, oracle_opts(c))}[solve]()
    assert ref.outer == (0 if solve == "raspen" else 5)
    h = gpu_problem(c, ras.RAS_MIXED, yd=zero)
    try:
        y, p = zeros(n), zeros(n)
        fn = {"raspen": ras.ras_raspen_solve, "newton_ras": ras.ras_newton_ras_solve,
              "newton": ras.ras_newton_solve}[solve]
        rc, st = fn(h, y, p)
        assert rc in (ras.RAS_OK, ras.RAS_OK_FLOOR)
        assert st.outer_its == ref.outer
        assert st.gmres_its == 0
        assert not y.any() and not p.any()
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_widest_block_matches_oracle(prec, tol):
    """One 80 x 80 subdomain: local block rows of 2 wx = 160 unknowns, the
    most the register-tile factorisations and the streaming solves take (the
    10 x 10 and 5 x 5 register tiles of 160)."""
    n = 80
    c = _cfg(n=n, sx=1, sy=1, overlap=0, nu=1e-4, mu=1e-3)
    prob = oracle_problem(c)
    subs = dd.subdomains(n, 1, 1, 0)
    ref = oras.ras_apply(prob, np.zeros((n, n)), np.zeros((n, n)), subs, oracle_opts(c), True)
    h = gpu_problem(c, prec)
    try:
        Fy, Fp = zeros(n), zeros(n)
        ras.ras_apply(h, zeros(n), zeros(n), 1, Fy, Fp)
        assert ras.ras_local_iterations(h)[0] == ref.iterations[0]
        assert rel_inf(Fy.cpu().numpy(), ref.Fy) <= tol
        assert rel_inf(Fp.cpu().numpy(), ref.Fp) <= tol
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_inactive_control(prec, tol):
    """mu much larger than |p|: the L1 term switches the control off (u ~ 0,
    P_eps in its flat region); the solve still matches the oracle."""
    n = 47
    c = _cfg(n=n, sx=3, sy=3, overlap=2, nu=1e-4, mu=10.0)
    ref = solvers.raspen(oracle_problem(c), c["sx"], c["sy"], c["overlap"], oracle_opts(c))
    assert np.abs(ref.P).max() < 0.1 * c["mu"]
    h = gpu_problem(c, prec)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
    finally:
        ras.ras_destroy(h)


def test_empty_batches_are_rejected():
    out = ras.ctypes.c_void_p()
    assert ras.lib().ras_batch_create(0, None, None, None, ras.ctypes.byref(out)) == ras.RAS_EINVAL
    s = ras.ras_server_create(1 << 30, 4)
    try:
        assert ras.ras_server_step(s) == (0, 0)
        assert ras.ras_server_counts(s) == (0, 0, 0)
        assert ras.ras_server_finished_ids(s) == []
    finally:
        ras.ras_server_destroy(s)
