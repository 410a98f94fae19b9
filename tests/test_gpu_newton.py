"""Newton and Newton_eps (Alg. 1 with unpreconditioned GMRES on the global
Jacobian, the paper's baselines) through ras_newton_solve, against the
oracle's newton_gmres on the same seeded inputs: same solution within the
stated tolerance, same Newton and GMRES counts."""
import numpy as np
import pytest

from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_problem, oracle_opts, oracle_problem, rel_inf, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402


def _cfg(n, eps0, phi):
    c = dict(inputs.problem("n63"))
    c.update(n=n, sx=2, sy=2, overlap=1, phi=phi, nu=1e-3, mu=2e-2, yd=("fourier", 300 + n), eps0=eps0)
    return c


CASES = [(15, 0.1, 0), (15, 1e-6, 0), (24, 0.1, 1)]


@pytest.fixture(scope="module")
def oracle_runs():
    out = {}
    for n, eps0, phi in CASES:
        c = _cfg(n, eps0, phi)
        out[n, eps0, phi] = solvers.newton_gmres(oracle_problem(c), oracle_opts(c, gmres_maxit=4000))
    return out


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)])
@pytest.mark.parametrize("n,eps0,phi", CASES)
def test_newton_solve_parity(oracle_runs, n, eps0, phi, prec, tol):
    c = _cfg(n, eps0, phi)
    ref = oracle_runs[n, eps0, phi]
    assert ref.status >= 0
    h = gpu_problem(c, prec, gmres_maxit=4000)
    try:
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_newton_solve(h, y, p)
        assert rc in (ras.RAS_OK, ras.RAS_OK_FLOOR)
        assert rel_inf(y.cpu().numpy(), ref.Y) <= tol
        assert rel_inf(p.cpu().numpy(), ref.P) <= tol
        assert st.outer_its == ref.outer
        assert st.gmres_its == sum(ref.gmres_its)
        assert st.halvings == ref.newton.halvings
    finally:
        ras.ras_destroy(h)


def test_newton_solve_host_method():
    """The host-buffer entry point runs the same solver (RAS_METHOD_NEWTON)."""
    n, eps0, phi = CASES[0]
    c = _cfg(n, eps0, phi)
    h = gpu_problem(c, ras.RAS_FP64, gmres_maxit=4000)
    try:
        y, p = zeros(n), zeros(n)
        ras.ras_newton_solve(h, y, p)
        yh = torch.zeros((n, n), dtype=torch.float64)
        ph = torch.zeros_like(yh)
        rc, st = ras.ras_solve_host(h, ras.RAS_METHOD_NEWTON, None, yh, ph)
        assert rc in (ras.RAS_OK, ras.RAS_OK_FLOOR)
        assert np.array_equal(yh.numpy(), y.cpu().numpy())
        assert np.array_equal(ph.numpy(), p.cpu().numpy())
    finally:
        ras.ras_destroy(h)
