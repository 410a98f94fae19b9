"""The layouts and schedules of the sensitivity studies against the oracle:
the weak-scaling layout (s x s subdomains of 50^2 nodes, overlap 2) at
s = 2 and 3, and eps-continuation schedules (eps0, gamma) other than the
default, full RASPEN solves in FP64 and mixed precision (same tolerances
and counts as the other parity tests)."""
import pytest

from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_problem, oracle_opts, oracle_problem, rel_inf, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)]
CASES = {"weak2": inputs.problem("weak2"), "weak3": inputs.problem("weak3"),
         "n63-eps1-gamma0.5": inputs.problem("n63", eps0=1.0, gamma=0.5),
         "n63-eps1e-3-gamma0.2": inputs.problem("n63", eps0=1e-3, gamma=0.2),
         "n63-eps1e-5-gamma0.1": inputs.problem("n63", eps0=1e-5, gamma=0.1)}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    cfg = CASES[request.param]
    return cfg, solvers.raspen(oracle_problem(cfg), cfg["sx"], cfg["sy"], cfg["overlap"], oracle_opts(cfg))


@pytest.mark.parametrize("prec,tol", PRECS)
def test_sweep_case_raspen_solve(case, prec, tol):
    cfg, ref = case
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
