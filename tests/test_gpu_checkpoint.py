"""Checkpoint / resume of the outer solves (ras_get_state / ras_set_state):
a solve stopped after K outer iterations and resumed in a fresh handle from
the saved state and iterate reproduces the uninterrupted solve bit for bit,
with the same counts."""
import numpy as np
import pytest

from paper_2411_00546_gb300 import inputs
from gpu_util import gpu_problem, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

CASES = {
    "raspen": (ras.ras_raspen_solve, "kmax_outer_raspen", 1, dict(inputs.problem("n63"))),
    "newton_ras": (ras.ras_newton_ras_solve, "kmax_outer_newton", 5, dict(inputs.problem("n63"))),
    "newton": (ras.ras_newton_solve, "kmax_outer_newton", 2,
               dict(inputs.problem("n63"), n=15, sx=2, sy=2, overlap=1, nu=1e-3, mu=2e-2, yd=("fourier", 315))),
}


@pytest.mark.parametrize("prec", [ras.RAS_FP64, ras.RAS_MIXED])
@pytest.mark.parametrize("name", sorted(CASES))
def test_resume_reproduces_the_uninterrupted_solve(name, prec):
    fn, cap, K, cfg = CASES[name]
    n = cfg["n"]
    extra = dict(gmres_maxit=4000) if name == "newton" else {}
    h = gpu_problem(cfg, prec, **extra)
    try:
        y, p = zeros(n), zeros(n)
        rc, full = fn(h, y, p)
        Yf, Pf = y.cpu().numpy(), p.cpu().numpy()
        assert full.outer_its > K
    finally:
        ras.ras_destroy(h)
    h2 = gpu_problem(cfg, prec, **dict(extra, **{cap: K}))
    try:
        y2, p2 = zeros(n), zeros(n)
        rc, part = fn(h2, y2, p2, check=False)
        assert rc == ras.RAS_ENOCONV and part.outer_its == K
        state = ras.ras_get_state(h2)
        assert state.k == K and state.res0 == full.res0
    finally:
        ras.ras_destroy(h2)
    h3 = gpu_problem(cfg, prec, **extra)
    try:
        ras.ras_set_state(h3, state)
        rc, rest = fn(h3, y2, p2)
        assert np.array_equal(y2.cpu().numpy(), Yf)
        assert np.array_equal(p2.cpu().numpy(), Pf)
        assert rest.outer_its == full.outer_its
        assert rest.res0 == full.res0 and rest.res == full.res
        end = ras.ras_get_state(h3)
        assert end.k == full.outer_its and end.stop == state.stop
    finally:
        ras.ras_destroy(h3)


def test_state_errors():
    cfg = dict(inputs.problem("n63"))
    h = gpu_problem(cfg, ras.RAS_MIXED)
    try:
        st = ras.ras_state()
        assert ras.lib().ras_get_state(h.ptr, st) == ras.RAS_ESTATE   # no solve yet
        bad = ras.ras_state(method=7, k=0, eps=1e-6, res0=1.0, stop=1e-10)
        assert ras.lib().ras_set_state(h.ptr, bad) == ras.RAS_EINVAL
        other = ras.ras_state(method=ras.RAS_METHOD_NEWTON_RAS, k=1, eps=1e-6, res0=1.0, stop=1e-10)
        ras.ras_set_state(h, other)
        n = cfg["n"]
        rc, _ = ras.ras_raspen_solve(h, zeros(n), zeros(n), check=False)
        assert rc == ras.RAS_ESTATE                                   # state of another method
        rc, _ = ras.ras_raspen_solve(h, zeros(n), zeros(n))          # one-shot: a fresh solve runs
        assert rc == ras.RAS_OK
    finally:
        ras.ras_destroy(h)
