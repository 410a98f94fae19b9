"""GMRES restart cycles as CUDA graphs (ras_use_graphs): the Arnoldi steps,
Givens updates and stop tests run on the device either way, so a solve with
graphs gives bit for bit the result, counts and iterates of the same solve
step by step, for RASPEN, Newton_RAS and a batch of problems of uneven size;
a profiled solve (step by step) gives the same result and per-kernel times."""
import numpy as np
import pytest

from paper_2411_00546_gb300 import inputs
from gpu_util import gpu_opts, gpu_problem, to_dev, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

SOLVERS = {"raspen": ras.ras_raspen_solve, "newton_ras": ras.ras_newton_ras_solve}


def _solve(cfg, prec, graphs, method):
    n = cfg["n"]
    h = gpu_problem(cfg, prec)
    try:
        ras.ras_use_graphs(h, graphs)
        y, p = zeros(n), zeros(n)
        rc, st = SOLVERS[method](h, y, p)
        return y.cpu().numpy(), p.cpu().numpy(), st.as_dict()
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("method", sorted(SOLVERS))
@pytest.mark.parametrize("prec", [ras.RAS_FP64, ras.RAS_MIXED])
@pytest.mark.parametrize("name", ["n63", "n255"])
def test_graph_cycles_equal_step_by_step(name, prec, method):
    cfg = inputs.problem(name)
    y0, p0, s0 = _solve(cfg, prec, False, method)
    y1, p1, s1 = _solve(cfg, prec, True, method)
    assert s0["gmres_its"] > 0
    assert np.array_equal(y0, y1) and np.array_equal(p0, p1)
    assert s0 == s1


def test_graph_cycles_equal_step_by_step_batch():
    base = inputs.problem("n63")
    specs = [(63, 4, 2, 0, 1e-4, 1e-3), (31, 2, 1, 1, 3e-5, 2e-3), (95, 3, 4, 0, 1e-3, 5e-4), (40, 2, 4, 1, 2e-4, 4e-3)]
    cfgs = []
    for k, (n, s, ov, phi, nu, mu) in enumerate(specs):
        c = dict(base)
        c.update(n=n, sx=s, sy=s, overlap=ov, phi=phi, nu=nu, mu=mu, yd=("fourier", 3000 + k))
        cfgs.append(c)
    out = []
    for graphs in (False, True):
        probs = [dict(n=c["n"], sx=c["sx"], sy=c["sy"], overlap=c["overlap"], phi=c["phi"], nu=c["nu"], mu=c["mu"],
                      y_d=to_dev(inputs.make_yd(c))) for c in cfgs]
        h = ras.ras_batch_create(probs, gpu_opts(cfgs[0], ras.RAS_MIXED))
        try:
            ras.ras_use_graphs(h, graphs)
            ys = [zeros(c["n"]) for c in cfgs]
            ps = [zeros(c["n"]) for c in cfgs]
            rc, stats = ras.ras_batch_raspen_solve(h, ys, ps)
            out.append(([y.cpu().numpy() for y in ys], [p.cpu().numpy() for p in ps], [s.as_dict() for s in stats]))
        finally:
            ras.ras_destroy(h)
    (Y0, P0, S0), (Y1, P1, S1) = out
    for k in range(len(cfgs)):
        assert np.array_equal(Y0[k], Y1[k]) and np.array_equal(P0[k], P1[k]), k
        assert S0[k] == S1[k], k


def test_profiled_solve_equals_graph_solve():
    cfg = inputs.problem("n63")
    n = cfg["n"]
    h = gpu_problem(cfg, ras.RAS_MIXED)
    try:
        y, p = zeros(n), zeros(n)
        ras.ras_raspen_solve(h, y, p)
        yg, pg = y.cpu().numpy(), p.cpu().numpy()
        ras.ras_profile(h, 1)
        y.zero_()
        p.zero_()
        rc, st = ras.ras_raspen_solve(h, y, p)
        prof = ras.ras_profile_all(h)
        ras.ras_profile(h, 0)
        assert np.array_equal(y.cpu().numpy(), yg) and np.array_equal(p.cpu().numpy(), pg)
        jvp_ms, jvp_n, jvp_work = prof["jvp"]
        kr_ms, kr_n, kr_work = prof["krylov"]
        # one Jacobian action per GMRES step (plus one per restart for the residual)
        assert jvp_n >= st.gmres_its and jvp_ms > 0 and jvp_work > 0
        assert kr_n >= 5 * st.gmres_its and kr_ms > 0
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("prec", [ras.RAS_FP64, ras.RAS_MIXED])
def test_graph_evaluation_equals_step_by_step(prec):
    """The RASPEN-function evaluation (local Newton sweeps under a graph WHILE
    node, the factor kernel chosen on the device) equals the host-driven loop."""
    cfg = inputs.problem("n255")
    n = cfg["n"]
    out = []
    for graphs in (False, True):
        h = gpu_problem(cfg, prec)
        try:
            ras.ras_use_graphs(h, graphs)
            Fy, Fp = zeros(n), zeros(n)
            ras.ras_apply(h, zeros(n), zeros(n), 1, Fy, Fp)
            out.append((Fy.cpu().numpy(), Fp.cpu().numpy(), list(ras.ras_local_iterations(h))))
        finally:
            ras.ras_destroy(h)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and max(out[0][2]) > 1
