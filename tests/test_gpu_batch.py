"""Batches of independent problems of uneven size in one handle (every sweep
step one launch for all problems, GMRES in lockstep): each problem's result
must equal the oracle's RASPEN solve of that problem alone (same tolerance
and counts as the single-problem parity tests) and the GPU's own
single-problem solve."""
import numpy as np
import pytest

from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_opts, gpu_problem, oracle_opts, oracle_problem, rel_inf, \
    to_dev, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402


def _batch_cfgs():
    """Small problems shaped like the uneven-batch workload: different n,
    mu, nu, phi, block sizes and overlaps (including a ragged layout)."""
    base = inputs.problem("n63")
    specs = [(63, 4, 2, 0, 1e-4, 1e-3), (31, 2, 1, 1, 3e-5, 2e-3), (47, 3, 3, 0, 1e-3, 5e-4),
             (40, 2, 4, 1, 2e-4, 4e-3), (63, 2, 2, 0, 1e-5, 1e-2), (24, 1, 2, 1, 1e-4, 1e-3)]
    out = []
    for k, (n, s, ov, phi, nu, mu) in enumerate(specs):
        c = dict(base)
        c.update(n=n, sx=s, sy=s, overlap=ov, phi=phi, nu=nu, mu=mu, yd=("fourier", 1000 + k))
        out.append(c)
    return out


@pytest.fixture(scope="module")
def oracle_solves():
    res = []
    for c in _batch_cfgs():
        prob = oracle_problem(c)
        res.append(solvers.raspen(prob, c["sx"], c["sy"], c["overlap"], oracle_opts(c)))
    return res


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)])
def test_batch_matches_individual_solves(oracle_solves, prec, tol):
    cfgs = _batch_cfgs()
    probs = [dict(n=c["n"], sx=c["sx"], sy=c["sy"], overlap=c["overlap"], phi=c["phi"], nu=c["nu"], mu=c["mu"],
                  y_d=to_dev(inputs.make_yd(c))) for c in cfgs]
    h = ras.ras_batch_create(probs, gpu_opts(cfgs[0], prec))
    try:
        assert ras.ras_problem_count(h) == len(cfgs)
        ys = [zeros(c["n"]) for c in cfgs]
        ps = [zeros(c["n"]) for c in cfgs]
        rc, stats = ras.ras_batch_raspen_solve(h, ys, ps)
        for k, (c, ref, st) in enumerate(zip(cfgs, oracle_solves, stats)):
            assert rel_inf(ys[k].cpu().numpy(), ref.Y) <= tol, k
            assert rel_inf(ps[k].cpu().numpy(), ref.P) <= tol, k
            assert st.outer_its == ref.outer, k
            assert st.inner_its_sum == sum(sum(i) for i in ref.inner_its), k
            # the same problem alone on the GPU
            h1 = gpu_problem(c, prec)
            try:
                y1, p1 = zeros(c["n"]), zeros(c["n"])
                rc1, st1 = ras.ras_raspen_solve(h1, y1, p1)
                assert rel_inf(ys[k].cpu().numpy(), y1.cpu().numpy()) <= tol
                assert rel_inf(ps[k].cpu().numpy(), p1.cpu().numpy()) <= tol
                assert st1.outer_its == st.outer_its and st1.inner_its_sum == st.inner_its_sum
            finally:
                ras.ras_destroy(h1)
    finally:
        ras.ras_destroy(h)


def test_batch_rejects_single_problem_calls():
    c = _batch_cfgs()[:2]
    probs = [dict(n=x["n"], sx=x["sx"], sy=x["sy"], overlap=x["overlap"], phi=x["phi"], nu=x["nu"], mu=x["mu"],
                  y_d=to_dev(inputs.make_yd(x))) for x in c]
    h = ras.ras_batch_create(probs)
    try:
        n = c[0]["n"]
        bufs = [zeros(n) for _ in range(4)]
        rc = ras.lib().ras_apply(h.ptr, bufs[0].data_ptr(), bufs[1].data_ptr(), 1, bufs[2].data_ptr(),
                                 bufs[3].data_ptr(), None)
        assert rc == ras.RAS_EINVAL
    finally:
        ras.ras_destroy(h)
