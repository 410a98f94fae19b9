"""Continuous batching (ras_server_*): requests submitted while others are on
the GPU are admitted between steps and advanced together; each result must be
the solve of that problem alone (the GPU's ras_raspen_solve, same counts) and
the oracle's, within the stated tolerance, whatever the mix."""
import numpy as np
import pytest

from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_opts, gpu_problem, oracle_opts, oracle_problem, rel_inf, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras, serve  # noqa: E402


def _cfgs():
    base = inputs.problem("n63")
    specs = [(63, 4, 2, 0, 1e-4, 1e-3), (31, 2, 1, 1, 3e-5, 2e-3), (47, 3, 3, 0, 1e-3, 5e-4),
             (40, 2, 4, 1, 2e-4, 4e-3), (63, 2, 2, 0, 1e-5, 1e-2), (24, 1, 2, 1, 1e-4, 1e-3)]
    out = []
    for k, (n, s, ov, phi, nu, mu) in enumerate(specs):
        c = dict(base)
        c.update(n=n, sx=s, sy=s, overlap=ov, phi=phi, nu=nu, mu=mu, yd=("fourier", 2000 + k))
        out.append(c)
    return out


def _req(c):
    return dict(n=c["n"], sx=c["sx"], sy=c["sy"], overlap=c["overlap"], phi=c["phi"], nu=c["nu"], mu=c["mu"],
                y_d=inputs.make_yd(c))


@pytest.fixture(scope="module")
def alone():
    """Each problem solved alone on the GPU, both precisions."""
    out = {}
    for prec in (ras.RAS_FP64, ras.RAS_MIXED):
        for k, c in enumerate(_cfgs()):
            h = gpu_problem(c, prec)
            try:
                y, p = zeros(c["n"]), zeros(c["n"])
                rc, st = ras.ras_raspen_solve(h, y, p)
                out[prec, k] = (y.cpu().numpy(), p.cpu().numpy(), st.as_dict())
            finally:
                ras.ras_destroy(h)
    return out


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)])
def test_staggered_arrivals_match_solves_alone(alone, prec, tol):
    cfgs = _cfgs()
    s = ras.ras_server_create(4 << 30, 16, gpu_opts(cfgs[0], prec))
    try:
        ids = {}
        # two requests before the first step, the others one per step while
        # earlier ones are still iterating
        for k in (0, 1):
            ids[ras.ras_server_submit(s, _req(cfgs[k]))] = k
        res = {}
        nxt, steps = 2, 0
        while len(res) < len(cfgs):
            act, _ = ras.ras_server_step(s)
            steps += 1
            if nxt < len(cfgs):
                ids[ras.ras_server_submit(s, _req(cfgs[nxt]))] = nxt
                nxt += 1
            for rid in ras.ras_server_finished_ids(s):
                rc, y, p, st = ras.ras_server_fetch(s, rid)
                assert rc == ras.RAS_OK
                res[ids[rid]] = (y, p, st.as_dict())
            assert steps < 200
        assert ras.ras_server_counts(s) == (0, 0, 0)
    finally:
        ras.ras_server_destroy(s)
    for k in range(len(cfgs)):
        y, p, st = res[k]
        ya, pa, sa = alone[prec, k]
        assert rel_inf(y, ya) <= tol, k
        assert rel_inf(p, pa) <= tol, k
        assert st["outer_its"] == sa["outer_its"], k
        assert st["inner_its_sum"] == sa["inner_its_sum"], k
        assert st["evaluations"] == sa["evaluations"], k


def test_served_results_match_oracle(alone):
    """Two of the served problems against the oracle's RASPEN (mixed)."""
    cfgs = _cfgs()
    reqs = [(0.0, _req(c)) for c in cfgs]
    out = serve.run_stream(reqs, 4 << 30, 16, gpu_opts(cfgs[0], ras.RAS_MIXED), keep_results=True)
    for k in (1, 4):
        c = cfgs[k]
        ref = solvers.raspen(oracle_problem(c), c["sx"], c["sy"], c["overlap"], oracle_opts(c))
        y, p = out["results"][k]
        assert rel_inf(y, ref.Y) <= MIXED_TOL
        assert rel_inf(p, ref.P) <= MIXED_TOL
        assert out["stats"][k]["outer_its"] == ref.outer
        assert out["stats"][k]["inner_its_sum"] == sum(sum(i) for i in ref.inner_its)


def test_budget_limits_admission(alone):
    """A budget that holds about two of the requests: admission waits for
    memory, the held bytes stay within the budget, every request finishes."""
    cfgs = _cfgs()
    opts = gpu_opts(cfgs[0], ras.RAS_MIXED)
    need = [a + 2 * b for a, b in (ras.ras_server_request_bytes(_req(c), opts) for c in cfgs)]
    budget = int(sorted(need)[-1] + sorted(need)[-2] + 1)
    s = ras.ras_server_create(budget, 16, opts)
    try:
        ids = {ras.ras_server_submit(s, _req(c)): k for k, c in enumerate(cfgs)}
        got, peak = {}, 0
        for _ in range(400):
            act, _ = ras.ras_server_step(s)
            peak = max(peak, act)
            assert ras.ras_server_device_bytes(s) <= budget
            for rid in ras.ras_server_finished_ids(s):
                rc, y, p, st = ras.ras_server_fetch(s, rid)
                got[ids[rid]] = (y, p)
            if len(got) == len(cfgs):
                break
        assert len(got) == len(cfgs)
        assert peak < len(cfgs)
    finally:
        ras.ras_server_destroy(s)
    for k in range(len(cfgs)):
        ya, pa, _ = alone[ras.RAS_MIXED, k]
        assert rel_inf(got[k][0], ya) <= MIXED_TOL
        assert rel_inf(got[k][1], pa) <= MIXED_TOL


def test_server_rejects_bad_requests():
    cfgs = _cfgs()
    s = ras.ras_server_create(1 << 20, 4)
    try:
        with pytest.raises(ras.RasError) as e:
            ras.ras_server_submit(s, _req(cfgs[0]))   # larger than a 1 MiB budget
        assert e.value.code == ras.RAS_ENOMEM
        assert ras.lib().ras_server_fetch(s.ptr, 12345, None, None, None) == ras.RAS_EINVAL   # unknown id
        assert ras.ras_server_step(s) == (0, 0)
    finally:
        ras.ras_server_destroy(s)


def test_easy_request_is_not_held_by_a_hard_one():
    """A request that needs few GMRES steps, admitted with one that needs many,
    finishes first (its steps are restart cycles, not the other's whole GMRES
    solve) and still equals its solve alone."""
    base = inputs.problem("n63")
    hard = dict(base, n=63, sx=4, sy=4, overlap=2, phi=0, nu=1e-6, mu=1e-3, yd=("fourier", 77))
    easy = dict(base, n=24, sx=2, sy=2, overlap=1, phi=0, nu=1e-3, mu=1e-2, yd=("fourier", 78))
    opts = gpu_opts(base, ras.RAS_MIXED)
    s = ras.ras_server_create(4 << 30, 8, opts)
    try:
        ih = ras.ras_server_submit(s, _req(hard))
        ie = ras.ras_server_submit(s, _req(easy))
        order, res = [], {}
        for _ in range(2000):
            ras.ras_server_step(s)
            for rid in ras.ras_server_finished_ids(s):
                rc, y, p, st = ras.ras_server_fetch(s, rid)
                assert rc == ras.RAS_OK
                order.append(rid)
                res[rid] = (y, p, st.as_dict())
            if len(order) == 2:
                break
        assert order == [ie, ih]
    finally:
        ras.ras_server_destroy(s)
    for rid, c in ((ie, easy), (ih, hard)):
        h = gpu_problem(c, ras.RAS_MIXED)
        try:
            y1, p1 = zeros(c["n"]), zeros(c["n"])
            rc, st1 = ras.ras_raspen_solve(h, y1, p1)
            y, p, st = res[rid]
            assert rel_inf(y, y1.cpu().numpy()) <= MIXED_TOL
            assert rel_inf(p, p1.cpu().numpy()) <= MIXED_TOL
            assert st["outer_its"] == st1.outer_its and st["inner_its_sum"] == st1.inner_its_sum
        finally:
            ras.ras_destroy(h)


def test_cancel_waiting_and_admitted_requests():
    """Cancelling a waiting and an admitted request frees them; the others
    still finish with their solve-alone results."""
    cfgs = _cfgs()
    opts = gpu_opts(cfgs[0], ras.RAS_MIXED)
    s = ras.ras_server_create(4 << 30, 2, opts)   # two admitted at a time
    try:
        ids = [ras.ras_server_submit(s, _req(c)) for c in cfgs[:4]]
        ras.ras_server_step(s)                     # admits ids[0], ids[1]
        assert ras.ras_server_counts(s)[:2] == (2, 2)
        ras.ras_server_cancel(s, ids[1])           # admitted
        ras.ras_server_cancel(s, ids[3])           # waiting
        with pytest.raises(ras.RasError):
            ras.ras_server_cancel(s, 999)
        got = {}
        for _ in range(2000):
            ras.ras_server_step(s)
            for rid in ras.ras_server_finished_ids(s):
                got[rid] = ras.ras_server_fetch(s, rid)
            if len(got) == 2:
                break
        assert sorted(got) == sorted([ids[0], ids[2]])
        assert ras.ras_server_counts(s) == (0, 0, 0)
    finally:
        ras.ras_server_destroy(s)
