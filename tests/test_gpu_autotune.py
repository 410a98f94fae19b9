"""Launch-shape tuning (ras_autotune / ras_set_tuning) changes how the kernels
are launched, never what they compute: every shape the tuner can install gives
the oracle's solution of every problem of an uneven batch (same tolerance and
counts as the other parity tests), the autotuner's choice follows from its own
timings by the documented rule, and bad tunings are refused."""
import numpy as np
import pytest

from oracle import solvers
from paper_2411_00546_gb300 import inputs
from gpu_util import FP64_TOL, MIXED_TOL, gpu_opts, oracle_opts, oracle_problem, rel_inf, to_dev, zeros

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402


def _cfgs():
    """One problem per register-tile class: subdomains of 2 wx = 32, 40, 80,
    112 and 144 unknowns per grid line (padded to 32, 64, 96, 128, 160)."""
    base = inputs.problem("n63")
    specs = [(24, 2, 2, 0, 1e-4, 1e-3), (63, 4, 2, 1, 3e-5, 2e-3), (95, 3, 4, 0, 1e-3, 5e-4),
             (96, 2, 4, 1, 2e-4, 4e-3), (127, 2, 8, 0, 1e-5, 1e-2)]
    out = []
    for k, (n, s, ov, phi, nu, mu) in enumerate(specs):
        c = dict(base)
        c.update(n=n, sx=s, sy=s, overlap=ov, phi=phi, nu=nu, mu=mu, yd=("fourier", 2000 + k))
        out.append(c)
    return out


@pytest.fixture(scope="module")
def oracle_solves():
    return [solvers.raspen(oracle_problem(c), c["sx"], c["sy"], c["overlap"], oracle_opts(c)) for c in _cfgs()]


def _batch(prec):
    cfgs = _cfgs()
    probs = [dict(n=c["n"], sx=c["sx"], sy=c["sy"], overlap=c["overlap"], phi=c["phi"], nu=c["nu"], mu=c["mu"],
                  y_d=to_dev(inputs.make_yd(c))) for c in cfgs]
    return cfgs, ras.ras_batch_create(probs, gpu_opts(cfgs[0], prec))


def _solve(h, cfgs):
    ys = [zeros(c["n"]) for c in cfgs]
    ps = [zeros(c["n"]) for c in cfgs]
    rc, stats = ras.ras_batch_raspen_solve(h, ys, ps)
    return [y.cpu().numpy() for y in ys], [p.cpu().numpy() for p in ps], stats


def _check(cfgs, ref, Y, P, stats, tol):
    for k, (c, r, st) in enumerate(zip(cfgs, ref, stats)):
        assert rel_inf(Y[k], r.Y) <= tol, k
        assert rel_inf(P[k], r.P) <= tol, k
        assert st.outer_its == r.outer, k
        assert st.inner_its_sum == sum(sum(i) for i in r.inner_its), k


SHAPES = {
    "default": {},
    "factor_always_1024": dict(factor_wide_max=(10 ** 6,) * ras.RAS_NTILE),
    "factor_always_256": dict(factor_wide_max=(0,) * ras.RAS_NTILE),
    "solve_1_cta_per_sm": dict(solve_ctas_per_sm=1),
    "vec_blocks_152": dict(vec_blocks=152),
    "vec_blocks_1": dict(vec_blocks=1),
}


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)])
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_every_shape_matches_the_oracle(oracle_solves, shape, prec, tol):
    cfgs, h = _batch(prec)
    try:
        ras.ras_set_tuning(h, ras.make_tuning(**SHAPES[shape]))
        assert ras.ras_get_tuning(h).as_dict() == ras.make_tuning(**SHAPES[shape]).as_dict()
        Y, P, stats = _solve(h, cfgs)
        _check(cfgs, oracle_solves, Y, P, stats, tol)
    finally:
        ras.ras_destroy(h)


def test_solve_grid_does_not_change_results():
    """One CTA computes each subdomain whatever the persistent grid: bit-identical."""
    cfgs, h = _batch(ras.RAS_MIXED)
    try:
        Y0, P0, s0 = _solve(h, cfgs)
        ras.ras_set_tuning(h, ras.make_tuning(solve_ctas_per_sm=1))
        Y1, P1, s1 = _solve(h, cfgs)
        for k in range(len(cfgs)):
            assert np.array_equal(Y0[k], Y1[k]) and np.array_equal(P0[k], P1[k]), k
            assert s0[k].gmres_its == s1[k].gmres_its
    finally:
        ras.ras_destroy(h)


def _follows_report(t, rep, sms):
    """The installed tuning is the one the documented rule derives from the timings."""
    d = rep.as_dict()
    for c in range(ras.RAS_NTILE):
        rows = d["factor"].get(32 * (c + 1), [])
        differs, run, thr = False, True, 0
        for k, t256, t1024 in rows:
            default = 1 if k <= sms else 0
            times = (t256, t1024)
            use = default if times[1 - default] > 0.98 * times[default] else 1 - default
            differs = differs or use != default
            if run and use == 1:
                thr = k
            else:
                run = False
        assert t.factor_wide_max[c] == (thr if differs else -1), c
    solve = d["solve"]
    assert solve, "no solve-grid candidate timed"
    ms = [x[1] for x in solve]
    best = min(range(len(ms)), key=lambda i: ms[i])
    want = 0 if ms[best] > 0.98 * ms[-1] or best == len(ms) - 1 else solve[best][0]
    assert t.solve_ctas_per_sm == want
    vec = d["vectors"]
    assert [v for v, _ in vec] == [152, 304, 456, 608]
    ms = [x[1] for x in vec]
    best = min(range(len(ms)), key=lambda i: ms[i])
    want = vec[best][0] if ms[best] <= 0.98 * ms[-1] else 608
    assert t.vec_blocks == want


@pytest.mark.parametrize("prec,tol", [(ras.RAS_FP64, FP64_TOL), (ras.RAS_MIXED, MIXED_TOL)])
def test_autotune_choice_and_tuned_solve(oracle_solves, prec, tol):
    cfgs, h = _batch(prec)
    try:
        t, rep = ras.ras_autotune(h)
        assert ras.ras_get_tuning(h).as_dict() == t.as_dict()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        _follows_report(t, rep, sms)
        d = rep.as_dict()
        if prec == ras.RAS_MIXED:
            # every tile class of the batch was timed, at its full subdomain count last
            assert sorted(d["factor"]) == [32, 64, 96, 128, 160]
            for c, rows in d["factor"].items():
                assert all(a > 0 and b > 0 for _, a, b in rows)
        else:
            assert d["factor"] == {} and list(t.factor_wide_max) == [-1] * ras.RAS_NTILE
        Y, P, stats = _solve(h, cfgs)
        _check(cfgs, oracle_solves, Y, P, stats, tol)
    finally:
        ras.ras_destroy(h)


def test_autotune_leaves_solve_state():
    """Autotuning overwrites the internal iterate and factors only: the
    checkpoint state stays, a JVP needs a new evaluation, and the next solve
    agrees with the untuned one within the mixed tolerance."""
    cfg = inputs.problem("n63")
    yd = to_dev(inputs.make_yd(cfg))
    n = cfg["n"]
    h = ras.ras_create(n, cfg["sx"], cfg["sy"], cfg["overlap"], cfg["phi"], cfg["nu"], cfg["mu"], yd, None,
                       gpu_opts(cfg, ras.RAS_MIXED))
    try:
        y, p = zeros(n), zeros(n)
        ras.ras_raspen_solve(h, y, p)
        state = ras.ras_get_state(h).as_dict()
        t, _ = ras.ras_autotune(h)
        assert ras.ras_get_state(h).as_dict() == state
        oy, op = zeros(n), zeros(n)
        rc = ras.lib().ras_jvp(h.ptr, y.data_ptr(), p.data_ptr(), oy.data_ptr(), op.data_ptr())
        assert rc == ras.RAS_ESTATE
        y2, p2 = zeros(n), zeros(n)
        ras.ras_raspen_solve(h, y2, p2)
        assert rel_inf(y2.cpu().numpy(), y.cpu().numpy()) <= MIXED_TOL
        assert rel_inf(p2.cpu().numpy(), p.cpu().numpy()) <= MIXED_TOL
    finally:
        ras.ras_destroy(h)


@pytest.mark.parametrize("bad", [dict(factor_wide_max=(-2, -1, -1, -1, -1)), dict(solve_ctas_per_sm=-1),
                                 dict(solve_ctas_per_sm=65), dict(vec_blocks=0), dict(vec_blocks=609)])
def test_set_tuning_rejects_bad_values(bad):
    cfg = inputs.problem("n63")
    yd = to_dev(inputs.make_yd(cfg))
    h = ras.ras_create(cfg["n"], cfg["sx"], cfg["sy"], cfg["overlap"], cfg["phi"], cfg["nu"], cfg["mu"], yd, None,
                       gpu_opts(cfg, ras.RAS_MIXED))
    try:
        before = ras.ras_get_tuning(h).as_dict()
        assert ras.ras_set_tuning(h, ras.make_tuning(**bad), check=False) == ras.RAS_EINVAL
        assert ras.ras_get_tuning(h).as_dict() == before
    finally:
        ras.ras_destroy(h)
