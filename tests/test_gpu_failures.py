"""Failure paths of the C ABI, each made on the host; none faults or hangs the GPU.

* RAS_ETIMEOUT: with ras_opts.wait_test = 1 the first slab wait of every
  streamed local solve gives up at once, with its bulk copy still in flight.
  The kernel drains the copies it issued (normal wait limit), records the
  timeout and returns; the call reports RAS_ETIMEOUT. After
  ras_set_opts(wait_test = 0) the same handle gives the results of a fresh one.
* RAS_ESINGULAR: in mixed precision the local factors are FP32; a problem with
  1/nu = 1e40 (beyond the FP32 range) on an active control has local Jacobian
  entries the FP32 factorisation cannot hold, and it finds no usable pivot.
  The FP64 path factors the same problem.
"""
import numpy as np
import pytest

from gpu_util import gpu_opts, gpu_problem, to_dev, zeros
from paper_2411_00546_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402

PRECS = [ras.RAS_FP64, ras.RAS_MIXED]


def _apply(h, n, cont=1):
    Fy, Fp = zeros(n), zeros(n)
    rc, st = ras.ras_apply(h, zeros(n), zeros(n), cont, Fy, Fp, check=False)
    return rc, Fy.cpu().numpy(), Fp.cpu().numpy(), ras.ras_local_iterations(h)


@pytest.mark.parametrize("prec", PRECS)
def test_wait_timeout_is_reported_and_the_handle_recovers(prec):
    cfg = inputs.problem("n63")
    n = cfg["n"]
    ref = gpu_problem(cfg, prec)
    h = gpu_problem(cfg, prec, wait_test=1)
    try:
        rc0, Fy0, Fp0, its0 = _apply(ref, n)
        assert rc0 == ras.RAS_OK
        rc, _, _, _ = _apply(h, n)
        assert rc == ras.RAS_ETIMEOUT, rc
        assert "wait" in ras.ras_last_error(h)
        # the switch also stops a whole solve at its first local solve
        y, p = zeros(n), zeros(n)
        rc, st = ras.ras_raspen_solve(h, y, p, check=False)
        assert rc == ras.RAS_ETIMEOUT and st.status == ras.RAS_ETIMEOUT
        # and the linear RAS preconditioner (its local solves stream the same way)
        rY = to_dev(np.ones((n, n)))
        with pytest.raises(ras.RasError) as e:
            ras.ras_precondition(h, zeros(n), zeros(n), cfg["eps_min"], rY, rY.clone(), zeros(n), zeros(n))
        assert e.value.code == ras.RAS_ETIMEOUT
        # switched off, the same handle computes what a fresh one does
        ras.ras_set_opts(h, gpu_opts(cfg, prec, wait_test=0))
        rc1, Fy1, Fp1, its1 = _apply(h, n)
        assert rc1 == ras.RAS_OK
        np.testing.assert_array_equal(Fy1, Fy0)
        np.testing.assert_array_equal(Fp1, Fp0)
        assert its1 == its0
    finally:
        ras.ras_destroy(h)
        ras.ras_destroy(ref)


def test_wait_timeout_inside_the_jacobian_action():
    """Switching the test on between an evaluation and its Jacobian action
    keeps the evaluation's factors; the action's first local solve times out,
    and once switched off the action equals the undisturbed one."""
    cfg = inputs.problem("n63")
    n = cfg["n"]
    h = gpu_problem(cfg, ras.RAS_MIXED)
    try:
        assert _apply(h, n)[0] == ras.RAS_OK
        rng = np.random.default_rng(4)
        dy, dp = to_dev(rng.standard_normal((n, n))), to_dev(1e-3 * rng.standard_normal((n, n)))
        oy0, op0 = zeros(n), zeros(n)
        ras.ras_jvp(h, dy, dp, oy0, op0)
        ras.ras_set_opts(h, gpu_opts(cfg, ras.RAS_MIXED, wait_test=1))
        with pytest.raises(ras.RasError) as e:
            ras.ras_jvp(h, dy, dp, zeros(n), zeros(n))
        assert e.value.code == ras.RAS_ETIMEOUT
        ras.ras_set_opts(h, gpu_opts(cfg, ras.RAS_MIXED, wait_test=0))
        oy1, op1 = zeros(n), zeros(n)
        ras.ras_jvp(h, dy, dp, oy1, op1)
        assert torch.equal(oy0, oy1) and torch.equal(op0, op1)
    finally:
        ras.ras_destroy(h)


def test_wait_test_switch_is_validated():
    cfg = inputs.problem("n63")
    with pytest.raises(ras.RasError):
        gpu_problem(cfg, ras.RAS_FP64, wait_test=2)


def test_fp32_unrepresentable_local_jacobian_is_singular():
    n = 31
    nu, mu = 1e-40, 1e-3
    yd = to_dev(inputs.yd_fourier(n, 2))
    P0 = to_dev(np.full((n, n), 0.5))          # |p| >> mu: active control, 1 - P_eps' = 1
    out = {}
    for prec in PRECS:
        h = ras.ras_create(n, 2, 2, 2, ras.RAS_PHI_CUBIC, nu, mu, yd, None,
                           ras.make_opts(precision=prec, eps0=1e-6, eps_min=1e-6))
        try:
            Fy, Fp = zeros(n), zeros(n)
            rc, st = ras.ras_apply(h, zeros(n), P0, 0, Fy, Fp, check=False)
            out[prec] = (rc, st.status)
        finally:
            ras.ras_destroy(h)
    assert out[ras.RAS_MIXED][0] == ras.RAS_ESINGULAR, out
    assert out[ras.RAS_FP64][0] != ras.RAS_ESINGULAR, out
