"""The allocation-free residual entry point (ras_residual_static) against the
handle-based ras_residual and against the oracle's residual.

Some callers cannot allocate device memory (another allocator owns it, or an
allocation's device synchronisation is not acceptable in their loop); they
use ras_residual_static, whose scratch is a fixed array inside the library.
This file is collected last on purpose, and it runs the same alone in a fresh
process: two calls in a row, each checked against the handle-based result
and the oracle's F within the tolerance of the other residual tests, a check
that the second call leaves the device's free memory unchanged, plus the size
limit."""
import numpy as np
import pytest

from gpu_util import to_dev, zeros
from oracle import discretization as fd
from paper_2411_00546_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2411_00546_gb300 import ras  # noqa: E402


def test_static_residual_matches_handle_residual_twice():
    n, phi, nu, mu, kappa = 100, ras.RAS_PHI_KAPPA, 1e-5, 2e-3, 0.1
    rng = np.random.default_rng(21)
    yd_h = inputs.yd_fourier(n, 3)
    f_h = 0.4 * rng.standard_normal((n, n))
    yd, f = to_dev(yd_h), to_dev(f_h)
    prob = fd.Problem(n, phi, nu, mu, yd_h, f_h, kappa=kappa)
    h = ras.ras_create(n, 3, 3, 2, phi, nu, mu, yd, f, ras.make_opts(kappa=kappa))
    stream = torch.cuda.current_stream().cuda_stream
    try:
        cases = []
        for eps in (1e-2, 1e-7):
            Y = 0.5 * rng.standard_normal((n, n))
            P = 3e-3 * rng.standard_normal((n, n))
            cases.append((eps, Y, P, to_dev(Y), to_dev(P), zeros(n), zeros(n), zeros(n), zeros(n),
                          torch.full((1,), -1.0, dtype=torch.float64, device="cuda")))
        torch.cuda.synchronize()
        free = []
        for call, (eps, Y, P, y, p, ry, rp, sy, sp, nd) in enumerate(cases):
            ref = ras.ras_residual(h, y, p, eps, ry, rp)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            ras.ras_residual_static(n, phi, nu, mu, kappa, eps, y, p, yd, f, sy, sp, nd, stream=stream)
            torch.cuda.synchronize()
            free.append((free_before, torch.cuda.mem_get_info()[0]))
            scale = (n + 1) ** 2 * max(np.abs(Y).max(), np.abs(P).max())
            oy, op = fd.residual(prob, Y, P, eps)
            for got, want, orc in ((sy, ry, oy), (sp, rp, op)):
                g, w = got.cpu().numpy(), want.cpu().numpy()
                assert np.max(np.abs(g - w)) <= 1e-13 * scale + 1e-12 * np.abs(w).max(), call
                assert np.max(np.abs(g - orc)) <= 1e-13 * scale + 1e-12 * np.abs(orc).max(), call
            assert abs(float(nd.item()) - ref) <= 1e-12 * ref, call
            onrm = float(np.sqrt(np.sum(oy ** 2) + np.sum(op ** 2)))
            assert abs(float(nd.item()) - onrm) <= 1e-12 * onrm, call
        # the second call (the device code is loaded by then) takes no device memory
        assert free[1][0] == free[1][1], free
    finally:
        ras.ras_destroy(h)


def test_static_residual_rejects_oversized_grid():
    rc = ras.lib().ras_residual_static(ras.RAS_STATIC_MAX_N + 1, 0, 1e-4, 1e-3, 0.1, 1e-3,
                                       None, None, None, None, None, None, None, None)
    assert rc == ras.RAS_EINVAL
    with pytest.raises(ras.RasError):
        ras.ras_residual_static(ras.RAS_STATIC_MAX_N + 1, 0, 1e-4, 1e-3, 0.1, 1e-3, None, None, None)
