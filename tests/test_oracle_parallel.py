"""The process-parallel oracle engine (oracle/parallel.py) against the serial
oracle: Alg. 3 computes every local correction from x alone and the
restricted prolongation writes each node from its one owner, so spreading the
subdomains over processes must change no value and no count."""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import discretization as fd
from oracle import parallel
from oracle import pointwise as pw
from oracle import ras as oras
from oracle import solvers
from paper_2411_00546_gb300 import inputs


@pytest.mark.parametrize("name,layout,workers", [("n63", None, 3), ("n63", (3, 2, 3), 4)])
def test_parallel_raspen_equals_serial(name, layout, workers):
    cfg = inputs.problem(name)
    if layout is not None:
        cfg["sx"], cfg["sy"], cfg["overlap"] = layout
    prob = fd.Problem(cfg["n"], cfg["phi"], cfg["nu"], cfg["mu"], inputs.make_yd(cfg))
    o = oras.Options(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"], eps0=cfg["eps0"],
                     gamma=cfg["gamma"], eps_min=cfg["eps_min"])
    ref = solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], o)
    subs = dd.subdomains(cfg["n"], cfg["sx"], cfg["sy"], cfg["overlap"])
    with parallel.ParallelEngine(prob, subs, o, workers) as eng:
        got = solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], o, engine=eng)
        assert eng.workers == workers
    np.testing.assert_array_equal(got.Y, ref.Y)
    np.testing.assert_array_equal(got.P, ref.P)
    assert got.outer == ref.outer and got.gmres_its == ref.gmres_its
    assert got.inner_its == ref.inner_its
    assert got.norms == ref.norms


def test_parallel_engine_reports_worker_errors_and_stale_states():
    n = 12
    prob = fd.Problem(n, pw.PHI_CUBIC, 1e-2, 0.05, np.random.default_rng(1).standard_normal((n, n)))
    subs = dd.subdomains(n, 2, 2, 1)
    o = oras.Options(eps0=1e-2, gamma=0.1, eps_min=1e-4)
    Z = np.zeros((n, n))
    with parallel.ParallelEngine(prob, subs, o, 2) as eng:
        st1 = eng.apply(Z, Z, True)
        eng.apply(Z, Z, False)
        with pytest.raises(RuntimeError):
            eng.jvp(st1, Z, Z)        # factors of a later evaluation
        bad = Z.copy()
        bad[3, 4] = np.nan
        st = eng.apply(bad, Z, False)  # non-finite local residuals end with a status, not a hang
        assert any(s != 0 for s in st.statuses)
