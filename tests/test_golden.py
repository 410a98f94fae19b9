"""The stored oracle solves under tests/golden (written by
tests/golden/make_raspen_golden.py, which calls only the oracle) against what
they claim to be: the parameters of the named workload, a converged RASPEN_eps
history (one more evaluation than outer steps, statuses OK), and a final
iterate at which the oracle's own residual F (Sec. 3.3) is at the solve's
accuracy."""
import ast
import glob
import os

import numpy as np
import pytest

from oracle import discretization as fd
from paper_2411_00546_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(glob.glob(os.path.join(HERE, "raspen_*.npz")))


def test_goldens_exist():
    names = [os.path.basename(f)[len("raspen_"):-len(".npz")] for f in FILES]
    assert "n1023" in names and "n1023_active" in names


@pytest.mark.parametrize("path", FILES, ids=os.path.basename)
def test_stored_solve_is_a_converged_oracle_solve(path):
    name = os.path.basename(path)[len("raspen_"):-len(".npz")]
    g = np.load(path)
    cfg = inputs.problem(name)
    assert ast.literal_eval(str(g["params"])) == cfg
    outer = int(g["outer"])
    assert int(g["status"]) == 0
    assert g["inner_its"].shape == (outer + 1, cfg["sx"] * cfg["sy"])
    assert g["gmres_its"].shape == (outer,) and np.all(g["gmres_its"] > 0)
    norms = g["norms"]
    assert norms[-1] <= cfg["tol"] * norms[0]        # Alg. 2 is undamped: the history need not fall monotonically
    n = cfg["n"]
    prob = fd.Problem(n, cfg["phi"], cfg["nu"], cfg["mu"], inputs.make_yd(cfg))
    Fy, Fp = fd.residual(prob, g["Y"], g["P"], cfg["eps_min"])
    F0 = np.sqrt(np.sum(prob.y_d ** 2))          # ||F(0)||: f = 0, only F_p = y_d
    res = np.sqrt(np.sum(Fy ** 2) + np.sum(Fp ** 2))
    # the local solves stop at inner_tol, so F itself is at that level, not at tol
    assert res <= 10 * cfg["inner_tol"] * F0, (res, F0)
