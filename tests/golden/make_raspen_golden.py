"""Writes the stored oracle solves that the full-size parity tests compare with.

For each named workload it runs the oracle's RASPEN_eps (Alg. 2, with Alg. 3
and Alg. 4 spread over worker processes by oracle.parallel, identical to the
serial oracle) from x0 = 0 to convergence and stores, in
tests/golden/raspen_<name>.npz:

* Y, P: the final iterate (n x n, FP64);
* inner_its: the local Newton iteration counts of every evaluation of the
  RASPEN function (evaluations x subdomains), in subdomain order;
* gmres_its, norms, outer, status: the outer history;
* the workload's parameters, the worker count and the wall time.

It calls only oracle/ and the seeded input generator; nothing here comes from
the CUDA path. Usage: python tests/golden/make_raspen_golden.py [name ...]
(default: n1023), with an optional --workers N.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import decomposition as dd  # noqa: E402
from oracle import discretization as fd  # noqa: E402
from oracle import parallel  # noqa: E402
from oracle import ras as oras  # noqa: E402
from oracle import solvers  # noqa: E402
from paper_2411_00546_gb300 import inputs  # noqa: E402


def solve(name, workers=None):
    cfg = inputs.problem(name)
    n = cfg["n"]
    prob = fd.Problem(n, cfg["phi"], cfg["nu"], cfg["mu"], inputs.make_yd(cfg), kappa=cfg["kappa"])
    opts = oras.Options(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"], eps0=cfg["eps0"],
                        gamma=cfg["gamma"], eps_min=cfg["eps_min"])
    subs = dd.subdomains(n, cfg["sx"], cfg["sy"], cfg["overlap"])
    with parallel.ParallelEngine(prob, subs, opts, workers) as eng:
        t0 = time.perf_counter()
        r = solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"], opts, engine=eng)
        wall = time.perf_counter() - t0
        nw = eng.workers
    return cfg, r, wall, nw


def main(argv):
    workers = None
    if "--workers" in argv:
        k = argv.index("--workers")
        workers = int(argv[k + 1])
        argv = argv[:k] + argv[k + 2:]
    names = argv or ["n1023"]
    for name in names:
        cfg, r, wall, nw = solve(name, workers)
        path = os.path.join(HERE, "raspen_%s.npz" % name)
        np.savez_compressed(
            path, Y=r.Y, P=r.P, inner_its=np.array(r.inner_its, dtype=np.int32),
            gmres_its=np.array(r.gmres_its, dtype=np.int32), norms=np.array(r.norms),
            outer=r.outer, status=r.status, wall_s=wall, workers=nw,
            params=np.array(repr({k: v for k, v in cfg.items()})))
        print("%s: outer %d, gmres %s, local its per evaluation %s, %.1f s on %d workers -> %s"
              % (name, r.outer, r.gmres_its, [int(np.sum(i)) for i in r.inner_its], wall, nw, path))


if __name__ == "__main__":
    main(sys.argv[1:])
