"""Alg. 3 and Alg. 4 with the subdomains spread over worker processes.
Test infrastructure.

Alg. 3 computes the local corrections C_i(x) "in parallel": each depends only
on x. ParallelEngine gives each of its worker processes a fixed set of
subdomains (dealt largest first to the least loaded worker). A worker keeps
the local results of its subdomains (C_i, x^(i) and the factorisation of J_i
at x^(i)) between calls, so the Jacobian action of Alg. 4 runs where Alg. 3
left its factors. Grid vectors pass through shared memory. Every node of an
output is written by its one owner (restricted prolongation, sum_i tilde P_i
R_i = I), so the result does not depend on the number of workers and equals
the serial oracle's (oracle.ras.SerialEngine) value for value.

The arithmetic is the serial oracle's own: the workers call
oracle.ras.local_correction and oracle.ras.local_jvp unchanged. Processes are
started with the 'spawn' method, which is safe after CUDA has been initialised
in the parent.
"""
import multiprocessing as mp
import os
import time
import traceback
from multiprocessing import shared_memory

import numpy as np

from . import decomposition as dd
from . import discretization as fd
from . import ras as oras


class ParallelState:
    """What Alg. 2 reads from an evaluation of Alg. 3: F(x) and the local counts."""

    def __init__(self, Fy, Fp, iterations, statuses, eps_min, generation):
        self.Fy, self.Fp = Fy, Fp
        self.iterations = iterations
        self.statuses = statuses
        self.eps_min = eps_min
        self.generation = generation


_BLAS_ENV = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def _owned_pieces(sub, zy, zp):
    x0, _, y0, _ = sub.box
    ox0, ox1, oy0, oy1 = sub.owned
    return ((slice(oy0, oy1), slice(ox0, ox1)),
            zy[oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0], zp[oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0])


def _serve(conn, X, D, OUT, prob, subs, opts):
    locs = {}
    while True:
        cmd = conn.recv()
        c0 = time.process_time()
        try:
            if cmd[0] == "stop":
                return
            if cmd[0] == "apply":
                Y, P = X[0].copy(), X[1].copy()
                eps0 = opts.eps0 if cmd[1] else opts.eps_min
                locs = {}
                info = []
                for sub in subs:
                    loc = oras.local_correction(prob, Y, P, sub, eps0, opts.eps_min, opts, True)
                    cy, cp = fd.deinterleave(loc.C, sub.wx, sub.wy)
                    sl, oy, op = _owned_pieces(sub, cy, cp)
                    OUT[0][sl] = oy
                    OUT[1][sl] = op
                    locs[sub.index] = loc
                    info.append((sub.index, loc.newton.iterations, loc.newton.status))
                conn.send(("ok", (info, time.process_time() - c0)))
            elif cmd[0] == "jvp":
                for sub in subs:
                    zy, zp = oras.local_jvp(prob, locs[sub.index], opts.eps_min, D[0], D[1])
                    sl, oy, op = _owned_pieces(sub, zy, zp)
                    OUT[0][sl] = oy
                    OUT[1][sl] = op
                conn.send(("ok", (None, time.process_time() - c0)))
            else:
                conn.send(("err", "unknown command %r" % (cmd[0],)))
        except Exception:
            conn.send(("err", traceback.format_exc()))


def _worker(conn, names, n, prob_args, sub_args, opts_kw):
    shms = [shared_memory.SharedMemory(name=nm) for nm in names]
    try:
        views = [np.ndarray((2, n, n), dtype=np.float64, buffer=s.buf) for s in shms]
        prob = fd.Problem(*prob_args[:6], kappa=prob_args[6])
        opts = oras.Options(**opts_kw)
        subs = [dd.Subdomain(i, owned, box) for i, owned, box in sub_args]
        _serve(conn, *views, prob, subs, opts)
        del views
    finally:
        for s in shms:
            try:
                s.close()
            except BufferError:
                pass


def _deal(subs, workers):
    """Largest subdomain first, each to the worker with the fewest nodes so far."""
    load = [0] * workers
    parts = [[] for _ in range(workers)]
    for sub in sorted(subs, key=lambda s: (-s.wx * s.wy, s.index)):
        w = min(range(workers), key=lambda k: (load[k], k))
        parts[w].append(sub)
        load[w] += sub.wx * sub.wy
    return [p for p in parts if p]


class ParallelEngine:
    """Alg. 3 / Alg. 4 engine for oracle.solvers.raspen over worker processes."""

    def __init__(self, prob, subs, opts, workers=None):
        n = prob.n
        self.n = n
        self.eps_min = opts.eps_min
        self.nsub = len(subs)
        workers = max(1, min(int(workers or os.cpu_count() or 1), len(subs)))
        nbytes = 2 * n * n * 8
        self._shms = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(3)]
        self.X, self.D, self.OUT = (np.ndarray((2, n, n), dtype=np.float64, buffer=s.buf) for s in self._shms)
        ctx = mp.get_context("spawn")
        prob_args = (n, prob.phi_kind, prob.nu, prob.mu, prob.y_d, prob.f, prob.kappa)
        self._conns, self._procs = [], []
        self.generation = 0
        self.cpu_seconds = 0.0    # CPU time the workers spent in Alg. 3 / Alg. 4
        # one BLAS thread per worker process (the children read this at start)
        saved = {k: os.environ.get(k) for k in _BLAS_ENV}
        os.environ.update({k: "1" for k in _BLAS_ENV})
        try:
            for part in _deal(subs, workers):
                a, b = ctx.Pipe()
                pr = ctx.Process(target=_worker, daemon=True,
                                 args=(b, [s.name for s in self._shms], n, prob_args,
                                       [(s.index, s.owned, s.box) for s in part], dict(vars(opts))))
                pr.start()
                b.close()
                self._conns.append(a)
                self._procs.append(pr)
        except Exception:
            self.close()
            raise
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.workers = len(self._procs)

    def _call(self, cmd):
        for c in self._conns:
            c.send(cmd)
        out, errs = [], []
        for c in self._conns:
            tag, val = c.recv()
            if tag == "ok":
                out.append(val[0])
                self.cpu_seconds += val[1]
            else:
                errs.append(val)
        if errs:
            raise RuntimeError("oracle worker failed:\n" + errs[0])
        return out

    def apply(self, Y, P, continuation):
        self.X[0] = Y
        self.X[1] = P
        self.OUT.fill(0.0)
        infos = self._call(("apply", bool(continuation)))
        its = [0] * self.nsub
        sts = [0] * self.nsub
        for info in infos:
            for i, k, st in info:
                its[i] = k
                sts[i] = st
        self.generation += 1
        return ParallelState(self.OUT[0].copy(), self.OUT[1].copy(), its, sts, self.eps_min, self.generation)

    def jvp(self, state, dY, dP):
        if state.generation != self.generation:
            raise RuntimeError("the workers hold the factors of a later evaluation")
        self.D[0] = dY
        self.D[1] = dP
        self.OUT.fill(0.0)
        self._call(("jvp",))
        return self.OUT[0].copy(), self.OUT[1].copy()

    def close(self):
        for c in getattr(self, "_conns", []):
            try:
                c.send(("stop",))
            except (OSError, BrokenPipeError):
                pass
        for pr in getattr(self, "_procs", []):
            pr.join(timeout=30)
            if pr.is_alive():
                pr.kill()
                pr.join()
        self._conns, self._procs = [], []
        self.X = self.D = self.OUT = None
        for s in getattr(self, "_shms", []):
            s.close()
            try:
                s.unlink()
            except FileNotFoundError:
                pass
        self._shms = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
