"""Helpers shared by the GPU tests: problem construction on both sides from the
same seeded inputs, and the error metric (relative infinity norm per field)."""
import numpy as np

from oracle import discretization as fd
from oracle import ras as oras
from paper_2411_00546_gb300 import inputs

FP64_TOL = 1e-10     # relative inf-norm per field, pure FP64 path
MIXED_TOL = 1e-8     # relative inf-norm per field, FP32-factor / FP64-refinement path


def rel_inf(a, b):
    """max|a - b| / max|b|: the relative infinity norm of one field, each field
    (y or p) on its own scale."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    diff = np.max(np.abs(a - b))
    if scale == 0.0:
        return diff
    return diff / scale


def oracle_problem(cfg, yd=None, f=None):
    yd = inputs.make_yd(cfg) if yd is None else yd
    return fd.Problem(cfg["n"], cfg["phi"], cfg["nu"], cfg["mu"], yd, f, kappa=cfg.get("kappa", 0.1))


def oracle_opts(cfg, **over):
    kw = dict(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"], eps0=cfg["eps0"],
              gamma=cfg["gamma"], eps_min=cfg["eps_min"])
    kw.update(over)
    return oras.Options(**kw)


def gpu_opts(cfg, precision, **over):
    from paper_2411_00546_gb300 import ras
    kw = dict(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"], eps0=cfg["eps0"],
              gamma=cfg["gamma"], eps_min=cfg["eps_min"], precision=precision, kappa=cfg.get("kappa", 0.1))
    kw.update(over)
    return ras.make_opts(**kw)


def gpu_problem(cfg, precision, yd=None, f=None, **over):
    import torch
    from paper_2411_00546_gb300 import ras
    yd = inputs.make_yd(cfg) if yd is None else yd
    n = cfg["n"]
    yd_t = torch.tensor(np.ascontiguousarray(yd), dtype=torch.float64, device="cuda")
    f_t = None if f is None else torch.tensor(np.ascontiguousarray(f), dtype=torch.float64, device="cuda")
    h = ras.ras_create(n, cfg["sx"], cfg["sy"], cfg["overlap"], cfg["phi"], cfg["nu"], cfg["mu"], yd_t, f_t,
                       gpu_opts(cfg, precision, **over))
    return h


def zeros(n):
    import torch
    return torch.zeros((n, n), dtype=torch.float64, device="cuda")


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
