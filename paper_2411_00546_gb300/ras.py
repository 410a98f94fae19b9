"""Thin ctypes binding of libras.so (include/ras.h), with the C ABI's names.

Argument marshalling only: every step of the solver runs in the CUDA library.
Grid functions are torch CUDA float64 tensors of n*n elements (any shape,
contiguous, row-major with the x1 index fastest). Host buffers for
ras_solve_host are CPU float64 tensors (pinned for speed). There is no CPU
fallback: if libras.so is missing, loading fails with an error.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libras.so")

RAS_OK = 0
RAS_OK_FLOOR = 1
RAS_EINVAL = -1
RAS_ENOMEM = -2
RAS_ENOCONV = -3
RAS_ESINGULAR = -5
RAS_ENONFINITE = -6
RAS_ETIMEOUT = -7
RAS_ENOTIMPL = -8
RAS_ECUDA = -9
RAS_ESTATE = -10

RAS_PHI_CUBIC = 0
RAS_PHI_EXP = 1
RAS_PHI_KAPPA = 2

RAS_FP64 = 0
RAS_MIXED = 1

RAS_METHOD_RASPEN = 0
RAS_METHOD_NEWTON_RAS = 1
RAS_METHOD_NEWTON = 2


class ras_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("sigma", ctypes.c_double),
                ("eps0", ctypes.c_double), ("gamma", ctypes.c_double), ("eps_min", ctypes.c_double),
                ("kmax_outer_raspen", ctypes.c_int), ("kmax_outer_newton", ctypes.c_int),
                ("kmax_inner", ctypes.c_int), ("max_halvings", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("gmres_rtol", ctypes.c_double), ("floor_factor", ctypes.c_double),
                ("precision", ctypes.c_int), ("ir_max", ctypes.c_int), ("ir_rtol", ctypes.c_double),
                ("kappa", ctypes.c_double), ("jvp_ir", ctypes.c_int), ("wait_test", ctypes.c_int)]


class ras_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
                ("evaluations", ctypes.c_int), ("inner_its_max", ctypes.c_int),
                ("inner_its_sum", ctypes.c_longlong), ("halvings", ctypes.c_int),
                ("exhausted", ctypes.c_int), ("local_failures", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("eps_final", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ras_problem_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("sx", ctypes.c_int), ("sy", ctypes.c_int), ("overlap", ctypes.c_int),
                ("phi", ctypes.c_int), ("nu", ctypes.c_double), ("mu", ctypes.c_double),
                ("y_d", ctypes.c_void_p), ("f", ctypes.c_void_p)]


class ras_state(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("k", ctypes.c_int), ("eps", ctypes.c_double), ("res0", ctypes.c_double),
                ("stop", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


RAS_NTILE = 5
RAS_TUNE_MAX = 8
RAS_VEC_BLOCKS_MAX = 608


class ras_tuning(ctypes.Structure):
    _fields_ = [("factor_wide_max", ctypes.c_int * RAS_NTILE), ("solve_ctas_per_sm", ctypes.c_int),
                ("vec_blocks", ctypes.c_int)]

    def as_dict(self):
        return {"factor_wide_max": list(self.factor_wide_max), "solve_ctas_per_sm": self.solve_ctas_per_sm,
                "vec_blocks": self.vec_blocks}


class ras_tune_report(ctypes.Structure):
    _fields_ = [("factor_count", (ctypes.c_int * RAS_TUNE_MAX) * RAS_NTILE),
                ("factor_ms", ((ctypes.c_double * 2) * RAS_TUNE_MAX) * RAS_NTILE),
                ("solve_ctas_per_sm", ctypes.c_int * RAS_TUNE_MAX), ("solve_ms", ctypes.c_double * RAS_TUNE_MAX),
                ("vec_blocks", ctypes.c_int * RAS_TUNE_MAX), ("vec_ms", ctypes.c_double * RAS_TUNE_MAX)]

    def as_dict(self):
        """Timed candidates only (entries with a zero count are unused)."""
        fac = {}
        for c in range(RAS_NTILE):
            rows = [(self.factor_count[c][i], self.factor_ms[c][i][0], self.factor_ms[c][i][1])
                    for i in range(RAS_TUNE_MAX) if self.factor_count[c][i] > 0]
            if rows:
                fac[32 * (c + 1)] = rows
        solve = [(self.solve_ctas_per_sm[i], self.solve_ms[i]) for i in range(RAS_TUNE_MAX)
                 if self.solve_ctas_per_sm[i] > 0]
        vec = [(self.vec_blocks[i], self.vec_ms[i]) for i in range(RAS_TUNE_MAX) if self.vec_blocks[i] > 0]
        return {"factor": fac, "solve": solve, "vectors": vec}


class RasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ras error %d: %s" % (code, msg))
        self.code = code


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGS = {
    "ras_default_opts": (_I, [ctypes.POINTER(ras_opts)]),
    "ras_create": (_I, [_I, _I, _I, _I, _I, _D, _D, _P, _P, ctypes.POINTER(ras_opts), _P, ctypes.POINTER(_P)]),
    "ras_create3": (_I, [_I, _I, _I, _I, _I, _I, _D, _D, _P, _P, ctypes.POINTER(ras_opts), _P,
                         ctypes.POINTER(_P)]),
    "ras_problem_dim": (_I, [_P]),
    "ras_batch_create": (_I, [_I, ctypes.POINTER(ras_problem_desc), ctypes.POINTER(ras_opts), _P,
                              ctypes.POINTER(_P)]),
    "ras_problem_count": (_I, [_P]),
    "ras_batch_raspen_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(ras_stats)]),
    "ras_set_eps": (_I, [_P, _D]),
    "ras_set_opts": (_I, [_P, ctypes.POINTER(ras_opts)]),
    "ras_set_data": (_I, [_P, _P, _P]),
    "ras_residual": (_I, [_P, _P, _P, _D, _P, _P, ctypes.POINTER(_D)]),
    "ras_apply": (_I, [_P, _P, _P, _I, _P, _P, ctypes.POINTER(ras_stats)]),
    "ras_jvp": (_I, [_P, _P, _P, _P, _P]),
    "ras_precondition": (_I, [_P, _P, _P, _D, _P, _P, _P, _P]),
    "ras_raspen_solve": (_I, [_P, _P, _P, ctypes.POINTER(ras_stats)]),
    "ras_newton_ras_solve": (_I, [_P, _P, _P, ctypes.POINTER(ras_stats)]),
    "ras_newton_solve": (_I, [_P, _P, _P, ctypes.POINTER(ras_stats)]),
    "ras_get_state": (_I, [_P, ctypes.POINTER(ras_state)]),
    "ras_set_state": (_I, [_P, ctypes.POINTER(ras_state)]),
    "ras_use_graphs": (_I, [_P, _I]),
    "ras_manufacture": (_I, [_P, _P, _D, _P, _P]),
    "ras_autotune": (_I, [_P, ctypes.POINTER(ras_tuning), ctypes.POINTER(ras_tune_report)]),
    "ras_get_tuning": (_I, [_P, ctypes.POINTER(ras_tuning)]),
    "ras_set_tuning": (_I, [_P, ctypes.POINTER(ras_tuning)]),
    "ras_solve_host": (_I, [_P, _I, _P, _P, _P, ctypes.POINTER(ras_stats)]),
    "ras_local_iterations": (_I, [_P, ctypes.POINTER(_I), _I]),
    "ras_subdomain_count": (_I, [_P]),
    "ras_device_bytes": (ctypes.c_size_t, [_P]),
    "ras_last_error": (ctypes.c_char_p, [_P]),
    "ras_destroy": (None, [_P]),
    "ras_launch_count": (ctypes.c_longlong, []),
    "ras_profile": (_I, [_P, _I]),
    "ras_profile_read": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D)]),
    "ras_residual_static": (_I, [_I, _I, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ras_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(ras_opts), _P, ctypes.POINTER(_P)]),
    "ras_server_request_bytes": (_I, [ctypes.POINTER(ras_problem_desc), ctypes.POINTER(ras_opts),
                                      ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "ras_server_submit": (_I, [_P, ctypes.POINTER(ras_problem_desc), ctypes.POINTER(ctypes.c_longlong)]),
    "ras_server_step": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ras_server_counts": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ras_server_finished_ids": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), _I]),
    "ras_server_fetch": (_I, [_P, ctypes.c_longlong, _P, _P, ctypes.POINTER(ras_stats)]),
    "ras_server_cancel": (_I, [_P, ctypes.c_longlong]),
    "ras_server_use_graphs": (_I, [_P, _I]),
    "ras_server_device_bytes": (ctypes.c_size_t, [_P]),
    "ras_server_last_error": (ctypes.c_char_p, [_P]),
    "ras_server_destroy": (None, [_P]),
}

RAS_STATIC_MAX_N = 8192

RAS_K_NAMES = ["init", "factor", "direction", "linesearch", "jvp", "precond", "residual", "krylov", "other"]

_lib = None


def lib():
    """Load libras.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libras.so not found at %s; build it with __graft_entry__.build() "
                               "or python -m paper_2411_00546_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t, n=None, device=True):
    if t is None:
        return None
    if device and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError("expected a CPU tensor")
    import torch
    if t.dtype != torch.float64:
        raise ValueError("expected float64")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """Opaque ras_problem* plus the grid size, for argument checks (nn: grid
    nodes, n^2 on the square, n^3 on the cube)."""

    def __init__(self, ptr, n, dim=2):
        self.ptr = ptr
        self.n = n
        self.dim = dim
        self.nn = None if n is None else n ** dim

    def _check(self, rc, ok=(RAS_OK, RAS_OK_FLOOR)):
        if rc not in ok:
            raise RasError(rc, ras_last_error(self))
        return rc


def ras_default_opts():
    o = ras_opts()
    lib().ras_default_opts(ctypes.byref(o))
    return o


def ras_create(n, sx, sy, overlap, phi, nu, mu, y_d, f=None, opts=None, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    rc = lib().ras_create(n, sx, sy, overlap, phi, nu, mu, _ptr(y_d, n * n), _ptr(f, n * n),
                          ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(stream),
                          ctypes.byref(out))
    if rc != RAS_OK:
        raise RasError(rc, "ras_create failed")
    return Handle(out, n)


def ras_create3(n, sx, sy, sz, overlap, phi, nu, mu, y_d, f=None, opts=None, stream=None):
    """A problem on the n x n x n cube (7-point stencil), sx x sy x sz boxes;
    y_d, f: CUDA float64 tensors of n^3 entries (x1 fastest)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    nn = n ** 3
    rc = lib().ras_create3(n, sx, sy, sz, overlap, phi, nu, mu, _ptr(y_d, nn), _ptr(f, nn),
                           ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(stream),
                           ctypes.byref(out))
    if rc != RAS_OK:
        raise RasError(rc, "ras_create3 failed")
    return Handle(out, n, 3)


def ras_problem_dim(h):
    return lib().ras_problem_dim(h.ptr)


class BatchHandle(Handle):
    """Handle of a batch: ns = grid sizes of its problems."""

    def __init__(self, ptr, ns):
        super().__init__(ptr, None)
        self.ns = list(ns)


def ras_batch_create(problems, opts=None, stream=None):
    """problems: list of dicts with n, sx, sy, overlap, phi, nu, mu, y_d (CUDA
    float64 tensor, n*n) and optionally f."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    arr = (ras_problem_desc * len(problems))()
    for k, d in enumerate(problems):
        n = d["n"]
        arr[k].n, arr[k].sx, arr[k].sy, arr[k].overlap, arr[k].phi = n, d["sx"], d["sy"], d["overlap"], d["phi"]
        arr[k].nu, arr[k].mu = d["nu"], d["mu"]
        arr[k].y_d = _ptr(d["y_d"], n * n)
        arr[k].f = _ptr(d.get("f"), n * n)
    out = ctypes.c_void_p()
    rc = lib().ras_batch_create(len(problems), arr, ctypes.byref(opts) if opts is not None else None,
                                ctypes.c_void_p(stream), ctypes.byref(out))
    if rc != RAS_OK:
        raise RasError(rc, "ras_batch_create failed")
    return BatchHandle(out, [d["n"] for d in problems])


def ras_problem_count(h):
    return lib().ras_problem_count(h.ptr)


def ras_batch_raspen_solve(h, ys, ps, check=True):
    """Solve every problem of the batch; ys, ps: lists of CUDA tensors."""
    k = len(h.ns)
    Y = (_P * k)(*[_ptr(y, n * n) for y, n in zip(ys, h.ns)])
    Pp = (_P * k)(*[_ptr(p, n * n) for p, n in zip(ps, h.ns)])
    st = (ras_stats * k)()
    rc = lib().ras_batch_raspen_solve(h.ptr, Y, Pp, st)
    if check:
        h._check(rc)
    return rc, list(st)


def ras_set_eps(h, eps_min):
    return h._check(lib().ras_set_eps(h.ptr, eps_min))


def ras_set_opts(h, opts):
    return h._check(lib().ras_set_opts(h.ptr, ctypes.byref(opts)))


def ras_set_data(h, y_d, f=None):
    nn = h.nn
    return h._check(lib().ras_set_data(h.ptr, _ptr(y_d, nn), _ptr(f, nn)))


def ras_residual(h, y, p, eps, Fy=None, Fp=None):
    nn = h.nn
    nrm = ctypes.c_double()
    h._check(lib().ras_residual(h.ptr, _ptr(y, nn), _ptr(p, nn), eps, _ptr(Fy, nn), _ptr(Fp, nn),
                                ctypes.byref(nrm)))
    return nrm.value


def ras_apply(h, y, p, continuation, Fy, Fp, check=True):
    nn = h.nn
    st = ras_stats()
    rc = lib().ras_apply(h.ptr, _ptr(y, nn), _ptr(p, nn), int(continuation), _ptr(Fy, nn), _ptr(Fp, nn),
                         ctypes.byref(st))
    if check:
        h._check(rc)
    return rc, st


def ras_jvp(h, dy, dp, oy, op):
    nn = h.nn
    return h._check(lib().ras_jvp(h.ptr, _ptr(dy, nn), _ptr(dp, nn), _ptr(oy, nn), _ptr(op, nn)))


def ras_precondition(h, y, p, eps, ry, rp, zy, zp):
    nn = h.nn
    return h._check(lib().ras_precondition(h.ptr, _ptr(y, nn), _ptr(p, nn), eps, _ptr(ry, nn), _ptr(rp, nn),
                                           _ptr(zy, nn), _ptr(zp, nn)))


def ras_raspen_solve(h, y, p, check=True):
    nn = h.nn
    st = ras_stats()
    rc = lib().ras_raspen_solve(h.ptr, _ptr(y, nn), _ptr(p, nn), ctypes.byref(st))
    if check:
        h._check(rc)
    return rc, st


def ras_newton_ras_solve(h, y, p, check=True):
    nn = h.nn
    st = ras_stats()
    rc = lib().ras_newton_ras_solve(h.ptr, _ptr(y, nn), _ptr(p, nn), ctypes.byref(st))
    if check:
        h._check(rc)
    return rc, st


def ras_newton_solve(h, y, p, check=True):
    nn = h.nn
    st = ras_stats()
    rc = lib().ras_newton_solve(h.ptr, _ptr(y, nn), _ptr(p, nn), ctypes.byref(st))
    if check:
        h._check(rc)
    return rc, st


def ras_get_state(h):
    st = ras_state()
    h._check(lib().ras_get_state(h.ptr, ctypes.byref(st)))
    return st


def ras_set_state(h, st):
    return h._check(lib().ras_set_state(h.ptr, ctypes.byref(st)))


def ras_manufacture(h, pbar, eps=1e-15, y_out=None, yd_out=None):
    """Sec. 4's manufactured solution for the adjoint pbar: sets the handle's
    y_d and writes ybar / y_d into y_out / yd_out (device tensors, optional)."""
    nn = h.nn
    return h._check(lib().ras_manufacture(h.ptr, _ptr(pbar, nn), float(eps), _ptr(y_out, nn), _ptr(yd_out, nn)))


def ras_use_graphs(h, enable):
    """CUDA-graph execution of the GMRES restart cycles on (default) or off."""
    return h._check(lib().ras_use_graphs(h.ptr, 1 if enable else 0))


def ras_autotune(h):
    """Time the launch-shape candidates on h's subdomains and install the
    fastest; returns (ras_tuning, ras_tune_report)."""
    t, rep = ras_tuning(), ras_tune_report()
    h._check(lib().ras_autotune(h.ptr, ctypes.byref(t), ctypes.byref(rep)))
    return t, rep


def ras_get_tuning(h):
    t = ras_tuning()
    h._check(lib().ras_get_tuning(h.ptr, ctypes.byref(t)))
    return t


def ras_set_tuning(h, t, check=True):
    rc = lib().ras_set_tuning(h.ptr, ctypes.byref(t))
    if check:
        h._check(rc)
    return rc


def make_tuning(factor_wide_max=(-1,) * RAS_NTILE, solve_ctas_per_sm=0, vec_blocks=RAS_VEC_BLOCKS_MAX):
    t = ras_tuning()
    for c, v in enumerate(factor_wide_max):
        t.factor_wide_max[c] = int(v)
    t.solve_ctas_per_sm = int(solve_ctas_per_sm)
    t.vec_blocks = int(vec_blocks)
    return t


def ras_solve_host(h, method, y_d_host, y_host, p_host, check=True):
    nn = h.nn
    st = ras_stats()
    rc = lib().ras_solve_host(h.ptr, int(method), _ptr(y_d_host, nn, device=False),
                              _ptr(y_host, nn, device=False), _ptr(p_host, nn, device=False),
                              ctypes.byref(st))
    if check:
        h._check(rc)
    return rc, st


def ras_local_iterations(h):
    k = ras_subdomain_count(h)
    buf = (ctypes.c_int * k)()
    got = lib().ras_local_iterations(h.ptr, buf, k)
    return list(buf)[:got]


def ras_subdomain_count(h):
    return lib().ras_subdomain_count(h.ptr)


def ras_device_bytes(h):
    return lib().ras_device_bytes(h.ptr)


def ras_last_error(h):
    r = lib().ras_last_error(h.ptr)
    return r.decode() if r else ""


def ras_destroy(h):
    if h.ptr:
        lib().ras_destroy(h.ptr)
        h.ptr = None


def ras_launch_count():
    return lib().ras_launch_count()


def ras_profile(h, enable):
    return h._check(lib().ras_profile(h.ptr, int(enable)))


def ras_profile_read(h, kind):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    w = ctypes.c_double()
    h._check(lib().ras_profile_read(h.ptr, int(kind), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return ms.value, n.value, w.value


def ras_profile_all(h):
    return {name: ras_profile_read(h, k) for k, name in enumerate(RAS_K_NAMES)}


def ras_residual_static(n, phi, nu, mu, kappa, eps, y, p, y_d, f=None, Fy=None, Fp=None, norm_dev=None,
                        stream=None):
    """F(x, eps) and its norm with no device allocation (for callers that
    cannot allocate, see include/ras.h). norm_dev: 1-element CUDA float64
    tensor or None. Only enqueues work on `stream`."""
    if n > RAS_STATIC_MAX_N:
        raise RasError(RAS_EINVAL, "n=%d exceeds RAS_STATIC_MAX_N=%d" % (n, RAS_STATIC_MAX_N))
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    nn = n * n
    rc = lib().ras_residual_static(n, phi, nu, mu, kappa, eps, _ptr(y, nn), _ptr(p, nn), _ptr(y_d, nn),
                                   _ptr(f, nn), _ptr(Fy, nn), _ptr(Fp, nn), _ptr(norm_dev, 1),
                                   ctypes.c_void_p(stream))
    if rc != RAS_OK:
        raise RasError(rc, "ras_residual_static rejected its arguments (n=%d, limit %d)" % (n, RAS_STATIC_MAX_N))
    return rc


def make_opts(**kw):
    """ras_default_opts() with fields overridden by keyword."""
    o = ras_default_opts()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------ serving

def _host_ptr(a, n):
    """Pointer to a host float64 array of n elements (numpy array or CPU tensor)."""
    import numpy as np
    if hasattr(a, "is_cuda"):
        if a.is_cuda:
            raise ValueError("expected host data")
        a = a.numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError("expected %d elements, got %d" % (n, a.size))
    return a, ctypes.c_void_p(a.ctypes.data)


def _desc(d, host):
    """ras_problem_desc from a dict (n, sx, sy, overlap, phi, nu, mu, y_d[, f]);
    returns the struct and the arrays it points to (keep them alive)."""
    n = d["n"]
    c = ras_problem_desc()
    c.n, c.sx, c.sy, c.overlap, c.phi = n, d["sx"], d["sy"], d["overlap"], d["phi"]
    c.nu, c.mu = d["nu"], d["mu"]
    keep = []
    if host:
        for key in ("y_d", "f"):
            if d.get(key) is not None:
                arr, ptr = _host_ptr(d[key], n * n)
                keep.append(arr)
                setattr(c, key, ptr)
    else:
        c.y_d = _ptr(d["y_d"], n * n)
        c.f = _ptr(d.get("f"), n * n)
    return c, keep


class Server:
    """Opaque ras_server* (continuous batching of RASPEN solves)."""

    def __init__(self, ptr):
        self.ptr = ptr
        self.sizes = {}

    def _check(self, rc, ok=(RAS_OK,)):
        if rc not in ok:
            raise RasError(rc, lib().ras_server_last_error(self.ptr).decode())
        return rc


def ras_server_create(hbm_budget, max_active, opts=None, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    rc = lib().ras_server_create(int(hbm_budget), int(max_active), ctypes.byref(opts) if opts is not None else None,
                                 ctypes.c_void_p(stream), ctypes.byref(out))
    if rc != RAS_OK:
        raise RasError(rc, "ras_server_create rejected its arguments")
    return Server(out)


def ras_server_request_bytes(d, opts=None):
    """(slot_bytes, workspace_bytes) estimate of one request (host only)."""
    c, _ = _desc(dict(d, y_d=None, f=None), host=True)
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    rc = lib().ras_server_request_bytes(ctypes.byref(c), ctypes.byref(opts) if opts is not None else None,
                                        ctypes.byref(a), ctypes.byref(b))
    if rc != RAS_OK:
        raise RasError(rc, "invalid problem description")
    return a.value, b.value


def ras_server_submit(s, d):
    """Queue one request; d: dict with n, sx, sy, overlap, phi, nu, mu and host
    y_d (and optional f) arrays. Returns its id."""
    c, keep = _desc(d, host=True)
    rid = ctypes.c_longlong()
    s._check(lib().ras_server_submit(s.ptr, ctypes.byref(c), ctypes.byref(rid)))
    s.sizes[rid.value] = d["n"]
    del keep
    return rid.value


def ras_server_step(s):
    """Admission and one outer iteration; returns (admitted, finished_now)."""
    a, f = _I(), _I()
    s._check(lib().ras_server_step(s.ptr, ctypes.byref(a), ctypes.byref(f)))
    return a.value, f.value


def ras_server_counts(s):
    p, a, f = _I(), _I(), _I()
    s._check(lib().ras_server_counts(s.ptr, ctypes.byref(p), ctypes.byref(a), ctypes.byref(f)))
    return p.value, a.value, f.value


def ras_server_finished_ids(s, cap=4096):
    ids = (ctypes.c_longlong * cap)()
    k = lib().ras_server_finished_ids(s.ptr, ids, cap)
    if k < 0:
        s._check(k)
    return list(ids[:k])


def ras_server_fetch(s, rid):
    """Result of a finished request: (status, y, p, stats) with host float64
    numpy arrays of shape (n, n)."""
    import numpy as np
    n = s.sizes.pop(rid)
    y = np.empty((n, n), dtype=np.float64)
    p = np.empty((n, n), dtype=np.float64)
    st = ras_stats()
    rc = lib().ras_server_fetch(s.ptr, rid, ctypes.c_void_p(y.ctypes.data), ctypes.c_void_p(p.ctypes.data),
                                ctypes.byref(st))
    if rc == RAS_EINVAL:
        raise RasError(rc, lib().ras_server_last_error(s.ptr).decode())
    return rc, y, p, st


def ras_server_cancel(s, rid):
    s._check(lib().ras_server_cancel(s.ptr, rid))
    s.sizes.pop(rid, None)


def ras_server_use_graphs(s, enable):
    s._check(lib().ras_server_use_graphs(s.ptr, 1 if enable else 0))


def ras_server_device_bytes(s):
    return lib().ras_server_device_bytes(s.ptr)


def ras_server_destroy(s):
    if s.ptr:
        lib().ras_server_destroy(s.ptr)
        s.ptr = None
