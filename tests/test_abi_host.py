"""Host-side behaviour of the C ABI, without a GPU: every argument check that
include/ras.h promises runs before any device work, so these calls return
RAS_EINVAL here and leave the output handle NULL; the null-handle rules; and
the server's per-request memory estimate (host arithmetic only) against a
lower bound counted from the oracle's subdomain boxes."""
import ctypes
import os

import numpy as np
import pytest

from oracle import decomposition as dd
from paper_2411_00546_gb300 import ras

BUF = np.zeros(16, dtype=np.float64)
PTR = ctypes.c_void_p(BUF.ctypes.data)   # never dereferenced: the checks fail first


class _Lib:
    """libras.so, built on first use (collection needs no library)."""

    def __getattr__(self, name):
        if not os.path.exists(ras.LIB_PATH):
            from paper_2411_00546_gb300 import build
            build.build()
        return getattr(ras.lib(), name)


L = _Lib()


def _create(n, sx, sy, overlap, phi=0, nu=1e-5, mu=1e-3, yd=PTR, opts=None):
    out = ctypes.c_void_p(1)
    rc = L.ras_create(n, sx, sy, overlap, phi, nu, mu, yd, None,
                      ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("args,kw", [
    ((1, 1, 1, 0), {}),                      # n < 2
    ((10, 0, 1, 0), {}),                     # sx < 1
    ((10, 1, 11, 0), {}),                    # sy > n
    ((10, 1, 1, -1), {}),                    # negative overlap
    ((10, 1, 1, 0), {"phi": 3}),             # unknown phi
    ((10, 1, 1, 0), {"nu": 0.0}),            # nu <= 0
    ((10, 1, 1, 0), {"mu": float("nan")}),   # mu not finite
    ((10, 1, 1, 0), {"yd": None}),           # y_d NULL
    ((300, 1, 2, 2), {}),                    # block rows of 600 unknowns (> 512)
])
def test_create_rejects_invalid_arguments(args, kw):
    assert _create(*args, **kw) == (ras.RAS_EINVAL, None)


@pytest.mark.parametrize("field,value", [("eps_min", 0.0), ("eps0", 1e-9), ("gamma", 1.5), ("sigma", 0.5),
                                         ("gmres_restart", 31), ("precision", 7), ("jvp_ir", 9)])
def test_create_rejects_invalid_options(field, value):
    o = ras.make_opts(eps_min=1e-6)
    setattr(o, field, value)
    assert _create(10, 2, 2, 1, opts=o) == (ras.RAS_EINVAL, None)


def test_create3_rejects_bad_x3_split():
    for sz in (0, 11):
        out = ctypes.c_void_p(1)
        rc = L.ras_create3(10, 2, 2, sz, 1, 0, 1e-5, 1e-3, PTR, None, None, None, ctypes.byref(out))
        assert (rc, out.value) == (ras.RAS_EINVAL, None)


def test_null_handle_rules():
    assert L.ras_problem_dim(None) == ras.RAS_EINVAL
    assert L.ras_last_error(None) == b"null handle"
    L.ras_destroy(None)   # a no-op


def test_server_create_rejects_invalid_arguments():
    out = ctypes.c_void_p(1)
    assert L.ras_server_create(0, 4, None, None, ctypes.byref(out)) == ras.RAS_EINVAL
    assert out.value is None
    assert L.ras_server_create(1 << 30, 0, None, None, ctypes.byref(out)) == ras.RAS_EINVAL
    bad = ras.make_opts(gamma=0.0)
    assert L.ras_server_create(1 << 30, 4, ctypes.byref(bad), None, ctypes.byref(out)) == ras.RAS_EINVAL


def test_static_residual_rejects_sizes_before_device_work():
    args = (0, 1e-5, 1e-3, 0.1, 1e-6, PTR, PTR, PTR, None, PTR, PTR, PTR, None)
    assert L.ras_residual_static(1, *args) == ras.RAS_EINVAL
    assert L.ras_residual_static(ras.RAS_STATIC_MAX_N + 1, *args) == ras.RAS_EINVAL
    assert L.ras_residual_static(16, 0, 1e-5, 1e-3, 0.1, 1e-6, None, PTR, PTR, None, PTR, PTR, PTR,
                                 None) == ras.RAS_EINVAL


def _request_bytes(n, sx, sy, overlap, precision):
    d = ras.ras_problem_desc(n=n, sx=sx, sy=sy, overlap=overlap, phi=0, nu=1e-5, mu=1e-3)
    o = ras.make_opts(precision=precision)
    a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    rc = L.ras_server_request_bytes(ctypes.byref(d), ctypes.byref(o), ctypes.byref(a), ctypes.byref(b))
    return rc, a.value, b.value


@pytest.mark.parametrize("n,sx,sy,overlap", [(127, 4, 4, 2), (255, 8, 8, 4), (450, 10, 10, 2), (450, 2, 5, 2)])
def test_request_bytes_cover_the_factors_and_the_iterate(n, sx, sy, overlap):
    """What a request keeps between steps holds at least its iterate (y, p)
    and y_d in FP64 and one m x m block per grid line of every subdomain
    (m = 2 wx unknowns), in FP32 for mixed precision and FP64 otherwise."""
    lines = sum(s.wy * (2 * s.wx) ** 2 for s in dd.subdomains(n, sx, sy, overlap))
    for prec, es in ((ras.RAS_MIXED, 4), (ras.RAS_FP64, 8)):
        rc, slot, scratch = _request_bytes(n, sx, sy, overlap, prec)
        assert rc == ras.RAS_OK
        assert slot >= lines * es + 3 * n * n * 8
        assert scratch > 0
    assert _request_bytes(n, sx, sy, overlap, ras.RAS_MIXED)[1] < _request_bytes(n, sx, sy, overlap,
                                                                                  ras.RAS_FP64)[1]


def test_request_bytes_reject_invalid_and_too_wide_requests():
    assert _request_bytes(300, 1, 2, 2, ras.RAS_MIXED)[0] == ras.RAS_EINVAL
    assert _request_bytes(1, 1, 1, 0, ras.RAS_MIXED)[0] == ras.RAS_EINVAL
