"""Host-only parts of the serving API: the per-request memory estimate used
for admission (no GPU needed)."""
import pytest

from paper_2411_00546_gb300 import inputs

ras = pytest.importorskip("paper_2411_00546_gb300.ras")


def _d(n, b=64, overlap=8, **kw):
    s = -(-n // b)
    d = dict(n=n, sx=s, sy=s, overlap=overlap, phi=0, nu=1e-6, mu=1e-2)
    d.update(kw)
    return d


def _lib_or_skip():
    try:
        ras.lib()
    except (RuntimeError, OSError) as exc:
        pytest.skip("libras.so not built: %s" % exc)


def test_request_bytes_grow_with_size():
    """A request's own storage holds x, y_d, the GMRES right-hand side and
    iterate (7 n^2 doubles) plus its local factors and coefficients."""
    _lib_or_skip()
    prev = (0, 0)
    for n in (63, 127, 255, 511, 1023):
        slot, ws = ras.ras_server_request_bytes(_d(n))
        assert slot >= 7 * n * n * 8
        assert ws > prev[1] and slot > prev[0]
        prev = (slot, ws)


def test_mixed_precision_needs_less_storage():
    """FP32 local factors and solve scratch: less request storage and workspace."""
    _lib_or_skip()
    o64 = ras.make_opts(precision=ras.RAS_FP64)
    o32 = ras.make_opts(precision=ras.RAS_MIXED)
    d = _d(511)
    s32, w32 = ras.ras_server_request_bytes(d, o32)
    s64, w64 = ras.ras_server_request_bytes(d, o64)
    assert s32 < s64 and w32 < w64


def test_request_bytes_rejects_invalid_and_too_wide():
    _lib_or_skip()
    with pytest.raises(ras.RasError):
        ras.ras_server_request_bytes(_d(63, nu=-1.0))
    with pytest.raises(ras.RasError):
        ras.ras_server_request_bytes(dict(n=300, sx=1, sy=1, overlap=2, phi=0, nu=1e-4, mu=1e-3))   # 2 wx > 512


def test_uneven_batch_fits_the_serving_budget():
    """The uneven-batch workload's requests each fit a 150 GB budget many times over."""
    _lib_or_skip()
    o = ras.make_opts(precision=ras.RAS_MIXED)
    tot = sum(sum(ras.ras_server_request_bytes(c, o)) for c in inputs.uneven_batch())
    assert tot < 150e9
