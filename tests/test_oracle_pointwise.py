"""Pins of the oracle's pointwise functions against the paper's definitions and
Lemma 5, evaluated independently in 50-digit arithmetic (mpmath)."""
import numpy as np
import pytest

from oracle import pointwise as pw

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50

EPSS = [1.0, 1e-2, 1e-6, 1e-10, 1e-15]
XS = np.concatenate([np.linspace(-5, 5, 101), [-1e3, -37.5, -1.0, -1e-9, 0.0, 1e-9, 1.0, 2.5, 1e3]])


def _P_mp(x, eps):
    """The smoothed projection exactly as first defined in Sec. 3.1 (difference
    of the two shifted square roots), in 50 digits."""
    x = mpmath.mpf(x)
    e = mpmath.mpf(eps)
    return (mpmath.sqrt((x + 1) ** 2 + e) - mpmath.sqrt((x - 1) ** 2 + e)) / 2


@pytest.mark.parametrize("eps", EPSS)
def test_P_eps_matches_definition_in_high_precision(eps):
    got = pw.P_eps(XS, eps)
    for x, g in zip(XS, got):
        ref = float(_P_mp(x, eps))
        assert abs(g - ref) <= 8 * 2.0 ** -53 * abs(ref) + 1e-300, (x, eps, g, ref)


@pytest.mark.parametrize("eps", EPSS)
def test_dP_eps_is_derivative_of_P_eps(eps):
    got = pw.dP_eps(XS, eps)
    for x, g in zip(XS, got):
        ref = float(mpmath.diff(lambda t: _P_mp(t, eps), mpmath.mpf(x)))
        # absolute bound: the printed difference of two quotients loses relative
        # accuracy where both are near +-1, never absolute accuracy
        assert abs(g - ref) <= 4e-16, (x, eps, g, ref)


def _rel_ok(got, ref, ulps):
    return abs(got - ref) <= ulps * 2.0 ** -53 * abs(ref) + 1e-300


@pytest.mark.parametrize("eps", EPSS)
def test_P_eps_minus_id_full_relative_accuracy(eps):
    """P_eps(x) - x against the 50-digit definition, to a few ulp of itself
    (the printed difference p + mu P_eps(-p/mu) misses this by 2^-53/eps)."""
    got = pw.P_eps_minus_id(XS, eps)
    for x, g in zip(XS, got):
        ref = float(_P_mp(x, eps) - mpmath.mpf(x))
        assert _rel_ok(g, ref, 16), (x, eps, g, ref)


@pytest.mark.parametrize("eps", EPSS)
def test_one_minus_dP_eps_full_relative_accuracy(eps):
    """1 - P_eps'(x) against 1 minus the 50-digit derivative of the definition."""
    got = pw.one_minus_dP_eps(XS, eps)
    for x, g in zip(XS, got):
        ref = float(1 - mpmath.diff(lambda t: _P_mp(t, eps), mpmath.mpf(x)))
        assert _rel_ok(g, ref, 16), (x, eps, g, ref)


@pytest.mark.parametrize("eps", [1e-2, 1e-6, 1e-15])
@pytest.mark.parametrize("nu,mu", [(1e-4, 1e-3), (1e-6, 1e-2), (1e-6, 1.0)])
def test_u_eps_full_relative_accuracy(eps, nu, mu):
    """u = -(1/nu)(p + mu P_eps(-p/mu)) (Sec. 3.2) in 50 digits: the oracle's
    control keeps a few ulp of relative accuracy also where |p| < mu, where it
    is O(eps) and drives the state alone. The reference is taken at
    p' = -mu fl(-p/mu), within one rounding of p: near |p| = mu, u is
    ill-conditioned in p (condition ~ 1/|1 - |p|/mu|), which no evaluation
    from FP64 data escapes."""
    ps = mu * np.concatenate([np.linspace(-3, 3, 61), [-1e-7, 1e-7, 0.35, -0.999, 1.0000001]])
    got = pw.u_eps(ps, eps, nu, mu)
    for p, g in zip(ps, got):
        X = mpmath.mpf(float(-p / mu))
        M, N, E = (mpmath.mpf(float(v)) for v in (mu, nu, eps))
        P = -M * X
        ref = float(-(P + M * _P_mp(-P / M, E)) / N)
        assert _rel_ok(g, ref, 24), (p, eps, g, ref)


@pytest.mark.parametrize("eps", EPSS)
def test_lemma5_properties(eps):
    x = np.linspace(-10, 10, 20001)
    P = pw.P_eps(x, eps)
    dP = pw.dP_eps(x, eps)
    # range [-1, 1], odd, strictly increasing (Lemma 5 (i))
    assert np.all(np.abs(P) <= 1.0 + 4 * 2.0 ** -53)  # exact range [-1, 1]; rounding may add an ulp
    np.testing.assert_array_equal(P, -pw.P_eps(-x, eps))
    assert np.all(np.diff(P) > 0) or eps < 1e-8  # tiny eps: flat within rounding far out
    # P' in (0, 1/sqrt(1+eps)] with the maximum at 0 (Lemma 5 (ii))
    # positive; the printed difference of quotients has absolute rounding ~1e-16
    assert np.all(dP > -4e-16)
    assert np.all(dP[np.abs(x) < 1] > 0)
    assert np.all(dP <= 1.0 / np.sqrt(1.0 + eps) * (1 + 4e-16))
    assert abs(pw.dP_eps(0.0, eps) - 1.0 / np.sqrt(1.0 + eps)) <= 4e-16
    # |proj - P_eps| <= sqrt(eps) (Lemma 5 (iv))
    assert np.all(np.abs(pw.proj(x) - P) <= np.sqrt(eps) * (1 + 1e-12) + 1e-16)


def test_lemma5_limits_as_eps_vanishes():
    eps = 1e-14
    x = np.array([-3.0, -0.5, 0.0, 0.7, 2.0])
    np.testing.assert_allclose(pw.P_eps(x, eps), pw.proj(x), atol=1e-7)
    np.testing.assert_allclose(pw.dP_eps(np.array([-0.5, 0.3, 1.0, -1.0, 1.5, -4.0]), eps),
                               [1.0, 1.0, 0.5, 0.5, 0.0, 0.0], atol=1e-7)


@pytest.mark.parametrize("nu,mu", [(1e-4, 1e-3), (1e-6, 1e-2), (1.0, 0.3)])
def test_u_eps_tends_to_soft_threshold(nu, mu):
    """As eps -> 0, u_eps(p) -> -(1/nu) sign(p) max(|p| - mu, 0) (the reduced
    non-smooth system, Sec. 2) within (mu/nu) sqrt(eps) (Lemma 5 (iv))."""
    p = np.linspace(-5 * mu, 5 * mu, 1001)
    soft = -(1.0 / nu) * np.sign(p) * np.maximum(np.abs(p) - mu, 0.0)
    np.testing.assert_allclose(pw.u_limit(p, nu, mu), soft, atol=1e-12 * mu / nu)
    for eps in (1e-4, 1e-8, 1e-12):
        err = np.abs(pw.u_eps(p, eps, nu, mu) - soft)
        assert np.all(err <= (mu / nu) * np.sqrt(eps) * (1 + 1e-9) + 1e-12 * mu / nu)
    # sparsity: zero control wherever |p| <= mu, up to that bound
    inside = np.abs(p) <= mu
    assert np.all(np.abs(pw.u_eps(p[inside], 1e-15, nu, mu)) <= (mu / nu) * np.sqrt(1e-15) * 1.01)


@pytest.mark.parametrize("kind", [pw.PHI_CUBIC, pw.PHI_EXP, pw.PHI_KAPPA])
def test_phi_derivatives(kind):
    kappa = 0.1
    fmp = {pw.PHI_CUBIC: lambda t: t ** 3,
           pw.PHI_EXP: lambda t: mpmath.exp(t),
           pw.PHI_KAPPA: lambda t: kappa * (t ** 3 + mpmath.exp(kappa * t))}[kind]
    for y in (-1.7, -0.2, 0.0, 0.4, 2.3):
        v, d1, d2 = pw.phi(kind, np.array(y), kappa)
        assert abs(float(v) - float(fmp(mpmath.mpf(y)))) <= 1e-14 * max(1, abs(float(v)))
        assert abs(float(d1) - float(mpmath.diff(fmp, mpmath.mpf(y)))) <= 1e-13 * max(1, abs(float(d1)))
        assert abs(float(d2) - float(mpmath.diff(fmp, mpmath.mpf(y), 2))) <= 1e-13 * max(1, abs(float(d2)))


def test_phi_monotone_assumption():
    """Assumption 1: phi is monotonically increasing (phi' >= 0)."""
    y = np.linspace(-20, 20, 4001)
    for kind in (pw.PHI_CUBIC, pw.PHI_EXP, pw.PHI_KAPPA):
        assert np.all(pw.phi(kind, y)[1] >= 0)
