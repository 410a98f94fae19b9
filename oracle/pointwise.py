"""Pointwise (Nemytskii) functions of the method, FP64 numpy. Test infrastructure.

* P_eps:   the smoothed projection of Sec. 3.1, evaluated in the quotient form
           that Lemma 5's proof gives, 2x / (sqrt((x+1)^2+eps) + sqrt((x-1)^2+eps)),
           which has no cancellation.
* dP_eps:  its derivative, Sec. 3.1, exactly as printed there.
* P_eps_minus_id, one_minus_dP_eps: P_eps(x) - x and 1 - P_eps'(x), the two
           combinations in which the reduced system uses P_eps, written without
           cancellation (see below).
* proj:    the projection onto [-1, 1] (Sec. 1), used only by the eps -> 0 pins.
* u_eps:   the control eliminated from the smoothed stationarity condition
           (Sec. 3.2, smoothed optimality system, third line):
           u = -(1/nu) (p + mu P_eps(-p/mu)) = -(mu/nu) (P_eps(x) - x), x = -p/mu.

Where |x| < 1 (the adjoint below the L1 threshold mu), P_eps(x) = x (1 - O(eps)),
so p + mu P_eps(-p/mu) and 1 - P_eps'(x) are O(eps) differences of O(1)
numbers: written as printed they lose a relative 2^-53 / eps of accuracy
(1e-10 at eps = 1e-6), and with them the state y, which the inactive control
alone drives. Lemma 5's proof removes the cancellation of P_eps itself by the
quotient form; the same device, applied to the differences
|s| - sqrt(s^2 + eps) = -eps / (|s| + sqrt(s^2 + eps)), removes it here, so
both combinations keep full relative accuracy at every x.
* u_limit: the eps = 0 control from the reduced non-smooth system (Sec. 2,
           Lemma 4): u = -(1/nu) (p + mu proj(-p/mu)).
* phi:     the nonlinearities used by the workloads: y^3, exp(y), and the
           paper's model nonlinearity kappa (y^3 + exp(kappa y)) (Sec. 4).
"""
import numpy as np

PHI_CUBIC = 0   # phi(y) = y^3
PHI_EXP = 1     # phi(y) = exp(y)
PHI_KAPPA = 2   # phi(y) = kappa (y^3 + exp(kappa y)), the model problem of Sec. 4


def P_eps(x, eps):
    """Smoothed projection P_eps(x) (Sec. 3.1), quotient form from Lemma 5's proof."""
    x = np.asarray(x, dtype=np.float64)
    s_plus = np.sqrt((x + 1.0) ** 2 + eps)
    s_minus = np.sqrt((x - 1.0) ** 2 + eps)
    return 2.0 * x / (s_plus + s_minus)


def dP_eps(x, eps):
    """Derivative P_eps'(x) (Sec. 3.1), the printed difference of two quotients."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * ((x + 1.0) / np.sqrt((x + 1.0) ** 2 + eps)
                  - (x - 1.0) / np.sqrt((x - 1.0) ** 2 + eps))


def P_eps_minus_id(x, eps):
    """P_eps(x) - x without cancellation.

    With a = sqrt((x+1)^2 + eps), b = sqrt((x-1)^2 + eps) the quotient form
    gives P_eps(x) - x = x (2 - a - b) / (a + b), and
        2 - a - b = (2 - |x+1| - |x-1|) + (|x+1| - a) + (|x-1| - b),
    where the first term is 2 (1 - max(1, |x|)) (zero for |x| <= 1) and each
    of the others is -eps / (|s| + sqrt(s^2 + eps)): three terms of one sign.
    """
    x = np.asarray(x, dtype=np.float64)
    a = np.sqrt((x + 1.0) ** 2 + eps)
    b = np.sqrt((x - 1.0) ** 2 + eps)
    gap = 2.0 * (1.0 - np.maximum(1.0, np.abs(x)))
    two_minus_ab = gap - eps / (np.abs(x + 1.0) + a) - eps / (np.abs(x - 1.0) + b)
    return x * two_minus_ab / (a + b)


def one_minus_dP_eps(x, eps):
    """1 - P_eps'(x) without cancellation.

    With g(s) = s / sqrt(s^2 + eps), P_eps'(x) = (g(x+1) - g(x-1)) / 2, so
    1 - P_eps'(x) = ((1 - g(x+1)) + (1 + g(x-1))) / 2. For r = sqrt(s^2 + eps):
    1 - g(s) = (r - s)/r, where r - s = eps/(r + s) if s > 0 and r + |s| if
    s <= 0; 1 + g(s) = (r + s)/r, where r + s = eps/(r - s) if s < 0 and r + s
    if s >= 0. Every branch adds numbers of one sign.
    """
    x = np.asarray(x, dtype=np.float64)
    sp_, sm = x + 1.0, x - 1.0
    a = np.sqrt(sp_ * sp_ + eps)
    b = np.sqrt(sm * sm + eps)
    with np.errstate(divide="ignore", invalid="ignore"):
        r1 = np.where(sp_ > 0.0, eps / (a + sp_), a - sp_)     # a - (x+1)
        r2 = np.where(sm < 0.0, eps / (b - sm), b + sm)        # b + (x-1)
    return 0.5 * (r1 / a + r2 / b)


def proj(x):
    """proj_[-1,1](x) (Sec. 1)."""
    return np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0)


def u_eps(p, eps, nu, mu):
    """Control u as a function of the adjoint p, smoothed stationarity (Sec. 3.2):
    u = -(1/nu)(p + mu P_eps(-p/mu)) = -(mu/nu)(P_eps(x) - x) with x = -p/mu
    (p = -mu x), evaluated through P_eps_minus_id."""
    p = np.asarray(p, dtype=np.float64)
    return -(mu / nu) * P_eps_minus_id(-p / mu, eps)


def u_limit(p, nu, mu):
    """Control of the non-smooth reduced system (Sec. 2): soft threshold of p at mu."""
    return -(1.0 / nu) * (p + mu * proj(-p / mu))


def phi(kind, y, kappa=0.1):
    """phi(y), phi'(y), phi''(y) for the three nonlinearities (closed forms)."""
    y = np.asarray(y, dtype=np.float64)
    if kind == PHI_CUBIC:
        return y ** 3, 3.0 * y ** 2, 6.0 * y
    if kind == PHI_EXP:
        e = np.exp(y)
        return e, e, e
    if kind == PHI_KAPPA:
        e = np.exp(kappa * y)
        return (kappa * (y ** 3 + e),
                kappa * (3.0 * y ** 2 + kappa * e),
                kappa * (6.0 * y + kappa * kappa * e))
    raise ValueError("unknown phi kind %r" % (kind,))
