"""Pointwise (Nemytskii) functions of the method, FP64 numpy. Test infrastructure.

* P_eps:   the smoothed projection of Sec. 3.1, evaluated in the quotient form
           that Lemma 5's proof gives, 2x / (sqrt((x+1)^2+eps) + sqrt((x-1)^2+eps)),
           which has no cancellation.
* dP_eps:  its derivative, Sec. 3.1, exactly as printed there.
* proj:    the projection onto [-1, 1] (Sec. 1), used only by the eps -> 0 pins.
* u_eps:   the control eliminated from the smoothed stationarity condition
           (Sec. 3.2, smoothed optimality system, third line):
           u = -(1/nu) (p + mu P_eps(-p/mu)).
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


def proj(x):
    """proj_[-1,1](x) (Sec. 1)."""
    return np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0)


def u_eps(p, eps, nu, mu):
    """Control u as a function of the adjoint p, smoothed stationarity (Sec. 3.2)."""
    return -(1.0 / nu) * (p + mu * P_eps(-p / mu, eps))


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
