"""Manufactured solutions of (FL-1) on the unit ball (Section 5, (exam-0) and
(exam-2)), shared by the oracle and GPU convergence tests.

For k >= 0 the pair

    f = 2^{2s} Gamma(1+s+k) Gamma(d/2+s+k) / (k! Gamma(d/2+k)) P_k^{(s, d/2-1)}(2|x|^2 - 1)
    u = (1 - |x|^2)_+^s P_k^{(s, d/2-1)}(2|x|^2 - 1)

solves (-Delta)^s u = f in the ball with u = 0 outside (P_k^{(a,b)} the
Jacobi polynomial).  k = 0 gives f = 1 / C with C the ball constant.
"""
import math

import numpy as np
from scipy import special


def jacobi(k, s, d, r2):
    return special.eval_jacobi(k, s, d / 2.0 - 1.0, 2.0 * r2 - 1.0)


def rhs(k, s, d, x):
    x = np.asarray(x, dtype=np.float64).reshape(len(x), -1)
    r2 = np.sum(x * x, axis=1)
    c = 2.0 ** (2 * s) * math.gamma(1 + s + k) * math.gamma(d / 2 + s + k) / (math.factorial(k) * math.gamma(d / 2 + k))
    return c * jacobi(k, s, d, r2)


def exact(k, s, d, x):
    x = np.asarray(x, dtype=np.float64).reshape(len(x), -1)
    r2 = np.sum(x * x, axis=1)
    return np.maximum(0.0, 1.0 - r2) ** s * jacobi(k, s, d, r2)
