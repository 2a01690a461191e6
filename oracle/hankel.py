"""Hankel-type functions of the HB ansatz (Eq. termf).

Test infrastructure (see ``oracle/__init__``).

f_q(omega, tau) = i (sqrt(pi)/2) e^{i q pi} (2 tau / omega)^q H^(1)_q(omega tau).
In 2D the ansatz truncated at N = 1 uses q = s - (d-2)/2 = 0 and 1 (Eq. babich):
  f0 = i sqrt(pi)/2 H0(omega tau),
  f1 = -i sqrt(pi)/2 (2 tau / omega) H1(omega tau)      (e^{i pi} = -1).
H^(1)_q is scipy.special.hankel1 (AMOS), the library primitive of this step.
"""
import math

import numpy as np
from scipy import special

SQRT_PI_2 = math.sqrt(math.pi) / 2.0


def f0(omega, tau):
    return 1j * SQRT_PI_2 * special.hankel1(0, omega * np.asarray(tau))


def f1(omega, tau):
    tau = np.asarray(tau)
    return -1j * SQRT_PI_2 * (2.0 * tau / omega) * special.hankel1(1, omega * tau)
