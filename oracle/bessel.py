"""Modified Bessel function of the first kind, integer order, by power series.

TEST INFRASTRUCTURE (oracle).  The thesis expands every Boltzmann factor with
the Jacobi-Anger identity exp(x cos t) = sum_n I_n(x) e^{int} (§3.2, Eq. 3.3;
§3.3, Eq. 3.9), so I_n(x) of integer order is the only special function the
method needs.  It is computed here from its defining series

    I_n(x) = sum_{k>=0} (x/2)^{2k+|n|} / (k! (k+|n|)!),      I_{-n} = I_n,

which has only positive terms for x >= 0 (no cancellation), so the partial sum
is accurate to a few ulp.  Pins: scipy.special.iv (an independent library
routine), the trapezoid rule on (1/pi) int_0^pi e^{x cos t} cos(nt) dt, and
the Wronskian-type identity sum_n I_n(x) = e^x (tests/test_oracle_bessel.py).
"""

import math


def bessel_i(n: int, x: float) -> float:
    """I_n(x) for integer n and real x (I_n(-x) = (-1)^n I_n(x))."""
    n = abs(int(n))
    x = float(x)
    if x == 0.0:
        return 1.0 if n == 0 else 0.0
    sign = 1.0
    if x < 0.0:
        x = -x
        sign = -1.0 if (n % 2) else 1.0
    half = 0.5 * x
    # first term (x/2)^n / n! as a running product (one rounding per factor)
    if n * math.log(half) - math.lgamma(n + 1) < -740.0:
        return 0.0
    term = 1.0
    for k in range(1, n + 1):
        term *= half / k
    total = term
    q = half * half
    k = 0
    while True:
        k += 1
        term *= q / (k * (k + n))
        total += term
        if term <= 1e-18 * total:
            break
    return sign * total
