"""Pins of the oracle's renormalized associated Legendre functions (GenASiS II Sec. 2.2)."""
import math

import numpy as np
import pytest
from scipy import special

from analytic import legendre_p
from oracle import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def scipy_ptilde(l, m, x):
    """Textbook route: sqrt((2l+1)/(4pi) (l-m)!/(l+m)!) P_l^m(x), CS phase included."""
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))
    return norm * special.lpmv(m, l, x)


@pytest.mark.parametrize("x", [-0.93, -0.2, 0.0, 0.41, 0.999])
def test_closed_forms(x):
    P = O.legendre(2, x)
    s = math.sqrt(1 - x * x)
    assert P[O.tri(0, 0)] == pytest.approx(1 / math.sqrt(4 * math.pi), rel=1e-15)
    assert P[O.tri(1, 0)] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * x, rel=1e-14, abs=1e-16)
    assert P[O.tri(1, 1)] == pytest.approx(-math.sqrt(3 / (8 * math.pi)) * s, rel=1e-14)
    assert P[O.tri(2, 0)] == pytest.approx(math.sqrt(5 / (4 * math.pi)) * 0.5 * (3 * x * x - 1), rel=1e-13, abs=1e-16)
    assert P[O.tri(2, 2)] == pytest.approx(math.sqrt(15 / (32 * math.pi)) * (1 - x * x), rel=1e-14)


@pytest.mark.parametrize("L", [8, 20, 40])
def test_matches_textbook_routine(L):
    rng = np.random.default_rng(L)
    for x in rng.uniform(-1, 1, 7):
        P = O.legendre(L, x)
        ref = np.array([scipy_ptilde(l, m, x) for l in range(L + 1) for m in range(l + 1)])
        scale = np.abs(ref).max()
        assert np.abs(P - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("l", [0, 1, 3, 7, 16, 33])
def test_addition_theorem(l):
    """sum_m Delta_m sum_a A^a_lm(O) A^a_lm(O') = (2l+1)/(4pi) P_l(cos gamma)."""
    rng = np.random.default_rng(100 + l)
    for _ in range(5):
        t1, t2 = rng.uniform(0, math.pi, 2)
        p1, p2 = rng.uniform(0, 2 * math.pi, 2)
        P1 = O.legendre(l, math.cos(t1), math.sin(t1))
        P2 = O.legendre(l, math.cos(t2), math.sin(t2))
        acc = 0.0
        for m in range(l + 1):
            d = 1.0 if m == 0 else 2.0
            pp = P1[O.tri(l, m)] * P2[O.tri(l, m)]
            acc += d * pp * (math.cos(m * p1) * math.cos(m * p2) + (math.sin(m * p1) * math.sin(m * p2) if m else 0.0))
        cosg = math.cos(t1) * math.cos(t2) + math.sin(t1) * math.sin(t2) * math.cos(p1 - p2)
        ref = (2 * l + 1) / (4 * math.pi) * float(legendre_p(l, cosg))
        assert acc == pytest.approx(ref, abs=1e-12 * (2 * l + 1) / (4 * math.pi))


def test_rejects_out_of_range_degree():
    with pytest.raises(ValueError):
        O.legendre(86, 0.3)
