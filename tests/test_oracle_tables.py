"""Pins of the oracle's cell-integrated angular and radial kernels (GenASiS II Sec. 2.2)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_2602_02507_gb300 import workloads as W


def scipy_ptilde(l, m, x):
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))
    return norm * special.lpmv(m, l, x)


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_theta_integrals_match_adaptive_quadrature():
    L = 12
    th = np.array([0.0, 0.05, 0.4, 1.2, 1.5707963267948966, 2.3, 3.0, math.pi])
    Ith = O.theta_integrals(L, th)
    scale = np.abs(Ith).max()
    for j in range(th.size - 1):
        for l in range(L + 1):
            for m in range(l + 1):
                ref, _ = integrate.quad(lambda t: scipy_ptilde(l, m, math.cos(t)) * math.sin(t),
                                        th[j], th[j + 1], epsabs=1e-16, epsrel=1e-14, limit=200)
                assert abs(Ith[O.tri(l, m), j] - ref) <= 2e-14 * scale


@pytest.mark.parametrize("n_t", [1, 7, 32])
def test_theta_integrals_full_sphere(n_t):
    """Summed over a full polar range, int_{-1}^{1} P~_l^0 dmu is 2/sqrt(4 pi) for l = 0
    and 0 for l >= 1 (orthogonality to P~_0^0); odd l+m vanish by mirror symmetry."""
    L = 16
    th = W.uniform_edges(0.0, math.pi, n_t)
    Ith = O.theta_integrals(L, th)
    tot = Ith.sum(axis=1)
    assert tot[O.tri(0, 0)] == pytest.approx(2 / math.sqrt(4 * math.pi), rel=1e-14)
    for l in range(1, L + 1):
        assert abs(tot[O.tri(l, 0)]) < 1e-14
        for m in range(l + 1):
            if (l + m) % 2 == 1:
                assert abs(tot[O.tri(l, m)]) < 1e-14


def test_phi_integrals_closed_form():
    L = 20
    ph = np.sort(np.concatenate([[0.0, 2 * math.pi], np.random.default_rng(3).uniform(0, 2 * math.pi, 9)]))
    Iph = O.phi_integrals(L, ph)
    for k in range(ph.size - 1):
        a, b = ph[k], ph[k + 1]
        assert Iph[0, k] == pytest.approx(b - a, rel=1e-14)
        for m in range(1, L + 1):
            c = (math.sin(m * b) - math.sin(m * a)) / m
            s = (math.cos(m * a) - math.cos(m * b)) / m
            assert abs(Iph[O.pcol(m, 0), k] - c) < 1e-14
            assert abs(Iph[O.pcol(m, 1), k] - s) < 1e-14


def test_phi_discrete_orthogonality():
    """On a uniform phi mesh, projecting the cell average of cos|sin(m'phi) with the
    cell integral of cos|sin(m phi) gives zero for m != m' when m + m' < n_phi."""
    n_p, L = 16, 7
    ph = W.uniform_edges(0.0, 2 * math.pi, n_p)
    Iph = O.phi_integrals(L, ph)
    dph = np.diff(ph)
    gram = Iph @ (Iph / dph).T
    for p in range(2 * L + 1):
        for p2 in range(2 * L + 1):
            if p != p2:
                assert abs(gram[p, p2]) < 1e-14


@pytest.mark.parametrize("r0", [0.0, 0.3])
def test_radial_integrals_gauss(r0):
    L = 10
    r = np.concatenate([[r0], r0 + np.cumsum(np.random.default_rng(5).uniform(0.05, 0.4, 6))])
    r_ref = 0.7
    WR, WI, V = O.radial_integrals(L, r, r_ref)
    x, w = np.polynomial.legendre.leggauss(40)
    for i in range(r.size - 1):
        a, b = r[i], r[i + 1]
        rr = 0.5 * (b - a) * x + 0.5 * (a + b)
        ww = 0.5 * (b - a) * w
        assert V[i] == pytest.approx(np.sum(ww * rr ** 2), rel=1e-14)
        for l in range(L + 1):
            assert WR[l, i] == pytest.approx(np.sum(ww * rr ** 2 * (rr / r_ref) ** l), rel=1e-13)
            if a == 0.0 and l >= 2:
                assert math.isinf(WI[l, i])
            elif a == 0.0:
                exact = r_ref ** l * b ** (2 - l) / (2 - l)
                assert WI[l, i] == pytest.approx(exact, rel=1e-14)
            else:
                assert WI[l, i] == pytest.approx(np.sum(ww * rr ** 2 * r_ref ** l / rr ** (l + 1)), rel=1e-12)


def test_default_reference_radius():
    assert O.default_r_ref([0.0, 1.0, 4.0]) == pytest.approx(2.0)
    assert O.default_r_ref([1e5, 1e7, 1e10]) == pytest.approx(math.sqrt(1e15))
