"""The spheroid study's closed form (paper_2602_02507_gb300.spheroids) against an
independent restatement (tests/analytic.py) and the paper's printed axes (Sec. 3.1)."""
import math

import numpy as np
import pytest

from analytic import sphere_potential, spheroid_potential
from paper_2602_02507_gb300 import spheroids as S


@pytest.mark.parametrize("e", [0.0, 0.01, 0.049, 0.051, 0.3, 0.6, 0.9])
def test_closed_form_matches_independent_restatement(e):
    a1, a3 = S.axes(e)
    rng = np.random.default_rng(1)
    rp = rng.uniform(0.0, 3 * a1, 4000)
    z = rng.uniform(-3 * a1, 3 * a1, 4000)
    got = S.potential(rp, z, a1, a3)
    want = spheroid_potential(rp, z, a1, a3, S.RHO)
    # the restatement uses the closed forms down to e = 1e-6 (cancellation near 1e-16 / e^2)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-10


def test_sphere_limit_and_mass():
    a1, a3 = S.axes(0.0)
    assert a1 == a3
    assert math.isclose(4.0 / 3.0 * math.pi * a1 ** 3 * S.RHO, S.MASS, rel_tol=1e-14)
    r = np.linspace(0.0, 4 * a1, 101)
    assert np.allclose(S.potential(r, 0.0 * r, a1, a3), sphere_potential(r, a1, S.RHO), rtol=1e-13, atol=0)


def test_paper_axes_for_e_09():
    # Sec. 3.1 prints a1 ~ 8.182 and a3 ~ 3.566 for e = 0.9, rho = 1e-3, M = 1
    a1, a3 = S.axes(0.9)
    assert round(a1, 3) == 8.182 and round(a3, 3) == 3.566


def test_coefficients_series_meets_closed_form():
    I, A1, A3 = S.coefficients(np.array([0.04999999, 0.05000001]))
    assert np.allclose(I[0], I[1], rtol=1e-9) and np.allclose(A1[0], A1[1], rtol=1e-9)
    assert np.allclose(A3[0], A3[1], rtol=1e-8)
    I, A1, A3 = S.coefficients(np.array([0.0, 0.2, 0.7]))
    assert np.allclose(2 * A1 + A3, 2.0, rtol=1e-13)


@pytest.mark.parametrize("e", [0.0, 0.3, 0.6, 0.9])
@pytest.mark.parametrize("n_theta", [16, 33])
def test_exact_volume_fractions_hold_the_whole_mass(e, n_theta):
    from paper_2602_02507_gb300 import workloads as W
    a1, a3 = S.axes(e)
    mesh = W.paper_mesh(n_theta, S.R_CORE, S.R_RADIAL, 0, 2)
    f = W.spheroid_fraction_exact(mesh.r, mesh.theta, a1, a3)
    assert f.min() >= 0.0 and f.max() <= 1.0
    vol = np.outer(np.diff(mesh.r ** 3) / 3.0, np.diff(-np.cos(mesh.theta))) * 2.0 * math.pi
    assert math.isclose(float(np.sum(f * vol)) * S.RHO, S.MASS, rel_tol=1e-13)
    # the sub-cell estimate converges to it (64 x 64 sub-cells: within a few 1/64 steps)
    fs = W.spheroid_fraction(mesh.r, mesh.theta, a1, a3, sub=64)
    assert np.abs(f - fs).max() < 4.0 / 64
