"""Pins of the coarsening-block oracle (Sec. 2.1 blocks, Sec. 2.3 volume-weighted means)."""
import math

import numpy as np
import pytest

from oracle import coarsen as O
from paper_2602_02507_gb300 import workloads as W

GOLDEN = {}
with open(__file__.replace("test_oracle_coarsen.py", "golden/paper_values.txt")) as f:
    for line in f:
        if line.strip() and not line.startswith("#"):
            k, v, digits = line.split()[:3]
            GOLDEN[k] = (float(v), int(digits))


def _agrees(x, key):
    v, d = GOLDEN[key]
    return float(f"{x:.{d - 1}e}") == float(f"{v:.{d - 1}e}")


def test_required_factors_at_the_first_cell_are_the_printed_gains():
    # Sec. 3: physical mesh N_theta = 192, r_core = 16 km, R_radial = 5.9
    m = W.paper_mesh(192, 16.0, 5.9, 0, 3)
    polar, azim = O.required_factors(m.r, m.theta, m.phi)
    assert _agrees(polar[0], "coarsening_gain_2d")
    assert _agrees(azim[0, 0], "coarsening_gain_3d")


def _mesh(n_theta=16):
    return W.paper_mesh(n_theta, 0.25, 3.68, 0, 3)


def test_blocks_are_powers_of_two_dividing_the_counts_and_cover_the_need():
    m = _mesh(24)
    c_t, c_p = O.factors(m.r, m.theta, m.phi)
    polar, azim = O.required_factors(m.r, m.theta, m.phi)
    n_t, n_p = m.theta.size - 1, m.phi.size - 1
    for i in range(c_t.size):
        assert n_t % c_t[i] == 0
        assert c_t[i] >= polar[i] or c_t[i] == n_t
        assert c_t[i] == 1 or c_t[i] // 2 < polar[i] or n_t % (c_t[i] // 2) != 0
        for j in range(n_t):
            assert n_p % c_p[i, j] == 0
            assert c_p[i, j] >= azim[i, j] or c_p[i, j] == n_p
    # near the origin everything is coarsened; far out the equatorial cells are not
    assert c_t[0] > 1 and c_p[0, 0] > 1
    assert c_t[-1] == 1 and c_p[-1, n_t // 2] == 1


def test_conserves_each_shell_and_is_constant_on_blocks():
    m = _mesh(16)
    rng = np.random.default_rng(1)
    shape = (m.r.size - 1, m.theta.size - 1, m.phi.size - 1)
    f = rng.normal(size=shape)
    g = O.coarsen(f, m.r, m.theta, m.phi)
    dmu = -np.diff(np.cos(m.theta))
    dph = np.diff(m.phi)
    w = dmu[:, None] * dph[None, :]
    assert np.allclose((g * w).sum(axis=(1, 2)), (f * w).sum(axis=(1, 2)), rtol=1e-13, atol=1e-13)
    c_t, c_p = O.factors(m.r, m.theta, m.phi)
    for i in range(shape[0]):
        for j0 in range(0, shape[1], c_t[i]):
            cp = c_p[i, j0]
            for k0 in range(0, shape[2], cp):
                blk = g[i, j0:j0 + c_t[i], k0:k0 + cp]
                assert np.ptp(blk) <= 1e-12 * max(1.0, np.abs(blk).max())
    # coarsening a coarsened field changes nothing
    assert np.allclose(O.coarsen(g, m.r, m.theta, m.phi), g, rtol=1e-14, atol=1e-15)


def test_cells_wide_enough_are_left_alone():
    m = _mesh(16)
    rng = np.random.default_rng(2)
    f = rng.normal(size=(m.r.size - 1, m.theta.size - 1, m.phi.size - 1))
    g = O.coarsen(f, m.r, m.theta, m.phi)
    c_t, c_p = O.factors(m.r, m.theta, m.phi)
    alone = (c_t[:, None] == 1) & (c_p == 1)
    assert alone.any()
    assert np.array_equal(g[alone], f[alone])


def test_one_block_by_brute_force():
    m = _mesh(16)
    rng = np.random.default_rng(3)
    f = rng.normal(size=(m.r.size - 1, m.theta.size - 1, m.phi.size - 1))
    g = O.coarsen(f, m.r, m.theta, m.phi)
    c_t, c_p = O.factors(m.r, m.theta, m.phi)
    i = 3
    ct, cp = c_t[i], c_p[i, 0]
    num = den = 0.0
    for j in range(ct):
        for k in range(cp):
            vol = (math.cos(m.theta[j]) - math.cos(m.theta[j + 1])) * (m.phi[k + 1] - m.phi[k])
            num += vol * f[i, j, k]
            den += vol
    assert math.isclose(g[i, 0, 0], num / den, rel_tol=1e-13)
    assert math.isclose(g[i, ct - 1, cp - 1], num / den, rel_tol=1e-13)


@pytest.mark.parametrize("value", [2.5, -1.0])
def test_block_constant_field_is_unchanged(value):
    m = _mesh(16)
    f = np.full((m.r.size - 1, m.theta.size - 1, m.phi.size - 1), value)
    assert np.allclose(O.coarsen(f, m.r, m.theta, m.phi), value, rtol=1e-15, atol=0)
