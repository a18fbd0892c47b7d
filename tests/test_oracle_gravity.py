"""Pins of the gravitational-source oracle (Sec. 3, Eq. (BalancedVariablesGravitational)
with the two-nearest-neighbour centred difference), each against a closed form."""
import numpy as np
import pytest

from oracle import gravity as O


def _mesh(n_r=6, n_t=5, n_p=8, geometric=True):
    r = np.geomspace(1.0, 50.0, n_r + 1) if geometric else np.linspace(0.0, 2.0, n_r + 1)
    th = np.linspace(0.0, np.pi, n_t + 1)
    ph = np.linspace(0.0, 2 * np.pi, n_p + 1)
    return r, th, ph


def test_linear_in_radius_is_exact_everywhere_edges_included():
    r, th, ph = _mesh()
    rc = O.centres(r)
    a, b = 3.25, -7.0
    phi = np.broadcast_to((a * rc + b)[:, None, None], (rc.size, th.size - 1, ph.size - 1)).copy()
    g = O.gradient(phi, r, th, ph)
    assert np.allclose(g[0], a, rtol=1e-13, atol=0)
    assert np.all(g[1] == 0.0) and np.all(g[2] == 0.0)


def test_point_mass_on_geometric_mesh_interior_closed_form():
    # (-1/x+ + 1/x-)/(x+ - x-) = 1/(x+ x-): the neighbours and their spacing, not the cell itself
    r, th, ph = _mesh(n_r=9)
    rc = O.centres(r)
    phi = np.broadcast_to((-1.0 / rc)[:, None, None], (rc.size, 3, 4)).copy()
    g = O.gradient(phi, r, np.linspace(0, np.pi, 4), np.linspace(0, 2 * np.pi, 5))
    want = 1.0 / (rc[2:] * rc[:-2])
    assert np.allclose(g[0][1:-1, 0, 0], want, rtol=1e-13, atol=0)
    # one-sided at both radial edges
    assert np.isclose(g[0][0, 0, 0], (-1 / rc[1] + 1 / rc[0]) / (rc[1] - rc[0]), rtol=1e-13)
    assert np.isclose(g[0][-1, 0, 0], (-1 / rc[-1] + 1 / rc[-2]) / (rc[-1] - rc[-2]), rtol=1e-13)


def test_azimuthal_cosine_closed_form_with_wrap():
    n_p = 16
    r, th, ph = _mesh(n_r=2, n_t=3, n_p=n_p)
    pc = O.centres(ph)
    h = 2 * np.pi / n_p
    phi = np.broadcast_to(np.cos(pc)[None, None, :], (2, 3, n_p)).copy()
    g = O.gradient(phi, r, th, ph)
    assert np.allclose(g[2][0, 0], -np.sin(pc) * np.sin(h) / h, rtol=0, atol=1e-14)


def test_polar_cosine_closed_form_and_one_sided_poles():
    n_t = 12
    r, th, ph = _mesh(n_r=2, n_t=n_t, n_p=3)
    tc = O.centres(th)
    h = np.pi / n_t
    phi = np.broadcast_to(np.cos(tc)[None, :, None], (2, n_t, 3)).copy()
    g = O.gradient(phi, r, th, ph)
    assert np.allclose(g[1][0, 1:-1, 0], -np.sin(tc[1:-1]) * np.sin(h) / h, rtol=0, atol=1e-14)
    assert np.isclose(g[1][0, 0, 0], (np.cos(tc[1]) - np.cos(tc[0])) / h, rtol=1e-13)
    assert np.isclose(g[1][0, -1, 0], (np.cos(tc[-1]) - np.cos(tc[-2])) / h, rtol=1e-13)


def test_sources_of_a_radial_potential():
    rng = np.random.default_rng(3)
    r, th, ph = _mesh()
    rc = O.centres(r)
    a = -2.5
    shape = (rc.size, th.size - 1, ph.size - 1)
    phi = np.broadcast_to((a * rc)[:, None, None], shape).copy()
    rho = rng.uniform(0.5, 2.0, shape)
    v = rng.normal(size=(3,) + shape)
    s = O.sources(phi, rho, v, r, th, ph)
    assert np.allclose(s["S"][0], -rho * a, rtol=1e-13, atol=0)
    assert np.all(s["S"][1] == 0.0) and np.all(s["S"][2] == 0.0)
    assert np.allclose(s["E"], -rho * a * v[0], rtol=1e-13, atol=0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_cell_along_an_axis_gives_zero(axis):
    sizes = [4, 5, 6]
    sizes[axis] = 1
    r = np.linspace(1.0, 2.0, sizes[0] + 1)
    th = np.linspace(0.0, np.pi, sizes[1] + 1)
    ph = np.linspace(0.0, 2 * np.pi, sizes[2] + 1)
    phi = np.random.default_rng(1).normal(size=sizes)
    g = O.gradient(phi, r, th, ph)
    assert np.all(g[axis] == 0.0)


def test_two_azimuthal_cells_give_zero():
    r, th, ph = _mesh(n_r=3, n_t=2, n_p=2)
    phi = np.random.default_rng(2).normal(size=(3, 2, 2))
    assert np.all(O.gradient(phi, r, th, ph)[2] == 0.0)


def test_energy_source_of_a_separable_potential_uses_all_three_components():
    # Phi = a r_c + b cos(theta_c) + c cos(phi_c): each component has a closed form, so
    # E = -rho (v^r g_r + v^theta g_theta + v^phi g_phi) is pinned term by term
    n_r, n_t, n_p = 5, 10, 12
    r, th, ph = _mesh(n_r=n_r, n_t=n_t, n_p=n_p)
    rc, tc, pc = O.centres(r), O.centres(th), O.centres(ph)
    a, b, c = 1.5, -0.75, 2.0
    phi = a * rc[:, None, None] + b * np.cos(tc)[None, :, None] + c * np.cos(pc)[None, None, :]
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.5, 2.0, phi.shape)
    v = rng.normal(size=(3,) + phi.shape)
    s = O.sources(phi, rho, v, r, th, ph)
    ht, hp = np.pi / n_t, 2 * np.pi / n_p
    g_t = (-b * np.sin(tc) * np.sin(ht) / ht)[None, :, None]
    g_p = (-c * np.sin(pc) * np.sin(hp) / hp)[None, None, :]
    want = -rho * (v[0] * a + v[1] * g_t + v[2] * g_p)
    inner = slice(1, -1)  # interior polar cells (the poles are one-sided)
    assert np.allclose(s["E"][:, inner], want[:, inner], rtol=1e-12, atol=1e-13)
    assert np.allclose(s["S"][2], -rho * g_p, rtol=1e-12, atol=1e-13)


def test_azimuthal_range_short_of_a_full_circle_is_one_sided_at_its_ends():
    n_p = 8
    ph = np.linspace(0.0, np.pi, n_p + 1)  # half a circle
    r, th, _ = _mesh(n_r=2, n_t=3, n_p=n_p)
    pc = O.centres(ph)
    h = np.pi / n_p
    phi = np.broadcast_to(np.cos(pc)[None, None, :], (2, 3, n_p)).copy()
    g = O.gradient(phi, r, th, ph)[2][0, 0]
    assert np.allclose(g[1:-1], -np.sin(pc[1:-1]) * np.sin(h) / h, rtol=0, atol=1e-14)
    assert np.isclose(g[0], (np.cos(pc[1]) - np.cos(pc[0])) / h, rtol=1e-13)
    assert np.isclose(g[-1], (np.cos(pc[-1]) - np.cos(pc[-2])) / h, rtol=1e-13)
