"""Pins of the oracle's whole solve: steps (a) moments, (b)+(c) radial recurrences,
(d) potential (GenASiS II Sec. 2.2), against invariants, exact discrete closed
forms, a dense brute-force restatement and continuum solutions."""
import math

import numpy as np
import pytest

import analytic as A
from oracle import oracle as O
from paper_2602_02507_gb300 import workloads as W


def _solve(w, literal=False, r_ref=None):
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L, r_ref=r_ref)
    return tab, O.solve(tab, w.rho, m.G, literal=literal)


def _cell_volumes(r, th, ph):
    V = np.diff(r ** 3) / 3.0
    dmu = np.cos(th[:-1]) - np.cos(th[1:])
    dph = np.diff(ph)
    return V[:, None, None] * dmu[None, :, None] * dph[None, None, :]


@pytest.mark.parametrize("r0", [0.0, 0.2])
def test_monopole_moment_is_enclosed_mass(r0):
    """M^R_00 at edge i = sqrt(4 pi) G M_enc(r_i)."""
    w = W.random_small((7, 5, 6), 4, seed=11, r0=r0, r1=2.0, uneven=True)
    tab, s = _solve(w)
    mass = (w.rho * _cell_volumes(w.mesh.r, w.mesh.theta, w.mesh.phi)).sum(axis=(1, 2))
    menc = np.concatenate([[0.0], np.cumsum(mass)])
    assert np.allclose(s["MR"][:, 0], math.sqrt(4 * math.pi) * w.mesh.G * menc, rtol=1e-13, atol=0)


def _spherical(n_r, shape_ang, r0, r1, L, hollow=0, seed=0):
    rng = np.random.default_rng(seed)
    prof = 0.5 + rng.random(n_r)
    prof[:hollow] = 0.0
    n_t, n_p = shape_ang
    rho = np.repeat(np.repeat(prof[:, None, None], n_t, 1), n_p, 2)
    r = W.uniform_edges(r0, r1, n_r)
    th, ph = W.angular_edges(n_t, n_p)
    return W.Workload(W.Mesh(r, th, ph, L, 1.0), np.ascontiguousarray(rho), {"prof": prof})


def test_spherical_density_has_only_monopole():
    w = _spherical(6, (8, 10), 0.0, 1.0, 6)
    _, s = _solve(w)
    assert np.abs(s["A"][:, 1:]).max() <= 1e-14 * np.abs(s["A"][:, 0]).max()


def test_spherical_potential_is_the_same_in_every_polar_cell():
    """A spherically symmetric density gives each shell one potential value: the cell
    mean of the monopole kernel is the constant P~_0^0 in every polar cell, including
    the polar caps of a fine theta mesh, whose solid-angle factor
    cos(theta_j) - cos(theta_{j+1}) is a difference of nearly equal numbers (formed
    as that difference, it costs the cap cells of 512 polar cells 1.8e-12; the bound
    leaves room for the 1e-14 tolerance of the Romberg theta integrals)."""
    w = _spherical(4, (512, 4), 0.1, 1.0, 2)
    _, s = _solve(w)
    phi = s["phi"]
    spread = np.abs(phi - phi[:, 256:257, :1]).max(axis=(1, 2)) / np.abs(phi).max(axis=(1, 2))
    assert spread.max() <= 2e-13, spread


def test_exterior_potential_of_spherical_mass():
    """Outside all mass: Phi_i = -G M_tot <1/r>_i, <1/r> the shell volume mean."""
    w = _spherical(9, (4, 6), 0.0, 3.0, 4)
    w.rho[5:] = 0.0
    tab, s = _solve(w)
    r = w.mesh.r
    M = (w.rho * _cell_volumes(r, w.mesh.theta, w.mesh.phi)).sum()
    inv_r = 1.5 * np.diff(r ** 2) / np.diff(r ** 3)
    for i in range(5, 9):
        assert np.allclose(s["phi"][i], -M * inv_r[i], rtol=1e-13, atol=0)


def test_cavity_potential_is_constant():
    """Inside an empty central cavity the l = 0 potential is
    -G sum_i' M_i' <1/r>_i', the same in every cavity cell."""
    w = _spherical(8, (4, 6), 0.0, 2.0, 3, hollow=3)
    tab, s = _solve(w)
    r = w.mesh.r
    Mi = (w.rho * _cell_volumes(r, w.mesh.theta, w.mesh.phi)).sum(axis=(1, 2))
    inv_r = 1.5 * np.diff(r ** 2) / np.diff(r ** 3)
    expect = -np.sum(Mi * inv_r)
    for i in range(3):
        assert np.allclose(s["phi"][i], expect, rtol=1e-13, atol=0)


@pytest.mark.parametrize("r0,L", [(0.0, 4), (0.3, 3), (0.0, 0)])
def test_literal_and_factored_sums_agree(r0, L):
    w = W.random_small((5, 6, 8), L, seed=3, r0=r0, r1=1.7, uneven=True)
    _, a = _solve(w, literal=False)
    _, b = _solve(w, literal=True)
    for key in ("A", "MR", "MI", "C"):
        assert np.abs(a[key] - b[key]).max() <= 1e-13 * np.abs(b[key]).max()
    assert np.abs(a["phi"] - b["phi"]).max() <= 1e-13 * np.abs(b["phi"]).max()


@pytest.mark.parametrize("r0,L", [(0.0, 4), (0.4, 4), (0.0, 2)])
def test_recurrences_match_dense_green_matrix(r0, L):
    """The outward/inward recurrences and the midpoint split equal the dense
    Green's-matrix sum over all source cells (no recurrences)."""
    w = W.random_small((6, 4, 8), L, seed=7, r0=r0, r1=1.5, uneven=True)
    tab, s = _solve(w)
    g = O.green_matrix_potential(tab, w.rho, w.mesh.G)
    assert np.abs(s["phi"] - g).max() <= 1e-13 * np.abs(g).max()


def test_linearity():
    w1 = W.random_small((5, 4, 6), 5, seed=1, r0=0.0, r1=1.0)
    w2 = W.random_small((5, 4, 6), 5, seed=2, r0=0.0, r1=1.0)
    tab = O.build_tables(w1.mesh.r, w1.mesh.theta, w1.mesh.phi, 5)
    p1 = O.solve(tab, w1.rho, 1.0)["phi"]
    p2 = O.solve(tab, w2.rho, 1.0)["phi"]
    p12 = O.solve(tab, 2.5 * w1.rho - 0.75 * w2.rho, 1.0)["phi"]
    assert np.abs(p12 - (2.5 * p1 - 0.75 * p2)).max() <= 1e-13 * np.abs(p12).max()


def test_z_rotation_equivariance():
    """A one-cell azimuthal shift of rho on a uniform phi mesh shifts Phi by one cell
    and rotates every (cos, sin) moment pair by m dphi."""
    n_p, L = 12, 6
    w = W.random_small((4, 5, n_p), L, seed=9, r0=0.1, r1=1.0)
    tab = O.build_tables(w.mesh.r, w.mesh.theta, w.mesh.phi, L)
    a = O.solve(tab, w.rho, 1.0)
    b = O.solve(tab, np.roll(w.rho, 1, axis=2), 1.0)
    assert np.abs(b["phi"] - np.roll(a["phi"], 1, axis=2)).max() <= 1e-13 * np.abs(a["phi"]).max()
    dphi = 2 * math.pi / n_p
    scale = np.abs(a["A"]).max()
    for l in range(L + 1):
        for m in range(1, l + 1):
            qc, qs = O.qidx(l, m, 0), O.qidx(l, m, 1)
            c, s = math.cos(m * dphi), math.sin(m * dphi)
            assert np.allclose(b["A"][:, qc], c * a["A"][:, qc] - s * a["A"][:, qs], atol=1e-13 * scale)
            assert np.allclose(b["A"][:, qs], s * a["A"][:, qc] + c * a["A"][:, qs], atol=1e-13 * scale)


def test_equatorial_mirror():
    """rho(theta) -> rho(pi - theta) on a symmetric theta mesh flips moments with
    l + m odd and mirrors Phi."""
    L = 7
    w = W.random_small((4, 6, 8), L, seed=4, r0=0.0, r1=1.0)
    tab = O.build_tables(w.mesh.r, w.mesh.theta, w.mesh.phi, L)
    a = O.solve(tab, w.rho, 1.0)
    b = O.solve(tab, w.rho[:, ::-1, :].copy(), 1.0)
    scale = np.abs(a["A"]).max()
    for l in range(L + 1):
        for m in range(l + 1):
            for aa in range(1 if m == 0 else 2):
                q = O.qidx(l, m, aa)
                sign = -1.0 if (l + m) % 2 else 1.0
                assert np.allclose(b["A"][:, q], sign * a["A"][:, q], atol=1e-13 * scale)
    assert np.abs(b["phi"] - a["phi"][:, ::-1, :]).max() <= 1e-13 * np.abs(a["phi"]).max()


@pytest.mark.parametrize("r0", [0.0, 1e5])
def test_reference_radius_invariance(r0):
    if r0 == 0.0:
        w = W.random_small((6, 4, 6), 8, seed=5, r0=0.0, r1=2.0)
    else:
        w = W.random_small((6, 4, 6), 12, seed=5, r0=1e5, r1=1e9, geometric=True)
    m = w.mesh
    ref = O.default_r_ref(m.r)
    _, a = _solve(w, r_ref=ref)
    _, b = _solve(w, r_ref=7.3 * ref)
    assert np.abs(a["phi"] - b["phi"]).max() <= 1e-13 * np.abs(a["phi"]).max()
    assert np.abs(a["A"] - b["A"]).max() <= 1e-15 * np.abs(a["A"]).max()


def test_direct_green_quadrature_converges_in_L():
    """Exterior cells: the solve tends, as L grows, to the cell-averaged direct
    Green's-function integral of the piecewise-constant source (sub-cell Gauss
    quadrature), down to the quadrature's own floor."""
    n_r, n_t, n_p = 8, 4, 6
    r = W.uniform_edges(0.0, 2.0, n_r)
    th, ph = W.angular_edges(n_t, n_p)
    rng = np.random.default_rng(1)
    rho = np.zeros((n_r, n_t, n_p))
    rho[:3] = 0.5 + rng.random((3, n_t, n_p))
    targets = [(i, j, k) for i in (6, 7) for j in range(n_t) for k in range(0, n_p, 2)]
    ref = A.direct_cell_average_potential(r, th, ph, rho, targets, n_src=6, n_tgt=5)
    errs = []
    for L in (0, 2, 4, 8, 12, 16):
        tab = O.build_tables(r, th, ph, L)
        phi = O.solve(tab, rho, 1.0)["phi"]
        num = np.array([phi[c] for c in targets])
        errs.append(np.abs(num - ref).max() / np.abs(ref).max())
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[0] > 1e-2 and errs[-1] < 1e-7


def test_homogeneous_sphere_converges():
    """Homogeneous sphere (surface on a shell edge): per-cell error against the closed
    form falls under radial refinement (second order in the interior)."""
    errs = []
    for n in (16, 32, 64):
        r = W.uniform_edges(0.0, 2.0, n)
        th, ph = W.angular_edges(4, 4)
        rho = np.zeros((n, 4, 4))
        rho[: n // 2] = 1.0
        tab = O.build_tables(r, th, ph, 2)
        phi = O.solve(tab, rho, 1.0)["phi"][:, 0, 0]
        ex = A.sphere_potential(W.midpoints(r), 1.0, 1.0)
        errs.append(np.abs(phi - ex).max() / np.abs(ex).max())
    assert errs[0] < 1e-2
    assert errs[1] < 0.3 * errs[0] and errs[2] < 0.3 * errs[1]


def test_spheroid_closed_form_and_refinement():
    """Homogeneous oblate spheroid a1 = 1, a3 = 0.6, L = 8 (the solver's small
    benchmark case): L1 error (Eq. L1error) below 1e-3 and falling under refinement."""
    l1 = []
    for fac in (1, 2):
        w = W.spheroid(n_r=64 * fac, n_theta=32 * fac, n_phi=4, L=8)
        m = w.mesh
        _, s = _solve(w)
        R, T = np.meshgrid(W.midpoints(m.r), W.midpoints(m.theta), indexing="ij")
        ex = A.spheroid_potential(R * np.sin(T), R * np.cos(T), 1.0, 0.6, 1.0)
        num = s["phi"][:, :, 0]
        l1.append(np.abs(num - ex).sum() / np.abs(ex).sum())
    assert l1[0] < 1e-3
    assert l1[1] < 0.75 * l1[0]


def test_truncation_error_carries_next_even_degree():
    """With L = 12 and equatorial symmetry the residual's polar pattern is P_14
    (GenASiS II Sec. 3.1): just outside the equator, the P_14 component of the
    relative error dominates every other degree up to 21."""
    e = 0.9
    a1, a3 = 1.0, math.sqrt(1 - e * e)
    w = W.spheroid(n_r=96, n_theta=96, n_phi=4, L=12, a1=a1, a3=a3, r_max=2.0)
    m = w.mesh
    _, s = _solve(w)
    rc, tc = W.midpoints(m.r), W.midpoints(m.theta)
    R, T = np.meshgrid(rc, tc, indexing="ij")
    ex = A.spheroid_potential(R * np.sin(T), R * np.cos(T), a1, a3, 1.0)
    err = (s["phi"][:, :, 0] - ex) / np.abs(ex)
    dmu = np.cos(m.theta[:-1]) - np.cos(m.theta[1:])
    i = int(np.searchsorted(rc, 1.05))
    coef = np.array([(2 * l + 1) / 2 * np.sum(err[i] * A.legendre_p(l, np.cos(tc)) * dmu) for l in range(22)])
    assert int(np.argmax(np.abs(coef))) == 14
