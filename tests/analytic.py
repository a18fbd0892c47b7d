"""Closed-form potentials and direct Green's-function quadrature used to pin the oracle.

Everything here is written from textbook formulas, independently of the oracle
and of the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np


def spheroid_coefficients(e: float):
    """(I, A1, A3) of a homogeneous oblate spheroid of eccentricity e
    (GenASiS II Sec. 3.1, Eq. SpheroidPotential); sphere limit (2, 2/3, 2/3)."""
    if e < 1e-6:
        return 2.0, 2.0 / 3.0, 2.0 / 3.0
    s = math.sqrt(1.0 - e * e)
    ase = math.asin(e)
    I = 2.0 * s / e * ase
    A1 = s / (e * e) * (ase / e - s)
    A3 = 2.0 * s / (e * e) * (1.0 / s - ase / e)
    return I, A1, A3


def spheroid_lambda(rperp2, z2, a1, a3):
    """Positive root of r_perp^2/(a1^2+lam) + z^2/(a3^2+lam) = 1 (exterior points)."""
    b = a1 * a1 + a3 * a3 - rperp2 - z2
    c = a1 * a1 * a3 * a3 - rperp2 * a3 * a3 - z2 * a1 * a1
    disc = np.sqrt(b * b - 4.0 * c)
    return np.where(b > 0.0, -2.0 * c / (b + disc), 0.5 * (-b + disc))


def spheroid_potential(rperp, z, a1, a3, rho, G=1.0):
    """Potential of a homogeneous oblate spheroid (a1 >= a3) at (r_perp, z)."""
    rperp = np.asarray(rperp, float)
    z = np.asarray(z, float)
    rp2, z2 = rperp * rperp, z * z
    inside = rp2 / a1 ** 2 + z2 / a3 ** 2 <= 1.0
    e = math.sqrt(max(0.0, 1.0 - a3 * a3 / (a1 * a1)))
    I, A1, A3 = spheroid_coefficients(e)
    phi_in = -math.pi * G * rho * (I * a1 * a1 - A1 * rp2 - A3 * z2)
    lam = spheroid_lambda(rp2, z2, a1, a3)
    lam = np.where(inside, 0.0, lam)
    a1p2 = a1 * a1 + lam
    a3p2 = a3 * a3 + lam
    ep = np.sqrt(np.clip(1.0 - a3p2 / a1p2, 0.0, None))
    coef = np.vectorize(spheroid_coefficients, otypes=[float, float, float])(ep)
    Ip, A1p, A3p = coef
    phi_out = -math.pi * G * rho * (a1 * a1 * a3) / (a1p2 * np.sqrt(a3p2)) * (Ip * a1p2 - A1p * rp2 - A3p * z2)
    return np.where(inside, phi_in, phi_out)


def sphere_potential(r, R, rho, G=1.0):
    r = np.asarray(r, float)
    return np.where(r <= R, -2.0 * math.pi * G * rho * (R * R - r * r / 3.0),
                    -4.0 * math.pi * G * rho * R ** 3 / (3.0 * np.maximum(r, 1e-300)))


def legendre_p(l: int, x):
    """Legendre polynomial P_l(x) by Bonnet's recursion."""
    x = np.asarray(x, float)
    p0, p1 = np.ones_like(x), x.copy()
    if l == 0:
        return p0
    for n in range(1, l):
        p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
    return p1


def gauss_nodes(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def cell_quadrature(r0, r1, t0, t1, p0, p1, n):
    """Cartesian points and volume weights of an n^3 Gauss rule on a spherical cell."""
    rr, wr = gauss_nodes(r0, r1, n)
    tt, wt = gauss_nodes(t0, t1, n)
    pp, wp = gauss_nodes(p0, p1, n)
    R, T, P = np.meshgrid(rr, tt, pp, indexing="ij")
    W = (wr[:, None, None] * wt[None, :, None] * wp[None, None, :]) * R * R * np.sin(T)
    X = np.stack([R * np.sin(T) * np.cos(P), R * np.sin(T) * np.sin(P), R * np.cos(T)], axis=-1)
    return X.reshape(-1, 3), W.reshape(-1)


def direct_cell_average_potential(r, th, ph, rho, target_cells, G=1.0, n_src=4, n_tgt=4):
    """Cell-volume average of Phi(x) = -G sum_c' rho_c' int_c' dV'/|x - x'| over each
    target cell (i, j, k); sources are the cells with rho != 0.  Only meaningful
    when no target cell overlaps a source cell (the integrand is then smooth)."""
    src_pts, src_w = [], []
    n_r, n_t, n_p = rho.shape
    for i in range(n_r):
        for j in range(n_t):
            for k in range(n_p):
                if rho[i, j, k] != 0.0:
                    X, Wt = cell_quadrature(r[i], r[i + 1], th[j], th[j + 1], ph[k], ph[k + 1], n_src)
                    src_pts.append(X)
                    src_w.append(Wt * rho[i, j, k])
    S = np.concatenate(src_pts)
    SW = np.concatenate(src_w)
    out = []
    for (i, j, k) in target_cells:
        X, Wt = cell_quadrature(r[i], r[i + 1], th[j], th[j + 1], ph[k], ph[k + 1], n_tgt)
        d = np.sqrt(((X[:, None, :] - S[None, :, :]) ** 2).sum(-1))
        pot = -G * (SW[None, :] / d).sum(1)
        out.append(np.sum(pot * Wt) / np.sum(Wt))
    return np.asarray(out)
