"""FP64 CPU oracle of the gravitational source terms of the fluid equations.

TEST INFRASTRUCTURE ONLY: the test suite and the benchmark's CPU-baseline leg use
it; the CUDA product path never imports it.

GenASiS II, Sec. 3, Eq. (BalancedVariablesGravitational): the potential enters
the balance equations of the fluid through the momentum source -rho grad(Phi)
(a covector: its components are rho times the coordinate derivatives
d(Phi)/dr, d(Phi)/dtheta, d(Phi)/dphi, negated) and the energy source
-rho v . grad(Phi) (v the contravariant 3-velocity).  The paper takes each
component of grad(Phi) as the simplest centred difference, the one formed from
the two nearest neighbours along that coordinate.

Readings where the paper is silent (listed with R13 in the design notes):

* Phi lives at cell centres, the coordinate midpoints of the cell edges (the
  midpoint reading of the Poisson solver), so the difference along x is
  (Phi[i+1] - Phi[i-1]) / (x_c[i+1] - x_c[i-1]) on any (non-uniform) mesh.
* phi is periodic when the azimuthal edges span 2 pi: the neighbours of the
  first and last azimuthal cells wrap around, their coordinate shifted by 2 pi.
  With one azimuthal cell the phi derivative is zero; with two, both neighbours
  are the same cell and the difference is zero.  A mesh spanning less than 2 pi
  is treated like r and theta at its ends.
* At the first and last cell along r and theta the two nearest cells along that
  coordinate are the cell itself and its one neighbour: a one-sided difference.
  With one cell along the coordinate the derivative is zero.

Pins (tests/test_oracle_gravity.py): a potential linear in r_c has the exact
derivative everywhere, edges included; -1/r_c on a geometric mesh has the
closed-form interior difference 1/(r_c[i+1] r_c[i-1]); cos(phi_c) and
cos(theta_c) on uniform meshes have the closed forms -sin(x) sin(h)/h (the
azimuthal wrap included) and the one-sided edge values (also at the ends of an
azimuthal range short of 2 pi); a potential of r alone
gives zero theta and phi components and E = v^r S_r; one cell along an axis
gives a zero component.
"""
from __future__ import annotations

import numpy as np


def centres(edges) -> np.ndarray:
    """Cell-centre coordinates: midpoints of consecutive edges."""
    e = np.asarray(edges, dtype=np.float64)
    return 0.5 * (e[:-1] + e[1:])


def stencil(edges, periodic: bool):
    """Per cell along one axis: indices (lo, hi) of the two cells the difference
    uses and the coordinate distance x_c[hi] - x_c[lo] between them (0 where the
    derivative is zero: a single cell, or two azimuthal cells)."""
    xc = centres(edges)
    n = xc.size
    lo = np.empty(n, dtype=np.int64)
    hi = np.empty(n, dtype=np.int64)
    dx = np.zeros(n)
    if n == 1:
        lo[0] = hi[0] = 0
        return lo, hi, dx
    period = float(np.asarray(edges, dtype=np.float64)[-1] - np.asarray(edges, dtype=np.float64)[0])
    for i in range(n):
        if periodic:
            lo[i], hi[i] = (i - 1) % n, (i + 1) % n
            x_lo = xc[lo[i]] - (period if i == 0 else 0.0)
            x_hi = xc[hi[i]] + (period if i == n - 1 else 0.0)
            dx[i] = 0.0 if lo[i] == hi[i] else x_hi - x_lo
        else:
            lo[i], hi[i] = max(i - 1, 0), min(i + 1, n - 1)
            dx[i] = xc[hi[i]] - xc[lo[i]]
    return lo, hi, dx


def gradient(phi, r_edges, theta_edges, phi_edges) -> np.ndarray:
    """[3][n_r][n_theta][n_phi]: d(Phi)/dr, d(Phi)/dtheta, d(Phi)/dphi by the
    centred difference over the two nearest cells along each coordinate."""
    phi = np.asarray(phi, dtype=np.float64)
    out = np.zeros((3,) + phi.shape)
    pe = np.asarray(phi_edges, dtype=np.float64)
    full_circle = abs((pe[-1] - pe[0]) - 2.0 * np.pi) <= 1e-12 * 2.0 * np.pi
    for axis, (edges, periodic) in enumerate(((r_edges, False), (theta_edges, False), (phi_edges, full_circle))):
        lo, hi, dx = stencil(edges, periodic)
        for i in range(lo.size):
            if dx[i] == 0.0:
                continue
            sel_hi = [slice(None)] * 3
            sel_lo = [slice(None)] * 3
            sel_out = [slice(None)] * 3
            sel_hi[axis], sel_lo[axis], sel_out[axis] = hi[i], lo[i], i
            out[axis][tuple(sel_out)] = (phi[tuple(sel_hi)] - phi[tuple(sel_lo)]) / dx[i]
    return out


def sources(phi, rho, v, r_edges, theta_edges, phi_edges) -> dict:
    """The momentum source S_a = -rho d(Phi)/dx^a (covariant components) and, when
    the contravariant velocity v [3][...] is given, the energy source
    E = -rho (v^r d_r Phi + v^theta d_theta Phi + v^phi d_phi Phi)."""
    g = gradient(phi, r_edges, theta_edges, phi_edges)
    rho = np.asarray(rho, dtype=np.float64)
    out = {"grad": g, "S": -rho[None] * g}
    if v is not None:
        v = np.asarray(v, dtype=np.float64)
        out["E"] = -rho * (v[0] * g[0] + v[1] * g[1] + v[2] * g[2])
    return out
