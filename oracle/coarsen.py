"""FP64 CPU oracle of coarsening-block averaging (GenASiS II Sec. 2.1 and Sec. 2.3).

TEST INFRASTRUCTURE ONLY: the test suite uses it; the CUDA product path never
imports it.

Sec. 2.1: where angular cell widths fall below the minimum radial width
Delta r_min, cells are grouped into angular blocks at each radius and fields are
averaged over the blocks.  Sec. 2.3 states the average: each cell of a block
takes the volume-weighted mean sum_j V_j K_j / sum_j V_j of the block, which
conserves the block's integral.

Reading (R15 in the design notes; the paper shows the blocks only in figures):

* Delta r_min is the smallest radial cell width of the mesh; widths are taken
  at the cell-centre radius r_c (the coordinate midpoint).
* Polar blocks at shell i: consecutive runs of p polar cells, p the smallest
  power of two dividing n_theta with p r_c min(Delta theta) >= Delta r_min;
  when none does, the whole polar range is one block.
* Azimuthal blocks within a polar block: runs of q azimuthal cells, q the
  smallest power of two dividing n_phi with
  q r_c sin(theta_c) min(Delta phi) >= Delta r_min, theta_c the centre of the
  block's polar cell nearest the axis; when none does, the whole ring.
* Cell volumes are separable, V = dV_r(i) dmu_j dphi_k with dmu the difference
  of cos(theta) over the cell, so within a shell the weights are dmu_j dphi_k.

The required (real-valued) factors Delta r_min / (r_c Delta theta) and
Delta r_min / (r_c sin(theta_c) Delta phi) at the first shell and polar cell are
the time-step gains the paper prints for its physical mesh (Sec. 3).

Pins (tests/test_oracle_coarsen.py): those printed gains; a field constant on
every block is unchanged; the volume integral of every shell is conserved;
the result is constant on each block; cells wide enough are left alone;
a brute-force mean over the cells of one hand-picked block.
"""
from __future__ import annotations

import math

import numpy as np


def _centres(e):
    e = np.asarray(e, dtype=np.float64)
    return 0.5 * (e[:-1] + e[1:])


def required_factors(r_edges, theta_edges, phi_edges):
    """Real-valued ratios Delta r_min / (r_c dtheta_min) [n_r] and
    Delta r_min / (r_c sin(theta_c) dphi_min) [n_r][n_theta]."""
    r = np.asarray(r_edges, dtype=np.float64)
    dr_min = float(np.min(np.diff(r)))
    rc = _centres(r)
    tc = _centres(theta_edges)
    dth = float(np.min(np.diff(np.asarray(theta_edges, dtype=np.float64))))
    dph = float(np.min(np.diff(np.asarray(phi_edges, dtype=np.float64))))
    polar = dr_min / (rc * dth)
    azim = dr_min / (rc[:, None] * np.sin(tc)[None, :] * dph)
    return polar, azim


def _pow2_block(need: float, n: int) -> int:
    p = 1
    while p <= n:
        if n % p == 0 and p >= need:
            return p
        p *= 2
    return n


def factors(r_edges, theta_edges, phi_edges):
    """Block sizes: c_theta [n_r] and c_phi [n_r][n_theta] (the azimuthal size of the
    polar block each polar cell belongs to)."""
    n_t = len(theta_edges) - 1
    n_p = len(phi_edges) - 1
    polar, azim = required_factors(r_edges, theta_edges, phi_edges)
    n_r = polar.size
    c_t = np.empty(n_r, dtype=np.int64)
    c_p = np.empty((n_r, n_t), dtype=np.int64)
    for i in range(n_r):
        c_t[i] = _pow2_block(polar[i], n_t)
        for j0 in range(0, n_t, int(c_t[i])):
            need = float(np.max(azim[i, j0:j0 + c_t[i]]))  # the cell nearest the axis needs most
            c_p[i, j0:j0 + c_t[i]] = _pow2_block(need, n_p)
    return c_t, c_p


def coarsen(field, r_edges, theta_edges, phi_edges) -> np.ndarray:
    """Every cell of a block takes the block's volume-weighted mean (Sec. 2.3)."""
    f = np.array(field, dtype=np.float64, copy=True)
    dmu = -np.diff(np.cos(np.asarray(theta_edges, dtype=np.float64)))
    dph = np.diff(np.asarray(phi_edges, dtype=np.float64))
    c_t, c_p = factors(r_edges, theta_edges, phi_edges)
    n_r, n_t, n_p = f.shape
    for i in range(n_r):
        ct = int(c_t[i])
        for j0 in range(0, n_t, ct):
            cp = int(c_p[i, j0])
            if ct == 1 and cp == 1:
                continue
            for k0 in range(0, n_p, cp):
                w = dmu[j0:j0 + ct, None] * dph[None, k0:k0 + cp]
                block = f[i, j0:j0 + ct, k0:k0 + cp]
                f[i, j0:j0 + ct, k0:k0 + cp] = np.sum(w * block) / np.sum(w)
    return f
