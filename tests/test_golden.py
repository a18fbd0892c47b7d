"""Values the paper prints for worked examples (tests/golden/paper_values.txt)."""
import math
import os

import numpy as np
import pytest

import analytic as A
from paper_2602_02507_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val, digits = line.split()[:3]
            out[key] = (float(val), int(digits))
    return out


GOLD = _golden()


def _agrees(x, key):
    val, digits = GOLD[key]
    return float(f"{x:.{digits - 1}e}") == pytest.approx(val, rel=1e-12)


def test_spheroid_axes_from_mass():
    """M = 4/3 pi a1^2 a3 rho with a3 = a1 sqrt(1 - e^2)."""
    e, rho, M = 0.9, 1e-3, 1.0
    a1 = (3 * M / (4 * math.pi * rho * math.sqrt(1 - e * e))) ** (1 / 3)
    a3 = a1 * math.sqrt(1 - e * e)
    assert _agrees(a1, "spheroid_e09_a1")
    assert _agrees(a3, "spheroid_e09_a3")
    # the closed form is continuous across the surface and matches the
    # point-mass field far away
    phi_in = A.spheroid_potential(a1 * (1 - 1e-12), 0.0, a1, a3, rho)
    phi_out = A.spheroid_potential(a1 * (1 + 1e-12), 0.0, a1, a3, rho)
    assert float(phi_in) == pytest.approx(float(phi_out), rel=1e-9)
    far = A.spheroid_potential(1e4, 3e3, a1, a3, rho)
    assert float(far) == pytest.approx(-M / math.hypot(1e4, 3e3), rel=1e-6)


@pytest.mark.parametrize("n_theta,r_core,rr,kd,ko", [
    (256, 0.25, 3.68, "mesh_dr_min_256", "mesh_r_out_256"),
    (192, 0.25, 3.68, "mesh_dr_min_192", "mesh_r_out_192"),
    (192, 16.0, 5.9, "mesh_dr_min_phys", "mesh_r_out_phys"),
])
def test_mesh_rule(n_theta, r_core, rr, kd, ko):
    e = W.paper_radial_edges(n_theta, r_core, rr)
    assert _agrees(e[1] - e[0], kd)
    assert _agrees(e[-1], ko)


def test_coarsening_gains_use_first_cell_midpoint():
    n_theta = 192
    e = W.paper_radial_edges(n_theta, 16.0, 5.9)
    dr = e[1] - e[0]
    r_min = 0.5 * dr
    dth = math.pi / n_theta
    assert _agrees(dr / (r_min * dth), "coarsening_gain_2d")
    assert _agrees(dr / (r_min * math.sin(0.5 * dth) * dth), "coarsening_gain_3d")
    assert _agrees(math.pi * (25 * 128 // 32) / 128, "core_aspect_ratio")
