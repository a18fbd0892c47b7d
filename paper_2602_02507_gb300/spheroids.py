"""Convergence study of the homogeneous spheroids of GenASiS II Sec. 3.1 on the GPU solver.

The paper measures its multipole solver on homogeneous oblate spheroids of
density rho = 1e-3 and mass M = 1 (G = 1) with eccentricities 0, 0.3, 0.6 and
0.9: the L1 error (Sec. 3, Eq. (L1error): sum |Phi - Phi_0| / sum |Phi_0| over the
cells) of the potential against the closed form, Eq. (SpheroidPotential), as a
function of resolution at L = 20 and as a function of L at N_theta = 384.  The
meshes follow the rule of Sec. 2.1 with the dimensionless set-up of Sec. 3:
N_core = 25/32 N_theta uniform shells inside r_core = 0.25, Delta r proportional
to r outside, N_r = 3.68 N_theta shells, N_phi = 2 N_theta (``dims=3``) or one
azimuthal cell over 2 pi (``dims=2``: the spheroid is axisymmetric, so every
m >= 1 moment vanishes and the 2-D mesh gives the 3-D potential).

Cells cut by the spheroid's surface carry their exact volume fraction
(``workloads.spheroid_fraction_exact``; a sub-cell estimate of the fraction puts
mass errors of order 1e-3 into the density, which would hide the solver's
convergence); Phi_0 is evaluated at cell centres, the coordinate midpoints.
The paper's figure of this study is not available as numbers, so the study
reproduces its set-up, not its values.

    python -m paper_2602_02507_gb300.spheroids --nthetas 32 64 128 256 384 --ls 0 2 4 8 12 16 20
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads as W

R_CORE = 0.25
R_RADIAL = 3.68
RHO = 1e-3
MASS = 1.0


def axes(e: float, rho: float = RHO, mass: float = MASS):
    """Semi-axes (a1, a3) of the oblate spheroid of eccentricity e, density rho and
    mass M: (4/3) pi a1^2 a3 rho = M with a3 = a1 sqrt(1 - e^2)."""
    a1 = (3.0 * mass / (4.0 * math.pi * rho * math.sqrt(1.0 - e * e))) ** (1.0 / 3.0)
    return a1, a1 * math.sqrt(1.0 - e * e)


def coefficients(e):
    """(I, A1, A3) of Eq. (SpheroidPotential) for eccentricity e (array or scalar).
    Below e = 0.05 the closed forms cancel: there their Taylor series in e^2 is used
    (from asin(e)/e = 1 + e^2/6 + 3e^4/40 + 5e^6/112 and the binomial series of
    sqrt(1 - e^2)); at e = 0 both give the sphere's (2, 2/3, 2/3)."""
    e = np.asarray(e, dtype=np.float64)
    s = np.sqrt(1.0 - e * e)
    small = e < 0.05
    es = np.where(small, 0.1, e)  # keeps the closed forms finite where the series is used
    g = np.arcsin(es) / es
    I_c = 2.0 * s * g
    A1_c = s / (es * es) * (g - s)
    A3_c = 2.0 / (es * es) * (1.0 - s * g)
    e2 = e * e
    I_s = 2.0 * (1.0 - e2 / 3.0 - 2.0 * e2 ** 2 / 15.0 - 8.0 * e2 ** 3 / 105.0)
    A1_s = s * (2.0 / 3.0 + e2 / 5.0 + 3.0 * e2 ** 2 / 28.0 + 5.0 * e2 ** 3 / 72.0)
    A3_s = 2.0 - 2.0 * A1_s  # 2 A1 + A3 = 2 for every e
    return (np.where(small, I_s, I_c), np.where(small, A1_s, A1_c), np.where(small, A3_s, A3_c))


def potential(r_perp, z, a1: float, a3: float, rho: float = RHO, G: float = 1.0):
    """Eq. (SpheroidPotential): the interior quadratic form, and outside the exterior
    form with a'_i^2 = a_i^2 + lambda, lambda the positive root of
    r_perp^2 / (a1^2 + lambda) + z^2 / (a3^2 + lambda) = 1."""
    rp2 = np.asarray(r_perp, dtype=np.float64) ** 2
    z2 = np.asarray(z, dtype=np.float64) ** 2
    inside = rp2 / a1 ** 2 + z2 / a3 ** 2 <= 1.0
    e = math.sqrt(max(0.0, 1.0 - (a3 / a1) ** 2))
    I, A1, A3 = (float(x) for x in coefficients(e))
    phi_in = -math.pi * G * rho * (I * a1 * a1 - A1 * rp2 - A3 * z2)
    # lambda^2 + b lambda + c = 0; c < 0 outside, so one positive root, taken without cancellation
    b = a1 * a1 + a3 * a3 - rp2 - z2
    c = a1 * a1 * a3 * a3 - rp2 * a3 * a3 - z2 * a1 * a1
    root = np.sqrt(np.maximum(b * b - 4.0 * c, 0.0))
    lam = np.where(b > 0.0, -2.0 * c / np.where(b + root > 0.0, b + root, 1.0), 0.5 * (root - b))
    lam = np.where(inside, 0.0, lam)
    a1p2, a3p2 = a1 * a1 + lam, a3 * a3 + lam
    ep = np.sqrt(np.clip(1.0 - a3p2 / a1p2, 0.0, None))
    Ip, A1p, A3p = coefficients(ep)
    phi_out = -math.pi * G * rho * (a1 * a1 * a3) / (a1p2 * np.sqrt(a3p2)) * (Ip * a1p2 - A1p * rp2 - A3p * z2)
    return np.where(inside, phi_in, phi_out)


def density(mesh: W.Mesh, a1: float, a3: float, rho: float = RHO) -> np.ndarray:
    """rho times the volume fraction of each cell inside the spheroid, [n_r][n_theta][n_phi]."""
    frac = W.spheroid_fraction_exact(mesh.r, mesh.theta, a1, a3)
    n_p = mesh.phi.size - 1
    return np.ascontiguousarray(np.repeat((rho * frac)[:, :, None], n_p, axis=2))


def exact_at_centres(mesh: W.Mesh, a1: float, a3: float, rho: float = RHO) -> np.ndarray:
    """Phi_0 at the cells' coordinate midpoints, [n_r][n_theta] (independent of phi)."""
    rc, tc = W.midpoints(mesh.r), W.midpoints(mesh.theta)
    return potential(rc[:, None] * np.sin(tc)[None, :], rc[:, None] * np.cos(tc)[None, :], a1, a3, rho)


def l1_error(phi: np.ndarray, phi0_rt: np.ndarray) -> float:
    """Eq. (L1error) over all cells; phi [n_r][n_theta][n_phi], phi0 [n_r][n_theta]."""
    diff = np.abs(phi - phi0_rt[:, :, None]).sum()
    return float(diff / (np.abs(phi0_rt).sum() * phi.shape[2]))


def run(nthetas, ls, eccentricities=(0.0, 0.3, 0.6, 0.9), dims: int = 2, precision: str = "fp64",
        n_theta_for_l: int | None = None, l_for_n: int = 20):
    """The two sweeps: L1 vs N_theta at L = l_for_n, and L1 vs L at N_theta = n_theta_for_l
    (default: the largest N_theta).  Returns a list of records."""
    import torch
    from . import multipole as mpl
    n_theta_for_l = n_theta_for_l or max(nthetas)
    jobs = {}
    for n in nthetas:
        jobs.setdefault(n, set()).add(l_for_n)
    for L in ls:
        jobs.setdefault(n_theta_for_l, set()).add(L)
    out = []
    for n_theta in sorted(jobs):
        base = W.paper_mesh(n_theta, R_CORE, R_RADIAL, 0, dims)
        for e in eccentricities:
            a1, a3 = axes(e)
            rho_np = density(base, a1, a3)
            phi0 = exact_at_centres(base, a1, a3)
            rho = torch.from_numpy(rho_np.reshape(-1)).cuda()
            phi = torch.empty_like(rho)
            for L in sorted(jobs[n_theta]):
                with mpl.Mesh(base.r, base.theta, base.phi, L, 1.0, precision=precision) as mesh:
                    mesh.set_density(rho)
                    mesh.set_phi_output(phi)
                    mesh.solve()
                    mesh.synchronize()
                    t0 = time.perf_counter()
                    mesh.solve()
                    mesh.synchronize()
                    dt = time.perf_counter() - t0
                err = l1_error(phi.cpu().numpy().reshape(rho_np.shape), phi0)
                out.append({"e": e, "n_theta": n_theta, "n_r": base.r.size - 1, "n_phi": base.phi.size - 1,
                            "inv_dr_min": 1.0 / (base.r[1] - base.r[0]), "L": L, "l1": err,
                            "solve_s": dt, "precision": precision, "dims": dims})
    return out


def _table(records, key, fixed_name, fixed_value):
    es = sorted({r["e"] for r in records})
    rows = sorted({r[key] for r in records if r[fixed_name] == fixed_value})
    lines = [f"| {key} | " + " | ".join(f"e = {e:g}" for e in es) + " |",
             "|---:|" + "---:|" * len(es)]
    for v in rows:
        vals = []
        for e in es:
            m = [r["l1"] for r in records if r["e"] == e and r[key] == v and r[fixed_name] == fixed_value]
            vals.append(f"{m[0]:.3e}" if m else "")
        lines.append(f"| {v} | " + " | ".join(vals) + " |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--nthetas", type=int, nargs="+", default=[32, 48, 64, 96, 128, 192, 256, 384])
    ap.add_argument("--ls", type=int, nargs="+", default=[0, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
    ap.add_argument("--eccentricities", type=float, nargs="+", default=[0.0, 0.3, 0.6, 0.9])
    ap.add_argument("--dims", type=int, default=2, choices=(2, 3))
    ap.add_argument("--precision", default="fp64", choices=("fp64", "bf16x3", "bf16x6"))
    ap.add_argument("--json", default=None, help="write the records to this file")
    a = ap.parse_args(argv)
    rec = run(a.nthetas, a.ls, a.eccentricities, a.dims, a.precision)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rec, f, indent=1)
    nmax = max(a.nthetas)
    print(f"L1 error of Phi vs N_theta at L = 20 ({a.dims}-D, {a.precision}):")
    print(_table(rec, "n_theta", "L", 20))
    print(f"\nL1 error of Phi vs L at N_theta = {nmax}:")
    print(_table(rec, "L", "n_theta", nmax))


if __name__ == "__main__":
    main()
