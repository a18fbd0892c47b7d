"""Seeded synthetic meshes and densities for the multipole Poisson solve.

This module is the only code shared by the tests' oracle side and the CUDA
side: it builds inputs (mesh edges and a density field) and holds none of the
solve's arithmetic.  Spherical harmonics needed to shape a density come from
scipy's textbook associated-Legendre routine, not from either solver.

Workloads (sizes as the solver's benchmark configurations name them):

* ``spheroid``   homogeneous oblate spheroid a1 = 1, a3 = 0.6 (e = 0.8), rho = 1,
                 G = 1, on 64 uniform shells over [0, 1.5] x 32 polar x 64
                 azimuthal cells, L = 8; cells cut by the surface carry their
                 volume fraction (GenASiS II Sec. 3.1 smooths the spheroid edge
                 with a sub-grid volume fraction; its resolution is unstated,
                 here 16 x 16 sub-cells uniform in (r^3, cos theta)).
* ``presn``      presupernova-like core rho_c / (1 + (r/r_c)^2)^1.5 with
                 rho_c = 1e10 g/cm^3, r_c = 1e8 cm, times
                 (1 + sum_{1<=l<=4, m, a} 1e-2 N(0,1) Y^a_lm), 512 geometric
                 shells over [1e5, 1e10] cm x 128 x 256, L = 16, seed 2.
* ``lognormal``  ln rho = ln rho0(r) + sigma g - sigma^2/2, sigma = 1, g a unit-
                 variance Gaussian angular field with C_l ~ l^-2 (1 <= l <= 64),
                 drawn independently per shell; 1024 geometric shells over
                 [1e5, 1e12] cm x 256 x 512, L = 32, seed 3.
* ``large``      2048 x 512 x 1024 cells, L = 64, presn profile plus l <= 64
                 perturbations of amplitude 1e-3, seed 4.
* ``batch``      64 instances, shapes from {(256,64,128), (512,128,256),
                 (768,192,384), (1024,256,512)}, L from {8, 16, 32}, presn
                 densities with log-uniform rho_c in [1e9, 1e11] and r_c in
                 [5e7, 2e8], seed 5.

Real orthonormal harmonics: Y^c_lm = sqrt(Delta_m) Pbar_l^m(cos th) cos(m phi),
Y^s_lm = sqrt(2) Pbar_l^m(cos th) sin(m phi), with Pbar the unit-sphere-
normalised associated Legendre function (Condon-Shortley phase included).
All densities are evaluated at cell coordinate midpoints.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import special

G_CGS = 6.674e-8
TWO_PI = 2.0 * math.pi


@dataclass
class Mesh:
    r: np.ndarray
    theta: np.ndarray
    phi: np.ndarray
    L: int
    G: float = 1.0
    name: str = ""

    @property
    def shape(self):
        return (self.r.size - 1, self.theta.size - 1, self.phi.size - 1)

    @property
    def cells(self) -> int:
        n_r, n_t, n_p = self.shape
        return n_r * n_t * n_p

    @property
    def KL(self) -> int:
        return (self.L + 1) ** 2


@dataclass
class Workload:
    mesh: Mesh
    rho: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def uniform_edges(lo: float, hi: float, n: int) -> np.ndarray:
    e = lo + (hi - lo) * np.arange(n + 1, dtype=np.float64) / n
    e[0], e[-1] = lo, hi
    return e


def geometric_edges(lo: float, hi: float, n: int) -> np.ndarray:
    e = lo * np.exp(np.log(hi / lo) * np.arange(n + 1, dtype=np.float64) / n)
    e[0], e[-1] = lo, hi
    return e


def angular_edges(n_theta: int, n_phi: int):
    return uniform_edges(0.0, math.pi, n_theta), uniform_edges(0.0, TWO_PI, n_phi)


def paper_radial_edges(n_theta: int, r_core: float, r_radial: float) -> np.ndarray:
    """Radial edges of the GenASiS II mesh rule (Sec. 2.1): N_core = 25/32 N_theta
    uniform cells inside r_core, then cells growing with Delta r proportional to r
    (r_{n+1} = r_n (1 + Delta r_min / r_core)), N_r = R_radial N_theta cells."""
    n_core = (25 * n_theta) // 32
    n_r = int(math.floor(r_radial * n_theta))
    dr_min = r_core / n_core
    e = np.empty(n_r + 1)
    e[: n_core + 1] = dr_min * np.arange(n_core + 1)
    e[n_core] = r_core
    g = 1.0 + dr_min / r_core
    for n in range(n_core, n_r):
        e[n + 1] = e[n] * g
    return e


def paper_mesh(n_theta: int, r_core: float, r_radial: float, L: int, dims: int = 3) -> Mesh:
    """Mesh of the paper's rule: N_phi = 2 N_theta (3-D), or 1 azimuthal cell (2-D)."""
    r = paper_radial_edges(n_theta, r_core, r_radial)
    th = uniform_edges(0.0, math.pi, n_theta)
    ph = uniform_edges(0.0, TWO_PI, 2 * n_theta if dims == 3 else 1)
    return Mesh(r, th, ph, L, 1.0, f"paper-{n_theta}")


def midpoints(e: np.ndarray) -> np.ndarray:
    return 0.5 * (e[:-1] + e[1:])


# --------------------------------------------------------------------------
# real spherical harmonics from scipy (input shaping only)
# --------------------------------------------------------------------------
def _pbar(l: int, m: int, x: np.ndarray) -> np.ndarray:
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))
    return norm * special.lpmv(m, l, x)


def real_ylm_modes(lmin: int, lmax: int):
    """(l, m, a) triples in draw order: l ascending, m ascending, cosine then sine."""
    out = []
    for l in range(lmin, lmax + 1):
        for m in range(0, l + 1):
            out.append((l, m, 0))
            if m > 0:
                out.append((l, m, 1))
    return out


def angular_field(theta_c: np.ndarray, phi_c: np.ndarray, coeffs: dict) -> np.ndarray:
    """sum_{(l,m,a)} coeffs * Y^a_lm(theta_c, phi_c) on the [n_theta, n_phi] grid,
    evaluated as (Legendre part) x (trig part) per m."""
    x = np.cos(theta_c)
    out = np.zeros((theta_c.size, phi_c.size))
    by_m: dict = {}
    for (l, m, a), c in coeffs.items():
        by_m.setdefault((m, a), []).append((l, c))
    for (m, a), terms in by_m.items():
        g = np.zeros(theta_c.size)
        for l, c in terms:
            g += c * _pbar(l, m, x)
        if m == 0:
            trig = np.ones(phi_c.size)
        else:
            trig = math.sqrt(2.0) * (np.cos(m * phi_c) if a == 0 else np.sin(m * phi_c))
        out += np.outer(g, trig)
    return out


# --------------------------------------------------------------------------
# densities
# --------------------------------------------------------------------------
def presn_profile(r_c_mid: np.ndarray, rho_c: float = 1e10, r_c: float = 1e8) -> np.ndarray:
    return rho_c / (1.0 + (r_c_mid / r_c) ** 2) ** 1.5


def spheroid_fraction(r_edges, theta_edges, a1: float, a3: float, sub: int = 16) -> np.ndarray:
    """Volume fraction [n_r, n_theta] of each (axisymmetric) cell inside
    r_perp^2/a1^2 + z^2/a3^2 < 1; sub x sub equal-volume sub-cells uniform in
    (r^3, cos theta) are tested only in cells the surface cuts."""
    r = np.asarray(r_edges, float)
    th = np.asarray(theta_edges, float)
    n_r, n_t = r.size - 1, th.size - 1

    def Rsurf(t):
        return 1.0 / np.sqrt(np.sin(t) ** 2 / a1 ** 2 + np.cos(t) ** 2 / a3 ** 2)

    frac = np.zeros((n_r, n_t))
    for j in range(n_t):
        t0, t1 = th[j], th[j + 1]
        cand = [Rsurf(t0), Rsurf(t1)]
        if t0 < 0.5 * math.pi < t1:
            cand.append(Rsurf(0.5 * math.pi))
        Rmin, Rmax = min(cand), max(cand)
        for i in range(n_r):
            if r[i + 1] <= Rmin:
                frac[i, j] = 1.0
            elif r[i] >= Rmax:
                frac[i, j] = 0.0
            else:
                s = (np.arange(sub) + 0.5) / sub
                rs = np.cbrt(r[i] ** 3 + s * (r[i + 1] ** 3 - r[i] ** 3))
                mus = np.cos(t0) + s * (np.cos(t1) - np.cos(t0))
                rr, mm = np.meshgrid(rs, mus, indexing="ij")
                rperp2 = rr ** 2 * (1.0 - mm ** 2)
                z2 = rr ** 2 * mm ** 2
                frac[i, j] = np.mean(rperp2 / a1 ** 2 + z2 / a3 ** 2 < 1.0)
    return frac


def spheroid_fraction_exact(r_edges, theta_edges, a1: float, a3: float) -> np.ndarray:
    """Exact volume fraction [n_r, n_theta] of each (axisymmetric) cell inside the oblate
    spheroid r_perp^2/a1^2 + z^2/a3^2 < 1 (a1 >= a3).  With mu = cos(theta) the surface
    radius is R(mu) = (A + B mu^2)^(-1/2), A = 1/a1^2, B = 1/a3^2 - 1/a1^2, and the part of
    cell (i, j) inside is (2 pi / 3) int [clamp(R^3, r_i^3, r_{i+1}^3) - r_i^3] d(mu) over
    the cell's mu range.  The clamp changes form where R(mu) = r_i or r_{i+1}
    (mu^2 = (1/r^2 - A) / B); between those points R^3 integrates in closed form,
    int (A + B mu^2)^(-3/2) d(mu) = mu / (A sqrt(A + B mu^2))."""
    r = np.asarray(r_edges, float)
    th = np.asarray(theta_edges, float)
    n_r, n_t = r.size - 1, th.size - 1
    A = 1.0 / (a1 * a1)
    B = 1.0 / (a3 * a3) - A

    def R3(mu):
        return (A + B * mu * mu) ** -1.5

    def F(mu):  # antiderivative of R^3
        return mu / (A * math.sqrt(A + B * mu * mu))

    def crossings(rad):
        if B <= 0.0:
            return []
        m2 = (1.0 / (rad * rad) - A) / B
        if m2 <= 0.0 or m2 >= 1.0:
            return []
        m = math.sqrt(m2)
        return [-m, m]

    frac = np.zeros((n_r, n_t))
    r_in, r_out = a3, a1  # the surface lies between these radii
    for j in range(n_t):
        mu_a, mu_b = sorted((math.cos(th[j]), math.cos(th[j + 1])))
        # surface radii over the cell's polar range: extremes at its ends or at mu = 0
        cand = [R3(mu_a) ** (1 / 3), R3(mu_b) ** (1 / 3)]
        if mu_a < 0.0 < mu_b:
            cand.append(a1)
        Rmin, Rmax = max(min(cand), r_in * (1 - 1e-15)), min(max(cand), r_out * (1 + 1e-15))
        for i in range(n_r):
            lo, hi = r[i], r[i + 1]
            if hi <= Rmin:
                frac[i, j] = 1.0
                continue
            if lo >= Rmax:
                continue
            lo3, hi3 = lo ** 3, hi ** 3
            pts = sorted({mu_a, mu_b, *[m for rad in (lo, hi) if rad > 0.0 for m in crossings(rad)
                                         if mu_a < m < mu_b]})
            vol = 0.0
            for u0, u1 in zip(pts[:-1], pts[1:]):
                mid = R3(0.5 * (u0 + u1))
                if mid <= lo3:
                    continue
                if mid >= hi3:
                    vol += (hi3 - lo3) * (u1 - u0)
                else:
                    vol += F(u1) - F(u0) - lo3 * (u1 - u0)
            frac[i, j] = vol / ((hi3 - lo3) * (mu_b - mu_a))
    return frac


def spheroid(n_r=64, n_theta=32, n_phi=64, L=8, a1=1.0, a3=0.6, rho0=1.0, r_max=1.5) -> Workload:
    r = uniform_edges(0.0, r_max, n_r)
    th, ph = angular_edges(n_theta, n_phi)
    frac = spheroid_fraction(r, th, a1, a3)
    rho = np.ascontiguousarray(np.repeat((rho0 * frac)[:, :, None], n_phi, axis=2))
    return Workload(Mesh(r, th, ph, L, 1.0, "spheroid"), rho, {"a1": a1, "a3": a3, "rho0": rho0})


def presn(n_r=512, n_theta=128, n_phi=256, L=16, seed=2, rho_c=1e10, r_c=1e8,
          r_lo=1e5, r_hi=1e10, amp=1e-2, lmax_pert=4, amp_hi=0.0, lmax_hi=0,
          materialize=True) -> Workload:
    r = geometric_edges(r_lo, r_hi, n_r)
    th, ph = angular_edges(n_theta, n_phi)
    rng = np.random.default_rng(seed)
    coeffs = {mode: amp * rng.standard_normal() for mode in real_ylm_modes(1, lmax_pert)}
    if amp_hi > 0.0:
        for mode in real_ylm_modes(1, lmax_hi):
            coeffs[mode] = coeffs.get(mode, 0.0) + amp_hi * rng.standard_normal()
    ang = 1.0 + angular_field(midpoints(th), midpoints(ph), coeffs)
    prof = presn_profile(midpoints(r), rho_c, r_c)
    rho = None
    if materialize:
        rho = np.ascontiguousarray(prof[:, None, None] * ang[None, :, :])
    return Workload(Mesh(r, th, ph, L, G_CGS, "presn"), rho, {"profile": prof, "angular": ang})


def unit_variance_cl(lmax: int):
    """C_l proportional to l^-2 for 1 <= l <= lmax, scaled so that the real
    field sum a_lm Y_lm with a_lm ~ N(0, C_l) has unit point variance."""
    ls = np.arange(1, lmax + 1)
    cl = ls.astype(float) ** -2
    var = np.sum(cl * (2 * ls + 1) / (4 * math.pi))
    return dict(zip(ls.tolist(), (cl / var).tolist()))


def lognormal(n_r=1024, n_theta=256, n_phi=512, L=32, seed=3, sigma=1.0, lmax_field=64,
              r_lo=1e5, r_hi=1e12) -> Workload:
    r = geometric_edges(r_lo, r_hi, n_r)
    th, ph = angular_edges(n_theta, n_phi)
    thc, phc = midpoints(th), midpoints(ph)
    prof = presn_profile(midpoints(r))
    cl = unit_variance_cl(lmax_field)
    modes = real_ylm_modes(1, lmax_field)
    # Legendre x trig basis once; one coefficient draw per shell.
    x = np.cos(thc)
    cols = []
    leg = np.zeros((len(modes), thc.size))
    trig = np.zeros((len(modes), phc.size))
    for n, (l, m, a) in enumerate(modes):
        leg[n] = _pbar(l, m, x)
        if m == 0:
            trig[n] = 1.0
        else:
            trig[n] = math.sqrt(2.0) * (np.cos(m * phc) if a == 0 else np.sin(m * phc))
        cols.append(math.sqrt(cl[l]))
    sd = np.asarray(cols)
    rho = np.empty((n_r, thc.size, phc.size))
    for i in range(n_r):
        rng = np.random.default_rng([seed, i])
        c = sd * rng.standard_normal(len(modes))
        g = (leg * c[:, None]).T @ trig
        rho[i] = prof[i] * np.exp(sigma * g - 0.5 * sigma * sigma)
    return Workload(Mesh(r, th, ph, L, G_CGS, "lognormal"), rho)


def large(materialize=False, n_r=2048) -> Workload:
    """2048 x 512 x 1024 cells, L = 64; returned as the separable factors
    rho = profile[i] * angular[j, k] unless materialize is set (8.6 GB).  A smaller n_r
    keeps the angular grid, l_max and density recipe (profiling captures of its kernels)."""
    return presn(n_r=n_r, n_theta=512, n_phi=1024, L=64, seed=4, amp=1e-2, lmax_pert=4,
                 amp_hi=1e-3, lmax_hi=64, materialize=materialize)


BATCH_SHAPES = [(256, 64, 128), (512, 128, 256), (768, 192, 384), (1024, 256, 512)]
BATCH_L = [8, 16, 32]


def batch_draws(count=64, seed=5):
    """Per-instance (shape, L, rho_c, r_c) of the batched workload."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        shape = BATCH_SHAPES[int(rng.integers(len(BATCH_SHAPES)))]
        L = BATCH_L[int(rng.integers(len(BATCH_L)))]
        rho_c = float(10.0 ** rng.uniform(9.0, 11.0))
        r_c = float(10.0 ** rng.uniform(math.log10(5e7), math.log10(2e8)))
        out.append((shape, L, rho_c, r_c))
    return out


def batch_instance(n: int, draws=None, seed=5, materialize=True) -> Workload:
    draws = draws or batch_draws(seed=seed)
    (n_r, n_t, n_p), L, rho_c, r_c = draws[n]
    return presn(n_r=n_r, n_theta=n_t, n_phi=n_p, L=L, seed=seed * 1000 + n, rho_c=rho_c, r_c=r_c,
                 materialize=materialize)


def random_small(shape, L, seed=0, r0=0.0, r1=1.0, geometric=False, uneven=False) -> Workload:
    """Small positive random density on a (possibly uneven) mesh, for parity cases."""
    n_r, n_t, n_p = shape
    rng = np.random.default_rng(seed)
    if geometric:
        r = geometric_edges(r0, r1, n_r)
    else:
        r = uniform_edges(r0, r1, n_r)

    def jitter(e):
        if not uneven or e.size < 3:
            return e
        d = np.diff(e) * (1.0 + 0.5 * rng.random(e.size - 1))
        out = np.concatenate([[e[0]], e[0] + np.cumsum(d) * (e[-1] - e[0]) / d.sum()])
        out[-1] = e[-1]
        return out

    r = jitter(r)
    th = jitter(uniform_edges(0.0, math.pi, n_t))
    ph = jitter(uniform_edges(0.0, TWO_PI, n_p))
    rho = 0.5 + rng.random(shape)
    return Workload(Mesh(r, th, ph, L, 1.0, "random"), np.ascontiguousarray(rho))
