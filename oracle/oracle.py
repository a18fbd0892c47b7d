"""Python front of the FP64 CPU oracle of the multipole Poisson solve.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the CUDA product path never imports it.

Every function follows GenASiS II, Sec. 2.2 (see ``multipole_oracle.c`` for the
equation each C routine restates and for the readings R1-R7 where the paper
is silent).  Pins (tests that tie each function to something other than
itself):

* ``legendre``            -- closed forms of P~_0^0, P~_1^0, P~_1^1, the textbook
                             associated Legendre routine (scipy), the addition
                             theorem.
* ``theta_integrals``     -- adaptive quadrature (scipy.integrate.quad),
                             sum over a full polar range equals the closed
                             form of int P~_l^0 d(mu), orthonormality.
* ``phi_integrals``       -- closed-form antiderivatives of cos, sin.
* ``radial_integrals``    -- Gauss-Legendre quadrature of r^(l+2), r^(1-l).
* ``solve``               -- l = 0 enclosed-mass invariant, exact discrete
                             exterior / cavity potentials of shell-constant
                             densities, dense Green's matrix brute force,
                             literal vs factored sums, linearity, z-rotation,
                             mirror symmetry, r_ref invariance, direct
                             Green's-function quadrature converging in L,
                             homogeneous sphere / spheroid closed forms.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None
_dptr = ctypes.POINTER(ctypes.c_double)
_iptr = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d, i = ctypes.c_double, ctypes.c_int
        lib.orc_legendre_xs.argtypes = [i, d, d, _dptr]
        lib.orc_legendre_xs.restype = i
        lib.orc_theta_integrals.argtypes = [i, i, _dptr, d, _dptr, _iptr]
        lib.orc_theta_integrals.restype = i
        lib.orc_phi_integrals.argtypes = [i, i, _dptr, d, _dptr, _iptr]
        lib.orc_phi_integrals.restype = i
        lib.orc_radial.argtypes = [i, i, _dptr, d, _dptr, _dptr, _dptr]
        lib.orc_radial.restype = i
        lib.orc_default_r_ref.argtypes = [i, _dptr]
        lib.orc_default_r_ref.restype = d
        lib.orc_solve.argtypes = [i, i, i, i, _dptr, _dptr, _dptr, _dptr, _dptr, _dptr, _dptr,
                                  _dptr, d, _dptr, i, _dptr, _dptr, _dptr, _dptr, _dptr]
        lib.orc_solve.restype = i
        lib.orc_potential_shells.argtypes = [i, i, i, i, _dptr, _dptr, _dptr, _dptr, _dptr, i,
                                             _iptr, _dptr]
        lib.orc_potential_shells.restype = None
        lib.orc_potential_green.argtypes = [i, i, i, i, _dptr, _dptr, _dptr, _dptr, _dptr, _dptr,
                                            _dptr, _dptr, d, _dptr, _dptr]
        lib.orc_potential_green.restype = None
        lib.orc_set_threads.argtypes = [i]
        lib.orc_set_threads.restype = None
        lib.orc_get_threads.argtypes = []
        lib.orc_get_threads.restype = i
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dptr)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (0 = OpenMP default)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def tri(l: int, m: int) -> int:
    """Legendre triangle index t(l, m)."""
    return l * (l + 1) // 2 + m


def pcol(m: int, a: int) -> int:
    """Real moment column p(m, a): (0,c) -> 0, (m,c) -> 2m-1, (m,s) -> 2m."""
    return 0 if m == 0 else 2 * m - 1 + a


def qidx(l: int, m: int, a: int) -> int:
    """Moment index q(l, m, a) = l^2 + p(m, a)."""
    return l * l + pcol(m, a)


def legendre(L: int, x: float, s: float | None = None) -> np.ndarray:
    """P~_l^m(x) for all 0 <= m <= l <= L, indexed by tri(l, m) (Sec. 2.2)."""
    if s is None:
        s = np.sqrt((1.0 - x) * (1.0 + x))
    out = np.zeros((L + 1) * (L + 2) // 2)
    rc = _load().orc_legendre_xs(int(L), float(x), float(s), _p(out))
    if rc != 0:
        raise ValueError(f"oracle Legendre recursion supports 0 <= L <= 85, got {L}")
    return out


def theta_integrals(L: int, theta_edges, tol: float = 1e-14) -> np.ndarray:
    """Ith[t(l,m), j] = int P~_l^m(cos th) sin th dth over polar cell j (Romberg)."""
    th = _c(theta_edges)
    n_t = th.size - 1
    out = np.zeros(((L + 1) * (L + 2) // 2, n_t))
    lev = ctypes.c_int(0)
    rc = _load().orc_theta_integrals(int(L), n_t, _p(th), float(tol), _p(out), ctypes.byref(lev))
    if rc != 0:
        raise RuntimeError(f"Romberg theta integrals failed (rc={rc})")
    return out


def phi_integrals(L: int, phi_edges, tol: float = 1e-14) -> np.ndarray:
    """Iph[p(m,a), k] = int cos|sin(m phi) dphi over azimuthal cell k (Romberg)."""
    ph = _c(phi_edges)
    n_p = ph.size - 1
    out = np.zeros((2 * L + 1, n_p))
    lev = ctypes.c_int(0)
    rc = _load().orc_phi_integrals(int(L), n_p, _p(ph), float(tol), _p(out), ctypes.byref(lev))
    if rc != 0:
        raise RuntimeError(f"Romberg phi integrals failed (rc={rc})")
    return out


def default_r_ref(r_edges) -> float:
    r = _c(r_edges)
    return float(_load().orc_default_r_ref(r.size - 1, _p(r)))


def radial_integrals(L: int, r_edges, r_ref: float | None = None):
    """(WR[l,i], WI[l,i], V[i]): shell integrals of r^2 (r/r_ref)^l, r^2 r_ref^l / r^(l+1), r^2."""
    r = _c(r_edges)
    n_r = r.size - 1
    if r_ref is None:
        r_ref = default_r_ref(r)
    WR = np.zeros((L + 1, n_r))
    WI = np.zeros((L + 1, n_r))
    V = np.zeros(n_r)
    rc = _load().orc_radial(int(L), n_r, _p(r), float(r_ref), _p(WR), _p(WI), _p(V))
    if rc != 0:
        raise ValueError("bad radial arguments")
    return WR, WI, V


@dataclass
class Tables:
    """Per-mesh tables of the oracle (computed once, as the paper stores them)."""
    r: np.ndarray
    theta: np.ndarray
    phi: np.ndarray
    L: int
    r_ref: float
    Ith: np.ndarray
    Iph: np.ndarray
    WR: np.ndarray
    WI: np.ndarray
    V: np.ndarray

    @property
    def shape(self):
        return (self.r.size - 1, self.theta.size - 1, self.phi.size - 1)

    @property
    def KL(self):
        return (self.L + 1) ** 2


def build_tables(r_edges, theta_edges, phi_edges, L: int, r_ref: float | None = None,
                 tol: float = 1e-14) -> Tables:
    r, th, ph = _c(r_edges), _c(theta_edges), _c(phi_edges)
    if r_ref is None:
        r_ref = default_r_ref(r)
    WR, WI, V = radial_integrals(L, r, r_ref)
    return Tables(r=r, theta=th, phi=ph, L=int(L), r_ref=float(r_ref),
                  Ith=theta_integrals(L, th, tol), Iph=phi_integrals(L, ph, tol), WR=WR, WI=WI, V=V)


def solve(tab: Tables, rho, G: float, literal: bool = False, want_phi: bool = True) -> dict:
    """Full multipole solve: moments A[i,q], edge moments MR/MI[n_r+1,q],
    solution coefficients C[i,q] and potential phi[i,j,k]."""
    n_r, n_t, n_p = tab.shape
    rho = _c(rho).reshape(n_r, n_t, n_p)
    KL = tab.KL
    A = np.zeros((n_r, KL))
    MR = np.zeros((n_r + 1, KL))
    MI = np.zeros((n_r + 1, KL))
    C = np.zeros((n_r, KL))
    phi = np.zeros((n_r, n_t, n_p)) if want_phi else None
    rc = _load().orc_solve(n_r, n_t, n_p, tab.L, _p(tab.r), _p(tab.theta), _p(tab.phi),
                           _p(tab.Ith), _p(tab.Iph), _p(tab.WR), _p(tab.WI), _p(tab.V),
                           float(G), _p(rho), int(bool(literal)), _p(A), _p(MR), _p(MI), _p(C),
                           _p(phi) if want_phi else ctypes.cast(None, _dptr))
    if rc != 0:
        raise ValueError("oracle solve rejected its arguments")
    return {"A": A, "MR": MR, "MI": MI, "C": C, "phi": phi}


def potential_shells(tab: Tables, C: np.ndarray, shells) -> np.ndarray:
    """Potential of the listed shells only, from the coefficients of ``solve``."""
    n_r, n_t, n_p = tab.shape
    sel = np.ascontiguousarray(np.asarray(shells, dtype=np.int32))
    out = np.zeros((sel.size, n_t, n_p))
    C = _c(C)
    _load().orc_potential_shells(n_r, n_t, n_p, tab.L, _p(tab.theta), _p(tab.phi), _p(tab.Ith),
                                 _p(tab.Iph), _p(C), int(sel.size),
                                 sel.ctypes.data_as(_iptr), _p(out))
    return out


def green_matrix_potential(tab: Tables, rho, G: float) -> np.ndarray:
    """Dense O(N^2 K_L) restatement of the discrete solve without recurrences."""
    n_r, n_t, n_p = tab.shape
    rho = _c(rho).reshape(n_r, n_t, n_p)
    phi = np.zeros((n_r, n_t, n_p))
    _load().orc_potential_green(n_r, n_t, n_p, tab.L, _p(tab.r), _p(tab.theta), _p(tab.phi),
                                _p(tab.Ith), _p(tab.Iph), _p(tab.WR), _p(tab.WI), _p(tab.V),
                                float(G), _p(rho), _p(phi))
    return phi
