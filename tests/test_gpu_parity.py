"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

float64 path: Phi within 1e-12 (pointwise relative), moments within 1e-12 per degree.
split-precision paths: Phi within 1e-6 (pointwise relative).

Meshes keep shells moderately thin: the midpoint split of Eq. (Solution) weighs a
shell's own degree-l moment by about (r_{i+1}/r_i)^l, so on meshes with a few
shells per decade any rounding difference in high-degree moments is amplified
by that factor (the float64 path and the oracle then differ beyond 1e-12 for
reasons of conditioning, not of arithmetic).
"""
import numpy as np
import pytest

from gpu_helpers import (edge_moment_errors, edge_term_errors, gpu_solve, moment_term_errors, oracle_solve,
                         per_l_errors, phi_rel_err, split_moment_bar, term_scales)
from paper_2602_02507_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()


def _axisym():
    w = W.random_small((6, 10, 1), 6, seed=4, r0=0.0, r1=1.0)
    return w


def _one_polar_cell():
    return W.random_small((6, 1, 12), 5, seed=5, r0=0.1, r1=1.0)


FP64_CASES = {
    "spheroid_64x32x64_L8": lambda: W.spheroid(),
    "ragged_7x19x37_L5_origin": lambda: W.random_small((7, 19, 37), 5, seed=1, r0=0.0, r1=2.0, uneven=True),
    "geometric_9x23x40_L9": lambda: W.random_small((9, 23, 40), 9, seed=2, r0=1e5, r1=1e9, geometric=True,
                                                   uneven=True),
    "monopole_L0": lambda: W.random_small((5, 8, 16), 0, seed=3),
    "axisymmetric_nphi1": _axisym,
    "one_polar_cell": _one_polar_cell,
    "presn_64x32x64_L16": lambda: W.presn(n_r=64, n_theta=32, n_phi=64, L=16),
    # more shells than the register-resident scan holds (16 per thread x 128 threads): the
    # general chunked scan
    "long_radial_2100x2x4_L3": lambda: W.random_small((2100, 2, 4), 3, seed=9, r0=1.0, r1=2.0),
    # many moment columns (K_L = 2601): the recurrences take four adjacent columns per block
    "many_moments_40x64x128_L50": lambda: W.presn(n_r=40, n_theta=64, n_phi=128, L=50, r_lo=1e7, r_hi=3e7),
}


@pytest.mark.parametrize("name", list(FP64_CASES))
def test_fp64_path_matches_oracle(name):
    w = FP64_CASES[name]()
    ref = oracle_solve(w)
    got = gpu_solve(w, "fp64")
    assert got["info"]["effective_precision"] == 0
    assert phi_rel_err(got["phi"], ref["phi"]) <= 1e-12
    L = w.mesh.L
    assert max(per_l_errors(got["A"], ref["A"], L)) <= 1e-12
    # edge moments: per degree, against the size of the terms each recurrence adds
    for key, errs in edge_moment_errors(got, ref).items():
        assert max(errs) <= 1e-12, (key, errs)


SPLIT_CASES = {
    "spheroid_64x32x64_L8": (lambda: W.spheroid(), ("bf16x3", "bf16x6")),
    "presn_64x32x64_L16": (lambda: W.presn(n_r=64, n_theta=32, n_phi=64, L=16), ("bf16x3", "bf16x6")),
    "ragged_rows_5x27x48_L7": (lambda: W.presn(n_r=5, n_theta=27, n_phi=48, L=7, r_lo=1e7, r_hi=2e7),
                               ("bf16x3", "bf16x6")),
    "two_phi_chunks_3x48x320_L6": (lambda: W.presn(n_r=3, n_theta=48, n_phi=320, L=6, r_lo=1e7, r_hi=1.5e7),
                                   ("bf16x3", "bf16x6")),
    # 100 azimuthal cells in synthesis chunks of 64 columns: a ragged second chunk (its third
    # 16-column store box holds 4 cells, its fourth none)
    "ragged_phi_chunks_6x40x100_L6": (lambda: W.presn(n_r=6, n_theta=40, n_phi=100, L=6, r_lo=1e7, r_hi=2e7),
                                      ("bf16x3", "bf16x6")),
    "monopole_L0_8x16x32": (lambda: W.presn(n_r=8, n_theta=16, n_phi=32, L=0), ("bf16x3",)),
    "random_rough_6x32x64_L8": (lambda: W.random_small((6, 32, 64), 8, seed=8, r0=0.2, r1=1.0), ("bf16x6",)),
    "many_moments_40x64x128_L50": (lambda: W.presn(n_r=40, n_theta=64, n_phi=128, L=50, r_lo=1e7, r_hi=3e7),
                                   ("bf16x3",)),
    # more 128-row tiles than the projection's persistent grid has CTAs, the last tile ragged
    "multi_wave_200x100x32_L8": (lambda: W.presn(n_r=200, n_theta=100, n_phi=32, L=8), ("bf16x3", "bf16x6")),
    # three tiles per CTA of the projection, three K chunks per tile (the two converter groups
    # take one or two chunks of a tile, alternately) and three accumulators per tile: the
    # epilogue steps of a tile interleave with the next tile's chunks or run at its end
    "odd_chunks_3_tiles_per_cta_456x128x96_L12": (lambda: W.presn(n_r=456, n_theta=128, n_phi=96, L=12),
                                                  ("bf16x3",)),
    # tables too large for shared memory: the direct theta contraction and the per-row
    # theta synthesis
    "high_L_fallback_4x96x64_L30": (lambda: W.presn(n_r=4, n_theta=96, n_phi=64, L=30, r_lo=1e7, r_hi=1.3e7),
                                    ("bf16x3",)),
}


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
@pytest.mark.parametrize("name,prec", [(n, p) for n, (_, ps) in SPLIT_CASES.items() for p in ps])
def test_split_path_matches_oracle(name, prec, engine):
    """Both engines of the theta stages: tcgen05 GEMMs per order (m >= 1) and CUDA cores."""
    w = SPLIT_CASES[name][0]()
    if engine == "tensor" and w.mesh.L == 0:
        pytest.skip("l_max = 0 has no orders m >= 1")
    ref = oracle_solve(w)
    got = gpu_solve(w, prec, engine=engine)
    assert got["info"]["effective_precision"] == {"bf16x3": 1, "bf16x6": 2}[prec]
    assert got["info"]["theta_tensor_cores"] == (1 if engine == "tensor" else 0)
    err = phi_rel_err(got["phi"], ref["phi"])
    assert err <= 1e-6, err
    # every exported moment, per degree: the angular moments of step (a) and the edge
    # moments M^R, M^I of step (c), against the error model's bar relative to the sum of
    # the magnitudes of each moment's terms
    L = w.mesh.L
    S = term_scales(w.rho, ref["tables"], w.mesh.G)
    bar = split_moment_bar(w.mesh, prec)
    eA = moment_term_errors(got["A"], ref["A"], S, L)
    eM = edge_term_errors(got, ref, S)
    print(f"{name} {prec} {engine}: phi {err:.2e}; per-l A/S max {max(eA):.2e}, M^R {max(eM['MR']):.2e}, "
          f"M^I {max(eM['MI']):.2e} (bar {bar:.2e}); per-l A vs degree max {max(per_l_errors(got['A'], ref['A'], L)):.2e}")
    assert max(eA) <= bar, eA
    assert max(eM["MR"]) <= bar, eM["MR"]
    assert max(eM["MI"]) <= bar, eM["MI"]
    # the monopole, which carries most of Phi, against its own size
    assert per_l_errors(got["A"], ref["A"], L)[0] <= 1e-6


def test_presn_full_size_split_and_fp64():
    """512 x 128 x 256 cells, L = 16: every cell against the oracle, both paths (the split
    path with both theta engines)."""
    w = W.presn()
    ref = oracle_solve(w)
    for prec, tol, engine in (("bf16x3", 1e-6, "tensor"), ("bf16x3", 1e-6, "cuda"), ("fp64", 1e-12, None)):
        got = gpu_solve(w, prec, want_moments=False, engine=engine)
        assert phi_rel_err(got["phi"], ref["phi"]) <= tol, (prec, engine)


def test_theta_engine_requests_that_cannot_be_served():
    from paper_2602_02507_gb300 import multipole as mpl
    for prec, L in (("fp64", 4), ("bf16x3", 0)):
        w = W.presn(n_r=8, n_theta=16, n_phi=32, L=L, materialize=False)
        m = w.mesh
        with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
            with pytest.raises(mpl.MultipoleError) as ei:
                mesh.set_theta_engine("tensor")
            assert ei.value.name == "MP_ERR_UNSUPPORTED"
            mesh.set_theta_engine("cuda")
            mesh.set_theta_engine("auto")
            assert mesh.info()["theta_tensor_cores"] == 0


def test_split_falls_back_to_fp64_for_odd_nphi():
    w = W.random_small((6, 24, 37), 4, seed=6, r0=0.0, r1=1.0)
    got = gpu_solve(w, "bf16x3")
    assert got["info"]["effective_precision"] == 0
    assert phi_rel_err(got["phi"], oracle_solve(w)["phi"]) <= 1e-12
