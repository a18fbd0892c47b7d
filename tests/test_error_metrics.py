"""The error metrics the parity tests and the benchmark use, pinned on tiny meshes by
brute force (explicit loops over every term of the sums they bound)."""
import numpy as np

from oracle import oracle as O
from oracle.error_metrics import edge_term_errors, moment_term_errors, split_moment_bar, term_scales
from paper_2602_02507_gb300 import workloads as W


def _brute_scales(rho, tab, G):
    n_r, n_t, n_p = tab.shape
    L = tab.L
    S = np.zeros((n_r, (L + 1) ** 2))
    for i in range(n_r):
        for l in range(L + 1):
            for p in range(2 * l + 1):
                m = (p + 1) // 2
                t = l * (l + 1) // 2 + m
                acc = 0.0
                for j in range(n_t):
                    for k in range(n_p):
                        acc += abs(tab.Ith[t, j]) * abs(tab.Iph[p, k]) * abs(rho[i, j, k])
                S[i, l * l + p] = 4.0 * np.pi * G * acc
    return S


def test_term_scales_equal_the_brute_force_sum_of_term_magnitudes():
    w = W.random_small((3, 5, 6), 3, seed=11, r0=0.2, r1=1.0)
    rho = w.rho.copy()
    rho[1, 2, 3] = -rho[1, 2, 3]  # a negative value: magnitudes, not values
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    np.testing.assert_allclose(term_scales(rho, tab, 2.5, chunk=2), _brute_scales(rho, tab, 2.5),
                               rtol=1e-13, atol=0)


def test_term_scales_bound_every_moment_and_the_relative_errors_follow():
    w = W.random_small((4, 6, 8), 4, seed=12, r0=0.0, r1=1.0)
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    ref = O.solve(tab, w.rho, m.G)
    ref["tables"] = tab
    S = term_scales(w.rho, tab, m.G)
    assert np.all(np.abs(ref["A"]) <= S * (1 + 1e-14))
    # a perturbation of known size relative to S per degree
    got = {k: ref[k].copy() for k in ("A", "MR", "MI")}
    got["A"][2, 5] += 3e-7 * S[2, 5]                       # l = 2
    e = moment_term_errors(got["A"], ref["A"], S, m.L)
    assert abs(e[2] - 3e-7) < 1e-12 and max(e[:2] + e[3:]) == 0.0
    got["MR"][3, 1] += 1e-9 * abs(ref["MR"][3, 1])          # l = 1
    eM = edge_term_errors(got, ref, S)
    assert eM["MR"][1] > 0 and max(eM["MR"][:1] + eM["MR"][2:]) == 0.0 and max(eM["MI"]) == 0.0


def test_split_bar_grows_with_the_accumulation_chain():
    small = W.presn(n_r=4, n_theta=8, n_phi=64, L=8, materialize=False).mesh
    large = W.presn(n_r=4, n_theta=8, n_phi=1024, L=64, materialize=False).mesh
    assert split_moment_bar(small, "bf16x3") < split_moment_bar(large, "bf16x3")
    assert split_moment_bar(small, "bf16x6") < split_moment_bar(small, "bf16x3")
    assert split_moment_bar(large, "bf16x3") < 2e-4
