"""Input generators: deterministic, positive, the shapes the configurations name."""
import numpy as np

from paper_2602_02507_gb300 import workloads as W


def test_presn_is_seeded_and_positive():
    a = W.presn(n_r=16, n_theta=8, n_phi=16, L=4)
    b = W.presn(n_r=16, n_theta=8, n_phi=16, L=4)
    assert np.array_equal(a.rho, b.rho)
    assert a.rho.min() > 0
    assert a.mesh.r[0] == 1e5 and a.mesh.r[-1] == 1e10


def test_spheroid_fraction_bounds():
    w = W.spheroid()
    assert w.rho.shape == (64, 32, 64)
    assert w.rho.min() >= 0.0 and w.rho.max() <= 1.0
    vol = (np.diff(w.mesh.r ** 3) / 3)[:, None] * (np.cos(w.mesh.theta[:-1]) - np.cos(w.mesh.theta[1:]))[None, :]
    mass = 2 * np.pi * np.sum(w.rho[:, :, 0] * vol)
    assert abs(mass - 4 / 3 * np.pi * 0.6) < 2e-3


def test_lognormal_unit_variance_field():
    w = W.lognormal(n_r=3, n_theta=32, n_phi=64, L=8, lmax_field=16)
    g = np.log(w.rho[1] / W.presn_profile(W.midpoints(w.mesh.r))[1]) + 0.5
    assert 0.3 < np.var(g) < 3.0


def test_batch_draws_deterministic():
    d1, d2 = W.batch_draws(), W.batch_draws()
    assert d1 == d2 and len(d1) == 64
    assert {s for s, *_ in d1} <= set(W.BATCH_SHAPES)
