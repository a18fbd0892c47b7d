"""Gravitational source terms on the GPU (mp_gravity_sources) against the FP64 oracle.

The kernel and the oracle take the same centred differences (Sec. 3, Eq.
(BalancedVariablesGravitational)); the kernel multiplies by 1/dx where the oracle
divides by dx, so components agree to a few float64 ulps.  The energy source is a
sum of three products that may cancel: its bound is relative to rho sum |v^a g_a|.
"""
import zlib

import numpy as np
import pytest

from paper_2602_02507_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()


def _edges(n_r, n_t, n_p, r0=1e5, r1=1e10, phi_span=2 * np.pi):
    r = np.geomspace(r0, r1, n_r + 1) if r0 > 0 else np.linspace(0.0, r1, n_r + 1)
    th = np.linspace(0.0, np.pi, n_t + 1)
    ph = np.linspace(0.0, phi_span, n_p + 1)
    return r, th, ph


def _compare(got, ref, v, rho, tol):
    for key in ("grad", "S"):
        if key in got:
            g, r = got[key].reshape(ref[key].shape), ref[key]
            scale = np.abs(r).max() if np.abs(r).max() > 0 else 1.0
            err = np.abs(g - r)
            assert np.all(err <= tol * np.abs(r) + 1e-15 * scale), (key, float(err.max()))
    if "E" in got:
        terms = np.abs(rho) * (np.abs(v[0] * ref["grad"][0]) + np.abs(v[1] * ref["grad"][1]) +
                               np.abs(v[2] * ref["grad"][2]))
        e = got["E"].reshape(ref["E"].shape)
        err = np.abs(e - ref["E"])
        assert np.all(err <= tol * terms + 1e-300), ("E", float(err.max()))


def _run(r, th, ph, phi_np, rho_np, v_np, outputs=("grad", "S", "E"), L=4):
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    n = phi_np.size
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    phi, rho = dev(phi_np), dev(rho_np)
    v = dev(v_np) if v_np is not None else None
    out = {k: torch.full((3 * n if k != "E" else n,), np.nan, dtype=torch.float64, device="cuda") for k in outputs}
    with mpl.Mesh(r, th, ph, L, 1.0, precision="fp64") as mesh:
        mesh.gravity_sources(phi=phi, rho=rho, v=v, grad=out.get("grad"), S=out.get("S"), E=out.get("E"))
        mesh.synchronize()
    shape = phi_np.shape
    return {k: (t.cpu().numpy().reshape((3,) + shape) if k != "E" else t.cpu().numpy().reshape(shape))
            for k, t in out.items()}


CASES = {
    "geometric_full_circle_16x24x32": (16, 24, 32, 1e5, 1e10, 2 * np.pi),
    "phi_rows_past_one_block_5x6x300": (5, 6, 300, 1e7, 2e7, 2 * np.pi),
    "origin_shell_12x8x16": (12, 8, 16, 0.0, 1.5, 2 * np.pi),
    "half_circle_6x7x10": (6, 7, 10, 1.0, 3.0, np.pi),
    "one_azimuthal_cell_8x9x1": (8, 9, 1, 1.0, 3.0, 2 * np.pi),
    "two_azimuthal_cells_8x9x2": (8, 9, 2, 1.0, 3.0, 2 * np.pi),
    "one_polar_cell_8x1x16": (8, 1, 16, 1.0, 3.0, 2 * np.pi),
    "one_shell_1x8x16": (1, 8, 16, 1.0, 3.0, 2 * np.pi),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sources_match_oracle(name):
    from oracle import gravity as O
    n_r, n_t, n_p, r0, r1, span = CASES[name]
    r, th, ph = _edges(n_r, n_t, n_p, r0, r1, span)
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    shape = (n_r, n_t, n_p)
    rc = O.centres(r)
    # a smooth potential times a small random modulation: large common part, small differences
    phi = (-1e3 / (1.0 + rc))[:, None, None] * (1.0 + 1e-2 * rng.normal(size=shape))
    rho = rng.uniform(0.1, 10.0, shape)
    v = rng.normal(size=(3,) + shape)
    ref = O.sources(phi, rho, v, r, th, ph)
    got = _run(r, th, ph, phi, rho, v)
    _compare(got, ref, v, rho, 1e-13)


@pytest.mark.parametrize("outputs", [("E",), ("grad",), ("S",), ("grad", "E")])
def test_output_subsets(outputs):
    from oracle import gravity as O
    r, th, ph = _edges(6, 10, 24)
    rng = np.random.default_rng(5)
    shape = (6, 10, 24)
    phi = rng.normal(size=shape)
    rho = rng.uniform(0.5, 2.0, shape)
    v = rng.normal(size=(3,) + shape) if "E" in outputs else None
    ref = O.sources(phi, rho, v, r, th, ph)
    got = _run(r, th, ph, phi, rho, v, outputs=outputs)
    assert set(got) == set(outputs)
    _compare(got, ref, v, rho, 1e-13)


def test_argument_errors():
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    r, th, ph = _edges(4, 4, 8)
    n = 4 * 4 * 8
    S = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    rho = torch.ones(n, dtype=torch.float64, device="cuda")
    with mpl.Mesh(r, th, ph, 2, 1.0, precision="fp64") as mesh:
        with pytest.raises(mpl.MultipoleError, match="MP_ERR_NOT_READY"):
            mesh.gravity_sources(rho=rho, S=S)          # no solve yet, no potential given
        with pytest.raises(mpl.MultipoleError, match="MP_ERR_INVALID_ARG"):
            mesh.gravity_sources(phi=rho, rho=rho, E=E)  # energy source without velocity
        with pytest.raises(mpl.MultipoleError, match="MP_ERR_INVALID_ARG"):
            mesh.gravity_sources(phi=rho, rho=rho)       # no output


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_full_size_presn_after_solve(prec):
    """512 x 128 x 256 cells: the potential of the preceding solve (phi = None) and the
    bound density (rho = None), every cell against the oracle on that same potential."""
    import torch
    from oracle import gravity as O
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn()
    m = w.mesh
    rho = torch.from_numpy(np.ascontiguousarray(w.rho).reshape(-1)).cuda()
    phi = torch.empty_like(rho)
    n = rho.numel()
    rng = np.random.default_rng(11)
    v_np = rng.normal(size=(3, n)) * 1e8
    v = torch.from_numpy(v_np.reshape(-1)).cuda()
    S = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    E = torch.empty(n, dtype=torch.float64, device="cuda")
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        mesh.solve()
        mesh.gravity_sources(v=v, S=S, E=E)
        mesh.synchronize()
    shape = w.rho.shape
    phi_np = phi.cpu().numpy().reshape(shape)
    vv = v_np.reshape((3,) + shape)
    ref = O.sources(phi_np, w.rho, vv, m.r, m.theta, m.phi)
    got = {"S": S.cpu().numpy().reshape((3,) + shape), "E": E.cpu().numpy().reshape(shape)}
    _compare(got, ref, vv, w.rho, 1e-13)
