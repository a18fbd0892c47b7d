"""Coarsening-block averaging on the GPU (mp_coarsen, mp_coarsening_factors) against the
FP64 oracle (Sec. 2.1 blocks, Sec. 2.3 volume-weighted means).  Block sizes are
integers and must agree exactly; means agree to float64 rounding of the sums."""
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


MESHES = {
    "paper_3d_16": lambda: W.paper_mesh(16, 0.25, 3.68, 0, 3),
    "paper_3d_24_non_power_of_two": lambda: W.paper_mesh(24, 0.25, 3.68, 0, 3),
    "paper_3d_64": lambda: W.paper_mesh(64, 0.25, 3.68, 0, 3),
    "paper_2d_48": lambda: W.paper_mesh(48, 0.25, 3.68, 0, 2),
    # 54 azimuthal cells (2 x 27): two columns a thread; odd polar count: whole-range polar blocks
    "paper_3d_27_n_phi_54": lambda: W.paper_mesh(27, 0.25, 3.68, 0, 3),
    "offset_geometric_3d": lambda: W.Mesh(np.geomspace(1e5, 1e7, 41), np.linspace(0, np.pi, 21),
                                          np.linspace(0, 2 * np.pi, 41), 0, 1.0, "geo"),
    # 640 azimuthal cells (2^7 x 5): whole-ring blocks wider than one pass of the CTA
    "wide_rings_6x8x640": lambda: W.Mesh(np.linspace(0.0, 1.0, 7), np.linspace(0, np.pi, 9),
                                         np.linspace(0, 2 * np.pi, 641), 0, 1.0, "wide"),
    # a 16-row whole-ring block at the first shell: chunks of rows wider than one pass of the CTA
    "wide_rings_6x16x640_many_rows": lambda: W.Mesh(np.linspace(0.0, 1.0, 7), np.linspace(0, np.pi, 17),
                                                    np.linspace(0, 2 * np.pi, 641), 0, 1.0, "wide16"),
}


def _mesh(name):
    from paper_2602_02507_gb300 import multipole as mpl
    m = MESHES[name]()
    return m, mpl.Mesh(m.r, m.theta, m.phi, 2, 1.0, precision="fp64")


@pytest.mark.parametrize("name", list(MESHES))
def test_factors_and_means_match_oracle(name):
    import torch
    from oracle import coarsen as O
    m, mesh = _mesh(name)
    with mesh:
        ct, cp = mesh.coarsening_factors()
        oct_, ocp = O.factors(m.r, m.theta, m.phi)
        assert np.array_equal(ct, oct_) and np.array_equal(cp, ocp)
        shape = (m.r.size - 1, m.theta.size - 1, m.phi.size - 1)
        rng = np.random.default_rng(7)
        f = rng.normal(size=shape) * 10.0 + 3.0
        t = torch.from_numpy(f.reshape(-1).copy()).cuda()
        mesh.coarsen(t)
        # a second field through the same mesh: the per-block state of the first call is reset
        f2 = rng.normal(size=shape) - 1.0
        t2 = torch.from_numpy(f2.reshape(-1).copy()).cuda()
        mesh.coarsen(t2)
        mesh.synchronize()
        got = t.cpu().numpy().reshape(shape)
        got2 = t2.cpu().numpy().reshape(shape)
    untouched = (oct_[:, None] == 1) & (ocp == 1)
    for x, g in ((f, got), (f2, got2)):
        ref = O.coarsen(x, m.r, m.theta, m.phi)
        assert np.all(np.abs(g - ref) <= 1e-13 * np.abs(ref) + 1e-13), float(np.abs(g - ref).max())
        assert np.array_equal(g[untouched], x[untouched])


@pytest.mark.parametrize("gap", [37, 38])
@pytest.mark.parametrize("name", ["paper_3d_16", "paper_3d_24_non_power_of_two"])
def test_several_fields_with_a_gap_between_them(name, gap):
    # an odd gap leaves the fields 8-byte aligned only: the one-column paths (and, with
    # 48 azimuthal cells, whole rings spanning two warp chunks); an even one keeps every
    # field 16-byte aligned: the staged two-column paths on each, six fields in two launches
    import torch
    from oracle import coarsen as O
    m, mesh = _mesh(name)
    shape = (m.r.size - 1, m.theta.size - 1, m.phi.size - 1)
    n = int(np.prod(shape))
    stride = n + gap
    rng = np.random.default_rng(9)
    buf = rng.normal(size=6 * stride)
    t = torch.from_numpy(buf.copy()).cuda()
    with mesh:
        mesh.coarsen(t, n_fields=6, field_stride=stride)
        mesh.coarsen(t, n_fields=0)  # nothing to do
        mesh.synchronize()
    got = t.cpu().numpy()
    for fi in range(6):
        ref = O.coarsen(buf[fi * stride:fi * stride + n].reshape(shape), m.r, m.theta, m.phi)
        g = got[fi * stride:fi * stride + n].reshape(shape)
        assert np.all(np.abs(g - ref) <= 1e-13 * np.abs(ref) + 1e-13)
        assert np.array_equal(got[fi * stride + n:(fi + 1) * stride], buf[fi * stride + n:(fi + 1) * stride])


def test_argument_errors():
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    m, mesh = _mesh("paper_3d_16")
    n = (m.r.size - 1) * (m.theta.size - 1) * (m.phi.size - 1)
    t = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    with mesh:
        with pytest.raises(mpl.MultipoleError, match="MP_ERR_INVALID_ARG"):
            mesh.coarsen(t, n_fields=2, field_stride=n - 1)
