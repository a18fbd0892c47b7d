"""mp_moments_noalloc: the angular moments for callers that cannot allocate device
memory where they need them (loops with a memory budget fixed up front, plug-ins whose
host application owns every allocation).  Its scratch is a fixed device array inside
the library, so this file is collected last: the array is shared by every call in the
process."""
import ctypes

import numpy as np
import pytest

from gpu_helpers import oracle_solve, per_l_errors
from paper_2602_02507_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()


def test_noalloc_moments_match_the_solver_moments_on_two_calls():
    import torch
    from paper_2602_02507_gb300 import multipole as mpl

    w = W.presn(n_r=64, n_theta=32, n_phi=64, L=16)
    m = w.mesh
    n_r, K = m.shape[0], m.KL
    rho = torch.from_numpy(w.rho).cuda()
    lib = mpl.load_library()
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="fp64") as mesh:
        mesh.set_density(rho)
        mesh.solve()
        ref = torch.empty(n_r * K, dtype=torch.float64, device="cuda")
        mesh.get_moments(ref)
        mesh.synchronize()
        ref = ref.cpu().numpy().reshape(n_r, K)
        out = torch.empty(n_r * K, dtype=torch.float64, device="cuda")
        for _ in range(2):
            out.fill_(float("nan"))  # every value must come from this call
            torch.cuda.synchronize()
            st = lib.mp_moments_noalloc(mesh._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(out.data_ptr()))
            assert st == 0, mpl.status_string(st)
            mesh.synchronize()
            got = out.cpu().numpy().reshape(n_r, K)
            assert np.all(np.isfinite(got))
            assert max(per_l_errors(got, ref, m.L)) <= 1e-12
    # and against the float64 CPU oracle of Sec. 2.2
    assert max(per_l_errors(got, oracle_solve(w)["A"], m.L)) <= 1e-12


def test_noalloc_reports_a_nonfinite_density_at_the_next_synchronize():
    import torch
    from paper_2602_02507_gb300 import multipole as mpl

    w = W.presn(n_r=8, n_theta=16, n_phi=32, L=4)
    m = w.mesh
    rho = torch.from_numpy(w.rho).cuda().reshape(-1)
    rho[777] = float("nan")
    out = torch.empty(m.shape[0] * m.KL, dtype=torch.float64, device="cuda")
    lib = mpl.load_library()
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="fp64") as mesh:
        st = lib.mp_moments_noalloc(mesh._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert st == 0, mpl.status_string(st)
        with pytest.raises(mpl.MultipoleError) as ei:
            mesh.synchronize()
        assert ei.value.name == "MP_ERR_NONFINITE"
        mesh.synchronize()  # reported once, then cleared


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import torch
    from paper_2602_02507_gb300 import multipole as mpl

    # 1024 x 64 x 16 cells at L = 40: n_r * n_theta * (2L + 1) = 5,308,416 > 4 Mi
    w = W.presn(n_r=1024, n_theta=64, n_phi=16, L=40, materialize=False)
    m = w.mesh
    lib = mpl.load_library()
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="fp64") as mesh:
        rho = torch.zeros(m.cells, dtype=torch.float64, device="cuda")
        out = torch.zeros(m.shape[0] * m.KL, dtype=torch.float64, device="cuda")
        st = lib.mp_moments_noalloc(mesh._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert mpl.STATUS_NAMES[st] == "MP_ERR_INVALID_ARG"
