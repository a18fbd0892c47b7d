"""Radial-shell sharding of one solve on the GPU: the slabs of a mesh solved one after the
other on one device (mp_slab_moments, the exclusive prefix of their totals on the host,
mp_slab_potential) give the whole mesh's potential and edge moments."""
import numpy as np
import pytest

from gpu_helpers import edge_term_errors, oracle_solve, phi_rel_err, split_moment_bar, term_scales
from paper_2602_02507_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()


def _slab_solve(w, prec, world, engine=None):
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    from paper_2602_02507_gb300.sharding import outer_from_totals, slab_of
    m = w.mesh
    n_r, K = m.shape[0], m.KL
    meshes, rhos, phis, totals = [], [], [], []
    for rank in range(world):
        i0, i1 = slab_of(n_r, rank, world)
        ms = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec, slab=(i0, i1))
        if engine is not None:
            ms.set_theta_engine(engine)
        rho = torch.from_numpy(np.ascontiguousarray(w.rho[i0:i1])).cuda()
        phi = torch.empty_like(rho)
        ms.set_density(rho)
        ms.set_phi_output(phi)
        t = torch.empty(2 * K, dtype=torch.float64, device="cuda")
        ms.slab_moments(t)
        meshes.append(ms)
        rhos.append(rho)
        phis.append(phi)
        totals.append(t.view(2, K))
    all_totals = torch.stack(totals)
    MR, MI = [], []
    for rank, ms in enumerate(meshes):
        ms.slab_potential(outer_from_totals(all_totals, rank).reshape(-1).contiguous())
        n = ms.shape[0]
        mr = torch.empty((n + 1) * K, dtype=torch.float64, device="cuda")
        mi = torch.empty((n + 1) * K, dtype=torch.float64, device="cuda")
        ms.get_moments(None, mr, mi)
        ms.synchronize()
        MR.append(mr.cpu().numpy().reshape(n + 1, K))
        MI.append(mi.cpu().numpy().reshape(n + 1, K))
    phi = np.concatenate([p.cpu().numpy() for p in phis])
    for ms in meshes:
        ms.close()
    return phi, MR, MI


CASES = {
    "presn_64x32x64_L16_3_slabs": (lambda: W.presn(n_r=64, n_theta=32, n_phi=64, L=16), 3,
                                   (("fp64", None), ("bf16x3", "tensor"), ("bf16x3", "cuda"))),
    "origin_ragged_7x19x37_L5_2_slabs": (lambda: W.random_small((7, 19, 37), 5, seed=1, r0=0.0, r1=2.0, uneven=True),
                                         2, (("fp64", None),)),
    "geometric_200x100x32_L8_4_slabs": (lambda: W.presn(n_r=200, n_theta=100, n_phi=32, L=8), 4,
                                        (("fp64", None), ("bf16x3", "tensor"))),
}


@pytest.mark.parametrize("name", list(CASES))
def test_slabs_equal_the_whole_mesh_and_the_oracle(name):
    make, world, runs = CASES[name]
    w = make()
    ref = oracle_solve(w)
    S = term_scales(w.rho, ref["tables"], w.mesh.G)
    for prec, engine in runs:
        phi, MR, MI = _slab_solve(w, prec, world, engine)
        err = phi_rel_err(phi, ref["phi"])
        tol = 1e-12 if prec == "fp64" else 1e-6
        # the edges of the whole mesh: each slab's inner edges, then the last slab's outer edge
        got = {"MR": np.concatenate([mr[:-1] for mr in MR] + [MR[-1][-1:]]),
               "MI": np.concatenate([mi[:-1] for mi in MI] + [MI[-1][-1:]])}
        eM = edge_term_errors(got, ref, S)
        bar = 1e-12 if prec == "fp64" else split_moment_bar(w.mesh, prec)
        print(f"{name} {prec} {engine}: phi {err:.2e}, edge moments per degree M^R {max(eM['MR']):.2e}, "
              f"M^I {max(eM['MI']):.2e} (bar {bar:.1e})")
        assert err <= tol, (prec, engine, err)
        assert max(eM["MR"]) <= bar and max(eM["MI"]) <= bar, (prec, engine, eM)
