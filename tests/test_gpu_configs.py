"""The larger workloads at full size, through the C ABI, against the FP64 CPU oracle.

- log-normal precision stress, 1024 x 256 x 512, L = 32: every cell against the oracle.
- large single solve, 2048 x 512 x 1024 (1.07e9 cells), L = 64: oracle moments of the
  whole mesh and the potential of sampled shells (the oracle computes shells one by one).
- 64 uneven meshes solved as one graph-launched batch: the batch equals the meshes'
  own solves bit for bit (sampled), and the smallest instances match the oracle.

Phi errors are max_c |dPhi_c| / |Phi_c| (pointwise; the max-norm error max |dPhi| /
max |Phi| is printed beside it for the large mesh).  Per-degree moment errors are
printed for the record.
"""
import numpy as np
import pytest

from gpu_helpers import (edge_term_errors, moment_term_errors, per_l_errors, phi_rel_err, split_moment_bar,
                         term_scales)
from paper_2602_02507_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()


def _solve(w, prec, rho_dev=None, shells=None, engine=None):
    """Phi (whole mesh, or the listed shells), the angular and edge moments of one GPU solve
    (engine: theta stages of the split path, "tensor" or "cuda"; None: the default)."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    m = w.mesh
    rho = rho_dev if rho_dev is not None else torch.from_numpy(np.ascontiguousarray(w.rho)).cuda()
    phi = torch.empty_like(rho)
    n_r, K = m.shape[0], m.KL
    A = torch.empty(n_r * K, dtype=torch.float64, device="cuda")
    MR = torch.empty((n_r + 1) * K, dtype=torch.float64, device="cuda")
    MI = torch.empty((n_r + 1) * K, dtype=torch.float64, device="cuda")
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
        if engine is not None:
            mesh.set_theta_engine(engine)
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        mesh.solve()
        mesh.get_moments(A, MR, MI)
        mesh.synchronize()
        eff = mesh.info()["effective_precision"]
    out = phi.view(n_r, -1) if shells is None else phi.view(n_r, -1)[shells]
    mom = {"A": A.cpu().numpy().reshape(n_r, K), "MR": MR.cpu().numpy().reshape(n_r + 1, K),
           "MI": MI.cpu().numpy().reshape(n_r + 1, K)}
    return out.cpu().numpy().reshape(-1 if shells is None else len(shells), *m.shape[1:]), mom, eff


def _check_moments(tag, w, prec, mom, ref, S, L):
    """Per-degree moment errors of a split solve against the error model's bar; float64
    solves against 1e-12 of the same term scale."""
    bar = split_moment_bar(w.mesh, prec) if prec != "fp64" else 1e-12
    eA = moment_term_errors(mom["A"], ref["A"], S, L)
    eM = edge_term_errors(mom, ref, S)
    print(f"{tag} {prec}: per-l A/S max {max(eA):.2e}, M^R {max(eM['MR']):.2e}, M^I {max(eM['MI']):.2e} "
          f"(bar {bar:.2e})")
    assert max(eA) <= bar, (prec, eA)
    assert max(eM["MR"]) <= bar, (prec, eM["MR"])
    assert max(eM["MI"]) <= bar, (prec, eM["MI"])


def test_lognormal_full_size_1024x256x512_L32():
    from oracle import oracle as O
    w = W.lognormal()
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    ref = O.solve(tab, w.rho, m.G)
    ref["tables"] = tab
    S = term_scales(w.rho, tab, m.G)
    for prec, tol, engine in (("fp64", 1e-12, None), ("bf16x3", 1e-6, "tensor"), ("bf16x6", 1e-6, "tensor"),
                              ("bf16x3", 1e-6, "cuda")):
        phi, mom, eff = _solve(w, prec, engine=engine)
        assert eff == {"fp64": 0, "bf16x3": 1, "bf16x6": 2}[prec]
        err = phi_rel_err(phi, ref["phi"])
        print(f"lognormal {prec} {engine}: phi {err:.3e}, per-l A vs degree max "
              f"{max(per_l_errors(mom['A'], ref['A'], m.L)):.3e}")
        assert err <= tol, (prec, engine, err)
        _check_moments(f"lognormal {engine}", w, prec, mom, ref, S, m.L)


LARGE_SHELLS = sorted(set([0, 1, 2046, 2047] + list(range(0, 2048, 32))))


def test_large_full_size_2048x512x1024_L64_sampled_shells():
    """Every moment of the whole mesh against the oracle; Phi on every 32nd shell plus the
    first and last two (68 of 2048 shells, 35.7 M cells)."""
    from oracle import oracle as O
    w = W.large(materialize=True)
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    ref = O.solve(tab, w.rho, m.G, want_phi=False)
    ref["tables"] = tab
    S = term_scales(w.rho, tab, m.G)
    shells = LARGE_SHELLS
    ref_phi = O.potential_shells(tab, ref["C"], shells)
    import torch
    rho = torch.from_numpy(w.rho).cuda()
    del w
    for prec, engine in (("fp64", None), ("bf16x3", "tensor"), ("bf16x3", "cuda")):
        phi, mom, _ = _solve(W.large(), prec, rho_dev=rho, shells=shells, engine=engine)
        pointwise = phi_rel_err(phi, ref_phi)
        maxnorm = float(np.abs(phi - ref_phi).max() / np.abs(ref_phi).max())
        A = mom["A"]
        mono = float(np.max(np.abs(A[:, 0] - ref["A"][:, 0]) / np.abs(ref["A"][:, 0])))
        print(f"large {prec} {engine}: phi pointwise {pointwise:.3e}, max-norm {maxnorm:.3e}, A_00 {mono:.3e}")
        assert pointwise <= (1e-12 if prec == "fp64" else 1e-6), (prec, engine, pointwise, maxnorm, mono)
        _check_moments(f"large {engine}", W.large(), prec, mom, ref, S, m.L)
        torch.cuda.empty_cache()


def test_batch_of_64_uneven_meshes():
    import torch
    from oracle import oracle as O
    from paper_2602_02507_gb300 import multipole as mpl
    draws = W.batch_draws()
    meshes, rhos, phis = [], [], []
    for n in range(len(draws)):
        w = W.batch_instance(n, draws)
        m = w.mesh
        rho = torch.from_numpy(w.rho).cuda()
        phi = torch.empty_like(rho)
        ms = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3")
        ms.set_density(rho)
        ms.set_phi_output(phi)
        meshes.append(ms)
        rhos.append(rho)
        phis.append(phi)
    # the meshes' own solves, one at a time
    own = []
    for ms, phi in zip(meshes, phis):
        ms.solve()
        ms.synchronize()
        own.append(phi.clone())
    # the batch runs its meshes on parallel branches, so kernels of different meshes share the
    # SMs: every instance must still give its own solve's bits, launch after launch
    b = mpl.Batch(meshes)
    for rep in range(3):
        for phi in phis:
            phi.fill_(float("nan"))
        b.solve()
        torch.cuda.synchronize()
        for n, (ms, phi) in enumerate(zip(meshes, phis)):
            ms.synchronize()  # no device-side error
            assert torch.equal(phi, own[n]), (rep, n)
    b.close()
    # against the oracle: the three smallest instances, and the smallest instance of each
    # l_max value (8, 16, 32)
    order = sorted(range(len(draws)), key=lambda n: np.prod(draws[n][0]) * draws[n][1])
    picks = list(order[:3])
    for L in sorted({d[1] for d in draws}):
        n = min((k for k in range(len(draws)) if draws[k][1] == L), key=lambda k: np.prod(draws[k][0]))
        if n not in picks:
            picks.append(n)
    for n in picks:
        w = W.batch_instance(n, draws)
        m = w.mesh
        ref = O.solve(O.build_tables(m.r, m.theta, m.phi, m.L), w.rho, m.G)
        err = phi_rel_err(phis[n].cpu().numpy(), ref["phi"])
        print(f"batch instance {n} {draws[n][0]} L={draws[n][1]}: phi {err:.3e}")
        assert err <= 1e-6, (n, err)
    for ms in meshes:
        ms.close()
