"""Helpers of the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np


def gpu_solve(w, precision, want_moments=True, engine=None):
    """One solve through the C ABI; engine selects the theta stages of the split path
    ("tensor" or "cuda"; None keeps the mesh's default)."""
    import torch

    from paper_2602_02507_gb300 import multipole as mpl

    m = w.mesh
    rho = torch.from_numpy(np.ascontiguousarray(w.rho)).cuda()
    phi = torch.empty_like(rho)
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=precision) as mesh:
        if engine is not None:
            mesh.set_theta_engine(engine)
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        mesh.solve()
        out = {"info": mesh.info()}
        if want_moments:
            n_r, K = m.shape[0], m.KL
            A = torch.empty(n_r * K, dtype=torch.float64, device="cuda")
            MR = torch.empty((n_r + 1) * K, dtype=torch.float64, device="cuda")
            MI = torch.empty((n_r + 1) * K, dtype=torch.float64, device="cuda")
            mesh.get_moments(A, MR, MI)
        mesh.synchronize()
        out["phi"] = phi.cpu().numpy()
        if want_moments:
            out["A"] = A.cpu().numpy().reshape(n_r, K)
            out["MR"] = MR.cpu().numpy().reshape(n_r + 1, K)
            out["MI"] = MI.cpu().numpy().reshape(n_r + 1, K)
    return out


def oracle_solve(w):
    from oracle import oracle as O

    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    out = O.solve(tab, w.rho, m.G)
    out["tables"] = tab
    return out


from oracle.error_metrics import (edge_moment_errors, edge_term_errors, moment_term_errors,  # noqa: E402,F401
                                  per_l_errors, phi_rel_err, significant_degrees, split_moment_bar,
                                  term_scales)
