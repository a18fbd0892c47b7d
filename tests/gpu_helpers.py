"""Helpers of the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np


def gpu_solve(w, precision, want_moments=True):
    import torch

    from paper_2602_02507_gb300 import multipole as mpl

    m = w.mesh
    rho = torch.from_numpy(np.ascontiguousarray(w.rho)).cuda()
    phi = torch.empty_like(rho)
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=precision) as mesh:
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


def phi_rel_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def per_l_errors(got, ref, L, floor=1e-2):
    """max over (i, m, a) of |dA| / max over (i, m, a) of |A_ref|, for each degree l.
    Degrees whose moments are below floor * max |A_ref| (vanishing by symmetry or
    by the smoothness of the density) are measured against that floor instead:
    their values are rounding noise of sums of terms of the leading size."""
    out = []
    top = np.abs(ref).max()
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        den = max(np.abs(ref[:, sl]).max(), floor * top)
        out.append(float(np.abs(got[:, sl] - ref[:, sl]).max() / den) if den > 0 else 0.0)
    return out


def significant_degrees(A_ref, L, floor=1e-2):
    """Degrees whose angular moments reach floor * the largest moment."""
    top = np.abs(A_ref).max()
    return [l for l in range(L + 1) if np.abs(A_ref[:, l * l:(l + 1) * (l + 1)]).max() >= floor * top]


def edge_moment_errors(got, ref):
    """Per-degree error of the edge moments M^R, M^I against the size of the terms
    their recurrences add: each shell contributes |W_l,i| times its largest angular
    moment, so a degree whose own moments vanish (to rounding) is measured against
    the rounding scale of the recurrence rather than against its own noise."""
    tab = ref["tables"]
    A = ref["A"]
    L = tab.L
    amax = np.abs(A).max(axis=1)                               # largest moment of each shell
    WR = np.where(np.isfinite(tab.WR), np.abs(tab.WR), 0.0)
    WI = np.where(np.isfinite(tab.WI), np.abs(tab.WI), 0.0)
    out = {}
    for key, W, forward in (("MR", WR, True), ("MI", WI, False)):
        errs = []
        for l in range(L + 1):
            terms = W[l] * amax
            scale = np.cumsum(terms) if forward else np.cumsum(terms[::-1])[::-1]
            sl = slice(l * l, (l + 1) * (l + 1))
            d = np.abs(got[key][:, sl] - ref[key][:, sl]).max()
            errs.append(float(d / scale.max()) if scale.max() > 0 else 0.0)
        out[key] = errs
    return out
