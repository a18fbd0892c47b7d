"""Error metrics of a GPU solve against the FP64 oracle (test infrastructure only).

Used by the test suite and by the benchmark's oracle leg; the CUDA product path never
imports anything under oracle/.  Phi is compared pointwise, max_c |dPhi_c| / |Phi_c|
(Phi < 0 everywhere); moments per degree l, either against the largest moment of that
degree, or against the sum of the magnitudes of each moment's terms (the natural scale of
the rounding error of any evaluation of the double sum of Eq. (AngularMomentsDiscrete)).
"""
import numpy as np


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


# ---------------------------------------------------------------- error model of the split path
FOUR_PI = 4.0 * np.pi


def term_scales(rho, tab, G, chunk=64):
    """S[i, q] = 4 pi G sum_j |Ith[t(l,m)][j]| sum_k |Iph[p][k]| |rho[i,j,k]|: the sum of the
    magnitudes of the terms of the angular moment A_q(i) of Eq. (AngularMomentsDiscrete), the
    scale of the rounding error of any floating-point evaluation of that double sum.  Uses
    the oracle's tables (shells taken in chunks to bound host memory)."""
    n_r, n_t, n_p = tab.shape
    L = tab.L
    P = 2 * L + 1
    aIph = np.abs(tab.Iph).T                                    # [n_p, P]
    aIth = np.abs(tab.Ith)                                      # [T, n_t]
    S = np.empty((n_r, (L + 1) ** 2))
    rho = np.asarray(rho).reshape(n_r, n_t, n_p)
    rows = {m: aIth[[l * (l + 1) // 2 + m for l in range(m, L + 1)]] for m in range(L + 1)}
    for i0 in range(0, n_r, chunk):
        i1 = min(n_r, i0 + chunk)
        absF = (np.abs(rho[i0:i1]).reshape(-1, n_p) @ aIph).reshape(i1 - i0, n_t, P)
        for m in range(L + 1):
            tm = rows[m]                                        # [L+1-m, n_t]
            for p in ((0,) if m == 0 else (2 * m - 1, 2 * m)):
                vals = absF[:, :, p] @ tm.T                     # [shells, L+1-m]
                for k, l in enumerate(range(m, L + 1)):
                    S[i0:i1, l * l + p] = vals[:, k]
    return FOUR_PI * G * S


def moment_term_errors(got_A, ref_A, S, L):
    """Per degree l: max over (shell, m, a) of |A_gpu - A_oracle| / S (S from term_scales)."""
    d = np.abs(got_A - ref_A)
    # a moment whose terms all vanish must come out exactly zero
    rel = np.where(S > 0, d / np.where(S > 0, S, 1.0), np.where(d > 0, np.inf, 0.0))
    return [float(rel[:, l * l:(l + 1) * (l + 1)].max()) for l in range(L + 1)]


def edge_term_errors(got, ref, S):
    """Per degree l, for the edge moments M^R (outward sums of W^R A) and M^I (inward sums
    of W^I A): max |M_gpu - M_oracle| over the edges and (m, a), relative to the same sums
    taken over |W| S, which bound the error the moments' own errors carry into them."""
    tab = ref["tables"]
    L = tab.L
    n_r = S.shape[0]
    out = {}
    for key, W, forward in (("MR", tab.WR, True), ("MI", tab.WI, False)):
        aW = np.where(np.isfinite(W), np.abs(W), 0.0)          # [L+1, n_r]
        lq = np.repeat(np.arange(L + 1), 2 * np.arange(L + 1) + 1)
        terms = aW[lq].T * S                                    # [n_r, K_L]
        scale = np.zeros((n_r + 1, S.shape[1]))
        if forward:
            scale[1:] = np.cumsum(terms, axis=0)
        else:
            scale[:-1] = np.cumsum(terms[::-1], axis=0)[::-1]
        d = np.abs(got[key] - ref[key])
        rel = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0))
        out[key] = [float(rel[:, l * l:(l + 1) * (l + 1)].max()) for l in range(L + 1)]
    return out


def split_moment_bar(mesh, precision):
    """Bound of the split path's moment errors relative to the term scale S, from its
    error model.  Both factors of step (a) are bf16 products with float32 accumulation on
    the tensor cores:
    - the phi projection multiplies density deviations (x - x_ref, split into 2 bf16
      terms for BF16X3, 3 for BF16X6) by the table (3 bf16 terms): the dropped low
      products and split residuals leave 3 * 2^-18 (BF16X3) or 5 * 2^-27 (BF16X6) of each
      |term|, doubled because |x - x_ref| <= |x| + |x_ref|; the accumulator adds each
      MMA's products with truncation, at most 2^-23 of the running sum per MMA, over
      chains of 2 * NPROD * ceil(n_kc / nacc) MMAs (32 azimuthal cells per K chunk, chunks
      dealt over nacc accumulators);
    - the theta contraction of the orders m >= 1 splits F the same way (its split error
      once more) over chains of 2 * NPROD * ceil(n_kc_theta / nacc_theta) MMAs (32 polar
      cells per chunk); the m = 0 column, in compensated float32, adds about 3 * 2^-24.
    The bar is twice the sum."""
    n_r, n_t, n_p = mesh.shape
    L = mesh.L
    x6 = precision == "bf16x6"
    nprod = 6 if x6 else 3
    eps_term = 5 * 2.0 ** -27 if x6 else 3 * 2.0 ** -18
    npad = -(-(2 * L + 1) // 16) * 16
    n_kc = -(-n_p // 32)
    nacc = max(1, min(4, 256 // npad, n_kc))
    eps_proj = 2.0 * eps_term + 2 * nprod * (-(-n_kc // nacc)) * 2.0 ** -23
    eps_theta = 3 * 2.0 ** -24
    if L >= 1:
        nmax = -(-L // 16) * 16
        n_kct = -(-n_t // 32)
        nacct = max(1, min(4, 256 // nmax, n_kct))
        eps_theta = max(eps_theta, eps_term + 2 * nprod * (-(-n_kct // nacct)) * 2.0 ** -23)
    return 2.0 * (eps_proj + eps_theta)
