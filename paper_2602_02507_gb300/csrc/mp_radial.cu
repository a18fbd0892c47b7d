// mp_radial.cu -- steps (b) and (c) of GenASiS II Sec. 2.2 and the per-shell
// coefficients of step (d), in float64 (they span many decades of radius), plus
// the float32 theta contraction of the split path.
//
// Radial recurrences on the n_r + 1 shell edges:
//   MR_0 = 0,      MR_{i+1} = MR_i + WR[l][i] A[i][q]      (outward, regular)
//   MI_{n_r} = 0,  MI_i     = MI_{i+1} + WI[l][i] A[i][q]  (inward, irregular)
// where WR = Delta(r^3/3) (R^R)_i and WI = Delta(r^3/3) (R^I)_i are the shell
// integrals.  Cell-centre moments are the edge means (linear interpolation to
// the coordinate midpoint), and Eq. (Solution) gives, per shell and moment,
//   C[i][q] = -(Delta_m / (2l+1)) [ (R^R)_i Mbar^I + (R^I)_i Mbar^R ].
// A shell touching r = 0 uses, for l >= 2, the exact own-shell value
// 6 r_1^2 / (5 (l+3)) A[0][q] in place of the divergent midpoint split.
#include "mp_internal.h"

namespace mp {

namespace {

// One block per 32 moment columns; warp w scans shells [w*chunk, (w+1)*chunk)
// and the chunk totals are combined through shared memory.
__global__ void k_scan(const double *__restrict__ A, const double *__restrict__ WR, const double *__restrict__ WI,
                       const double *__restrict__ RR, const double *__restrict__ RI, double *__restrict__ MR,
                       double *__restrict__ MI, double *__restrict__ C, float *__restrict__ C32, int n_r, int KL,
                       int origin, double r1sq)
{
    extern __shared__ double tot[];  // [2][NW][32]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    const bool valid = q < KL;
    int l = 0;
    if (valid)
        while ((l + 1) * (l + 1) <= q) ++l;
    const int p = q - l * l;
    const int m = pcol_m(p);
    const int chunk = (n_r + NW - 1) / NW;
    const int i0 = min(n_r, w * chunk), i1 = min(n_r, i0 + chunk);
    const double *wr = WR + (size_t)l * n_r;
    const double *wi = WI + (size_t)l * n_r;
    double sR = 0.0, sI = 0.0;
    if (valid)
        for (int i = i0; i < i1; ++i) {
            const double a = A[(size_t)i * KL + q];
            sR += wr[i] * a;
            sI += wi[i] * a;
        }
    tot[w * 32 + lane] = sR;
    tot[(NW + w) * 32 + lane] = sI;
    __syncthreads();
    if (!valid) return;
    double mr = 0.0, mi = 0.0;
    for (int w2 = 0; w2 < w; ++w2) mr += tot[w2 * 32 + lane];
    for (int w2 = NW - 1; w2 > w; --w2) mi += tot[(NW + w2) * 32 + lane];
    // outward: edges i0 .. i1-1 (and n_r for the last warp)
    for (int i = i0; i < i1; ++i) {
        MR[(size_t)i * KL + q] = mr;
        mr += wr[i] * A[(size_t)i * KL + q];
    }
    if (w == NW - 1) {
        MR[(size_t)n_r * KL + q] = mr;
        MI[(size_t)n_r * KL + q] = mi;
    }
    // inward: edges i1-1 .. i0, coefficients of every shell of the chunk
    const double pre = -((m == 0) ? 1.0 : 2.0) / (2.0 * l + 1.0);
    for (int i = i1 - 1; i >= i0; --i) {
        const double a = A[(size_t)i * KL + q];
        const double mi_hi = mi;
        mi += wi[i] * a;
        MI[(size_t)i * KL + q] = mi;
        const double mr_lo = MR[(size_t)i * KL + q];
        const double mr_hi = mr_lo + wr[i] * a;
        double c;
        if (origin && i == 0 && l >= 2) {
            const double sself = 6.0 * r1sq / (5.0 * (l + 3.0));
            c = pre * (RR[(size_t)l * n_r] * mi_hi + sself * a);
        } else {
            c = pre * (RR[(size_t)l * n_r + i] * 0.5 * (mi + mi_hi) + RI[(size_t)l * n_r + i] * 0.5 * (mr_lo + mr_hi));
        }
        C[(size_t)i * KL + q] = c;
        if (C32) C32[(size_t)i * KL + q] = (float)c;
    }
}

// Split path, theta part of step (a): A[i][q] = 4 pi G sum_j Ith[t][j] F[i n_t + j][p]
// in float32 with compensated (Kahan) summation; F comes from the tensor-core
// phi projection.
__global__ void __launch_bounds__(512) k32_theta(const float *__restrict__ F, const float *__restrict__ IthT,
                                                 double *__restrict__ A, int n_t, int KL, int T, int Npad,
                                                 double scale)
{
    const int i = blockIdx.x;
    for (int q = threadIdx.x; q < KL; q += blockDim.x) {
        int l = 0;
        while ((l + 1) * (l + 1) <= q) ++l;
        const int p = q - l * l;
        const int t = tri(l, pcol_m(p));
        const float *f = F + (size_t)i * n_t * Npad + p;
        float s = 0.0f, c = 0.0f;
        for (int j = 0; j < n_t; ++j) {
            const float y = __fmul_rn(IthT[(size_t)j * T + t], f[(size_t)j * Npad]) - c;
            const float tt = __fadd_rn(s, y);
            c = __fsub_rn(__fsub_rn(tt, s), y);
            s = tt;
        }
        A[(size_t)i * KL + q] = scale * ((double)s - (double)c);
    }
}

}  // namespace

cudaError_t launch_scan(mp_mesh *m, int want_f32)
{
    const int NW = m->plan.scan_warps;
    const int blocks = (m->KL + 31) / 32;
    const size_t smem = 2 * (size_t)NW * 32 * sizeof(double);
    const double r1sq = m->h_r[1] * m->h_r[1];
    cudaEvent_t ev;
    prof_begin(m, "radial_scan", &ev);
    k_scan<<<blocks, NW * 32, smem, m->stream>>>(m->d_A, m->d_WR, m->d_WI, m->d_RR, m->d_RI, m->d_MR, m->d_MI, m->d_C,
                                                 want_f32 ? m->d_C32 : nullptr, m->n_r, m->KL, m->origin, r1sq);
    prof_end(m, "radial_scan", ev);
    return cudaGetLastError();
}

cudaError_t launch_split_theta(mp_mesh *m)
{
    constexpr double kFourPi = 12.566370614359172954;
    const int threads = m->KL >= 512 ? 512 : ((m->KL + 31) / 32) * 32;
    cudaEvent_t ev;
    prof_begin(m, "split_theta_contract", &ev);
    k32_theta<<<m->n_r, threads, 0, m->stream>>>(m->d_F32, m->d_IthT32, m->d_A, m->n_t, m->KL, m->T, m->plan.Npad,
                                                 kFourPi * m->G);
    prof_end(m, "split_theta_contract", ev);
    return cudaGetLastError();
}

}  // namespace mp
