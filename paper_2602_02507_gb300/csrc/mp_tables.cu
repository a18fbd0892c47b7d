// mp_tables.cu -- per-mesh kernel tables, built once on the device in float64.
//
// GenASiS II Sec. 2.2 stores, at start-up, the angular kernels averaged over
// each angular cell and the radial kernels averaged over each shell.  Here:
//   Ith[t(l,m)][j] = int_{theta_j}^{theta_j+1} P~_l^m(cos th) sin th dth
//                    (Gauss-Legendre on sub-intervals short enough that the
//                    degree-(L+1) trigonometric integrand is integrated to
//                    rounding level);
//   Iph[p(m,a)][k] = int_{phi_k}^{phi_k+1} cos|sin(m phi) dphi, closed form in
//                    the cancellation-free product form 2 trig(m mid) sin(m h)/m;
//   WR[l][i], WI[l][i] = shell integrals of r^2 (r/r_ref)^l and
//                    r^2 r_ref^l / r^(l+1), V[i] = Delta(r^3/3), in
//                    x0^p expm1(p log1p(dx/x0)) form; R^R = WR/V, R^I = WI/V.
// The solid-angle mean of the kernel over cell (j, k) is
// (Ith/dmu_j)(Iph/dphi_k), dmu_j = cos th_j - cos th_j+1 = 2 sin(mid) sin(half).
#include <cmath>

#include "mp_internal.h"

namespace mp {

namespace {

constexpr int kGaussPoints = 12;

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
__global__ void k_gauss_legendre(int n, double *x, double *w)
{
    const int g = threadIdx.x;
    if (g >= n) return;
    double z = cos(M_PI * (g + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[g] = z;
    w[g] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// Recursion coefficients of P~ in l: a(l,m) = sqrt((4l^2-1)/(l^2-m^2)),
// b(l,m) = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)), stored at t(l, m) for l >= m+2.
__global__ void k_legendre_coefficients(int L, double *ca, double *cb)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int T = (L + 1) * (L + 2) / 2;
    if (t >= T) return;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= t) ++l;
    const int m = t - l * (l + 1) / 2;
    double a = 0.0, b = 0.0;
    if (l >= m + 2) {
        a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
    }
    ca[t] = a;
    cb[t] = b;
}

// One thread per (m, j): all l >= m of the polar cell integrals.
__global__ void k_theta_tables(int L, int n_t, const double *__restrict__ th, const double *__restrict__ glx,
                               const double *__restrict__ glw, const double *__restrict__ ca,
                               const double *__restrict__ cb, double *__restrict__ Ith, double *__restrict__ dmu)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (L + 1) * n_t) return;
    const int m = idx / n_t, j = idx % n_t;
    const double t0 = th[j], t1 = th[j + 1];
    if (m == 0) dmu[j] = 2.0 * sin(0.5 * (t0 + t1)) * sin(0.5 * (t1 - t0));
    const int nsub = max(1, (int)ceil((t1 - t0) * (L + 2) * 0.5));
    const double h = (t1 - t0) / nsub;
    for (int l = m; l <= L; ++l) Ith[(size_t)tri(l, m) * n_t + j] = 0.0;
    // sectoral factor sqrt((2k+1)/(2k)) products give P~_m^m = c_m (-sin)^m
    double cm = 0.28209479177387814347;  // 1/sqrt(4 pi)
    for (int k = 1; k <= m; ++k) cm *= sqrt((2.0 * k + 1.0) / (2.0 * k));
    const double sgn = (m & 1) ? -1.0 : 1.0;
    for (int s = 0; s < nsub; ++s) {
        const double a = t0 + s * h;
        for (int g = 0; g < kGaussPoints; ++g) {
            const double tt = a + 0.5 * h * (glx[g] + 1.0);
            const double w = 0.5 * h * glw[g];
            double sn, x;
            sincos(tt, &sn, &x);
            double pmm = sgn * cm;
            for (int k = 0; k < m; ++k) pmm *= sn;
            const double ws = w * sn;
            Ith[(size_t)tri(m, m) * n_t + j] += ws * pmm;
            if (m < L) {
                double p0 = pmm;
                double p1 = x * sqrt(2.0 * m + 3.0) * pmm;
                Ith[(size_t)tri(m + 1, m) * n_t + j] += ws * p1;
                for (int l = m + 2; l <= L; ++l) {
                    const int t = tri(l, m);
                    const double p2 = ca[t] * (x * p1 - cb[t] * p0);
                    Ith[(size_t)t * n_t + j] += ws * p2;
                    p0 = p1;
                    p1 = p2;
                }
            }
        }
    }
}

// One thread per (p, k): azimuthal cell integrals and cell means.
__global__ void k_phi_tables(int L, int n_p, const double *__restrict__ ph, double *__restrict__ Iph,
                             double *__restrict__ Iphc)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = 2 * L + 1;
    if (idx >= P * n_p) return;
    const int p = idx / n_p, k = idx % n_p;
    const double f0 = ph[k], f1 = ph[k + 1];
    const double mid = 0.5 * (f0 + f1), half = 0.5 * (f1 - f0), width = f1 - f0;
    double v;
    if (p == 0) {
        v = width;
    } else {
        const int m = (p + 1) >> 1;
        const double s = 2.0 * sin(m * half) / m;
        v = (p & 1) ? cos(m * mid) * s : sin(m * mid) * s;
    }
    Iph[(size_t)p * n_p + k] = v;
    Iphc[(size_t)p * n_p + k] = v / width;
}

// x1^p - x0^p without cancellation for x1 > x0 > 0.
__device__ double pow_diff(double x0, double x1, double p)
{
    return pow(x0, p) * expm1(p * log1p((x1 - x0) / x0));
}

// One thread per (l, i): radial shell integrals.  GR and GI are the
// cell-average radial factors R^R = WR/V and R^I = WI/V of Eq. (Solution)
// times the m = 0 coefficient prefactor h_l = -1/(2 (2l+1)).  At r_0 = 0 and
// l >= 2 the irregular integral diverges: WI is stored as 0 there (the inward
// recurrence then gives M^I_0 = M^I_1, the exported edge value without the
// own-shell term), and GI[l][0] carries the own-shell value instead.  The
// coefficient of that shell is 2 GR M^I_1 + 2 h_l S A with S = 6 r_1^2 /
// (5 (l+3)); the general formula GI (M^R_0 + M^R_1) + GR (M^I_0 + M^I_1) gives
// it when GI[l][0] = 2 h_l S / WR[l][0], since M^R_0 = 0 and M^R_1 = WR A.
__global__ void k_radial_tables(int L, int n_r, const double *__restrict__ r, double r_ref, double *__restrict__ WR,
                                double *__restrict__ WI, double *__restrict__ GR, double *__restrict__ GI,
                                double *__restrict__ V)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (L + 1) * n_r) return;
    const int l = idx / n_r, i = idx % n_r;
    const double r0 = r[i], r1 = r[i + 1];
    const double x0 = r0 / r_ref, x1 = r1 / r_ref;
    const double rr2 = r_ref * r_ref, rr3 = rr2 * r_ref;
    double vol;
    if (r0 > 0.0)
        vol = r0 * r0 * r0 * expm1(3.0 * log1p((r1 - r0) / r0)) / 3.0;
    else
        vol = r1 * r1 * r1 / 3.0;
    double wr, wi;
    const double pr = l + 3.0, pi = 2.0 - l;
    if (x0 > 0.0) {
        wr = rr3 * pow_diff(x0, x1, pr) / pr;
        if (l == 2)
            wi = rr2 * log1p((x1 - x0) / x0);
        else
            wi = rr2 * pow_diff(x0, x1, pi) / pi;
    } else {
        wr = rr3 * pow(x1, pr) / pr;
        wi = (l < 2) ? rr2 * pow(x1, pi) / pi : 0.0;
    }
    WR[(size_t)l * n_r + i] = wr;
    WI[(size_t)l * n_r + i] = wi;
    const double hp = -0.5 / (2.0 * l + 1.0);
    GR[(size_t)l * n_r + i] = hp * (wr / vol);
    if (x0 > 0.0 || l < 2)
        GI[(size_t)l * n_r + i] = hp * (wi / vol);
    else
        GI[(size_t)l * n_r + i] = 2.0 * hp * (6.0 * r1 * r1 / (5.0 * (l + 3.0))) / wr;
    if (l == 0) V[i] = vol;
}

}  // namespace

cudaError_t launch_tables(mp_mesh *m)
{
    const int L = m->L;
    double *glx = nullptr, *glw = nullptr, *ca = nullptr, *cb = nullptr;
    cudaError_t e = cudaMallocAsync(&glx, 2 * kGaussPoints * sizeof(double), m->stream);
    if (e != cudaSuccess) return e;
    glw = glx + kGaussPoints;
    e = cudaMallocAsync(&ca, 2 * (size_t)m->T * sizeof(double), m->stream);
    if (e != cudaSuccess) return e;
    cb = ca + m->T;
    k_gauss_legendre<<<1, 32, 0, m->stream>>>(kGaussPoints, glx, glw);
    k_legendre_coefficients<<<(m->T + 127) / 128, 128, 0, m->stream>>>(L, ca, cb);
    {
        const int n = (L + 1) * m->n_t;
        k_theta_tables<<<(n + 63) / 64, 64, 0, m->stream>>>(L, m->n_t, m->d_r + (m->n_r + 1), glx, glw, ca, cb,
                                                            m->d_Ith, m->d_dmu);
    }
    {
        const int n = m->P * m->n_p;
        k_phi_tables<<<(n + 255) / 256, 256, 0, m->stream>>>(L, m->n_p, m->d_r + (m->n_r + 1) + (m->n_t + 1),
                                                             m->d_Iph, m->d_Iphc);
    }
    {
        const int n = (L + 1) * m->n_r;
        k_radial_tables<<<(n + 255) / 256, 256, 0, m->stream>>>(L, m->n_r, m->d_r, m->r_ref, m->d_WR, m->d_WI,
                                                                m->d_GR, m->d_GI, m->d_V);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaFreeAsync(glx, m->stream);
    cudaFreeAsync(ca, m->stream);
    return cudaGetLastError();
}

}  // namespace mp
