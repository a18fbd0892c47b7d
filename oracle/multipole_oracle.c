/*
 * multipole_oracle.c -- plain FP64 CPU oracle of the multipole Poisson solve of
 * GenASiS II (Cardall, Budiardja, Murphy & Endeve), Sec. 2.2 "Poisson Solver".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * never includes, links or calls it, and the two share no code, header, table
 * or constant generator.  Every step below is written out from the paper's
 * definitions in the paper's order, in double precision, without blocking or
 * fusion; OpenMP only splits independent shells (or columns) across threads.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   R1  "averaged over each angular cell" = solid-angle mean, so
 *       (dOmega)_jk (A)_jk = [int P~ sin(theta) dtheta] * [int cos|sin(m phi) dphi].
 *   R2  radial cell averages are volume (r^2 dr) means, so
 *       (Delta(r^3/3))_i (R)_i = int r^2 R(r) dr over the shell.
 *   R3  "linear interpolation to the cell center": the coordinate midpoint,
 *       edge weights 1/2, 1/2.
 *   R4  origin shell (r_0 = 0) with l >= 2, where int_0 r^(1-l) dr diverges:
 *       the shell's own-term is replaced by its exact value for a moment that is
 *       uniform inside the ball, S_self(l) = 6 r_1^2 / (5 (l+3)); the exported
 *       irregular moment at edge 0 excludes the divergent own-shell term.
 *   R5  the (m = 0, sine) kernel vanishes identically and is not stored, so a
 *       shell carries K_L = (L+1)^2 real moments.
 *   R6  the Condon-Shortley phase (-1)^m of the P~_m^m seed is kept.
 *   R7  radial kernels are scaled by a reference radius r_ref:
 *       R^R -> (r/r_ref)^l and R^I -> r_ref^l / r^(l+1); Phi is unchanged
 *       because only products R^R(r) R^I(r') enter.
 *
 * Conventions (C row-major, double):
 *   shells i = 0..n_r-1 between radial edges r[0] < ... < r[n_r];
 *   polar cells j = 0..n_t-1, azimuthal cells k = 0..n_p-1;
 *   rho, phi: [n_r][n_t][n_p];
 *   real moment column p(m,a): p(0,c) = 0, p(m,c) = 2m-1, p(m,s) = 2m (m >= 1);
 *   moment index q(l,m,a) = l*l + p(m,a);
 *   Legendre triangle index t(l,m) = l(l+1)/2 + m.
 *
 * Parity status of every function is recorded in the oracle's Python front
 * (oracle.py) and the tests that pin it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* The literal seed uses (2m)! in double precision, finite for m <= 85. */
#define ORC_L_MAX 85

static int orc_threads = 0;

void orc_set_threads(int n) { orc_threads = n; }

int orc_get_threads(void)
{
#ifdef _OPENMP
    if (orc_threads > 0) return orc_threads;
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void orc_apply_threads(void)
{
#ifdef _OPENMP
    if (orc_threads > 0) omp_set_num_threads(orc_threads);
#endif
}

static int tri(int l, int m) { return l * (l + 1) / 2 + m; }
static int pcol(int m, int a) { return m == 0 ? 0 : 2 * m - 1 + a; }

/* ------------------------------------------------------------------------ */
/* Renormalized associated Legendre functions (Sec. 2.2).                   */
/* P~_m^m(x)     = (-1)^m sqrt((2m+1)/(4 pi (2m)!)) (2m-1)!! (1-x^2)^(m/2)   */
/* P~_{m+1}^m(x) = x sqrt(2m+3) P~_m^m(x)                                   */
/* P~_l^m(x)     = sqrt((4l^2-1)/(l^2-m^2))                                 */
/*                 [x P~_{l-1}^m - sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)) P~_{l-2}^m] */
/* s = (1-x^2)^(1/2) is passed in so that callers integrating in theta can  */
/* use sin(theta) directly.                                                 */
/* ------------------------------------------------------------------------ */
int orc_legendre_xs(int L, double x, double s, double *P)
{
    if (L < 0 || L > ORC_L_MAX) return -1;
    double fact2m = 1.0;   /* (2m)!    */
    double dfact = 1.0;    /* (2m-1)!! */
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            fact2m *= (double)(2 * m - 1) * (double)(2 * m);
            dfact *= (double)(2 * m - 1);
        }
        double sign = (m % 2 == 0) ? 1.0 : -1.0;
        double pmm = sign * sqrt((2.0 * m + 1.0) / (4.0 * ORC_PI * fact2m)) * dfact * pow(s, (double)m);
        P[tri(m, m)] = pmm;
        if (m + 1 <= L) P[tri(m + 1, m)] = x * sqrt(2.0 * m + 3.0) * pmm;
        for (int l = m + 2; l <= L; ++l) {
            double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
            double b = sqrt(((double)(l - 1) * (l - 1) - (double)m * m) / (4.0 * (l - 1) * (l - 1) - 1.0));
            P[tri(l, m)] = a * (x * P[tri(l - 1, m)] - b * P[tri(l - 2, m)]);
        }
    }
    return 0;
}

int orc_legendre(int L, double x, double *P)
{
    double s = sqrt((1.0 - x) * (1.0 + x));
    return orc_legendre_xs(L, x, s, P);
}

/* ------------------------------------------------------------------------ */
/* Romberg integration of a vector-valued integrand over [a, b].           */
/* The paper averages the angular kernels over each cell numerically, by     */
/* Romberg integration (Sec. 2.2).  Trapezoid rule with step halving plus    */
/* Richardson extrapolation; converged when the change of the diagonal is    */
/* below tol * max|component| (all components checked together).            */
/* ------------------------------------------------------------------------ */
typedef void (*orc_vfun)(double x, void *ctx, double *out);

static int romberg_vec(orc_vfun f, void *ctx, int nv, double a, double b, double tol,
                       int kmin, int kmax, double *result, double *work)
{
    double *prev = work;                       /* previous row, (kmax+1)*nv */
    double *cur = work + (size_t)(kmax + 1) * nv;
    double *fx = cur + (size_t)(kmax + 1) * nv;
    double *sum = fx + nv;
    double h = b - a;
    f(a, ctx, fx);
    for (int c = 0; c < nv; ++c) prev[c] = fx[c];
    f(b, ctx, fx);
    for (int c = 0; c < nv; ++c) prev[c] = 0.5 * h * (prev[c] + fx[c]);
    int k;
    for (k = 1; k <= kmax; ++k) {
        h *= 0.5;
        long npts = 1L << (k - 1);
        for (int c = 0; c < nv; ++c) sum[c] = 0.0;
        for (long i = 1; i <= npts; ++i) {
            f(a + (double)(2 * i - 1) * h, ctx, fx);
            for (int c = 0; c < nv; ++c) sum[c] += fx[c];
        }
        for (int c = 0; c < nv; ++c) cur[c] = 0.5 * prev[c] + h * sum[c];
        double pow4 = 1.0;
        for (int j = 1; j <= k; ++j) {
            pow4 *= 4.0;
            for (int c = 0; c < nv; ++c) {
                double rj1 = cur[(size_t)(j - 1) * nv + c];
                double pj1 = prev[(size_t)(j - 1) * nv + c];
                cur[(size_t)j * nv + c] = rj1 + (rj1 - pj1) / (pow4 - 1.0);
            }
        }
        if (k >= kmin) {
            double err = 0.0, scale = 0.0;
            for (int c = 0; c < nv; ++c) {
                double d = fabs(cur[(size_t)k * nv + c] - prev[(size_t)(k - 1) * nv + c]);
                if (d > err) err = d;
                double v = fabs(cur[(size_t)k * nv + c]);
                if (v > scale) scale = v;
            }
            if (err <= tol * scale || scale == 0.0) {
                for (int c = 0; c < nv; ++c) result[c] = cur[(size_t)k * nv + c];
                return k;
            }
        }
        double *t = prev; prev = cur; cur = t;
    }
    for (int c = 0; c < nv; ++c) result[c] = prev[(size_t)kmax * nv + c];
    return -1;
}

/* Integrand in theta: P~_l^m(cos theta) sin(theta) for every (l, m). */
typedef struct { int L; double *P; } theta_ctx;

static void theta_integrand(double th, void *vctx, double *out)
{
    theta_ctx *ctx = (theta_ctx *)vctx;
    double x = cos(th), s = sin(th);
    orc_legendre_xs(ctx->L, x, s, out);
    int T = (ctx->L + 1) * (ctx->L + 2) / 2;
    for (int t = 0; t < T; ++t) out[t] *= s;
}

/* Ith[t(l,m)][j] = int_{theta_j}^{theta_{j+1}} P~_l^m(cos theta) sin(theta) dtheta,
 * so that (dOmega)_jk (A^a_lm)_jk = Ith[t][j] * Iph[p(m,a)][k]  (reading R1). */
int orc_theta_integrals(int L, int n_t, const double *th, double tol, double *Ith, int *max_levels)
{
    if (L < 0 || L > ORC_L_MAX || n_t < 1) return -1;
    const int kmax = 24;
    int T = (L + 1) * (L + 2) / 2;
    int worst = 0, fail = 0;
    orc_apply_threads();
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * ((size_t)(2 * (kmax + 1) + 2) * T));
        double *res = (double *)malloc(sizeof(double) * T);
        theta_ctx ctx;
        ctx.L = L;
        ctx.P = NULL;
#pragma omp for schedule(dynamic)
        for (int j = 0; j < n_t; ++j) {
            int lev = romberg_vec(theta_integrand, &ctx, T, th[j], th[j + 1], tol, 4, kmax, res, work);
            for (int t = 0; t < T; ++t) Ith[(size_t)t * n_t + j] = res[t];
#pragma omp critical
            {
                if (lev < 0) fail = 1;
                if (lev > worst) worst = lev;
            }
        }
        free(work);
        free(res);
    }
    if (max_levels) *max_levels = worst;
    return fail ? -2 : 0;
}

/* Integrand in phi: 1, cos(m phi), sin(m phi) ordered by the column p(m,a). */
typedef struct { int L; } phi_ctx;

static void phi_integrand(double ph, void *vctx, double *out)
{
    phi_ctx *ctx = (phi_ctx *)vctx;
    out[0] = 1.0;
    for (int m = 1; m <= ctx->L; ++m) {
        out[pcol(m, 0)] = cos((double)m * ph);
        out[pcol(m, 1)] = sin((double)m * ph);
    }
}

/* Iph[p(m,a)][k] = int_{phi_k}^{phi_{k+1}} {cos|sin}(m phi) dphi (Eqs. AngularKernel_c/s). */
int orc_phi_integrals(int L, int n_p, const double *ph, double tol, double *Iph, int *max_levels)
{
    if (L < 0 || n_p < 1) return -1;
    const int kmax = 24;
    int P = 2 * L + 1;
    int worst = 0, fail = 0;
    orc_apply_threads();
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * ((size_t)(2 * (kmax + 1) + 2) * P));
        double *res = (double *)malloc(sizeof(double) * P);
        phi_ctx ctx;
        ctx.L = L;
#pragma omp for schedule(dynamic)
        for (int k = 0; k < n_p; ++k) {
            int lev = romberg_vec(phi_integrand, &ctx, P, ph[k], ph[k + 1], tol, 4, kmax, res, work);
            for (int p = 0; p < P; ++p) Iph[(size_t)p * n_p + k] = res[p];
#pragma omp critical
            {
                if (lev < 0) fail = 1;
                if (lev > worst) worst = lev;
            }
        }
        free(work);
        free(res);
    }
    if (max_levels) *max_levels = worst;
    return fail ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Radial cell integrals (Eqs. RadialRegular, RadialIrregular; reading R2,  */
/* R7), written as the plain antiderivative differences:                    */
/*   WR[l][i] = int r^2 (r/r_ref)^l dr       = r_ref^3 (x1^(l+3) - x0^(l+3))/(l+3) */
/*   WI[l][i] = int r^2 r_ref^l / r^(l+1) dr = r_ref^2 (x1^(2-l) - x0^(2-l))/(2-l) */
/*            (r_ref^2 ln(x1/x0) at l = 2),  x = r / r_ref                  */
/*   V[i]     = Delta(r^3/3)                                                */
/* At r_0 = 0 and l >= 2 the irregular integral diverges; WI is set to +inf */
/* there and the recurrences apply reading R4.                              */
/* ------------------------------------------------------------------------ */
double orc_default_r_ref(int n_r, const double *r)
{
    double rmin = r[0] > 0.0 ? r[0] : r[1];
    return sqrt(rmin * r[n_r]);
}

int orc_radial(int L, int n_r, const double *r, double r_ref, double *WR, double *WI, double *V)
{
    if (L < 0 || n_r < 1 || !(r_ref > 0.0)) return -1;
    for (int i = 0; i < n_r; ++i) {
        double r0 = r[i], r1 = r[i + 1];
        V[i] = (r1 * r1 * r1 - r0 * r0 * r0) / 3.0;
        double x0 = r0 / r_ref, x1 = r1 / r_ref;
        for (int l = 0; l <= L; ++l) {
            double pr = (double)(l + 3);
            WR[(size_t)l * n_r + i] = r_ref * r_ref * r_ref * (pow(x1, pr) - pow(x0, pr)) / pr;
            if (r0 == 0.0 && l >= 2) {
                WI[(size_t)l * n_r + i] = INFINITY;
            } else if (l == 2) {
                WI[(size_t)l * n_r + i] = r_ref * r_ref * log(x1 / x0);
            } else {
                double pi = (double)(2 - l);
                WI[(size_t)l * n_r + i] = r_ref * r_ref * (pow(x1, pi) - pow(x0, pi)) / pi;
            }
        }
    }
    return 0;
}

/* Solid-angle cell widths: dmu_j = cos(theta_j) - cos(theta_{j+1}) = integral of  */
/* sin(theta) over the polar cell, and dphi_k.  The difference of cosines is      */
/* evaluated as 2 sin(mid) sin(half width): near the poles the two cosines agree  */
/* in their leading digits and their plain difference would lose them.           */
static void cell_widths(int n_t, const double *th, int n_p, const double *ph, double *dmu, double *dph)
{
    for (int j = 0; j < n_t; ++j) dmu[j] = 2.0 * sin(0.5 * (th[j] + th[j + 1])) * sin(0.5 * (th[j + 1] - th[j]));
    for (int k = 0; k < n_p; ++k) dph[k] = ph[k + 1] - ph[k];
}

/* ------------------------------------------------------------------------ */
/* Step (a): angular moments, Eq. (AngularMomentsDiscrete)                 */
/*   A[i][q] = sum_jk (dOmega)_jk (A_q)_jk S_ijk,  S = 4 pi G rho          */
/* Literal form: the cell-averaged kernel (A_q)_jk = Ith/dmu * Iph/dphi and */
/* the solid angle dOmega_jk = dmu_j dphi_k are formed per cell.            */
/* ------------------------------------------------------------------------ */
void orc_moments_literal(int n_r, int n_t, int n_p, int L, const double *th, const double *ph,
                         const double *Ith, const double *Iph, double G, const double *rho, double *A)
{
    int KL = (L + 1) * (L + 1);
    double *dmu = (double *)malloc(sizeof(double) * n_t);
    double *dph = (double *)malloc(sizeof(double) * n_p);
    cell_widths(n_t, th, n_p, ph, dmu, dph);
    orc_apply_threads();
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n_r; ++i) {
        for (int l = 0; l <= L; ++l)
            for (int m = 0; m <= l; ++m)
                for (int a = 0; a < (m == 0 ? 1 : 2); ++a) {
                    int p = pcol(m, a), q = l * l + p, t = tri(l, m);
                    double acc = 0.0;
                    for (int j = 0; j < n_t; ++j)
                        for (int k = 0; k < n_p; ++k) {
                            double dOmega = dmu[j] * dph[k];
                            double Aavg = (Ith[(size_t)t * n_t + j] / dmu[j]) * (Iph[(size_t)p * n_p + k] / dph[k]);
                            double S = 4.0 * ORC_PI * G * rho[((size_t)i * n_t + j) * n_p + k];
                            acc += dOmega * Aavg * S;
                        }
                    A[(size_t)i * KL + q] = acc;
                }
    }
    free(dmu);
    free(dph);
}

/* Factored form of the same double sum: because (dOmega A_q)_jk is the
 * product Ith[t][j] Iph[p][k] (reading R1), sum_jk = sum_j Ith sum_k Iph S. */
void orc_moments_factored(int n_r, int n_t, int n_p, int L, const double *Ith, const double *Iph,
                          double G, const double *rho, double *A)
{
    int KL = (L + 1) * (L + 1), P = 2 * L + 1;
    orc_apply_threads();
#pragma omp parallel
    {
        double *F = (double *)malloc(sizeof(double) * (size_t)n_t * P);
#pragma omp for schedule(dynamic)
        for (int i = 0; i < n_r; ++i) {
            for (int j = 0; j < n_t; ++j)
                for (int p = 0; p < P; ++p) {
                    double acc = 0.0;
                    for (int k = 0; k < n_p; ++k)
                        acc += Iph[(size_t)p * n_p + k] * (4.0 * ORC_PI * G * rho[((size_t)i * n_t + j) * n_p + k]);
                    F[(size_t)j * P + p] = acc;
                }
            for (int l = 0; l <= L; ++l)
                for (int m = 0; m <= l; ++m)
                    for (int a = 0; a < (m == 0 ? 1 : 2); ++a) {
                        int p = pcol(m, a), t = tri(l, m);
                        double acc = 0.0;
                        for (int j = 0; j < n_t; ++j) acc += Ith[(size_t)t * n_t + j] * F[(size_t)j * P + p];
                        A[(size_t)i * KL + l * l + p] = acc;
                    }
        }
        free(F);
    }
}

/* ------------------------------------------------------------------------ */
/* Steps (b), (c): radial moments on the n_r + 1 shell edges (Sec. 2.2).    */
/*   MR_0 = 0,      MR_{i+1} = MR_i + (Delta(r^3/3))_i (R^R_l)_i A_i         */
/*   MI_{n_r} = 0,  MI_i     = MI_{i+1} + (Delta(r^3/3))_i (R^I_l)_i A_i     */
/* with (R)_i = W/V the volume-mean kernels.  Reading R4: at r_0 = 0 and    */
/* l >= 2 the divergent own-shell term of MI_0 is left out.                  */
/* ------------------------------------------------------------------------ */
void orc_radial_moments(int n_r, int L, const double *r, const double *WR, const double *WI,
                        const double *V, const double *A, double *MR, double *MI)
{
    int KL = (L + 1) * (L + 1);
    int origin = (r[0] == 0.0);
    for (int l = 0; l <= L; ++l)
        for (int p = 0; p <= 2 * l; ++p) {
            int q = l * l + p;
            MR[q] = 0.0;
            for (int i = 0; i < n_r; ++i) {
                double RR = WR[(size_t)l * n_r + i] / V[i];
                MR[(size_t)(i + 1) * KL + q] = MR[(size_t)i * KL + q] + V[i] * RR * A[(size_t)i * KL + q];
            }
            MI[(size_t)n_r * KL + q] = 0.0;
            for (int i = n_r - 1; i >= 0; --i) {
                if (i == 0 && origin && l >= 2) {
                    MI[q] = MI[(size_t)KL + q];
                    continue;
                }
                double RI = WI[(size_t)l * n_r + i] / V[i];
                MI[(size_t)i * KL + q] = MI[(size_t)(i + 1) * KL + q] + V[i] * RI * A[(size_t)i * KL + q];
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Step (d): cell-centre radial moments by linear interpolation (R3) and    */
/* the per-shell coefficient of every angular kernel in Eq. (Solution):     */
/*   C[i][q] = -(Delta_m/(2l+1)) [ (R^R)_i Mbar^I_i + (R^I)_i Mbar^R_i ]    */
/* Delta_m = 2 - delta_m0 (Eq. Delta).  Reading R4 at the origin shell.     */
/* ------------------------------------------------------------------------ */
void orc_solution_coefficients(int n_r, int L, const double *r, const double *WR, const double *WI,
                               const double *V, const double *A, const double *MR, const double *MI,
                               double *C)
{
    int KL = (L + 1) * (L + 1);
    int origin = (r[0] == 0.0);
    for (int i = 0; i < n_r; ++i)
        for (int l = 0; l <= L; ++l) {
            double RR = WR[(size_t)l * n_r + i] / V[i];
            double RI = WI[(size_t)l * n_r + i] / V[i];
            for (int p = 0; p <= 2 * l; ++p) {
                int q = l * l + p;
                int m = (p + 1) / 2;
                double Delta = (m == 0) ? 1.0 : 2.0;
                double pre = -Delta / (2.0 * l + 1.0);
                if (i == 0 && origin && l >= 2) {
                    double Sself = 6.0 * r[1] * r[1] / (5.0 * (l + 3.0));
                    C[(size_t)i * KL + q] = pre * (RR * MI[(size_t)1 * KL + q] + Sself * A[q]);
                } else {
                    double MbarR = 0.5 * (MR[(size_t)i * KL + q] + MR[(size_t)(i + 1) * KL + q]);
                    double MbarI = 0.5 * (MI[(size_t)i * KL + q] + MI[(size_t)(i + 1) * KL + q]);
                    C[(size_t)i * KL + q] = pre * (RR * MbarI + RI * MbarR);
                }
            }
        }
}

/* Phi_ijk = sum_q C[i][q] (A_q)_jk, cell-averaged kernels (Eq. Solution). */
void orc_potential_literal(int n_r, int n_t, int n_p, int L, const double *th, const double *ph,
                           const double *Ith, const double *Iph, const double *C, double *phi)
{
    int KL = (L + 1) * (L + 1);
    double *dmu = (double *)malloc(sizeof(double) * n_t);
    double *dph = (double *)malloc(sizeof(double) * n_p);
    cell_widths(n_t, th, n_p, ph, dmu, dph);
    orc_apply_threads();
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n_r; ++i)
        for (int j = 0; j < n_t; ++j)
            for (int k = 0; k < n_p; ++k) {
                double acc = 0.0;
                for (int l = 0; l <= L; ++l)
                    for (int m = 0; m <= l; ++m)
                        for (int a = 0; a < (m == 0 ? 1 : 2); ++a) {
                            int p = pcol(m, a), t = tri(l, m);
                            double Aavg = (Ith[(size_t)t * n_t + j] / dmu[j]) * (Iph[(size_t)p * n_p + k] / dph[k]);
                            acc += C[(size_t)i * KL + l * l + p] * Aavg;
                        }
                phi[((size_t)i * n_t + j) * n_p + k] = acc;
            }
    free(dmu);
    free(dph);
}

/* Same sum factored over the separable kernel: G[j][p] = sum_l Ith/dmu C,
 * then Phi_ijk = sum_p G[j][p] Iph/dphi. */
void orc_potential_factored(int n_r, int n_t, int n_p, int L, const double *th, const double *ph,
                            const double *Ith, const double *Iph, const double *C, double *phi)
{
    int KL = (L + 1) * (L + 1), P = 2 * L + 1;
    double *dmu = (double *)malloc(sizeof(double) * n_t);
    double *dph = (double *)malloc(sizeof(double) * n_p);
    cell_widths(n_t, th, n_p, ph, dmu, dph);
    orc_apply_threads();
#pragma omp parallel
    {
        double *Gp = (double *)malloc(sizeof(double) * P);
#pragma omp for schedule(dynamic)
        for (int i = 0; i < n_r; ++i)
            for (int j = 0; j < n_t; ++j) {
                for (int p = 0; p < P; ++p) {
                    int m = (p + 1) / 2;
                    double acc = 0.0;
                    for (int l = m; l <= L; ++l)
                        acc += (Ith[(size_t)tri(l, m) * n_t + j] / dmu[j]) * C[(size_t)i * KL + l * l + p];
                    Gp[p] = acc;
                }
                for (int k = 0; k < n_p; ++k) {
                    double acc = 0.0;
                    for (int p = 0; p < P; ++p) acc += Gp[p] * (Iph[(size_t)p * n_p + k] / dph[k]);
                    phi[((size_t)i * n_t + j) * n_p + k] = acc;
                }
            }
        free(Gp);
    }
    free(dmu);
    free(dph);
}

/* ------------------------------------------------------------------------ */
/* Whole solve: (a) moments, (b)+(c) radial recurrences, (d) potential.     */
/* literal != 0 selects the per-cell double sums, else the factored sums.   */
/* Tables come from orc_theta_integrals, orc_phi_integrals, orc_radial.     */
/* ------------------------------------------------------------------------ */
int orc_solve(int n_r, int n_t, int n_p, int L, const double *r, const double *th, const double *ph,
              const double *Ith, const double *Iph, const double *WR, const double *WI, const double *V,
              double G, const double *rho, int literal, double *A, double *MR, double *MI, double *C,
              double *phi)
{
    if (n_r < 1 || n_t < 1 || n_p < 1 || L < 0) return -1;
    if (literal)
        orc_moments_literal(n_r, n_t, n_p, L, th, ph, Ith, Iph, G, rho, A);
    else
        orc_moments_factored(n_r, n_t, n_p, L, Ith, Iph, G, rho, A);
    orc_radial_moments(n_r, L, r, WR, WI, V, A, MR, MI);
    orc_solution_coefficients(n_r, L, r, WR, WI, V, A, MR, MI, C);
    if (phi) {
        if (literal)
            orc_potential_literal(n_r, n_t, n_p, L, th, ph, Ith, Iph, C, phi);
        else
            orc_potential_factored(n_r, n_t, n_p, L, th, ph, Ith, Iph, C, phi);
    }
    return 0;
}

/* Potential of selected shells only, from precomputed coefficients C
 * (used to sample very large meshes shell by shell). */
void orc_potential_shells(int n_r, int n_t, int n_p, int L, const double *th, const double *ph,
                          const double *Ith, const double *Iph, const double *C, int n_sel,
                          const int *shells, double *phi_sel)
{
    int KL = (L + 1) * (L + 1);
    size_t cells = (size_t)n_t * n_p;
    (void)n_r;
    for (int s = 0; s < n_sel; ++s)
        orc_potential_factored(1, n_t, n_p, L, th, ph, Ith, Iph, C + (size_t)shells[s] * KL,
                               phi_sel + (size_t)s * cells);
}

/* ------------------------------------------------------------------------ */
/* Dense Green's-matrix restatement of the same discretisation, without     */
/* radial recurrences (tiny meshes only, O(N^2 K_L)):                       */
/*   Phi_c = sum_c' sum_q -(Delta_m/(2l+1)) (A_q)_c (dOmega A_q)_c' S_c'     */
/*                    g_l(i, i')                                            */
/*   g_l = (R^I)_i W^R_i'              for i' < i                           */
/*       = (R^R)_i W^I_i'              for i' > i                           */
/*       = [(R^R)_i W^I_i + (R^I)_i W^R_i] / 2   for i' = i (midpoint split)  */
/*       = S_self(l)                   for i = i' = 0, r_0 = 0, l >= 2 (R4) */
/* ------------------------------------------------------------------------ */
void orc_potential_green(int n_r, int n_t, int n_p, int L, const double *r, const double *th,
                         const double *ph, const double *Ith, const double *Iph, const double *WR,
                         const double *WI, const double *V, double G, const double *rho, double *phi)
{
    int origin = (r[0] == 0.0);
    double *dmu = (double *)malloc(sizeof(double) * n_t);
    double *dph = (double *)malloc(sizeof(double) * n_p);
    cell_widths(n_t, th, n_p, ph, dmu, dph);
    size_t N = (size_t)n_r * n_t * n_p;
    orc_apply_threads();
#pragma omp parallel for schedule(dynamic)
    for (long c = 0; c < (long)N; ++c) {
        int i = (int)(c / ((size_t)n_t * n_p));
        int j = (int)((c / n_p) % n_t);
        int k = (int)(c % n_p);
        double acc = 0.0;
        for (size_t c2 = 0; c2 < N; ++c2) {
            int i2 = (int)(c2 / ((size_t)n_t * n_p));
            int j2 = (int)((c2 / n_p) % n_t);
            int k2 = (int)(c2 % n_p);
            double S = 4.0 * ORC_PI * G * rho[c2];
            for (int l = 0; l <= L; ++l) {
                double g;
                double RRi = WR[(size_t)l * n_r + i] / V[i];
                double RIi = WI[(size_t)l * n_r + i] / V[i];
                if (i == 0 && i2 == 0 && origin && l >= 2)
                    g = 6.0 * r[1] * r[1] / (5.0 * (l + 3.0));
                else if (i2 < i)
                    g = RIi * WR[(size_t)l * n_r + i2];
                else if (i2 > i)
                    g = RRi * WI[(size_t)l * n_r + i2];
                else
                    g = 0.5 * (RRi * WI[(size_t)l * n_r + i] + RIi * WR[(size_t)l * n_r + i]);
                for (int m = 0; m <= l; ++m) {
                    double Delta = (m == 0) ? 1.0 : 2.0;
                    int t = tri(l, m);
                    for (int a = 0; a < (m == 0 ? 1 : 2); ++a) {
                        int p = pcol(m, a);
                        double Ac = (Ith[(size_t)t * n_t + j] / dmu[j]) * (Iph[(size_t)p * n_p + k] / dph[k]);
                        double dOA = Ith[(size_t)t * n_t + j2] * Iph[(size_t)p * n_p + k2];
                        acc += -(Delta / (2.0 * l + 1.0)) * Ac * dOA * S * g;
                    }
                }
            }
        }
        phi[c] = acc;
    }
    free(dmu);
    free(dph);
}
