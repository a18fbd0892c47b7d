// mp_fp64.cu -- the plain float64 path: every contraction on CUDA cores in
// float64 (GB300's float64 rate bounds it).  Steps of GenASiS II Sec. 2.2:
//   (a1) F[row][p]  = sum_k Iph[p][k] rho[row][k]                 (phi part of Eq. AngularMomentsDiscrete)
//   (a2) A[i][q]    = 4 pi G sum_j Ith[t][j] F[i n_t + j][p]      (theta part)
//   (d1) G[row][p]  = sum_{l>=m} (Ith[t][j] / dmu_j) C[i][q]       (theta part of Eq. Solution)
//   (d2) Phi[row][k]= sum_p G[row][p] Iph[p][k] / dphi_k           (phi part)
// with row = i n_t + j, q = l^2 + p, t = t(l, m(p)).
#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

constexpr double kFourPi = 12.566370614359172954;

// (a1): one block per group of rows; rho rows staged in shared memory.
constexpr int kRowsPerBlock = 4;

__global__ void __launch_bounds__(256) k64_project(const double *__restrict__ rho, const double *__restrict__ Iph,
                                                   double *__restrict__ F, long long R, int n_p, int P, int *err)
{
    extern __shared__ double srow[];  // [kRowsPerBlock][n_p]
    const long long row0 = (long long)blockIdx.x * kRowsPerBlock;
    const int nrows = (int)min((long long)kRowsPerBlock, R - row0);
    bool bad = false;
    for (int e = threadIdx.x; e < nrows * n_p; e += blockDim.x) {
        const double v = rho[row0 * n_p + e];
        bad |= !isfinite(v);
        srow[e] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, DEV_ERR_NONFINITE);
    for (int o = threadIdx.x; o < nrows * P; o += blockDim.x) {
        const int rr = o / P, p = o % P;
        const double *s = srow + (size_t)rr * n_p;
        const double *w = Iph + (size_t)p * n_p;
        double acc = 0.0;
        for (int k = 0; k < n_p; ++k) acc = fma(w[k], s[k], acc);
        F[(row0 + rr) * P + p] = acc;
    }
}

// (a2): one block per shell, one thread per moment.
__global__ void __launch_bounds__(256) k64_theta(const double *__restrict__ F, const double *__restrict__ Ith,
                                                 double *__restrict__ A, int n_t, int L, int KL, int P, double scale)
{
    const int i = blockIdx.x;
    for (int q = threadIdx.x; q < KL; q += blockDim.x) {
        int l = 0;
        while ((l + 1) * (l + 1) <= q) ++l;
        const int p = q - l * l;
        const int t = tri(l, pcol_m(p));
        const double *f = F + (size_t)i * n_t * P + p;
        const double *w = Ith + (size_t)t * n_t;
        double acc = 0.0;
        for (int j = 0; j < n_t; ++j) acc = fma(w[j], f[(size_t)j * P], acc);
        A[(size_t)i * KL + q] = scale * acc;
    }
}

// (d1): one thread per (row, p).
__global__ void __launch_bounds__(256) k64_synth_theta(const double *__restrict__ C, const double *__restrict__ Ith,
                                                       const double *__restrict__ dmu, double *__restrict__ Gm,
                                                       long long R, int n_t, int L, int KL, int P)
{
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= R * P) return;
    const long long row = o / P;
    const int p = (int)(o % P);
    const int i = (int)(row / n_t), j = (int)(row % n_t);
    const int m = pcol_m(p);
    const double inv = 1.0 / dmu[j];
    double acc = 0.0;
    for (int l = m; l <= L; ++l) acc = fma(Ith[(size_t)tri(l, m) * n_t + j] * inv, C[(size_t)i * KL + l * l + p], acc);
    Gm[o] = acc;
}

// (d2): one thread per cell.
__global__ void __launch_bounds__(256) k64_synth_phi(const double *__restrict__ Gm, const double *__restrict__ Iphc,
                                                     double *__restrict__ phi, long long N, int n_p, int P)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const long long row = c / n_p;
    const int k = (int)(c % n_p);
    const double *g = Gm + row * P;
    double acc = 0.0;
    for (int p = 0; p < P; ++p) acc = fma(g[p], Iphc[(size_t)p * n_p + k], acc);
    phi[c] = acc;
}

}  // namespace

cudaError_t launch_fp64_project(mp_mesh *m, const double *rho)
{
    const long long blocks = (m->R + kRowsPerBlock - 1) / kRowsPerBlock;
    const size_t smem = (size_t)kRowsPerBlock * m->n_p * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k64_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaEvent_t ev;
    prof_begin(m, "fp64_phi_project", &ev);
    k64_project<<<(unsigned)blocks, 256, smem, m->stream>>>(rho, m->d_Iph, m->d_F64, m->R, m->n_p, m->P, m->d_err);
    prof_end(m, "fp64_phi_project", ev);
    return cudaGetLastError();
}

cudaError_t launch_fp64_moments_into(const mp_mesh *m, const double *rho, double *F, double *A)
{
    const long long blocks = (m->R + kRowsPerBlock - 1) / kRowsPerBlock;
    const size_t smem = (size_t)kRowsPerBlock * m->n_p * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k64_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k64_project<<<(unsigned)blocks, 256, smem, m->stream>>>(rho, m->d_Iph, F, m->R, m->n_p, m->P, m->d_err);
    k64_theta<<<m->n_r, 256, 0, m->stream>>>(F, m->d_Ith, A, m->n_t, m->L, m->KL, m->P, kFourPi * m->G);
    return cudaGetLastError();
}

cudaError_t launch_fp64_theta(mp_mesh *m)
{
    cudaEvent_t ev;
    prof_begin(m, "fp64_theta_contract", &ev);
    k64_theta<<<m->n_r, 256, 0, m->stream>>>(m->d_F64, m->d_Ith, m->d_A, m->n_t, m->L, m->KL, m->P,
                                            kFourPi * m->G);
    prof_end(m, "fp64_theta_contract", ev);
    return cudaGetLastError();
}

cudaError_t launch_fp64_synth(mp_mesh *m, double *phi)
{
    cudaEvent_t ev;
    prof_begin(m, "fp64_theta_synth", &ev);
    {
        const long long n = m->R * m->P;
        k64_synth_theta<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_C, m->d_Ith, m->d_dmu, m->d_G64,
                                                                            m->R, m->n_t, m->L, m->KL, m->P);
    }
    prof_end(m, "fp64_theta_synth", ev);
    prof_begin(m, "fp64_phi_synth", &ev);
    k64_synth_phi<<<(unsigned)((m->N + 255) / 256), 256, 0, m->stream>>>(m->d_G64, m->d_Iphc, phi, m->N, m->n_p,
                                                                         m->P);
    prof_end(m, "fp64_phi_synth", ev);
    return cudaGetLastError();
}

}  // namespace mp
