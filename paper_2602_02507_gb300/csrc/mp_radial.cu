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

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanThreads = 128;  // threads per moment column

// Exclusive prefix (forward) and exclusive suffix (backward) of one value per
// thread over the block, by warp shuffles plus one shared-memory pass over the
// warp totals.  Only additions: no prefix is formed by subtracting from a total
// (inward moments of high degree fall by many decades, a difference would cancel).
template <int NT>
__device__ __forceinline__ void block_exclusive_scans(double xf, double xb, double &exf, double &exb,
                                                      double (*wt)[NT / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double inf = xf, inb = xb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double yf = __shfl_up_sync(kFull, inf, o);
        const double yb = __shfl_down_sync(kFull, inb, o);
        if (lane >= o) inf += yf;
        if (lane + o < 32) inb += yb;
    }
    double ef = __shfl_up_sync(kFull, inf, 1);
    double eb = __shfl_down_sync(kFull, inb, 1);
    if (lane == 0) ef = 0.0;
    if (lane == 31) eb = 0.0;
    if (lane == 31) wt[0][w] = inf;
    if (lane == 0) wt[1][w] = inb;
    __syncthreads();
    double of = 0.0, ob = 0.0;
    for (int w2 = 0; w2 < w; ++w2) of += wt[0][w2];
    for (int w2 = NT / 32 - 1; w2 > w; --w2) ob += wt[1][w2];
    exf = of + ef;
    exb = ob + eb;
}

// One block per moment column q; thread t owns shells [t*chunk, (t+1)*chunk).
template <int NT>
__global__ void __launch_bounds__(NT) k_scan(const double *__restrict__ A, const double *__restrict__ WR,
                                             const double *__restrict__ WI, const double *__restrict__ RR,
                                             const double *__restrict__ RI, double *__restrict__ MR,
                                             double *__restrict__ MI, double *__restrict__ C,
                                             float *__restrict__ C32, int n_r, int KL, int origin, double r1sq)
{
    __shared__ double wt[2][NT / 32];
    const int q = blockIdx.x;
    int l = (int)sqrtf((float)q);
    while (l * l > q) --l;
    while ((l + 1) * (l + 1) <= q) ++l;
    const int p = q - l * l;
    const int m = pcol_m(p);
    const int chunk = (n_r + NT - 1) / NT;
    const int i0 = min(n_r, (int)threadIdx.x * chunk), i1 = min(n_r, i0 + chunk);
    const double *wr = WR + (size_t)l * n_r;
    const double *wi = WI + (size_t)l * n_r;
    double sR = 0.0, sI = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double a = A[(size_t)i * KL + q];
        sR = fma(wr[i], a, sR);
        sI = fma(wi[i], a, sI);
    }
    double mr, mi;
    block_exclusive_scans<NT>(sR, sI, mr, mi, wt);
    // outward: edges i0 .. i1-1; the last thread also writes edge n_r
    for (int i = i0; i < i1; ++i) {
        MR[(size_t)i * KL + q] = mr;
        mr = fma(wr[i], A[(size_t)i * KL + q], mr);
    }
    if (threadIdx.x == NT - 1) {
        MR[(size_t)n_r * KL + q] = mr;
        MI[(size_t)n_r * KL + q] = mi;
    }
    // inward: edges i1-1 .. i0 and the coefficients of every shell of the chunk
    const double half_pre = -0.5 * ((m == 0) ? 1.0 : 2.0) / (2.0 * l + 1.0);
    for (int i = i1 - 1; i >= i0; --i) {
        const double a = A[(size_t)i * KL + q];
        const double mi_hi = mi;
        mi = fma(wi[i], a, mi);
        MI[(size_t)i * KL + q] = mi;
        const double mr_lo = MR[(size_t)i * KL + q];
        const double mr_hi = fma(wr[i], a, mr_lo);
        double c;
        if (origin && i == 0 && l >= 2) {
            const double sself = 6.0 * r1sq / (5.0 * (l + 3.0));
            c = 2.0 * half_pre * (RR[(size_t)l * n_r] * mi_hi + sself * a);
        } else {
            c = half_pre * (RR[(size_t)l * n_r + i] * (mi + mi_hi) + RI[(size_t)l * n_r + i] * (mr_lo + mr_hi));
        }
        C[(size_t)i * KL + q] = c;
        if (C32) C32[(size_t)i * KL + q] = (float)c;
    }
}

// Split path, theta part of step (a): A[i][q] = 4 pi G sum_j Ith[t][j] F[i n_t + j][p]
// in float32 with compensated (Kahan) summation.  Block (i, g) handles shell i
// and moments [g * 256 QPT, (g+1) * 256 QPT).  The shell's F rows and the
// matching table rows pass through shared memory in chunks of JC polar cells;
// each thread owns QPT moments and keeps two Kahan streams per moment (even and
// odd polar cells), merged in float64 at the end.
template <int QPT>
__global__ void __launch_bounds__(256) k32_theta(const float *__restrict__ F, const float *__restrict__ IthT,
                                                 double *__restrict__ A, int n_t, int KL, int T, int Npad, int JC,
                                                 double scale)
{
    extern __shared__ float smem_t[];
    float *sF = smem_t;                       // [JC][Npad]
    float *sT = smem_t + (size_t)JC * Npad;   // [JC][T]
    const int i = blockIdx.x;
    const int qbase = blockIdx.y * blockDim.x * QPT;
    int tq[QPT], pq[QPT];
    float s0[QPT], c0[QPT], s1[QPT], c1[QPT];
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
        const int q = qbase + threadIdx.x + u * blockDim.x;
        int l = (int)sqrtf((float)q);
        while (l * l > q) --l;
        while ((l + 1) * (l + 1) <= q) ++l;
        const int p = q - l * l;
        tq[u] = (q < KL) ? tri(l, pcol_m(p)) : 0;
        pq[u] = (q < KL) ? p : 0;
        s0[u] = c0[u] = s1[u] = c1[u] = 0.0f;
    }
    const float *Fi = F + (size_t)i * n_t * Npad;
    for (int j0 = 0; j0 < n_t; j0 += JC) {
        const int nj = min(JC, n_t - j0);
        __syncthreads();
        {
            const float4 *src = reinterpret_cast<const float4 *>(Fi + (size_t)j0 * Npad);
            float4 *dst = reinterpret_cast<float4 *>(sF);
            for (int e = threadIdx.x; e < nj * Npad / 4; e += blockDim.x) dst[e] = src[e];
            const float *tsrc = IthT + (size_t)j0 * T;
            for (int e = threadIdx.x; e < nj * T; e += blockDim.x) sT[e] = __ldg(tsrc + e);
        }
        __syncthreads();
        int j = 0;
        for (; j + 1 < nj; j += 2) {
            const float *ta = sT + (size_t)j * T, *tb = ta + T;
            const float *fa = sF + j * Npad, *fb = fa + Npad;
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const float ya = __fmul_rn(ta[tq[u]], fa[pq[u]]) - c0[u];
                const float yb = __fmul_rn(tb[tq[u]], fb[pq[u]]) - c1[u];
                const float xa = __fadd_rn(s0[u], ya);
                const float xb = __fadd_rn(s1[u], yb);
                c0[u] = __fsub_rn(__fsub_rn(xa, s0[u]), ya);
                c1[u] = __fsub_rn(__fsub_rn(xb, s1[u]), yb);
                s0[u] = xa;
                s1[u] = xb;
            }
        }
        if (j < nj) {
            const float *ta = sT + (size_t)j * T;
            const float *fa = sF + j * Npad;
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const float ya = __fmul_rn(ta[tq[u]], fa[pq[u]]) - c0[u];
                const float xa = __fadd_rn(s0[u], ya);
                c0[u] = __fsub_rn(__fsub_rn(xa, s0[u]), ya);
                s0[u] = xa;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
        const int q = qbase + threadIdx.x + u * blockDim.x;
        if (q < KL)
            A[(size_t)i * KL + q] = scale * (((double)s0[u] - (double)c0[u]) + ((double)s1[u] - (double)c1[u]));
    }
}

// Same contraction, persistent: the whole table IthT [n_t][T] stays in shared
// memory and each block walks shells i = blockIdx.x, blockIdx.x + gridDim.x, ...
// staging one shell's F rows at a time (used when the table fits).  Each thread
// owns moments q = threadIdx.x + k blockDim.x; terms are summed in float32 in
// blocks of eight polar cells and the block sums are added with Kahan
// compensation.
__global__ void __launch_bounds__(1024) k32_theta_res(const float *__restrict__ F, const float *__restrict__ IthT,
                                                      double *__restrict__ A, int n_r, int n_t, int KL, int T,
                                                      int Npad, double scale)
{
    extern __shared__ float smem_t[];
    float *sT = smem_t;                        // [n_t][T]
    float *sF = smem_t + (((size_t)n_t * T + 3) & ~(size_t)3);  // [n_t][Npad]
    const int nT = n_t * T;
    {
        const float4 *src = reinterpret_cast<const float4 *>(IthT);
        float4 *dst = reinterpret_cast<float4 *>(sT);
        const int n4 = nT / 4;
        for (int e0 = threadIdx.x; e0 < n4; e0 += 8 * blockDim.x) {
            float4 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = e0 + k * blockDim.x;
                if (e < n4) v[k] = __ldg(src + e);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = e0 + k * blockDim.x;
                if (e < n4) dst[e] = v[k];
            }
        }
        for (int e = n4 * 4 + threadIdx.x; e < nT; e += blockDim.x) sT[e] = __ldg(IthT + e);
    }
    const int n4F = n_t * Npad / 4;
    for (int i = blockIdx.x; i < n_r; i += gridDim.x) {
        __syncthreads();  // previous shell's rows fully read (and, the first time, the table stored)
        {
            const float4 *src = reinterpret_cast<const float4 *>(F + (size_t)i * n_t * Npad);
            float4 *dst = reinterpret_cast<float4 *>(sF);
            for (int e0 = threadIdx.x; e0 < n4F; e0 += 8 * blockDim.x) {
                float4 v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = e0 + k * blockDim.x;
                    if (e < n4F) v[k] = __ldcs(src + e);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = e0 + k * blockDim.x;
                    if (e < n4F) dst[e] = v[k];
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < KL; q += blockDim.x) {
            int l = (int)sqrtf((float)q);
            while (l * l > q) --l;
            while ((l + 1) * (l + 1) <= q) ++l;
            const int p = q - l * l;
            const float *tcol = sT + tri(l, pcol_m(p));
            const float *fcol = sF + p;
            float s = 0.0f, c = 0.0f;
            int j = 0;
            for (; j + 8 <= n_t; j += 8) {
                float b0 = 0.0f, b1 = 0.0f;
#pragma unroll
                for (int jj = 0; jj < 8; jj += 2) {
                    b0 = fmaf(tcol[(size_t)(j + jj) * T], fcol[(j + jj) * Npad], b0);
                    b1 = fmaf(tcol[(size_t)(j + jj + 1) * T], fcol[(j + jj + 1) * Npad], b1);
                }
                const float y = (b0 + b1) - c;
                const float t = s + y;
                c = (t - s) - y;
                s = t;
            }
            float b0 = 0.0f;
            for (; j < n_t; ++j) b0 = fmaf(tcol[(size_t)j * T], fcol[j * Npad], b0);
            const float y = b0 - c;
            const float t = s + y;
            c = (t - s) - y;
            s = t;
            A[(size_t)i * KL + q] = scale * ((double)s - (double)c);
        }
    }
}

}  // namespace

cudaError_t launch_scan(mp_mesh *m, int want_f32)
{
    const double r1sq = m->h_r[1] * m->h_r[1];
    cudaEvent_t ev;
    prof_begin(m, "radial_scan", &ev);
    k_scan<kScanThreads><<<m->KL, kScanThreads, 0, m->stream>>>(m->d_A, m->d_WR, m->d_WI, m->d_RR, m->d_RI, m->d_MR,
                                                                m->d_MI, m->d_C, want_f32 ? m->d_C32 : nullptr,
                                                                m->n_r, m->KL, m->origin, r1sq);
    prof_end(m, "radial_scan", ev);
    return cudaGetLastError();
}

template <int QPT>
static void theta_launch(mp_mesh *m, int JC, size_t smem, double scale)
{
    const dim3 grid(m->n_r, (m->KL + 256 * QPT - 1) / (256 * QPT));
    k32_theta<QPT><<<grid, 256, smem, m->stream>>>(m->d_F32, m->d_IthT32, m->d_A, m->n_t, m->KL, m->T,
                                                   m->plan.Npad, JC, scale);
}

static void theta_res_launch(mp_mesh *m, size_t smem, double scale)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k32_theta_res, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
        attr_set = true;
    }
    const int threads = std::min(1024, 32 * ((m->KL + 31) / 32));
    const int grid = std::min(m->n_r, 2 * m->num_sms);
    k32_theta_res<<<grid, threads, smem, m->stream>>>(m->d_F32, m->d_IthT32, m->d_A, m->n_r, m->n_t, m->KL, m->T,
                                                      m->plan.Npad, scale);
}

cudaError_t launch_split_theta(mp_mesh *m)
{
    constexpr double kFourPi = 12.566370614359172954;
    const int Npad = m->plan.Npad;
    // resident table: two blocks per SM when table + one shell's rows fit in 112 KB
    const size_t res_smem = ((((size_t)m->n_t * m->T + 3) & ~(size_t)3) + (size_t)m->n_t * Npad) * sizeof(float);
    if (res_smem <= 112 * 1024) {
        cudaEvent_t ev;
        prof_begin(m, "split_theta_contract", &ev);
        theta_res_launch(m, res_smem, kFourPi * m->G);
        prof_end(m, "split_theta_contract", ev);
        return cudaGetLastError();
    }
    // polar cells per chunk: F rows plus table rows within 48 KB of shared memory
    const int JC = std::max(1, std::min(m->n_t, (48 * 1024) / ((Npad + m->T) * 4)));
    const size_t smem = (size_t)JC * (Npad + m->T) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k32_theta<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k32_theta<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k32_theta<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k32_theta<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const int qpt = (m->KL + 255) / 256;
    const double scale = kFourPi * m->G;
    cudaEvent_t ev;
    prof_begin(m, "split_theta_contract", &ev);
    if (qpt <= 1)
        theta_launch<1>(m, JC, smem, scale);
    else if (qpt <= 2)
        theta_launch<2>(m, JC, smem, scale);
    else if (qpt <= 4)
        theta_launch<4>(m, JC, smem, scale);
    else
        theta_launch<8>(m, JC, smem, scale);
    prof_end(m, "split_theta_contract", ev);
    return cudaGetLastError();
}

}  // namespace mp
