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
//   C[i][q] = -(Delta_m / (2l+1)) [ (R^R)_i Mbar^I + (R^I)_i Mbar^R ]
//           = (Delta_m / 2) [ GR_i (MI_i + MI_{i+1}) + GI_i (MR_i + MR_{i+1}) ]
// with the tables GR, GI = -(R^R, R^I) / (2 (2l+1)) and Delta_m / 2 = 1 or 2
// (a doubling, exact).  The float64 pipe is narrow on this part, so the scans
// keep float64 operations to the recurrences themselves.
// A shell touching r = 0 uses, for l >= 2, the exact own-shell value
// 6 r_1^2 / (5 (l+3)) A[0][q] in place of the divergent midpoint split; the
// tables carry it (GI at the origin shell), so the scans have no special case.
#include "mp_internal.h"
#include "ptx.cuh"

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

// C[i][l^2 + p] (m >= 1) as the bf16 terms of the tensor-core theta synthesis B operand
// (layout: CbOut in mp_internal.h).
__device__ __forceinline__ void write_cb(const CbOut &o, int i, int l, int p, float c32)
{
    const int m = pcol_m(p), a = (p + 1) & 1;
    const int k = l - m, n_kcm = (o.L + 1 - m + 31) >> 5;
    const int sg = i / o.NS, n = 2 * (i - sg * o.NS) + a;
    const size_t c_term = (size_t)2 * o.NS * 64;
    uint8_t *base = o.cb + o.off[m] + ((size_t)sg * n_kcm + (k >> 5)) * o.terms * c_term + (size_t)(n >> 3) * 512 +
                    ((k & 31) >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(c32);
    const float r1 = c32 - __bfloat162float(h0);
    const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
    *reinterpret_cast<__nv_bfloat16 *>(base) = h0;
    *reinterpret_cast<__nv_bfloat16 *>(base + c_term) = h1;
    if (o.terms == 3) *reinterpret_cast<__nv_bfloat16 *>(base + 2 * c_term) = __float2bfloat16_rn(r1 - __bfloat162float(h1));
}

// One block per moment column q; thread t owns shells [t*chunk, (t+1)*chunk).
template <int NT>
__global__ void __launch_bounds__(NT) k_scan(const double *__restrict__ A, const double *__restrict__ WR,
                                             const double *__restrict__ WI, const double *__restrict__ GR,
                                             const double *__restrict__ GI, double *__restrict__ MR,
                                             double *__restrict__ MI, double *__restrict__ C,
                                             float *__restrict__ C32, float2 *__restrict__ C0, int n_r, int KL,
                                             const CbOut cbo, const double *__restrict__ off)
{
    __shared__ double wt[2][NT / 32];
    // the next kernel's blocks may start (and copy their tables) while this one runs
    pdl_trigger();
    pdl_wait();  // A comes from the previous kernel
    const int q = blockIdx.x;
    int l = (int)sqrtf((float)q);
    while (l * l > q) --l;
    while ((l + 1) * (l + 1) <= q) ++l;
    const int p = q - l * l;
    const int m = pcol_m(p);
    const int Lp1 = (int)sqrtf((float)KL + 0.5f);  // L + 1
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
    if (off) {  // the sums of the slabs below (regular) and above (irregular) this one
        mr += off[q];
        mi += off[KL + q];
    }
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
    for (int i = i1 - 1; i >= i0; --i) {
        const double a = A[(size_t)i * KL + q];
        const double mi_hi = mi;
        mi = fma(wi[i], a, mi);
        MI[(size_t)i * KL + q] = mi;
        const double mr_lo = MR[(size_t)i * KL + q];
        const double mr_hi = fma(wr[i], a, mr_lo);
        double c = fma(GI[(size_t)l * n_r + i], mr_lo + mr_hi, GR[(size_t)l * n_r + i] * (mi + mi_hi));
        if (m > 0) c += c;
        if (C) C[(size_t)i * KL + q] = c;
        const float c32 = f64_to_f32_alu(c);
        if (C32) C32[(size_t)i * KL + q] = c32;
        if (C0 && p == 0) C0[(size_t)i * Lp1 + l] = f32_pair(c);
        if (cbo.cb && p > 0) write_cb(cbo, i, l, p, c32);
    }
}

// Same recurrences with each thread's chunk of CH shells held in registers
// (moments, weights and edge values are loaded once, all loads up front).
template <int NT, int CH>
__global__ void __launch_bounds__(NT) k_scan_reg(const double *__restrict__ A, const double *__restrict__ WR,
                                                 const double *__restrict__ WI, const double *__restrict__ GR,
                                                 const double *__restrict__ GI, double *__restrict__ MR,
                                                 double *__restrict__ MI, double *__restrict__ C,
                                                 float *__restrict__ C32, float2 *__restrict__ C0, int n_r, int KL,
                                                 const CbOut cbo, const double *__restrict__ off)
{
    __shared__ double wt[2][NT / 32];
    // the next kernel's blocks may start (and copy their tables) while this one runs
    pdl_trigger();
    pdl_wait();  // A comes from the previous kernel
    const int q = blockIdx.x;
    int l = (int)sqrtf((float)q);
    while (l * l > q) --l;
    while ((l + 1) * (l + 1) <= q) ++l;
    const int p = q - l * l;
    const int m = pcol_m(p);
    const int Lp1 = (int)sqrtf((float)KL + 0.5f);  // L + 1
    const int i0 = (int)threadIdx.x * CH;
    const double *wr = WR + (size_t)l * n_r;
    const double *wi = WI + (size_t)l * n_r;
    const double *gr = GR + (size_t)l * n_r;
    const double *gi = GI + (size_t)l * n_r;
    double a[CH], w1[CH], w2[CH], g1[CH], g2[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        const int i = i0 + k;
        const bool in = i < n_r;
        a[k] = in ? A[(size_t)i * KL + q] : 0.0;
        w1[k] = in ? wr[i] : 0.0;
        w2[k] = in ? wi[i] : 0.0;
        g1[k] = in ? gr[i] : 0.0;
        g2[k] = in ? gi[i] : 0.0;
    }
    double sR = 0.0, sI = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        sR = fma(w1[k], a[k], sR);
        sI = fma(w2[k], a[k], sI);
    }
    double mr0, mi0;
    block_exclusive_scans<NT>(sR, sI, mr0, mi0, wt);
    if (off) {  // the sums of the slabs below (regular) and above (irregular) this one
        mr0 += off[q];
        mi0 += off[KL + q];
    }
    double er[CH + 1], ei[CH + 1];
    er[0] = mr0;
#pragma unroll
    for (int k = 0; k < CH; ++k) er[k + 1] = fma(w1[k], a[k], er[k]);
    ei[CH] = mi0;
#pragma unroll
    for (int k = CH - 1; k >= 0; --k) ei[k] = fma(w2[k], a[k], ei[k + 1]);
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        const int i = i0 + k;
        if (i < n_r) {
            MR[(size_t)i * KL + q] = er[k];
            MI[(size_t)i * KL + q] = ei[k];
            double c = fma(g2[k], er[k] + er[k + 1], g1[k] * (ei[k] + ei[k + 1]));
            if (m > 0) c += c;
            if (C) C[(size_t)i * KL + q] = c;
            const float c32 = f64_to_f32_alu(c);
            if (C32) C32[(size_t)i * KL + q] = c32;
            if (C0 && p == 0) C0[(size_t)i * Lp1 + l] = f32_pair(c);
            if (cbo.cb && p > 0) write_cb(cbo, i, l, p, c32);
        }
    }
    if (threadIdx.x == NT - 1) {
        // the last thread's chunk ends at or beyond the last shell: its final values are the totals
        MR[(size_t)n_r * KL + q] = er[CH];
        MI[(size_t)n_r * KL + q] = ei[CH];
    }
}

// The same recurrences for four adjacent moment columns per block (used when there are
// many columns): thread t owns column q0 + (t & 3) and shells [c CH, (c + 1) CH) with
// c = t >> 2, so the four columns of a shell row sit in one 32-byte sector of A, MR, MI
// and C (one column per block reads a quarter of every sector it touches).  The block
// scans run over the lanes of one column (stride 4 within a warp), then over the warps.
// (two blocks per SM: the kernel is latency-bound, and the second block hides more of it
// than the registers the cap takes away; at 2048 shells, CH = 16, with a few spills to
// local memory: 226 -> 207 us against one block of 124 registers per SM)
template <int NT, int CH>
__global__ void __launch_bounds__(4 * NT, 2) k_scan_q4(const double *__restrict__ A, const double *__restrict__ WR,
                                                    const double *__restrict__ WI, const double *__restrict__ GR,
                                                    const double *__restrict__ GI, double *__restrict__ MR,
                                                    double *__restrict__ MI, double *__restrict__ C,
                                                    float *__restrict__ C32, float2 *__restrict__ C0, int n_r, int KL,
                                                    const CbOut cbo, const double *__restrict__ off)
{
    constexpr int NW = 4 * NT / 32;
    __shared__ double wt[2][NW][4];
    pdl_trigger();
    pdl_wait();  // A comes from the previous kernel
    const int sub = threadIdx.x & 3, c = threadIdx.x >> 2, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = 4 * blockIdx.x + sub;
    const bool valid = q < KL;
    int l = (int)sqrtf((float)(valid ? q : 0));
    const int qq = valid ? q : 0;
    while (l * l > qq) --l;
    while ((l + 1) * (l + 1) <= qq) ++l;
    const int p = qq - l * l;
    const int m = pcol_m(p);
    const int Lp1 = (int)sqrtf((float)KL + 0.5f);  // L + 1
    const int i0 = c * CH;
    const double *wr = WR + (size_t)l * n_r;
    const double *wi = WI + (size_t)l * n_r;
    const double *gr = GR + (size_t)l * n_r;
    const double *gi = GI + (size_t)l * n_r;
    // registers hold the column's values and its inward edge moments; the small weight
    // tables are read again where needed (cache hits), which keeps 512 threads resident
    double a[CH];
    double sR = 0.0, sI = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        const int i = i0 + k;
        const bool in = valid && i < n_r;
        a[k] = in ? A[(size_t)i * KL + q] : 0.0;
        if (in) {
            sR = fma(__ldg(wr + i), a[k], sR);
            sI = fma(__ldg(wi + i), a[k], sI);
        }
    }
    // inclusive scans over the 8 chunks of this column in the warp (lanes sub, sub + 4, ...)
    double inf = sR, inb = sI;
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        const double yf = __shfl_up_sync(kFull, inf, o);
        const double yb = __shfl_down_sync(kFull, inb, o);
        if (lane >= o) inf += yf;
        if (lane + o < 32) inb += yb;
    }
    double ef = __shfl_up_sync(kFull, inf, 4);
    double eb = __shfl_down_sync(kFull, inb, 4);
    if (lane < 4) ef = 0.0;
    if (lane >= 28) eb = 0.0;
    if (lane >= 28) wt[0][w][sub] = inf;
    if (lane < 4) wt[1][w][sub] = inb;
    __syncthreads();
    double of = 0.0, ob = 0.0;
    for (int w2_ = 0; w2_ < w; ++w2_) of += wt[0][w2_][sub];
    for (int w2_ = NW - 1; w2_ > w; --w2_) ob += wt[1][w2_][sub];
    if (!valid) return;
    if (off) {  // the sums of the slabs below (regular) and above (irregular) this one
        of += off[q];
        ob += off[KL + q];
    }
    double ei[CH + 1];
    ei[CH] = ob + eb;
#pragma unroll
    for (int k = CH - 1; k >= 0; --k) {
        const int i = i0 + k;
        ei[k] = (i < n_r) ? fma(__ldg(wi + i), a[k], ei[k + 1]) : ei[k + 1];
    }
    double er = of + ef;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        const int i = i0 + k;
        if (i < n_r) {
            const double er1 = fma(__ldg(wr + i), a[k], er);
            MR[(size_t)i * KL + q] = er;
            MI[(size_t)i * KL + q] = ei[k];
            double cv = fma(__ldg(gi + i), er + er1, __ldg(gr + i) * (ei[k] + ei[k + 1]));
            if (m > 0) cv += cv;
            if (C) C[(size_t)i * KL + q] = cv;
            const float c32 = f64_to_f32_alu(cv);
            if (C32) C32[(size_t)i * KL + q] = c32;
            if (C0 && p == 0) C0[(size_t)i * Lp1 + l] = f32_pair(cv);
            if (cbo.cb && p > 0) write_cb(cbo, i, l, p, c32);
            er = er1;
        }
    }
    if (c == NT - 1) {
        // the last chunk ends at or beyond the last shell: its final values are the totals
        MR[(size_t)n_r * KL + q] = er;
        MI[(size_t)n_r * KL + q] = ei[CH];
    }
}

// Split path, theta part of step (a):
//   A[i][q] = 4 pi G sum_j Ith[t(l,m)][j] F[i][p][j],   q = l^2 + p, m = m(p)
// F holds each shell as P rows of polar cells ([n_r][P][ldF]; ldF = n_t rounded
// up to a multiple of four, plus four; padding is zero, as in the table Ith32
// [T][ldF]).
//
// Persistent blocks (one per SM) keep the table in shared memory (one bulk
// copy) and take one shell per pass, double-buffered: the next shell's rows
// arrive by bulk copy while the block works on the current one.  Work item
// (m, l0) covers order m, degrees l0 and l0 + 1, cos and sin: per four polar
// cells two table float4s and two F float4s feed sixteen multiply-adds.  The
// polar cells of an item are dealt round-robin (in float4 units) to JS = 2^jsh
// adjacent lanes; with ldF / 4 odd and JS = 8 the eight lanes of a
// shared-memory phase read eight different banks.  Terms are summed in float32
// over blocks of eight cells, block sums with Kahan compensation, and the lane
// partials are added by shuffles.  Every wait is bounded; after a failed wait
// the block drains its own copies (bounded) and returns.
__device__ __forceinline__ float dot4(float4 a, float4 b, float acc)
{
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Items (m, l0 = m, m + 2, ...) of order m come in ceil((L + 1 - m) / 2).
__device__ __forceinline__ short2 theta_item(int k, int L)
{
    int m = 0;
    for (;; ++m) {
        const int np = (L + 2 - m) / 2;
        if (k < np) break;
        k -= np;
    }
    return make_short2((short)m, (short)(m + 2 * k));
}

__global__ void __launch_bounds__(1024, 1) k32_theta_pipe(const float *__restrict__ F, const float *__restrict__ Ith,
                                                          double *__restrict__ A, int *err, int n_r, int n_t, int L,
                                                          int KL, int P, int ldF, int n_items, int jsh,
                                                          uint32_t tab_bytes, double scale)
{
    extern __shared__ __align__(16) uint8_t smem_tp[];
    const size_t shell_floats = (size_t)P * ldF;
    const uint32_t shell_bytes = (uint32_t)(shell_floats * 4);
    float *sT = reinterpret_cast<float *>(smem_tp);                                  // [T][ldF]
    float *sF = reinterpret_cast<float *>(smem_tp + tab_bytes);                      // [2][P][ldF]
    short2 *sItem = reinterpret_cast<short2 *>(sF + 2 * shell_floats);               // [n_items]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sItem + ((n_items + 1) & ~1));     // table, rows[2]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 3);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    const int JS = 1 << jsh;
    if (tid == 0) {
        for (int b = 0; b < 3; ++b) mbar_init(smem_u32(&bars[b]), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int it = tid; it < n_items; it += nthr) sItem[it] = theta_item(it, L);
    __syncthreads();
    int issued[2] = {0, 0};  // bulk copies issued per row buffer (thread 0)
    auto issue = [&](int i, int buf) {
        mbar_arrive_expect_tx(smem_u32(&bars[1 + buf]), shell_bytes);
        bulk_load(smem_u32(sF + (size_t)buf * shell_floats), F + (size_t)i * shell_floats, shell_bytes,
                  smem_u32(&bars[1 + buf]));
        ++issued[buf];
    };
    if (tid == 0) {
        mbar_arrive_expect_tx(smem_u32(&bars[0]), tab_bytes);
        bulk_load(smem_u32(sT), Ith, tab_bytes, smem_u32(&bars[0]));
    }
    // the table copy overlaps the previous kernel's tail; F rows only after it completed
    pdl_trigger();
    pdl_wait();
    if (tid == 0)
        for (int b = 0; b < 2; ++b)
            if ((int)blockIdx.x + b * (int)gridDim.x < n_r) issue(blockIdx.x + b * gridDim.x, b);
    const bool table_ok = mbar_wait(smem_u32(&bars[0]), 0, abort_flag, err);
    bool ok = table_ok;
    int consumed[2] = {0, 0};
    const int nq = (n_t + 3) / 4;  // float4 units of polar cells per row
    const int n_work = n_items << jsh;

    // one item's lane partial for shell buffer fb, summed over the JS lanes, written by lane js = 0
    auto item = [&](const float *fb, double *Ai, int w) {
        const int js = w & (JS - 1);
        const bool act = w < n_work;
        float part[4] = {0.f, 0.f, 0.f, 0.f};
        int m = 0, l0 = 0;
        if (act) {
            const short2 itm = sItem[w >> jsh];
            m = itm.x;
            l0 = itm.y;
            const int pc = (m == 0) ? 0 : 2 * m - 1, ps = (m == 0) ? 0 : 2 * m;
            const float4 *fc = reinterpret_cast<const float4 *>(fb + (size_t)pc * ldF);
            const float4 *fs = reinterpret_cast<const float4 *>(fb + (size_t)ps * ldF);
            const float4 *t0 = reinterpret_cast<const float4 *>(sT + (size_t)tri(l0, m) * ldF);
            const float4 *t1 = reinterpret_cast<const float4 *>(sT + (size_t)tri(min(l0 + 1, L), m) * ldF);
            float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
            for (int u = js; u < nq; u += 2 * JS) {
                const float4 x0 = fc[u], y0 = fs[u], a0 = t0[u], b0 = t1[u];
                float blk[4];
                blk[0] = dot4(a0, x0, 0.f);
                blk[1] = dot4(a0, y0, 0.f);
                blk[2] = dot4(b0, x0, 0.f);
                blk[3] = dot4(b0, y0, 0.f);
                if (u + JS < nq) {
                    const float4 x1 = fc[u + JS], y1 = fs[u + JS], a1 = t0[u + JS], b1 = t1[u + JS];
                    blk[0] = dot4(a1, x1, blk[0]);
                    blk[1] = dot4(a1, y1, blk[1]);
                    blk[2] = dot4(b1, x1, blk[2]);
                    blk[3] = dot4(b1, y1, blk[3]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) kahan_add(s[e], c[e], blk[e]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) part[e] = s[e] - c[e];
        }
        for (int o = 1; o < JS; o <<= 1)
#pragma unroll
            for (int e = 0; e < 4; ++e) part[e] += __shfl_xor_sync(0xFFFFFFFFu, part[e], o);
        // every lane holds the four sums; lane js writes outputs js, js + JS, ... (one float64
        // scaling per output, not per lane)
        if (act) {
            const int pc = (m == 0) ? 0 : 2 * m - 1;
            for (int e = js; e < 4; e += JS) {
                const int l = l0 + (e >> 1), sn = e & 1;
                if (l > L || (sn && m == 0)) continue;
                const float v = (e == 0) ? part[0] : (e == 1) ? part[1] : (e == 2) ? part[2] : part[3];
                Ai[l * l + pc + sn] = scale * f32_to_f64_alu(v);
            }
        }
    };

    int k = 0;
    for (int i = blockIdx.x; i < n_r; i += gridDim.x, ++k) {
        const int b = k & 1;
        if (ok) ok = mbar_wait(smem_u32(&bars[1 + b]), (uint32_t)(k >> 1) & 1u, abort_flag, err);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        ++consumed[b];
        const float *fb = sF + (size_t)b * shell_floats;
        // whole warps run the loop together (the lane partials meet by shuffles)
        for (int wb = tid - lane; wb < n_work; wb += nthr) item(fb, A + (size_t)i * KL, wb + lane);
        // buffer b consumed: its plain reads are ordered before the bulk copy (async proxy) that
        // refills it
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && i + 2 * (int)gridDim.x < n_r) issue(i + 2 * gridDim.x, b);
    }
    if (!ok && tid == 0) {
        // drain this block's copies still in flight (bounded waits)
        const long long t0 = clock64();
        if (!table_ok)
            while (!mbar_try_wait(smem_u32(&bars[0]), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
            }
        for (int b = 0; b < 2; ++b) {
            if (issued[b] > consumed[b]) {
                const uint32_t par = (uint32_t)(issued[b] - 1) & 1u;
                const long long t1 = clock64();
                while (!mbar_try_wait(smem_u32(&bars[1 + b]), par) && clock64() - t1 < MP_WAIT_BUDGET_CYCLES) {
                }
            }
        }
    }
}

// Same sums for tables and shells that exceed shared memory, as one GEMM per order m:
//   Out_m[l][col] = sum_j Ith[tri(l,m)][j] F[i(col)][p(col)][j],  l = m..L,
//   col = (shell i, cos | sin).
// Block (tile of kMgShells shells, m) computes a 64 x 64 tile (degrees x columns; more
// degree tiles in turn when L + 1 - m > 64) in K chunks of kMgK polar cells: the
// chunk's table rows and F rows pass through shared memory (coalesced float4 loads);
// thread (rg, cg) owns degrees rg + 16 a and columns cg + 16 b (a, b < 4), so the eight
// lanes of a shared-memory phase read eight different banks.  Products are summed in
// float32 over blocks of eight cells, block sums with Kahan compensation.
constexpr int kMgShells = 32, kMgCols = 2 * kMgShells, kMgRows = 64, kMgK = 32, kMgLd = kMgK + 4;

// One pass of degree tile [l0, l0 + 16 RT) of order m: thread (rg, cg) owns degrees
// rg + 16 a (a < RT) and columns cg + 16 b (b < 4).  The tile has only as many rows as
// the order has degrees left (rounded up to 16): an order m has L + 1 - m degrees, so a
// fixed 64-row tile would mostly multiply zeros at high m.
template <int RT>
__device__ __forceinline__ void theta_mg_pass(float (*sT)[kMgLd], float (*sF)[kMgLd], const float *__restrict__ F,
                                              const float *__restrict__ Ith, double *__restrict__ A, int n_r, int n_t,
                                              int KL, int P, int ldF, double scale, int m, int i0, int nl, int pc,
                                              int l0)
{
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    float s[RT][4], c[RT][4];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) s[a][b] = c[a][b] = 0.0f;
    // the next chunk's global loads go out before the current chunk's arithmetic (registers
    // hold them in between): a 256-thread block moves at most 2 + 2 float4 per thread
    constexpr int kT = (16 * RT * (kMgK / 4) + 255) / 256, kF = kMgCols * (kMgK / 4) / 256;
    float4 pt[kT], pf[kF];
    auto load_chunk = [&](int j0) {
#pragma unroll
        for (int n = 0; n < kT; ++n) {
            const int e = tid + 256 * n, r = e >> 3, q = e & 7, j = j0 + 4 * q;
            pt[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < 16 * RT * (kMgK / 4) && l0 + r < nl && j < ldF)
                pt[n] = __ldg(reinterpret_cast<const float4 *>(Ith + (size_t)tri(m + l0 + r, m) * ldF + j));
        }
#pragma unroll
        for (int n = 0; n < kF; ++n) {
            const int e = tid + 256 * n, col = e >> 3, q = e & 7, j = j0 + 4 * q;
            const int i = i0 + (col >> 1), sn = col & 1;
            pf[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n_r && j < ldF && (sn == 0 || m > 0))
                pf[n] = __ldg(reinterpret_cast<const float4 *>(F + ((size_t)i * P + pc + sn) * ldF + j));
        }
    };
    load_chunk(0);
    for (int j0 = 0; j0 < n_t; j0 += kMgK) {
        __syncthreads();  // the previous chunk is consumed
#pragma unroll
        for (int n = 0; n < kT; ++n) {
            const int e = tid + 256 * n;
            if (e < 16 * RT * (kMgK / 4)) *reinterpret_cast<float4 *>(&sT[e >> 3][4 * (e & 7)]) = pt[n];
        }
#pragma unroll
        for (int n = 0; n < kF; ++n) {
            const int e = tid + 256 * n;
            *reinterpret_cast<float4 *>(&sF[e >> 3][4 * (e & 7)]) = pf[n];
        }
        __syncthreads();
        if (j0 + kMgK < n_t) load_chunk(j0 + kMgK);
#pragma unroll
        for (int jb = 0; jb < kMgK; jb += 8) {
            float blk[RT][4];
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) blk[a][b] = 0.0f;
#pragma unroll
            for (int jj = jb; jj < jb + 8; jj += 4) {
                float4 t[RT], f[4];
#pragma unroll
                for (int a = 0; a < RT; ++a) t[a] = *reinterpret_cast<const float4 *>(&sT[rg + 16 * a][jj]);
#pragma unroll
                for (int b = 0; b < 4; ++b) f[b] = *reinterpret_cast<const float4 *>(&sF[cg + 16 * b][jj]);
#pragma unroll
                for (int a = 0; a < RT; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) blk[a][b] = dot4(t[a], f[b], blk[a][b]);
            }
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) kahan_add(s[a][b], c[a][b], blk[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < RT; ++a) {
        const int lr = l0 + rg + 16 * a;
        if (lr >= nl) continue;
        const int l = m + lr;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int col = cg + 16 * b, i = i0 + (col >> 1), sn = col & 1;
            if (i < n_r && (sn == 0 || m > 0))
                A[(size_t)i * KL + l * l + pc + sn] = scale * f32_to_f64_alu(s[a][b] - c[a][b]);
        }
    }
}

__global__ void __launch_bounds__(256) k32_theta_mgemm(const float *__restrict__ F, const float *__restrict__ Ith,
                                                       double *__restrict__ A, int n_r, int n_t, int L, int KL, int P,
                                                       int ldF, double scale)
{
    __shared__ __align__(16) float sT[kMgRows][kMgLd];
    __shared__ __align__(16) float sF[kMgCols][kMgLd];
    pdl_wait();  // F comes from the previous kernel
    const int m = blockIdx.y, i0 = blockIdx.x * kMgShells;
    const int nl = L + 1 - m;
    const int pc = (m == 0) ? 0 : 2 * m - 1;
    for (int l0 = 0; l0 < nl; l0 += kMgRows) {
        switch (min(4, (nl - l0 + 15) / 16)) {
        case 1: theta_mg_pass<1>(sT, sF, F, Ith, A, n_r, n_t, KL, P, ldF, scale, m, i0, nl, pc, l0); break;
        case 2: theta_mg_pass<2>(sT, sF, F, Ith, A, n_r, n_t, KL, P, ldF, scale, m, i0, nl, pc, l0); break;
        case 3: theta_mg_pass<3>(sT, sF, F, Ith, A, n_r, n_t, KL, P, ldF, scale, m, i0, nl, pc, l0); break;
        default: theta_mg_pass<4>(sT, sF, F, Ith, A, n_r, n_t, KL, P, ldF, scale, m, i0, nl, pc, l0); break;
        }
    }
}

}  // namespace

// The coefficients the synthesis that follows reads: float64 C on the float64 path; on the
// split path the float32 copy for the CUDA-core theta synthesis, the bf16 terms (cb_out) for
// the tensor-core one, and the m = 0 (hi, lo) pairs for both.
static double *scan_c(const mp_mesh *m, int want_f32) { return want_f32 ? nullptr : m->d_C; }
static float *scan_c32(const mp_mesh *m, int want_f32)
{
    return (want_f32 && !m->plan.use_theta_tc) ? m->d_C32 : nullptr;
}

// The coefficient terms of the tensor-core theta synthesis, when the split path uses it.
static CbOut cb_out(const mp_mesh *m, int want_f32)
{
    CbOut o;
    if (want_f32 && m->plan.use_theta_tc) {
        o.cb = m->d_Cb;
        o.off = m->d_cb_off;
        o.NS = m->plan.gs_NS;
        o.terms = m->plan.a_terms;
        o.L = m->L;
    }
    return o;
}

template <int NT, int CH>
static void scan_reg_launch(mp_mesh *m, int want_f32)
{
    launch_pdl(k_scan_reg<NT, CH>, dim3(m->KL), dim3(NT), 0, m->stream, m->d_A, m->d_WR, m->d_WI, m->d_GR, m->d_GI,
               m->d_MR, m->d_MI, scan_c(m, want_f32), scan_c32(m, want_f32), want_f32 ? m->d_C0 : nullptr, m->n_r,
               m->KL, cb_out(m, want_f32), m->use_slab_off ? (const double *)m->d_slab_off : nullptr);
}

// Shells per thread CH for NT threads per moment column; false when n_r > 16 NT.
template <int NT>
static bool scan_reg_dispatch(mp_mesh *m, int want_f32)
{
    const int ch = (m->n_r + NT - 1) / NT;
    if (ch <= 1)
        scan_reg_launch<NT, 1>(m, want_f32);
    else if (ch <= 2)
        scan_reg_launch<NT, 2>(m, want_f32);
    else if (ch <= 4)
        scan_reg_launch<NT, 4>(m, want_f32);
    else if (ch <= 8)
        scan_reg_launch<NT, 8>(m, want_f32);
    else if (ch <= 16)
        scan_reg_launch<NT, 16>(m, want_f32);
    else
        return false;
    return true;
}

// Shared memory of the persistent theta contraction (table, two shell buffers, item
// list, barriers); above 200 KB the per-order GEMM form runs instead.
static size_t theta_pipe_smem(const mp_mesh *m, int *n_items_out = nullptr, int *jsh_out = nullptr)
{
    const int ldF = m->plan.ldF, L = m->L, P = m->P;
    const size_t tab_bytes = (size_t)m->T * ldF * 4;
    int n_items = 0;
    for (int mm = 0; mm <= L; ++mm) n_items += (L + 2 - mm) / 2;
    // lanes per item: eight when a row has enough float4 units to go round
    const int nq = (m->n_t + 3) / 4;
    const int jsh = nq >= 16 ? 3 : (nq >= 8 ? 2 : (nq >= 4 ? 1 : 0));
    if (n_items_out) *n_items_out = n_items;
    if (jsh_out) *jsh_out = jsh;
    return tab_bytes + 2 * (size_t)P * ldF * 4 + (size_t)((n_items + 1) & ~1) * 4 + 3 * 8 + 16;
}

bool theta_pipe_fits(const mp_mesh *m) { return theta_pipe_smem(m) <= 200 * 1024; }

// Four columns per block when there are at least four such blocks per SM; 128 chunk
// threads per column (512 per block), CH shells each.  Not beside the persistent theta
// contraction of the split path: its blocks leave room for the small one-column scan
// blocks to start early, not for these (that early start is worth more than coalescing).
static bool scan_q4_dispatch(mp_mesh *m, int want_f32)
{
    if (m->KL < 4 * m->num_sms) return false;
    if (want_f32 && theta_pipe_smem(m) <= 200 * 1024) return false;
    const int ch = (m->n_r + 127) / 128;
    auto go = [&](auto kern) {
        launch_pdl(kern, dim3((m->KL + 3) / 4), dim3(512), 0, m->stream, m->d_A, m->d_WR, m->d_WI, m->d_GR, m->d_GI,
                   m->d_MR, m->d_MI, scan_c(m, want_f32), scan_c32(m, want_f32), want_f32 ? m->d_C0 : nullptr,
                   m->n_r, m->KL, cb_out(m, want_f32), m->use_slab_off ? (const double *)m->d_slab_off : nullptr);
    };
    if (ch <= 4)
        go(k_scan_q4<128, 4>);
    else if (ch <= 8)
        go(k_scan_q4<128, 8>);
    else if (ch <= 16)
        go(k_scan_q4<128, 16>);
    else
        return false;
    return true;
}

cudaError_t launch_scan(mp_mesh *m, int want_f32)
{
    cudaEvent_t ev;
    prof_begin(m, "radial_scan", &ev);
    bool done = scan_q4_dispatch(m, want_f32);
    if (!done) switch (m->plan.scan_threads) {
    case 64: done = scan_reg_dispatch<64>(m, want_f32); break;
    case 256: done = scan_reg_dispatch<256>(m, want_f32); break;
    default: done = scan_reg_dispatch<kScanThreads>(m, want_f32); break;
    }
    if (!done)
        k_scan<kScanThreads><<<m->KL, kScanThreads, 0, m->stream>>>(m->d_A, m->d_WR, m->d_WI, m->d_GR, m->d_GI,
                                                                    m->d_MR, m->d_MI, scan_c(m, want_f32),
                                                                    scan_c32(m, want_f32),
                                                                    want_f32 ? m->d_C0 : nullptr, m->n_r, m->KL,
                                                                    cb_out(m, want_f32),
                                                                    m->use_slab_off ? (const double *)m->d_slab_off : nullptr);
    prof_end(m, "radial_scan", ev);
    return cudaGetLastError();
}


// The theta contraction of the orders 0 .. orders_hi on CUDA cores (all of them when the
// tensor-core kernel does not apply).
static cudaError_t theta_cuda_cores(mp_mesh *m, int orders_hi)
{
    constexpr double kFourPi = 12.566370614359172954;
    const int ldF = m->plan.ldF, L = m->L, P = m->P;
    const uint32_t tab_bytes = (uint32_t)((size_t)m->T * ldF * 4);
    int n_items = 0, jsh = 0;
    const size_t smem = theta_pipe_smem(m, &n_items, &jsh);
    if (orders_hi == 0) n_items = (L + 2) / 2;  // the items of m = 0 come first
    if (smem <= 200 * 1024) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k32_theta_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set = true;
        }
        const int threads = std::min(1024, 32 * (((n_items << jsh) + 31) / 32));
        const int grid = std::min(m->n_r, m->num_sms);
        launch_pdl(k32_theta_pipe, dim3(grid), dim3(threads), smem, m->stream, m->d_F32, m->d_Ith32, m->d_A, m->d_err,
                   m->n_r, m->n_t, L, m->KL, P, ldF, n_items, jsh, tab_bytes, kFourPi * m->G);
    } else {
        const dim3 grid((m->n_r + kMgShells - 1) / kMgShells, orders_hi + 1);
        launch_pdl(k32_theta_mgemm, grid, dim3(256), 0, m->stream, m->d_F32, m->d_Ith32, m->d_A, m->n_r, m->n_t, L,
                   m->KL, P, ldF, kFourPi * m->G);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_theta(mp_mesh *m)
{
    cudaEvent_t ev;
    if (m->plan.use_theta_tc) return launch_theta_tc(m);  // profiles its two kernels itself
    prof_begin(m, "split_theta_contract", &ev);
    cudaError_t e = theta_cuda_cores(m, m->L);
    prof_end(m, "split_theta_contract", ev);
    return e;
}

}  // namespace mp
