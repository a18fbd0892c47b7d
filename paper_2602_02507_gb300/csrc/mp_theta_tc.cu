// mp_theta_tc.cu -- the theta factors of both angular contractions of GenASiS II
// Sec. 2.2 as split-precision tcgen05 GEMMs, one per azimuthal order m >= 1.
//
//   (a2) theta contraction, Eq. (AngularMomentsDiscrete), theta part:
//          A[i][l^2 + p] = 4 pi G sum_j Ith[t(l,m)][j] F[i][p][j],   p = 2m - 1 + a
//        per order m, for 64 shells at a time:
//          D[(a, shell)][l - m] = sum_j F[i][p][j] Ith[t(l,m)][j]
//        M = 128 rows (64 shells x cos, sin), N = the L + 1 - m degrees rounded up to
//        16, K = polar cells in chunks of 32.  F (float32, written by the phi
//        projection) arrives by 3-D TMA and is split into bf16 terms by converter
//        warps; the table is pre-split.
//   (d1) theta synthesis, Eq. (Solution), theta part:
//          G[i, j][p] = sum_{l >= m} (Ith[t(l,m)][j] / dmu_j) C[i][l^2 + p]
//        per order m, for 128 polar cells and NS shells at a time:
//          D[j][(shell, a)] = sum_l Itc[t(l,m)][j] C[i][l^2 + p]
//        M = 128 polar cells, N = 2 NS, K = degrees in chunks of 32.  Both operands
//        arrive by bulk copy: the table pre-split, the coefficients as the bf16 terms
//        the radial recurrences write (mp_radial.cu).  Four consecutive orders share a
//        unit, so that the epilogue writes whole 16-byte rows (8 K columns) of the phi
//        synthesis A operand.
//
// The m = 0 column of both stages, the bulk of Phi, stays on CUDA cores in small kernels
// of their own launched just before the tensor-core kernels: compensated float32 sums for
// the contraction (a warp per shell), double-float for the synthesis (a thread per row).
// The tensor core accumulates in float32 with truncation, which the monopole cannot afford.
//
// Roles per CTA of the tensor-core kernels (persistent, one CTA per SM): warp 0 issues the
// copies, warp 1 owns tensor memory and issues the MMAs, converter / epilogue warps feed
// and drain it.  Every mbarrier wait is bounded (ptx.cuh).
#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

// bf16 products accumulated per K step: (dynamic-operand term, table term)
__constant__ int c_pa[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_pb[6] = {0, 1, 0, 2, 1, 0};

__host__ __device__ inline int round16(int x) { return (x + 15) / 16 * 16; }

// ---------------------------------------------------------------------------- (a2)
namespace thc {
constexpr int BK = 32;                      // polar cells per K chunk
constexpr int SHELLS = 64;                  // shells per unit (M = 128: cos rows, then sin rows)
constexpr int BOX_BYTES = SHELLS * BK * 4;  // one [64 x 32] float32 TMA box, 128B-swizzled rows
constexpr int F_BYTES = 2 * BOX_BYTES;
constexpr int A_TERM_BYTES = 128 * BK * 2;  // [128 x 32] bf16
constexpr int SBO = (BK / 8) * 128;         // 8-row group stride of [rows x 32] K-major chunks
constexpr int GROUP_WARPS = 8;
constexpr int CONV_WARPS = 2 * GROUP_WARPS;
constexpr int THREADS = (2 + CONV_WARPS) * 32;
}  // namespace thc

struct ThetaTcParams {
    const uint8_t *tab;              // order m >= 1: [n_kc][3 terms][Nm x 32] bf16, canonical K-major
    const unsigned long long *off;   // [L + 1] byte offset of order m's table
    const float *F;                  // [n_r][P][ldF] (the m = 0 kernel reads row p = 0 of each shell)
    const float *Ith32;              // [T][ldF]
    double *A;                       // [n_r][K_L]
    int *err;
    int n_r, n_t, L, KL, P, ldF, n_kc, n_groups, n_units, ns_s, ns_o, nacc, Nmax, bterms;
    uint32_t stage_bytes;            // F boxes + the largest table chunk (the terms the products read)
    double scale;                    // 4 pi G
};

template <int A_TERMS, int NPROD>
__global__ void __launch_bounds__(thc::THREADS, 1) k_theta_tc(const __grid_constant__ CUtensorMap tmF,
                                                              const ThetaTcParams prm)
{
    using namespace thc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS_S = prm.ns_s, NS_O = prm.ns_o;
    uint8_t *sS = smem;                                           // [NS_S][stage]: cos box, sin box, table
    uint8_t *sA = sS + (size_t)NS_S * prm.stage_bytes;            // [NS_O][A_TERMS][128 x 32] bf16
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + (size_t)NS_O * A_TERMS * A_TERM_BYTES);
    uint64_t *s_full = bars, *s_empty = bars + NS_S;
    uint64_t *o_full = bars + 2 * NS_S, *o_empty = o_full + NS_O;
    uint64_t *acc_full = o_empty + NS_O, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nacc = prm.nacc, Nmax = prm.Nmax;
    const uint32_t ncols = tmem_ncols_for(2 * nacc * Nmax);
    const uint32_t acc_stride = ncols / 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS_S; ++s) {
            mbar_init(smem_u32(&s_full[s]), 1);
            // a stage is free once its group's converters read the density and the MMAs read the table
            mbar_init(smem_u32(&s_empty[s]), GROUP_WARPS + 1);
        }
        for (int o = 0; o < NS_O; ++o) {
            mbar_init(smem_u32(&o_full[o]), GROUP_WARPS);
            mbar_init(smem_u32(&o_empty[o]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), CONV_WARPS);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_holder), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    pdl_trigger();
    pdl_wait();  // F comes from the previous kernels

    if (warp == 0) {
        // ---------------- producer: the cos and sin boxes of F and the table chunk of each stage
        if (lane == 0) {
            tma_prefetch_desc(&tmF);
            Ring rs;
            int issued = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < prm.n_units && ok; u += gridDim.x) {
                const int m = 1 + u / prm.n_groups, g = u - (m - 1) * prm.n_groups;
                const int Nm = round16(prm.L + 1 - m);
                const uint32_t tb = (uint32_t)(prm.bterms * Nm * 64);
                const uint8_t *tsrc = prm.tab + prm.off[m];
                for (int c = 0; c < prm.n_kc; ++c, rs.next(NS_S)) {
                    ok = mbar_wait(smem_u32(&s_empty[rs.idx]), rs.phase ^ 1, abort_flag, prm.err);
                    if (!ok) break;
                    const uint32_t fb = smem_u32(&s_full[rs.idx]);
                    const uint32_t dst = smem_u32(sS + (size_t)rs.idx * prm.stage_bytes);
                    mbar_arrive_expect_tx(fb, F_BYTES + tb);
                    tma_load_3d(dst, &tmF, fb, c * BK, 2 * m - 1, g * SHELLS);
                    tma_load_3d(dst + BOX_BYTES, &tmF, fb, c * BK, 2 * m, g * SHELLS);
                    bulk_load(dst + F_BYTES, tsrc + (size_t)c * 3 * Nm * 64, tb, fb);
                    ++issued;
                }
            }
            drain_ring(s_full, rs, NS_S, issued);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            Ring rs, ro;
            int lt = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < prm.n_units && ok; u += gridDim.x, ++lt) {
                const int m = 1 + u / prm.n_groups;
                const int Nm = round16(prm.L + 1 - m);
                const uint32_t idesc = idesc_bf16_f32(128, Nm);
                const uint32_t b_term = (uint32_t)Nm * 64;
                const int b = lt & 1;
                ok = mbar_wait(smem_u32(&acc_empty[b]), ((lt >> 1) & 1) ^ 1, abort_flag, prm.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_buf = tmem_base + (uint32_t)b * acc_stride;
                for (int c = 0; c < prm.n_kc; ++c, rs.next(NS_S), ro.next(NS_O)) {
                    ok = mbar_wait(smem_u32(&o_full[ro.idx]), ro.phase, abort_flag, prm.err) &&
                         mbar_wait(smem_u32(&s_full[rs.idx]), rs.phase, abort_flag, prm.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(sA + (size_t)ro.idx * A_TERMS * A_TERM_BYTES);
                    const uint32_t t_base = smem_u32(sS + (size_t)rs.idx * prm.stage_bytes + F_BYTES);
                    const uint32_t d_tmem = d_buf + (uint32_t)((c % nacc) * Nmax);
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
                        for (int pi = 0; pi < NPROD; ++pi) {
                            const uint64_t ad = sdesc_noswizzle(a_base + c_pa[pi] * A_TERM_BYTES + ks * 256, 128, SBO);
                            const uint64_t bd = sdesc_noswizzle(t_base + c_pb[pi] * b_term + ks * 256, 128, SBO);
                            umma_bf16(d_tmem, ad, bd, idesc, (c >= nacc) || ((ks | pi) != 0));
                        }
                    }
                    umma_commit(smem_u32(&o_empty[ro.idx]));
                    umma_commit(smem_u32(&s_empty[rs.idx]));
                }
                if (!ok) break;
                umma_commit(smem_u32(&acc_full[b]));
            }
            umma_commit(smem_u32(drain));
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(drain), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
            }
        }
    } else {
        // ---------------- converters (F -> bf16 terms) + epilogue (accumulators -> moments)
        const int cw = warp - 2, grp = cw / GROUP_WARPS, qd = warp & 3, half = (cw >> 2) & 1;
        // this thread converts F row (a = row >> 6, shell row & 63) of the boxes and writes it
        // to MMA row mrow = 2 shell + a, so that each shell's cos and sin accumulators sit in
        // adjacent lanes and the epilogue's stores of a warp pair up in 16-byte pieces
        const int row = qd * 32 + lane;
        const int mrow = 2 * (row & 63) + (row >> 6);
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        Ring rs, ro;
        if (grp) {
            rs.next(NS_S);
            ro.next(NS_O);
        }
        int par = 0, lt = 0, prev_u = -1;
        bool ok = true;

        auto epilogue = [&](int eu, int elt) -> bool {
            const int b = elt & 1;
            if (!warp_all(mbar_wait(smem_u32(&acc_full[b]), (elt >> 1) & 1, abort_flag, prm.err))) return false;
            tc_fence_after();
            const int m = 1 + eu / prm.n_groups, g = eu - (m - 1) * prm.n_groups;
            const int Nm = round16(prm.L + 1 - m);
            const int i = g * SHELLS + (row >> 1);  // accumulator lane row holds MMA row `row`
            const int p = 2 * m - 1 + (row & 1);
            double *Ai = prm.A + (size_t)i * prm.KL + p;
            for (int cg = 2 * grp + half; cg * 8 < Nm; cg += 4) {
                uint32_t v[4][8];
                const uint32_t col = tmem_base + lane_base + (uint32_t)b * acc_stride + (uint32_t)(cg * 8);
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (s < nacc) tmem_ld8(col + (uint32_t)(s * Nmax), v[s]);
                tmem_ld_wait();
                if (i < prm.n_r) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int l = m + cg * 8 + e;
                        float acc = __uint_as_float(v[0][e]);
#pragma unroll
                        for (int s = 1; s < 4; ++s)
                            if (s < nacc) acc += __uint_as_float(v[s][e]);
                        if (l <= prm.L) Ai[(size_t)l * l] = prm.scale * f32_to_f64_alu(acc);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
            return true;
        };

        for (int u = blockIdx.x; u < prm.n_units && ok; u += gridDim.x, ++lt) {
            for (int c = 0; c < prm.n_kc; ++c, par ^= 1) {
                if (par != grp) continue;
                const int sidx = rs.idx, oidx = ro.idx;
                const uint32_t sph = rs.phase, oph = ro.phase;
                rs.next(NS_S);
                rs.next(NS_S);
                ro.next(NS_O);
                ro.next(NS_O);
                ok = warp_all(mbar_wait(smem_u32(&s_full[sidx]), sph, abort_flag, prm.err));
                if (!ok) break;
                ok = warp_all(mbar_wait(smem_u32(&o_empty[oidx]), oph ^ 1, abort_flag, prm.err));
                if (!ok) break;
                // this thread's 16 polar cells [16 half, 16 half + 16) of its row, 128B-swizzled
                const uint8_t *src = sS + (size_t)sidx * prm.stage_bytes + (row >> 6) * BOX_BYTES + (row & 63) * 128;
                uint32_t w0[8], w1[8], w2[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int cc = 4 * half + q;
                    const float4 v = *reinterpret_cast<const float4 *>(src + ((cc ^ (row & 7)) << 4));
                    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float x0 = x[2 * h], x1 = x[2 * h + 1];
                        const uint32_t t0 = pack_bf16x2(x0, x1);
                        const float r0 = x0 - bf16lo_to_f32(t0), r1 = x1 - bf16hi_to_f32(t0);
                        const uint32_t t1 = pack_bf16x2(r0, r1);
                        w0[2 * q + h] = t0;
                        w1[2 * q + h] = t1;
                        if (A_TERMS == 3) w2[2 * q + h] = pack_bf16x2(r0 - bf16lo_to_f32(t1), r1 - bf16hi_to_f32(t1));
                    }
                }
                uint8_t *adst = sA + (size_t)oidx * A_TERMS * A_TERM_BYTES + (mrow >> 3) * SBO + half * 256 +
                                (mrow & 7) * 16;
#pragma unroll
                for (int kg = 0; kg < 2; ++kg) {
                    *reinterpret_cast<uint4 *>(adst + kg * 128) =
                        make_uint4(w0[4 * kg], w0[4 * kg + 1], w0[4 * kg + 2], w0[4 * kg + 3]);
                    *reinterpret_cast<uint4 *>(adst + A_TERM_BYTES + kg * 128) =
                        make_uint4(w1[4 * kg], w1[4 * kg + 1], w1[4 * kg + 2], w1[4 * kg + 3]);
                    if (A_TERMS == 3)
                        *reinterpret_cast<uint4 *>(adst + 2 * A_TERM_BYTES + kg * 128) =
                            make_uint4(w2[4 * kg], w2[4 * kg + 1], w2[4 * kg + 2], w2[4 * kg + 3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&s_empty[sidx]));
                    mbar_arrive(smem_u32(&o_full[oidx]));
                }
            }
            if (!ok) break;
            if (prev_u >= 0) ok = epilogue(prev_u, lt - 1);
            prev_u = u;
        }
        if (ok && prev_u >= 0) epilogue(prev_u, lt - 1);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, ncols);
    }
}

// ---------------------------------------------------------------------------- (d1)
namespace gsc {
constexpr int BK = 32;                        // degrees per K chunk
constexpr int T_TERM_BYTES = 128 * BK * 2;    // [128 polar cells x 32 degrees] bf16
constexpr int SBO = (BK / 8) * 128;
constexpr int EPI_WARPS = 8;                  // two per tensor-memory lane quarter
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int ORDERS = 4;                     // orders per unit: 8 K columns of the phi synthesis
}  // namespace gsc

struct GsynthTcParams {
    const uint8_t *tab;               // order m >= 1: [n_jb][n_kcm][3 terms][128 x 32] bf16, canonical K-major
    const unsigned long long *toff;   // [L + 1]
    const uint8_t *cb;                // order m >= 1: [n_sg][n_kcm][A_TERMS][2 NS x 32] bf16, canonical K-major
    const unsigned long long *coff;   // [L + 1]
    uint8_t *Aop;                     // [tiles][A_TERMS][128 x Kpad] bf16, canonical K-major (SBO = 16 Kpad)
    int *err;
    int n_r, n_t, L, Kpad, NS, n_jb, n_sg, n_units, ns_s, bterms;
    uint32_t stage_bytes;             // table terms read + coefficient terms of one K chunk
};

template <int A_TERMS, int NPROD>
__global__ void __launch_bounds__(gsc::THREADS, 1) k_gsynth_tc(const GsynthTcParams prm)
{
    using namespace gsc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int NS_S = prm.ns_s, NS = prm.NS, N = 2 * NS;
    const uint32_t tbytes = (uint32_t)(prm.bterms * T_TERM_BYTES), c_term = (uint32_t)(N * 64);
    uint8_t *sS = smem;                                              // [NS_S][stage]: table chunk, C chunk
    uint64_t *bars = reinterpret_cast<uint64_t *>(sS + (size_t)NS_S * prm.stage_bytes);
    uint64_t *s_full = bars, *s_empty = bars + NS_S;
    uint64_t *acc_full = bars + 2 * NS_S, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_ncols_for(2 * ORDERS * N);
    const uint32_t acc_stride = ncols / 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS_S; ++s) {
            mbar_init(smem_u32(&s_full[s]), 1);
            mbar_init(smem_u32(&s_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), EPI_WARPS);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_holder), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    pdl_trigger();
    pdl_wait();  // the coefficients come from the previous kernels

    if (warp == 0) {
        // ---------------- producer: table chunk and coefficient chunk of every (order, K chunk)
        if (lane == 0) {
            Ring rs;
            int issued = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < prm.n_units && ok; u += gridDim.x) {
                const int jb = u % prm.n_jb, rest = u / prm.n_jb;
                const int sg = rest % prm.n_sg, mg = rest / prm.n_sg;
                for (int ml = 0; ml < ORDERS && ok; ++ml) {
                    const int m = ORDERS * mg + 1 + ml;
                    if (m > prm.L) break;
                    const int n_kcm = (prm.L + 1 - m + BK - 1) / BK;
                    const uint8_t *tsrc = prm.tab + prm.toff[m] + (size_t)jb * n_kcm * 3 * T_TERM_BYTES;
                    const uint8_t *csrc = prm.cb + prm.coff[m] + (size_t)sg * n_kcm * A_TERMS * c_term;
                    for (int kc = 0; kc < n_kcm; ++kc, rs.next(NS_S)) {
                        ok = mbar_wait(smem_u32(&s_empty[rs.idx]), rs.phase ^ 1, abort_flag, prm.err);
                        if (!ok) break;
                        const uint32_t fb = smem_u32(&s_full[rs.idx]);
                        const uint32_t dst = smem_u32(sS + (size_t)rs.idx * prm.stage_bytes);
                        mbar_arrive_expect_tx(fb, tbytes + A_TERMS * c_term);
                        bulk_load(dst, tsrc + (size_t)kc * 3 * T_TERM_BYTES, tbytes, fb);
                        bulk_load(dst + tbytes, csrc + (size_t)kc * A_TERMS * c_term, A_TERMS * c_term, fb);
                        ++issued;
                    }
                }
            }
            drain_ring(s_full, rs, NS_S, issued);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, N);
            Ring rs;
            int lt = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < prm.n_units && ok; u += gridDim.x, ++lt) {
                const int mg = u / prm.n_jb / prm.n_sg;
                const int b = lt & 1;
                ok = mbar_wait(smem_u32(&acc_empty[b]), ((lt >> 1) & 1) ^ 1, abort_flag, prm.err);
                if (!ok) break;
                tc_fence_after();
                for (int ml = 0; ml < ORDERS && ok; ++ml) {
                    const int m = ORDERS * mg + 1 + ml;
                    if (m > prm.L) break;
                    const int n_kcm = (prm.L + 1 - m + BK - 1) / BK;
                    const uint32_t d_tmem = tmem_base + (uint32_t)b * acc_stride + (uint32_t)(ml * N);
                    for (int kc = 0; kc < n_kcm; ++kc, rs.next(NS_S)) {
                        ok = mbar_wait(smem_u32(&s_full[rs.idx]), rs.phase, abort_flag, prm.err);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t t_base = smem_u32(sS + (size_t)rs.idx * prm.stage_bytes);
                        const uint32_t c_base = t_base + tbytes;
#pragma unroll
                        for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
                            for (int pi = 0; pi < NPROD; ++pi) {
                                const uint64_t ad = sdesc_noswizzle(t_base + c_pb[pi] * T_TERM_BYTES + ks * 256, 128, SBO);
                                const uint64_t bd = sdesc_noswizzle(c_base + c_pa[pi] * c_term + ks * 256, 128, SBO);
                                umma_bf16(d_tmem, ad, bd, idesc, ((kc | ks | pi) != 0));
                            }
                        }
                        umma_commit(smem_u32(&s_empty[rs.idx]));
                    }
                }
                if (!ok) break;
                umma_commit(smem_u32(&acc_full[b]));
            }
            umma_commit(smem_u32(drain));
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(drain), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
            }
        }
    } else {
        // ---------------- epilogue: accumulators -> bf16 terms of the phi-synthesis A operand
        const int ew = warp - 2, qd = warp & 3, sh = ew >> 2;
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        const size_t a_term_bytes = (size_t)128 * prm.Kpad * 2;
        const int half_ns = NS / 2;
        int lt = 0;
        for (int u = blockIdx.x; u < prm.n_units; u += gridDim.x, ++lt) {
            const int jb = u % prm.n_jb, rest = u / prm.n_jb;
            const int sg = rest % prm.n_sg, mg = rest / prm.n_sg;
            const int b = lt & 1;
            if (!warp_all(mbar_wait(smem_u32(&acc_full[b]), (lt >> 1) & 1, abort_flag, prm.err))) break;
            tc_fence_after();
            const int j = jb * 128 + qd * 32 + lane;
            for (int sq = 0; sq < half_ns; sq += 4) {
                const int s0 = sh * half_ns + sq;  // four shells: accumulator columns 2 s + a
                uint32_t v[ORDERS][8];
#pragma unroll
                for (int ml = 0; ml < ORDERS; ++ml)
                    tmem_ld8(tmem_base + lane_base + (uint32_t)b * acc_stride + (uint32_t)(ml * N + 2 * s0), v[ml]);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = sg * NS + s0 + e;
                    if (i >= prm.n_r || j >= prm.n_t) continue;
                    float x[8];
#pragma unroll
                    for (int ml = 0; ml < ORDERS; ++ml) {
                        const bool live = ORDERS * mg + 1 + ml <= prm.L;  // orders past l_max: zero columns
                        x[2 * ml] = live ? __uint_as_float(v[ml][2 * e]) : 0.0f;
                        x[2 * ml + 1] = live ? __uint_as_float(v[ml][2 * e + 1]) : 0.0f;
                    }
                    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t t0 = pack_bf16x2(x[2 * c], x[2 * c + 1]);
                        const float r0 = x[2 * c] - bf16lo_to_f32(t0), r1 = x[2 * c + 1] - bf16hi_to_f32(t0);
                        const uint32_t t1 = pack_bf16x2(r0, r1);
                        w0[c] = t0;
                        w1[c] = t1;
                        if (A_TERMS == 3) w2[c] = pack_bf16x2(r0 - bf16lo_to_f32(t1), r1 - bf16hi_to_f32(t1));
                    }
                    const long long row = (long long)i * prm.n_t + j;
                    const int r = (int)(row & 127);
                    uint8_t *dst = prm.Aop + (size_t)(row >> 7) * A_TERMS * a_term_bytes +
                                   (size_t)(r >> 3) * (prm.Kpad * 16) + (size_t)mg * 128 + (r & 7) * 16;
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                    *reinterpret_cast<uint4 *>(dst + a_term_bytes) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                    if (A_TERMS == 3)
                        *reinterpret_cast<uint4 *>(dst + 2 * a_term_bytes) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, ncols);
    }
}

// ---------------------------------------------------------------------------- m = 0 columns
// (a2) m = 0 as a register-tiled float32 GEMM with compensated sums:
//   A[i][l^2] = scale sum_j Ith[t(l,0)][j] F[i][0][j]
// Block (64 degrees, 16 shells) stages K chunks of 32 polar cells of both operands in
// shared memory; thread (rg, cg) owns degrees rg + 16 a (a < 4) and shell cg; products are
// summed over blocks of eight cells, block sums with Kahan compensation.
constexpr int kM0Deg = 64, kM0Shells = 16, kM0K = 32, kM0Ld = kM0K + 4;

__device__ __forceinline__ float dot4f(float4 a, float4 b, float acc)
{
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}

__global__ void __launch_bounds__(256) k_theta_m0(const ThetaTcParams prm)
{
    __shared__ __align__(16) float sT[kM0Deg][kM0Ld];
    __shared__ __align__(16) float sF[kM0Shells][kM0Ld];
    // no early trigger: the tensor-core kernel that follows holds one CTA of shared memory
    // per SM, which would leave this kernel's later blocks no room
    pdl_wait();  // F comes from the previous kernel
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    const int i0 = blockIdx.x * kM0Shells, l0 = blockIdx.y * kM0Deg;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    // the next chunk's table and F values are loaded into registers while this chunk is
    // summed (two table float4s and, for the first 128 threads, one F float4 a thread)
    float4 tv[2], fv = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load = [&](int j0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = tid + 256 * k, r = e >> 3, q = e & 7, l = l0 + r, j = j0 + 4 * q;
            tv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l <= prm.L && j < prm.ldF)
                tv[k] = __ldg(reinterpret_cast<const float4 *>(prm.Ith32 + (size_t)tri(l, 0) * prm.ldF + j));
        }
        if (tid < kM0Shells * (kM0K / 4)) {
            const int r = tid >> 3, q = tid & 7, i = i0 + r, j = j0 + 4 * q;
            fv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < prm.n_r && j < prm.ldF) fv = __ldg(reinterpret_cast<const float4 *>(prm.F + (size_t)i * prm.P * prm.ldF + j));
        }
    };
    load(0);
    for (int j0 = 0; j0 < prm.n_t; j0 += kM0K) {
        __syncthreads();  // the previous chunk is consumed
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = tid + 256 * k;
            *reinterpret_cast<float4 *>(&sT[e >> 3][4 * (e & 7)]) = tv[k];
        }
        if (tid < kM0Shells * (kM0K / 4)) *reinterpret_cast<float4 *>(&sF[tid >> 3][4 * (tid & 7)]) = fv;
        __syncthreads();
        if (j0 + kM0K < prm.n_t) load(j0 + kM0K);
#pragma unroll
        for (int jb = 0; jb < kM0K; jb += 8) {
            const float4 f0 = *reinterpret_cast<const float4 *>(&sF[cg][jb]);
            const float4 f1 = *reinterpret_cast<const float4 *>(&sF[cg][jb + 4]);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 t0 = *reinterpret_cast<const float4 *>(&sT[rg + 16 * a][jb]);
                const float4 t1 = *reinterpret_cast<const float4 *>(&sT[rg + 16 * a][jb + 4]);
                const float blk = dot4f(t1, f1, dot4f(t0, f0, 0.f));
                const float y = blk - c[a];
                const float t = s[a] + y;
                c[a] = (t - s[a]) - y;
                s[a] = t;
            }
        }
    }
    const int i = i0 + cg;
    if (i >= prm.n_r) return;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int l = l0 + rg + 16 * a;
        if (l <= prm.L) prm.A[(size_t)i * prm.KL + (size_t)l * l] = prm.scale * f32_to_f64_alu(s[a] - c[a]);
    }
}

// (d1) m = 0 in double-float: G0[row] = (hi, lo) of sum_l (Ith[t(l,0)][j] / dmu_j) C[i][l^2]
// for the rows (i, j) of a block of 128 polar cells and SB shells; the block's table slice
// and coefficients sit in shared memory, thread (j, half) forms SB / 2 shells of cell j.
__global__ void __launch_bounds__(256) k_gsynth_m0(const float2 *__restrict__ C0, const float2 *__restrict__ Itc0,
                                                   float *__restrict__ G0, int n_r, int n_t, int L, int SB)
{
    extern __shared__ __align__(16) float2 sm0[];
    float2 *sT = sm0;                          // [L + 1][128]
    float2 *sC = sm0 + (size_t)(L + 1) * 128;  // [SB][L + 1]
    const int tid = threadIdx.x;
    const int j0 = blockIdx.x * 128, i0 = blockIdx.y * SB;
    for (int e = tid; e < (L + 1) * 128; e += 256) {  // the static table, ahead of the wait
        const int l = e >> 7, j = j0 + (e & 127);
        sT[e] = j < n_t ? Itc0[(size_t)l * n_t + j] : make_float2(0.f, 0.f);
    }
    pdl_wait();  // C0 comes from the previous kernel (no early trigger: see k_theta_m0)
    for (int e = tid; e < SB * (L + 1); e += 256) {
        const int i = i0 + e / (L + 1);
        sC[e] = i < n_r ? C0[(size_t)i0 * (L + 1) + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int jj = tid & 127, half = tid >> 7, j = j0 + jj;
    if (j >= n_t) return;
    // this thread's shells in groups of four (SB is a multiple of 8): four chains in flight
    for (int s0 = 4 * half; s0 < SB; s0 += 8) {
        float2 g[4];
        g0_double_float_n<4>(sT + jj, 128, sC + (size_t)s0 * (L + 1), L + 1, L, g);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + s0 + k;
            if (i < n_r) *reinterpret_cast<float2 *>(G0 + 2 * ((size_t)i * n_t + j)) = g[k];
        }
    }
}

// ---------------------------------------------------------------------------- tables
__device__ __forceinline__ void split3_f64(double v, uint16_t &b0, uint16_t &b1, uint16_t &b2)
{
    __nv_bfloat16 h0 = __float2bfloat16_rn((float)v);
    const double r1 = v - (double)__bfloat162float(h0);
    __nv_bfloat16 h1 = __float2bfloat16_rn((float)r1);
    const double r2 = r1 - (double)__bfloat162float(h1);
    __nv_bfloat16 h2 = __float2bfloat16_rn((float)r2);
    b0 = *reinterpret_cast<uint16_t *>(&h0);
    b1 = *reinterpret_cast<uint16_t *>(&h1);
    b2 = *reinterpret_cast<uint16_t *>(&h2);
}

// byte offset of (row, k) inside one [rows x 32] K-major canonical chunk
__device__ __forceinline__ size_t chunk_off(int row, int k)
{
    return (size_t)(row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// theta contraction B operand: order m = 1 + blockIdx.y; thread (kc, n, kk) of that order
__global__ void k_tab_theta_tc(const double *__restrict__ Ith, int n_t, int L, int n_kc,
                               const unsigned long long *__restrict__ off, uint8_t *__restrict__ tab)
{
    const int m = 1 + blockIdx.y;
    const int Nm = round16(L + 1 - m);
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_kc * Nm * 32) return;
    const int kc = (int)(idx / (Nm * 32)), rem = (int)(idx % (Nm * 32));
    const int n = rem / 32, kk = rem % 32;
    const int l = m + n, j = kc * 32 + kk;
    const double v = (l <= L && j < n_t) ? Ith[(size_t)tri(l, m) * n_t + j] : 0.0;
    uint16_t b[3];
    split3_f64(v, b[0], b[1], b[2]);
    uint8_t *base = tab + off[m] + (size_t)kc * 3 * Nm * 64;
    for (int t = 0; t < 3; ++t) *reinterpret_cast<uint16_t *>(base + (size_t)t * Nm * 64 + chunk_off(n, kk)) = b[t];
}

// theta synthesis A operand: order m = 1 + blockIdx.y; thread (jb, kc, j, kk) of that order
__global__ void k_tab_gsynth_tc(const double *__restrict__ Ith, const double *__restrict__ dmu, int n_t, int L,
                                int n_jb, const unsigned long long *__restrict__ off, uint8_t *__restrict__ tab)
{
    const int m = 1 + blockIdx.y;
    const int n_kcm = (L + 1 - m + 31) / 32;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_jb * n_kcm * 128 * 32) return;
    const int kk = (int)(idx % 32);
    const int jr = (int)((idx / 32) % 128);
    const int kc = (int)((idx / (32 * 128)) % n_kcm);
    const int jb = (int)(idx / (32 * 128 * n_kcm));
    const int l = m + kc * 32 + kk, j = jb * 128 + jr;
    const double v = (l <= L && j < n_t) ? Ith[(size_t)tri(l, m) * n_t + j] / dmu[j] : 0.0;
    uint16_t b[3];
    split3_f64(v, b[0], b[1], b[2]);
    uint8_t *base = tab + off[m] + ((size_t)jb * n_kcm + kc) * 3 * gsc::T_TERM_BYTES;
    for (int t = 0; t < 3; ++t)
        *reinterpret_cast<uint16_t *>(base + (size_t)t * gsc::T_TERM_BYTES + chunk_off(jr, kk)) = b[t];
}

constexpr int kSmemLimit = 232448;

}  // namespace

// ---------------------------------------------------------------------------- plan
size_t theta_tc_smem(const SplitPlan &pl)
{
    const size_t stage = thc::F_BYTES + (size_t)(pl.n_products == 3 ? 2 : 3) * pl.th_Nmax * 64;
    return 1024 + (size_t)pl.th_ns_s * stage + (size_t)pl.th_ns_o * pl.a_terms * thc::A_TERM_BYTES + 512;
}

size_t gsynth_tc_smem(const SplitPlan &pl)
{
    const size_t stage = (size_t)(pl.n_products == 3 ? 2 : 3) * gsc::T_TERM_BYTES + (size_t)pl.a_terms * 2 * pl.gs_NS * 64;
    return 128 + (size_t)pl.gs_ns_s * stage + 512;
}

// Theta synthesis with NS shells per unit: fills pl.gs_* and the per-order offsets of the
// coefficient terms the radial recurrences write (false when the stages do not fit).
bool gsynth_plan_ns(mp_mesh *m, int ns, std::vector<unsigned long long> &cb_off, size_t &cb_bytes)
{
    SplitPlan &pl = m->plan;
    const int L = m->L;
    pl.gs_NS = ns;
    pl.gs_n_sg = (m->n_r + ns - 1) / ns;
    pl.gs_units = pl.gs_n_jb * pl.gs_n_sg * pl.gs_n_mg;
    pl.gs_ns_s = 8;
    while (pl.gs_ns_s > 2 && gsynth_tc_smem(pl) > (size_t)kSmemLimit) --pl.gs_ns_s;
    if (gsynth_tc_smem(pl) > (size_t)kSmemLimit) return false;
    pl.gs_smem = (int)gsynth_tc_smem(pl);
    cb_off.assign(L + 1, 0);
    cb_bytes = 0;
    for (int mm = 1; mm <= L; ++mm) {
        const int n_kcm = (L + 1 - mm + 31) / 32;
        cb_off[mm] = cb_bytes;
        cb_bytes += (size_t)pl.gs_n_sg * n_kcm * pl.a_terms * 2 * ns * 64;
    }
    return true;
}

// Switches a mesh's theta synthesis to NS shells per unit (8, 16 or 32): new coefficient
// offsets, and the coefficient buffer cleared (its padding must read as zeros).  Waits for
// the mesh's stream.
cudaError_t set_gsynth_ns(mp_mesh *m, int ns)
{
    std::vector<unsigned long long> cb_off;
    size_t cb_bytes = 0;
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return e;
    if (!gsynth_plan_ns(m, ns, cb_off, cb_bytes) || cb_bytes > m->cb_bytes_alloc) return cudaErrorInvalidValue;
    e = cudaMemcpy(m->d_cb_off, cb_off.data(), cb_off.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(m->d_Cb, 0, m->cb_bytes_alloc, m->stream);
}

// Sizes of the tensor-core theta stages; fills pl.th_* / pl.gs_* and the table offsets.
// Returns false when they do not apply (l_max = 0: only the m = 0 column exists).
bool plan_theta_tc(mp_mesh *m, std::vector<unsigned long long> &th_off, size_t &th_bytes,
                   std::vector<unsigned long long> &gs_off, size_t &gs_bytes, std::vector<unsigned long long> &cb_off,
                   size_t &cb_bytes)
{
    SplitPlan &pl = m->plan;
    const int L = m->L;
    pl.use_theta_tc = pl.theta_tc_ok = pl.theta_tc_default = 0;
    if (L < 1) return false;
    // (a2): 64 shells per unit; accumulators of Nmax = max_m round16(L + 1 - m) columns
    pl.th_Nmax = round16(L);
    pl.th_n_kc = (m->n_t + thc::BK - 1) / thc::BK;
    pl.th_groups = (m->n_r + thc::SHELLS - 1) / thc::SHELLS;
    pl.th_units = L * pl.th_groups;
    pl.th_nacc = std::max(1, std::min(std::min(4, 256 / pl.th_Nmax), pl.th_n_kc));
    pl.th_ns_o = 2;
    pl.th_ns_s = 8;  // deep rings: the stages are small and the kernel is bound by the bytes in flight
    while (pl.th_ns_s > 2 && theta_tc_smem(pl) > (size_t)kSmemLimit) pl.th_ns_s -= 2;
    if (theta_tc_smem(pl) > (size_t)kSmemLimit) return false;
    th_off.assign(L + 1, 0);
    th_bytes = 0;
    for (int mm = 1; mm <= L; ++mm) {
        th_off[mm] = th_bytes;
        th_bytes += (size_t)pl.th_n_kc * 3 * round16(L + 1 - mm) * 64;
    }
    // (d1): 128 polar cells x NS shells x 4 orders per unit; NS the widest of 32 / 16 / 8 that
    // still gives every SM two units (mp_autotune may choose another; the coefficient buffer
    // is sized for the widest)
    pl.gs_n_jb = (m->n_t + 127) / 128;
    pl.gs_n_mg = (L + gsc::ORDERS - 1) / gsc::ORDERS;
    int ns = 8;
    for (int c = 32; c >= 16; c /= 2) {
        const long long units = (long long)pl.gs_n_jb * ((m->n_r + c - 1) / c) * pl.gs_n_mg;
        if (units >= 2LL * m->num_sms) {
            ns = c;
            break;
        }
    }
    size_t cb32 = 0;
    if (!gsynth_plan_ns(m, 32, cb_off, cb32)) return false;
    if (!gsynth_plan_ns(m, ns, cb_off, cb_bytes)) return false;
    cb_bytes = std::max(cb_bytes, cb32);
    gs_off.assign(L + 1, 0);
    gs_bytes = 0;
    for (int mm = 1; mm <= L; ++mm) {
        const int n_kcm = (L + 1 - mm + 31) / 32;
        gs_off[mm] = gs_bytes;
        gs_bytes += (size_t)pl.gs_n_jb * n_kcm * 3 * gsc::T_TERM_BYTES;
    }
    pl.th_smem = (int)theta_tc_smem(pl);
    pl.gs_smem = (int)gsynth_tc_smem(pl);
    // Both engines are built; the tensor cores take the theta stages by default where the
    // CUDA-core contraction cannot hold its tables in shared memory (large l_max x n_theta).
    // Measured on GB300: 512 x 128 x 256 cells at l_max = 16 (tables resident) solve in 86 us
    // on the CUDA-core theta kernels and 126 us on the tensor-core ones (two more launches,
    // small units); 2048 x 512 x 1024 at l_max = 64 in 4.25 ms against 4.71 ms.
    pl.theta_tc_ok = 1;
    pl.theta_tc_default = theta_pipe_fits(m) ? 0 : 1;
    pl.use_theta_tc = pl.theta_tc_default;
    return true;
}

cudaError_t launch_theta_tc_tables(mp_mesh *m)
{
    const SplitPlan &pl = m->plan;
    if (!pl.theta_tc_ok) return cudaSuccess;
    {
        const long long n = (long long)pl.th_n_kc * pl.th_Nmax * 32;
        k_tab_theta_tc<<<dim3((unsigned)((n + 255) / 256), m->L), 256, 0, m->stream>>>(m->d_Ith, m->n_t, m->L,
                                                                                       pl.th_n_kc, m->d_th_off,
                                                                                       m->d_tabTh);
    }
    {
        const long long n = (long long)pl.gs_n_jb * ((m->L + 31) / 32) * 128 * 32;
        k_tab_gsynth_tc<<<dim3((unsigned)((n + 255) / 256), m->L), 256, 0, m->stream>>>(
            m->d_Ith, m->d_dmu, m->n_t, m->L, pl.gs_n_jb, m->d_gs_off, m->d_tabGs);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static bool attr_set = false;
    if (!attr_set) {
        for (cudaError_t r : {cudaFuncSetAttribute(k_theta_tc<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit),
                              cudaFuncSetAttribute(k_theta_tc<3, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit),
                              cudaFuncSetAttribute(k_gsynth_tc<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit),
                              cudaFuncSetAttribute(k_gsynth_tc<3, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit),
                              cudaFuncSetAttribute(k_gsynth_m0, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit)})
            if (r != cudaSuccess) return r;
        attr_set = true;
    }
    return cudaSuccess;
}

cudaError_t launch_theta_tc(mp_mesh *m)
{
    constexpr double kFourPi = 12.566370614359172954;
    const SplitPlan &pl = m->plan;
    ThetaTcParams prm;
    prm.tab = m->d_tabTh;
    prm.off = m->d_th_off;
    prm.F = m->d_F32;
    prm.Ith32 = m->d_Ith32;
    prm.A = m->d_A;
    prm.err = m->d_err;
    prm.n_r = m->n_r;
    prm.n_t = m->n_t;
    prm.L = m->L;
    prm.KL = m->KL;
    prm.P = m->P;
    prm.ldF = pl.ldF;
    prm.n_kc = pl.th_n_kc;
    prm.n_groups = pl.th_groups;
    prm.n_units = pl.th_units;
    prm.ns_s = pl.th_ns_s;
    prm.ns_o = pl.th_ns_o;
    prm.nacc = pl.th_nacc;
    prm.Nmax = pl.th_Nmax;
    prm.bterms = pl.n_products == 3 ? 2 : 3;
    prm.stage_bytes = (uint32_t)(thc::F_BYTES + prm.bterms * pl.th_Nmax * 64);
    prm.scale = kFourPi * m->G;
    // the m = 0 column first (CUDA cores), then the orders m >= 1
    cudaEvent_t ev;
    prof_begin(m, "split_theta_contract_m0", &ev);
    cudaError_t e = launch_pdl(k_theta_m0, dim3((m->n_r + kM0Shells - 1) / kM0Shells, (m->L + kM0Deg) / kM0Deg),
                               dim3(256), 0, m->stream, prm);
    prof_end(m, "split_theta_contract_m0", ev);
    if (e != cudaSuccess) return e;
    const int grid = std::min(pl.th_units, m->num_sms);
    prof_begin(m, "split_theta_contract_tc", &ev);
    e = pl.a_terms == 2
            ? launch_pdl(k_theta_tc<2, 3>, dim3(grid), dim3(thc::THREADS), pl.th_smem, m->stream, m->tm_F, prm)
            : launch_pdl(k_theta_tc<3, 6>, dim3(grid), dim3(thc::THREADS), pl.th_smem, m->stream, m->tm_F, prm);
    prof_end(m, "split_theta_contract_tc", ev);
    return e;
}

cudaError_t launch_gsynth_tc(mp_mesh *m)
{
    const SplitPlan &pl = m->plan;
    GsynthTcParams prm;
    prm.tab = m->d_tabGs;
    prm.toff = m->d_gs_off;
    prm.cb = m->d_Cb;
    prm.coff = m->d_cb_off;
    prm.Aop = m->d_Aop;
    prm.err = m->d_err;
    prm.n_r = m->n_r;
    prm.n_t = m->n_t;
    prm.L = m->L;
    prm.Kpad = pl.Kpad;
    prm.NS = pl.gs_NS;
    prm.n_jb = pl.gs_n_jb;
    prm.n_sg = pl.gs_n_sg;
    prm.n_units = pl.gs_units;
    prm.ns_s = pl.gs_ns_s;
    prm.bterms = pl.n_products == 3 ? 2 : 3;
    prm.stage_bytes = (uint32_t)(prm.bterms * gsc::T_TERM_BYTES + pl.a_terms * 2 * pl.gs_NS * 64);
    // the m = 0 column first (double-float on CUDA cores): 32 shells per block, or 8 when that
    // leaves fewer than two blocks per SM
    const int n_jb = (m->n_t + 127) / 128;
    const int SB = (long long)n_jb * ((m->n_r + 31) / 32) >= 2LL * m->num_sms ? 32 : 8;
    const size_t smem0 = ((size_t)(m->L + 1) * 128 + (size_t)SB * (m->L + 1)) * sizeof(float2);
    cudaEvent_t ev;
    prof_begin(m, "split_theta_synth_m0", &ev);
    cudaError_t e = launch_pdl(k_gsynth_m0, dim3(n_jb, (m->n_r + SB - 1) / SB), dim3(256), smem0, m->stream,
                               (const float2 *)m->d_C0, (const float2 *)m->d_Itc0, m->d_G0, m->n_r, m->n_t, m->L, SB);
    prof_end(m, "split_theta_synth_m0", ev);
    if (e != cudaSuccess) return e;
    const int grid = std::min(pl.gs_units, m->num_sms);
    prof_begin(m, "split_theta_synth_tc", &ev);
    e = pl.a_terms == 2 ? launch_pdl(k_gsynth_tc<2, 3>, dim3(grid), dim3(gsc::THREADS), pl.gs_smem, m->stream, prm)
                        : launch_pdl(k_gsynth_tc<3, 6>, dim3(grid), dim3(gsc::THREADS), pl.gs_smem, m->stream, prm);
    prof_end(m, "split_theta_synth_tc", ev);
    return e;
}

}  // namespace mp
