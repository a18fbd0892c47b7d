// mp_split.cu -- split-precision tensor-core path of the two angular
// contractions of GenASiS II Sec. 2.2 (the (L+1)^2 N hot loops):
//
//   (a1) phi projection, Eq. (AngularMomentsDiscrete), phi part:
//        F[row][p] = sum_k rho[row][k] Iph[p][k]            [R x n_phi] x [n_phi x (2L+1)]
//   (d)  reconstruction, Eq. (Solution):
//        G[row][p] = sum_{l>=m} (Ith[t][j]/dmu_j) C[i][q]   (float32, CUDA cores)
//        Phi[row][k] = G[row][0] + sum_{p>=1} G[row][p] Iph[p][k]/dphi_k
//                                                           [R x 2L] x [2L x n_phi]
//
// Both GEMMs run on tcgen05 (M = 128 rows per tile, fp32 accumulators in
// tensor memory) with bf16 operands split into terms: x = x0 + x1 (+ x2),
// x0 = bf16(x), x1 = bf16(x - x0), ...  The density (float64 in HBM) arrives
// through TMA in 128B-swizzled [128 x 16] tiles; converter warps turn each
// value into float32 with integer ops (no float64 pipe), subtract a per-row
// reference value (the row's first cell) so that only the deviation is split,
// and write the bf16 terms in the canonical no-swizzle K-major UMMA layout.
// The per-row reference enters again exactly through the column sums of the
// table.  The reconstruction's float32 accumulators leave tensor memory via
// tcgen05.ld, get the m = 0 term added, become float64 with integer ops and
// leave through TMA stores.
//
// Roles per CTA (persistent, one CTA per SM): warp 0 issues TMA / bulk copies,
// warp 1 owns tensor memory and issues the MMAs, warps 2..9 convert and run
// the epilogues.  Every mbarrier wait is bounded (ptx.cuh).
#include <cstdio>

#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

constexpr int kBM = 128;      // rows per tile (UMMA M)
constexpr int kConvWarps = 8; // converter / epilogue warps
constexpr int kThreads = (2 + kConvWarps) * 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

// bf16 product terms (a_term, b_term) accumulated per K step.
__constant__ int c_prod_a[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_prod_b[6] = {0, 1, 0, 2, 1, 0};

__device__ __forceinline__ uint32_t tmem_ncols_for(int cols)
{
    uint32_t n = 32;
    while (n < (uint32_t)cols) n <<= 1;
    return n;
}

__device__ __forceinline__ bool warp_all(bool v) { return __all_sync(kFull, v); }

// ----------------------------------------------------------------------------
// (a1) phi projection
// ----------------------------------------------------------------------------
namespace proj {
constexpr int BK = 32;                       // float64 cells per stage (two TMA boxes of 16)
constexpr int BOX_BYTES = kBM * 16 * 8;      // one [128 x 16] float64 box, 16 KB
constexpr int S_BYTES = 2 * BOX_BYTES;       // 32 KB
constexpr int A_TERM_BYTES = kBM * BK * 2;   // [128 x 32] bf16, 8 KB
constexpr int SBO = (BK / 8) * 128;          // 8-row group stride of A and B chunks
}  // namespace proj

// Position in a ring of mbarrier-guarded stages: index and phase advance together.
struct Ring {
    int idx = 0;
    uint32_t phase = 0;
    __device__ __forceinline__ void next(int n)
    {
        if (++idx == n) {
            idx = 0;
            phase ^= 1u;
        }
    }
};

struct ProjParams {
    const uint8_t *tabB;   // [n_kc][3][Npad x 32] bf16, canonical layout
    const float *colsum;   // [Npad]
    float *F;              // [R][Npad]
    int *err;
    long long R;
    int n_p, n_kc, Npad, n_tiles, ns_s, ns_o;
    uint32_t bchunk;       // bytes of one B chunk (3 terms)
};

template <int A_TERMS, int NPROD>
__global__ void __launch_bounds__(kThreads, 1) k_proj_tc(const __grid_constant__ CUtensorMap tmS, const ProjParams prm)
{
    using namespace proj;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS_S = prm.ns_s, NS_O = prm.ns_o;
    uint8_t *sS = smem;
    uint8_t *sB = sS + (size_t)NS_S * S_BYTES;
    uint8_t *sA = sB + (size_t)NS_S * prm.bchunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + (size_t)NS_O * A_TERMS * A_TERM_BYTES);
    uint64_t *s_full = bars, *s_empty = bars + NS_S;
    uint64_t *b_full = bars + 2 * NS_S, *b_empty = b_full + NS_S;
    uint64_t *o_full = bars + 4 * NS_S, *o_empty = o_full + NS_O;
    uint64_t *acc_full = o_empty + NS_O, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Npad = prm.Npad;
    const uint32_t ncols = tmem_ncols_for(2 * Npad);
    const uint32_t acc_stride = ncols / 2;  // accumulator buffers at power-of-two column offsets

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS_S; ++s) {
            mbar_init(smem_u32(&s_full[s]), 1);
            mbar_init(smem_u32(&s_empty[s]), kConvWarps);  // density stages: free once converted
            mbar_init(smem_u32(&b_full[s]), 1);
            mbar_init(smem_u32(&b_empty[s]), 1);           // table stages: free once the MMAs read them
        }
        for (int o = 0; o < NS_O; ++o) {
            mbar_init(smem_u32(&o_full[o]), kConvWarps);
            mbar_init(smem_u32(&o_empty[o]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kConvWarps);
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

    if (warp == 0) {
        // ---------------- producer: two TMA boxes of rho, and the table chunk on its own ring
        if (lane == 0) {
            tma_prefetch_desc(&tmS);
            Ring rs;
            int issued = 0;
            for (int tile = blockIdx.x; tile < prm.n_tiles && !*abort_flag; tile += gridDim.x) {
                for (int kc = 0; kc < prm.n_kc; ++kc, rs.next(NS_S)) {
                    if (!mbar_wait(smem_u32(&s_empty[rs.idx]), rs.phase ^ 1, abort_flag, prm.err)) break;
                    const uint32_t fb = smem_u32(&s_full[rs.idx]);
                    const bool two = kc * BK + 16 < prm.n_p;  // the second box holds cells
                    mbar_arrive_expect_tx(fb, two ? S_BYTES : BOX_BYTES);
                    const uint32_t dst = smem_u32(sS + (size_t)rs.idx * S_BYTES);
                    tma_load_2d(dst, &tmS, fb, kc * BK, tile * kBM);
                    if (two) tma_load_2d(dst + BOX_BYTES, &tmS, fb, kc * BK + 16, tile * kBM);
                    if (!mbar_wait(smem_u32(&b_empty[rs.idx]), rs.phase ^ 1, abort_flag, prm.err)) {
                        ++issued;
                        break;
                    }
                    const uint32_t bb = smem_u32(&b_full[rs.idx]);
                    mbar_arrive_expect_tx(bb, prm.bchunk);
                    bulk_load(smem_u32(sB + (size_t)rs.idx * prm.bchunk), prm.tabB + (size_t)kc * prm.bchunk,
                              prm.bchunk, bb);
                    ++issued;
                }
            }
            if (*abort_flag && issued > 0) {
                // drain copies still in flight into this CTA's shared memory
                Ring back = rs;
                for (int n = 0; n < NS_S && n < issued; ++n) {
                    back.idx = (back.idx == 0) ? NS_S - 1 : back.idx - 1;
                    if (back.idx == NS_S - 1) back.phase ^= 1u;
                    const long long t0 = clock64();
                    while ((!mbar_try_wait(smem_u32(&s_full[back.idx]), back.phase) ||
                            !mbar_try_wait(smem_u32(&b_full[back.idx]), back.phase)) &&
                           clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kBM, Npad);
            Ring rs, ro;
            int lt = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < prm.n_tiles && ok; tile += gridDim.x, ++lt) {
                const int b = lt & 1;
                ok = mbar_wait(smem_u32(&acc_empty[b]), ((lt >> 1) & 1) ^ 1, abort_flag, prm.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)b * acc_stride;
                for (int kc = 0; kc < prm.n_kc; ++kc, rs.next(NS_S), ro.next(NS_O)) {
                    ok = mbar_wait(smem_u32(&o_full[ro.idx]), ro.phase, abort_flag, prm.err) &&
                         mbar_wait(smem_u32(&b_full[rs.idx]), rs.phase, abort_flag, prm.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(sA + (size_t)ro.idx * A_TERMS * A_TERM_BYTES);
                    const uint32_t b_base = smem_u32(sB + (size_t)rs.idx * prm.bchunk);
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
                        for (int pi = 0; pi < NPROD; ++pi) {
                            const uint64_t ad =
                                sdesc_noswizzle(a_base + c_prod_a[pi] * A_TERM_BYTES + ks * 256, 128, SBO);
                            const uint64_t bd =
                                sdesc_noswizzle(b_base + c_prod_b[pi] * Npad * (BK * 2) + ks * 256, 128, SBO);
                            umma_bf16(d_tmem, ad, bd, idesc, (kc | ks | pi) != 0);
                        }
                    }
                    umma_commit(smem_u32(&o_empty[ro.idx]));
                    umma_commit(smem_u32(&b_empty[rs.idx]));
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
        // ---------------- converters + epilogue
        const int cw = warp - 2, qd = warp & 3, half = cw >> 2;
        const int row = qd * 32 + lane;
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        Ring rs, ro;
        int lt = 0, prev_tile = -1;
        float sref = 0.0f, sref_prev = 0.0f;
        uint32_t efmax = 0;  // largest float64 exponent field seen (flags values beyond float32)
        bool ok = true;

        auto epilogue = [&](int etile, int elt, float sr) -> bool {
            const int b = elt & 1;
            bool w_ok = warp_all(mbar_wait(smem_u32(&acc_full[b]), (elt >> 1) & 1, abort_flag, prm.err));
            if (!w_ok) return false;
            tc_fence_after();
            const long long grow = (long long)etile * kBM + row;
            const int ngroups = Npad / 8;
            for (int cg = half; cg < ngroups; cg += 2) {
                uint32_t v[8];
                tmem_ld8(tmem_base + lane_base + (uint32_t)b * acc_stride + (uint32_t)(cg * 8), v);
                tmem_ld_wait();
                if (grow < prm.R) {
                    const float4 c0 = *reinterpret_cast<const float4 *>(prm.colsum + cg * 8);
                    const float4 c1 = *reinterpret_cast<const float4 *>(prm.colsum + cg * 8 + 4);
                    float4 o0, o1;
                    o0.x = fmaf(sr, c0.x, __uint_as_float(v[0]));
                    o0.y = fmaf(sr, c0.y, __uint_as_float(v[1]));
                    o0.z = fmaf(sr, c0.z, __uint_as_float(v[2]));
                    o0.w = fmaf(sr, c0.w, __uint_as_float(v[3]));
                    o1.x = fmaf(sr, c1.x, __uint_as_float(v[4]));
                    o1.y = fmaf(sr, c1.y, __uint_as_float(v[5]));
                    o1.z = fmaf(sr, c1.z, __uint_as_float(v[6]));
                    o1.w = fmaf(sr, c1.w, __uint_as_float(v[7]));
                    float4 *dst = reinterpret_cast<float4 *>(prm.F + grow * Npad + cg * 8);
                    dst[0] = o0;
                    dst[1] = o1;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
            return true;
        };

        // this thread converts cells [16 half, 16 half + 16) of every stage: box `half`
        for (int tile = blockIdx.x; tile < prm.n_tiles && ok; tile += gridDim.x, ++lt) {
            for (int kc = 0; kc < prm.n_kc; ++kc, rs.next(NS_S), ro.next(NS_O)) {
                ok = warp_all(mbar_wait(smem_u32(&s_full[rs.idx]), rs.phase, abort_flag, prm.err));
                if (!ok) break;
                ok = warp_all(mbar_wait(smem_u32(&o_empty[ro.idx]), ro.phase ^ 1, abort_flag, prm.err));
                if (!ok) break;
                const uint8_t *sbox = sS + (size_t)rs.idx * S_BYTES + row * 128;
                if (kc == 0) {
                    const uint2 v0 = *reinterpret_cast<const uint2 *>(sbox + ((row & 7) << 4));
                    uint32_t e0;
                    sref = f64w_to_f32_fast(v0.x, v0.y, e0);
                }
                const uint8_t *srow = sbox + half * BOX_BYTES;
                const int kfirst = kc * BK + half * 16;           // first cell of this thread's box
                const bool full = kfirst + 16 <= prm.n_p;         // warp-uniform
                uint32_t w0[8], w1[8], w2[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(srow + ((c ^ (row & 7)) << 4));
                    uint32_t e0, e1;
                    float x0 = f64w_to_f32_fast(v.x, v.y, e0) - sref;
                    float x1 = f64w_to_f32_fast(v.z, v.w, e1) - sref;
                    if (!full) {
                        // cells past the last azimuthal cell hold no data: zero deviation
                        const bool in0 = kfirst + 2 * c < prm.n_p, in1 = kfirst + 2 * c + 1 < prm.n_p;
                        x0 = in0 ? x0 : 0.0f;
                        x1 = in1 ? x1 : 0.0f;
                        e0 = in0 ? e0 : 0u;
                        e1 = in1 ? e1 : 0u;
                    }
                    efmax = max(efmax, max(e0, e1));
                    const uint32_t t0 = pack_bf16x2(x0, x1);
                    const float r0 = x0 - bf16lo_to_f32(t0), r1 = x1 - bf16hi_to_f32(t0);
                    const uint32_t t1 = pack_bf16x2(r0, r1);
                    w0[c] = t0;
                    w1[c] = t1;
                    if (A_TERMS == 3) w2[c] = pack_bf16x2(r0 - bf16lo_to_f32(t1), r1 - bf16hi_to_f32(t1));
                }
                // K groups 2 half and 2 half + 1 of the [128 x 32] A tile, each term
                uint8_t *adst = sA + (size_t)ro.idx * A_TERMS * A_TERM_BYTES + (row >> 3) * SBO + half * 256 +
                                (row & 7) * 16;
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
                    mbar_arrive(smem_u32(&s_empty[rs.idx]));
                    mbar_arrive(smem_u32(&o_full[ro.idx]));
                }
            }
            if (!ok) break;
            if (prev_tile >= 0) ok = epilogue(prev_tile, lt - 1, sref_prev);
            prev_tile = tile;
            sref_prev = sref;
        }
        if (ok && prev_tile >= 0) epilogue(prev_tile, lt - 1, sref_prev);
        // exponent fields above float32's range (including inf / nan, 0x7FF) are reported
        if (efmax > (1150u << 20)) atomicOr(prm.err, DEV_ERR_NONFINITE);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, ncols);
    }
}

// ----------------------------------------------------------------------------
// (d) reconstruction: theta synthesis on CUDA cores + phi synthesis on tcgen05
// ----------------------------------------------------------------------------
namespace synth {
constexpr int STG_BYTES = 32 * 16 * 8;  // TMA store box [32 rows][16 float64], 128B swizzle
constexpr int JB = 32;                  // polar cells per tile in polar-block mode
}

struct SynthParams {
    const uint8_t *tabT;   // [n_nc][Kpad/16][3][NC x 16] bf16, canonical layout
    const float *C32;      // [n_r][KL]
    const float *Itc;      // [T][n_t]  Ith / dmu
    int *err;
    long long R;
    int n_r, n_t, L, KL, T, P, Kpad, NC, n_nc, ns_b;
    int jblock;            // 1: tiles of (128/JB shells x JB polar cells), table slice in shared memory
    int n_ib;              // shell blocks per polar block (polar-block mode)
    int n_items;           // tiles in total
    uint32_t bchunk;       // bytes of one B chunk (3 terms)
};

// Tile -> (first shell, first polar cell) in polar-block mode; rows r of the
// tile are (shell i0 + r / JB, polar cell j0 + r % JB).
__device__ __forceinline__ void synth_item(const SynthParams &prm, int item, int &i0, int &j0)
{
    const int jb = item / prm.n_ib, ib = item % prm.n_ib;
    i0 = ib * (kBM / synth::JB);
    j0 = jb * synth::JB;
}

template <int A_TERMS, int NPROD>
__global__ void __launch_bounds__(kThreads, 1)
    k_synth_tc(const __grid_constant__ CUtensorMap tmPhi, const SynthParams prm)
{
    using namespace synth;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS_B = prm.ns_b;
    const int Kpad = prm.Kpad, NC = prm.NC;
    const int a_term_bytes = kBM * Kpad * 2;
    const int SB = kBM / JB;
    uint8_t *stg = smem;                                          // [8 warps][2][4096]
    uint8_t *sA = stg + (size_t)kConvWarps * 2 * STG_BYTES;       // [A_TERMS][128 x Kpad]
    uint8_t *sB = sA + (size_t)A_TERMS * a_term_bytes;            // [NS_B][bchunk]
    float *sItc = reinterpret_cast<float *>(sB + (size_t)NS_B * prm.bchunk);  // [T][JB] (polar-block mode)
    float *sC = sItc + (prm.jblock ? (size_t)prm.T * JB : 0);     // [SB][KL] (polar-block mode)
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(sC + (prm.jblock ? (size_t)SB * prm.KL : 0)) + 15) & ~uintptr_t(15));
    uint64_t *a_full = bars, *a_empty = bars + 1;
    uint64_t *b_full = bars + 2, *b_empty = b_full + NS_B;
    uint64_t *acc_full = b_empty + NS_B, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint64_t *c_free = drain + 1, *c_ready = drain + 2;  // compute warps: staged rows free / loaded
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_ncols_for(2 * NC);
    const uint32_t acc_stride = ncols / 2;
    const int nkk = Kpad / 16;
    // contiguous range of tiles of this CTA (consecutive tiles share a polar block)
    const int it0 = (int)((long long)prm.n_items * blockIdx.x / gridDim.x);
    const int it1 = (int)((long long)prm.n_items * (blockIdx.x + 1) / gridDim.x);

    if (threadIdx.x == 0) {
        mbar_init(smem_u32(a_full), kConvWarps);
        mbar_init(smem_u32(a_empty), 1);
        for (int s = 0; s < NS_B; ++s) {
            mbar_init(smem_u32(&b_full[s]), 1);
            mbar_init(smem_u32(&b_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kConvWarps);
        }
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(c_free), kConvWarps);
        mbar_init(smem_u32(c_ready), kConvWarps);
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

    if (warp == 0) {
        // ---------------- producer: table chunks (nc, kk) for every tile
        if (lane == 0) {
            Ring rb;
            int issued = 0;
            bool ok = true;
            for (int it = it0; it < it1 && ok; ++it)
                for (int nc = 0; nc < prm.n_nc && ok; ++nc)
                    for (int kk = 0; kk < nkk; ++kk, rb.next(NS_B)) {
                        ok = mbar_wait(smem_u32(&b_empty[rb.idx]), rb.phase ^ 1, abort_flag, prm.err);
                        if (!ok) break;
                        mbar_arrive_expect_tx(smem_u32(&b_full[rb.idx]), prm.bchunk);
                        bulk_load(smem_u32(sB + (size_t)rb.idx * prm.bchunk),
                                  prm.tabT + ((size_t)nc * nkk + kk) * prm.bchunk, prm.bchunk,
                                  smem_u32(&b_full[rb.idx]));
                        ++issued;
                    }
            if (*abort_flag && issued > 0) {
                Ring back = rb;
                for (int n = 0; n < NS_B && n < issued; ++n) {
                    back.idx = (back.idx == 0) ? NS_B - 1 : back.idx - 1;
                    if (back.idx == NS_B - 1) back.phase ^= 1u;
                    const long long t0 = clock64();
                    while (!mbar_try_wait(smem_u32(&b_full[back.idx]), back.phase) &&
                           clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kBM, NC);
            const uint32_t sbo_a = (uint32_t)Kpad * 16;
            Ring rb;
            uint32_t u = 0;
            int lt = 0;
            bool ok = true;
            for (int it = it0; it < it1 && ok; ++it, ++lt) {
                ok = mbar_wait(smem_u32(a_full), lt & 1, abort_flag, prm.err);
                if (!ok) break;
                tc_fence_after();
                for (int nc = 0; nc < prm.n_nc && ok; ++nc, ++u) {
                    const int buf = u & 1;
                    ok = mbar_wait(smem_u32(&acc_empty[buf]), ((u >> 1) & 1) ^ 1, abort_flag, prm.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)buf * acc_stride;
                    for (int kk = 0; kk < nkk; ++kk, rb.next(NS_B)) {
                        ok = mbar_wait(smem_u32(&b_full[rb.idx]), rb.phase, abort_flag, prm.err);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t a_base = smem_u32(sA) + (uint32_t)(kk * 256);
                        const uint32_t b_base = smem_u32(sB + (size_t)rb.idx * prm.bchunk);
#pragma unroll
                        for (int pi = 0; pi < NPROD; ++pi) {
                            const uint64_t ad =
                                sdesc_noswizzle(a_base + (uint32_t)(c_prod_a[pi] * a_term_bytes), 128, sbo_a);
                            const uint64_t bd = sdesc_noswizzle(b_base + (uint32_t)(c_prod_b[pi] * NC * 32), 128, 256);
                            umma_bf16(d_tmem, ad, bd, idesc, (kk | pi) != 0);
                        }
                        umma_commit(smem_u32(&b_empty[rb.idx]));
                    }
                    if (!ok) break;
                    umma_commit(smem_u32(&acc_full[buf]));
                }
                if (!ok) break;
                umma_commit(smem_u32(a_empty));
            }
            umma_commit(smem_u32(drain));
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(drain), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
            }
        }
    } else {
        // ---------------- theta synthesis (A operand) + epilogue (Phi)
        const int cw = warp - 2, qd = warp & 3, half = cw >> 2;
        const int row = qd * 32 + lane;
        const int ctid = threadIdx.x - 64;  // 0..255 among the compute warps
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        const int n_t = prm.n_t, L = prm.L, KL = prm.KL;
        uint32_t u = 0, cs = 0;
        int lt = 0, cur_j0 = -1;
        bool ok = true;
        for (int it = it0; it < it1 && ok; ++it, ++lt) {
            ok = warp_all(mbar_wait(smem_u32(a_empty), (lt & 1) ^ 1, abort_flag, prm.err));
            if (!ok) break;
            // rows of this tile: (shell i, polar cell j) and the first memory row of this warp's box
            int i, j;
            long long box_row;
            bool valid;
            const float *crow;    // coefficients C[i][*] of this row's shell
            const float *itab;    // table Itc[t][j], stride tstride in t
            int tstride;
            if (prm.jblock) {
                int i0, j0;
                synth_item(prm, it, i0, j0);
                i = i0 + row / JB;
                j = j0 + row % JB;
                valid = i < prm.n_r;
                box_row = (long long)(i0 + (qd * 32) / JB) * n_t + j0 + (qd * 32) % JB;
                // every compute warp is done with the previous tile's staged rows
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(c_free));
                ok = warp_all(mbar_wait(smem_u32(c_free), lt & 1, abort_flag, prm.err));
                if (!ok) break;
                if (j0 != cur_j0) {
                    for (int e = ctid; e < prm.T * JB; e += 256)
                        sItc[e] = __ldg(prm.Itc + (size_t)(e / JB) * n_t + j0 + e % JB);
                    cur_j0 = j0;
                }
                for (int e = ctid; e < SB * KL; e += 256) {
                    const int si = i0 + e / KL;
                    sC[e] = (si < prm.n_r) ? __ldg(prm.C32 + (size_t)si * KL + e % KL) : 0.0f;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(c_ready));
                ok = warp_all(mbar_wait(smem_u32(c_ready), lt & 1, abort_flag, prm.err));
                if (!ok) break;
                crow = sC + (row / JB) * KL;
                itab = sItc + row % JB;
                tstride = JB;
            } else {
                const long long grow = (long long)it * kBM + row;
                valid = grow < prm.R;
                i = valid ? (int)(grow / n_t) : 0;
                j = valid ? (int)(grow % n_t) : 0;
                box_row = (long long)it * kBM + qd * 32;
                crow = prm.C32 + (size_t)i * KL;
                itab = prm.Itc + j;
                tstride = n_t;
            }
            (void)i;
            (void)j;
            float g0 = 0.0f, g1 = 0.0f;
            if (valid) {
                int l = 0;
                for (; l + 1 <= L; l += 2) {
                    g0 = fmaf(itab[(size_t)tri(l, 0) * tstride], crow[l * l], g0);
                    g1 = fmaf(itab[(size_t)tri(l + 1, 0) * tstride], crow[(l + 1) * (l + 1)], g1);
                }
                if (l <= L) g0 = fmaf(itab[(size_t)tri(l, 0) * tstride], crow[l * l], g0);
                g0 += g1;
            }
            // A operand: G[row][p], p = 1..2L, stored at K index p-1, in A_TERMS bf16 terms.
            // Group gi holds p = 8 gi + 1 .. 8 gi + 8, the cos/sin pairs of m = 4 gi + 1 .. 4 gi + 4;
            // each table value serves both members of a pair.
            for (int gi = half; gi < Kpad / 8; gi += 2) {
                float gv[8];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm) {
                    const int m = 4 * gi + mm + 1;
                    float ac = 0.0f, as = 0.0f, bc = 0.0f, bs = 0.0f;
                    if (valid && m <= L) {
                        const float *cc = crow + 2 * m - 1;  // C[i][l^2 + 2m - 1], C[i][l^2 + 2m]
                        int l = m;
                        for (; l + 1 <= L; l += 2) {
                            const float w0 = itab[(size_t)tri(l, m) * tstride];
                            const float w1 = itab[(size_t)tri(l + 1, m) * tstride];
                            ac = fmaf(w0, cc[l * l], ac);
                            as = fmaf(w0, cc[l * l + 1], as);
                            bc = fmaf(w1, cc[(l + 1) * (l + 1)], bc);
                            bs = fmaf(w1, cc[(l + 1) * (l + 1) + 1], bs);
                        }
                        if (l <= L) {
                            const float w0 = itab[(size_t)tri(l, m) * tstride];
                            ac = fmaf(w0, cc[l * l], ac);
                            as = fmaf(w0, cc[l * l + 1], as);
                        }
                    }
                    gv[2 * mm] = ac + bc;
                    gv[2 * mm + 1] = as + bs;
                }
                uint32_t w0[4], w1[4], w2[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const float x0 = gv[2 * cc], x1 = gv[2 * cc + 1];
                    const uint32_t t0 = pack_bf16x2(x0, x1);
                    const float r0 = x0 - bf16lo_to_f32(t0), r1 = x1 - bf16hi_to_f32(t0);
                    const uint32_t t1 = pack_bf16x2(r0, r1);
                    w0[cc] = t0;
                    w1[cc] = t1;
                    if (A_TERMS == 3) w2[cc] = pack_bf16x2(r0 - bf16lo_to_f32(t1), r1 - bf16hi_to_f32(t1));
                }
                uint8_t *adst = sA + (size_t)(row >> 3) * (Kpad * 16) + gi * 128 + (row & 7) * 16;
                *reinterpret_cast<uint4 *>(adst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *reinterpret_cast<uint4 *>(adst + a_term_bytes) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                if (A_TERMS == 3)
                    *reinterpret_cast<uint4 *>(adst + 2 * a_term_bytes) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(a_full));

            // a box of 32 rows is written only when its first row is a real row
            const bool box_valid = prm.jblock ? (__shfl_sync(kFull, valid ? 1 : 0, 0) != 0) : (box_row < prm.R);
            int nc_cur = 0;
            // converts 16 accumulator columns of this row (+ the m = 0 term) to float64 in a
            // swizzled staging box and hands the box to a TMA store
            auto store_chunk = [&](const uint32_t(&v)[16], int ch) {
                uint8_t *st = stg + (size_t)(cw * 2 + (cs & 1)) * STG_BYTES;
                ++cs;
                if (lane == 0) bulk_wait_read_le1();
                __syncwarp();
                uint8_t *srow = st + lane * 128;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    uint32_t lo0, hi0, lo1, hi1;
                    f32_to_f64w_finite(__uint_as_float(v[2 * e]) + g0, lo0, hi0);
                    f32_to_f64w_finite(__uint_as_float(v[2 * e + 1]) + g0, lo1, hi1);
                    *reinterpret_cast<uint4 *>(srow + ((e ^ (lane & 7)) << 4)) = make_uint4(lo0, hi0, lo1, hi1);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0 && box_valid) {
                    tma_store_2d(&tmPhi, smem_u32(st), nc_cur * NC + ch * 16, (int)box_row);
                    bulk_commit();
                }
            };
            for (int nc = 0; nc < prm.n_nc && ok; ++nc, ++u) {
                nc_cur = nc;
                const int buf = u & 1;
                ok = warp_all(mbar_wait(smem_u32(&acc_full[buf]), (u >> 1) & 1, abort_flag, prm.err));
                if (!ok) break;
                tc_fence_after();
                // 16-column chunks ch = half, half + 2, ...; the tensor-memory load of the
                // next chunk is in flight while the current one is converted and stored
                const int nch = NC / 16;
                const uint32_t tcol = tmem_base + lane_base + (uint32_t)buf * acc_stride;
                uint32_t va[16], vb[16];
                if (half < nch) tmem_ld16(tcol + (uint32_t)(half * 16), va);
                tmem_ld_wait();
                for (int ch = half; ch < nch; ch += 4) {
                    const bool nb = ch + 2 < nch, na = ch + 4 < nch;
                    if (nb) tmem_ld16(tcol + (uint32_t)((ch + 2) * 16), vb);
                    store_chunk(va, ch);
                    if (nb) {
                        tmem_ld_wait();
                        if (na) tmem_ld16(tcol + (uint32_t)((ch + 4) * 16), va);
                        store_chunk(vb, ch + 2);
                        if (na) tmem_ld_wait();
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
            }
        }
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, ncols);
    }
}

// ----------------------------------------------------------------------------
// split tables: bf16 x 3 terms in the canonical K-major no-swizzle layout
// ----------------------------------------------------------------------------
__device__ __forceinline__ void split3(double v, uint16_t &b0, uint16_t &b1, uint16_t &b2)
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

// byte offset of element (n, kk) inside one [rows x 16] K-major term
__device__ __forceinline__ size_t canon_off(int n, int kk)
{
    return (size_t)(n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2;
}

// projection B: chunk kc, term tb, row p (N), column kk (K = azimuthal cell), 32 cells per chunk
__global__ void k_tab_proj(const double *__restrict__ Iph, int n_p, int P, int Npad, int n_kc, uint8_t *__restrict__ tab,
                           float *__restrict__ colsum)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int BK = proj::BK;
    const long long total = (long long)n_kc * Npad * BK;
    if (idx < Npad && colsum) {
        double s = 0.0;
        if (idx < P)
            for (int k = 0; k < n_p; ++k) s += Iph[(size_t)idx * n_p + k];
        colsum[idx] = (float)s;
    }
    if (idx >= total) return;
    const int kc = (int)(idx / (Npad * BK));
    const int rem = (int)(idx % (Npad * BK));
    const int p = rem / BK, kk = rem % BK;
    const int k = kc * BK + kk;
    const double v = (p < P && k < n_p) ? Iph[(size_t)p * n_p + k] : 0.0;
    uint16_t b0, b1, b2;
    split3(v, b0, b1, b2);
    const size_t term = (size_t)Npad * BK * 2;
    uint8_t *base = tab + (size_t)kc * 3 * term;
    const size_t off = (size_t)(p >> 3) * proj::SBO + (kk >> 3) * 128 + (p & 7) * 16 + (kk & 7) * 2;
    *reinterpret_cast<uint16_t *>(base + off) = b0;
    *reinterpret_cast<uint16_t *>(base + term + off) = b1;
    *reinterpret_cast<uint16_t *>(base + 2 * term + off) = b2;
}

// synthesis B: chunk (nc, kc), term tb, row n (N = azimuthal cell), column kk (K = p - 1)
__global__ void k_tab_synth(const double *__restrict__ Iphc, int n_p, int P, int Kpad, int NC, int n_nc,
                            uint8_t *__restrict__ tab)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nkk = Kpad / 16;
    const long long total = (long long)n_nc * nkk * NC * 16;
    if (idx >= total) return;
    const long long chunk = idx / (NC * 16);
    const int rem = (int)(idx % (NC * 16));
    const int n = rem / 16, kk = rem % 16;
    const int nc = (int)(chunk / nkk), kc = (int)(chunk % nkk);
    const int k = nc * NC + n;
    const int p = kc * 16 + kk + 1;
    const double v = (p < P && k < n_p) ? Iphc[(size_t)p * n_p + k] : 0.0;
    uint16_t b0, b1, b2;
    split3(v, b0, b1, b2);
    uint8_t *base = tab + (size_t)chunk * 3 * NC * 32;
    const size_t off = canon_off(n, kk);
    *reinterpret_cast<uint16_t *>(base + off) = b0;
    *reinterpret_cast<uint16_t *>(base + (size_t)NC * 32 + off) = b1;
    *reinterpret_cast<uint16_t *>(base + (size_t)2 * NC * 32 + off) = b2;
}

// float32 theta tables: IthT[j][t] = Ith[t][j], Itc[t][j] = Ith[t][j] / dmu_j
__global__ void k_tab_theta32(const double *__restrict__ Ith, const double *__restrict__ dmu, int n_t, int T,
                              float *__restrict__ IthT, float *__restrict__ Itc)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)T * n_t) return;
    const int t = (int)(idx / n_t), j = (int)(idx % n_t);
    const double v = Ith[idx];
    IthT[(size_t)j * T + t] = (float)v;
    Itc[idx] = (float)(v / dmu[j]);
}

template <int A_TERMS, int NPROD>
cudaError_t set_smem_attrs(int proj_smem, int synth_smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_proj_tc<A_TERMS, NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         proj_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_synth_tc<A_TERMS, NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize, synth_smem);
}

int proj_smem_bytes(const SplitPlan &pl, int ns_s, int ns_o)
{
    const int bchunk = 3 * pl.Npad * proj::BK * 2;
    return 1024 + ns_s * proj::S_BYTES + ns_s * bchunk + ns_o * pl.a_terms * proj::A_TERM_BYTES + 512;
}

int synth_smem_bytes(const SplitPlan &pl, int ns_b, int jblock, int T, int KL)
{
    const int bchunk = 3 * pl.NC * 32;
    const int tabs = jblock ? (T * synth::JB + (kBM / synth::JB) * KL) * 4 + 16 : 0;
    return 1024 + kConvWarps * 2 * synth::STG_BYTES + pl.a_terms * kBM * pl.Kpad * 2 + ns_b * bchunk + tabs + 256;
}

constexpr int kSmemLimit = 232448;  // 227 KB opt-in per block on sm_100-class parts

}  // namespace

// Chooses ring depths that fit shared memory; fills plan.* sizes.
int split_smem_limits(mp_mesh *m)
{
    SplitPlan &pl = m->plan;
    int ns_s = 4;
    while (ns_s > 2 && proj_smem_bytes(pl, ns_s, 2) > kSmemLimit) --ns_s;
    if (proj_smem_bytes(pl, ns_s, 2) > kSmemLimit) return 1;
    // polar-block tiles when the polar cells split into blocks of 32 and the table slice fits
    int jblock = (m->n_t % synth::JB == 0) ? 1 : 0;
    int ns_b = 3;
    while (ns_b > 2 && synth_smem_bytes(pl, ns_b, jblock, m->T, m->KL) > kSmemLimit) --ns_b;
    if (jblock && synth_smem_bytes(pl, ns_b, jblock, m->T, m->KL) > kSmemLimit) {
        jblock = 0;
        ns_b = 3;
        while (ns_b > 2 && synth_smem_bytes(pl, ns_b, 0, m->T, m->KL) > kSmemLimit) --ns_b;
    }
    if (synth_smem_bytes(pl, ns_b, jblock, m->T, m->KL) > kSmemLimit) return 2;
    pl.jblock = jblock;
    pl.proj_smem = proj_smem_bytes(pl, ns_s, 2);
    pl.synth_smem = synth_smem_bytes(pl, ns_b, jblock, m->T, m->KL);
    pl.ns_s = ns_s;
    pl.ns_b = ns_b;
    return 0;
}

cudaError_t launch_split_tables(mp_mesh *m)
{
    SplitPlan &pl = m->plan;
    {
        const long long n = std::max<long long>((long long)pl.n_kc * pl.Npad * proj::BK, pl.Npad);
        k_tab_proj<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_Iph, m->n_p, m->P, pl.Npad, pl.n_kc,
                                                                       m->d_tabB, m->d_colsum);
    }
    {
        const long long n = (long long)pl.n_nc * (pl.Kpad / 16) * pl.NC * 16;
        k_tab_synth<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_Iphc, m->n_p, m->P, pl.Kpad, pl.NC,
                                                                        pl.n_nc, m->d_tabT);
    }
    {
        const long long n = (long long)m->T * m->n_t;
        k_tab_theta32<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_Ith, m->d_dmu, m->n_t, m->T,
                                                                          m->d_IthT32, m->d_Itc32);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (pl.a_terms == 2)
        return set_smem_attrs<2, 3>(pl.proj_smem, pl.synth_smem);
    return set_smem_attrs<3, 6>(pl.proj_smem, pl.synth_smem);
}

cudaError_t launch_split_project(mp_mesh *m, const double *rho)
{
    (void)rho;
    const SplitPlan &pl = m->plan;
    ProjParams prm;
    prm.tabB = m->d_tabB;
    prm.colsum = m->d_colsum;
    prm.F = m->d_F32;
    prm.err = m->d_err;
    prm.R = m->R;
    prm.n_p = m->n_p;
    prm.n_kc = pl.n_kc;
    prm.Npad = pl.Npad;
    prm.n_tiles = (int)((m->R + kBM - 1) / kBM);
    prm.ns_s = pl.ns_s;
    prm.ns_o = 2;
    prm.bchunk = (uint32_t)(3 * pl.Npad * proj::BK * 2);
    const int grid = std::min(prm.n_tiles, pl.proj_ctas);
    cudaEvent_t ev;
    prof_begin(m, "split_phi_project_tc", &ev);
    if (pl.a_terms == 2)
        k_proj_tc<2, 3><<<grid, kThreads, pl.proj_smem, m->stream>>>(m->tm_rho, prm);
    else
        k_proj_tc<3, 6><<<grid, kThreads, pl.proj_smem, m->stream>>>(m->tm_rho, prm);
    prof_end(m, "split_phi_project_tc", ev);
    return cudaGetLastError();
}

cudaError_t launch_split_synth(mp_mesh *m, double *phi)
{
    (void)phi;
    const SplitPlan &pl = m->plan;
    SynthParams prm;
    prm.tabT = m->d_tabT;
    prm.C32 = m->d_C32;
    prm.Itc = m->d_Itc32;
    prm.err = m->d_err;
    prm.R = m->R;
    prm.n_r = m->n_r;
    prm.n_t = m->n_t;
    prm.L = m->L;
    prm.KL = m->KL;
    prm.T = m->T;
    prm.P = m->P;
    prm.Kpad = pl.Kpad;
    prm.NC = pl.NC;
    prm.n_nc = pl.n_nc;
    prm.ns_b = pl.ns_b;
    prm.jblock = pl.jblock;
    if (pl.jblock) {
        const int SB = kBM / synth::JB;
        prm.n_ib = (m->n_r + SB - 1) / SB;
        prm.n_items = prm.n_ib * (m->n_t / synth::JB);
    } else {
        prm.n_ib = 0;
        prm.n_items = (int)((m->R + kBM - 1) / kBM);
    }
    prm.bchunk = (uint32_t)(3 * pl.NC * 32);
    const int grid = std::min(prm.n_items, pl.synth_ctas);
    cudaEvent_t ev;
    prof_begin(m, "split_synth_tc", &ev);
    if (pl.a_terms == 2)
        k_synth_tc<2, 3><<<grid, kThreads, pl.synth_smem, m->stream>>>(m->tm_phi, prm);
    else
        k_synth_tc<3, 6><<<grid, kThreads, pl.synth_smem, m->stream>>>(m->tm_phi, prm);
    prof_end(m, "split_synth_tc", ev);
    return cudaGetLastError();
}

}  // namespace mp
