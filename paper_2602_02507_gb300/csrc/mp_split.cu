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
// Roles per CTA (persistent, one CTA per SM): warp 0 issues the TMA / bulk copies
// of the streamed operand (the projection's table chunks come from warp 2),
// warp 1 owns tensor memory and issues the MMAs, the other warps convert and
// run the epilogues.  Every mbarrier wait is bounded (ptx.cuh).
#include <cstdio>

#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

constexpr int kBM = 128;      // rows per tile (UMMA M)
constexpr unsigned kFull = 0xFFFFFFFFu;

// bf16 product terms (a_term, b_term) accumulated per K step.
__constant__ int c_prod_a[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_prod_b[6] = {0, 1, 0, 2, 1, 0};


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

// Chunk order of a tile: a rotation by a tile-dependent offset, so that the SMs
// streaming different tiles address different parts of their rows at any moment
// (a common order sends every SM's requests to the same few memory channels).
__device__ __forceinline__ int rotated_chunk(int it, int tile, int n)
{
    int k = it + (int)(((unsigned)tile * 5u) % (unsigned)n);
    return k >= n ? k - n : k;
}

struct ProjParams {
    const uint8_t *tabB;   // [n_kc][3][Npad x 32] bf16, canonical layout
    const float *colsum;   // [Npad]
    const double *rho;     // [R][n_p], read directly only for the row reference values
    float *F;              // [n_r][P][ldF]: per shell, the P columns as rows of polar cells
    int *err;
    long long R;
    int n_p, n_kc, Npad, n_tiles, ns_s, ns_o;
    int n_t, P, ldF;
    int nacc;              // tensor-memory accumulators per tile (K chunks dealt round-robin)
    int b_resident;        // 1: every table chunk stays in shared memory for the whole launch
    int ns_b;              // table ring slots (when not resident)
    uint32_t bchunk;       // bytes of one B chunk in the table (3 terms)
    uint32_t bload;        // bytes of the terms the products read (a prefix of the chunk)
};

// Converter warps (warps 3 ..): two groups of kGroupWarps; group g converts the chunks
// whose CTA-wide sequence number c has c % 2 == g, so that each SM sub-partition holds
// four converter warps (their integer conversion chains hide each other's latency).
constexpr int kGroupWarps = 8;
constexpr int kProjConvWarps = 2 * kGroupWarps;
constexpr int kProjThreads = (3 + kProjConvWarps) * 32;

template <int A_TERMS, int NPROD>
__global__ void __launch_bounds__(kProjThreads, 1) k_proj_tc(const __grid_constant__ CUtensorMap tmS,
                                                             const ProjParams prm)
{
    using namespace proj;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS_S = prm.ns_s, NS_O = prm.ns_o, NS_B = prm.ns_b;
    uint8_t *sS = smem;
    uint8_t *sB = sS + (size_t)NS_S * S_BYTES;                        // table: n_kc chunks or NS_B slots
    uint8_t *sA = sB + (size_t)(prm.b_resident ? prm.n_kc : NS_B) * prm.bload;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + (size_t)NS_O * A_TERMS * A_TERM_BYTES);
    uint64_t *s_full = bars, *s_empty = bars + NS_S;
    uint64_t *b_full = bars + 2 * NS_S, *b_empty = b_full + NS_B;
    uint64_t *o_full = b_empty + NS_B, *o_empty = o_full + NS_O;
    uint64_t *acc_full = o_empty + NS_O, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Npad = prm.Npad;
    // per tile buffer, nacc accumulators of Npad columns: chunk it of a tile accumulates into
    // accumulator it % nacc, which shortens every float32 accumulation chain in the tensor core
    // nacc-fold (the epilogue adds the partials)
    const int nacc = prm.nacc;
    const uint32_t ncols = tmem_ncols_for(2 * nacc * Npad);
    const uint32_t acc_stride = ncols / 2;  // tile buffers at power-of-two column offsets

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS_S; ++s) {
            mbar_init(smem_u32(&s_full[s]), 1);
            mbar_init(smem_u32(&s_empty[s]), kGroupWarps);  // density stages: free once converted
        }
        for (int s = 0; s < NS_B; ++s) {
            mbar_init(smem_u32(&b_full[s]), 1);
            mbar_init(smem_u32(&b_empty[s]), 1);            // table stages: free once the MMAs read them
        }
        for (int o = 0; o < NS_O; ++o) {
            mbar_init(smem_u32(&o_full[o]), kGroupWarps);
            mbar_init(smem_u32(&o_empty[o]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kProjConvWarps);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        fence_mbar_init();
        if (prm.b_resident && (int)blockIdx.x < prm.n_tiles) {
            // the whole (static) table once, ahead of the wait for the previous kernel
            mbar_arrive_expect_tx(smem_u32(&b_full[0]), (uint32_t)prm.n_kc * prm.bload);
            for (int kc = 0; kc < prm.n_kc; ++kc)
                bulk_load(smem_u32(sB + (size_t)kc * prm.bload), prm.tabB + (size_t)kc * prm.bchunk, prm.bload,
                          smem_u32(&b_full[0]));
        }
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_holder), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    // barrier set-up, tensor memory and the table copy overlap the previous kernel's tail;
    // the density and the outputs are touched only after the previous kernel has completed
    pdl_trigger();
    pdl_wait();

    if (warp == 0) {
        // ---------------- density producer: lane 0 streams the two TMA boxes of rho per chunk
        if (lane == 0) {
            tma_prefetch_desc(&tmS);
            // rho is read once per solve: its lines go first, ahead of F, tables and moments
            const uint64_t l2_first = l2_evict_first_policy();
            Ring rs;
            int issued = 0;
            for (int tile = blockIdx.x; tile < prm.n_tiles && !*abort_flag; tile += gridDim.x) {
                for (int it = 0; it < prm.n_kc; ++it, rs.next(NS_S)) {
                    const int kc = rotated_chunk(it, tile, prm.n_kc);
                    if (!mbar_wait(smem_u32(&s_empty[rs.idx]), rs.phase ^ 1, abort_flag, prm.err)) break;
                    const uint32_t fb = smem_u32(&s_full[rs.idx]);
                    const bool two = kc * BK + 16 < prm.n_p;  // the second box holds cells
                    mbar_arrive_expect_tx(fb, two ? S_BYTES : BOX_BYTES);
                    const uint32_t dst = smem_u32(sS + (size_t)rs.idx * S_BYTES);
                    tma_load_2d_hint(dst, &tmS, fb, kc * BK, tile * kBM, l2_first);
                    if (two) tma_load_2d_hint(dst + BOX_BYTES, &tmS, fb, kc * BK + 16, tile * kBM, l2_first);
                    ++issued;
                }
            }
            // Every copy this thread issued has landed before the CTA can exit (another role may
            // abort after this loop ends; without an abort the phases are long complete).
            drain_ring(s_full, rs, NS_S, issued);
            if (prm.b_resident && (int)blockIdx.x < prm.n_tiles) {
                const long long t0 = clock64();
                while (!mbar_try_wait(smem_u32(&b_full[0]), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
                }
            }
        }
    } else if (warp == 2) {
        // ---------------- table producer (when the table is not resident): the table chunks on a
        // ring of their own, so that a shallow table ring does not hold back the density
        // prefetch.  A warp of its own: beside the density producer in one warp, each lane's
        // blocking barrier waits held up the other's copies (1567 -> 1525 us per launch at
        // 2048 x 512 x 1024 cells, l_max = 64)
        if (lane == 0 && !prm.b_resident) {
            Ring rb;
            int issued_b = 0;
            for (int tile = blockIdx.x; tile < prm.n_tiles && !*abort_flag; tile += gridDim.x) {
                for (int it = 0; it < prm.n_kc; ++it, rb.next(NS_B)) {
                    const int kc = rotated_chunk(it, tile, prm.n_kc);
                    if (!mbar_wait(smem_u32(&b_empty[rb.idx]), rb.phase ^ 1, abort_flag, prm.err)) break;
                    const uint32_t bb = smem_u32(&b_full[rb.idx]);
                    mbar_arrive_expect_tx(bb, prm.bload);
                    bulk_load(smem_u32(sB + (size_t)rb.idx * prm.bload), prm.tabB + (size_t)kc * prm.bchunk,
                              prm.bload, bb);
                    ++issued_b;
                }
            }
            drain_ring(b_full, rb, NS_B, issued_b);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kBM, Npad);
            const uint32_t b_term = (uint32_t)Npad * (BK * 2);
            Ring ro, rb;
            int lt = 0;
            bool ok = true;
            if (prm.b_resident && (int)blockIdx.x < prm.n_tiles) ok = mbar_wait(smem_u32(&b_full[0]), 0, abort_flag, prm.err);
            for (int tile = blockIdx.x; tile < prm.n_tiles && ok; tile += gridDim.x, ++lt) {
                const int b = lt & 1;
                ok = mbar_wait(smem_u32(&acc_empty[b]), ((lt >> 1) & 1) ^ 1, abort_flag, prm.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_buf = tmem_base + (uint32_t)b * acc_stride;
                for (int it = 0; it < prm.n_kc; ++it, ro.next(NS_O)) {
                    const uint32_t d_tmem = d_buf + (uint32_t)((it % nacc) * Npad);
                    ok = mbar_wait(smem_u32(&o_full[ro.idx]), ro.phase, abort_flag, prm.err) &&
                         (prm.b_resident || mbar_wait(smem_u32(&b_full[rb.idx]), rb.phase, abort_flag, prm.err));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(sA + (size_t)ro.idx * A_TERMS * A_TERM_BYTES);
                    const int bslot = prm.b_resident ? rotated_chunk(it, tile, prm.n_kc) : rb.idx;
                    const uint32_t b_base = smem_u32(sB + (size_t)bslot * prm.bload);
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
                        for (int pi = 0; pi < NPROD; ++pi) {
                            const uint64_t ad =
                                sdesc_noswizzle(a_base + c_prod_a[pi] * A_TERM_BYTES + ks * 256, 128, SBO);
                            const uint64_t bd = sdesc_noswizzle(b_base + c_prod_b[pi] * b_term + ks * 256, 128, SBO);
                            umma_bf16(d_tmem, ad, bd, idesc, (it >= nacc) || ((ks | pi) != 0));
                        }
                    }
                    umma_commit(smem_u32(&o_empty[ro.idx]));
                    if (!prm.b_resident) {
                        umma_commit(smem_u32(&b_empty[rb.idx]));
                        rb.next(NS_B);
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
        // ---------------- converters + epilogue
        const int cw = warp - 3, grp = cw / kGroupWarps, qd = warp & 3, half = (cw >> 2) & 1;
        const int row = qd * 32 + lane;
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        int lt = 0;
        // this group converts the chunks c = grp, grp + 2, ... of the CTA-wide sequence (the
        // producer's and the MMA's order): its ring positions advance two slots per own chunk
        Ring rs, ro;
        if (grp) {
            rs.next(NS_S);
            ro.next(NS_O);
        }
        int par = 0;  // parity of the CTA-wide chunk sequence number
        float sref = 0.0f;
        uint32_t efmax = 0;  // largest float64 exponent field seen (flags values beyond float32)
        bool ok = true;

        // The accumulator of a finished tile: F = D + sref colsum, stored per shell as rows of
        // polar cells (lanes hold consecutive cells: each store is coalesced); column groups
        // split four ways.  A tile's epilogue runs in steps of one column group, between the
        // own chunks of the next tile (from its second on, when the tile's last MMAs have
        // completed), so that the converters never leave the MMAs and the density ring idle
        // for a whole epilogue; what is left runs at the end of that tile.  Measured on GB300
        // at 2048 x 512 x 1024 cells, l_max = 64: 1537 -> 1447 us per launch against the
        // whole epilogue after each tile.
        struct {
            int tile = -1, lt = 0, cg = 0;
            float sr = 0.0f;
            bool ready = false;  // the tile's accumulator is complete
        } ep;
        const int ngroups = Npad / 8;
        auto ep_more = [&]() { return ep.cg < ngroups && ep.cg * 8 < prm.P; };
        auto ep_step = [&]() -> bool {
            if (ep.tile < 0) return true;
            const int b = ep.lt & 1;
            if (!ep.ready) {
                // also before a warp with no column group arrives: an arrival on acc_empty may
                // only follow the completion of this tile's MMAs, which follow every warp's
                // arrival for the buffer's previous tile
                if (!warp_all(mbar_wait(smem_u32(&acc_full[b]), (ep.lt >> 1) & 1, abort_flag, prm.err))) return false;
                tc_fence_after();
                ep.ready = true;
            }
            if (ep_more()) {
                const long long grow = (long long)ep.tile * kBM + row;
                const long long ish = grow / prm.n_t;
                float *fdst = prm.F + (size_t)ish * prm.P * prm.ldF + (grow - ish * prm.n_t);
                const int cg = ep.cg;
                const uint32_t col = tmem_base + lane_base + (uint32_t)b * acc_stride + (uint32_t)(cg * 8);
                // one accumulator at a time: these steps sit inside the conversion loop, whose
                // registers they must not crowd out
                float acc[8];
                {
                    uint32_t v[8];
                    tmem_ld8(col, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[e] = __uint_as_float(v[e]);
                    for (int s = 1; s < nacc; ++s) {
                        tmem_ld8(col + (uint32_t)(s * Npad), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 8; ++e) acc[e] += __uint_as_float(v[e]);
                    }
                }
                if (grow < prm.R) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int p = cg * 8 + e;
                        if (p < prm.P) fdst[(size_t)p * prm.ldF] = fmaf(ep.sr, prm.colsum[p], acc[e]);
                    }
                }
                ep.cg += 4;
            }
            if (!ep_more()) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
                ep.tile = -1;
            }
            return true;
        };
        auto ep_finish = [&]() -> bool {
            while (ep.tile >= 0)
                if (!ep_step()) return false;
            return true;
        };

        // this thread converts cells [16 half, 16 half + 16) of its group's stages: box `half`
        // reference value of a row: its first cell, read directly (both groups need it); the
        // next tile's is requested one tile ahead, so its HBM latency hides behind this tile
        auto load_ref = [&](int tile) -> uint2 {
            uint2 v = make_uint2(0u, 0u);
            const long long grow = (long long)tile * kBM + row;
            if (tile < prm.n_tiles && grow < prm.R) v = __ldg(reinterpret_cast<const uint2 *>(prm.rho + grow * prm.n_p));
            return v;
        };
        uint2 ref_next = load_ref(blockIdx.x);
        for (int tile = blockIdx.x; tile < prm.n_tiles && ok; tile += gridDim.x, ++lt) {
            {
                uint32_t e0;
                sref = f64w_to_f32_fast(ref_next.x, ref_next.y, e0);
                ref_next = load_ref(tile + gridDim.x);
            }
            const int rot = rotated_chunk(0, tile, prm.n_kc);
            int own = 0;  // own chunks of this tile so far
            for (int it = 0; it < prm.n_kc; ++it, par ^= 1) {
                if (par != grp) continue;
                const int kc = (it + rot >= prm.n_kc) ? it + rot - prm.n_kc : it + rot;
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
                const uint8_t *srow = sS + (size_t)sidx * S_BYTES + half * BOX_BYTES + row * 128;
                const int kfirst = kc * BK + half * 16;           // first cell of this thread's box
                const bool full = kfirst + 16 <= prm.n_p;         // warp-uniform
                uint32_t w0[8], w1[8], w2[8];
                // the deviations' bf16 terms of one pair of cells (packed float32 pairs)
                auto split_pair = [&](int cc, float2 x) {
                    const uint32_t t0 = pack_bf16x2(x.x, x.y);
                    const float2 r = sub_f32x2(x, make_float2(bf16lo_to_f32(t0), bf16hi_to_f32(t0)));
                    const uint32_t t1 = pack_bf16x2(r.x, r.y);
                    w0[cc] = t0;
                    w1[cc] = t1;
                    if (A_TERMS == 3) {
                        const float2 r2 = sub_f32x2(r, make_float2(bf16lo_to_f32(t1), bf16hi_to_f32(t1)));
                        w2[cc] = pack_bf16x2(r2.x, r2.y);
                    }
                };
                const float2 sref2 = make_float2(sref, sref);
                // Fast path (every magnitude in float32's normal range, the common case): the
                // conversion without per-value selects.  Two SWAR subtractions per pair of
                // values test the upper halves of their high words (exponent and four mantissa
                // bits) against 2^-126 (0x3810) and 2^128 (0x47F0); a value below the first, or
                // at or above the second (an infinity or a nan too), sends the chunk through the
                // checked conversion again, which zeroes the small ones and records the
                // exponent of the large ones for the report at the end.
                uint32_t bad = 0;  // bit 15 or 31: a magnitude outside [2^-126, 2^128)
                if (full) {
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(srow + ((cc ^ (row & 7)) << 4));
                        const uint32_t hh = __byte_perm(v.y, v.w, 0x7632) | 0x80008000u;
                        bad |= ~(hh - 0x38103810u) | (hh - 0x47F047F0u);
                        split_pair(cc, sub_f32x2(make_float2(f64w_to_f32_inrange(v.x, v.y),
                                                             f64w_to_f32_inrange(v.z, v.w)), sref2));
                    }
                }
                if (!full || (bad & 0x80008000u)) {
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(srow + ((cc ^ (row & 7)) << 4));
                        uint32_t e0, e1;
                        float x0 = f64w_to_f32_fast(v.x, v.y, e0) - sref;
                        float x1 = f64w_to_f32_fast(v.z, v.w, e1) - sref;
                        if (!full) {
                            // cells past the last azimuthal cell hold no data: zero deviation
                            const bool in0 = kfirst + 2 * cc < prm.n_p, in1 = kfirst + 2 * cc + 1 < prm.n_p;
                            x0 = in0 ? x0 : 0.0f;
                            x1 = in1 ? x1 : 0.0f;
                            e0 = in0 ? e0 : 0u;
                            e1 = in1 ? e1 : 0u;
                        }
                        efmax = max(efmax, max(e0, e1));
                        split_pair(cc, make_float2(x0, x1));
                    }
                }
                // K groups 2 half and 2 half + 1 of the [128 x 32] A tile, each term
                uint8_t *adst = sA + (size_t)oidx * A_TERMS * A_TERM_BYTES + (row >> 3) * SBO + half * 256 +
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
                    mbar_arrive(smem_u32(&s_empty[sidx]));
                    mbar_arrive(smem_u32(&o_full[oidx]));
                }
                if (own++ >= 1) {
                    ok = ep_step();
                    if (!ok) break;
                }
            }
            if (!ok) break;
            ok = ep_finish();
            if (!ok) break;
            ep.tile = tile;
            ep.lt = lt;
            ep.sr = sref;
            ep.cg = 2 * grp + half;
            ep.ready = false;
        }
        if (ok) ep_finish();
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
// (d) reconstruction, part 1: theta synthesis on CUDA cores
//   G[row][p] = sum_{l >= m(p)} (Ith[t(l,m)][j] / dmu_j) C[i][l^2 + p]
// written as the bf16 terms of the phi-synthesis A operand -- already in the
// canonical K-major layout of 128-row tiles (K = p - 1, p = 1 .. 2L) -- plus the
// m = 0 column G[row][0] in float32.  One block per (shell, 256 polar cells);
// the shell's coefficient row sits in shared memory, the table is read through
// L1 (coalesced along the polar cells).
// ----------------------------------------------------------------------------
// Register-tiled theta synthesis for n_t % 4 == 0 with the table Itc [T][n_t]
// resident in shared memory (persistent blocks walk the shells).  Thread
// (qd, g): polar cells j = 4 qd .. 4 qd + 3 and, for g < Kpad/8, the eight K
// columns p = 8 g + 1 .. 8 g + 8 (m = 4 g + 1 .. 4 g + 4, cos and sin); thread
// g = Kpad/8 forms the m = 0 column.  Per (l, m) one float4 table read feeds
// eight multiply-adds.
// Persistent form (one block per SM): the table Itc [T][ldF] (rows padded with
// zeros to ldF cells) arrives once by bulk copy and the block takes kGsS shells
// per pass.  Work unit u of a shell holds the orders m = u and m = L + 1 - u
// (u = 1 .. ceil(L/2); unit 0 is m = 0), so that every unit sums L + 1 terms
// per output pair and the warps finish together.  Lane t of a unit's warp forms
// four consecutive polar cells (one float4 table read feeds eight
// multiply-adds).  G collects in shared memory column-major ([K][ldF]) and
// leaves in a second pass as the bf16 terms of the canonical K-major MMA layout
// (16-byte stores, coalesced); the m = 0 column leaves as float32.  The next
// pass's coefficients are read into registers during the output pass.
constexpr int kGsS = 2;   // shells per pass
constexpr int kGsPre = 4; // coefficient registers per thread (kGsS * KL <= kGsPre * threads)

template <int A_TERMS>
__global__ void __launch_bounds__(1024, 1) k_gsynth_pipe(const float *__restrict__ C32, const float *__restrict__ Itc,
                                                         const float2 *__restrict__ C0, const float2 *__restrict__ Itc0,
                                                         uint8_t *__restrict__ Aop, float *__restrict__ G0, int *err,
                                                         int n_r, int n_t, int L, int KL, int Kpad, int ldF,
                                                         uint32_t tab_bytes)
{
    extern __shared__ __align__(16) uint8_t smem_gp[];
    float *sI = reinterpret_cast<float *>(smem_gp);                              // [T][ldF]
    float *sG = reinterpret_cast<float *>(smem_gp + tab_bytes);                  // [kGsS][Kpad][ldF]
    float *sC = sG + (size_t)kGsS * Kpad * ldF;                                  // [kGsS][KL]
    float2 *sT0 = reinterpret_cast<float2 *>(sC + (((size_t)kGsS * KL + 1) & ~(size_t)1));  // [L+1][n_t]
    float2 *sC0 = sT0 + (size_t)(L + 1) * n_t;                                   // [kGsS][L+1]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sC0 + (size_t)kGsS * (L + 1));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bar + 1);
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) {
        mbar_init(smem_u32(bar), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(smem_u32(bar), tab_bytes);
        bulk_load(smem_u32(sI), Itc, tab_bytes, smem_u32(bar));
    }
    for (int e = tid; e < (L + 1) * n_t; e += nthr) sT0[e] = Itc0[e];  // static table
    // the table copies overlap the previous kernel's tail; coefficients only after it completed
    pdl_trigger();
    pdl_wait();
    const int U = (L + 1) / 2;          // work units (order pairs, m >= 1) per group of 128 polar cells
    const int nq = (n_t + 3) / 4;       // float4 units of polar cells
    const int NJ = (nq + 31) / 32;
    const int n_work = kGsS * NJ * U * 32;
    const int ngk = Kpad / 8;
    const int n_out = kGsS * n_t * ngk;
    const int n_cf = kGsS * KL;
    const size_t a_term_bytes = (size_t)128 * Kpad * 2;
    const int n_pass = (n_r + kGsS - 1) / kGsS;
    // K columns past 2L never receive a term: zero once
    for (int e = tid; e < kGsS * (Kpad - 2 * L) * ldF; e += nthr) {
        const int kk = 2 * L + (e / ldF) % (Kpad - 2 * L), sh = e / ((Kpad - 2 * L) * ldF);
        sG[((size_t)sh * Kpad + kk) * ldF + e % ldF] = 0.0f;
    }
    float cv[kGsPre];
    float2 cv0 = make_float2(0.f, 0.f);  // thread e < kGsS (L+1): m = 0 coefficient pair
    auto load_coefficients = [&](int pass) {
#pragma unroll
        for (int k = 0; k < kGsPre; ++k) {
            const int e = tid + k * nthr;
            if (e < n_cf) {
                const int i = pass * kGsS + e / KL;
                cv[k] = (i < n_r) ? __ldg(C32 + (size_t)i * KL + e % KL) : 0.0f;
            }
        }
        if (tid < kGsS * (L + 1)) {
            const int i = pass * kGsS + tid / (L + 1);
            cv0 = (i < n_r) ? C0[(size_t)i * (L + 1) + tid % (L + 1)] : make_float2(0.f, 0.f);
        }
    };
    if ((int)blockIdx.x < n_pass) load_coefficients(blockIdx.x);
    const bool ok = mbar_wait(smem_u32(bar), 0, abort_flag, err);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(bar), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
            }
        }
        return;
    }
    // compute-phase work item w = tid + r nthr: (lane, unit u, 128-cell group jg, shell slot sh)
    auto compute = [&](int pass, int w) {
        const int lane = w & 31;
        int rest = w >> 5;
        const int u = 1 + rest % U;
        rest /= U;
        const int jg = rest % NJ, sh = rest / NJ;
        const int i = pass * kGsS + sh;
        const int uq = jg * 32 + lane;  // float4 unit of polar cells
        if (i >= n_r || uq >= nq) return;
        const float *cf = sC + (size_t)sh * KL;
        float *gs = sG + (size_t)sh * Kpad * ldF;
        for (int h = 0; h < 2; ++h) {
            const int m = (h == 0) ? u : L + 1 - u;
            if (h == 1 && m <= u) break;  // odd L: the middle order stands alone
            float4 ac = make_float4(0.f, 0.f, 0.f, 0.f), as = make_float4(0.f, 0.f, 0.f, 0.f);
            const float *tr = sI + (size_t)tri(m, m) * ldF + 4 * uq;
            const float *cp = cf + m * m + 2 * m - 1;  // C[i][l^2 + 2m - 1] at l = m
            for (int l = m; l <= L; ++l) {
                const float cc = cp[0], cs = cp[1];
                cp += 2 * l + 1;                      // (l+1)^2 - l^2
                const float4 t = *reinterpret_cast<const float4 *>(tr);
                tr += (size_t)(l + 1) * ldF;          // tri(l + 1, m) = tri(l, m) + l + 1
                ac.x = fmaf(t.x, cc, ac.x);
                ac.y = fmaf(t.y, cc, ac.y);
                ac.z = fmaf(t.z, cc, ac.z);
                ac.w = fmaf(t.w, cc, ac.w);
                as.x = fmaf(t.x, cs, as.x);
                as.y = fmaf(t.y, cs, as.y);
                as.z = fmaf(t.z, cs, as.z);
                as.w = fmaf(t.w, cs, as.w);
            }
            *reinterpret_cast<float4 *>(gs + (size_t)(2 * m - 2) * ldF + 4 * uq) = ac;
            *reinterpret_cast<float4 *>(gs + (size_t)(2 * m - 1) * ldF + 4 * uq) = as;
        }
    };
    // output-phase item o = tid + r nthr: polar cell j = o mod n_t, (shell slot, K group) = o div n_t,
    // advanced without divisions
    const int dj = nthr % n_t, dsg = nthr / n_t;
    const int j_first = tid % n_t, sg_first = tid / n_t;
    for (int pass = blockIdx.x; pass < n_pass; pass += gridDim.x) {
#pragma unroll
        for (int k = 0; k < kGsPre; ++k) {
            const int e = tid + k * nthr;
            if (e < n_cf) sC[e] = cv[k];
        }
        if (tid < kGsS * (L + 1)) sC0[tid] = cv0;
        __syncthreads();
        for (int w = tid; w < n_work; w += nthr) compute(pass, w);
        // the m = 0 column in double-float, one cell per thread
        for (int e = tid; e < kGsS * n_t; e += nthr) {
            const int sh = e / n_t, j = e - sh * n_t, i = pass * kGsS + sh;
            if (i < n_r)
                *reinterpret_cast<float2 *>(G0 + 2 * ((size_t)i * n_t + j)) =
                    g0_double_float(sT0 + j, n_t, sC0 + (size_t)sh * (L + 1), L);
        }
        __syncthreads();
        if (pass + (int)gridDim.x < n_pass) load_coefficients(pass + gridDim.x);
        int j = j_first, sg = sg_first;
        for (int o = tid; o < n_out; o += nthr) {
            int sh = 0, g = sg;
            while (g >= ngk) {
                g -= ngk;
                ++sh;
            }
            const int i = pass * kGsS + sh;
            if (i < n_r) {
                const float *gc = sG + ((size_t)sh * Kpad + 8 * g) * ldF + j;
                uint32_t w0[4], w1[4], w2[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float x0 = gc[(size_t)(2 * c) * ldF], x1 = gc[(size_t)(2 * c + 1) * ldF];
                    const uint32_t t0 = pack_bf16x2(x0, x1);
                    const float r0 = x0 - bf16lo_to_f32(t0), r1 = x1 - bf16hi_to_f32(t0);
                    const uint32_t t1 = pack_bf16x2(r0, r1);
                    w0[c] = t0;
                    w1[c] = t1;
                    if (A_TERMS == 3) w2[c] = pack_bf16x2(r0 - bf16lo_to_f32(t1), r1 - bf16hi_to_f32(t1));
                }
                const long long row = (long long)i * n_t + j;
                const int r = (int)(row & 127);
                uint8_t *dst = Aop + (size_t)(row >> 7) * A_TERMS * a_term_bytes + (size_t)(r >> 3) * (Kpad * 16) +
                               (r & 7) * 16 + g * 128;
                *reinterpret_cast<uint4 *>(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *reinterpret_cast<uint4 *>(dst + a_term_bytes) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                if (A_TERMS == 3)
                    *reinterpret_cast<uint4 *>(dst + 2 * a_term_bytes) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
            }
            j += dj;
            sg += dsg;
            if (j >= n_t) {
                j -= n_t;
                ++sg;
            }
        }
        __syncthreads();  // G columns and coefficients of this pass consumed
    }
}

// Theta synthesis for tables that exceed shared memory, one GEMM per order m:
//   G[i, j][p] = sum_{l = m..L} Itc[tri(l,m)][j] C32[i][l^2 + p],   p in {pc, ps},
// M = polar cells, N = shells (cos and sin together), K = degrees.  Block (128 polar
// cells, 64 shells, m) stages the table rows and the coefficients of K chunks of 32
// degrees in shared memory, the next chunk's loads in flight (registers) during the
// current chunk's arithmetic; thread (rg, cg) owns cells cg + 16 a (a < 8) and shells
// rg + 16 b (b < 4), cos and sin: 64 multiply-adds per 16 shared-memory reads.  The
// results leave as the bf16 terms of the canonical MMA layout ((cos, sin) pairs, 4 bytes
// per term); the m = 0 column (double-float) is shared by kGm0Parts blocks per tile and
// leaves as float32 (hi, lo) pairs.  K columns past 2L keep the zeros the buffer was
// created with.
constexpr int kGmCells = 128, kGmShells = 64, kGmK = 32, kGm0Parts = 4;

template <int A_TERMS>
__global__ void __launch_bounds__(256) k_gsynth_mgemm(const float *__restrict__ C32, const float *__restrict__ Itc,
                                                      const float2 *__restrict__ C0, const float2 *__restrict__ Itc0,
                                                      uint8_t *__restrict__ Aop, float *__restrict__ G0, int n_r,
                                                      int n_t, int L, int KL, int Kpad, int ldF)
{
    __shared__ __align__(16) float sT[kGmK][kGmCells + 4];
    __shared__ float sC[kGmK][2 * kGmShells + 1];
    pdl_wait();  // C32 comes from the previous kernel
    const int j0 = blockIdx.x * kGmCells, i0 = blockIdx.y * kGmShells, z = blockIdx.z;
    if (z < kGm0Parts) {
        // the m = 0 column in double-float (block-uniform branch), a quarter of the tile per block
        constexpr int per = kGmCells * kGmShells / kGm0Parts;
        for (int e = z * per + (int)threadIdx.x; e < (z + 1) * per; e += blockDim.x) {
            const int j = j0 + e % kGmCells, i = i0 + e / kGmCells;
            if (j < n_t && i < n_r)
                *reinterpret_cast<float2 *>(G0 + 2 * ((size_t)i * n_t + j)) =
                    g0_double_float(Itc0 + j, n_t, C0 + (size_t)i * (L + 1), L);
        }
        return;
    }
    const int m = z - kGm0Parts + 1;
    const int nl = L + 1 - m;
    const int pc = 2 * m - 1;
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    float gc[8][4], gs[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) gc[a][b] = gs[a][b] = 0.0f;
    // per chunk a thread moves 4 float4 of the table and 16 coefficients
    float4 pt[4];
    float pcf[16];
    auto load_chunk = [&](int l0) {
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const int e = tid + 256 * n, r = e >> 5, q = e & 31, j = j0 + 4 * q;
            pt[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l0 + r < nl && j < ldF) pt[n] = __ldg(reinterpret_cast<const float4 *>(Itc + (size_t)tri(m + l0 + r, m) * ldF + j));
        }
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            const int e = tid + 256 * n, r = e >> 7, col = e & 127;
            const int i = i0 + (col >> 1), sn = col & 1, l = m + l0 + r;
            pcf[n] = (l0 + r < nl && i < n_r) ? __ldg(C32 + (size_t)i * KL + l * l + pc + sn) : 0.0f;
        }
    };
    load_chunk(0);
    for (int l0 = 0; l0 < nl; l0 += kGmK) {
        __syncthreads();  // the previous chunk is consumed
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const int e = tid + 256 * n;
            *reinterpret_cast<float4 *>(&sT[e >> 5][4 * (e & 31)]) = pt[n];
        }
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            const int e = tid + 256 * n;
            sC[e >> 7][e & 127] = pcf[n];
        }
        __syncthreads();
        if (l0 + kGmK < nl) load_chunk(l0 + kGmK);
        const int kn = min(kGmK, nl - l0);
        for (int r = 0; r < kn; ++r) {
            float t[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) t[a] = sT[r][cg + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float cc = sC[r][2 * (rg + 16 * b)], cs = sC[r][2 * (rg + 16 * b) + 1];
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    gc[a][b] = fmaf(t[a], cc, gc[a][b]);
                    gs[a][b] = fmaf(t[a], cs, gs[a][b]);
                }
            }
        }
    }
    const size_t a_term_bytes = (size_t)128 * Kpad * 2;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int i = i0 + rg + 16 * b;
        if (i >= n_r) continue;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int j = j0 + cg + 16 * a;
            if (j >= n_t) continue;
            const long long row = (long long)i * n_t + j;
            const int k = 2 * m - 2;  // K column of the cos term; the sin term follows
            const int r = (int)(row & 127);
            uint8_t *dst = Aop + (size_t)(row >> 7) * A_TERMS * a_term_bytes + (size_t)(r >> 3) * (Kpad * 16) +
                           (size_t)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
            const float x0 = gc[a][b], x1 = gs[a][b];
            const uint32_t t0 = pack_bf16x2(x0, x1);
            const float r0 = x0 - bf16lo_to_f32(t0), r1 = x1 - bf16hi_to_f32(t0);
            const uint32_t t1 = pack_bf16x2(r0, r1);
            *reinterpret_cast<uint32_t *>(dst) = t0;
            *reinterpret_cast<uint32_t *>(dst + a_term_bytes) = t1;
            if (A_TERMS == 3)
                *reinterpret_cast<uint32_t *>(dst + 2 * a_term_bytes) =
                    pack_bf16x2(r0 - bf16lo_to_f32(t1), r1 - bf16hi_to_f32(t1));
        }
    }
}

// ----------------------------------------------------------------------------
// (d) reconstruction, part 2: phi synthesis on tcgen05
//   Phi[row][k] = G[row][0] + sum_{p>=1} G[row][p] Iph[p][k] / dphi_k
// Warp 0 bulk-copies each tile's A operand (+ its m = 0 column) into a 2-deep
// ring and the pre-split table (resident when it fits, else a ring); warp 1
// issues the MMAs into double-buffered [128 x NC] fp32 accumulators; warps
// 2..17 (four per tensor-memory lane quarter) drain the accumulators, add the
// m = 0 term, pack float64 with integer ops into swizzled staging boxes and
// write Phi with TMA stores.
// ----------------------------------------------------------------------------
namespace synth {
// TMA store boxes of [32 rows][16 float64] (128B swizzle) or [32 rows][8 float64] (64B swizzle)
__host__ __device__ constexpr int stg_bytes(int cols) { return 32 * cols * 8; }
constexpr int EPI_WARPS = 16;
constexpr int THREADS = (2 + EPI_WARPS) * 32;
}

struct SynthParams {
    const uint8_t *Aop;    // [tiles][A_TERMS][128 x Kpad] bf16, canonical layout
    const float *G0;       // [R]
    const uint8_t *tabT;   // [n_nc][Kpad/16][3][NC x 16] bf16, canonical layout
    int *err;
    long long R;
    int Kpad, NC, n_nc, n_tiles, ns_a, ns_b, stg_bufs, stg_cols;
    int b_resident;        // 1: every table chunk stays in shared memory for the whole launch
    uint32_t a_bytes;      // one tile's A operand (all terms)
    uint32_t bchunk;       // bytes of one B chunk in the table (3 terms)
    uint32_t bload;        // bytes of the terms the products read (a prefix of the chunk)
};

template <int A_TERMS, int NPROD>
__global__ void __launch_bounds__(synth::THREADS, 1)
    k_synth_tc(const __grid_constant__ CUtensorMap tmPhi, const SynthParams prm)
{
    using namespace synth;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS_A = prm.ns_a, NS_B = prm.ns_b, NSTG = prm.stg_bufs, STG_BYTES = stg_bytes(prm.stg_cols);
    const int Kpad = prm.Kpad, NC = prm.NC;
    const int nkk = Kpad / 16;
    const int n_chunks = prm.n_nc * nkk;
    // work units (tile, column chunk nc), dealt out round-robin: a tile's chunks may go to
    // different CTAs, each loading the tile's A operand, so that the last wave is a chunk
    // rather than a whole tile
    const int n_units = prm.n_tiles * prm.n_nc;
    const int b_slots = prm.b_resident ? n_chunks : NS_B;
    const uint32_t a_stage = prm.a_bytes + 1024;  // A operand terms + the tile's 128 m = 0 (hi, lo) pairs
    uint8_t *stg = smem;                                           // [16 warps][NSTG][STG_BYTES]
    uint8_t *sA = stg + (size_t)EPI_WARPS * NSTG * STG_BYTES;      // [NS_A][a_stage]
    uint8_t *sB = sA + (size_t)NS_A * a_stage;                     // [b_slots][bload]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)b_slots * prm.bload);
    uint64_t *a_full = bars, *a_empty = bars + NS_A;
    uint64_t *b_full = a_empty + NS_A, *b_empty = b_full + NS_B;
    uint64_t *acc_full = b_empty + NS_B, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_ncols_for(2 * NC);
    const uint32_t acc_stride = ncols / 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS_A; ++s) {
            mbar_init(smem_u32(&a_full[s]), 1);
            mbar_init(smem_u32(&a_empty[s]), 1 + EPI_WARPS);  // MMAs done and m = 0 values read
        }
        for (int s = 0; s < NS_B; ++s) {
            mbar_init(smem_u32(&b_full[s]), 1);
            mbar_init(smem_u32(&b_empty[s]), 1);
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
    // set-up (and, in the producer, the table copy) overlaps the previous kernel's tail; the
    // A tiles and the potential are touched only after it has completed
    pdl_trigger();
    if (warp != 0) pdl_wait();

    if (warp == 0) {
        // ---------------- producer: A tiles (+ m = 0 column) and table chunks
        if (lane == 0) {
            bool ok = true;
            if (prm.b_resident && blockIdx.x < n_units) {
                // the whole table once; b_full[0] completes when every chunk has landed
                mbar_arrive_expect_tx(smem_u32(&b_full[0]), (uint32_t)n_chunks * prm.bload);
                for (int c = 0; c < n_chunks; ++c)
                    bulk_load(smem_u32(sB + (size_t)c * prm.bload), prm.tabT + (size_t)c * prm.bchunk, prm.bload,
                              smem_u32(&b_full[0]));
            }
            pdl_wait();
            Ring ra, rb;
            int issued_a = 0, issued_b = 0;
            for (int unit = blockIdx.x; unit < n_units && ok; unit += gridDim.x, ra.next(NS_A)) {
                const int tile = unit / prm.n_nc, nc = unit - tile * prm.n_nc;
                ok = mbar_wait(smem_u32(&a_empty[ra.idx]), ra.phase ^ 1, abort_flag, prm.err);
                if (!ok) break;
                const uint32_t fb = smem_u32(&a_full[ra.idx]);
                uint8_t *dst = sA + (size_t)ra.idx * a_stage;
                mbar_arrive_expect_tx(fb, a_stage);
                bulk_load(smem_u32(dst), prm.Aop + (size_t)tile * prm.a_bytes, prm.a_bytes, fb);
                bulk_load(smem_u32(dst + prm.a_bytes), prm.G0 + (size_t)tile * 256, 1024, fb);
                ++issued_a;
                if (!prm.b_resident) {
                    for (int c = nc * nkk; c < (nc + 1) * nkk && ok; ++c, rb.next(NS_B)) {
                        ok = mbar_wait(smem_u32(&b_empty[rb.idx]), rb.phase ^ 1, abort_flag, prm.err);
                        if (!ok) break;
                        mbar_arrive_expect_tx(smem_u32(&b_full[rb.idx]), prm.bload);
                        bulk_load(smem_u32(sB + (size_t)rb.idx * prm.bload), prm.tabT + (size_t)c * prm.bchunk,
                                  prm.bload, smem_u32(&b_full[rb.idx]));
                        ++issued_b;
                    }
                }
            }
            // Every copy this thread issued has landed before the CTA can exit: another role may
            // abort after this loop ends, leaving stages nobody waits for.  In a run without an
            // abort these waits find the phases long complete.
            drain_ring(a_full, ra, NS_A, issued_a);
            if (prm.b_resident) {
                if (blockIdx.x < n_units) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(smem_u32(&b_full[0]), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
                    }
                }
            } else {
                drain_ring(b_full, rb, NS_B, issued_b);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kBM, NC);
            const uint32_t sbo_a = (uint32_t)Kpad * 16;
            const uint32_t a_term_bytes = (uint32_t)kBM * Kpad * 2;
            Ring ra, rb;
            uint32_t u = 0;
            bool ok = true;
            if (prm.b_resident && blockIdx.x < n_units) ok = mbar_wait(smem_u32(&b_full[0]), 0, abort_flag, prm.err);
            for (int unit = blockIdx.x; unit < n_units && ok; unit += gridDim.x, ra.next(NS_A)) {
                const int nc = unit % prm.n_nc;
                ok = mbar_wait(smem_u32(&a_full[ra.idx]), ra.phase, abort_flag, prm.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t a_base0 = smem_u32(sA + (size_t)ra.idx * a_stage);
                {
                    const int buf = u & 1;
                    ok = mbar_wait(smem_u32(&acc_empty[buf]), ((u >> 1) & 1) ^ 1, abort_flag, prm.err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)buf * acc_stride;
                    for (int kk = 0; kk < nkk; ++kk) {
                        uint32_t b_base;
                        if (prm.b_resident) {
                            b_base = smem_u32(sB + (size_t)(nc * nkk + kk) * prm.bload);
                        } else {
                            ok = mbar_wait(smem_u32(&b_full[rb.idx]), rb.phase, abort_flag, prm.err);
                            if (!ok) break;
                            tc_fence_after();
                            b_base = smem_u32(sB + (size_t)rb.idx * prm.bload);
                        }
                        const uint32_t a_base = a_base0 + (uint32_t)(kk * 256);
#pragma unroll
                        for (int pi = 0; pi < NPROD; ++pi) {
                            const uint64_t ad = sdesc_noswizzle(a_base + c_prod_a[pi] * a_term_bytes, 128, sbo_a);
                            const uint64_t bd = sdesc_noswizzle(b_base + (uint32_t)(c_prod_b[pi] * NC * 32), 128, 256);
                            umma_bf16(d_tmem, ad, bd, idesc, (kk | pi) != 0);
                        }
                        if (!prm.b_resident) {
                            umma_commit(smem_u32(&b_empty[rb.idx]));
                            rb.next(NS_B);
                        }
                    }
                    if (!ok) break;
                    umma_commit(smem_u32(&acc_full[buf]));
                    ++u;
                }
                if (!ok) break;
                umma_commit(smem_u32(&a_empty[ra.idx]));
            }
            umma_commit(smem_u32(drain));
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(drain), 0) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
            }
        }
    } else {
        // ---------------- epilogue: accumulators -> Phi
        const int cw = warp - 2, qd = warp & 3, quarter = cw >> 2;
        const int row = qd * 32 + lane;
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        // Phi is written once per solve: its lines leave L2 first (written back now, not
        // during the next solve's density stream)
        const uint64_t l2_first = l2_evict_first_policy();
        Ring ra;
        uint32_t u = 0;
        int cs = 0;  // staging box of this warp in use
        bool ok = true;
        const int nmine = (NC / 16 - quarter + 3) / 4;  // chunks quarter, quarter + 4, ...
        for (int unit = blockIdx.x; unit < n_units && ok; unit += gridDim.x, ra.next(NS_A)) {
            const int tile = unit / prm.n_nc, nc = unit - tile * prm.n_nc;
            const int rot = nmine > 0 ? rotated_chunk(0, tile, nmine) : 0;
            ok = warp_all(mbar_wait(smem_u32(&a_full[ra.idx]), ra.phase, abort_flag, prm.err));
            if (!ok) break;
            const float2 g0 = reinterpret_cast<const float2 *>(sA + (size_t)ra.idx * a_stage + prm.a_bytes)[row];
            // the stage is refilled by the bulk-copy engine (the async proxy): the m = 0 values just
            // read must be ordered before that write, or a late read returns the next unit's values
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&a_empty[ra.idx]));
            const long long box_row = (long long)tile * kBM + qd * 32;
            const bool box_valid = box_row < prm.R;
            {
                const int buf = u & 1;
                ok = warp_all(mbar_wait(smem_u32(&acc_full[buf]), (u >> 1) & 1, abort_flag, prm.err));
                if (!ok) break;
                tc_fence_after();
                const uint32_t tcol = tmem_base + lane_base + (uint32_t)buf * acc_stride;
                for (int it = 0; it < nmine; ++it) {
                    const int ch = quarter + 4 * ((it + rot >= nmine) ? it + rot - nmine : it + rot);
                    uint32_t v[16];
                    tmem_ld16(tcol + (uint32_t)(ch * 16), v);
                    tmem_ld_wait();
                    // one box of 16 columns or two of 8: with two or more staging boxes a warp
                    // fills one while the bulk-copy engine still reads another.  Phi = m >= 1 part
                    // + m = 0 column (low part first: one rounding of the sum).
                    auto next_box = [&]() -> uint8_t * {
                        uint8_t *st = stg + (size_t)(cw * NSTG + cs) * STG_BYTES;
                        if (++cs == NSTG) cs = 0;
                        if (lane == 0) {  // this box's last store has read it
                            if (NSTG >= 4)
                                bulk_wait_read_le3();
                            else if (NSTG > 1)
                                bulk_wait_read_le1();
                            else
                                bulk_wait_read_all();
                        }
                        __syncwarp();
                        return st;
                    };
                    auto store_box = [&](uint8_t *st, int col) {
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0 && box_valid) {
                            tma_store_2d_hint(&tmPhi, smem_u32(st), col, (int)box_row, l2_first);
                            bulk_commit();
                        }
                    };
                    if (prm.stg_cols == 16) {
                        // 128-byte swizzle: 16-byte piece e of row `lane` sits at e ^ (lane & 7)
                        uint8_t *st = next_box();
                        uint8_t *srow = st + lane * 128;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            uint32_t lo0, hi0, lo1, hi1;
                            f32_to_f64w_finite((__uint_as_float(v[2 * e]) + g0.y) + g0.x, lo0, hi0);
                            f32_to_f64w_finite((__uint_as_float(v[2 * e + 1]) + g0.y) + g0.x, lo1, hi1);
                            *reinterpret_cast<uint4 *>(srow + ((e ^ (lane & 7)) << 4)) = make_uint4(lo0, hi0, lo1, hi1);
                        }
                        store_box(st, nc * NC + ch * 16);
                    } else {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            // 64-byte swizzle: 16-byte piece e of row `lane` sits at e ^ ((lane >> 1) & 3)
                            uint8_t *st = next_box();
                            uint8_t *srow = st + lane * 64;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                uint32_t lo0, hi0, lo1, hi1;
                                f32_to_f64w_finite((__uint_as_float(v[8 * h + 2 * e]) + g0.y) + g0.x, lo0, hi0);
                                f32_to_f64w_finite((__uint_as_float(v[8 * h + 2 * e + 1]) + g0.y) + g0.x, lo1, hi1);
                                *reinterpret_cast<uint4 *>(srow + ((e ^ ((lane >> 1) & 3)) << 4)) =
                                    make_uint4(lo0, hi0, lo1, hi1);
                            }
                            store_box(st, nc * NC + ch * 16 + 8 * h);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
                ++u;
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

// float32 theta tables (rows of ldF cells): Ith32[t][j] = Ith[t][j], Itc[t][j] = Ith[t][j] / dmu_j
__global__ void k_tab_theta32(const double *__restrict__ Ith, const double *__restrict__ dmu, int n_t, int T, int ldF,
                              float *__restrict__ Ith32, float *__restrict__ Itc)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)T * n_t) return;
    const int t = (int)(idx / n_t), j = (int)(idx % n_t);
    const double v = Ith[idx];
    Ith32[(size_t)t * ldF + j] = (float)v;
    Itc[(size_t)t * ldF + j] = (float)(v / dmu[j]);
}

constexpr int kSmemLimit = 232448;  // 227 KB opt-in per block on sm_100-class parts

// theta table of the m = 0 column as (hi, lo) float pairs: Itc0[l][j] = Ith[tri(l,0)][j] / dmu_j
__global__ void k_tab_theta0(const double *__restrict__ Ith, const double *__restrict__ dmu, int n_t, int L,
                             float2 *__restrict__ Itc0)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (L + 1) * n_t) return;
    const int l = idx / n_t, j = idx % n_t;
    Itc0[idx] = f32_pair(Ith[(size_t)tri(l, 0) * n_t + j] / dmu[j]);
}

template <int A_TERMS, int NPROD>
cudaError_t set_smem_attrs()
{
    // the per-function limit is shared by every mesh: set it to the part's maximum once,
    // not to one mesh's need (a larger mesh created earlier would then fail to launch)
    cudaError_t e = cudaFuncSetAttribute(k_proj_tc<A_TERMS, NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_synth_tc<A_TERMS, NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

// B terms the products read: x3 uses b0 and b1, x6 also b2
int proj_b_terms(const SplitPlan &pl) { return pl.n_products == 3 ? 2 : 3; }

// The table ring (when the table is not resident) is as deep as the density ring: both
// loads of a chunk come from one thread, so a shallower table ring would cap the density
// prefetch depth.
int proj_smem_bytes(const SplitPlan &pl, int ns_s, int ns_o, int b_resident, int ns_b)
{
    const int bload = proj_b_terms(pl) * pl.Npad * proj::BK * 2;
    return 1024 + ns_s * proj::S_BYTES + (b_resident ? pl.n_kc : ns_b) * bload +
           ns_o * pl.a_terms * proj::A_TERM_BYTES + 512;
}

int synth_smem_bytes(const SplitPlan &pl, int ns_a, int b_slots, int stg_bufs, int stg_cols)
{
    const int bchunk = 3 * pl.NC * 32;
    const int a_stage = pl.a_terms * kBM * pl.Kpad * 2 + 1024;
    return 1024 + synth::EPI_WARPS * stg_bufs * synth::stg_bytes(stg_cols) + ns_a * a_stage + b_slots * bchunk + 512;
}


}  // namespace

namespace {

// Stage configurations of the phi synthesis: A-operand stages, table resident or its ring
// slots, staging boxes per epilogue warp and their columns (16: 128B swizzle, 8: 64B).
struct SynthCfg {
    int ns_a, resident, ns_b, stg, cols;
};
constexpr SynthCfg kSynthCfgs[] = {
    {2, 1, 0, 2, 16}, {2, 0, 3, 2, 16}, {2, 0, 2, 2, 16}, {1, 0, 2, 2, 16},  // 8 KB of staging a warp
    {2, 1, 0, 2, 8},  {2, 0, 3, 2, 8},  {2, 0, 2, 2, 8},  {1, 0, 2, 2, 8},   // 4 KB, double-buffered
    {2, 0, 2, 1, 16}, {2, 0, 2, 1, 8},  {1, 0, 2, 1, 16}, {1, 0, 2, 1, 8},   // one box
};

}  // namespace

int synth_cfg_count() { return (int)(sizeof(kSynthCfgs) / sizeof(kSynthCfgs[0])); }

bool synth_cfg_fits(const SplitPlan &pl, int k)
{
    if (k < 0 || k >= synth_cfg_count()) return false;
    const SynthCfg &c = kSynthCfgs[k];
    const int b_slots = c.resident ? pl.n_nc * (pl.Kpad / 16) : c.ns_b;
    return synth_smem_bytes(pl, c.ns_a, b_slots, c.stg, c.cols) <= kSmemLimit;
}

void synth_cfg_apply(SplitPlan &pl, int k)
{
    const SynthCfg &c = kSynthCfgs[k];
    const int b_slots = c.resident ? pl.n_nc * (pl.Kpad / 16) : c.ns_b;
    pl.synth_cfg = k;
    pl.ns_a = c.ns_a;
    pl.b_resident = c.resident;
    pl.ns_b = c.resident ? 1 : c.ns_b;
    pl.stg_bufs = c.stg;
    pl.stg_cols = c.cols;
    pl.synth_smem = synth_smem_bytes(pl, c.ns_a, b_slots, c.stg, c.cols);
}

// Preferred order of the synthesis stage configurations.  Where a tile's A operand is large
// (>= 48 KB: l_max >= 48), a second A stage comes first, so the next unit's operand arrives
// while the current one is multiplied; else the staging volume does.  Measured on GB300:
// 2048 x 512 x 1024 cells at l_max = 64 (66.5 KB A stages) ran the synthesis in 1414 us with
// two A stages beside one 8-column box a warp against 1553 us with one A stage beside two; a
// log-normal 1024 x 256 x 512 mesh at l_max = 32 (33.8 KB) in 176 us with one A stage beside
// two 16-column boxes against 189 us with four 8-column ones and 207 us with two A stages
// beside two 8-column boxes.
std::vector<int> synth_cfg_order(const SplitPlan &pl)
{
    const int a_stage = pl.a_terms * kBM * pl.Kpad * 2 + 1024;
    if (a_stage >= 48 * 1024) return {0, 1, 2, 4, 5, 6, 8, 9, 3, 7, 10, 11};
    return {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11};
}

// Chooses ring depths that fit shared memory; fills plan.* sizes.
int split_smem_limits(mp_mesh *m)
{
    SplitPlan &pl = m->plan;
    // projection: (density stages, A-operand stages, table ring slots) in order of
    // preference, the table resident when it fits beside them, else on a ring of its own
    // (its own producer thread: a shallower ring than the density's is fine).  The density and
    // A-operand depths are even: the two converter groups take alternate chunks, so with an
    // even depth each slot belongs to one group, and a group can never run a whole ring ahead
    // of the other (a parity wait on a slot two phases behind would pass at once)
    static const int kProjCfg[][3] = {{4, 2, 4}, {4, 2, 3}, {4, 2, 2}, {2, 2, 2}};
    int ns_s = 0, ns_o = 0, b_res = 0, ns_bp = 2;
    for (const auto &c : kProjCfg) {
        if (proj_smem_bytes(pl, c[0], c[1], 1, 0) <= kSmemLimit) {
            ns_s = c[0];
            ns_o = c[1];
            b_res = 1;
            ns_bp = c[2];
            break;
        }
        if (proj_smem_bytes(pl, c[0], c[1], 0, c[2]) <= kSmemLimit) {
            ns_s = c[0];
            ns_o = c[1];
            b_res = 0;
            ns_bp = c[2];
            break;
        }
    }
    if (ns_s == 0) return 1;
    // synthesis: the first stage configuration of the preferred order that fits
    bool found = false;
    for (int k : synth_cfg_order(pl)) {
        if (synth_cfg_fits(pl, k)) {
            synth_cfg_apply(pl, k);
            found = true;
            break;
        }
    }
    if (!found) return 2;
    pl.ns_s = ns_s;
    pl.ns_s_max = ns_s;
    pl.ns_o = ns_o;
    pl.proj_ns_b = ns_bp;
    pl.proj_b_resident = b_res;
    pl.proj_res_ok = proj_smem_bytes(pl, ns_s, ns_o, 1, 0) <= kSmemLimit;
    pl.proj_ring_ok = proj_smem_bytes(pl, ns_s, ns_o, 0, ns_bp) <= kSmemLimit;
    // the launch reserves the larger of the table modes that fit, so the tuner may switch them
    pl.proj_smem = std::max(pl.proj_res_ok ? proj_smem_bytes(pl, ns_s, ns_o, 1, 0) : 0,
                            pl.proj_ring_ok ? proj_smem_bytes(pl, ns_s, ns_o, 0, ns_bp) : 0);
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
        k_tab_theta32<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_Ith, m->d_dmu, m->n_t, m->T, pl.ldF,
                                                                          m->d_Ith32, m->d_Itc32);
        const int n0 = (m->L + 1) * m->n_t;
        k_tab_theta0<<<(n0 + 255) / 256, 256, 0, m->stream>>>(m->d_Ith, m->d_dmu, m->n_t, m->L, m->d_Itc0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (pl.a_terms == 2)
        return set_smem_attrs<2, 3>();
    return set_smem_attrs<3, 6>();
}

cudaError_t launch_split_project(mp_mesh *m, const double *rho)
{
    const SplitPlan &pl = m->plan;
    ProjParams prm;
    prm.tabB = m->d_tabB;
    prm.colsum = m->d_colsum;
    prm.rho = rho;
    prm.n_t = m->n_t;
    prm.P = m->P;
    prm.ldF = pl.ldF;
    prm.F = m->d_F32;
    prm.err = m->d_err;
    prm.R = m->R;
    prm.n_p = m->n_p;
    prm.n_kc = pl.n_kc;
    prm.Npad = pl.Npad;
    prm.n_tiles = (int)((m->R + kBM - 1) / kBM);
    prm.ns_s = pl.ns_s;
    prm.ns_o = pl.ns_o;
    if ((prm.ns_s & 1) || (prm.ns_o & 1) || prm.ns_s < 2 || prm.ns_o < 2) return cudaErrorInvalidValue;
    prm.bchunk = (uint32_t)(3 * pl.Npad * proj::BK * 2);
    prm.bload = (uint32_t)(proj_b_terms(pl) * pl.Npad * proj::BK * 2);
    prm.nacc = std::max(1, std::min(pl.proj_nacc, pl.proj_nacc_max));
    prm.b_resident = pl.proj_b_resident;
    prm.ns_b = pl.proj_ns_b;
    const int grid = std::min(prm.n_tiles, pl.proj_ctas);
    cudaEvent_t ev;
    prof_begin(m, "split_phi_project_tc", &ev);
    if (pl.a_terms == 2)
        launch_pdl(k_proj_tc<2, 3>, dim3(grid), dim3(kProjThreads), pl.proj_smem, m->stream, m->tm_rho, prm);
    else
        launch_pdl(k_proj_tc<3, 6>, dim3(grid), dim3(kProjThreads), pl.proj_smem, m->stream, m->tm_rho, prm);
    prof_end(m, "split_phi_project_tc", ev);
    return cudaGetLastError();
}

static cudaError_t launch_phi_synth(mp_mesh *m);

cudaError_t launch_split_synth(mp_mesh *m, double *phi)
{
    (void)phi;
    cudaEvent_t ev;
    if (m->plan.use_theta_tc) {
        cudaError_t e = launch_gsynth_tc(m);  // profiles its two kernels itself
        if (e != cudaSuccess) return e;
        return launch_phi_synth(m);
    }
    const SplitPlan &pl = m->plan;
    prof_begin(m, "split_theta_synth", &ev);
    const uint32_t tab_bytes = (uint32_t)((size_t)m->T * pl.ldF * 4);
    const int U = (m->L + 1) / 2, NJ = ((m->n_t + 3) / 4 + 31) / 32;
    const int pipe_threads = std::max(64, std::min(1024, kGsS * NJ * U * 32));
    const size_t pipe_smem = (size_t)tab_bytes + (size_t)kGsS * pl.Kpad * pl.ldF * 4 +
                             (((size_t)kGsS * m->KL + 1) & ~(size_t)1) * 4 +
                             ((size_t)(m->L + 1) * m->n_t + (size_t)kGsS * (m->L + 1)) * 8 + 16;
    if (pipe_smem <= 200 * 1024 && kGsS * m->KL <= kGsPre * pipe_threads && kGsS * (m->L + 1) <= pipe_threads) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_gsynth_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            cudaFuncSetAttribute(k_gsynth_pipe<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set = true;
        }
        const int grid = std::min((m->n_r + kGsS - 1) / kGsS, m->num_sms);
        if (pl.a_terms == 2)
            launch_pdl(k_gsynth_pipe<2>, dim3(grid), dim3(pipe_threads), pipe_smem, m->stream, m->d_C32, m->d_Itc32,
                       m->d_C0, m->d_Itc0, m->d_Aop, m->d_G0, m->d_err, m->n_r, m->n_t, m->L, m->KL, pl.Kpad,
                       pl.ldF, tab_bytes);
        else
            launch_pdl(k_gsynth_pipe<3>, dim3(grid), dim3(pipe_threads), pipe_smem, m->stream, m->d_C32, m->d_Itc32,
                       m->d_C0, m->d_Itc0, m->d_Aop, m->d_G0, m->d_err, m->n_r, m->n_t, m->L, m->KL, pl.Kpad,
                       pl.ldF, tab_bytes);
    } else {
        // z < kGm0Parts: the m = 0 column; z >= kGm0Parts: order m = z - kGm0Parts + 1
        const dim3 grid((m->n_t + kGmCells - 1) / kGmCells, (m->n_r + kGmShells - 1) / kGmShells,
                        m->L + kGm0Parts);
        if (pl.a_terms == 2)
            launch_pdl(k_gsynth_mgemm<2>, grid, dim3(256), 0, m->stream, m->d_C32, m->d_Itc32, m->d_C0, m->d_Itc0,
                       m->d_Aop, m->d_G0,
                       m->n_r, m->n_t, m->L, m->KL, pl.Kpad, pl.ldF);
        else
            launch_pdl(k_gsynth_mgemm<3>, grid, dim3(256), 0, m->stream, m->d_C32, m->d_Itc32, m->d_C0, m->d_Itc0,
                       m->d_Aop, m->d_G0,
                       m->n_r, m->n_t, m->L, m->KL, pl.Kpad, pl.ldF);
    }
    prof_end(m, "split_theta_synth", ev);
    return launch_phi_synth(m);
}

static cudaError_t launch_phi_synth(mp_mesh *m)
{
    const SplitPlan &pl = m->plan;
    const int n_tiles = (int)((m->R + kBM - 1) / kBM);
    cudaEvent_t ev;
    SynthParams prm;
    prm.Aop = m->d_Aop;
    prm.G0 = m->d_G0;
    prm.tabT = m->d_tabT;
    prm.err = m->d_err;
    prm.R = m->R;
    prm.Kpad = pl.Kpad;
    prm.NC = pl.NC;
    prm.n_nc = pl.n_nc;
    prm.n_tiles = n_tiles;
    prm.ns_a = pl.ns_a;
    prm.ns_b = pl.ns_b;
    prm.stg_bufs = pl.stg_bufs;
    prm.stg_cols = pl.stg_cols;
    prm.b_resident = pl.b_resident;
    prm.a_bytes = (uint32_t)(pl.a_terms * kBM * pl.Kpad * 2);
    prm.bchunk = (uint32_t)(3 * pl.NC * 32);
    // every term of a chunk is copied: copying only the terms the products read (BF16X3)
    // measured slower on GB300 (2048 x 512 x 1024, l_max = 64: 1566 -> 1634 us)
    prm.bload = prm.bchunk;
    const int grid = std::min(n_tiles * pl.n_nc, pl.synth_ctas);  // work units: (tile, column chunk)
    prof_begin(m, "split_synth_tc", &ev);
    if (pl.a_terms == 2)
        launch_pdl(k_synth_tc<2, 3>, dim3(grid), dim3(synth::THREADS), pl.synth_smem, m->stream, m->tm_phi, prm);
    else
        launch_pdl(k_synth_tc<3, 6>, dim3(grid), dim3(synth::THREADS), pl.synth_smem, m->stream, m->tm_phi, prm);
    prof_end(m, "split_synth_tc", ev);
    return cudaGetLastError();
}

}  // namespace mp
