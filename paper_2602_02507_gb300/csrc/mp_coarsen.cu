// mp_coarsen.cu -- coarsening-block averaging (GenASiS II Sec. 2.1: angular blocks
// where angular cell widths fall below the minimum radial width; Sec. 2.3: every
// cell of a block takes the volume-weighted mean sum V_j K_j / sum V_j).
//
// Block rule (the paper shows the blocks only in figures):
//   Delta r_min = the smallest radial width; widths at the cell-centre radius r_c.
//   polar: runs of p cells, p the smallest power of two dividing n_theta with
//          p r_c min(dtheta) >= Delta r_min, else the whole polar range;
//   azimuthal, within a polar block: runs of q cells, q the smallest power of two
//          dividing n_phi with q r_c sin(theta_c) min(dphi) >= Delta r_min (theta_c
//          of the block's polar cell nearest the axis), else the whole ring.
// Volumes are separable, so within a shell the weights are dmu_j dphi_k.
//
// The host turns the rule into a work list once per mesh: one entry per polar
// block that is coarsened (p > 1 or q > 1); cells outside every block are not
// touched.  Each cell's mean is the normalised polar weights (dmu_j / sum dmu, none
// for a single polar cell) applied along theta, then the normalised azimuthal
// weights along phi, so that a single-row block of two cells costs one float64
// multiply and one multiply-add: the float64 pipe of this part (about 0.5 T
// instructions/s), not HBM, bounds the kernel.  On 16-byte aligned fields (even
// n_phi) one launch holds three kinds of CTA:
//   * blocks of more than kStageRows rows: one CTA per chunk of kStageRows rows
//     (partial polar sums to scratch; the CTA that finishes an entry's last chunk
//     forms and writes the means), so that the whole-sphere block near the origin
//     is not one long chain of loads on one SM;
//   * wide blocks (a power of two above 64 cells, or the whole ring): one CTA each,
//     reduced across the CTA;
//   * the rest (power-of-two azimuthal blocks up to 64 cells): runs of consecutive
//     entries of at most kStageRows rows, all their rows copied to shared memory by
//     cp.async at once, two columns a thread, shuffles within each azimuthal block.
// On other fields (odd n_phi, 2-D meshes, odd offsets) the same chunks for blocks of
// many rows, then one CTA per entry, one column a thread.  Every coarsened cell is read
// once and written once.  Float64 throughout.
#include <algorithm>
#include <cmath>

#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

constexpr int kCoarsenThreads = 256;
constexpr int kCoarsenLevels = 7;  // azimuthal block sizes 1, 2, 4, ..., 64 have normalised weights
constexpr int kStageRows = 8;      // rows a CTA stages at once (16 bytes a thread each)
constexpr int kFieldBatch = 4;     // fields per launch on aligned fields (scratch and counters for each)

struct CoarsenArgs {
    double *f;
    long long stride;
    const int4 *work;      // entries: shell, first polar cell, polar size ct, azimuthal size cp
    const int2 *groups;    // runs: first entry, number of entries
    const int4 *chunks;    // chunks of many-row blocks: entry, chunk, first scratch row, counter
    double *scratch;       // [field][scratch row][n_phi] polar sums of the chunks
    int *counters;         // [field][many-row block] finished chunks
    const double *dmu, *dph, *nph, *inv_mu, *nth;
    int n_th_rows, n_t, n_p;
    int e_wide_first;      // first entry taken one per CTA
    int n_chunk_ctas, n_wide_ctas, n_big, n_scratch_rows;
};

// The block's mean is sum_j sum_k (dmu_j / sum dmu) (dphi_k / sum_{block} dphi) K_jk: the
// normalised polar weights nth[row][j] (row log2 of the polar block size, or the last row for
// the whole polar range) and azimuthal weights nph[level][k] (block size 2^level) come from
// the host.

__device__ __forceinline__ void cp_async16(double2 *dst, const double *src) { cp_async16_zfill(smem_u32(dst), src, 16); }
__device__ __forceinline__ void cp_async_wait_all()
{
    cp_async_commit();
    cp_async_wait<0>();
}

// The mean of one power-of-two azimuthal block (up to 64 cells) from the polar sums c0, c1 of a
// thread's two columns k, k + 1: the cp / 2 lanes of the block (aligned: 64 columns per warp,
// a multiple of cp) add their sums, weighted by the normalised azimuthal weights, by shuffles;
// every cell of the block's ct rows takes it.  All lanes of the warp call this together.
__device__ __forceinline__ void coarsen_finish(double *base, int ct, int cp, const double *__restrict__ nph, int n_p,
                                               int k, bool in, double c0, double c1)
{
    double2 out = make_double2(c0, c1);
    if (cp > 1) {
        const double *w_phi = nph + (size_t)(__ffs(cp) - 1) * n_p;
        double num = in ? fma(__ldg(w_phi + k + 1), c1, __ldg(w_phi + k) * c0) : 0.0;
        for (int o = 1; o < cp / 2; o <<= 1) num += __shfl_xor_sync(0xFFFFFFFFu, num, o);
        out = make_double2(num, num);
    }
    if (in)
        for (int j = 0; j < ct; ++j) *reinterpret_cast<double2 *>(base + (long long)j * n_p + k) = out;
}

// A run of consecutive entries with power-of-two azimuthal blocks up to 64 cells and at most
// kStageRows rows in all (16-byte aligned fields).  Each thread owns two adjacent columns
// along phi and copies its 16 bytes of every row of the run into its own shared-memory
// slots (cp.async: all the rows' loads in flight together, no registers held for them),
// then sums its columns over each block's rows with the normalised polar weights (none for
// a single polar cell).
__device__ __forceinline__ void coarsen_run(double *fld, const int4 *__restrict__ work, int2 g,
                                            const double *__restrict__ nph, const double *__restrict__ nth,
                                            int n_th_rows, int n_t, int n_p, double2 *stage)
{
    const int nthr = (int)blockDim.x, tid = (int)threadIdx.x;
    for (int k0 = 0; k0 < n_p; k0 += 2 * nthr) {
        const int k = k0 + 2 * tid;
        const bool in = k < n_p;
        int row = 0;
        for (int q = 0; q < g.y; ++q) {
            const int4 wk = work[g.x + q];
            const double *base = fld + ((long long)wk.x * n_t + wk.y) * n_p + k;
            if (in)
                for (int j = 0; j < wk.z; ++j) cp_async16(stage + (row + j) * nthr + tid, base + (long long)j * n_p);
            row += wk.z;
        }
        cp_async_wait_all();
        row = 0;
        for (int q = 0; q < g.y; ++q) {
            const int4 wk = work[g.x + q];
            const int j0 = wk.y, ct = wk.z;
            double c0 = 0.0, c1 = 0.0;
            if (in) {
                if (ct == 1) {
                    const double2 v = stage[row * nthr + tid];
                    c0 = v.x;
                    c1 = v.y;
                } else {
                    const double *w_th = nth + (size_t)((ct & (ct - 1)) == 0 ? __ffs(ct) - 1 : n_th_rows - 1) * n_t + j0;
                    for (int j = 0; j < ct; ++j) {
                        const double2 v = stage[(row + j) * nthr + tid];
                        const double w = __ldg(w_th + j);
                        c0 = fma(w, v.x, c0);
                        c1 = fma(w, v.y, c1);
                    }
                }
            }
            coarsen_finish(fld + ((long long)wk.x * n_t + j0) * n_p, ct, wk.w, nph, n_p, k, in, c0, c1);
            row += ct;
        }
    }
}

// Polar blocks of more than kStageRows rows (16-byte aligned fields): one CTA per chunk of
// kStageRows rows, so that such a block is not one long chain of loads on one SM.  Chunk
// d = (entry, chunk, first scratch row of the entry, counter) writes the polar sums of its
// rows per column (normalised polar weights) to scratch; the CTA that finishes an entry's
// last chunk (a counter per entry and field, reset by that CTA) adds the chunks' sums in
// chunk order, forms each azimuthal block's mean sum dphi_k S_k / sum dphi_k (any block
// width) and writes it to every cell of the block.  No CTA waits for another.
template <int V>
__device__ __forceinline__ void coarsen_chunk(double *fld, const CoarsenArgs &a, int4 d, double *sm)
{
    const int nthr = (int)blockDim.x, tid = (int)threadIdx.x, n_t = a.n_t, n_p = a.n_p;
    const int4 wk = a.work[d.x];
    const int j0 = wk.y, ct = wk.z, cp = wk.w;
    const int n_ch = (ct + kStageRows - 1) / kStageRows, r0 = d.y * kStageRows, nr = min(kStageRows, ct - r0);
    double *base = fld + ((long long)wk.x * n_t + j0) * n_p;
    const double *w_th = a.nth + (size_t)((ct & (ct - 1)) == 0 ? __ffs(ct) - 1 : a.n_th_rows - 1) * n_t + j0;
    double *part = a.scratch + ((long long)blockIdx.y * a.n_scratch_rows + d.z) * n_p;
    for (int k = V * tid; k < n_p; k += V * nthr) {
        double c0 = 0.0, c1 = 0.0;
#pragma unroll
        for (int r = 0; r < kStageRows; ++r)
            if (r < nr) {
                const double w = __ldg(w_th + r0 + r);
                if (V == 2) {
                    const double2 v = *reinterpret_cast<const double2 *>(base + (long long)(r0 + r) * n_p + k);
                    c0 = fma(w, v.x, c0);
                    c1 = fma(w, v.y, c1);
                } else {
                    c0 = fma(w, base[(long long)(r0 + r) * n_p + k], c0);
                }
            }
        if (V == 2)
            __stcg(reinterpret_cast<double2 *>(part + (long long)d.y * n_p + k), make_double2(c0, c1));
        else
            __stcg(part + (long long)d.y * n_p + k, c0);
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    int *cnt = a.counters + blockIdx.y * a.n_big + d.w;
    if (tid == 0) s_last = atomicAdd(cnt, 1) == n_ch - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double *sS = sm, *sM = sm + n_p;  // column sums, block means
    for (int k = tid; k < n_p; k += nthr) {
        double acc = 0.0;
        for (int c = 0; c < n_ch; ++c) acc += __ldcg(part + (long long)c * n_p + k);
        sS[k] = acc;
    }
    __syncthreads();
    const int lane = tid & 31, nkb = n_p / cp;
    for (int b = tid >> 5; b < nkb; b += nthr >> 5) {
        double num = 0.0, den = 0.0;
        for (int k = b * cp + lane; k < (b + 1) * cp; k += 32) {
            const double dp = __ldg(a.dph + k);
            num = fma(dp, sS[k], num);
            den += dp;
        }
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xFFFFFFFFu, num, o);
            den += __shfl_xor_sync(0xFFFFFFFFu, den, o);
        }
        if (lane == 0) sM[b] = num / den;  // one division per block
    }
    __syncthreads();
    if (V == 2) {
        for (int k = 2 * tid; k < n_p; k += 2 * nthr) {
            const double2 out = make_double2(sM[k / cp], sM[(k + 1) / cp]);
            for (int j = 0; j < ct; ++j) *reinterpret_cast<double2 *>(base + (long long)j * n_p + k) = out;
        }
    } else if (n_p >= nthr) {
        for (int k = tid; k < n_p; k += nthr)  // one column a thread
            for (int j = 0; j < ct; ++j) base[(long long)j * n_p + k] = sM[k / cp];
    } else {
        // fewer columns than threads (n_phi = 1 on 2-D meshes): the rows are dealt out too
        const int per = nthr / n_p, k = tid % n_p, j1 = tid / n_p;
        if (j1 < per)
            for (int j = j1; j < ct; j += per) base[(long long)j * n_p + k] = sM[k / cp];
    }
    if (tid == 0) *cnt = 0;  // ready for the next launch
}

// The CTAs take, in this order, one chunk of a block of many rows each, then, for VEC = 2
// (16-byte aligned fields, even n_phi), one entry of a wide block each (a power of two above
// 64 cells, or the whole ring) and one run of groups[] each; for VEC = 1, one entry of every
// other block each.
template <int VEC>
__global__ void __launch_bounds__(kCoarsenThreads, 6) k_coarsen(const CoarsenArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    double *fld = a.f + (long long)blockIdx.y * a.stride;
    const int n_t = a.n_t, n_p = a.n_p;
    int x = (int)blockIdx.x;
    if (x < a.n_chunk_ctas) {
        coarsen_chunk<VEC>(fld, a, a.chunks[x], reinterpret_cast<double *>(dsm));
        return;
    }
    x -= a.n_chunk_ctas;
    if (VEC == 2) {
        if (x >= a.n_wide_ctas) {
            coarsen_run(fld, a.work, a.groups[x - a.n_wide_ctas], a.nph, a.nth, a.n_th_rows, n_t, n_p,
                        reinterpret_cast<double2 *>(dsm));
            return;
        }
    }
    const double *__restrict__ dmu = a.dmu, *__restrict__ dph = a.dph, *__restrict__ nph = a.nph;
    const int e = a.e_wide_first + x;
    const int4 wk = a.work[e];  // shell, first polar cell, polar size, azimuthal size
    const int j0 = wk.y, ct = wk.z, cp = wk.w;
    double *base = fld + ((long long)wk.x * n_t + j0) * n_p;
    const int lane = threadIdx.x & 31;
    const bool pow2 = (cp & (cp - 1)) == 0;
    const double inv = a.inv_mu[e];  // 1 / sum of dmu over the polar block (no divisions here:
                                     // they are slow on the float64 pipe of this part)
    if (VEC == 1 && pow2 && cp <= 32) {
        // one column per thread (odd n_phi or unaligned fields)
        const double *w_phi = nph + (size_t)(__ffs(cp) - 1) * n_p;
        for (int k0 = 0; k0 < n_p; k0 += (int)blockDim.x) {
            const int k = k0 + (int)threadIdx.x;
            const bool in = k < n_p;
            double col = 0.0;
            if (in)
#pragma unroll 4
                for (int j = 0; j < ct; ++j) col = fma(dmu[j0 + j], base[(long long)j * n_p + k], col);
            double num = in ? w_phi[k] * col : 0.0;
            for (int o = 1; o < cp; o <<= 1) num += __shfl_xor_sync(0xFFFFFFFFu, num, o);
            if (in) {
                const double mean = num * inv;
                for (int j = 0; j < ct; ++j) base[(long long)j * n_p + k] = mean;
            }
        }
        return;
    }
    // wider blocks (a power of two above 64, above 32 on unaligned fields, or the whole
    // ring): threads again take columns along phi (two at a time when aligned) and sum them
    // over the polar block; each warp reduces its chunk of 32 V columns, and one thread per
    // azimuthal block adds its chunks in order (a chunk never straddles two blocks: cp is a
    // multiple of 32 V, or the block is the whole ring)
    double *chunk = reinterpret_cast<double *>(dsm);  // per chunk of 32 V columns: num, den; then per block: the mean
    constexpr int V = VEC;
    const int per_warp = 32 * V, warp = threadIdx.x >> 5;
    const int n_chunks = (n_p + per_warp - 1) / per_warp;
    for (int k0 = 0; k0 < n_p; k0 += V * (int)blockDim.x) {
        const int k = k0 + V * (int)threadIdx.x;
        double c0 = 0.0, c1 = 0.0;
        // eight rows' loads in flight a thread: a block of many rows is a long chain of them,
        // and its CTA sets the kernel's length when few others are left
        if (k < n_p)
#pragma unroll 8
            for (int j = 0; j < ct; ++j) {
                const double w = dmu[j0 + j];
                if (V == 2) {
                    const double2 v = *reinterpret_cast<const double2 *>(base + (long long)j * n_p + k);
                    c0 = fma(w, v.x, c0);
                    c1 = fma(w, v.y, c1);
                } else {
                    c0 = fma(w, base[(long long)j * n_p + k], c0);
                }
            }
        double num = 0.0, den = 0.0;  // den: the block's dphi sum
        if (k < n_p) {
            num = dph[k] * c0;
            den = dph[k];
            if (V == 2) {
                num = fma(dph[k + 1], c1, num);
                den += dph[k + 1];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xFFFFFFFFu, num, o);
            den += __shfl_xor_sync(0xFFFFFFFFu, den, o);
        }
        const int ci = (k0 + warp * per_warp) / per_warp;
        if (lane == 0 && ci < n_chunks) {
            chunk[ci] = num;
            chunk[n_chunks + ci] = den;
        }
    }
    __syncthreads();
    const int nkb = n_p / cp, cpc = (cp + per_warp - 1) / per_warp;  // chunks per block
    for (int b = threadIdx.x; b < nkb; b += blockDim.x) {
        double n_ = 0.0, d_ = 0.0;
        for (int c = b * cpc; c < min((b + 1) * cpc, n_chunks); ++c) {
            n_ += chunk[c];
            d_ += chunk[n_chunks + c];
        }
        chunk[2 * n_chunks + b] = n_ / d_ * inv;  // one division per block
    }
    __syncthreads();
    for (int k0 = 0; k0 < n_p; k0 += V * (int)blockDim.x) {
        const int k = k0 + V * (int)threadIdx.x;
        if (k >= n_p) continue;
        const double mean = chunk[2 * n_chunks + k / cp];
        for (int j = 0; j < ct; ++j) {
            if (V == 2)
                *reinterpret_cast<double2 *>(base + (long long)j * n_p + k) = make_double2(mean, mean);
            else
                base[(long long)j * n_p + k] = mean;
        }
    }
}

// rows of the normalised polar weights: block sizes 2^0 .. 2^floor(log2 n_t), then the whole range
int coarsen_theta_rows(int n_t)
{
    int rows = 1;
    while ((1 << rows) <= n_t) ++rows;
    return rows + 1;
}

int pow2_block(double need, int n)
{
    for (int p = 1; p <= n; p *= 2)
        if (n % p == 0 && (double)p >= need) return p;
    return n;
}

}  // namespace

cudaError_t coarsen_prepare(mp_mesh *m)
{
    const int n_r = m->n_r, n_t = m->n_t, n_p = m->n_p;
    double dr_min = m->h_r[1] - m->h_r[0], dth = m->h_th[1] - m->h_th[0], dph = m->h_ph[1] - m->h_ph[0];
    for (int i = 1; i < n_r; ++i) dr_min = std::min(dr_min, m->h_r[i + 1] - m->h_r[i]);
    for (int j = 1; j < n_t; ++j) dth = std::min(dth, m->h_th[j + 1] - m->h_th[j]);
    for (int k = 1; k < n_p; ++k) dph = std::min(dph, m->h_ph[k + 1] - m->h_ph[k]);
    m->h_ctheta.assign(n_r, 1);
    m->h_cphi.assign((size_t)n_r * n_t, 1);
    std::vector<int4> work;
    for (int i = 0; i < n_r; ++i) {
        const double rc = 0.5 * (m->h_r[i] + m->h_r[i + 1]);
        const int ct = pow2_block(dr_min / (rc * dth), n_t);
        m->h_ctheta[i] = ct;
        for (int j0 = 0; j0 < n_t; j0 += ct) {
            double need = 0.0;  // the block's cell nearest the axis needs the widest azimuthal block
            for (int j = j0; j < j0 + ct; ++j) {
                const double tc = 0.5 * (m->h_th[j] + m->h_th[j + 1]);
                need = std::max(need, dr_min / (rc * std::sin(tc) * dph));
            }
            const int cp = pow2_block(need, n_p);
            for (int j = j0; j < j0 + ct; ++j) m->h_cphi[(size_t)i * n_t + j] = cp;
            if (ct > 1 || cp > 1) work.push_back(make_int4(i, j0, ct, cp));
        }
    }
    // order of the entries: power-of-two azimuthal blocks up to 64 cells of at most kStageRows
    // rows (staged in runs on aligned fields), other blocks of at most kStageRows rows (one
    // CTA each), blocks of more rows (chunks of kStageRows rows); each part in mesh order
    const auto is_run = [](const int4 &e) { return e.z <= kStageRows && (e.w & (e.w - 1)) == 0 && e.w <= 64; };
    const auto is_short = [](const int4 &e) { return e.z <= kStageRows; };
    std::stable_partition(work.begin(), work.end(), is_short);
    std::stable_partition(work.begin(), work.end(), is_run);
    m->n_cwork = (int)work.size();
    m->n_cwork_fast = (int)std::count_if(work.begin(), work.end(), is_run);
    m->n_cwork_wide = (int)std::count_if(work.begin(), work.end(), is_short) - m->n_cwork_fast;
    std::vector<int2> groups;  // runs of consecutive entries of at most kStageRows rows in all
    int open_rows = kStageRows + 1;  // rows in the last run (above kStageRows: none open)
    for (int e = 0; e < m->n_cwork_fast; ++e) {
        const int ct = work[e].z;
        if (open_rows + ct > kStageRows) {
            groups.push_back(make_int2(e, 1));
            open_rows = ct;
        } else {
            ++groups.back().y;
            open_rows += ct;
        }
    }
    std::vector<int4> chunks;  // entry, chunk, first scratch row, counter
    m->n_cbig = 0;
    m->n_cscratch_rows = 0;
    for (int e = m->n_cwork_fast + m->n_cwork_wide; e < m->n_cwork; ++e) {
        const int n_ch = (work[e].z + kStageRows - 1) / kStageRows;
        for (int c = 0; c < n_ch; ++c) chunks.push_back(make_int4(e, c, m->n_cscratch_rows, m->n_cbig));
        m->n_cscratch_rows += n_ch;
        ++m->n_cbig;
    }
    m->n_cchunks = (int)chunks.size();
    m->n_cgroups = (int)groups.size();
    std::vector<double> inv_mu(std::max<size_t>(1, work.size()), 0.0);
    for (size_t e = 0; e < work.size(); ++e) {
        double sum = 0.0;
        for (int j = work[e].y; j < work[e].y + work[e].z; ++j) sum += std::cos(m->h_th[j]) - std::cos(m->h_th[j + 1]);
        inv_mu[e] = 1.0 / sum;
    }
    // weights: dmu [n_t], dphi [n_p], per block size 2^level the normalised dphi, per work entry
    // 1 / (sum of dmu over its polar block), then the normalised dmu per polar block size 2^level
    // (level < n_th_rows - 1) and for the whole polar range (the last row)
    const int n_th_rows = coarsen_theta_rows(n_t);
    const size_t off_nth = (size_t)n_t + (size_t)n_p * (1 + kCoarsenLevels) + inv_mu.size();
    std::vector<double> w(off_nth + (size_t)n_th_rows * n_t, 0.0);
    for (int j = 0; j < n_t; ++j) w[j] = std::cos(m->h_th[j]) - std::cos(m->h_th[j + 1]);
    for (int k = 0; k < n_p; ++k) w[(size_t)n_t + k] = m->h_ph[k + 1] - m->h_ph[k];
    for (int lv = 0; lv < kCoarsenLevels; ++lv) {
        const int q = 1 << lv;
        if (n_p % q) continue;  // no blocks of this size on this mesh
        for (int k0 = 0; k0 < n_p; k0 += q) {
            double sum = 0.0;
            for (int k = k0; k < k0 + q; ++k) sum += w[(size_t)n_t + k];
            for (int k = k0; k < k0 + q; ++k)
                w[(size_t)n_t + (size_t)n_p * (1 + lv) + k] = w[(size_t)n_t + k] / sum;
        }
    }
    std::copy(inv_mu.begin(), inv_mu.end(), w.begin() + n_t + (size_t)n_p * (1 + kCoarsenLevels));
    for (int row = 0; row < n_th_rows; ++row) {
        const int q = row < n_th_rows - 1 ? 1 << row : n_t;
        if (n_t % q) continue;  // no polar blocks of this size on this mesh
        for (int j0 = 0; j0 < n_t; j0 += q) {
            double sum = 0.0;
            for (int j = j0; j < j0 + q; ++j) sum += w[j];
            for (int j = j0; j < j0 + q; ++j) w[off_nth + (size_t)row * n_t + j] = w[j] / sum;
        }
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&m->d_cwork), std::max<size_t>(1, work.size()) * sizeof(int4));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(reinterpret_cast<void **>(&m->d_cweights), w.size() * sizeof(double));
    if (e != cudaSuccess) return e;
    m->device_bytes += std::max<size_t>(1, work.size()) * sizeof(int4) + w.size() * sizeof(double);
    if (!work.empty()) {
        e = cudaMemcpy(m->d_cwork, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    e = cudaMalloc(reinterpret_cast<void **>(&m->d_cgroups), std::max<size_t>(1, groups.size()) * sizeof(int2));
    if (e != cudaSuccess) return e;
    m->device_bytes += std::max<size_t>(1, groups.size()) * sizeof(int2);
    if (!groups.empty()) {
        e = cudaMemcpy(m->d_cgroups, groups.data(), groups.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    if (m->n_cbig > 0) {
        e = cudaMalloc(reinterpret_cast<void **>(&m->d_cchunks), chunks.size() * sizeof(int4));
        if (e != cudaSuccess) return e;
        e = cudaMalloc(reinterpret_cast<void **>(&m->d_cscratch),
                       (size_t)kFieldBatch * m->n_cscratch_rows * n_p * sizeof(double));
        if (e != cudaSuccess) return e;
        e = cudaMalloc(reinterpret_cast<void **>(&m->d_ccount), (size_t)kFieldBatch * m->n_cbig * sizeof(int));
        if (e != cudaSuccess) return e;
        m->device_bytes += chunks.size() * sizeof(int4) + (size_t)kFieldBatch * m->n_cscratch_rows * n_p * sizeof(double) +
                           (size_t)kFieldBatch * m->n_cbig * sizeof(int);
        e = cudaMemset(m->d_ccount, 0, (size_t)kFieldBatch * m->n_cbig * sizeof(int));
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(m->d_cchunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpy(m->d_cweights, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
}

cudaError_t launch_coarsen(mp_mesh *m, double *fields, int n_fields, long long stride)
{
    if (m->n_cwork == 0 || n_fields == 0) return cudaSuccess;
    cudaEvent_t ev;
    prof_begin(m, "coarsen_blocks", &ev);
    // 16-byte accesses need even n_phi and 16-byte aligned fields
    const int vec = (m->n_p % 2 == 0) && (reinterpret_cast<uintptr_t>(fields) % 16 == 0) && (stride % 2 == 0) ? 2 : 1;
    // as many threads as one pass along a ring takes (at most 256)
    const int threads = std::min(kCoarsenThreads, std::max(32, 32 * ((m->n_p + 32 * vec - 1) / (32 * vec))));
    // wide blocks keep per-chunk sums and per-block means in dynamic shared memory; runs, the
    // staged rows; the last chunk of a many-row block, column sums and block means
    const int per_warp = 32 * vec;
    const int n_chunks = (m->n_p + per_warp - 1) / per_warp;
    size_t smem = (size_t)3 * n_chunks * sizeof(double);
    smem = std::max(smem, (size_t)2 * m->n_p * sizeof(double));
    if (vec == 2) smem = std::max(smem, (size_t)kStageRows * threads * 16);
    if (smem > 48 * 1024) {
        const cudaError_t e = vec == 2 ? cudaFuncSetAttribute(k_coarsen<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                                       : cudaFuncSetAttribute(k_coarsen<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const double *w = m->d_cweights;
    const size_t off_inv = (size_t)m->n_t + (size_t)m->n_p * (1 + kCoarsenLevels);
    CoarsenArgs a;
    a.f = fields;
    a.stride = stride;
    a.work = m->d_cwork;
    a.groups = m->d_cgroups;
    a.chunks = m->d_cchunks;
    a.scratch = m->d_cscratch;
    a.counters = m->d_ccount;
    a.dmu = w;
    a.dph = w + m->n_t;
    a.nph = w + m->n_t + m->n_p;
    a.inv_mu = w + off_inv;
    a.nth = w + off_inv + std::max(1, m->n_cwork);
    a.n_th_rows = coarsen_theta_rows(m->n_t);
    a.n_t = m->n_t;
    a.n_p = m->n_p;
    a.n_big = m->n_cbig;
    a.n_scratch_rows = m->n_cscratch_rows;
    // chunks of many-row blocks first, then (aligned) wide blocks one per CTA and runs, or
    // (unaligned) every other block one per CTA; kFieldBatch fields a launch (the scratch and
    // counters are per field of a launch)
    a.n_chunk_ctas = m->n_cchunks;
    a.e_wide_first = vec == 2 ? m->n_cwork_fast : 0;
    a.n_wide_ctas = vec == 2 ? m->n_cwork_wide : m->n_cwork_fast + m->n_cwork_wide;
    const unsigned gx = (unsigned)(m->n_cchunks + a.n_wide_ctas + (vec == 2 ? m->n_cgroups : 0));
    for (int f0 = 0; f0 < n_fields; f0 += kFieldBatch) {
        a.f = fields + (long long)f0 * stride;
        const dim3 grid(gx, (unsigned)std::min(kFieldBatch, n_fields - f0));
        if (vec == 2)
            k_coarsen<2><<<grid, threads, smem, m->stream>>>(a);
        else
            k_coarsen<1><<<grid, threads, smem, m->stream>>>(a);
    }
    prof_end(m, "coarsen_blocks", ev);
    return cudaGetLastError();
}

}  // namespace mp
