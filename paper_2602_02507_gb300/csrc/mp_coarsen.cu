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
// touched.  One CTA per (entry, field).  Azimuthal blocks of a power of two up to
// 128 cells (n_phi a multiple of 4): threads run along phi four columns at a time
// (two 16-byte accesses), each sums its columns over the polar block with the
// block's normalised polar weights (none for a single polar cell), and the block's
// lanes add their sums, weighted by normalised azimuthal weights, by shuffles: about
// 1.2 float64 operations a cell on the paper mesh, the float64 pipe of this part being
// the bound before HBM.  Two columns (odd multiples of 2) or one column per thread
// (odd n_phi, unaligned fields) otherwise; wider blocks: the whole CTA reduces each
// one.  Every coarsened cell is read once and written once.  Float64 throughout.
#include <algorithm>
#include <cmath>

#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

constexpr int kCoarsenThreads = 256;
constexpr int kCoarsenLevels = 7;  // azimuthal block sizes 1, 2, 4, ..., 64 have normalised weights

// The block's mean is sum_j sum_k (dmu_j / sum dmu) (dphi_k / sum_{block} dphi) K_jk: the
// normalised azimuthal weights nph[level][k] (block size 2^level) come from the host.
// VEC = 2: 16-byte accesses (two columns a thread), VEC = 1: one column a thread.
template <int VEC>
__global__ void __launch_bounds__(kCoarsenThreads) k_coarsen(double *__restrict__ f, long long stride,
                                                             const int4 *__restrict__ work,
                                                             const double *__restrict__ dmu,
                                                             const double *__restrict__ dph,
                                                             const double *__restrict__ nph,
                                                             const double *__restrict__ inv_mu,
                                                             const double *__restrict__ nth, int n_th_rows, int n_t,
                                                             int n_p)
{
    const int4 wk = work[blockIdx.x];  // shell, first polar cell, polar size, azimuthal size
    const int j0 = wk.y, ct = wk.z, cp = wk.w;
    double *base = f + (long long)blockIdx.y * stride + ((long long)wk.x * n_t + j0) * n_p;
    const int lane = threadIdx.x & 31;
    const bool pow2 = (cp & (cp - 1)) == 0;
    const double inv = inv_mu[blockIdx.x];  // 1 / sum of dmu over the polar block (no divisions here:
                                            // they are slow on the float64 pipe of this part)
    if (VEC == 2 && pow2 && cp <= 64) {
        // two adjacent columns per thread (16-byte accesses along phi): each sums its columns
        // over the polar block with the block's normalised polar weights (none for a single
        // polar cell); the cp / 2 lanes of an azimuthal block (aligned: 64 columns per warp, a
        // multiple of cp) add their sums, weighted by the normalised azimuthal weights, by shuffles
        const double *w_phi = nph + (size_t)(__ffs(cp) - 1) * n_p;
        const double *w_th = nth + (size_t)((ct & (ct - 1)) == 0 ? __ffs(ct) - 1 : n_th_rows - 1) * n_t + j0;
        for (int k0 = 0; k0 < n_p; k0 += 2 * (int)blockDim.x) {
            const int k = k0 + 2 * (int)threadIdx.x;
            const bool in = k < n_p;
            double c0 = 0.0, c1 = 0.0;
            if (in) {
                if (ct == 1) {
                    const double2 v = *reinterpret_cast<const double2 *>(base + k);
                    c0 = v.x;
                    c1 = v.y;
                } else {
#pragma unroll 4
                    for (int j = 0; j < ct; ++j) {
                        const double2 v = *reinterpret_cast<const double2 *>(base + (long long)j * n_p + k);
                        const double w = __ldg(w_th + j);
                        c0 = fma(w, v.x, c0);
                        c1 = fma(w, v.y, c1);
                    }
                }
            }
            double2 out;
            if (cp == 1) {
                out = make_double2(c0, c1);
            } else {
                double num = in ? fma(__ldg(w_phi + k + 1), c1, __ldg(w_phi + k) * c0) : 0.0;
                for (int o = 1; o < cp / 2; o <<= 1) num += __shfl_xor_sync(0xFFFFFFFFu, num, o);
                out = make_double2(num, num);
            }
            if (in)
                for (int j = 0; j < ct; ++j) *reinterpret_cast<double2 *>(base + (long long)j * n_p + k) = out;
        }
        return;
    }
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
    // wider blocks (a power of two above 64, or the whole ring): threads again take columns
    // along phi (two at a time when aligned) and sum them over the polar block; each warp
    // reduces its chunk of 32 V columns, and one thread per azimuthal block adds its chunks
    // in order (a chunk never straddles two blocks: cp is a multiple of 32 V, or the block
    // is the whole ring)
    extern __shared__ double chunk[];  // per chunk of 32 V columns: num, den; then per block: the mean
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
    // the polar blocks with the most rows first: their CTAs run longest (a chain of row loads)
    // and so start while the many short ones stream past them
    std::stable_sort(work.begin(), work.end(), [](const int4 &a, const int4 &b) { return a.z > b.z; });
    m->n_cwork = (int)work.size();
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
    return cudaMemcpy(m->d_cweights, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
}

cudaError_t launch_coarsen(mp_mesh *m, double *fields, int n_fields, long long stride)
{
    if (m->n_cwork == 0 || n_fields == 0) return cudaSuccess;
    cudaEvent_t ev;
    prof_begin(m, "coarsen_blocks", &ev);
    // 16-byte accesses need even n_phi and 16-byte aligned fields; four columns a thread also
    // need n_phi a multiple of 4
    const bool al = (m->n_p % 2 == 0) && (reinterpret_cast<uintptr_t>(fields) % 16 == 0) && (stride % 2 == 0);
    const int vec = !al ? 1 : 2;
    // as many threads as one pass along a ring takes at the widest access (at most 256)
    const int threads = std::min(kCoarsenThreads, std::max(32, 32 * ((m->n_p + 32 * vec - 1) / (32 * vec))));
    // wide blocks keep per-chunk sums and per-block means in dynamic shared memory
    const int per_warp = vec >= 2 ? 64 : 32;
    const int n_chunks = (m->n_p + per_warp - 1) / per_warp;
    const size_t smem = (size_t)3 * n_chunks * sizeof(double);  // blocks here span whole chunks
    const double *w = m->d_cweights;
    const size_t off_inv = (size_t)m->n_t + (size_t)m->n_p * (1 + kCoarsenLevels);
    const dim3 grid((unsigned)m->n_cwork, (unsigned)n_fields);
    if (vec == 2)
        k_coarsen<2><<<grid, threads, smem, m->stream>>>(fields, stride, m->d_cwork, w, w + m->n_t, w + m->n_t + m->n_p,
                                                         w + off_inv, w + off_inv + std::max(1, m->n_cwork),
                                                         coarsen_theta_rows(m->n_t), m->n_t, m->n_p);
    else
        k_coarsen<1><<<grid, threads, smem, m->stream>>>(fields, stride, m->d_cwork, w, w + m->n_t, w + m->n_t + m->n_p,
                                                         w + off_inv, w + off_inv + std::max(1, m->n_cwork),
                                                         coarsen_theta_rows(m->n_t), m->n_t, m->n_p);
    prof_end(m, "coarsen_blocks", ev);
    return cudaGetLastError();
}

}  // namespace mp
