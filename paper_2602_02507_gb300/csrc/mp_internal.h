// mp_internal.h -- private state of a mesh and the launchers of every kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <utility>
#include <algorithm>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "multipole.h"
#include "mp_errors.h"

namespace mp {

// Column p of a real moment: p(0,c) = 0, p(m,c) = 2m-1, p(m,s) = 2m.
__host__ __device__ inline int pcol_m(int p) { return (p + 1) >> 1; }
__host__ __device__ inline int tri(int l, int m) { return l * (l + 1) / 2 + m; }
inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Split-path geometry of one mesh (tcgen05 tensor-core contractions).
struct SplitPlan {
    int a_terms = 2;      // bf16 terms of the streaming operand (density deviation / G)
    int n_products = 3;   // bf16 products accumulated per K step
    int Npad = 0;         // projection GEMM N: 2L+1 rounded up to 16
    int n_kc = 0;         // projection K chunks of 16 azimuthal cells
    int Kpad = 0;         // synthesis GEMM K: 2L rounded up to 16 (m >= 1 columns)
    int ldF = 0;          // theta contraction: padded polar-cell row of F and Ith32
    int NC = 0;           // synthesis GEMM N per work unit: 64, 128 or 256 (n_phi rounded to 16 below 64)
    int n_nc = 0;         // synthesis N chunks
    int proj_ctas = 0;    // persistent grid sizes
    int synth_ctas = 0;
    int proj_smem = 0;    // dynamic shared memory bytes
    int synth_smem = 0;
    int ns_s = 6;         // projection: TMA stages of the density
    int ns_o = 2;         // projection: stages of converted A operands (bf16 terms)
    int proj_ns_b = 2;    // projection: table ring slots (when the table is not resident)
    int ns_s_max = 0;     // projection: the deepest density ring the reserved shared memory holds
    int proj_b_resident = 0;  // projection: whole pre-split table held in shared memory
    int proj_res_ok = 0, proj_ring_ok = 0;  // projection: which table modes fit the reserved memory
    int ns_b = 3;         // synthesis: table stages (when not resident)
    int ns_a = 2;         // synthesis: A-operand stages
    int b_resident = 0;   // synthesis: whole table held in shared memory
    int stg_bufs = 2;     // synthesis: TMA store staging boxes per epilogue warp
    int stg_cols = 16;    // synthesis: float64 columns of a staging box (16: 128B swizzle, 8: 64B)
    int synth_cfg = 0;    // synthesis: index of the stage configuration above (synth_cfg_apply)
    int proj_nacc = 1;    // projection: accumulators per tile (K chunks dealt round-robin)
    int proj_nacc_max = 1;
    int scan_threads = 128;  // radial recurrences: threads (shell chunks) per moment column
    // theta stages on the tensor cores (orders m >= 1; mp_theta_tc.cu): possible for this mesh
    // (tables built), in use, and the choice the rule makes
    int theta_tc_ok = 0, use_theta_tc = 0, theta_tc_default = 0;
    int th_Nmax = 0, th_n_kc = 0, th_groups = 0, th_units = 0, th_nacc = 1, th_ns_s = 4, th_ns_o = 2, th_smem = 0;
    int gs_NS = 8, gs_n_jb = 0, gs_n_sg = 0, gs_n_mg = 0, gs_units = 0, gs_ns_s = 4, gs_smem = 0;
};

// Where the radial recurrences write the solution coefficients C[i][l^2 + p] (m >= 1) as
// the bf16 terms of the theta synthesis B operand: order m's block at cb + off[m], then
// [shell group i / NS][K chunk (l - m) / 32][term][2 NS rows (shell, cos | sin) x 32]
// canonical K-major (nullptr cb: not written).
struct CbOut {
    uint8_t *cb = nullptr;
    const unsigned long long *off = nullptr;
    int NS = 8, terms = 2, L = 0;
};

// Centred difference along one axis at one cell: (Phi[hi] - Phi[lo]) * w, w = 1 / (x_c[hi] - x_c[lo])
// (0 where the derivative is zero)
struct GradStencil {
    int lo, hi;
    double w;
};

struct ProfileEntry {
    const char *name = nullptr;
    int launches = 0;
    double total_ms = 0.0;
};

}  // namespace mp

struct mp_mesh {
    int n_r = 0, n_t = 0, n_p = 0, L = 0;
    int KL = 0, P = 0, T = 0;  // (L+1)^2, 2L+1, (L+1)(L+2)/2
    long long R = 0;           // rows n_r * n_t
    long long N = 0;           // cells
    double G = 1.0, r_ref = 1.0;
    int prec = 0, eff_prec = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    std::vector<double> h_r, h_th, h_ph;

    // float64 tables
    double *d_r = nullptr;
    double *d_Ith = nullptr;   // [T][n_t]  int P~ sin dtheta over polar cells
    double *d_dmu = nullptr;   // [n_t]
    double *d_Iph = nullptr;   // [P][n_p]  int cos|sin(m phi) over azimuthal cells
    double *d_Iphc = nullptr;  // [P][n_p]  Iph / dphi (cell mean)
    double *d_WR = nullptr, *d_WI = nullptr;  // [L+1][n_r]
    double *d_GR = nullptr, *d_GI = nullptr;  // [L+1][n_r]  -(R^R, R^I) / (2 (2l+1))
    double *d_V = nullptr;     // [n_r]

    // moments (both paths)
    double *d_A = nullptr;     // [n_r][KL]
    double *d_MR = nullptr;    // [n_r+1][KL]
    double *d_MI = nullptr;    // [n_r+1][KL]
    double *d_C = nullptr;     // [n_r][KL]

    // float64 path workspace
    double *d_F64 = nullptr;   // [R][P]
    double *d_G64 = nullptr;   // [R][P]

    // split path tables and workspace
    mp::SplitPlan plan;
    float *d_F32 = nullptr;       // [R][Npad]
    float *d_C32 = nullptr;       // [n_r][KL]
    float *d_Ith32 = nullptr;     // [T][ldF]   Ith, float, zero padding
    float *d_Itc32 = nullptr;     // [T][n_t]   Ith / dmu, float
    float *d_colsum = nullptr;    // [Npad]     sum_k Iph[p][k]
    uint8_t *d_Aop = nullptr;     // synthesis A operand, bf16 terms per 128-row tile, canonical layout
    float *d_G0 = nullptr;        // [tiles * 128] x (hi, lo) float pairs: m = 0 column of the theta synthesis
    float2 *d_Itc0 = nullptr;     // [L+1][n_t] Ith[tri(l,0)][j] / dmu_j as (hi, lo) float pairs
    float2 *d_C0 = nullptr;       // [n_r][L+1] m = 0 coefficients C[i][l^2] as (hi, lo) float pairs
    mp::GradStencil *d_gst = nullptr;  // gravity sources: [n_r + n_theta + n_phi] difference stencils
    // coarsening blocks: per shell the polar block size, per (shell, polar cell) the azimuthal
    // one; the device work list (shell, first polar cell, polar size, azimuthal size) of the
    // coarsened polar blocks and the weights dmu [n_theta], dphi [n_phi]
    std::vector<int> h_ctheta, h_cphi;
    int4 *d_cwork = nullptr;
    int n_cwork = 0;
    int n_cwork_fast = 0;   // leading entries of d_cwork staged in runs (short blocks of up to 64 cells)
    int n_cwork_wide = 0;   // then short blocks taken one per CTA; then blocks of many rows
    int2 *d_cgroups = nullptr;  // runs: first entry, count
    int n_cgroups = 0;
    int4 *d_cchunks = nullptr;  // chunks of many-row blocks: entry, chunk, first scratch row, counter
    int n_cchunks = 0, n_cbig = 0, n_cscratch_rows = 0;
    double *d_cscratch = nullptr;  // per field of a launch: polar sums of the chunks
    int *d_ccount = nullptr;       // per field of a launch and many-row block: finished chunks
    double *d_cweights = nullptr;
    // tensor-core theta stages: pre-split tables, their per-order byte offsets, the coefficient
    // terms written by the radial recurrences, and the TMA map of F ([n_r][P][ldF] float32)
    uint8_t *d_tabTh = nullptr, *d_tabGs = nullptr, *d_Cb = nullptr;
    unsigned long long *d_th_off = nullptr, *d_gs_off = nullptr, *d_cb_off = nullptr;
    CUtensorMap tm_F{};
    size_t cb_bytes_alloc = 0;
    uint8_t *d_tabB = nullptr;    // projection B operand, bf16 x 3 terms, canonical layout
    uint8_t *d_tabT = nullptr;    // synthesis B operand, bf16 x 3 terms, canonical layout
    size_t tabB_chunk_bytes = 0, tabT_chunk_bytes = 0;

    // bindings
    const double *rho = nullptr;
    double *phi_user = nullptr;
    double *phi_own = nullptr;
    // host round trips (mp_solve_host, mp_solve_host_async): two device staging pairs used
    // in turn, uploads and downloads on streams of their own, events for buffer reuse
    double *h_rho[2] = {nullptr, nullptr}, *h_phi[2] = {nullptr, nullptr};
    cudaStream_t h_up = nullptr, h_down = nullptr;
    cudaEvent_t h_uploaded[2] = {nullptr, nullptr}, h_solved[2] = {nullptr, nullptr};
    cudaEvent_t h_downloaded[2] = {nullptr, nullptr};
    int h_slot = 0;
    const double *last_phi = nullptr;  // device buffer holding the last solve's Phi
    int *d_err = nullptr;
    int solved = 0;
    // radial-shell slab of a larger mesh: the other slabs' radial sums [2][K_L] (sum of
    // W^R A below this slab, sum of W^I A above it), added to the recurrences when
    // use_slab_off is set
    int slab = 0, use_slab_off = 0, slab_moments_ready = 0;
    double *d_slab_off = nullptr;

    // TMA descriptors, cached per bound pointer
    CUtensorMap tm_rho{}, tm_phi{};
    const void *tm_rho_ptr = nullptr, *tm_phi_ptr = nullptr;
    // the solve's kernel chain as CUDA graphs, one per (density, potential) binding in use
    // (captured on g_cap), least recently used replaced
    struct GraphSlot {
        const void *rho = nullptr, *phi = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long used = 0;
    };
    static constexpr int kGraphSlots = 4;
    GraphSlot g_slots[kGraphSlots];
    unsigned long long g_clock = 0;
    cudaStream_t g_cap = nullptr;

    // profiling
    int profiling = 0;
    int tuned_candidates = 0;  // configurations the last mp_autotune timed
    std::vector<std::pair<const char *, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::map<std::string, mp::ProfileEntry> prof;
    std::vector<cudaEvent_t> event_pool;

    size_t device_bytes = 0;
};

#ifndef MP_PDL_ALLOWED
#define MP_PDL_ALLOWED 1
#endif

namespace mp {

// error detail of the calling host thread
mp_status set_error(mp_status st, const char *fmt, ...);

// ---- tables (float64, on the device) ----
// Launch with programmatic stream serialization: the kernel may begin while
// the previous kernel on the stream finishes; it calls pdl_wait() (ptx.cuh)
// before it touches anything that kernel produced.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = MP_PDL_ALLOWED;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

cudaError_t launch_tables(mp_mesh *m);
cudaError_t launch_split_tables(mp_mesh *m);

// ---- float64 path ----
cudaError_t launch_fp64_project(mp_mesh *m, const double *rho);
cudaError_t launch_fp64_theta(mp_mesh *m);
cudaError_t launch_fp64_synth(mp_mesh *m, double *phi);
// step (a) in float64 with caller-provided workspace F [R][2L+1] and output A [n_r][K_L]
cudaError_t launch_fp64_moments_into(const mp_mesh *m, const double *rho, double *F, double *A);

// ---- shared radial recurrences ----
cudaError_t launch_scan(mp_mesh *m, int want_f32);
// the CUDA-core theta contraction keeps its tables in shared memory (its fast form)
bool theta_pipe_fits(const mp_mesh *m);

// ---- split path ----
cudaError_t launch_split_project(mp_mesh *m, const double *rho);
cudaError_t launch_split_theta(mp_mesh *m);
cudaError_t launch_split_synth(mp_mesh *m, double *phi);
int split_smem_limits(mp_mesh *m);  // 0 when the plan fits, else an error
// stage configurations of the phi synthesis (A stages, table residency / ring, staging boxes)
int synth_cfg_count();
bool synth_cfg_fits(const SplitPlan &pl, int k);
void synth_cfg_apply(SplitPlan &pl, int k);
std::vector<int> synth_cfg_order(const SplitPlan &pl);

// ---- tensor-core theta stages (orders m >= 1)
bool plan_theta_tc(mp_mesh *m, std::vector<unsigned long long> &th_off, size_t &th_bytes,
                   std::vector<unsigned long long> &gs_off, size_t &gs_bytes, std::vector<unsigned long long> &cb_off,
                   size_t &cb_bytes);
bool gsynth_plan_ns(mp_mesh *m, int ns, std::vector<unsigned long long> &cb_off, size_t &cb_bytes);
cudaError_t set_gsynth_ns(mp_mesh *m, int ns);
cudaError_t launch_theta_tc_tables(mp_mesh *m);
cudaError_t launch_theta_tc(mp_mesh *m);   // theta contraction, m >= 1
cudaError_t launch_gsynth_tc(mp_mesh *m);  // theta synthesis, m >= 1
// tiled TMA map of a float32 array of up to 3 dimensions (innermost first)
mp_status make_map_f32(CUtensorMap *map, const void *ptr, int rank, const unsigned long long *dims,
                       const unsigned long long *strides_bytes, const unsigned *box, int swizzle128);

// ---- gravitational source terms ----
cudaError_t gravity_prepare(mp_mesh *m);  // stencils from the host edges (once per mesh)
cudaError_t launch_gravity(mp_mesh *m, const double *phi, const double *rho, const double *v, double *grad,
                           double *S, double *E);

// ---- coarsening blocks ----
cudaError_t coarsen_prepare(mp_mesh *m);  // block sizes and work list from the host edges (once per mesh)
cudaError_t launch_coarsen(mp_mesh *m, double *fields, int n_fields, long long stride);

// profiling hooks used by the launchers
void prof_begin(mp_mesh *m, const char *name, cudaEvent_t *ev_start);
void prof_end(mp_mesh *m, const char *name, cudaEvent_t ev_start);

}  // namespace mp
