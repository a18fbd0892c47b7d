// mp_api.cu -- the C ABI of include/multipole.h: argument checks, device
// memory, TMA descriptors, dispatch of the float64 and split-precision paths,
// per-kernel timing, graph-captured batches and the launch-parameter tuner.
#include <cudaTypedefs.h>

#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "mp_internal.h"

namespace mp {

namespace {
thread_local char g_detail[512] = "";
constexpr double kPi = 3.14159265358979323846;
}  // namespace

mp_status set_error(mp_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return st;
}

static mp_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MP_OK;
    cudaGetLastError();  // clear a sticky launch error of this thread
    return set_error(e == cudaErrorMemoryAllocation ? MP_ERR_OOM : MP_ERR_CUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

#define MP_TRY(call)                                        \
    do {                                                    \
        mp_status st_ = cuda_status((call), #call);         \
        if (st_ != MP_OK) return st_;                       \
    } while (0)

// ---------------------------------------------------------------- profiling
static cudaEvent_t pool_get(mp_mesh *m)
{
    if (!m->event_pool.empty()) {
        cudaEvent_t e = m->event_pool.back();
        m->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(mp_mesh *m, const char *name, cudaEvent_t *ev)
{
    (void)name;
    *ev = nullptr;
    if (!m->profiling) return;
    *ev = pool_get(m);
    cudaEventRecord(*ev, m->stream);
}

void prof_end(mp_mesh *m, const char *name, cudaEvent_t ev0)
{
    if (!m->profiling || !ev0) return;
    cudaEvent_t ev1 = pool_get(m);
    cudaEventRecord(ev1, m->stream);
    m->prof_pending.push_back({name, {ev0, ev1}});
}

static void prof_collect(mp_mesh *m)
{
    for (auto &pe : m->prof_pending) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
        ProfileEntry &e = m->prof[pe.first];
        e.name = pe.first;
        e.launches += 1;
        e.total_ms += ms;
        m->event_pool.push_back(pe.second.first);
        m->event_pool.push_back(pe.second.second);
    }
    m->prof_pending.clear();
}

// ---------------------------------------------------------------- TMA descriptors
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// [rows][cols] float64 in boxes of [box_rows][box_cols]: 16 columns with a 128-byte swizzle,
// 8 with a 64-byte one.
static mp_status make_map(CUtensorMap *map, const void *ptr, long long rows, int cols, int box_rows,
                          int box_cols = 16)
{
    auto fn = encode_fn();
    if (!fn) return set_error(MP_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (reinterpret_cast<uintptr_t>(ptr) & 15)
        return set_error(MP_ERR_INVALID_ARG, "split precision needs 16-byte aligned density/potential buffers");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(double)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(ptr), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                    box_cols == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MP_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MP_OK;
}

mp_status make_map_f32(CUtensorMap *map, const void *ptr, int rank, const unsigned long long *dims,
                       const unsigned long long *strides_bytes, const unsigned *box, int swizzle128)
{
    auto fn = encode_fn();
    if (!fn) return set_error(MP_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t d[3], st[2];
    cuuint32_t b[3], es[3] = {1u, 1u, 1u};
    for (int k = 0; k < rank; ++k) {
        d[k] = dims[k];
        b[k] = box[k];
        if (k + 1 < rank) st[k] = strides_bytes[k];
    }
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(ptr), d, st, b, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MP_ERR_CUDA, "cuTensorMapEncodeTiled (float32) failed (%d)", (int)r);
    return MP_OK;
}

// ---------------------------------------------------------------- helpers
static bool finite_increasing(const double *e, int n)
{
    for (int i = 0; i <= n; ++i)
        if (!std::isfinite(e[i])) return false;
    for (int i = 0; i < n; ++i)
        if (!(e[i + 1] > e[i])) return false;
    return true;
}

template <class T>
static mp_status dalloc(mp_mesh *m, T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(MP_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    m->device_bytes += count * sizeof(T);
    return MP_OK;
}

static void free_mesh_buffers(mp_mesh *m)
{
    void *ptrs[] = {m->d_r,   m->d_Ith,  m->d_dmu,    m->d_Iph,   m->d_Iphc,   m->d_WR,    m->d_WI,
                    m->d_GR,  m->d_GI,   m->d_V,      m->d_A,     m->d_MR,     m->d_MI,    m->d_C,
                    m->d_F64, m->d_G64,  m->d_F32,    m->d_C32,   m->d_Ith32, m->d_Itc32, m->d_Itc0, m->d_C0, m->d_colsum,
                    m->d_tabB, m->d_tabT, m->d_Aop, m->d_G0, m->phi_own, m->h_rho[0], m->h_rho[1],
                    m->h_phi[0], m->h_phi[1], m->d_err, m->d_gst, m->d_cwork, m->d_cweights, m->d_cgroups,
                    m->d_cchunks, m->d_cscratch, m->d_ccount, m->d_tabTh, m->d_tabGs, m->d_Cb, m->d_th_off,
                    m->d_gs_off, m->d_cb_off, m->d_slab_off};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &pe : m->prof_pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (cudaEvent_t e : m->event_pool) cudaEventDestroy(e);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

static void drop_graph(mp_mesh *m)
{
    for (auto &g : m->g_slots) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = mp_mesh::GraphSlot();
    }
}

static mp_status ensure_phi_own(mp_mesh *m)
{
    if (m->phi_own) return MP_OK;
    return dalloc(m, &m->phi_own, (size_t)m->N);
}

// Step (a): the angular moments of rho.
static mp_status run_moments(mp_mesh *m, const double *rho)
{
    if (m->eff_prec == MP_PREC_FP64) {
        MP_TRY(launch_fp64_project(m, rho));
        MP_TRY(launch_fp64_theta(m));
    } else {
        if (m->tm_rho_ptr != rho) {
            mp_status st = make_map(&m->tm_rho, rho, m->R, m->n_p, 128);
            if (st != MP_OK) return st;
            m->tm_rho_ptr = rho;
        }
        MP_TRY(launch_split_project(m, rho));
        MP_TRY(launch_split_theta(m));
    }
    return MP_OK;
}

// Steps (b)-(d): the radial recurrences (from the other slabs' sums when use_slab_off is
// set) and the potential.
static mp_status run_potential(mp_mesh *m, double *phi)
{
    if (m->eff_prec == MP_PREC_FP64) {
        MP_TRY(launch_scan(m, 0));
        MP_TRY(launch_fp64_synth(m, phi));
    } else {
        if (m->tm_phi_ptr != phi) {
            mp_status st = make_map(&m->tm_phi, phi, m->R, m->n_p, 32, m->plan.stg_cols);
            if (st != MP_OK) return st;
            m->tm_phi_ptr = phi;
        }
        MP_TRY(launch_scan(m, 1));
        MP_TRY(launch_split_synth(m, phi));
    }
    return MP_OK;
}

static mp_status run_solve(mp_mesh *m, const double *rho, double *phi)
{
    mp_status st = run_moments(m, rho);
    if (st != MP_OK) return st;
    st = run_potential(m, phi);
    if (st != MP_OK) return st;
    m->solved = 1;
    return MP_OK;
}

// The solve's kernel chain replayed as one CUDA graph launch on the mesh stream.
// A graph is captured on a private stream (the caller's stream may be the legacy
// default stream, which cannot be captured) per (density, potential) binding; a
// few bindings stay cached (the host round trips alternate two), the least
// recently used one is captured over.
static mp_status solve_graph(mp_mesh *m, const double *rho, double *phi)
{
    mp_mesh::GraphSlot *slot = nullptr;
    for (auto &g : m->g_slots)
        if (g.exec && g.rho == rho && g.phi == phi) slot = &g;
    if (!slot) {
        slot = &m->g_slots[0];
        for (auto &g : m->g_slots)
            if (!g.exec || g.used < slot->used) slot = &g;
        if (slot->exec) cudaGraphExecDestroy(slot->exec);
        if (slot->graph) cudaGraphDestroy(slot->graph);
        *slot = mp_mesh::GraphSlot();
        if (!m->g_cap) MP_TRY(cudaStreamCreateWithFlags(&m->g_cap, cudaStreamNonBlocking));
        cudaStream_t saved = m->stream;
        m->stream = m->g_cap;
        cudaError_t e = cudaStreamBeginCapture(m->g_cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            m->stream = saved;
            return cuda_status(e, "cudaStreamBeginCapture");
        }
        mp_status st = run_solve(m, rho, phi);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(m->g_cap, &g);
        m->stream = saved;
        if (st != MP_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&slot->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            slot->exec = nullptr;
            return cuda_status(e, "cudaGraphInstantiate");
        }
        slot->graph = g;
        slot->rho = rho;
        slot->phi = phi;
    }
    slot->used = ++m->g_clock;
    MP_TRY(cudaGraphLaunch(slot->exec, m->stream));
    return MP_OK;
}

static mp_status plan_split(mp_mesh *m)
{
    SplitPlan &pl = m->plan;
    pl.a_terms = (m->prec == MP_PREC_BF16X6) ? 3 : 2;
    pl.n_products = (m->prec == MP_PREC_BF16X6) ? 6 : 3;
    pl.Npad = round_up(m->P, 16);
    pl.n_kc = (m->n_p + 31) / 32;
    pl.Kpad = std::max(16, round_up(2 * m->L, 16));
    {
        // polar rows of F and the theta tables: whole float4 units plus an odd pad unit count,
        // so that consecutive rows start on different shared-memory banks
        const int nq = (m->n_t + 3) / 4;
        pl.ldF = 4 * ((nq % 2 == 0) ? nq + 1 : nq + 2);
    }
    {
        // synthesis column chunk NC (<= 256 accumulator columns): the CTAs take (tile, chunk)
        // units round-robin.  Take the widest NC in {256, 128, 64} that still gives every CTA
        // about 12 units or more (the last wave then costs at most about a twelfth), else 64:
        // wide chunks fetch a tile's A operand fewer times, narrow ones balance the CTAs.
        // Measured on GB300: 512 x 128 x 256 cells at l_max = 16 (512 tiles) ran the synthesis
        // in 27.1 / 28.6 / 28.9 us at NC = 64 / 128 / 256; 1024 x 256 x 512 cells at
        // l_max = 32 (2048 tiles) in 262 / 208 / 173 us.
        const long long n_tiles = (m->R + 127) / 128;
        const int nc_max = std::min(256, round_up(m->n_p, 16));
        pl.NC = nc_max;
        if (nc_max >= 64) {
            pl.NC = 64;
            for (int nc = 256; nc >= 128; nc /= 2) {
                if (nc > nc_max) continue;
                const long long units = n_tiles * ((m->n_p + nc - 1) / nc);
                if (units >= 12LL * m->num_sms) {
                    pl.NC = nc;
                    break;
                }
            }
        }
    }
    pl.n_nc = (m->n_p + pl.NC - 1) / pl.NC;
    // projection accumulators per tile: as many as tensor memory holds (up to 4), each chain of
    // float32 additions in the tensor core that many times shorter
    pl.proj_nacc_max = std::max(1, std::min(std::min(4, 256 / pl.Npad), pl.n_kc));
    pl.proj_nacc = pl.proj_nacc_max;
    pl.proj_ctas = m->num_sms;
    pl.synth_ctas = m->num_sms;
    if (split_smem_limits(m) != 0)
        return set_error(MP_ERR_UNSUPPORTED, "split-precision tiles of l_max = %d do not fit in shared memory", m->L);
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" {

int mp_version(void) { return 100; }

const char *mp_status_string(mp_status s)
{
    switch (s) {
    case MP_OK: return "MP_OK";
    case MP_ERR_INVALID_ARG: return "MP_ERR_INVALID_ARG: invalid argument";
    case MP_ERR_RANGE: return "MP_ERR_RANGE: radial kernels leave the float64 range";
    case MP_ERR_CUDA: return "MP_ERR_CUDA: CUDA runtime error";
    case MP_ERR_OOM: return "MP_ERR_OOM: out of memory";
    case MP_ERR_NOT_READY: return "MP_ERR_NOT_READY: no density bound";
    case MP_ERR_NONFINITE: return "MP_ERR_NONFINITE: density holds NaN or infinity";
    case MP_ERR_TIMEOUT: return "MP_ERR_TIMEOUT: a device-side wait gave up";
    case MP_ERR_UNSUPPORTED: return "MP_ERR_UNSUPPORTED: request not supported";
    }
    return "unknown mp_status";
}

mp_status mp_last_error_detail(char *buf, int len)
{
    if (!buf || len <= 0) return MP_ERR_INVALID_ARG;
    snprintf(buf, (size_t)len, "%s", g_detail);
    return MP_OK;
}

}  // extern "C"

// Mesh creation; r_ref_given > 0 fixes the reference radius of the radial kernels (a slab
// of a larger mesh takes the whole mesh's), otherwise sqrt(r_min+ r_max) of these edges.
static mp_status create_mesh(const double *r_edges, int n_r, const double *theta_edges, int n_theta,
                             const double *phi_edges, int n_phi, int l_max, double G, mp_precision prec,
                             void *cuda_stream, double r_ref_given, mp_mesh **out)
{
    g_detail[0] = 0;
    if (!out) return set_error(MP_ERR_INVALID_ARG, "out is NULL");
    if (!r_edges || !theta_edges || !phi_edges) return set_error(MP_ERR_INVALID_ARG, "edge array is NULL");
    if (n_r < 1 || n_theta < 1 || n_phi < 1) return set_error(MP_ERR_INVALID_ARG, "mesh needs at least one cell per dimension");
    if (l_max < 0 || l_max > 128) return set_error(MP_ERR_INVALID_ARG, "l_max must be in [0, 128]");
    if (!(G > 0.0) || !std::isfinite(G)) return set_error(MP_ERR_INVALID_ARG, "G must be positive and finite");
    if (prec != MP_PREC_FP64 && prec != MP_PREC_BF16X3 && prec != MP_PREC_BF16X6)
        return set_error(MP_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if ((long long)n_r * n_theta * (long long)n_phi > (1LL << 40))
        return set_error(MP_ERR_INVALID_ARG, "mesh too large");
    if (!finite_increasing(r_edges, n_r) || r_edges[0] < 0.0)
        return set_error(MP_ERR_INVALID_ARG, "radial edges must be finite, >= 0 and strictly increasing");
    if (!finite_increasing(theta_edges, n_theta) || theta_edges[0] < -1e-12 || theta_edges[n_theta] > kPi + 1e-12)
        return set_error(MP_ERR_INVALID_ARG, "polar edges must be strictly increasing within [0, pi]");
    if (!finite_increasing(phi_edges, n_phi) || phi_edges[n_phi] - phi_edges[0] > 2.0 * kPi * (1.0 + 1e-12))
        return set_error(MP_ERR_INVALID_ARG, "azimuthal edges must be strictly increasing and span at most 2 pi");
    if (prec != MP_PREC_FP64 && 2 * l_max + 1 > 256)
        return set_error(MP_ERR_UNSUPPORTED, "split precision supports l_max <= 127");

    // reference radius and float64 range of the scaled radial kernels
    const double rmin = r_edges[0] > 0.0 ? r_edges[0] : r_edges[1];
    const double rmax = r_edges[n_r];
    const double r_ref = r_ref_given > 0.0 ? r_ref_given : std::sqrt(rmin * rmax);
    {
        const double lx_hi = std::log10(rmax / r_ref), lx_lo = std::log10(rmin / r_ref), lr = std::log10(r_ref);
        const double e_reg = 3.0 * lr + (l_max + 3.0) * lx_hi;
        const double e_irr = 2.0 * lr + std::max(0.0, (l_max - 2.0)) * (-lx_lo);
        if (e_reg > 290.0 || e_irr > 290.0 || 3.0 * std::log10(rmax) > 300.0)
            return set_error(MP_ERR_RANGE, "r^l or r^-(l+1) over [%g, %g] at l_max = %d exceeds float64", rmin, rmax,
                             l_max);
    }

    mp_mesh *m = new (std::nothrow) mp_mesh();
    if (!m) return set_error(MP_ERR_OOM, "host allocation failed");
    m->n_r = n_r;
    m->n_t = n_theta;
    m->n_p = n_phi;
    m->L = l_max;
    m->KL = (l_max + 1) * (l_max + 1);
    m->P = 2 * l_max + 1;
    m->T = (l_max + 1) * (l_max + 2) / 2;
    m->R = (long long)n_r * n_theta;
    m->N = m->R * n_phi;
    m->G = G;
    m->r_ref = r_ref;
    m->prec = prec;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    m->h_r.assign(r_edges, r_edges + n_r + 1);
    m->h_th.assign(theta_edges, theta_edges + n_theta + 1);
    m->h_ph.assign(phi_edges, phi_edges + n_phi + 1);

    auto fail = [&](mp_status st) {
        free_mesh_buffers(m);
        delete m;
        return st;
    };
    if (cudaGetDevice(&m->device) != cudaSuccess) return fail(cuda_status(cudaGetLastError(), "cudaGetDevice"));
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, m->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, m->device);

    // split precision runs where its TMA tiles apply; otherwise float64
    m->eff_prec = prec;
    if (prec != MP_PREC_FP64 && (n_phi % 2 != 0 || n_phi < 16 || m->R < 128)) m->eff_prec = MP_PREC_FP64;
    if (m->eff_prec != MP_PREC_FP64 && !(major == 10 && minor == 3))
        return fail(set_error(MP_ERR_UNSUPPORTED, "split precision needs an sm_103 device (found sm_%d%d)", major, minor));

    const size_t nedges = (size_t)(n_r + 1) + (n_theta + 1) + (n_phi + 1);
    mp_status st;
#define ALLOC(ptr, count)                             \
    st = dalloc(m, &(ptr), (size_t)(count));          \
    if (st != MP_OK) return fail(st);
    ALLOC(m->d_r, nedges);
    ALLOC(m->d_Ith, (size_t)m->T * n_theta);
    ALLOC(m->d_dmu, n_theta);
    ALLOC(m->d_Iph, (size_t)m->P * n_phi);
    ALLOC(m->d_Iphc, (size_t)m->P * n_phi);
    ALLOC(m->d_WR, (size_t)(l_max + 1) * n_r);
    ALLOC(m->d_WI, (size_t)(l_max + 1) * n_r);
    ALLOC(m->d_GR, (size_t)(l_max + 1) * n_r);
    ALLOC(m->d_GI, (size_t)(l_max + 1) * n_r);
    ALLOC(m->d_V, n_r);
    ALLOC(m->d_A, (size_t)n_r * m->KL);
    ALLOC(m->d_MR, (size_t)(n_r + 1) * m->KL);
    ALLOC(m->d_MI, (size_t)(n_r + 1) * m->KL);
    ALLOC(m->d_C, (size_t)n_r * m->KL);
    ALLOC(m->d_err, 4);
    ALLOC(m->d_slab_off, (size_t)2 * m->KL);  // radial sums of the other slabs (slab meshes)  // [0] error word, [2..3] budget of the pipeline waits (int64, 0: default)
    if (m->eff_prec == MP_PREC_FP64) {
        ALLOC(m->d_F64, (size_t)m->R * m->P);
        ALLOC(m->d_G64, (size_t)m->R * m->P);
    } else {
        st = plan_split(m);
        if (st != MP_OK) return fail(st);
        const SplitPlan &pl = m->plan;
        ALLOC(m->d_F32, (size_t)n_r * m->P * pl.ldF);
        ALLOC(m->d_C32, (size_t)n_r * m->KL);
        ALLOC(m->d_Ith32, (size_t)m->T * pl.ldF);
        ALLOC(m->d_Itc32, (size_t)m->T * pl.ldF);
        ALLOC(m->d_Itc0, (size_t)(l_max + 1) * n_theta);
        ALLOC(m->d_C0, (size_t)n_r * (l_max + 1));
        ALLOC(m->d_colsum, pl.Npad);
        m->tabB_chunk_bytes = (size_t)3 * pl.Npad * 64;
        m->tabT_chunk_bytes = (size_t)3 * pl.NC * 32;
        ALLOC(m->d_tabB, m->tabB_chunk_bytes * pl.n_kc);
        ALLOC(m->d_tabT, m->tabT_chunk_bytes * pl.n_nc * (pl.Kpad / 16));
        {
            const size_t tiles = (size_t)((m->R + 127) / 128);
            ALLOC(m->d_Aop, tiles * pl.a_terms * 128 * pl.Kpad * 2);
            ALLOC(m->d_G0, tiles * 256);
            // rows past the last one in the final tile are never written by the theta synthesis
            cudaMemsetAsync(m->d_Aop, 0, tiles * pl.a_terms * 128 * pl.Kpad * 2, m->stream);
            cudaMemsetAsync(m->d_G0, 0, tiles * 256 * sizeof(float), m->stream);
            // padding cells of the polar rows stay zero: the theta contraction sums over them
            cudaMemsetAsync(m->d_F32, 0, (size_t)n_r * m->P * pl.ldF * sizeof(float), m->stream);
            cudaMemsetAsync(m->d_Ith32, 0, (size_t)m->T * pl.ldF * sizeof(float), m->stream);
            cudaMemsetAsync(m->d_Itc32, 0, (size_t)m->T * pl.ldF * sizeof(float), m->stream);
        }
        // orders m >= 1 of both theta stages on the tensor cores: pre-split tables, the
        // coefficient terms (zero padding never written), the 3-D TMA map of F
        std::vector<unsigned long long> th_off, gs_off, cb_off;
        size_t th_bytes = 0, gs_bytes = 0, cb_bytes = 0;
        if (plan_theta_tc(m, th_off, th_bytes, gs_off, gs_bytes, cb_off, cb_bytes)) {
            ALLOC(m->d_tabTh, th_bytes);
            ALLOC(m->d_tabGs, gs_bytes);
            ALLOC(m->d_Cb, cb_bytes);
            m->cb_bytes_alloc = cb_bytes;
            ALLOC(m->d_th_off, (size_t)(l_max + 1));
            ALLOC(m->d_gs_off, (size_t)(l_max + 1));
            ALLOC(m->d_cb_off, (size_t)(l_max + 1));
            st = cuda_status(cudaMemsetAsync(m->d_Cb, 0, cb_bytes, m->stream), "clear coefficient terms");
            if (st != MP_OK) return fail(st);
            const size_t ob = (size_t)(l_max + 1) * sizeof(unsigned long long);
            st = cuda_status(cudaMemcpy(m->d_th_off, th_off.data(), ob, cudaMemcpyHostToDevice), "table offsets");
            if (st == MP_OK)
                st = cuda_status(cudaMemcpy(m->d_gs_off, gs_off.data(), ob, cudaMemcpyHostToDevice), "table offsets");
            if (st == MP_OK)
                st = cuda_status(cudaMemcpy(m->d_cb_off, cb_off.data(), ob, cudaMemcpyHostToDevice), "table offsets");
            if (st != MP_OK) return fail(st);
            const unsigned long long dims[3] = {(unsigned long long)pl.ldF, (unsigned long long)m->P,
                                                (unsigned long long)n_r};
            const unsigned long long strides[2] = {(unsigned long long)pl.ldF * 4,
                                                   (unsigned long long)m->P * pl.ldF * 4};
            const unsigned box[3] = {32u, 1u, 64u};
            st = make_map_f32(&m->tm_F, m->d_F32, 3, dims, strides, box, 1);
            if (st != MP_OK) return fail(st);
        }
    }
#undef ALLOC
    {
        std::vector<double> edges;
        edges.reserve(nedges);
        edges.insert(edges.end(), r_edges, r_edges + n_r + 1);
        edges.insert(edges.end(), theta_edges, theta_edges + n_theta + 1);
        edges.insert(edges.end(), phi_edges, phi_edges + n_phi + 1);
        st = cuda_status(cudaMemcpyAsync(m->d_r, edges.data(), nedges * sizeof(double), cudaMemcpyHostToDevice,
                                         m->stream),
                         "copy edges");
        if (st != MP_OK) return fail(st);
        st = cuda_status(cudaMemsetAsync(m->d_err, 0, 4 * sizeof(int), m->stream), "clear error word");
        if (st != MP_OK) return fail(st);
        st = cuda_status(launch_tables(m), "build tables");
        if (st != MP_OK) return fail(st);
        if (m->eff_prec != MP_PREC_FP64) {
            st = cuda_status(launch_split_tables(m), "build split tables");
            if (st != MP_OK) return fail(st);
            st = cuda_status(launch_theta_tc_tables(m), "build tensor-core theta tables");
            if (st != MP_OK) return fail(st);
        }
        st = cuda_status(cudaStreamSynchronize(m->stream), "table build");
        if (st != MP_OK) return fail(st);
        st = cuda_status(gravity_prepare(m), "gravity stencils");
        if (st != MP_OK) return fail(st);
        st = cuda_status(coarsen_prepare(m), "coarsening blocks");
        if (st != MP_OK) return fail(st);
    }
    *out = m;
    return MP_OK;
}

extern "C" {

mp_status mp_mesh_create(const double *r_edges, int n_r, const double *theta_edges, int n_theta,
                         const double *phi_edges, int n_phi, int l_max, double G, mp_precision prec, void *cuda_stream,
                         mp_mesh **out)
{
    return create_mesh(r_edges, n_r, theta_edges, n_theta, phi_edges, n_phi, l_max, G, prec, cuda_stream, 0.0, out);
}

mp_status mp_mesh_create_slab(const double *r_edges, int n_r, int i0, int i1, const double *theta_edges,
                              int n_theta, const double *phi_edges, int n_phi, int l_max, double G, mp_precision prec,
                              void *cuda_stream, mp_mesh **out)
{
    g_detail[0] = 0;
    if (!r_edges || n_r < 1) return set_error(MP_ERR_INVALID_ARG, "radial edges of the whole mesh are missing");
    if (i0 < 0 || i1 > n_r || i1 <= i0) return set_error(MP_ERR_INVALID_ARG, "slab shells [%d, %d) outside [0, %d)", i0, i1, n_r);
    if (!finite_increasing(r_edges, n_r) || r_edges[0] < 0.0)
        return set_error(MP_ERR_INVALID_ARG, "radial edges must be finite, >= 0 and strictly increasing");
    const double rmin = r_edges[0] > 0.0 ? r_edges[0] : r_edges[1];
    mp_status st = create_mesh(r_edges + i0, i1 - i0, theta_edges, n_theta, phi_edges, n_phi, l_max, G, prec,
                               cuda_stream, std::sqrt(rmin * r_edges[n_r]), out);
    if (st != MP_OK) return st;
    (*out)->slab = 1;
    return MP_OK;
}

mp_status mp_mesh_destroy(mp_mesh *m)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    cudaStreamSynchronize(m->stream);
    if (m->h_up) cudaStreamSynchronize(m->h_up);
    if (m->h_down) cudaStreamSynchronize(m->h_down);
    drop_graph(m);
    if (m->g_cap) cudaStreamDestroy(m->g_cap);
    for (int b = 0; b < 2; ++b) {
        if (m->h_uploaded[b]) cudaEventDestroy(m->h_uploaded[b]);
        if (m->h_solved[b]) cudaEventDestroy(m->h_solved[b]);
        if (m->h_downloaded[b]) cudaEventDestroy(m->h_downloaded[b]);
    }
    if (m->h_up) cudaStreamDestroy(m->h_up);
    if (m->h_down) cudaStreamDestroy(m->h_down);
    free_mesh_buffers(m);
    delete m;
    return MP_OK;
}

mp_status mp_mesh_set_stream(mp_mesh *m, void *cuda_stream)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    MP_TRY(cudaStreamSynchronize(m->stream));
    if (m->profiling) prof_collect(m);
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    return MP_OK;
}

mp_status mp_mesh_get_info(const mp_mesh *m, mp_mesh_info *info)
{
    if (!m || !info) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    info->n_r = m->n_r;
    info->n_theta = m->n_t;
    info->n_phi = m->n_p;
    info->l_max = m->L;
    info->n_moments = m->KL;
    info->precision = m->prec;
    info->effective_precision = m->eff_prec;
    info->r_ref = m->r_ref;
    info->G = m->G;
    info->device_bytes = m->device_bytes;
    info->tuned_candidates = m->tuned_candidates;
    info->theta_tensor_cores = m->eff_prec != MP_PREC_FP64 ? m->plan.use_theta_tc : 0;
    return MP_OK;
}

mp_status mp_set_density(mp_mesh *m, const double *rho_dev)
{
    if (!m || !rho_dev) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    m->rho = rho_dev;
    return MP_OK;
}

mp_status mp_set_phi_output(mp_mesh *m, double *phi_dev)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    m->phi_user = phi_dev;
    return MP_OK;
}

mp_status mp_solve(mp_mesh *m)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (!m->rho) return set_error(MP_ERR_NOT_READY, "no density bound (mp_set_density)");
    DeviceGuard dg(m->device);
    double *phi = m->phi_user;
    if (!phi) {
        mp_status st = ensure_phi_own(m);
        if (st != MP_OK) return st;
        phi = m->phi_own;
    }
    m->last_phi = phi;
    // per-kernel timing needs events between the kernels: launch them one by one
    if (m->profiling) return run_solve(m, m->rho, phi);
    return solve_graph(m, m->rho, phi);
}

mp_status mp_get_phi(mp_mesh *m, double *phi_dev)
{
    if (!m || !phi_dev) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    if (!m->solved) return set_error(MP_ERR_NOT_READY, "no solve has run");
    const double *src = m->last_phi;
    if (src == phi_dev) return MP_OK;
    DeviceGuard dg(m->device);
    MP_TRY(cudaMemcpyAsync(phi_dev, src, (size_t)m->N * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    return MP_OK;
}

mp_status mp_gravity_sources(mp_mesh *m, const double *phi_dev, const double *rho_dev, const double *v_dev,
                             double *grad_dev, double *S_dev, double *E_dev)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (!grad_dev && !S_dev && !E_dev) return set_error(MP_ERR_INVALID_ARG, "no output requested");
    if (E_dev && !v_dev) return set_error(MP_ERR_INVALID_ARG, "the energy source needs the velocity");
    if (!phi_dev) {
        if (!m->solved || !m->last_phi) return set_error(MP_ERR_NOT_READY, "no solve has run");
        phi_dev = m->last_phi;
    }
    if (!rho_dev) {
        if (!m->rho) return set_error(MP_ERR_NOT_READY, "no density bound");
        rho_dev = m->rho;
    }
    DeviceGuard dg(m->device);
    MP_TRY(launch_gravity(m, phi_dev, rho_dev, v_dev, grad_dev, S_dev, E_dev));
    return MP_OK;
}

mp_status mp_coarsen(mp_mesh *m, double *fields_dev, int n_fields, long long field_stride)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (n_fields < 0 || n_fields > 65535) return set_error(MP_ERR_INVALID_ARG, "n_fields must be in [0, 65535]");
    if (n_fields == 0) return MP_OK;
    if (!fields_dev) return set_error(MP_ERR_INVALID_ARG, "fields_dev is NULL");
    if (n_fields > 1 && field_stride < m->N)
        return set_error(MP_ERR_INVALID_ARG, "field_stride must be at least n_r * n_theta * n_phi");
    DeviceGuard dg(m->device);
    MP_TRY(launch_coarsen(m, fields_dev, n_fields, field_stride));
    return MP_OK;
}

mp_status mp_coarsening_factors(const mp_mesh *m, int *c_theta, int *c_phi)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (c_theta) std::copy(m->h_ctheta.begin(), m->h_ctheta.end(), c_theta);
    if (c_phi) std::copy(m->h_cphi.begin(), m->h_cphi.end(), c_phi);
    return MP_OK;
}

mp_status mp_get_moments(mp_mesh *m, double *ang_dev, double *mr_dev, double *mi_dev)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (!m->solved) return set_error(MP_ERR_NOT_READY, "no solve has run");
    DeviceGuard dg(m->device);
    const size_t a = (size_t)m->n_r * m->KL * sizeof(double), e = (size_t)(m->n_r + 1) * m->KL * sizeof(double);
    if (ang_dev) MP_TRY(cudaMemcpyAsync(ang_dev, m->d_A, a, cudaMemcpyDeviceToDevice, m->stream));
    if (mr_dev) MP_TRY(cudaMemcpyAsync(mr_dev, m->d_MR, e, cudaMemcpyDeviceToDevice, m->stream));
    if (mi_dev) MP_TRY(cudaMemcpyAsync(mi_dev, m->d_MI, e, cudaMemcpyDeviceToDevice, m->stream));
    return MP_OK;
}

mp_status mp_mesh_synchronize(mp_mesh *m)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    MP_TRY(cudaStreamSynchronize(m->stream));
    if (m->h_up) MP_TRY(cudaStreamSynchronize(m->h_up));
    if (m->h_down) MP_TRY(cudaStreamSynchronize(m->h_down));
    int err = 0;
    MP_TRY(cudaMemcpy(&err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        MP_TRY(cudaMemset(m->d_err, 0, sizeof(int)));
        if (err & DEV_ERR_TIMEOUT) return set_error(MP_ERR_TIMEOUT, "a device-side pipeline wait ran out of time");
        if (err & DEV_ERR_NONFINITE) return set_error(MP_ERR_NONFINITE, "density holds NaN or infinity");
        return set_error(MP_ERR_CUDA, "device error word %d", err);
    }
    return MP_OK;
}

mp_status mp_slab_moments(mp_mesh *m, double *totals_dev)
{
    if (!m || !totals_dev) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    if (!m->rho) return set_error(MP_ERR_NOT_READY, "no density bound (mp_set_density)");
    DeviceGuard dg(m->device);
    mp_status st = run_moments(m, m->rho);
    if (st != MP_OK) return st;
    // the recurrences of this slab alone: its totals are M^R at its outer edge and M^I at its
    // inner edge
    m->use_slab_off = 0;
    MP_TRY(launch_scan(m, 0));
    const size_t kb = (size_t)m->KL * sizeof(double);
    MP_TRY(cudaMemcpyAsync(totals_dev, m->d_MR + (size_t)m->n_r * m->KL, kb, cudaMemcpyDeviceToDevice, m->stream));
    MP_TRY(cudaMemcpyAsync(totals_dev + m->KL, m->d_MI, kb, cudaMemcpyDeviceToDevice, m->stream));
    m->slab_moments_ready = 1;
    return MP_OK;
}

mp_status mp_slab_potential(mp_mesh *m, const double *outer_dev)
{
    if (!m || !outer_dev) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    if (!m->slab_moments_ready) return set_error(MP_ERR_NOT_READY, "mp_slab_moments has not run on this slab");
    DeviceGuard dg(m->device);
    double *phi = m->phi_user;
    if (!phi) {
        mp_status st = ensure_phi_own(m);
        if (st != MP_OK) return st;
        phi = m->phi_own;
    }
    MP_TRY(cudaMemcpyAsync(m->d_slab_off, outer_dev, (size_t)2 * m->KL * sizeof(double), cudaMemcpyDeviceToDevice,
                           m->stream));
    m->use_slab_off = 1;
    mp_status st = run_potential(m, phi);
    m->use_slab_off = 0;
    if (st != MP_OK) return st;
    m->last_phi = phi;
    m->solved = 1;
    m->slab_moments_ready = 0;
    return MP_OK;
}

mp_status mp_set_theta_engine(mp_mesh *m, int engine)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (engine < 0 || engine > 2) return set_error(MP_ERR_INVALID_ARG, "engine must be 0, 1 or 2");
    if (engine == 1 && !m->plan.theta_tc_ok)
        return set_error(MP_ERR_UNSUPPORTED, "the tensor-core theta stages need the split path and l_max >= 1");
    DeviceGuard dg(m->device);
    MP_TRY(cudaStreamSynchronize(m->stream));
    const int want = engine == 0 ? m->plan.theta_tc_default : (engine == 1 ? 1 : 0);
    if (want != m->plan.use_theta_tc) {
        m->plan.use_theta_tc = want;
        drop_graph(m);
    }
    return MP_OK;
}

mp_status mp_set_wait_budget(mp_mesh *m, long long cycles)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    const long long v = cycles > 0 ? cycles : 0;
    MP_TRY(cudaStreamSynchronize(m->stream));
    MP_TRY(cudaMemcpy(m->d_err + 2, &v, sizeof(v), cudaMemcpyHostToDevice));
    return MP_OK;
}

mp_status mp_solve_host_async(mp_mesh *m, const double *rho_host, double *phi_host)
{
    if (!m || !rho_host || !phi_host) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(m->device);
    if (!m->h_up) {
        MP_TRY(cudaStreamCreateWithFlags(&m->h_up, cudaStreamNonBlocking));
        MP_TRY(cudaStreamCreateWithFlags(&m->h_down, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            MP_TRY(cudaEventCreateWithFlags(&m->h_uploaded[b], cudaEventDisableTiming));
            MP_TRY(cudaEventCreateWithFlags(&m->h_solved[b], cudaEventDisableTiming));
            MP_TRY(cudaEventCreateWithFlags(&m->h_downloaded[b], cudaEventDisableTiming));
        }
    }
    const int b = m->h_slot;
    for (double **buf : {&m->h_rho[b], &m->h_phi[b]})
        if (!*buf) {
            mp_status st = dalloc(m, buf, (size_t)m->N);
            if (st != MP_OK) return st;
        }
    const size_t bytes = (size_t)m->N * sizeof(double);
    // upload into staging pair b once the solve that last read it has run
    MP_TRY(cudaStreamWaitEvent(m->h_up, m->h_solved[b], 0));
    MP_TRY(cudaMemcpyAsync(m->h_rho[b], rho_host, bytes, cudaMemcpyHostToDevice, m->h_up));
    MP_TRY(cudaEventRecord(m->h_uploaded[b], m->h_up));
    // solve on the mesh stream once the upload landed and the last download of pair b left
    MP_TRY(cudaStreamWaitEvent(m->stream, m->h_uploaded[b], 0));
    MP_TRY(cudaStreamWaitEvent(m->stream, m->h_downloaded[b], 0));
    mp_status st = m->profiling ? run_solve(m, m->h_rho[b], m->h_phi[b]) : solve_graph(m, m->h_rho[b], m->h_phi[b]);
    if (st != MP_OK) return st;
    m->last_phi = m->h_phi[b];
    MP_TRY(cudaEventRecord(m->h_solved[b], m->stream));
    // download on its own stream: it overlaps the next call's upload
    MP_TRY(cudaStreamWaitEvent(m->h_down, m->h_solved[b], 0));
    MP_TRY(cudaMemcpyAsync(phi_host, m->h_phi[b], bytes, cudaMemcpyDeviceToHost, m->h_down));
    MP_TRY(cudaEventRecord(m->h_downloaded[b], m->h_down));
    m->h_slot = b ^ 1;
    return MP_OK;
}

mp_status mp_solve_host(mp_mesh *m, const double *rho_host, double *phi_host)
{
    mp_status st = mp_solve_host_async(m, rho_host, phi_host);
    if (st != MP_OK) return st;
    return mp_mesh_synchronize(m);
}

mp_status mp_profile_enable(mp_mesh *m, int enable)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    cudaStreamSynchronize(m->stream);
    prof_collect(m);
    m->prof.clear();
    m->profiling = enable ? 1 : 0;
    return MP_OK;
}

mp_status mp_profile_read(mp_mesh *m, const char **names, int *launches, double *total_ms, int cap, int *n_out)
{
    if (!m || !n_out) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(m->device);
    MP_TRY(cudaStreamSynchronize(m->stream));
    prof_collect(m);
    int n = 0;
    for (auto &kv : m->prof) {
        if (n < cap) {
            if (names) names[n] = kv.second.name;
            if (launches) launches[n] = kv.second.launches;
            if (total_ms) total_ms[n] = kv.second.total_ms;
        }
        ++n;
    }
    *n_out = n;
    return MP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches
struct mp_batch {
#ifndef MP_BATCH_BRANCHES
#define MP_BATCH_BRANCHES 4
#endif
    static constexpr int kBranches = MP_BATCH_BRANCHES;  // parallel chains of meshes in the captured graph
    std::vector<mp_mesh *> meshes;
    std::vector<const void *> bound;  // rho / phi pointers the graph was captured with
    cudaStream_t stream = nullptr;    // caller's stream (that of the first mesh)
    cudaStream_t cap = nullptr;       // private stream the graph is captured on and runs on
    cudaStream_t side[kBranches] = {};                        // capture streams of the branches
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

static void batch_bindings(const mp_batch *b, std::vector<const void *> &out)
{
    out.clear();
    for (mp_mesh *m : b->meshes) {
        out.push_back(m->rho);
        out.push_back(m->phi_user ? m->phi_user : m->phi_own);
    }
}

extern "C" {

mp_status mp_batch_create(mp_mesh *const *meshes, int count, mp_batch **out)
{
    if (!meshes || count < 1 || !out) return set_error(MP_ERR_INVALID_ARG, "need count >= 1 meshes and out");
    for (int i = 0; i < count; ++i)
        if (!meshes[i]) return set_error(MP_ERR_INVALID_ARG, "mesh %d is NULL", i);
    for (int i = 1; i < count; ++i)
        if (meshes[i]->device != meshes[0]->device)
            return set_error(MP_ERR_INVALID_ARG, "all meshes of a batch must live on one device");
    mp_batch *b = new (std::nothrow) mp_batch();
    if (!b) return set_error(MP_ERR_OOM, "host allocation failed");
    b->meshes.assign(meshes, meshes + count);
    b->stream = meshes[0]->stream;
    b->device = meshes[0]->device;
    DeviceGuard dg(b->device);
    bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < mp_batch::kBranches && ok; ++k)
        ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        mp_status st = cuda_status(cudaGetLastError(), "batch streams/events");
        mp_batch_destroy(b);
        return st == MP_OK ? set_error(MP_ERR_CUDA, "batch streams/events") : st;
    }
    *out = b;
    return MP_OK;
}

mp_status mp_batch_solve(mp_batch *b)
{
    if (!b) return set_error(MP_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard dg(b->device);
    for (mp_mesh *m : b->meshes) {
        if (!m->rho) return set_error(MP_ERR_NOT_READY, "a mesh of the batch has no density bound");
        if (!m->phi_user) {
            mp_status st = ensure_phi_own(m);
            if (st != MP_OK) return st;
        }
    }
    std::vector<const void *> now;
    batch_bindings(b, now);
    if (b->exec && now != b->bound) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    if (!b->exec) {
        // eager first pass (builds TMA descriptors), then capture the batch
        std::vector<cudaStream_t> saved;
        std::vector<int> prof;
        // the meshes go to kBranches parallel chains of the graph, largest first, each to the
        // chain with the fewest cells so far: small meshes then share the SMs instead of each
        // leaving most of them idle between its kernels
        const int nb = std::min<int>(mp_batch::kBranches, (int)b->meshes.size());
        std::vector<int> order(b->meshes.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (double)b->meshes[x]->N * b->meshes[x]->KL > (double)b->meshes[y]->N * b->meshes[y]->KL;
        });
        std::vector<double> load(nb, 0.0);
        std::vector<int> branch(b->meshes.size(), 0);
        for (int i : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            branch[i] = k;
            load[k] += (double)b->meshes[i]->N * b->meshes[i]->KL;
        }
        for (size_t i = 0; i < b->meshes.size(); ++i) {
            mp_mesh *m = b->meshes[i];
            saved.push_back(m->stream);
            prof.push_back(m->profiling);
            m->stream = b->side[branch[i]];
            m->profiling = 0;
        }
        auto restore = [&] {
            for (size_t i = 0; i < b->meshes.size(); ++i) {
                b->meshes[i]->stream = saved[i];
                b->meshes[i]->profiling = prof[i];
            }
        };
        mp_status st = MP_OK;
        cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
        cudaError_t e = cudaStreamBeginCapture(b->cap, mode);
        if (e != cudaSuccess) {
            restore();
            return cuda_status(e, "cudaStreamBeginCapture");
        }
        // fork: every branch starts after the capture stream's start, and the capture stream
        // waits for every branch at the end
        e = cudaEventRecord(b->fork, b->cap);
        for (int k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
        if (e != cudaSuccess) st = cuda_status(e, "batch fork");
        for (size_t i = 0; i < b->meshes.size() && st == MP_OK; ++i) {
            mp_mesh *m = b->meshes[order[i]];
            m->last_phi = m->phi_user ? m->phi_user : m->phi_own;
            st = run_solve(m, m->rho, m->phi_user ? m->phi_user : m->phi_own);
        }
        for (int k = 0; k < nb; ++k) {
            cudaError_t e2 = cudaEventRecord(b->join[k], b->side[k]);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(b->cap, b->join[k], 0);
            if (e2 != cudaSuccess && st == MP_OK) st = cuda_status(e2, "batch join");
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap, &graph);
        restore();
        if (st != MP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_status(e, "cudaGraphInstantiate");
        }
        b->graph = graph;
        b->bound = now;
    }
    // order the replay after earlier work on the caller's stream, and later work after it
    MP_TRY(cudaEventRecord(b->ev_in, b->stream));
    MP_TRY(cudaStreamWaitEvent(b->cap, b->ev_in, 0));
    MP_TRY(cudaGraphLaunch(b->exec, b->cap));
    MP_TRY(cudaEventRecord(b->ev_out, b->cap));
    MP_TRY(cudaStreamWaitEvent(b->stream, b->ev_out, 0));
    return MP_OK;
}

mp_status mp_batch_destroy(mp_batch *b)
{
    if (!b) return set_error(MP_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard dg(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->cap) cudaStreamSynchronize(b->cap);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : {b->ev_in, b->ev_out, b->fork})
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < mp_batch::kBranches; ++k) {
        if (b->join[k]) cudaEventDestroy(b->join[k]);
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return MP_OK;
}

// ---------------------------------------------------------------- tuner
static std::string tune_key(const mp_mesh *m)
{
    std::ostringstream k;
    k << m->n_r << ' ' << m->n_t << ' ' << m->n_p << ' ' << m->L << ' ' << m->eff_prec;
    return k.str();
}

}  // extern "C"

// One point of the tuner's search space: density ring depth, synthesis stage configuration
// (synth_cfg_apply), threads per moment column of the recurrences, projection table
// residency, theta engine, theta synthesis shells per unit, projection accumulators.
struct TuneCfg {
    int ns_s, sy, sw, br, tc, gs_ns, nacc;
};

static TuneCfg current_cfg(const mp_mesh *m)
{
    const SplitPlan &p = m->plan;
    return {p.ns_s, p.synth_cfg, p.scan_threads, p.proj_b_resident, p.use_theta_tc, p.gs_NS, p.proj_nacc};
}

// Whether a configuration (a cache line, or a tuner candidate) fits this mesh's plan.
static bool cfg_fits(const mp_mesh *m, const TuneCfg &c)
{
    const SplitPlan &p = m->plan;
    if (!(c.sw == 64 || c.sw == 128 || c.sw == 256)) return false;
    if (m->eff_prec == MP_PREC_FP64) return true;
    // the density ring is even (the two converter groups alternate over its slots)
    return c.ns_s >= 2 && !(c.ns_s & 1) && c.ns_s <= p.ns_s_max && synth_cfg_fits(p, c.sy) &&
           (c.br ? p.proj_res_ok : p.proj_ring_ok) && (c.tc == 0 || p.theta_tc_ok) &&
           (c.gs_ns == 8 || c.gs_ns == 16 || c.gs_ns == 32) && c.nacc >= 1 && c.nacc <= p.proj_nacc_max;
}

static mp_status apply_cfg(mp_mesh *m, const TuneCfg &c)
{
    SplitPlan &p = m->plan;
    p.ns_s = c.ns_s;
    if (m->eff_prec != MP_PREC_FP64) {
        const int cols = p.stg_cols;
        synth_cfg_apply(p, c.sy);
        if (p.stg_cols != cols) m->tm_phi_ptr = nullptr;  // the Phi map's box follows the staging
    }
    p.scan_threads = c.sw;
    p.proj_b_resident = c.br;
    p.use_theta_tc = c.tc;
    p.proj_nacc = c.nacc;
    if (p.theta_tc_ok && c.gs_ns != p.gs_NS) MP_TRY(set_gsynth_ns(m, c.gs_ns));
    drop_graph(m);
    return MP_OK;
}

extern "C" {

mp_status mp_autotune(mp_mesh *m, const char *cache_path)
{
    if (!m) return set_error(MP_ERR_INVALID_ARG, "mesh is NULL");
    if (!m->rho) return set_error(MP_ERR_NOT_READY, "autotune needs a bound density");
    DeviceGuard dg(m->device);
    const std::string key = tune_key(m);
    // cached choice?
    if (cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream is(line);
            int a, b, c, d, e;
            TuneCfg t;
            std::string tag;  // lines of this format end in "s2"
            if (is >> a >> b >> c >> d >> e >> t.ns_s >> t.sy >> t.sw >> t.br >> t.tc >> t.gs_ns >> t.nacc >> tag &&
                tag == "s2") {
                std::ostringstream k;
                k << a << ' ' << b << ' ' << c << ' ' << d << ' ' << e;
                // a line that does not fit this plan's reserved memory is not used
                if (k.str() == key && cfg_fits(m, t)) {
                    mp_status st = apply_cfg(m, t);
                    if (st != MP_OK) return st;
                    m->tuned_candidates = 0;
                    return MP_OK;
                }
            }
        }
    }
    double *phi = m->phi_user;
    if (!phi) {
        mp_status st = ensure_phi_own(m);
        if (st != MP_OK) return st;
        phi = m->phi_own;
    }
    const SplitPlan base = m->plan;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_prof = m->profiling;
    m->profiling = 0;
    int timed = 0;
    // device time of three solves (after one warm-up) in configuration c
    auto time_cfg = [&](const TuneCfg &c, float *ms) -> mp_status {
        mp_status st = apply_cfg(m, c);
        if (st != MP_OK) return st;
        st = run_solve(m, m->rho, phi);
        if (st != MP_OK) return st;
        cudaEventRecord(e0, m->stream);
        for (int it = 0; it < 3 && st == MP_OK; ++it) st = run_solve(m, m->rho, phi);
        if (st != MP_OK) return st;
        cudaEventRecord(e1, m->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_status(cudaGetLastError(), "autotune timing");
        cudaEventElapsedTime(ms, e0, e1);
        ++timed;
        return MP_OK;
    };
    // Coordinate descent over the choices, most consequential first: the theta engine, the
    // theta synthesis shells per unit (a tile shape: N = 2 NS), the projection accumulators
    // per tile, the density ring depth with the table residency, the synthesis table ring,
    // the threads per moment column of the recurrences.  Each dimension is swept with the
    // others held at the best so far.
    TuneCfg best = current_cfg(m);
    float best_ms = FLT_MAX;
    mp_status st = time_cfg(best, &best_ms);
    auto sweep = [&](const std::vector<TuneCfg> &cands) {
        for (const TuneCfg &c : cands) {
            if (st != MP_OK) return;
            if (!cfg_fits(m, c)) continue;
            float ms = 0.0f;
            st = time_cfg(c, &ms);
            if (st == MP_OK && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    };
    std::vector<TuneCfg> cands;
    if (m->eff_prec != MP_PREC_FP64) {
        cands.clear();
        for (int tc = 0; tc <= base.theta_tc_ok; ++tc) cands.push_back({best.ns_s, best.sy, best.sw, best.br, tc, best.gs_ns, best.nacc});
        sweep(cands);
        if (best.tc) {
            cands.clear();
            for (int ns : {8, 16, 32}) cands.push_back({best.ns_s, best.sy, best.sw, best.br, best.tc, ns, best.nacc});
            sweep(cands);
        }
        cands.clear();
        for (int na = 1; na <= base.proj_nacc_max; ++na) cands.push_back({best.ns_s, best.sy, best.sw, best.br, best.tc, best.gs_ns, na});
        sweep(cands);
        cands.clear();
        for (int ns_s = 2; ns_s <= base.ns_s_max; ns_s += 2)
            for (int br = 0; br <= 1; ++br) cands.push_back({ns_s, best.sy, best.sw, br, best.tc, best.gs_ns, best.nacc});
        sweep(cands);
        cands.clear();
        for (int k = 0; k < synth_cfg_count(); ++k) cands.push_back({best.ns_s, k, best.sw, best.br, best.tc, best.gs_ns, best.nacc});
        sweep(cands);
    }
    cands.clear();
    for (int sw : {64, 128, 256}) cands.push_back({best.ns_s, best.sy, sw, best.br, best.tc, best.gs_ns, best.nacc});
    sweep(cands);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->profiling = saved_prof;
    m->tuned_candidates = timed;
    if (st != MP_OK) {
        m->plan = base;
        if (base.theta_tc_ok) set_gsynth_ns(m, base.gs_NS);
        drop_graph(m);
        return st;
    }
    st = apply_cfg(m, best);
    if (st != MP_OK) return st;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        f << key << ' ' << best.ns_s << ' ' << best.sy << ' ' << best.sw << ' ' << best.br << ' ' << best.tc << ' '
          << best.gs_ns << ' ' << best.nacc << " s2\n";
    }
    return mp_mesh_synchronize(m);
}

}  // extern "C"
