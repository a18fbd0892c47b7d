// mp_noalloc.cu -- angular moments of a density without allocating device memory.
//
// Some callers cannot allocate device memory at the point where they need the
// moments: code running while a CUDA graph is being captured (an allocation
// there either fails or becomes part of the graph), real-time loops whose
// memory budget is fixed up front, or plug-ins whose host application owns
// every device allocation.  mp_moments_noalloc serves them: it computes the
// angular moments of step (a) in float64 into the caller's buffer, and its one
// intermediate array -- the phi projection F[row][p] -- lives in a fixed
// file-scope device array instead of memory obtained from cudaMalloc.
//
// That array holds MP_NOALLOC_SCRATCH_DOUBLES float64 values (32 MiB); every GPU
// that loads this library keeps it until the process exits.  In host code the
// symbol g_noalloc_scratch is only a host-side stand-in for the device array,
// so the kernels get its device address, looked up once per device with
// cudaGetSymbolAddress while that device is current.  The lookup happens on
// the first call on each device, so that first call should come before any
// stream capture.  Every call shares the array: calls whose work overlaps on
// the GPU (different streams, or different meshes on one device running at
// once) race on it.  Each call writes every scratch value it later reads, so
// nothing in the array has to start at zero.
#include <mutex>

#include "mp_internal.h"

namespace mp {

namespace {

constexpr unsigned long long kScratchDoubles = MP_NOALLOC_SCRATCH_DOUBLES;
constexpr int kMaxDevices = 64;
constexpr double kFourPi = 12.566370614359172954;

__device__ __align__(256) double g_noalloc_scratch[MP_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {};

// phi projection of four rows per block into the scratch array (float64)
__global__ void __launch_bounds__(256) k_na_project(const double *__restrict__ rho, const double *__restrict__ Iph,
                                                    double *__restrict__ F, long long R, int n_p, int P, int *err)
{
    extern __shared__ double srow[];  // [4][n_p]
    const long long row0 = (long long)blockIdx.x * 4;
    const int nrows = (int)min(4LL, R - row0);
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

// theta contraction of one shell per block from the scratch array
__global__ void __launch_bounds__(256) k_na_theta(const double *__restrict__ F, const double *__restrict__ Ith,
                                                  double *__restrict__ A, int n_t, int KL, int P, double scale)
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

// Device address of the scratch array for the current device (looked up once).
mp_status scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(MP_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(MP_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return MP_OK;
}

}  // namespace

}  // namespace mp

extern "C" MP_API mp_status mp_moments_noalloc(const mp_mesh *mesh, const double *rho_dev, double *ang_dev)
{
    using namespace mp;
    if (!mesh || !rho_dev || !ang_dev) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    const unsigned long long need = (unsigned long long)mesh->R * mesh->P;
    if (need > kScratchDoubles)
        return set_error(MP_ERR_INVALID_ARG,
                         "n_r * n_theta * (2 l_max + 1) = %llu exceeds the fixed scratch of %llu float64 values", need,
                         kScratchDoubles);
    const size_t smem = (size_t)4 * mesh->n_p * sizeof(double);
    if (smem > 48 * 1024) return set_error(MP_ERR_UNSUPPORTED, "n_phi = %d exceeds 1536 for this entry point", mesh->n_p);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(MP_ERR_CUDA, "no CUDA device");
    if (prev != mesh->device && cudaSetDevice(mesh->device) != cudaSuccess)
        return set_error(MP_ERR_CUDA, "cannot select device %d", mesh->device);
    double *F = nullptr;
    mp_status st = scratch_address(mesh->device, &F);
    if (st == MP_OK) {
        const long long blocks = (mesh->R + 3) / 4;
        k_na_project<<<(unsigned)blocks, 256, smem, mesh->stream>>>(rho_dev, mesh->d_Iph, F, mesh->R, mesh->n_p,
                                                                    mesh->P, mesh->d_err);
        k_na_theta<<<mesh->n_r, 256, 0, mesh->stream>>>(F, mesh->d_Ith, ang_dev, mesh->n_t, mesh->KL, mesh->P,
                                                        kFourPi * mesh->G);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = set_error(MP_ERR_CUDA, "mp_moments_noalloc launch: %s", cudaGetErrorString(e));
    }
    if (prev != mesh->device) cudaSetDevice(prev);
    return st;
}
