// mp_noalloc.cu -- angular moments of a density without allocating device memory.
//
// Some callers cannot allocate device memory at the point where they need the
// moments: real-time loops whose memory budget is fixed up front (an allocation
// mid-run can fail or stall), or plug-ins embedded in a host application that
// owns every device allocation and forbids them to call cudaMalloc.
// mp_moments_noalloc serves them: it computes the angular moments of step (a) in
// float64 into the caller's buffer with the float64 path's own kernels, and their
// one intermediate array -- the phi projection F[row][p] -- lives in a fixed
// file-scope device array instead of memory obtained from cudaMalloc.  A
// non-finite density sets the mesh's device error word, which the next
// mp_mesh_synchronize reports as MP_ERR_NONFINITE.
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

__device__ __align__(256) double g_noalloc_scratch[MP_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {};

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
    if (mesh->n_p > 1536) return set_error(MP_ERR_UNSUPPORTED, "n_phi = %d exceeds 1536 for this entry point", mesh->n_p);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return set_error(MP_ERR_CUDA, "no CUDA device");
    if (prev != mesh->device && cudaSetDevice(mesh->device) != cudaSuccess)
        return set_error(MP_ERR_CUDA, "cannot select device %d", mesh->device);
    double *F = nullptr;
    mp_status st = scratch_address(mesh->device, &F);
    if (st == MP_OK) {
        // the float64 path's own projection and theta contraction, with the fixed array as
        // their workspace
        const cudaError_t e = launch_fp64_moments_into(mesh, rho_dev, F, ang_dev);
        if (e != cudaSuccess) st = set_error(MP_ERR_CUDA, "mp_moments_noalloc launch: %s", cudaGetErrorString(e));
    }
    if (prev != mesh->device) cudaSetDevice(prev);
    return st;
}
