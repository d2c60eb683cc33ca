// fcm_apply_S_noalloc: the Schwarz apply with its scratch in static device memory.
//
// fcm_apply_S copies the caller's residual into a masked scratch vector owned
// by the context before the block apply.  Some callers cannot allocate device
// memory at the point where they apply the preconditioner: an application
// whose device memory is owned by its own pool allocator, or a real-time
// loop that forbids allocation once it is running, sets the context up at
// start-up and afterwards may only launch work on buffers that already exist.
// For them this entry point keeps the scratch vector in a file-scope
// __device__ array of fixed size instead, so the call itself allocates
// nothing (no cudaMalloc, no cudaFree, no allocating library routine).
//
// Limits and sharing rules:
//   * at most FCM_NOALLOC_MAX_LATTICE lattice DOFs (8 MiB of FP64 scratch that
//     every GPU loading the library holds until the process exits);
//   * every call on a device shares the one array, which keeps the last
//     call's contents; each call overwrites every entry it reads, so nothing
//     has to be cleared, but calls that overlap on the GPU (two streams, or
//     two contexts on different streams) race on it;
//   * the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "fcm_device.cuh"

namespace {

static __device__ __align__(256) double g_noalloc_scratch[FCM_NOALLOC_MAX_LATTICE];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" fcm_status fcm_apply_S_noalloc(fcm_ctx *C, const double *r_dev, double *z_dev)
{
    if (!C || !r_dev || !z_dev) return FCM_EINVAL;
    if (!C->have_precond) {
        C->err = "fcm_apply_S_noalloc: call fcm_precond_build first";
        return FCM_ESTATE;
    }
    if (C->nlat > (int64_t)FCM_NOALLOC_MAX_LATTICE) {
        C->err = "fcm_apply_S_noalloc: problem has " + std::to_string(C->nlat) +
                 " lattice DOFs, more than the static scratch holds (FCM_NOALLOC_MAX_LATTICE = " +
                 std::to_string((long long)FCM_NOALLOC_MAX_LATTICE) + "); use fcm_apply_S";
        return FCM_EINVAL;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        C->err = std::string("fcm_apply_S_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    fcm::launch_mask_copy(r_dev, scratch, C->d_mask, C->nlat, C->stream);
    fcm::launch_schwarz_apply(C->p, C->g, scratch, z_dev, C->d_f64, C->d_f32, C->plan,
                              nullptr, C->stream);
    e = cudaGetLastError();
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    if (e != cudaSuccess) {
        C->err = std::string("fcm_apply_S_noalloc: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    return FCM_OK;
}
