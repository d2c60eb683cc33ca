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
//   * host code cannot use the array's name as a device address (in host code
//     it names a host-side shadow).  fcm_precond_build looks the device
//     address up with cudaGetSymbolAddress, with the context's device current
//     and outside any stream capture, and keeps it in the context, so the
//     address lives exactly as long as the context's own device allocations.
#include <cuda_runtime.h>

#include "fcm_device.cuh"

namespace {

static __device__ __align__(256) double g_noalloc_scratch[FCM_NOALLOC_MAX_LATTICE];

}  // namespace

namespace fcm {

// Device address of the scratch array on the current device.
cudaError_t noalloc_scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    *out = e == cudaSuccess ? static_cast<double *>(p) : nullptr;
    return e;
}

}  // namespace fcm

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
    double *scratch = C->noalloc_scratch;
    if (!scratch) {
        C->err = "fcm_apply_S_noalloc: the static scratch address was not found at fcm_precond_build (" +
                 C->noalloc_err + ")";
        return FCM_ECUDA;
    }
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    fcm::launch_mask_copy(r_dev, scratch, C->d_mask, C->nlat, C->stream);
    fcm::launch_schwarz_apply(C->p, C->g, scratch, z_dev, C->d_f64, C->d_f32, C->plan,
                              nullptr, C->stream);
    const cudaError_t e = cudaGetLastError();
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    if (e != cudaSuccess) {
        C->err = std::string("fcm_apply_S_noalloc: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    return FCM_OK;
}
