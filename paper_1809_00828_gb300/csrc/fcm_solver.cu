// Fused CG vector kernels of the preconditioned conjugate gradient method
// (PCG with x0 = 0, Sec. 5 of Jomo et al.: stopping on the relative
// preconditioned residual ||S r_i|| / ||S b||, Eq. (14)).
//
// All CG scalars stay on the device.  Every dot product is a deterministic
// two-level reduction: warp shuffles, one partial per CTA, and the last CTA to
// finish (ticket counter) sums the partials in a fixed order and performs the
// scalar part of the iteration (alpha, breakdown test, convergence test,
// beta).  Every kernel returns at once when the solve has finished, so a
// captured CUDA graph of several iterations can run past convergence for free.
#include <cuda_runtime.h>

#include "fcm_device.cuh"

namespace fcm {

namespace {

constexpr int RT = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = (threadIdx.x < RT / 32) ? sh[threadIdx.x] : 0.0;
    if (warp == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// Publishes the CTA partials and tells whether this CTA is the last one.
__device__ __forceinline__ bool publish(double a, double b, double *partial, unsigned *counter, bool *last)
{
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
        __threadfence();
        *last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return *last;
}

// Fixed-order sum of the partials (run by the last CTA only).
__device__ __forceinline__ void gather(const double *partial, double *sh, double &a, double &b)
{
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += RT) {
        x += __ldcg(partial + 2 * i);
        y += __ldcg(partial + 2 * i + 1);
    }
    a = block_sum(x, sh);
    b = block_sum(y, sh);
}

__global__ void __launch_bounds__(RT) init_kernel(double *x, double *r, const double *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        x[i] = 0.0;
        r[i] = b[i];
    }
}

// rz = r.z, zz0 = z.z, p = z; finishes at once when S b = 0 (then x = 0 is exact).
__global__ void __launch_bounds__(RT) first_kernel(const double *r, const double *z, double *p, int64_t n,
                                                    double *partial, unsigned *counter, CgScalars *S)
{
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double zi = z[i];
        a = fma(r[i], zi, a);
        b = fma(zi, zi, b);
        p[i] = zi;
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (!publish(a, b, partial, counter, &last)) return;
    gather(partial, sh, a, b);
    if (threadIdx.x == 0) {
        *counter = 0u;
        S->rz = a;
        S->zz0 = b;
        S->zz = b;
        S->relres = 1.0;
        S->it = 0;
        S->status = FCM_OK;
        S->done = 0;
        if (!(b == b) || !(a == a)) {
            S->status = FCM_EBREAKDOWN;
            S->done = 1;
        } else if (b == 0.0) {
            S->relres = 0.0;
            S->done = 1;
        }
    }
}

// pq = p.q and alpha = rz / pq; breakdown when pq <= 0 or alpha is not finite.
__global__ void __launch_bounds__(RT) pq_kernel(const double *p, const double *q, int64_t n, double *partial,
                                                 unsigned *counter, CgScalars *S)
{
    if (S->done) return;
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double a = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) a = fma(p[i], q[i], a);
    a = block_sum(a, sh);
    if (!publish(a, 0.0, partial, counter, &last)) return;
    double b;
    gather(partial, sh, a, b);
    if (threadIdx.x == 0) {
        *counter = 0u;
        S->pq = a;
        const double alpha = S->rz / a;
        S->alpha = alpha;
        if (!(a > 0.0) || !isfinite(alpha)) {
            S->status = FCM_EBREAKDOWN;
            S->done = 1;
        }
    }
}

// x += alpha p, r -= alpha q
__global__ void __launch_bounds__(RT) xr_kernel(double *x, double *r, const double *p, const double *q, int64_t n,
                                                 const CgScalars *S)
{
    if (S->done) return;
    const double alpha = S->alpha;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// rz' = r.z, zz = z.z; convergence on sqrt(zz / zz0) <= tol (Eq. (14)); beta = rz' / rz.
__global__ void __launch_bounds__(RT) rz_kernel(const double *r, const double *z, int64_t n, double *partial,
                                                 unsigned *counter, CgScalars *S)
{
    if (S->done) return;
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double zi = z[i];
        a = fma(r[i], zi, a);
        b = fma(zi, zi, b);
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (!publish(a, b, partial, counter, &last)) return;
    gather(partial, sh, a, b);
    if (threadIdx.x == 0) {
        *counter = 0u;
        S->zz = b;
        S->it += 1;
        const double rel = sqrt(b / S->zz0);
        S->relres = rel;
        const double beta = a / S->rz;
        S->beta = beta;
        S->rz = a;
        if (!(rel == rel) || !isfinite(beta)) {
            S->status = FCM_EBREAKDOWN;
            S->done = 1;
        } else if (rel <= S->tol) {
            S->status = FCM_OK;
            S->done = 1;
        } else if (S->it >= S->maxit) {
            S->status = FCM_ENOTCONV;
            S->done = 1;
        }
    }
}

// p = z + beta p
__global__ void __launch_bounds__(RT) p_kernel(double *p, const double *z, int64_t n, const CgScalars *S)
{
    if (S->done) return;
    const double beta = S->beta;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) p[i] = fma(beta, p[i], z[i]);
}

// out2 = (||b - Kx||^2, ||b||^2) with Kx in kx.
__global__ void __launch_bounds__(RT) resid_kernel(const double *kx, const double *b, int64_t n, double *partial,
                                                    unsigned *counter, double *out2)
{
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double a = 0.0, c = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double d = b[i] - kx[i];
        a = fma(d, d, a);
        c = fma(b[i], b[i], c);
    }
    a = block_sum(a, sh);
    c = block_sum(c, sh);
    if (!publish(a, c, partial, counter, &last)) return;
    gather(partial, sh, a, c);
    if (threadIdx.x == 0) {
        *counter = 0u;
        out2[0] = a;
        out2[1] = c;
    }
}

}  // namespace

void cg_init_kernels(const CgWork &w, cudaStream_t s)
{
    init_kernel<<<w.red_blocks, RT, 0, s>>>(w.x, w.r, w.b, w.n);
}

void cg_after_first_S(const CgWork &w, cudaStream_t s)
{
    first_kernel<<<w.red_blocks, RT, 0, s>>>(w.r, w.z, w.p, w.n, w.partial, w.counter, w.s);
}

void cg_after_K(const CgWork &w, cudaStream_t s)
{
    pq_kernel<<<w.red_blocks, RT, 0, s>>>(w.p, w.q, w.n, w.partial, w.counter, w.s);
    xr_kernel<<<w.red_blocks, RT, 0, s>>>(w.x, w.r, w.p, w.q, w.n, w.s);
}

void cg_after_S(const CgWork &w, cudaStream_t s)
{
    rz_kernel<<<w.red_blocks, RT, 0, s>>>(w.r, w.z, w.n, w.partial, w.counter, w.s);
    p_kernel<<<w.red_blocks, RT, 0, s>>>(w.p, w.z, w.n, w.s);
}

void cg_residual_norms(const CgWork &w, const double *kx, const double *b, double *out2, cudaStream_t s)
{
    resid_kernel<<<w.red_blocks, RT, 0, s>>>(kx, b, w.n, w.partial, w.counter, out2);
}

}  // namespace fcm
