// Coarse transfer between lattice DOFs and the cell grid, and the flexible
// PCG that uses the learned coarse correction.
//
// R (restriction): cell value = mean of the vector at the 8 vertex nodes of
// the cell, per component.  P (prolongation) = R^T: a free vertex DOF
// receives 1/8 of the sum of the values of the cells that contain the vertex;
// higher-order DOFs receive nothing.
//
// The preconditioner of the flexible PCG is z = S r + gamma sigma P N(R r /
// sigma, eta), with S the Additive-Schwarz operator (Sec. 3.1 Eq. (5)) and N
// the U-Net.  Because N is nonlinear, each new search direction is
// K-orthogonalised explicitly against the last four (truncated flexible CG,
// Notay, SIAM J. Sci. Comput. 22, 2000).  Convergence is judged on ||S r|| / ||S b|| (Sec. 5 Eq. (14))
// with the plain Schwarz part, so the judge is the same as for plain PCG.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fcm_device.cuh"


namespace fcm {
namespace {

constexpr int RT = 256;

__global__ void restrict_kernel(const double *__restrict__ v, const uint8_t *__restrict__ mask, const float *__restrict__ eta,
                                float *__restrict__ out, Grid3 g, int p, float s, int with_eta, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.n[0]), cy = (int)((c / g.n[0]) % g.n[1]), cz = (int)(c / ((int64_t)g.n[0] * g.n[1]));
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 8; ++k) {
            const int64_t node = (int64_t)p * (cx + (k & 1)) +
                                 (int64_t)g.M[0] * ((int64_t)p * (cy + ((k >> 1) & 1)) + (int64_t)g.M[1] * p * (cz + (k >> 2)));
            for (int a = 0; a < 3; ++a)
                if (mask[3 * node + a]) acc[a] += v[3 * node + a];
        }
        for (int a = 0; a < 3; ++a) out[a * ncell + c] = (float)(0.125 * s * acc[a]);
        if (with_eta) out[3 * ncell + c] = eta[c];
    }
}

// y = s * P cells (scale s from host, or from *s_dev when non-null)
__global__ void prolong_kernel(const float *__restrict__ cells, const uint8_t *__restrict__ mask, double *__restrict__ y,
                               Grid3 g, int p, double s, const double *__restrict__ s_dev, int64_t nnode)
{
    const double sc = s_dev ? *s_dev : s;
    const int64_t ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nnode;
         node += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(node % g.M[0]), j = (int)((node / g.M[0]) % g.M[1]), k = (int)(node / ((int64_t)g.M[0] * g.M[1]));
        double acc[3] = {0.0, 0.0, 0.0};
        if (i % p == 0 && j % p == 0 && k % p == 0) {
            const int vi = i / p, vj = j / p, vk = k / p;
            for (int t = 0; t < 8; ++t) {
                const int cx = vi - 1 + (t & 1), cy = vj - 1 + ((t >> 1) & 1), cz = vk - 1 + (t >> 2);
                if (cx < 0 || cy < 0 || cz < 0 || cx >= g.n[0] || cy >= g.n[1] || cz >= g.n[2]) continue;
                const int64_t c = cx + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
                for (int a = 0; a < 3; ++a) acc[a] += cells[a * ncell + c];
            }
        }
        for (int a = 0; a < 3; ++a) y[3 * node + a] = mask[3 * node + a] ? 0.125 * sc * acc[a] : 0.0;
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < RT / 32 ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32) v = warp_sum(v);
    __syncthreads();
    return v;
}

// out[0] = a.b, out[1] = c.d (c may be null); deterministic two-level reduction.
__global__ void __launch_bounds__(RT) dot2_kernel(const double *a, const double *b, const double *c, const double *d,
                                                   int64_t n, double *partial, unsigned *counter, double *out)
{
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double x = 0.0, y = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        x = fma(a[i], b[i], x);
        if (c) y = fma(c[i], d[i], y);
    }
    x = block_sum(x, sh);
    y = block_sum(y, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = x;
        partial[2 * blockIdx.x + 1] = y;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    x = 0.0;
    y = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += RT) {
        x += __ldcg(partial + 2 * i);
        y += __ldcg(partial + 2 * i + 1);
    }
    x = block_sum(x, sh);
    y = block_sum(y, sh);
    if (threadIdx.x == 0) {
        out[0] = x;
        out[1] = y;
        *counter = 0u;
    }
}

// sum of squares of a float array into out[0] (single block, fixed order)
__global__ void __launch_bounds__(RT) sumsq_kernel(const float *a, int64_t n, double *out)
{
    __shared__ double sh[RT / 32];
    double x = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += RT) x += (double)a[i] * a[i];
    x = block_sum(x, sh);
    if (threadIdx.x == 0) out[0] = x;
}

__global__ void scale_f_kernel(float *a, int64_t n, float s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] *= s;
}

// x += alpha p, r -= alpha q
__global__ void axpy2_kernel(double *x, double *r, const double *p, const double *q, int64_t n, double alpha)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// z = a + b
__global__ void add_kernel(double *z, const double *a, const double *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) z[i] = a[i] + b[i];
}

// p = z + beta p
__global__ void xpby_kernel(double *p, const double *z, int64_t n, double beta)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = fma(beta, p[i], z[i]);
}

// y += a u (+ b v when v is non-null)
__global__ void xpby_acc_kernel(double *y, const double *u, double a, const double *v, double b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = fma(a, u[i], y[i]);
        if (v) t = fma(b, v[i], t);
        y[i] = t;
    }
}

// r = b - q (explicit residual)
__global__ void sub_kernel(double *r, const double *b, const double *q, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) r[i] = b[i] - q[i];
}

int nblk(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace
}  // namespace fcm

using namespace fcm;

namespace {

struct CoarseWs {
    double *z = nullptr, *c = nullptr, *red = nullptr;
    float *cin = nullptr, *cout = nullptr, *f = nullptr;
};

#define CO_CUDA(C, call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            (C)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return e_ == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;                    \
        }                                                                                       \
    } while (0)

fcm_status dot2(fcm_ctx *C, const double *a, const double *b, const double *c, const double *d, double *h2)
{
    dot2_kernel<<<C->red_blocks, RT, 0, C->stream>>>(a, b, c, d, C->nlat, C->d_partial, C->d_counter, C->d_out2);
    CO_CUDA(C, cudaMemcpyAsync(h2, C->d_out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
    CO_CUDA(C, cudaStreamSynchronize(C->stream));
    return FCM_OK;
}

// c = P y with y ~ K_H^-1 R r: the initial guess is gamma sigma N(R r / sigma, eta) (zero without a
// network), refined by `iters` coarse CG steps (iters = 0: the network's prediction alone).
fcm_status coarse_correction(fcm_ctx *C, fcm_unet *net, double gamma, int iters, const double *r, CoarseWs &ws,
                             double *c)
{
    const int64_t ncell = C->hp.ncells;
    cudaStream_t st = C->stream;
    restrict_kernel<<<nblk(ncell), 256, 0, st>>>(r, C->d_mask, C->d_eta, ws.cin, C->g, C->p, 1.0f, 1, ncell);
    if (net) {
        sumsq_kernel<<<1, RT, 0, st>>>(ws.cin, 3 * ncell, ws.red);
        double ss = 0.0;
        CO_CUDA(C, cudaMemcpyAsync(&ss, ws.red, sizeof(double), cudaMemcpyDeviceToHost, st));
        CO_CUDA(C, cudaStreamSynchronize(st));
        const double sigma = std::sqrt(ss / (3.0 * ncell));
        if (!(sigma > 0.0) || !std::isfinite(sigma)) {
            CO_CUDA(C, cudaMemsetAsync(c, 0, sizeof(double) * C->nlat, st));
            return FCM_OK;
        }
        CO_CUDA(C, cudaMemcpyAsync(ws.f, ws.cin, sizeof(float) * 3 * ncell, cudaMemcpyDeviceToDevice, st));
        scale_f_kernel<<<nblk(3 * ncell), 256, 0, st>>>(ws.cin, 3 * ncell, (float)(1.0 / sigma));
        fcm_status s = fcm_unet_forward(net, ws.cin, 1, C->g.n[0], C->g.n[1], C->g.n[2], ws.cout);
        if (s != FCM_OK) {
            C->err = "fcm_fpcg_solve: " + fcm_unet_last_error();
            return s;
        }
        scale_f_kernel<<<nblk(3 * ncell), 256, 0, st>>>(ws.cout, 3 * ncell, (float)(gamma * sigma));
    } else {
        CO_CUDA(C, cudaMemcpyAsync(ws.f, ws.cin, sizeof(float) * 3 * ncell, cudaMemcpyDeviceToDevice, st));
        CO_CUDA(C, cudaMemsetAsync(ws.cout, 0, sizeof(float) * 3 * ncell, st));
    }
    if (iters > 0) coarse_solve(C, ws.f, ws.cout, iters);
    prolong_kernel<<<nblk(C->nlat / 3), 256, 0, st>>>(ws.cout, C->d_mask, c, C->g, C->p, 1.0, nullptr, C->nlat / 3);
    CO_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

}  // namespace

extern "C" {

fcm_status fcm_coarse_restrict(fcm_ctx *C, const double *v, float s, int eta_channel, float *cells)
{
    if (!C || !v || !cells) return FCM_EINVAL;
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    const int64_t ncell = C->hp.ncells;
    restrict_kernel<<<nblk(ncell), 256, 0, C->stream>>>(v, C->d_mask, C->d_eta, cells, C->g, C->p, s, eta_channel, ncell);
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    CO_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_coarse_prolong(fcm_ctx *C, const float *cells, double s, double *y)
{
    if (!C || !cells || !y) return FCM_EINVAL;
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    prolong_kernel<<<nblk(C->nlat / 3), 256, 0, C->stream>>>(cells, C->d_mask, y, C->g, C->p, s, nullptr, C->nlat / 3);
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    CO_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_fpcg_solve(fcm_ctx *C, fcm_unet *net, double gamma, int coarse_iters, const double *rhs, double tol,
                          int maxit, double *u,
                          int *iterations, double *final_relres)
{
    if (!C || !rhs || !u || !(tol > 0.0) || maxit < 1 || !std::isfinite(gamma) || coarse_iters < 0 ||
        (!net && coarse_iters == 0)) {
        if (C) C->err = "fcm_fpcg_solve: invalid argument";
        return FCM_EINVAL;
    }
    if (!C->have_precond) {
        C->err = "fcm_fpcg_solve: call fcm_precond_build first";
        return FCM_ESTATE;
    }
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    cudaStream_t st = C->stream;
    const int64_t n = C->nlat, ncell = C->hp.ncells;
    CoarseWs ws;
    struct Free {
        CoarseWs &w;
        ~Free()
        {
            cudaFree(w.z);
            cudaFree(w.c);
            cudaFree(w.red);
            cudaFree(w.cin);
            cudaFree(w.cout);
            cudaFree(w.f);
        }
    } freer{ws};
    CO_CUDA(C, cudaMalloc(&ws.z, sizeof(double) * n));
    CO_CUDA(C, cudaMalloc(&ws.c, sizeof(double) * n));
    CO_CUDA(C, cudaMalloc(&ws.red, sizeof(double) * 2));
    CO_CUDA(C, cudaMalloc(&ws.cin, sizeof(float) * 4 * ncell));
    CO_CUDA(C, cudaMalloc(&ws.cout, sizeof(float) * 3 * ncell));
    CO_CUDA(C, cudaMalloc(&ws.f, sizeof(float) * 3 * ncell));
    if (coarse_iters > 0) {
        fcm_status se = coarse_ensure(C);
        if (se != FCM_OK) return se;
    }
    // the network runs on the solver's stream for the duration of the solve
    struct Restore {
        fcm_unet *n;
        cudaStream_t s;
        ~Restore()
        {
            if (n) unet_set_stream(n, s);
        }
    } restore{net, net ? unet_set_stream(net, st) : nullptr};

    cudaEventRecord(C->ev_t0, st);
    double *x = C->d_x, *r = C->d_r, *zS = C->d_z, *p = C->d_p, *q = C->d_q, *b = C->d_b;
    launch_mask_copy(rhs, b, C->d_mask, n, st);
    CO_CUDA(C, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CO_CUDA(C, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double h2[2];
    fcm_status s;
    if ((s = dot2(C, b, b, nullptr, nullptr, h2)) != FCM_OK) return s;
    if (!std::isfinite(h2[0])) {
        C->err = "fcm_fpcg_solve: right-hand side has non-finite entries";
        return FCM_EINVAL;
    }
    ctx_apply_S(C, r, zS);
    if ((s = dot2(C, zS, zS, nullptr, nullptr, h2)) != FCM_OK) return s;
    const double judge0 = std::sqrt(h2[0]);
    double rel = 0.0, best = 1.0, mark = 1.0;
    int it = 0, mark_it = 0;
    constexpr int kStallWindow = 100;
    bool converged = judge0 == 0.0, fallback = false;
    // truncated flexible CG, FCG(m) (Notay 2000): each new direction is K-orthogonalised
    // against the last kTrunc ones; ring of kTrunc + 1 direction slots (slot 0 = C->d_p/d_q)
    constexpr int kTrunc = 4, kRing = kTrunc + 1;
    double *P[kRing], *Q[kRing], pqs[kRing] = {0.0};
    P[0] = p;
    Q[0] = q;
    std::vector<double *> extra;
    struct FreeRing {
        std::vector<double *> &v;
        ~FreeRing()
        {
            for (double *a : v) cudaFree(a);
        }
    } free_ring{extra};
    for (int k = 1; k < kRing; ++k) {
        CO_CUDA(C, cudaMalloc(&P[k], sizeof(double) * n));
        extra.push_back(P[k]);
        CO_CUDA(C, cudaMalloc(&Q[k], sizeof(double) * n));
        extra.push_back(Q[k]);
    }
    if (!converged) {
        if ((s = coarse_correction(C, net, gamma, coarse_iters, r, ws, ws.c)) != FCM_OK) return s;
        add_kernel<<<nblk(n), 256, 0, st>>>(P[0], zS, ws.c, n);
        rel = 1.0;
    }
    while (!converged && !fallback && it < maxit) {
        const int cur = it % kRing;
        double *pc = P[cur], *qc = Q[cur];
        ctx_apply_K(C, pc, qc);
        if ((s = dot2(C, pc, qc, pc, r, h2)) != FCM_OK) return s;
        const double pq = h2[0], pr = h2[1];
        pqs[cur] = pq;
        ++it;
        if (!(pq > 0.0) || !std::isfinite(pr)) {
            fallback = true;
            break;
        }
        const double alpha = pr / pq;
        axpy2_kernel<<<nblk(n), 256, 0, st>>>(x, r, pc, qc, n, alpha);
        ctx_apply_S(C, r, zS);
        if ((s = dot2(C, zS, zS, nullptr, nullptr, h2)) != FCM_OK) return s;
        rel = std::sqrt(h2[0]) / judge0;
        if (!std::isfinite(rel)) {
            fallback = true;
            break;
        }
        best = std::min(best, rel);
        if (rel <= tol) {
            converged = true;
            break;
        }
        if (rel <= 0.5 * mark) {
            mark = rel;
            mark_it = it;
        }
        // a harmful or useless correction: growth, or no halving within kStallWindow iterations
        if (rel > 100.0 * best || it - mark_it >= kStallWindow) {
            fallback = true;
            break;
        }
        if ((s = coarse_correction(C, net, gamma, coarse_iters, r, ws, ws.c)) != FCM_OK) return s;
        add_kernel<<<nblk(n), 256, 0, st>>>(ws.z, zS, ws.c, n);
        // p_new = z - sum_j (z.q_j / p_j.q_j) p_j over the last min(it, kTrunc) directions
        const int nxt = it % kRing;
        CO_CUDA(C, cudaMemcpyAsync(P[nxt], ws.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        const int nprev = std::min(it, kTrunc);
        for (int j0 = 0; j0 < nprev; j0 += 2) {
            const int a = (it - 1 - j0 + kRing) % kRing;
            const int b2 = (it - 2 - j0 + kRing) % kRing;
            const bool two = j0 + 1 < nprev;
            if ((s = dot2(C, ws.z, Q[a], two ? ws.z : nullptr, two ? Q[b2] : nullptr, h2)) != FCM_OK) return s;
            xpby_acc_kernel<<<nblk(n), 256, 0, st>>>(P[nxt], P[a], -h2[0] / pqs[a], two ? P[b2] : nullptr,
                                                      two ? -h2[1] / pqs[b2] : 0.0, n);
        }
    }
    int total = it;
    fcm_status status = converged ? FCM_OK : FCM_ENOTCONV;
    if (fallback && it < maxit) {
        // plain Schwarz-PCG on K dx = b - K x, to the same absolute judged residual
        ctx_apply_K(C, x, q);
        sub_kernel<<<nblk(n), 256, 0, st>>>(ws.c, b, q, n);  // ws.c = explicit residual
        ctx_apply_S(C, ws.c, zS);
        if ((s = dot2(C, zS, zS, nullptr, nullptr, h2)) != FCM_OK) return s;
        const double jr = std::sqrt(h2[0]);
        CO_CUDA(C, cudaMemcpyAsync(ws.z, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));  // keep x
        fcm_solve_info inner = {};
        const double tol2 = jr > 0.0 ? std::min(1.0, tol * judge0 / jr) : 1.0;
        // the plain solve consumes its right-hand side first, so ws.c also receives dx
        fcm_status s2 = ctx_solve_one(C, ws.c, tol2, maxit - it, ws.c, inner);
        if (s2 == FCM_EINVAL || s2 == FCM_ECUDA || s2 == FCM_ENOMEM) return s2;
        add_kernel<<<nblk(n), 256, 0, st>>>(x, ws.z, ws.c, n);
        total += inner.iterations;
        rel = inner.relres * (jr / judge0);
        status = (fcm_status)inner.status;
        // ctx_solve_one left b = masked ws.c; restore the caller's b for the true residual
        launch_mask_copy(rhs, b, C->d_mask, n, st);
    }
    cudaEventRecord(C->ev_t1, st);
    CO_CUDA(C, cudaMemcpyAsync(u, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    ctx_apply_K(C, x, q);
    if ((s = dot2(C, b, b, nullptr, nullptr, h2)) != FCM_OK) return s;
    const double bb = h2[0];
    sub_kernel<<<nblk(n), 256, 0, st>>>(ws.c, b, q, n);
    if ((s = dot2(C, ws.c, ws.c, nullptr, nullptr, h2)) != FCM_OK) return s;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C->ev_t0, C->ev_t1);
    C->last.iterations = total;
    C->last.relres = rel;
    C->last.true_relres = bb > 0.0 ? std::sqrt(h2[0] / bb) : 0.0;
    C->last.status = status;
    C->last.seconds = ms * 1e-3;
    C->last.fallback = fallback ? 1 : 0;
    C->last.flexible_iterations = it;
    if (iterations) *iterations = total;
    if (final_relres) *final_relres = rel;
    cudaEventRecord(C->ev_out, st);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    if (status == FCM_ENOTCONV) C->err = "fcm_fpcg_solve: maxit reached";
    return status;
}

}  // extern "C"
