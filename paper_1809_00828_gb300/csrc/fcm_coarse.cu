// Coarse transfer between lattice DOFs and the cell grid, and the flexible
// PCG that uses the coarse correction.
//
// R (restriction): cell value = mean of the vector at the 8 vertex nodes of
// the cell, per component.  P (prolongation) = R^T: a free vertex DOF
// receives 1/8 of the sum of the values of the cells that contain the vertex;
// higher-order DOFs receive nothing.
//
// The preconditioner of the flexible PCG is z = S r + P y, with S the
// Additive-Schwarz operator (Sec. 3.1 Eq. (5)) and y an approximation of
// K_H^-1 R r (K_H = P^T K P): the U-Net's prediction gamma sigma N(R r / sigma,
// eta) (sigma the RMS of R r), scaled by the coarse energy-minimising step,
// refined by a few coarse CG steps (or those steps from zero without a
// network).  z depends nonlinearly on r, so each new search direction is
// K-orthogonalised explicitly against the last four (truncated flexible CG,
// FCG(4), Notay, SIAM J. Sci. Comput. 22, 2000).  Convergence is tested on
// ||S r|| / ||S b|| (Sec. 5 Eq. (14)) with the plain Schwarz part, so the
// stopping test is the same as for plain PCG.
//
// The iteration runs on the device: every scalar (alpha, the
// orthogonalisation coefficients, the convergence and stall tests) is
// computed by the last CTA of a deterministic two-level reduction, and every
// kernel returns at once when the device flag `stop` is set.  Four
// iterations are captured in one CUDA graph, kept on the context between
// solves; the host polls the flag once per graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "fcm_device.cuh"

namespace fcm {

constexpr int kM = 4;          // FCG(m): directions kept for the explicit K-orthogonalisation
constexpr double kL2Bytes = 129e6;  // GB300's L2
constexpr int kFcgChunk = 4;   // iterations per captured graph

struct FcgScalars {
    double pq[kM];     // p_j . K p_j, by ring slot
    double beta[kM];   // z . K p_j / pq_j for the j-th previous direction
    double alpha, sb_norm, rel, best, mark, tol, sigma;
    int it, maxit, mark_it, window, stop, status, fallback, pad;
};

struct FcgState {
    int64_t n = 0, ncell = 0;
    double *ring = nullptr;      // kM direction slots P, then kM slots Q = K P
    double *c = nullptr;         // P y on the lattice
    double *partial = nullptr;   // kM partials per CTA
    unsigned *counter = nullptr;
    float *cin = nullptr, *cout = nullptr, *f = nullptr;
    FcgScalars *d = nullptr, *h = nullptr;
    cudaGraphExec_t graph = nullptr;
    // the coarse correction without a network runs on `side`, beside the Schwarz apply (both read r only)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_r = nullptr, ev_c = nullptr;
    // what the graph was captured for
    uint64_t net_serial = 0, net_gen = 0;
    const fcm_unet *net = nullptr;
    double gamma = 0.0;
    int coarse_iters = -1;
};

// device address of the stop flag
const int *stop_flag(const FcgState *F)
{
    return reinterpret_cast<const int *>(reinterpret_cast<const char *>(F->d) + offsetof(FcgScalars, stop));
}

void fcg_forget_graph(FcgState *F)
{
    if (!F) return;
    if (F->graph) cudaGraphExecDestroy(F->graph);
    F->graph = nullptr;
    F->coarse_iters = -1;
}

void fcg_free(FcgState *F)
{
    if (!F) return;
    if (F->graph) cudaGraphExecDestroy(F->graph);
    void *ps[] = {F->ring, F->c, F->partial, F->counter, F->cin, F->cout, F->f, F->d};
    for (void *q : ps)
        if (q) cudaFree(q);
    if (F->h) cudaFreeHost(F->h);
    if (F->ev_r) cudaEventDestroy(F->ev_r);
    if (F->ev_c) cudaEventDestroy(F->ev_c);
    if (F->side) cudaStreamDestroy(F->side);
    delete F;
}

namespace {

constexpr int RT = 256;

#define STOP_RETURN \
    if (stop && *stop) return

__global__ void restrict_kernel(const double *__restrict__ v, const uint8_t *__restrict__ mask, const float *__restrict__ eta,
                                float *__restrict__ out, Grid3 g, int p, float s, int with_eta, int64_t ncell,
                                const int *stop)
{
    STOP_RETURN;
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

// y = s * P cells
__global__ void prolong_kernel(const float *__restrict__ cells, const uint8_t *__restrict__ mask, double *__restrict__ y,
                               Grid3 g, int p, double s, int64_t nnode, const int *stop)
{
    STOP_RETURN;
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
        for (int a = 0; a < 3; ++a) y[3 * node + a] = mask[3 * node + a] ? 0.125 * s * acc[a] : 0.0;
    }
}

// z += P cells on the free vertex DOFs (the only DOFs P reaches): one thread per vertex node, the 8
// cells around it summed in the same fixed order as prolong_kernel, so z + P y here equals the sum
// zS[i] + (P y)[i] formed from a separate prolongation
__global__ void prolong_add_kernel(const float *__restrict__ cells, const uint8_t *__restrict__ mask,
                                   double *__restrict__ z, Grid3 g, int p, const int *stop)
{
    STOP_RETURN;
    const int vx = g.n[0] + 1, vy = g.n[1] + 1, vz = g.n[2] + 1;
    const int64_t nv = (int64_t)vx * vy * vz, ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int vi = (int)(v % vx), vj = (int)((v / vx) % vy), vk = (int)(v / ((int64_t)vx * vy));
        double acc[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < 8; ++t) {
            const int cx = vi - 1 + (t & 1), cy = vj - 1 + ((t >> 1) & 1), cz = vk - 1 + (t >> 2);
            if (cx < 0 || cy < 0 || cz < 0 || cx >= g.n[0] || cy >= g.n[1] || cz >= g.n[2]) continue;
            const int64_t c = cx + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
            for (int a = 0; a < 3; ++a) acc[a] += cells[a * ncell + c];
        }
        const int64_t node = (int64_t)p * vi + (int64_t)g.M[0] * ((int64_t)p * vj + (int64_t)g.M[1] * p * vk);
        for (int a = 0; a < 3; ++a)
            if (mask[3 * node + a]) z[3 * node + a] += 0.125 * acc[a];
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; valid in thread 0.
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

// K sums over the grid in a fixed order: every CTA publishes its partials, the last CTA
// to arrive adds them up (thread 0 then holds the totals) and returns true.
template <int K>
__device__ bool grid_sums(double (&v)[K], double *partial, unsigned *counter)
{
    __shared__ double sh[RT / 32];
    __shared__ bool last;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = block_sum(v[k], sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partial[K * blockIdx.x + k] = v[k];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += RT) x += __ldcg(partial + K * i + k);
        v[k] = block_sum(x, sh);
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// sb_norm = ||S b||; resets the iteration state
__global__ void __launch_bounds__(RT) fk_first_kernel(const double *zS, int64_t n, double *partial, unsigned *counter,
                                                       FcgScalars *F)
{
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) v[0] = fma(zS[i], zS[i], v[0]);
    if (!grid_sums<1>(v, partial, counter) || threadIdx.x) return;
    const double j0 = sqrt(v[0]);
    F->sb_norm = j0;
    F->it = 0;
    F->rel = 1.0;
    F->best = 1.0;
    F->mark = 1.0;
    F->mark_it = 0;
    F->fallback = 0;
    F->status = FCM_OK;
    F->stop = 0;
    F->sigma = 0.0;
    if (!isfinite(j0)) {
        F->status = FCM_EBREAKDOWN;
        F->stop = 1;
    } else if (j0 == 0.0) {
        F->rel = 0.0;
        F->stop = 1;
    }
}

// pq = p.q, alpha = p.r / pq; stores p and q in the ring slot of this iteration
__global__ void __launch_bounds__(RT) fk_pq_kernel(const double *p, const double *q, const double *r, double *ring, int64_t n,
                                                    double *partial, unsigned *counter, FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    const int slot = F->it % kM;
    double *Ps = ring + (int64_t)slot * n, *Qs = ring + (int64_t)(kM + slot) * n;
    double v[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double pi = p[i], qi = q[i];
        v[0] = fma(pi, qi, v[0]);
        v[1] = fma(pi, r[i], v[1]);
        Ps[i] = pi;
        Qs[i] = qi;
    }
    if (!grid_sums<2>(v, partial, counter) || threadIdx.x) return;
    F->pq[slot] = v[0];
    const double alpha = v[1] / v[0];
    F->alpha = alpha;
    if (!(v[0] > 0.0) || !isfinite(alpha)) {
        F->fallback = 1;
        F->stop = 1;
    }
}

// x += alpha p, r -= alpha q
__global__ void __launch_bounds__(RT) fk_xr_kernel(double *x, double *r, const double *p, const double *q, int64_t n,
                                                    const FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    const double alpha = F->alpha;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// stopping residual ||S r|| / ||S b|| (Eq. (14)); convergence, growth, stall and iteration-limit tests
__global__ void __launch_bounds__(RT) fk_conv_kernel(const double *zS, int64_t n, double *partial, unsigned *counter,
                                                      FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) v[0] = fma(zS[i], zS[i], v[0]);
    if (!grid_sums<1>(v, partial, counter) || threadIdx.x) return;
    const int it = F->it + 1;
    F->it = it;
    const double rel = sqrt(v[0]) / F->sb_norm;
    F->rel = rel;
    if (!isfinite(rel)) {
        F->fallback = 1;
        F->stop = 1;
        return;
    }
    F->best = fmin(F->best, rel);
    if (rel <= F->tol) {
        F->status = FCM_OK;
        F->stop = 1;
        return;
    }
    if (rel <= 0.5 * F->mark) {
        F->mark = rel;
        F->mark_it = it;
    }
    // a harmful or useless correction: growth, or no halving within `window` iterations
    if (rel > 100.0 * F->best || it - F->mark_it >= F->window) {
        F->fallback = 1;
        F->stop = 1;
    } else if (it >= F->maxit) {
        F->status = FCM_ENOTCONV;
        F->stop = 1;
    }
}

// beta_j = z . q_j / pq_j over the last min(it, kM) directions (z = S r + P y)
__global__ void __launch_bounds__(RT) fk_dots_kernel(const double *zv, const double *ring, int64_t n,
                                                      double *partial, unsigned *counter, FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    const int it = F->it, np = min(it, kM);
    const double *Q[kM];
#pragma unroll
    for (int j = 0; j < kM; ++j) Q[j] = ring + (int64_t)(kM + (it - 1 - j + 2 * kM) % kM) * n;
    double v[kM] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        const double z = zv[i];
#pragma unroll
        for (int j = 0; j < kM; ++j)
            if (j < np) v[j] = fma(z, Q[j][i], v[j]);
    }
    if (!grid_sums<kM>(v, partial, counter) || threadIdx.x) return;
#pragma unroll
    for (int j = 0; j < kM; ++j) F->beta[j] = j < np ? v[j] / F->pq[(it - 1 - j + 2 * kM) % kM] : 0.0;
}

// p = z - sum_j beta_j p_j (z = S r + P y)
__global__ void __launch_bounds__(RT) fk_newp_kernel(double *p, const double *zv, const double *ring, int64_t n,
                                                      const FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    const int it = F->it, np = min(it, kM);
    const double *P[kM];
    double b[kM];
#pragma unroll
    for (int j = 0; j < kM; ++j) {
        P[j] = ring + (int64_t)((it - 1 - j + 2 * kM) % kM) * n;
        b[j] = j < np ? F->beta[j] : 0.0;
    }
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        double z = zv[i];
#pragma unroll
        for (int j = 0; j < kM; ++j)
            if (j < np) z = fma(-b[j], P[j][i], z);
        p[i] = z;
    }
}

// sigma = RMS of the 3 residual channels of the network input
__global__ void __launch_bounds__(RT) fk_sigma_kernel(const float *cin, int64_t n3, double *partial, unsigned *counter,
                                                       FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n3; i += (int64_t)gridDim.x * RT)
        v[0] += (double)cin[i] * cin[i];
    if (!grid_sums<1>(v, partial, counter) || threadIdx.x) return;
    const double s = sqrt(v[0] / (double)n3);
    F->sigma = isfinite(s) ? s : 0.0;
}

// f = R r (unscaled); the network input channels become R r / sigma
__global__ void fk_prep_kernel(float *cin, float *f, int64_t n3, const FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    const float inv = F->sigma > 0.0 ? (float)(1.0 / F->sigma) : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = cin[i];
        f[i] = v;
        cin[i] = v * inv;
    }
}

// network output times gamma sigma
__global__ void fk_post_kernel(float *cout, int64_t n3, double gamma, const FcgScalars *F)
{
    const int *stop = &F->stop;
    STOP_RETURN;
    const float s = (float)(gamma * F->sigma);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
        cout[i] *= s;
}

// out = a.b, c.d (c may be null); deterministic
__global__ void __launch_bounds__(RT) dot2_kernel(const double *a, const double *b, const double *c, const double *d,
                                                   int64_t n, double *partial, unsigned *counter, double *out)
{
    double v[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        v[0] = fma(a[i], b[i], v[0]);
        if (c) v[1] = fma(c[i], d[i], v[1]);
    }
    if (!grid_sums<2>(v, partial, counter) || threadIdx.x) return;
    out[0] = v[0];
    out[1] = v[1];
}

// z = a + b
__global__ void add_kernel(double *z, const double *a, const double *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) z[i] = a[i] + b[i];
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
    FcgState *F = C->fcg;
    dot2_kernel<<<C->red_blocks, RT, 0, C->stream>>>(a, b, c, d, C->nlat, F->partial, F->counter, C->d_out2);
    CO_CUDA(C, cudaMemcpyAsync(h2, C->d_out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
    CO_CUDA(C, cudaStreamSynchronize(C->stream));
    return FCM_OK;
}

fcm_status fcg_ensure(fcm_ctx *C)
{
    if (C->fcg) return FCM_OK;
    FcgState *F = new FcgState();
    F->n = C->nlat;
    F->ncell = C->hp.ncells;
    auto fail = [&](cudaError_t e) {
        C->err = std::string("flexible PCG workspace: ") + cudaGetErrorString(e);
        fcg_free(F);
        return e == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&F->side, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&F->ev_r, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&F->ev_c, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->ring, sizeof(double) * 2 * kM * F->n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->c, sizeof(double) * F->n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->partial, sizeof(double) * kM * 152 * 8)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->counter, sizeof(unsigned))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->cin, sizeof(float) * 4 * F->ncell)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->cout, sizeof(float) * 3 * F->ncell)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->f, sizeof(float) * 3 * F->ncell)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&F->d, sizeof(FcgScalars))) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&F->h, sizeof(FcgScalars))) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(F->counter, 0, sizeof(unsigned), C->stream)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(F->d, 0, sizeof(FcgScalars), C->stream)) != cudaSuccess) return fail(e);
    C->fcg = F;
    return FCM_OK;
}

// z += P y, y ~ K_H^-1 R r (see the file comment); every launch is stream-ordered and capturable
fcm_status coarse_correction(fcm_ctx *C, fcm_unet *net, double gamma, int iters)
{
    FcgState *F = C->fcg;
    const int64_t ncell = F->ncell, n3 = 3 * ncell;
    cudaStream_t st = C->stream;
    const int *stop = stop_flag(F);
    if (net) {
        restrict_kernel<<<nblk(ncell), 256, 0, st>>>(C->d_r, C->d_mask, C->d_eta, F->cin, C->g, C->p, 1.0f, 1, ncell, stop);
        fk_sigma_kernel<<<nblk(n3), RT, 0, st>>>(F->cin, n3, F->partial, F->counter, F->d);
        fk_prep_kernel<<<nblk(n3), 256, 0, st>>>(F->cin, F->f, n3, F->d);
        fcm_status s = fcm_unet_forward(net, F->cin, 1, C->g.n[0], C->g.n[1], C->g.n[2], F->cout);
        if (s != FCM_OK) {
            C->err = "fcm_fpcg_solve: " + fcm_unet_last_error();
            return s;
        }
        fk_post_kernel<<<nblk(n3), 256, 0, st>>>(F->cout, n3, gamma, F->d);
        coarse_solve(C, F->f, F->cout, iters, 2, stop);
    } else {
        restrict_kernel<<<nblk(ncell), 256, 0, st>>>(C->d_r, C->d_mask, C->d_eta, F->f, C->g, C->p, 1.0f, 0, ncell, stop);
        coarse_solve(C, F->f, F->cout, iters, 0, stop);
    }
    // z = zS + P y in place (zS's norm has been taken for the convergence test)
    const int64_t nv = (int64_t)(C->g.n[0] + 1) * (C->g.n[1] + 1) * (C->g.n[2] + 1);
    prolong_add_kernel<<<nblk(nv), 256, 0, st>>>(F->cout, C->d_mask, C->d_z, C->g, C->p, stop);
    return FCM_OK;
}

// one iteration: q = K p, x and r, zS = S r and its norm (the convergence test), c = P y, the next direction
fcm_status fcg_iteration(fcm_ctx *C, fcm_unet *net, double gamma, int iters)
{
    FcgState *F = C->fcg;
    cudaStream_t st = C->stream;
    const int64_t n = C->nlat;
    const int rb = C->red_blocks;
    const int *stop = stop_flag(F);
    ctx_apply_K_flag(C, C->d_p, C->d_q, stop);
    fk_pq_kernel<<<rb, RT, 0, st>>>(C->d_p, C->d_q, C->d_r, F->ring, n, F->partial, F->counter, F->d);
    fk_xr_kernel<<<rb, RT, 0, st>>>(C->d_x, C->d_r, C->d_p, C->d_q, n, F->d);
    // K_H in bytes: 63 stored 3x3 FP32 blocks per cell
    const double kh_bytes = (double)F->ncell * 63 * 9 * 4;
    if (!net && kh_bytes > kL2Bytes) {
        // R r and the coarse solve on the side stream while the Schwarz apply streams its factors; both
        // only read r, and they share no scratch (separate reduction buffers).  Only where K_H streams
        // from HBM anyway: a K_H that fits the L2 stays there across the coarse steps, and the Schwarz
        // apply's stream beside them would evict it.
        const int64_t ncell = F->ncell;
        CO_CUDA(C, cudaEventRecord(F->ev_r, st));
        CO_CUDA(C, cudaStreamWaitEvent(F->side, F->ev_r, 0));
        restrict_kernel<<<nblk(ncell), 256, 0, F->side>>>(C->d_r, C->d_mask, C->d_eta, F->f, C->g, C->p, 1.0f, 0, ncell,
                                                          stop);
        coarse_solve(C, F->f, F->cout, iters, 0, stop, F->side);
        CO_CUDA(C, cudaEventRecord(F->ev_c, F->side));
        ctx_apply_S_flag(C, C->d_r, C->d_z, stop);
        fk_conv_kernel<<<rb, RT, 0, st>>>(C->d_z, n, F->partial, F->counter, F->d);
        CO_CUDA(C, cudaStreamWaitEvent(st, F->ev_c, 0));
        const int64_t nv = (int64_t)(C->g.n[0] + 1) * (C->g.n[1] + 1) * (C->g.n[2] + 1);
        prolong_add_kernel<<<nblk(nv), 256, 0, st>>>(F->cout, C->d_mask, C->d_z, C->g, C->p, stop);
    } else {
        ctx_apply_S_flag(C, C->d_r, C->d_z, stop);
        fk_conv_kernel<<<rb, RT, 0, st>>>(C->d_z, n, F->partial, F->counter, F->d);
        fcm_status s = coarse_correction(C, net, gamma, iters);
        if (s != FCM_OK) return s;
    }
    fk_dots_kernel<<<rb, RT, 0, st>>>(C->d_z, F->ring, n, F->partial, F->counter, F->d);
    fk_newp_kernel<<<rb, RT, 0, st>>>(C->d_p, C->d_z, F->ring, n, F->d);
    return FCM_OK;
}

fcm_status fcg_graph(fcm_ctx *C, fcm_unet *net, double gamma, int iters)
{
    FcgState *F = C->fcg;
    uint64_t serial = 0, gen = 0;
    unet_identity(net, &serial, &gen);
    if (F->graph && F->net == net && F->net_serial == serial && F->net_gen == gen && F->gamma == gamma &&
        F->coarse_iters == iters)
        return FCM_OK;
    if (F->graph) cudaGraphExecDestroy(F->graph);
    F->graph = nullptr;
    CO_CUDA(C, cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal));
    fcm_status s = FCM_OK;
    for (int k = 0; k < kFcgChunk && s == FCM_OK; ++k) s = fcg_iteration(C, net, gamma, iters);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(C->stream, &graph);
    if (s != FCM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    CO_CUDA(C, e);
    e = cudaGraphInstantiate(&F->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        F->graph = nullptr;
        C->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    F->net = net;
    F->net_serial = serial;
    F->net_gen = gen;
    F->gamma = gamma;
    F->coarse_iters = iters;
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
    restrict_kernel<<<nblk(ncell), 256, 0, C->stream>>>(v, C->d_mask, C->d_eta, cells, C->g, C->p, s, eta_channel, ncell,
                                                        nullptr);
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
    prolong_kernel<<<nblk(C->nlat / 3), 256, 0, C->stream>>>(cells, C->d_mask, y, C->g, C->p, s, C->nlat / 3, nullptr);
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    CO_CUDA(C, cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_fpcg_set_stall_window(fcm_ctx *C, int window)
{
    if (!C) return FCM_EINVAL;
    if (window < 1) {
        C->err = "fcm_fpcg_set_stall_window: window must be >= 1";
        return FCM_EINVAL;
    }
    C->fcg_window = window;
    return FCM_OK;
}

fcm_status fcm_fpcg_solve(fcm_ctx *C, fcm_unet *net, double gamma, int coarse_iters, const double *rhs, double tol,
                          int maxit, double *u, int *iterations, double *final_relres)
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
    fcm_status s;
    if ((s = fcg_ensure(C)) != FCM_OK) return s;
    if ((s = coarse_ensure(C)) != FCM_OK) return s;
    FcgState *F = C->fcg;
    cudaStream_t st = C->stream;
    const int64_t n = C->nlat;
    // the network runs on the solver's stream for the duration of the solve
    struct Restore {
        fcm_unet *n;
        cudaStream_t s;
        ~Restore()
        {
            if (n) unet_set_stream(n, s);
        }
    } restore{net, net ? unet_set_stream(net, st) : nullptr};

    double *x = C->d_x, *r = C->d_r, *zS = C->d_z, *q = C->d_q, *b = C->d_b;
    CO_CUDA(C, cudaMemsetAsync(C->d_err, 0, sizeof(int), st));  // earlier fcm_apply_S failures are not this solve's
    launch_mask_copy(rhs, b, C->d_mask, n, st);
    double h2[2];
    if ((s = dot2(C, b, b, nullptr, nullptr, h2)) != FCM_OK) return s;
    if (!std::isfinite(h2[0])) {
        C->err = "fcm_fpcg_solve: right-hand side has non-finite entries";
        return FCM_EINVAL;
    }
    FcgScalars &h = *F->h;
    std::memset(&h, 0, sizeof h);
    h.tol = tol;
    h.maxit = maxit;
    h.window = C->fcg_window;
    CO_CUDA(C, cudaMemcpyAsync(F->d, &h, sizeof h, cudaMemcpyHostToDevice, st));
    CO_CUDA(C, cudaEventRecord(C->ev_f0, st));
    CO_CUDA(C, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CO_CUDA(C, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    ctx_apply_S_flag(C, r, zS, nullptr);
    fk_first_kernel<<<C->red_blocks, RT, 0, st>>>(zS, n, F->partial, F->counter, F->d);
    // first direction p = S r + P y (also the warm-up of the network's buffers before any capture)
    if ((s = coarse_correction(C, net, gamma, coarse_iters)) != FCM_OK) return s;
    fk_newp_kernel<<<C->red_blocks, RT, 0, st>>>(C->d_p, zS, F->ring, n, F->d);
    CO_CUDA(C, cudaGetLastError());
    if ((s = fcg_graph(C, net, gamma, coarse_iters)) != FCM_OK) return s;
    for (;;) {
        CO_CUDA(C, cudaMemcpyAsync(&h, F->d, sizeof h, cudaMemcpyDeviceToHost, st));
        CO_CUDA(C, cudaMemcpyAsync(C->h_err, C->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CO_CUDA(C, cudaStreamSynchronize(st));
        if (*C->h_err) {
            // a Schwarz apply gave up waiting for a factor copy: the iterate is not valid
            CO_CUDA(C, cudaMemsetAsync(C->d_err, 0, sizeof(int), st));
            C->err = "fcm_fpcg_solve: a Schwarz apply gave up waiting for a factor copy (bounded mbarrier wait)";
            C->last.status = FCM_ETIMEOUT;
            cudaEventRecord(C->ev_out, st);
            cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
            return FCM_ETIMEOUT;
        }
        if (h.stop) break;
        CO_CUDA(C, cudaGraphLaunch(F->graph, st));
    }
    const int it = h.it;
    const bool fallback = h.fallback != 0;
    const double sb_norm = h.sb_norm;
    double rel = h.rel;
    int total = it;
    fcm_status status = (fcm_status)h.status;
    if (fallback && it < maxit) {
        // plain Schwarz-PCG on K dx = b - K x, to the same absolute stopping residual
        double *res = F->c, *keep = F->ring;
        ctx_apply_K_flag(C, x, q, nullptr);
        sub_kernel<<<nblk(n), 256, 0, st>>>(res, b, q, n);
        ctx_apply_S_flag(C, res, zS, nullptr);
        if ((s = dot2(C, zS, zS, nullptr, nullptr, h2)) != FCM_OK) return s;
        const double jr = std::sqrt(h2[0]);
        CO_CUDA(C, cudaMemcpyAsync(keep, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        fcm_solve_info inner = {};
        const double tol2 = jr > 0.0 ? std::min(1.0, tol * sb_norm / jr) : 1.0;
        // the plain solve copies its right-hand side first, so `res` also receives dx
        fcm_status s2 = ctx_solve_one(C, res, tol2, maxit - it, res, inner);
        if (s2 == FCM_EINVAL || s2 == FCM_ECUDA || s2 == FCM_ENOMEM || s2 == FCM_ETIMEOUT) return s2;
        add_kernel<<<nblk(n), 256, 0, st>>>(x, keep, res, n);
        total += inner.iterations;
        rel = inner.relres * (jr / sb_norm);
        status = (fcm_status)inner.status;
        // the plain solve left b = masked res; restore the caller's b for the true residual
        launch_mask_copy(rhs, b, C->d_mask, n, st);
    } else if (fallback) {
        status = FCM_ENOTCONV;
    }
    cudaEventRecord(C->ev_f1, st);
    CO_CUDA(C, cudaMemcpyAsync(u, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    ctx_apply_K_flag(C, x, q, nullptr);
    if ((s = dot2(C, b, b, nullptr, nullptr, h2)) != FCM_OK) return s;
    const double bb = h2[0];
    sub_kernel<<<nblk(n), 256, 0, st>>>(F->c, b, q, n);
    if ((s = dot2(C, F->c, F->c, nullptr, nullptr, h2)) != FCM_OK) return s;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C->ev_f0, C->ev_f1);
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

fcm_status fcm_fpcg_solve_host(fcm_ctx *C, fcm_unet *net, double gamma, int coarse_iters, const double *rhs_host,
                               double tol, int maxit, double *u_host, int *iterations, double *final_relres)
{
    if (!C || !rhs_host || !u_host) {
        if (C) C->err = "fcm_fpcg_solve_host: invalid argument";
        return FCM_EINVAL;
    }
    if (!C->have_precond) {
        C->err = "fcm_fpcg_solve_host: call fcm_precond_build first";
        return FCM_ESTATE;
    }
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    // the coarse operator's assembly uses the scratch vector d_t: build it before the rhs goes there
    fcm_status s;
    if ((s = fcg_ensure(C)) != FCM_OK) return s;
    if ((s = coarse_ensure(C)) != FCM_OK) return s;
    CO_CUDA(C, cudaMemcpyAsync(C->d_t, rhs_host, sizeof(double) * C->nlat, cudaMemcpyHostToDevice, C->stream));
    // the device solve reads its right-hand side before it writes the solution, so both may be d_t
    s = fcm_fpcg_solve(C, net, gamma, coarse_iters, C->d_t, tol, maxit, C->d_t, iterations, final_relres);
    if (s == FCM_EINVAL || s == FCM_ECUDA || s == FCM_ENOMEM || s == FCM_ESTATE) return s;
    CO_CUDA(C, cudaMemcpyAsync(u_host, C->d_t, sizeof(double) * C->nlat, cudaMemcpyDeviceToHost, C->stream));
    CO_CUDA(C, cudaStreamSynchronize(C->stream));
    return s;
}

}  // extern "C"
