// Galerkin coarse operator K_H = P^T K P on the cell grid and its CG solver.
//
// P maps cell values (3 components per cell) to the free vertex DOFs of the
// lattice (each vertex gets 1/8 of the sum over the cells that contain it);
// P^T = R is the cell restriction of fcm_coarse.cu.  Because a vertex hat
// couples to the vertices of the neighbouring cells only, K_H has a 5x5x5
// cell stencil of 3x3 blocks.  It is assembled once by probing: for each of
// the 5^3 cell classes (c mod 5 per axis) and each component, P of the class
// indicator is multiplied by K and restricted; every restricted value then
// belongs to exactly one probed cell within distance 2.  375 applications
// of K in total.
//
// The coarse system K_H y = R r is solved approximately by a fixed number of
// block-Jacobi-preconditioned CG steps whose scalars stay on the device, from
// an initial guess (the learned network's prediction, or zero).  Storage and
// arithmetic are FP32 with FP64 dot products: the coarse solve is part of a
// preconditioner inside flexible CG, which tolerates its inexactness.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "fcm_device.cuh"

namespace fcm {

struct CoarseOp {
    int64_t ncell = 0;
    float *KH = nullptr;     // [cell][125][3][3]
    float *Dinv = nullptr;   // [cell][3][3] inverse of the diagonal block (0 where singular)
    float *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;  // 3 x ncell each, [comp][cell]
    double *partial = nullptr;
    unsigned *counter = nullptr;
    double *sc = nullptr;    // rz, pq, alpha, beta
};

namespace {

constexpr int RT = 256;
constexpr int NOFF = 125;

int nb(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// e[b][c] = 1 for the cells of class (ox, oy, oz) (c mod 5 per axis) and component b, else 0 (double cells)
__global__ void probe_cells_kernel(double *e, Grid3 g, int ox, int oy, int oz, int b, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.n[0]), cy = (int)((c / g.n[0]) % g.n[1]), cz = (int)(c / ((int64_t)g.n[0] * g.n[1]));
        const bool on = cx % 5 == ox && cy % 5 == oy && cz % 5 == oz;
        for (int a = 0; a < 3; ++a) e[a * ncell + c] = (on && a == b) ? 1.0 : 0.0;
    }
}

// y = P cells (double cells), s = 1
__global__ void prolong_d_kernel(const double *__restrict__ cells, const uint8_t *__restrict__ mask,
                                 double *__restrict__ y, Grid3 g, int p, int64_t nnode)
{
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
        for (int a = 0; a < 3; ++a) y[3 * node + a] = mask[3 * node + a] ? 0.125 * acc[a] : 0.0;
    }
}

// KH[c'][off][a][b] = (R K P e)[a][c'] for the probed cell c within distance 2 of c'
__global__ void probe_scatter_kernel(const double *__restrict__ v, const uint8_t *__restrict__ mask, float *KH, Grid3 g,
                                     int p, int ox, int oy, int oz, int b, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cc[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((int64_t)g.n[0] * g.n[1]))};
        const int o[3] = {ox, oy, oz};
        int off[3];
        bool ok = true;
        for (int ax = 0; ax < 3; ++ax) {
            int d = ((o[ax] - cc[ax]) % 5 + 5) % 5;  // 0..4
            if (d > 2) d -= 5;                       // -2..2
            off[ax] = d;
            const int t = cc[ax] + d;
            ok = ok && t >= 0 && t < g.n[ax];
        }
        if (!ok) continue;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 8; ++k) {
            const int64_t node = (int64_t)p * (cc[0] + (k & 1)) +
                                 (int64_t)g.M[0] * ((int64_t)p * (cc[1] + ((k >> 1) & 1)) + (int64_t)g.M[1] * p * (cc[2] + (k >> 2)));
            for (int a = 0; a < 3; ++a)
                if (mask[3 * node + a]) acc[a] += v[3 * node + a];
        }
        const int oi = (off[0] + 2) + 5 * ((off[1] + 2) + 5 * (off[2] + 2));
        for (int a = 0; a < 3; ++a) KH[((c * NOFF + oi) * 3 + a) * 3 + b] = (float)(0.125 * acc[a]);
    }
}

__global__ void diag_inverse_kernel(const float *KH, float *Dinv, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const float *A = KH + (c * NOFF + 62) * 9;  // offset (0,0,0)
        const double a = A[0], b = A[1], d = A[2], e = A[3], f = A[4], h = A[5], k = A[6], l = A[7], m = A[8];
        const double c00 = f * m - h * l, c01 = -(e * m - h * k), c02 = e * l - f * k;
        const double det = a * c00 + b * c01 + d * c02;
        const double tr = fabs(a) + fabs(f) + fabs(m);
        float *D = Dinv + c * 9;
        if (!(fabs(det) > 1e-30 * tr * tr * tr) || tr == 0.0) {
            for (int t = 0; t < 9; ++t) D[t] = 0.f;
            continue;
        }
        const double id = 1.0 / det;
        D[0] = (float)(c00 * id);
        D[1] = (float)(-(b * m - d * l) * id);
        D[2] = (float)((b * h - d * f) * id);
        D[3] = (float)(c01 * id);
        D[4] = (float)((a * m - d * k) * id);
        D[5] = (float)(-(a * h - d * e) * id);
        D[6] = (float)(c02 * id);
        D[7] = (float)(-(a * l - b * k) * id);
        D[8] = (float)((a * f - b * e) * id);
    }
}

// y = K_H x (FP32, [comp][cell])
__global__ void kh_apply_kernel(const float *__restrict__ KH, const float *__restrict__ x, float *__restrict__ y, Grid3 g,
                                int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.n[0]), cy = (int)((c / g.n[0]) % g.n[1]), cz = (int)(c / ((int64_t)g.n[0] * g.n[1]));
        float acc[3] = {0.f, 0.f, 0.f};
        const float *A = KH + c * NOFF * 9;
        for (int dz = -2; dz <= 2; ++dz) {
            const int zz = cz + dz;
            if (zz < 0 || zz >= g.n[2]) continue;
            for (int dy = -2; dy <= 2; ++dy) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= g.n[1]) continue;
                for (int dx = -2; dx <= 2; ++dx) {
                    const int xx = cx + dx;
                    if (xx < 0 || xx >= g.n[0]) continue;
                    const int64_t nc = xx + (int64_t)g.n[0] * (yy + (int64_t)g.n[1] * zz);
                    const float *B = A + ((dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2))) * 9;
                    const float x0 = x[nc], x1 = x[ncell + nc], x2 = x[2 * ncell + nc];
                    for (int a = 0; a < 3; ++a) acc[a] = fmaf(B[3 * a], x0, fmaf(B[3 * a + 1], x1, fmaf(B[3 * a + 2], x2, acc[a])));
                }
            }
        }
        for (int a = 0; a < 3; ++a) y[a * ncell + c] = acc[a];
    }
}

// z = Dinv r
__global__ void jacobi_kernel(const float *Dinv, const float *r, float *z, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const float *D = Dinv + c * 9;
        const float r0 = r[c], r1 = r[ncell + c], r2 = r[2 * ncell + c];
        for (int a = 0; a < 3; ++a) z[a * ncell + c] = D[3 * a] * r0 + D[3 * a + 1] * r1 + D[3 * a + 2] * r2;
    }
}

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double bsum(double v, double *sh)
{
    v = wsum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < RT / 32 ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32) v = wsum(v);
    __syncthreads();
    return v;
}

// mode 0: sc[0] = a.b (rz of the start);  mode 1: pq = a.b, alpha = rz / pq;
// mode 2: rz' = a.b, beta = rz' / rz, rz = rz'.  Deterministic two-level reduction.
__global__ void __launch_bounds__(RT) cdot_kernel(const float *a, const float *b, int64_t n, double *partial,
                                                   unsigned *counter, double *sc, int mode)
{
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    double x = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) x += (double)a[i] * b[i];
    x = bsum(x, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = x;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    x = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += RT) x += __ldcg(partial + i);
    x = bsum(x, sh);
    if (threadIdx.x == 0) {
        *counter = 0u;
        if (mode == 0) {
            sc[0] = x;
        } else if (mode == 1) {
            sc[1] = x;
            sc[2] = (x > 0.0 && isfinite(sc[0] / x)) ? sc[0] / x : 0.0;
        } else {
            sc[3] = (sc[0] > 0.0 && isfinite(x / sc[0])) ? x / sc[0] : 0.0;
            sc[0] = x;
        }
    }
}

// y += alpha p, r -= alpha q
__global__ void cupd_kernel(float *y, float *r, const float *p, const float *q, int64_t n, const double *sc)
{
    const float al = (float)sc[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        y[i] = fmaf(al, p[i], y[i]);
        r[i] = fmaf(-al, q[i], r[i]);
    }
}

// p = z + beta p (beta = 0 on the first call: p = z)
__global__ void cp_kernel(float *p, const float *z, int64_t n, const double *sc, int first)
{
    const float be = first ? 0.f : (float)sc[3];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : fmaf(be, p[i], z[i]);
}

// r = f - r  (r holds K_H y on entry)
__global__ void csub_kernel(const float *f, float *r, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) r[i] = f[i] - r[i];
}

}  // namespace

// Build the coarse operator once per context (375 applications of K).
fcm_status coarse_ensure(fcm_ctx *C)
{
    if (C->coarse) return FCM_OK;
    const int64_t ncell = C->hp.ncells, n3 = 3 * ncell;
    CoarseOp *op = new CoarseOp();
    op->ncell = ncell;
    auto fail = [&](cudaError_t e) {
        C->err = std::string("coarse operator: ") + cudaGetErrorString(e);
        coarse_free(op);
        return e == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&op->KH, sizeof(float) * ncell * NOFF * 9)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->Dinv, sizeof(float) * ncell * 9)) != cudaSuccess) return fail(e);
    float **vs[] = {&op->r, &op->z, &op->p, &op->q};
    for (float **v : vs)
        if ((e = cudaMalloc(v, sizeof(float) * n3)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->partial, sizeof(double) * 152 * 8)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->counter, sizeof(unsigned))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->sc, sizeof(double) * 4)) != cudaSuccess) return fail(e);
    cudaStream_t st = C->stream;
    cudaMemsetAsync(op->counter, 0, sizeof(unsigned), st);
    cudaMemsetAsync(op->KH, 0, sizeof(float) * ncell * NOFF * 9, st);
    double *ecell = nullptr;
    if ((e = cudaMalloc(&ecell, sizeof(double) * n3)) != cudaSuccess) return fail(e);
    // lattice scratch: the context's d_t (probe) and d_q (K times probe)
    for (int oz = 0; oz < 5; ++oz)
        for (int oy = 0; oy < 5; ++oy)
            for (int ox = 0; ox < 5; ++ox)
                for (int b = 0; b < 3; ++b) {
                    probe_cells_kernel<<<nb(ncell), 256, 0, st>>>(ecell, C->g, ox, oy, oz, b, ncell);
                    prolong_d_kernel<<<nb(C->nlat / 3), 256, 0, st>>>(ecell, C->d_mask, C->d_t, C->g, C->p, C->nlat / 3);
                    ctx_apply_K(C, C->d_t, C->d_q);
                    probe_scatter_kernel<<<nb(ncell), 256, 0, st>>>(C->d_q, C->d_mask, op->KH, C->g, C->p, ox, oy, oz, b,
                                                                     ncell);
                }
    diag_inverse_kernel<<<nb(ncell), 256, 0, st>>>(op->KH, op->Dinv, ncell);
    e = cudaStreamSynchronize(st);
    cudaFree(ecell);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return fail(e);
    C->coarse = op;
    return FCM_OK;
}

void coarse_free(CoarseOp *op)
{
    if (!op) return;
    void *ps[] = {op->KH, op->Dinv, op->r, op->z, op->p, op->q, op->partial, op->counter, op->sc};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete op;
}

// y <- approximate solution of K_H y = f after `iters` block-Jacobi CG steps from the given y
// (FP32 cells, [comp][cell]); asynchronous on the context's stream.
void coarse_solve(fcm_ctx *C, const float *f, float *y, int iters)
{
    CoarseOp *op = C->coarse;
    const int64_t n3 = 3 * op->ncell;
    cudaStream_t st = C->stream;
    const int rb = nb(n3);
    kh_apply_kernel<<<nb(op->ncell), 256, 0, st>>>(op->KH, y, op->r, C->g, op->ncell);
    csub_kernel<<<nb(n3), 256, 0, st>>>(f, op->r, n3);
    jacobi_kernel<<<nb(op->ncell), 256, 0, st>>>(op->Dinv, op->r, op->z, op->ncell);
    cp_kernel<<<nb(n3), 256, 0, st>>>(op->p, op->z, n3, op->sc, 1);
    cdot_kernel<<<rb, RT, 0, st>>>(op->r, op->z, n3, op->partial, op->counter, op->sc, 0);
    for (int i = 0; i < iters; ++i) {
        kh_apply_kernel<<<nb(op->ncell), 256, 0, st>>>(op->KH, op->p, op->q, C->g, op->ncell);
        cdot_kernel<<<rb, RT, 0, st>>>(op->p, op->q, n3, op->partial, op->counter, op->sc, 1);
        cupd_kernel<<<nb(n3), 256, 0, st>>>(y, op->r, op->p, op->q, n3, op->sc);
        if (i + 1 == iters) break;
        jacobi_kernel<<<nb(op->ncell), 256, 0, st>>>(op->Dinv, op->r, op->z, op->ncell);
        cdot_kernel<<<rb, RT, 0, st>>>(op->r, op->z, n3, op->partial, op->counter, op->sc, 2);
        cp_kernel<<<nb(n3), 256, 0, st>>>(op->p, op->z, n3, op->sc, 0);
    }
}

void coarse_apply(fcm_ctx *C, const float *x, float *y)
{
    kh_apply_kernel<<<nb(C->coarse->ncell), 256, 0, C->stream>>>(C->coarse->KH, x, y, C->g, C->coarse->ncell);
}

}  // namespace fcm

extern "C" fcm_status fcm_coarse_apply(fcm_ctx *C, const float *x_dev, float *y_dev)
{
    if (!C || !x_dev || !y_dev) return FCM_EINVAL;
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    fcm_status s = fcm::coarse_ensure(C);
    if (s == FCM_OK) fcm::coarse_apply(C, x_dev, y_dev);
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    if (s != FCM_OK) return s;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        C->err = std::string("fcm_coarse_apply: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    return FCM_OK;
}
