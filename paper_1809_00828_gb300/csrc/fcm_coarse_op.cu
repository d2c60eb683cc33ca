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
// an initial guess: zero, or the learned network's prediction scaled by the
// step t = f.y0 / y0.K_H y0 that minimises the coarse energy along y0 (so the
// start is never worse than zero in the K_H norm).  Storage and arithmetic are
// FP32 with FP64 dot products: the coarse solve is part of a preconditioner
// inside flexible CG, which tolerates its inexactness.  K_H is symmetric, so
// only the 63 blocks of the offsets from (0,0,0) on (in z, y, x order) are
// stored, as structure of arrays, KH[(s * 9 + 3 a + b) * n_cells + cell], so
// that consecutive threads (cells) read consecutive words; at 32^3 cells the
// 74 MB stay in L2 across the steps of a coarse solve.  Every kernel returns at
// once when the device flag `stop` (may be null) is set, so the solve can be
// captured in a CUDA graph that runs past the end of the outer iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "fcm_device.cuh"

namespace fcm {

struct CoarseOp {
    int64_t ncell = 0;
    float *KH = nullptr;     // [63 * 9][cell]: the blocks of offsets 0..62 (see kStored)
    float *Dinv = nullptr;   // [cell][3][3] inverse of the diagonal block (0 where singular)
    float *r = nullptr, *z = nullptr, *q = nullptr, *p[2] = {nullptr, nullptr};  // 3 x ncell each, [comp][cell]
    double *partial = nullptr;
    int64_t npartial = 0;
    unsigned *counter = nullptr;
    double *sc = nullptr;    // rz, pq, alpha, beta, t
    double seconds = 0.0;    // assembly time
};

namespace {

constexpr int RT = 256;
constexpr int kCenter = 62;               // offset index of (0, 0, 0) in the 5x5x5 stencil
constexpr int kStored = 63;               // offsets kCenter..124 are stored; the others by symmetry
constexpr int kTileCells = 32;            // cells per CTA of the K_H apply (one per lane)
constexpr int kTileWarps = RT / 32;       // warps of that CTA, splitting the offsets

int nb(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

#define STOP_RETURN \
    if (stop && *stop) return

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

// KH[s][a][b][c'] = (R K P e)[a][c'] for the probed cell c = c' + off within distance 2 of c',
// kept for the offsets with index kCenter + s, s >= 0
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
        const int oi = (off[0] + 2) + 5 * ((off[1] + 2) + 5 * (off[2] + 2));
        if (!ok || oi < kCenter) continue;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 8; ++k) {
            const int64_t node = (int64_t)p * (cc[0] + (k & 1)) +
                                 (int64_t)g.M[0] * ((int64_t)p * (cc[1] + ((k >> 1) & 1)) + (int64_t)g.M[1] * p * (cc[2] + (k >> 2)));
            for (int a = 0; a < 3; ++a)
                if (mask[3 * node + a]) acc[a] += v[3 * node + a];
        }
        const int s = oi - kCenter;
        for (int a = 0; a < 3; ++a) KH[(int64_t)(s * 9 + 3 * a + b) * ncell + c] = (float)(0.125 * acc[a]);
    }
}

__global__ void diag_inverse_kernel(const float *KH, float *Dinv, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        double A[9];
        for (int t = 0; t < 9; ++t) A[t] = KH[(int64_t)t * ncell + c];  // s = 0: offset (0,0,0)
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

// Two sums over the grid in a fixed order; true in the last CTA, whose thread 0 then holds the totals.
__device__ bool grid_sums2(double &x, double &y, double *partial, unsigned *counter)
{
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    x = bsum(x, sh);
    y = bsum(y, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = x;
        partial[2 * blockIdx.x + 1] = y;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += RT) {
        a += __ldcg(partial + 2 * i);
        b += __ldcg(partial + 2 * i + 1);
    }
    x = bsum(a, sh);
    y = bsum(b, sh);
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// y = K_H v over a tile of 32 cells per CTA; the 8 warps split the 63 stored offsets, each
// stored block used twice: directly (row cell c, column cell c + off) and transposed for the
// mirrored offset (row c, column c - off), since K_H is symmetric.  The loads carry no
// branches: a neighbour outside the grid is replaced by the cell itself (an in-bounds address)
// and its vector value weighted by 0, so all 24 loads of an offset can be in flight at once.
//   mode 0: v = x
//   mode 1: v = x + beta xb (beta = sc[3]); v is written to pout; pq = v.y, alpha = rz / pq
//   mode 2: v = x;                          v is written to pout; pq = v.y, alpha = rz / pq
__global__ void __launch_bounds__(RT) kh_kernel(const float *__restrict__ KH, const float *__restrict__ x,
                                                 const float *__restrict__ xb, float *__restrict__ pout,
                                                 float *__restrict__ y, Grid3 g, int64_t ncell, int mode,
                                                 double *partial, unsigned *counter, double *sc, const int *stop)
{
    STOP_RETURN;
    __shared__ float red[kTileWarps][3][kTileCells];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * kTileCells + lane;
    const bool live = c0 < ncell;
    const int64_t c = live ? c0 : ncell - 1;
    const float beta = mode == 1 ? (float)sc[3] : 0.f;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int cx = (int)(c % nx), cy = (int)((c / nx) % ny), cz = (int)(c / ((int64_t)nx * ny));
    // bit d + 2 set when the coordinate + d lies in the grid, d = -2..2
    unsigned mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int d = -2; d <= 2; ++d) {
        mx |= (unsigned)(cx + d >= 0 && cx + d < nx) << (d + 2);
        my |= (unsigned)(cy + d >= 0 && cy + d < ny) << (d + 2);
        mz |= (unsigned)(cz + d >= 0 && cz + d < nz) << (d + 2);
    }
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    if (live) {
#pragma unroll 2
        for (int s = w; s < kStored; s += kTileWarps) {
            const int oi = kCenter + s, dx = oi % 5 - 2, dy = (oi / 5) % 5 - 2, dz = oi / 25 - 2;
            const int64_t d = dx + (int64_t)nx * (dy + (int64_t)ny * dz);
            const bool vd = (mx >> (dx + 2)) & (my >> (dy + 2)) & (mz >> (dz + 2)) & 1u;
            const bool vm = s > 0 && ((mx >> (2 - dx)) & (my >> (2 - dy)) & (mz >> (2 - dz)) & 1u);
            const int64_t n = vd ? c + d : c, m = vm ? c - d : c;
            const float wd = vd ? 1.f : 0.f, wm = vm ? 1.f : 0.f;
            const float *Bc = KH + (int64_t)s * 9 * ncell + c;
            const float *Bm = KH + (int64_t)s * 9 * ncell + m;
            float u0 = __ldg(x + n), u1 = __ldg(x + ncell + n), u2 = __ldg(x + 2 * ncell + n);
            float v0 = __ldg(x + m), v1 = __ldg(x + ncell + m), v2 = __ldg(x + 2 * ncell + m);
            if (mode == 1) {
                u0 = fmaf(beta, __ldg(xb + n), u0);
                u1 = fmaf(beta, __ldg(xb + ncell + n), u1);
                u2 = fmaf(beta, __ldg(xb + 2 * ncell + n), u2);
                v0 = fmaf(beta, __ldg(xb + m), v0);
                v1 = fmaf(beta, __ldg(xb + ncell + m), v1);
                v2 = fmaf(beta, __ldg(xb + 2 * ncell + m), v2);
            }
            u0 *= wd;
            u1 *= wd;
            u2 *= wd;
            v0 *= wm;
            v1 *= wm;
            v2 *= wm;
            a0 = fmaf(__ldg(Bc), u0, fmaf(__ldg(Bc + ncell), u1, fmaf(__ldg(Bc + 2 * ncell), u2, a0)));
            a1 = fmaf(__ldg(Bc + 3 * ncell), u0, fmaf(__ldg(Bc + 4 * ncell), u1, fmaf(__ldg(Bc + 5 * ncell), u2, a1)));
            a2 = fmaf(__ldg(Bc + 6 * ncell), u0, fmaf(__ldg(Bc + 7 * ncell), u1, fmaf(__ldg(Bc + 8 * ncell), u2, a2)));
            a0 = fmaf(__ldg(Bm), v0, fmaf(__ldg(Bm + 3 * ncell), v1, fmaf(__ldg(Bm + 6 * ncell), v2, a0)));
            a1 = fmaf(__ldg(Bm + ncell), v0, fmaf(__ldg(Bm + 4 * ncell), v1, fmaf(__ldg(Bm + 7 * ncell), v2, a1)));
            a2 = fmaf(__ldg(Bm + 2 * ncell), v0, fmaf(__ldg(Bm + 5 * ncell), v1, fmaf(__ldg(Bm + 8 * ncell), v2, a2)));
        }
    }
    red[w][0][lane] = a0;
    red[w][1][lane] = a1;
    red[w][2][lane] = a2;
    __syncthreads();
    double dot = 0.0, unused = 0.0;
    if (w < 3) {
        // warp w finishes component w of the 32 cells
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTileWarps; ++k) acc += red[k][w][lane];
        if (live) {
            y[w * ncell + c] = acc;
            if (mode != 0) {
                float v = x[w * ncell + c];
                if (mode == 1) v = fmaf(beta, xb[w * ncell + c], v);
                pout[w * ncell + c] = v;
                dot = (double)v * acc;
            }
        }
    }
    if (mode == 0) return;
    if (!grid_sums2(dot, unused, partial, counter) || threadIdx.x) return;
    sc[1] = dot;
    sc[2] = (dot > 0.0 && isfinite(sc[0] / dot)) ? sc[0] / dot : 0.0;
}

// line search t = f.y / y.q (0 when y.q <= 0), into sc[4]
__global__ void __launch_bounds__(RT) line_kernel(const float *f, const float *y, const float *q, int64_t n,
                                                   double *partial, unsigned *counter, double *sc, const int *stop)
{
    STOP_RETURN;
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        a += (double)f[i] * y[i];
        b += (double)y[i] * q[i];
    }
    if (!grid_sums2(a, b, partial, counter) || threadIdx.x) return;
    sc[4] = (b > 0.0 && isfinite(a / b)) ? a / b : 0.0;
}

// Start of the coarse CG, one thread per cell:
//   start 0: y = 0, r = f;  start 1: r = f - q (q = K_H y);  start 2: y *= t, r = f - t q.
// With want_z: z = Dinv r and rz = r.z into sc[0].
__global__ void __launch_bounds__(RT) cstart_kernel(const float *f, float *y, float *r, float *z, const float *q,
                                                     const float *Dinv, int64_t ncell, int start, int want_z,
                                                     double *partial, unsigned *counter, double *sc, const int *stop)
{
    STOP_RETURN;
    const float t = start == 2 ? (float)sc[4] : 1.f;
    double dot = 0.0, unused = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)RT + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * RT) {
        float rv[3];
        for (int a = 0; a < 3; ++a) {
            const int64_t i = a * ncell + c;
            if (start == 0) {
                y[i] = 0.f;
                rv[a] = f[i];
            } else {
                y[i] *= t;
                rv[a] = fmaf(-t, q[i], f[i]);
            }
            r[i] = rv[a];
        }
        if (want_z) {
            const float *D = Dinv + c * 9;
            for (int a = 0; a < 3; ++a) {
                const float zv = D[3 * a] * rv[0] + D[3 * a + 1] * rv[1] + D[3 * a + 2] * rv[2];
                z[a * ncell + c] = zv;
                dot += (double)rv[a] * zv;
            }
        }
    }
    if (!want_z) return;
    if (!grid_sums2(dot, unused, partial, counter) || threadIdx.x) return;
    sc[0] = dot;
}

// y += alpha p, r -= alpha q; unless last: z = Dinv r, rz' = r.z, beta = rz' / rz, rz = rz'
__global__ void __launch_bounds__(RT) cupd_kernel(float *y, float *r, float *z, const float *p, const float *q,
                                                   const float *Dinv, int64_t ncell, int last_step, double *partial,
                                                   unsigned *counter, double *sc, const int *stop)
{
    STOP_RETURN;
    const float al = (float)sc[2];
    double dot = 0.0, unused = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)RT + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * RT) {
        float rv[3];
        for (int a = 0; a < 3; ++a) {
            const int64_t i = a * ncell + c;
            y[i] = fmaf(al, p[i], y[i]);
            rv[a] = fmaf(-al, q[i], r[i]);
            r[i] = rv[a];
        }
        if (!last_step) {
            const float *D = Dinv + c * 9;
            for (int a = 0; a < 3; ++a) {
                const float zv = D[3 * a] * rv[0] + D[3 * a + 1] * rv[1] + D[3 * a + 2] * rv[2];
                z[a * ncell + c] = zv;
                dot += (double)rv[a] * zv;
            }
        }
    }
    if (last_step) return;
    if (!grid_sums2(dot, unused, partial, counter) || threadIdx.x) return;
    sc[3] = (sc[0] > 0.0 && isfinite(dot / sc[0])) ? dot / sc[0] : 0.0;
    sc[0] = dot;
}

int tiles(int64_t ncell) { return (int)((ncell + kTileCells - 1) / kTileCells); }

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
    const size_t kh_words = (size_t)ncell * kStored * 9;
    if ((e = cudaMalloc(&op->KH, sizeof(float) * kh_words)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->Dinv, sizeof(float) * ncell * 9)) != cudaSuccess) return fail(e);
    float **vs[] = {&op->r, &op->z, &op->q, &op->p[0], &op->p[1]};
    for (float **v : vs)
        if ((e = cudaMalloc(v, sizeof(float) * n3)) != cudaSuccess) return fail(e);
    op->npartial = std::max<int64_t>(tiles(ncell), 152 * 8);
    if ((e = cudaMalloc(&op->partial, sizeof(double) * 2 * op->npartial)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->counter, sizeof(unsigned))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&op->sc, sizeof(double) * 8)) != cudaSuccess) return fail(e);
    cudaStream_t st = C->stream;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, st);
    cudaMemsetAsync(op->counter, 0, sizeof(unsigned), st);
    cudaMemsetAsync(op->sc, 0, sizeof(double) * 8, st);
    cudaMemsetAsync(op->KH, 0, sizeof(float) * kh_words, st);
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
    cudaEventRecord(t1, st);
    e = cudaStreamSynchronize(st);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    op->seconds = ms * 1e-3;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(ecell);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return fail(e);
    C->coarse = op;
    return FCM_OK;
}

void coarse_free(CoarseOp *op)
{
    if (!op) return;
    void *ps[] = {op->KH, op->Dinv, op->r, op->z, op->q, op->p[0], op->p[1], op->partial, op->counter, op->sc};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete op;
}

double coarse_seconds(const CoarseOp *op) { return op ? op->seconds : 0.0; }

// y <- approximate solution of K_H y = f after `iters` block-Jacobi CG steps (FP32 cells,
// [comp][cell]) from the start `start` (0 zero, 1 the given y, 2 the given y scaled by the
// energy-minimising step); asynchronous on the context's stream, capturable.  Two launches
// per step: the K_H apply (which also forms the new direction and alpha) and the update
// (which also applies Dinv and forms beta).
void coarse_solve(fcm_ctx *C, const float *f, float *y, int iters, int start, const int *stop)
{
    CoarseOp *op = C->coarse;
    const int64_t n3 = 3 * op->ncell, nc = op->ncell;
    cudaStream_t st = C->stream;
    if (start != 0)
        kh_kernel<<<tiles(nc), RT, 0, st>>>(op->KH, y, nullptr, nullptr, op->q, C->g, nc, 0, op->partial, op->counter,
                                            op->sc, stop);
    if (start == 2) line_kernel<<<nb(n3), RT, 0, st>>>(f, y, op->q, n3, op->partial, op->counter, op->sc, stop);
    cstart_kernel<<<nb(nc), RT, 0, st>>>(f, y, op->r, op->z, op->q, op->Dinv, nc, start, iters > 0 ? 1 : 0, op->partial,
                                         op->counter, op->sc, stop);
    for (int i = 0; i < iters; ++i) {
        float *pn = op->p[i & 1];
        const float *po = op->p[(i + 1) & 1];
        kh_kernel<<<tiles(nc), RT, 0, st>>>(op->KH, op->z, i == 0 ? nullptr : po, pn, op->q, C->g, nc, i == 0 ? 2 : 1,
                                            op->partial, op->counter, op->sc, stop);
        cupd_kernel<<<nb(nc), RT, 0, st>>>(y, op->r, op->z, pn, op->q, op->Dinv, nc, i + 1 == iters ? 1 : 0, op->partial,
                                           op->counter, op->sc, stop);
    }
}

void coarse_apply(fcm_ctx *C, const float *x, float *y)
{
    CoarseOp *op = C->coarse;
    kh_kernel<<<tiles(op->ncell), RT, 0, C->stream>>>(op->KH, x, nullptr, nullptr, y, C->g, op->ncell, 0, op->partial,
                                                      op->counter, op->sc, nullptr);
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
