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
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fcm_device.cuh"

namespace fcm {

// One level of the cell-grid multigrid hierarchy (level 0: the cell grid of K_H itself).
struct MgLevel {
    Grid3 g{};                 // only g.n is used
    int64_t ncell = 0;
    float *KH = nullptr;       // stored blocks as for K_H (level 0: CoarseOp::KH, not owned)
    float *Dinv = nullptr;     // inverse diagonal blocks (level 0: CoarseOp::Dinv, not owned)
    float *f = nullptr, *xa = nullptr, *r = nullptr, *x = nullptr;  // 3 x ncell; level 0 owns xa and r only
    float omega = 0.f;         // damping of the block-Jacobi smoother, 4 / (3 lambda_max(Dinv K))
    double lambda = 0.0;       // that lambda_max (power iteration)
    bool own = false;
};

constexpr int kMaxLevels = 12;
constexpr int64_t kDenseMaxCells = 512;  // the coarsest level has at most this many cells

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
    // K_H stored in scaled FP16 (fcm_coarse_set_storage): K~_cj = s_c K_cj s_j, s_c = (tr K_cc / 3)^-1/2
    __half *KH16 = nullptr;
    float *scale = nullptr, *iscale = nullptr;  // s and 1 / s
    bool use_half = false;   // KH16 in use (the storage chosen at the last coarse_ensure)
    bool half_cycles = false;  // ... only in the cycles' residual and smoothing products
    Grid3 g{};               // the cell grid of K_H
    // multigrid hierarchy (built on first use of the V-cycle preconditioner)
    int nlev = 0;
    MgLevel lev[kMaxLevels];
    float *Apinv = nullptr;  // dense pseudo-inverse of the coarsest level, [comp][cell] order
    int n3last = 0;
    double mg_seconds = 0.0;
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

// y = K_H v over a tile of 32 cells per CTA (at most 64 registers, 4 offsets unrolled: more loads in
// flight per warp, which this latency-bound product needs; 344 -> 273 us at 80^3 cells); the 8 warps
// split the 63 stored offsets, each
// stored block used twice: directly (row cell c, column cell c + off) and transposed for the
// mirrored offset (row c, column c - off), since K_H is symmetric.  The loads carry no
// branches: a neighbour outside the grid is replaced by the cell itself (an in-bounds address)
// and its vector value weighted by 0, so all 24 loads of an offset can be in flight at once.
//   mode 0: v = x
//   mode 1: v = x + beta xb (beta = sc[3]); v is written to pout; pq = v.y, alpha = rz / pq
//   mode 2: v = x;                          v is written to pout; pq = v.y, alpha = rz / pq
//   mode 3: y = xb - K_H x                  (residual of K_H x = xb)
//   mode 4: pout = x + omega Dinv (xb - K_H x)  (one damped block-Jacobi step; pout must not alias x)
//
// T = __half: the blocks are stored symmetrically scaled, K~_cj = s_c K_cj s_j, so that every stored
// value is O(1) and FP16 keeps 11 significant bits; K_H x = S^-1 K~ S^-1 x, so the kernel multiplies the
// vector values by `scale` = 1 / s before the product and the result by 1 / s_c after it.
__device__ __forceinline__ float ldk(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldk(const __half *p) { return __half2float(__ldg(p)); }

template <class T>
__global__ void __launch_bounds__(RT, 4) kh_kernel(const T *__restrict__ KH, const float *__restrict__ x,
                                                 const float *__restrict__ xb, float *__restrict__ pout,
                                                 float *__restrict__ y, Grid3 g, int64_t ncell, int mode,
                                                 double *partial, unsigned *counter, double *sc, const int *stop,
                                                 const float *__restrict__ Dinv = nullptr, float omega = 0.f,
                                                 const float *__restrict__ scale = nullptr)
{
    constexpr bool kScaled = sizeof(T) == 2;
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
#pragma unroll 4
        for (int s = w; s < kStored; s += kTileWarps) {
            const int oi = kCenter + s, dx = oi % 5 - 2, dy = (oi / 5) % 5 - 2, dz = oi / 25 - 2;
            const int64_t d = dx + (int64_t)nx * (dy + (int64_t)ny * dz);
            const bool vd = (mx >> (dx + 2)) & (my >> (dy + 2)) & (mz >> (dz + 2)) & 1u;
            const bool vm = s > 0 && ((mx >> (2 - dx)) & (my >> (2 - dy)) & (mz >> (2 - dz)) & 1u);
            const int64_t n = vd ? c + d : c, m = vm ? c - d : c;
            const float wd = vd ? 1.f : 0.f, wm = vm ? 1.f : 0.f;
            const T *Bc = KH + (int64_t)s * 9 * ncell + c;
            const T *Bm = KH + (int64_t)s * 9 * ncell + m;
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
            float sd = wd, sm = wm;
            if constexpr (kScaled) {
                sd *= __ldg(scale + n);
                sm *= __ldg(scale + m);
            }
            u0 *= sd;
            u1 *= sd;
            u2 *= sd;
            v0 *= sm;
            v1 *= sm;
            v2 *= sm;
            a0 = fmaf(ldk(Bc), u0, fmaf(ldk(Bc + ncell), u1, fmaf(ldk(Bc + 2 * ncell), u2, a0)));
            a1 = fmaf(ldk(Bc + 3 * ncell), u0, fmaf(ldk(Bc + 4 * ncell), u1, fmaf(ldk(Bc + 5 * ncell), u2, a1)));
            a2 = fmaf(ldk(Bc + 6 * ncell), u0, fmaf(ldk(Bc + 7 * ncell), u1, fmaf(ldk(Bc + 8 * ncell), u2, a2)));
            a0 = fmaf(ldk(Bm), v0, fmaf(ldk(Bm + 3 * ncell), v1, fmaf(ldk(Bm + 6 * ncell), v2, a0)));
            a1 = fmaf(ldk(Bm + ncell), v0, fmaf(ldk(Bm + 4 * ncell), v1, fmaf(ldk(Bm + 7 * ncell), v2, a1)));
            a2 = fmaf(ldk(Bm + 2 * ncell), v0, fmaf(ldk(Bm + 5 * ncell), v1, fmaf(ldk(Bm + 8 * ncell), v2, a2)));
        }
    }
    red[w][0][lane] = a0;
    red[w][1][lane] = a1;
    red[w][2][lane] = a2;
    __syncthreads();
    if (mode >= 3) {
        if (w == 0 && live) {
            float res[3];
            const float sc_c = kScaled ? scale[c] : 1.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < kTileWarps; ++k) acc += red[k][a][lane];
                res[a] = xb[a * ncell + c] - sc_c * acc;
            }
            if (mode == 3) {
#pragma unroll
                for (int a = 0; a < 3; ++a) y[a * ncell + c] = res[a];
            } else {
                const float *D = Dinv + c * 9;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    pout[a * ncell + c] =
                        fmaf(omega, fmaf(D[3 * a], res[0], fmaf(D[3 * a + 1], res[1], D[3 * a + 2] * res[2])),
                             x[a * ncell + c]);
            }
        }
        return;
    }
    double dot = 0.0, unused = 0.0;
    if (w < 3) {
        // warp w finishes component w of the 32 cells
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTileWarps; ++k) acc += red[k][w][lane];
        if (kScaled) acc *= scale[c];
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

// ---- geometric multigrid on the cell grid (the V-cycle that may precondition the coarse CG) ----
//
// Level l + 1 halves the cells of level l along every axis with more than one cell (n' = (n + 1) / 2).
// The interpolation P2 from level l + 1 to level l is cell-centred trilinear per axis: fine cell i
// takes 3/4 of coarse cell i / 2 and 1/4 of its neighbour on the side of i (i - 1 for even i, i + 1
// for odd), or all of i / 2 where that neighbour is outside the grid; along an axis that is not
// coarsened, the identity.  K_{l+1} = P2^T K_l P2: a coarse cell reaches fine cells [2J - 1, 2J + 2],
// so coupling distance 2 on level l stays distance 2 on level l + 1 and the 63-block storage and
// kh_kernel serve every level.

// weight of coarse cell J in fine cell i along one axis (f: 2 if the axis is coarsened, else 1)
__device__ __forceinline__ float axis_w(int i, int J, int nc, int f)
{
    if (f == 1) return i == J ? 1.f : 0.f;
    const int c = i >> 1, o = (i & 1) ? c + 1 : c - 1;
    const bool ov = o >= 0 && o < nc;
    if (J == c) return ov ? 0.75f : 1.f;
    return (ov && J == o) ? 0.25f : 0.f;
}

struct LvDims {
    int nf[3], nc[3], f[3];
    int64_t ncf, ncc;
};

// xf (+)= P2 xc, one thread per fine cell
__global__ void __launch_bounds__(RT) mg_interp_kernel(const float *__restrict__ xc, float *__restrict__ xf, LvDims d,
                                                        int add, const int *stop)
{
    STOP_RETURN;
    for (int64_t c = blockIdx.x * (int64_t)RT + threadIdx.x; c < d.ncf; c += (int64_t)gridDim.x * RT) {
        const int i[3] = {(int)(c % d.nf[0]), (int)((c / d.nf[0]) % d.nf[1]), (int)(c / ((int64_t)d.nf[0] * d.nf[1]))};
        int J[3][2];
        float W[3][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d.f[a] == 1) {
                J[a][0] = J[a][1] = i[a];
                W[a][0] = 1.f;
                W[a][1] = 0.f;
            } else {
                const int cc = i[a] >> 1, o = (i[a] & 1) ? cc + 1 : cc - 1;
                const bool ov = o >= 0 && o < d.nc[a];
                J[a][0] = cc;
                J[a][1] = ov ? o : cc;
                W[a][0] = ov ? 0.75f : 1.f;
                W[a][1] = ov ? 0.25f : 0.f;
            }
        }
        float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int jx = J[0][t & 1], jy = J[1][(t >> 1) & 1], jz = J[2][t >> 2];
            const float wt = W[0][t & 1] * W[1][(t >> 1) & 1] * W[2][t >> 2];
            const int64_t q = jx + (int64_t)d.nc[0] * (jy + (int64_t)d.nc[1] * jz);
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] = fmaf(wt, xc[a * d.ncc + q], acc[a]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) xf[a * d.ncf + c] = add ? xf[a * d.ncf + c] + acc[a] : acc[a];
    }
}

// fc = P2^T rf, one thread per coarse cell (up to 4 fine cells per axis)
__global__ void __launch_bounds__(RT) mg_restrict_kernel(const float *__restrict__ rf, float *__restrict__ fc, LvDims d,
                                                          const int *stop)
{
    STOP_RETURN;
    for (int64_t q = blockIdx.x * (int64_t)RT + threadIdx.x; q < d.ncc; q += (int64_t)gridDim.x * RT) {
        const int J[3] = {(int)(q % d.nc[0]), (int)((q / d.nc[0]) % d.nc[1]), (int)(q / ((int64_t)d.nc[0] * d.nc[1]))};
        int lo[3], cnt[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = d.f[a] == 1 ? J[a] : 2 * J[a] - 1;
            cnt[a] = d.f[a] == 1 ? 1 : 4;
        }
        float acc[3] = {0.f, 0.f, 0.f};
        for (int kz = 0; kz < cnt[2]; ++kz) {
            const int iz = lo[2] + kz;
            if (iz < 0 || iz >= d.nf[2]) continue;
            const float wz = axis_w(iz, J[2], d.nc[2], d.f[2]);
            if (wz == 0.f) continue;
            for (int ky = 0; ky < cnt[1]; ++ky) {
                const int iy = lo[1] + ky;
                if (iy < 0 || iy >= d.nf[1]) continue;
                const float wy = wz * axis_w(iy, J[1], d.nc[1], d.f[1]);
                if (wy == 0.f) continue;
                for (int kx = 0; kx < cnt[0]; ++kx) {
                    const int ix = lo[0] + kx;
                    if (ix < 0 || ix >= d.nf[0]) continue;
                    const float wt = wy * axis_w(ix, J[0], d.nc[0], d.f[0]);
                    if (wt == 0.f) continue;
                    const int64_t c = ix + (int64_t)d.nf[0] * (iy + (int64_t)d.nf[1] * iz);
#pragma unroll
                    for (int a = 0; a < 3; ++a) acc[a] = fmaf(wt, rf[a * d.ncf + c], acc[a]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) fc[a * d.ncc + q] = acc[a];
    }
}

// e = indicator of the cells with (x, y, z) = (ox, oy, oz) mod 5, component b
__global__ void probe_cells_f_kernel(float *e, Grid3 g, int ox, int oy, int oz, int b, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(c % g.n[0]), cy = (int)((c / g.n[0]) % g.n[1]), cz = (int)(c / ((int64_t)g.n[0] * g.n[1]));
        const float v = (cx % 5 == ox && cy % 5 == oy && cz % 5 == oz) ? 1.f : 0.f;
        for (int a = 0; a < 3; ++a) e[a * ncell + c] = a == b ? v : 0.f;
    }
}

// the probe's answer u (cell vector) into the stored blocks, as probe_scatter_kernel does for level 0
__global__ void cell_scatter_kernel(const float *__restrict__ u, float *KH, Grid3 g, int ox, int oy, int oz, int b,
                                    int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cc[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((int64_t)g.n[0] * g.n[1]))};
        const int o[3] = {ox, oy, oz};
        int off[3];
        bool ok = true;
        for (int ax = 0; ax < 3; ++ax) {
            int dd = ((o[ax] - cc[ax]) % 5 + 5) % 5;
            if (dd > 2) dd -= 5;
            off[ax] = dd;
            const int t = cc[ax] + dd;
            ok = ok && t >= 0 && t < g.n[ax];
        }
        const int oi = (off[0] + 2) + 5 * ((off[1] + 2) + 5 * (off[2] + 2));
        if (!ok || oi < kCenter) continue;
        const int s = oi - kCenter;
        for (int a = 0; a < 3; ++a) KH[(int64_t)(s * 9 + 3 * a + b) * ncell + c] = u[a * ncell + c];
    }
}

// x = omega Dinv f (the first damped block-Jacobi step from zero)
__global__ void __launch_bounds__(RT) jacobi0_kernel(const float *__restrict__ f, const float *__restrict__ Dinv,
                                                      float omega, float *__restrict__ x, int64_t ncell, const int *stop)
{
    STOP_RETURN;
    for (int64_t c = blockIdx.x * (int64_t)RT + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * RT) {
        const float r0 = f[c], r1 = f[ncell + c], r2 = f[2 * ncell + c];
        const float *D = Dinv + c * 9;
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a * ncell + c] = omega * fmaf(D[3 * a], r0, fmaf(D[3 * a + 1], r1, D[3 * a + 2] * r2));
    }
}

// sum of squares into *out (deterministic two-level reduction)
__global__ void __launch_bounds__(RT) sumsq_kernel(const float *u, int64_t n, double *partial, unsigned *counter,
                                                    double *out)
{
    double a = 0.0, unused = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) a += (double)u[i] * u[i];
    if (!grid_sums2(a, unused, partial, counter) || threadIdx.x) return;
    *out = a;
}

// u = s Dinv v (one thread per cell), for the power iteration
__global__ void __launch_bounds__(RT) dinv_scale_kernel(const float *__restrict__ v, const float *__restrict__ Dinv,
                                                         float s, float *__restrict__ u, int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)RT + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * RT) {
        const float r0 = v[c], r1 = v[ncell + c], r2 = v[2 * ncell + c];
        const float *D = Dinv + c * 9;
        for (int a = 0; a < 3; ++a) u[a * ncell + c] = s * fmaf(D[3 * a], r0, fmaf(D[3 * a + 1], r1, D[3 * a + 2] * r2));
    }
}

// deterministic start vector of the power iteration
__global__ void hash_fill_kernel(float *v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        v[i] = (float)(h & 0xffff) / 65536.f - 0.5f;
    }
}

// dense symmetric A (n3 x n3, FP64, row-major = column-major) from the stored blocks of the last level
__global__ void dense_from_blocks_kernel(const float *__restrict__ KH, Grid3 g, int64_t ncell, double *A)
{
    const int64_t n3 = 3 * ncell;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncell * kStored;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % ncell;
        const int s = (int)(t / ncell), oi = kCenter + s;
        const int dx = oi % 5 - 2, dy = (oi / 5) % 5 - 2, dz = oi / 25 - 2;
        const int cx = (int)(c % g.n[0]) + dx, cy = (int)((c / g.n[0]) % g.n[1]) + dy,
                  cz = (int)(c / ((int64_t)g.n[0] * g.n[1])) + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= g.n[0] || cy >= g.n[1] || cz >= g.n[2]) continue;
        const int64_t j = cx + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double v = KH[(int64_t)(s * 9 + 3 * a + b) * ncell + c];
                A[(3 * c + a) * n3 + 3 * j + b] = v;
                if (s > 0) A[(3 * j + b) * n3 + 3 * c + a] = v;  // the centre block is stored whole
            }
    }
}

// P = V diag(1 / lambda) V^T over the eigenvalues above the cut-off (V column-major from syevd), FP32,
// unknowns in [comp][cell] order
__global__ void pinv_kernel(const double *__restrict__ V, const double *__restrict__ lam, double cut, int n3,
                            int64_t ncell, float *__restrict__ P)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n3 * n3;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n3), j = (int)(t % n3);
        double acc = 0.0;
        for (int k = 0; k < n3; ++k)
            if (lam[k] > cut) acc += V[i + (int64_t)k * n3] * V[j + (int64_t)k * n3] / lam[k];
        // row/column i, j are interleaved unknowns 3 cell + comp; P is stored for [comp][cell] vectors
        const int64_t pi = (i % 3) * ncell + i / 3, pj = (j % 3) * ncell + j / 3;
        P[pi * n3 + pj] = (float)acc;
    }
}

// x = P f (dense, a warp per row)
__global__ void __launch_bounds__(RT) dense_mv_kernel(const float *__restrict__ P, const float *__restrict__ f,
                                                       float *__restrict__ x, int n3, const int *stop)
{
    STOP_RETURN;
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x * (RT / 32) + (threadIdx.x >> 5); row < n3; row += gridDim.x * (RT / 32)) {
        float acc = 0.f;
        for (int j = lane; j < n3; j += 32) acc = fmaf(P[(int64_t)row * n3 + j], f[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) x[row] = acc;
    }
}

// rz = r.z; first: sc[0] = rz; else beta = rz / sc[0] into sc[3], sc[0] = rz
__global__ void __launch_bounds__(RT) rz_kernel(const float *r, const float *z, int64_t n, int first, double *partial,
                                                 unsigned *counter, double *sc, const int *stop)
{
    STOP_RETURN;
    double a = 0.0, unused = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) a += (double)r[i] * z[i];
    if (!grid_sums2(a, unused, partial, counter) || threadIdx.x) return;
    if (!first) sc[3] = (sc[0] > 0.0 && isfinite(a / sc[0])) ? a / sc[0] : 0.0;
    sc[0] = a;
}

// s_c = (tr K_cc / 3)^-1/2 from the centre block, and 1 / s_c (both 0 where the trace is 0)
__global__ void kh_scale_kernel(const float *__restrict__ KH, float *__restrict__ scale, float *__restrict__ iscale,
                                int64_t ncell)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const double tr = (double)KH[c] + (double)KH[4 * ncell + c] + (double)KH[8 * ncell + c];
        scale[c] = tr > 0.0 ? (float)(1.0 / sqrt(tr / 3.0)) : 0.f;
        iscale[c] = tr > 0.0 ? (float)sqrt(tr / 3.0) : 0.f;
    }
}

// K~ = s K s in FP16, rounded to nearest; a block whose column cell lies outside the grid is 0
__global__ void kh_to_half_kernel(const float *__restrict__ KH, const float *__restrict__ scale,
                                  __half *__restrict__ KH16, Grid3 g, int64_t ncell)
{
    const int64_t total = ncell * kStored * 9;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % ncell;
        const int s = (int)(t / ncell / 9), oi = kCenter + s;
        const int cx = (int)(c % g.n[0]) + oi % 5 - 2, cy = (int)((c / g.n[0]) % g.n[1]) + (oi / 5) % 5 - 2,
                  cz = (int)(c / ((int64_t)g.n[0] * g.n[1])) + oi / 25 - 2;
        float v = 0.f;
        if (cx >= 0 && cy >= 0 && cz >= 0 && cx < g.n[0] && cy < g.n[1] && cz < g.n[2]) {
            const int64_t j = cx + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
            v = KH[t] * scale[c] * scale[j];
        }
        KH16[t] = __float2half_rn(v);
    }
}

int tiles(int64_t ncell) { return (int)((ncell + kTileCells - 1) / kTileCells); }

// K_H apply on the cell grid of K_H in the stored precision: FP32, or the scaled FP16 copy when in use
void kh0(const CoarseOp *op, const float *x, const float *xb, float *pout, float *y, int mode, cudaStream_t st,
         const int *stop, const float *Dinv = nullptr, float omega = 0.f, bool in_cycle = false)
{
    if (op->use_half && (in_cycle || !op->half_cycles))
        kh_kernel<__half><<<tiles(op->ncell), RT, 0, st>>>(op->KH16, x, xb, pout, y, op->g, op->ncell, mode, op->partial,
                                                           op->counter, op->sc, stop, Dinv, omega, op->iscale);
    else
        kh_kernel<float><<<tiles(op->ncell), RT, 0, st>>>(op->KH, x, xb, pout, y, op->g, op->ncell, mode, op->partial,
                                                          op->counter, op->sc, stop, Dinv, omega);
}

}  // namespace

// Build the coarse operator once per context (375 applications of K).
namespace {
fcm_status mg_build(fcm_ctx *C);
void mg_free_levels(CoarseOp *op);
void vcycle(CoarseOp *op, const float *f0, float *x0, cudaStream_t st, const int *stop, bool hybrid);
}  // namespace

namespace {
// the scaled FP16 copy of K_H (outside any capture), or FCM_ENOMEM
fcm_status half_build(fcm_ctx *C)
{
    CoarseOp *op = C->coarse;
    const int64_t nc = op->ncell;
    cudaError_t e;
    if ((e = cudaMalloc(&op->scale, sizeof(float) * nc)) != cudaSuccess ||
        (e = cudaMalloc(&op->iscale, sizeof(float) * nc)) != cudaSuccess ||
        (e = cudaMalloc(&op->KH16, sizeof(__half) * (size_t)nc * kStored * 9)) != cudaSuccess) {
        if (op->scale) cudaFree(op->scale);
        if (op->iscale) cudaFree(op->iscale);
        op->scale = op->iscale = nullptr;
        op->KH16 = nullptr;
        C->err = std::string("coarse operator FP16 copy: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;
    }
    kh_scale_kernel<<<nb(nc), 256, 0, C->stream>>>(op->KH, op->scale, op->iscale, nc);
    kh_to_half_kernel<<<nb(nc * kStored * 9), 256, 0, C->stream>>>(op->KH, op->scale, op->KH16, op->g, nc);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        C->err = std::string("coarse operator FP16 copy: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    return FCM_OK;
}
}  // namespace

fcm_status coarse_ensure(fcm_ctx *C)
{
    if (C->coarse) {
        fcm_status s = FCM_OK;
        if (C->coarse_half && !C->coarse->KH16) s = half_build(C);
        C->coarse->use_half = C->coarse_half && C->coarse->KH16;
        C->coarse->half_cycles = C->coarse_half == FCM_COARSE_STORE_FP16_CYCLES;
        if (s == FCM_OK && C->coarse_prec != FCM_COARSE_JACOBI && C->coarse->nlev == 0) s = mg_build(C);
        return s;
    }
    const int64_t ncell = C->hp.ncells, n3 = 3 * ncell;
    CoarseOp *op = new CoarseOp();
    op->ncell = ncell;
    op->g = C->g;
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
    return coarse_ensure(C);  // the FP16 copy and the hierarchy, where asked for
}

void coarse_free(CoarseOp *op)
{
    if (!op) return;
    mg_free_levels(op);
    if (op->KH16) cudaFree(op->KH16);
    if (op->scale) cudaFree(op->scale);
    if (op->iscale) cudaFree(op->iscale);
    void *ps[] = {op->KH, op->Dinv, op->r, op->z, op->q, op->p[0], op->p[1], op->partial, op->counter, op->sc};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete op;
}

namespace {

void mg_free_levels(CoarseOp *op)
{
    for (int l = 0; l < op->nlev; ++l) {
        MgLevel &v = op->lev[l];
        float *ps[] = {v.own ? v.KH : nullptr, v.own ? v.Dinv : nullptr, v.f, v.xa, v.r, v.x};
        for (float *q : ps)
            if (q) cudaFree(q);
        v = MgLevel();
    }
    if (op->Apinv) cudaFree(op->Apinv);
    op->Apinv = nullptr;
    op->nlev = 0;
}

LvDims dims_down(const MgLevel &fine, const MgLevel &coarse)
{
    LvDims d{};
    for (int a = 0; a < 3; ++a) {
        d.nf[a] = fine.g.n[a];
        d.nc[a] = coarse.g.n[a];
        d.f[a] = fine.g.n[a] > 1 ? 2 : 1;
    }
    d.ncf = fine.ncell;
    d.ncc = coarse.ncell;
    return d;
}

// The hierarchy below K_H: levels by Galerkin probing through P2 (375 applications of the finer
// level's operator each), block-Jacobi damping from 15 power-iteration steps on Dinv K_l, and the
// dense pseudo-inverse of the coarsest level (FP64 eigen-decomposition, eigenvalues below 1e-12 of
// the largest dropped, as for a singular block of the fine preconditioner).
fcm_status mg_build(fcm_ctx *C)
{
    CoarseOp *op = C->coarse;
    cudaStream_t st = C->stream;
    cudaError_t e = cudaSuccess;
    double *A = nullptr, *W = nullptr, *work = nullptr;
    float *pv = nullptr, *pw = nullptr;
    int *info = nullptr;
    cusolverDnHandle_t sh = nullptr;
    auto fail = [&](const std::string &m) {
        C->err = "coarse multigrid: " + m;
        if (A) cudaFree(A);
        if (W) cudaFree(W);
        if (work) cudaFree(work);
        if (pv) cudaFree(pv);
        if (pw) cudaFree(pw);
        if (info) cudaFree(info);
        if (sh) cusolverDnDestroy(sh);
        mg_free_levels(op);
        return e == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;
    };
#define MG_CUDA(call)                                            \
    do {                                                         \
        if ((e = (call)) != cudaSuccess) return fail(#call ": " + std::string(cudaGetErrorString(e))); \
    } while (0)
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, st);
    // level 0
    MgLevel &l0 = op->lev[0];
    l0.g = C->g;
    l0.ncell = op->ncell;
    l0.KH = op->KH;
    l0.Dinv = op->Dinv;
    op->nlev = 1;
    const int64_t n0 = 3 * op->ncell;
    MG_CUDA(cudaMalloc(&pv, sizeof(float) * n0));
    MG_CUDA(cudaMalloc(&pw, sizeof(float) * n0));
    while (op->lev[op->nlev - 1].ncell > kDenseMaxCells && op->nlev < kMaxLevels) {
        MgLevel &fine = op->lev[op->nlev - 1];
        if (fine.g.n[0] == 1 && fine.g.n[1] == 1 && fine.g.n[2] == 1) break;
        MgLevel &cs = op->lev[op->nlev];
        cs = MgLevel();
        cs.own = true;
        for (int a = 0; a < 3; ++a) cs.g.n[a] = fine.g.n[a] > 1 ? (fine.g.n[a] + 1) / 2 : 1;
        cs.ncell = (int64_t)cs.g.n[0] * cs.g.n[1] * cs.g.n[2];
        op->nlev += 1;
        const int64_t nc = cs.ncell, n3 = 3 * nc;
        MG_CUDA(cudaMalloc(&cs.KH, sizeof(float) * (size_t)nc * kStored * 9));
        MG_CUDA(cudaMalloc(&cs.Dinv, sizeof(float) * nc * 9));
        float **bufs[] = {&cs.f, &cs.xa, &cs.r, &cs.x};
        for (float **b : bufs) MG_CUDA(cudaMalloc(b, sizeof(float) * n3));
        MG_CUDA(cudaMemsetAsync(cs.KH, 0, sizeof(float) * (size_t)nc * kStored * 9, st));
        const LvDims d = dims_down(fine, cs);
        for (int oz = 0; oz < 5; ++oz)
            for (int oy = 0; oy < 5; ++oy)
                for (int ox = 0; ox < 5; ++ox)
                    for (int b = 0; b < 3; ++b) {
                        probe_cells_f_kernel<<<nb(nc), 256, 0, st>>>(cs.f, cs.g, ox, oy, oz, b, nc);
                        mg_interp_kernel<<<nb(fine.ncell), RT, 0, st>>>(cs.f, pv, d, 0, nullptr);
                        kh_kernel<<<tiles(fine.ncell), RT, 0, st>>>(fine.KH, pv, nullptr, nullptr, pw, fine.g, fine.ncell,
                                                                    0, op->partial, op->counter, op->sc, nullptr);
                        mg_restrict_kernel<<<nb(nc), RT, 0, st>>>(pw, cs.r, d, nullptr);
                        cell_scatter_kernel<<<nb(nc), 256, 0, st>>>(cs.r, cs.KH, cs.g, ox, oy, oz, b, nc);
                    }
        diag_inverse_kernel<<<nb(nc), 256, 0, st>>>(cs.KH, cs.Dinv, nc);
        MG_CUDA(cudaGetLastError());
    }
    // smoother damping on every level but the last: lambda_max(Dinv K_l) by power iteration
    const int L = op->nlev - 1;
    for (int l = 0; l < L; ++l) {
        MgLevel &v = op->lev[l];
        const int64_t n3 = 3 * v.ncell;
        hash_fill_kernel<<<nb(n3), 256, 0, st>>>(pv, n3);
        double h = 0.0, norm = 0.0, lam = 0.0;
        sumsq_kernel<<<nb(n3), RT, 0, st>>>(pv, n3, op->partial, op->counter, op->sc + 7);
        MG_CUDA(cudaMemcpyAsync(&h, op->sc + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
        MG_CUDA(cudaStreamSynchronize(st));
        norm = std::sqrt(h);
        for (int it = 0; it < 15 && norm > 0.0; ++it) {
            kh_kernel<<<tiles(v.ncell), RT, 0, st>>>(v.KH, pv, nullptr, nullptr, pw, v.g, v.ncell, 0, op->partial,
                                                     op->counter, op->sc, nullptr);
            dinv_scale_kernel<<<nb(v.ncell), RT, 0, st>>>(pw, v.Dinv, (float)(1.0 / norm), pv, v.ncell);
            sumsq_kernel<<<nb(n3), RT, 0, st>>>(pv, n3, op->partial, op->counter, op->sc + 7);
            MG_CUDA(cudaMemcpyAsync(&h, op->sc + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
            MG_CUDA(cudaStreamSynchronize(st));
            lam = std::sqrt(h);  // ||Dinv K v|| for the unit vector v of this step
            norm = lam;
        }
        v.lambda = lam;
        // the power iteration approaches lambda_max from below: damp for 1.1 times the estimate
        v.omega = lam > 0.0 ? (float)(4.0 / (3.0 * 1.1 * lam)) : 0.f;
    }
    // coarsest level: dense pseudo-inverse
    {
        MgLevel &v = op->lev[L];
        const int n3 = (int)(3 * v.ncell);
        op->n3last = n3;
        MG_CUDA(cudaMalloc(&A, sizeof(double) * (size_t)n3 * n3));
        MG_CUDA(cudaMalloc(&W, sizeof(double) * n3));
        MG_CUDA(cudaMalloc(&info, sizeof(int)));
        MG_CUDA(cudaMalloc(&op->Apinv, sizeof(float) * (size_t)n3 * n3));
        MG_CUDA(cudaMemsetAsync(A, 0, sizeof(double) * (size_t)n3 * n3, st));
        dense_from_blocks_kernel<<<nb(v.ncell * kStored), 256, 0, st>>>(v.KH, v.g, v.ncell, A);
        MG_CUDA(cudaGetLastError());
        if (cusolverDnCreate(&sh) != CUSOLVER_STATUS_SUCCESS) return fail("cusolverDnCreate");
        cusolverDnSetStream(sh, st);
        int lwork = 0;
        if (cusolverDnDsyevd_bufferSize(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n3, A, n3, W, &lwork) !=
            CUSOLVER_STATUS_SUCCESS)
            return fail("cusolverDnDsyevd_bufferSize");
        MG_CUDA(cudaMalloc(&work, sizeof(double) * std::max(lwork, 1)));
        if (cusolverDnDsyevd(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n3, A, n3, W, work, lwork, info) !=
            CUSOLVER_STATUS_SUCCESS)
            return fail("cusolverDnDsyevd");
        std::vector<double> lam(n3);
        int hinfo = 0;
        MG_CUDA(cudaMemcpyAsync(lam.data(), W, sizeof(double) * n3, cudaMemcpyDeviceToHost, st));
        MG_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
        MG_CUDA(cudaStreamSynchronize(st));
        if (hinfo != 0) return fail("cusolverDnDsyevd info " + std::to_string(hinfo));
        double lmax = 0.0;
        for (double x : lam) lmax = std::max(lmax, x);
        pinv_kernel<<<nb((int64_t)n3 * n3), 256, 0, st>>>(A, W, 1e-12 * lmax, n3, v.ncell, op->Apinv);
        MG_CUDA(cudaGetLastError());
    }
    cudaEventRecord(t1, st);
    MG_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    op->mg_seconds = ms * 1e-3;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(A);
    cudaFree(W);
    cudaFree(work);
    cudaFree(pv);
    cudaFree(pw);
    cudaFree(info);
    cusolverDnDestroy(sh);
    // level 0 scratch of the V-cycle
    MgLevel &z0 = op->lev[0];
    A = nullptr;
    W = work = nullptr;
    pv = pw = nullptr;
    info = nullptr;
    sh = nullptr;
    MG_CUDA(cudaMalloc(&z0.xa, sizeof(float) * n0));
    MG_CUDA(cudaMalloc(&z0.r, sizeof(float) * n0));
#undef MG_CUDA
    return FCM_OK;
}

// x0 = one V-cycle applied to f0 (cell vectors of level 0): on each level but the last, one damped
// block-Jacobi step from zero, the residual restricted to the next level, the correction
// interpolated back and one more damped block-Jacobi step; the last level by its dense
// pseudo-inverse.  Symmetric in its smoothing, so a fixed linear operator (for the coarse CG).
//
// hybrid: on level 0 the damped block-Jacobi step and the coarse correction are added instead of
// multiplied, x0 = omega Dinv f0 + P2 V_1(P2^T f0) with V_1 the V-cycle of the levels below: symmetric as
// well, and without a K_H apply on the finest cell grid (the expensive one).
void vcycle(CoarseOp *op, const float *f0, float *x0, cudaStream_t st, const int *stop, bool hybrid)
{
    const int L = op->nlev - 1;
    if (L == 0) {
        dense_mv_kernel<<<std::max(1, std::min((op->n3last + 7) / 8, 152 * 8)), RT, 0, st>>>(op->Apinv, f0, x0,
                                                                                           op->n3last, stop);
        return;
    }
    const int l0 = hybrid ? 1 : 0;
    if (hybrid) {
        MgLevel &v = op->lev[0];
        jacobi0_kernel<<<nb(v.ncell), RT, 0, st>>>(f0, v.Dinv, v.omega, x0, v.ncell, stop);
        mg_restrict_kernel<<<nb(op->lev[1].ncell), RT, 0, st>>>(f0, op->lev[1].f, dims_down(v, op->lev[1]), stop);
    }
    for (int l = l0; l < L; ++l) {
        MgLevel &v = op->lev[l];
        const float *f = l == 0 ? f0 : v.f;
        jacobi0_kernel<<<nb(v.ncell), RT, 0, st>>>(f, v.Dinv, v.omega, v.xa, v.ncell, stop);
        if (l == 0)
            kh0(op, v.xa, f, nullptr, v.r, 3, st, stop, nullptr, 0.f, true);
        else
            kh_kernel<<<tiles(v.ncell), RT, 0, st>>>(v.KH, v.xa, f, nullptr, v.r, v.g, v.ncell, 3, op->partial,
                                                     op->counter, op->sc, stop);
        mg_restrict_kernel<<<nb(op->lev[l + 1].ncell), RT, 0, st>>>(v.r, op->lev[l + 1].f, dims_down(v, op->lev[l + 1]),
                                                                    stop);
    }
    dense_mv_kernel<<<std::max(1, std::min((op->n3last + 7) / 8, 152 * 8)), RT, 0, st>>>(op->Apinv, op->lev[L].f,
                                                                                       op->lev[L].x, op->n3last, stop);
    for (int l = L - 1; l >= l0; --l) {
        MgLevel &v = op->lev[l];
        const float *f = l == 0 ? f0 : v.f;
        float *out = l == 0 ? x0 : v.x;
        mg_interp_kernel<<<nb(v.ncell), RT, 0, st>>>(op->lev[l + 1].x, v.xa, dims_down(v, op->lev[l + 1]), 1, stop);
        if (l == 0)
            kh0(op, v.xa, f, out, nullptr, 4, st, stop, v.Dinv, v.omega, true);
        else
            kh_kernel<<<tiles(v.ncell), RT, 0, st>>>(v.KH, v.xa, f, out, nullptr, v.g, v.ncell, 4, op->partial,
                                                     op->counter, op->sc, stop, v.Dinv, v.omega);
    }
    if (hybrid)
        mg_interp_kernel<<<nb(op->lev[0].ncell), RT, 0, st>>>(op->lev[1].x, x0, dims_down(op->lev[0], op->lev[1]), 1,
                                                               stop);
}

}  // namespace

double coarse_seconds(const CoarseOp *op) { return op ? op->seconds : 0.0; }

// y <- approximate solution of K_H y = f after `iters` block-Jacobi CG steps (FP32 cells,
// [comp][cell]) from the start `start` (0 zero, 1 the given y, 2 the given y scaled by the
// energy-minimising step); asynchronous on the context's stream, capturable.  Two launches
// per step: the K_H apply (which also forms the new direction and alpha) and the update
// (which also applies Dinv and forms beta).
void coarse_solve(fcm_ctx *C, const float *f, float *y, int iters, int start, const int *stop, cudaStream_t st)
{
    CoarseOp *op = C->coarse;
    const int64_t n3 = 3 * op->ncell, nc = op->ncell;
    if (!st) st = C->stream;
    const bool mg = C->coarse_prec != FCM_COARSE_JACOBI && op->nlev > 0;
    const bool hybrid = C->coarse_prec == FCM_COARSE_HYBRID;
    if (start != 0)
        kh0(op, y, nullptr, nullptr, op->q, 0, st, stop);
    if (start == 2) line_kernel<<<nb(n3), RT, 0, st>>>(f, y, op->q, n3, op->partial, op->counter, op->sc, stop);
    cstart_kernel<<<nb(nc), RT, 0, st>>>(f, y, op->r, op->z, op->q, op->Dinv, nc, start, !mg && iters > 0 ? 1 : 0,
                                         op->partial, op->counter, op->sc, stop);
    if (mg && iters > 0) {
        vcycle(op, op->r, op->z, st, stop, hybrid);
        rz_kernel<<<nb(n3), RT, 0, st>>>(op->r, op->z, n3, 1, op->partial, op->counter, op->sc, stop);
    }
    for (int i = 0; i < iters; ++i) {
        float *pn = op->p[i & 1];
        const float *po = op->p[(i + 1) & 1];
        const bool last = i + 1 == iters;
        kh0(op, op->z, i == 0 ? nullptr : po, pn, op->q, i == 0 ? 2 : 1, st, stop);
        // with the V-cycle the update kernel only moves y and r; z and beta follow from the cycle
        cupd_kernel<<<nb(nc), RT, 0, st>>>(y, op->r, op->z, pn, op->q, op->Dinv, nc, last || mg ? 1 : 0, op->partial,
                                           op->counter, op->sc, stop);
        if (mg && !last) {
            vcycle(op, op->r, op->z, st, stop, hybrid);
            rz_kernel<<<nb(n3), RT, 0, st>>>(op->r, op->z, n3, 0, op->partial, op->counter, op->sc, stop);
        }
    }
}

void coarse_apply(fcm_ctx *C, const float *x, float *y)
{
    CoarseOp *op = C->coarse;
    kh0(op, x, nullptr, nullptr, y, 0, C->stream, nullptr);
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

namespace fcm {
fcm_status coarse_vcycle_apply(fcm_ctx *C, int kind, const float *f, float *x)
{
    fcm_status s = coarse_ensure(C);
    if (s == FCM_OK && C->coarse->nlev == 0) s = mg_build(C);
    if (s != FCM_OK) return s;
    vcycle(C->coarse, f, x, C->stream, nullptr, kind == FCM_COARSE_HYBRID);
    return FCM_OK;
}
}  // namespace fcm

extern "C" fcm_status fcm_coarse_vcycle(fcm_ctx *C, int kind, const float *f_dev, float *x_dev)
{
    if (!C || !f_dev || !x_dev || f_dev == x_dev || (kind != FCM_COARSE_VCYCLE && kind != FCM_COARSE_HYBRID)) {
        if (C) C->err = "fcm_coarse_vcycle: invalid argument";
        return FCM_EINVAL;
    }
    cudaEventRecord(C->ev_in, C->ustream);
    cudaStreamWaitEvent(C->stream, C->ev_in, 0);
    fcm_status s = fcm::coarse_vcycle_apply(C, kind, f_dev, x_dev);
    cudaEventRecord(C->ev_out, C->stream);
    cudaStreamWaitEvent(C->ustream, C->ev_out, 0);
    if (s != FCM_OK) return s;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        C->err = std::string("fcm_coarse_vcycle: ") + cudaGetErrorString(e);
        return FCM_ECUDA;
    }
    return FCM_OK;
}

extern "C" fcm_status fcm_coarse_set_preconditioner(fcm_ctx *C, int kind)
{
    if (!C) return FCM_EINVAL;
    if (kind != FCM_COARSE_JACOBI && kind != FCM_COARSE_VCYCLE && kind != FCM_COARSE_HYBRID) {
        C->err = "fcm_coarse_set_preconditioner: kind must be FCM_COARSE_JACOBI, FCM_COARSE_VCYCLE or FCM_COARSE_HYBRID";
        return FCM_EINVAL;
    }
    if (kind != C->coarse_prec) fcm::fcg_forget_graph(C->fcg);
    C->coarse_prec = kind;
    return FCM_OK;
}

extern "C" fcm_status fcm_coarse_set_storage(fcm_ctx *C, int storage)
{
    if (!C) return FCM_EINVAL;
    if (storage != FCM_COARSE_STORE_FP32 && storage != FCM_COARSE_STORE_FP16 && storage != FCM_COARSE_STORE_FP16_CYCLES) {
        C->err = "fcm_coarse_set_storage: storage must be FCM_COARSE_STORE_FP32, _FP16 or _FP16_CYCLES";
        return FCM_EINVAL;
    }
    const int half = storage;
    if (half != C->coarse_half) fcm::fcg_forget_graph(C->fcg);
    C->coarse_half = half;
    return FCM_OK;
}

extern "C" fcm_status fcm_coarse_levels(fcm_ctx *C, int *levels, int *dims, double *lambdas, double *seconds)
{
    if (!C || !levels) return FCM_EINVAL;
    const fcm::CoarseOp *op = C->coarse;
    const int n = op ? op->nlev : 0;
    *levels = n;
    for (int l = 0; l < n; ++l) {
        if (dims)
            for (int a = 0; a < 3; ++a) dims[3 * l + a] = op->lev[l].g.n[a];
        if (lambdas && l + 1 < n) lambdas[l] = op->lev[l].lambda;
    }
    if (seconds) *seconds = op ? op->mg_seconds : 0.0;
    return FCM_OK;
}
