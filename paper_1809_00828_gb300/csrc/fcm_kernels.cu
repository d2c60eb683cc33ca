// Hot kernels of the finite cell Schwarz-PCG on sm_103a:
//  * element-by-element stiffness apply y = K x (Sec. 2.1 Eq. (1)), one CTA
//    per active cell, cells processed in 8 parity colours so that cells of one
//    launch share no lattice DOF and the scatter needs no atomics;
//  * Additive-Schwarz apply z = sum_B R_B^T A_B+^-1 R_B r (Sec. 3.1 Eq. (5)):
//    gather r over the vertex patch box, dense symmetric block apply, scatter
//    into z, patches processed in 8 parity colours (patches of one colour are
//    DOF-disjoint).
#include <cuda_runtime.h>

#include "fcm_device.cuh"

namespace fcm {

namespace {

constexpr int round32(int v) { return (v + 31) / 32 * 32; }
// One thread per row up to 512 rows; larger blocks loop over rows.
constexpr int threads_for(int rows) { return round32(rows) < 512 ? round32(rows) : 512; }

// y += K_e x_e over the active cells of one colour; rows that are not free stay untouched.
template <int P>
__global__ void __launch_bounds__(threads_for(3 * (P + 1) * (P + 1) * (P + 1)))
    ebe_apply_kernel(const double *__restrict__ x, double *__restrict__ y, const uint8_t *__restrict__ mask,
                     const double *__restrict__ elem, const int2 *__restrict__ cells, Grid3 g,
                     const int *__restrict__ done)
{
    constexpr int Q = P + 1, NL = Q * Q * Q, NE = 3 * NL;
    if (done && *done) return;
    __shared__ double xe[NE];
    __shared__ int64_t node[NL];
    const int2 ce = cells[blockIdx.x];
    const int cx = ce.x % g.n[0], cy = (ce.x / g.n[0]) % g.n[1], cz = ce.x / (g.n[0] * g.n[1]);
    for (int t = threadIdx.x; t < NL; t += blockDim.x) {
        const int ix = t % Q, iy = (t / Q) % Q, iz = t / (Q * Q);
        node[t] = (P * cx + ix) + (int64_t)g.M[0] * ((P * cy + iy) + (int64_t)g.M[1] * (P * cz + iz));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NE; t += blockDim.x) xe[t] = x[3 * node[t / 3] + t % 3];
    __syncthreads();
    const double *__restrict__ K = elem + (size_t)ce.y * NE * NE;
    for (int t = threadIdx.x; t < NE; t += blockDim.x) {
        double s = 0.0;
#pragma unroll 8
        for (int j = 0; j < NE; ++j) s = fma(__ldg(K + (size_t)j * NE + t), xe[j], s);
        const int64_t gi = 3 * node[t / 3] + t % 3;
        if (mask[gi]) y[gi] += s;
    }
}

// z += F_B r_B for the patches of one colour.  F_B is the dense symmetric
// pseudo inverse over the patch box (zero rows/columns for DOFs outside B).
template <int P>
__global__ void __launch_bounds__(threads_for(3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1)))
    schwarz_apply_kernel(const double *__restrict__ r, double *__restrict__ z, const double *__restrict__ f64,
                         const float *__restrict__ f32, const PatchRec *__restrict__ patches, Grid3 g,
                         const int *__restrict__ done)
{
    constexpr int W = 2 * P - 1, NB = 3 * W * W * W;
    if (done && *done) return;
    __shared__ double rb[NB];
    __shared__ float rbf[NB];
    __shared__ int64_t gidx[NB];
    const PatchRec pr = patches[blockIdx.x];
    const int nvx = g.n[0] + 1, nvy = g.n[1] + 1;
    const int v[3] = {pr.v % nvx, (pr.v / nvx) % nvy, pr.v / (nvx * nvy)};
    int lo[3], d[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(0, P * v[a] - (P - 1));
        const int hi = min(g.M[a] - 1, P * v[a] + (P - 1));
        d[a] = hi - lo[a] + 1;
    }
    const int n = 3 * d[0] * d[1] * d[2];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int nl = t / 3, comp = t % 3;
        const int ix = nl % d[0], iy = (nl / d[0]) % d[1], iz = nl / (d[0] * d[1]);
        const int64_t gi = 3 * ((lo[0] + ix) + (int64_t)g.M[0] * ((lo[1] + iy) + (int64_t)g.M[1] * (lo[2] + iz))) + comp;
        gidx[t] = gi;
        const double v = r[gi];
        rb[t] = v;
        rbf[t] = (float)v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double s = 0.0;
        if (pr.prec == 0) {
            const double *__restrict__ F = f64 + pr.off;
#pragma unroll 8
            for (int j = 0; j < n; ++j) s = fma(__ldg(F + (size_t)j * n + t), rb[j], s);
        } else {
            const float *__restrict__ F = f32 + pr.off;
            float acc = 0.0f;
#pragma unroll 8
            for (int j = 0; j < n; ++j) acc = fmaf(__ldg(F + (size_t)j * n + t), rbf[j], acc);
            s = acc;
        }
        z[gidx[t]] += s;
    }
}

__global__ void mask_copy_kernel(const double *__restrict__ in, double *__restrict__ out,
                                 const uint8_t *__restrict__ mask, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mask[i] ? in[i] : 0.0;
}

__global__ void zero_kernel(double *__restrict__ v, int64_t n, const int *__restrict__ done)
{
    if (done && *done) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 0.0;
}

template <int P>
void ebe_launch(const Grid3 &g, const double *x, double *y, const uint8_t *mask, const double *elem,
                const int2 *cells, const int *off, const int *done, cudaStream_t s)
{
    constexpr int NE = 3 * (P + 1) * (P + 1) * (P + 1);
    for (int c = 0; c < 8; ++c) {
        const int cnt = off[c + 1] - off[c];
        if (cnt > 0) ebe_apply_kernel<P><<<cnt, threads_for(NE), 0, s>>>(x, y, mask, elem, cells + off[c], g, done);
    }
}

template <int P>
void schwarz_launch(const Grid3 &g, const double *r, double *z, const double *f64, const float *f32,
                    const PatchRec *patches, const int *off, const int *done, cudaStream_t s)
{
    constexpr int NB = 3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1);
    for (int c = 0; c < 8; ++c) {
        const int cnt = off[c + 1] - off[c];
        if (cnt > 0) schwarz_apply_kernel<P><<<cnt, threads_for(NB), 0, s>>>(r, z, f64, f32, patches + off[c], g, done);
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_ebe_apply(int p, const Grid3 &g, const double *x, double *y, const uint8_t *mask, const double *elem,
                      const int2 *cells, const int *colour_off, const int *done, cudaStream_t s)
{
    switch (p) {
    case 1: ebe_launch<1>(g, x, y, mask, elem, cells, colour_off, done, s); break;
    case 2: ebe_launch<2>(g, x, y, mask, elem, cells, colour_off, done, s); break;
    case 3: ebe_launch<3>(g, x, y, mask, elem, cells, colour_off, done, s); break;
    case 4: ebe_launch<4>(g, x, y, mask, elem, cells, colour_off, done, s); break;
    default: break;
    }
}

void launch_schwarz_apply(int p, const Grid3 &g, const double *r, double *z, const double *f64, const float *f32,
                          const PatchRec *patches, const int *colour_off, const int *done, cudaStream_t s)
{
    switch (p) {
    case 1: schwarz_launch<1>(g, r, z, f64, f32, patches, colour_off, done, s); break;
    case 2: schwarz_launch<2>(g, r, z, f64, f32, patches, colour_off, done, s); break;
    case 3: schwarz_launch<3>(g, r, z, f64, f32, patches, colour_off, done, s); break;
    case 4: schwarz_launch<4>(g, r, z, f64, f32, patches, colour_off, done, s); break;
    default: break;
    }
}

void launch_mask_copy(const double *in, double *out, const uint8_t *mask, int64_t n, cudaStream_t s)
{
    mask_copy_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, mask, n);
}

void launch_zero(double *v, int64_t n, const int *done, cudaStream_t s)
{
    zero_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n, done);
}

}  // namespace fcm
