// Stiffness apply y = K x of the finite cell Schwarz-PCG on sm_103a (Sec. 2.1 Eq. (1)): cells
// processed in 8 parity colours so that cells of one launch share no lattice DOF and the scatter
// needs no atomics; uncut cells matrix-free by sum factorisation, cut cells with their own dense
// element matrix.  (The Schwarz apply is in fcm_schwarz.cu.)
#include <cuda_runtime.h>

#include <algorithm>

#include "fcm_device.cuh"

namespace fcm {

namespace {

__host__ __device__ constexpr int round32(int v) { return (v + 31) / 32 * 32; }
// One thread per row up to 512 rows; larger blocks loop over rows.
__host__ __device__ constexpr int threads_for(int rows) { return round32(rows) < 512 ? round32(rows) : 512; }

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

// Barrier among the threads of one cell: a warp when the cell's points fit one warp (p <= 2), else
// the CTA.  Only the table load at the start needs the whole CTA.
template <int TPC>
__device__ __forceinline__ void cell_sync()
{
    if constexpr (TPC == 32)
        __syncwarp();
    else
        __syncthreads();
}

// y += K_ref x_e for uncut cells of one colour, without the matrix.  Each displacement
// component is interpolated to the (p+1)^3 Gauss points by one-dimensional contractions along
// x, y, z (sum factorisation); its gradient there follows from the collocation derivative on
// the Gauss points (exact: the field has degree <= p per axis).  The weighted stress
// sigma = lam tr(eps) I + 2 mu eps is formed per point, and the transposed steps give the
// nodal forces.  Exact for the uncut integrand (degree <= 2p per axis), so it equals
// K_ref x_e up to rounding, with 36 (p+1)^4 FP64 multiply-adds per cell (the dense product
// takes 9 (p+1)^6) and no matrix traffic.  Threads of a cell: one per point.
template <int P>
__global__ void __launch_bounds__(256)
    sf_apply_kernel(const double *__restrict__ x, double *__restrict__ y, const uint8_t *__restrict__ mask,
                    const int *__restrict__ cells, int ncells, Grid3 g, SfTables T, const int *__restrict__ done)
{
    constexpr int Q = P + 1, Q3 = Q * Q * Q, TPC = round32(Q3), CPC = 256 / TPC;
    if (done && *done) return;
    __shared__ double sB[Q][Q], sG[3][Q][Q], sW[Q];
    __shared__ double U[CPC][3][Q3];   // nodal values; then the point values per component
    __shared__ double A[CPC][Q3], Bq[CPC][Q3];
    for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) {
        const int q = t / Q, i = t % Q;
        sB[q][i] = T.B[q][i];
        for (int a = 0; a < 3; ++a) sG[a][q][i] = T.G[a][q][i];
    }
    if (threadIdx.x < Q) sW[threadIdx.x] = T.W[threadIdx.x];
    const int lc = threadIdx.x / TPC, t = threadIdx.x % TPC;
    const int cidx = blockIdx.x * CPC + lc;
    const bool on = cidx < ncells && t < Q3;
    const int tx = t % Q, ty = (t / Q) % Q, tz = t / (Q * Q);
    int64_t node = 0;
    if (on) {
        const int cell = cells[cidx];
        const int cx = cell % g.n[0], cy = (cell / g.n[0]) % g.n[1], cz = cell / (g.n[0] * g.n[1]);
        node = (P * cx + tx) + (int64_t)g.M[0] * ((P * cy + ty) + (int64_t)g.M[1] * (P * cz + tz));
        for (int c = 0; c < 3; ++c) U[lc][c][t] = x[3 * node + c];
    }
    __syncthreads();
    // interpolation to the points: (ix,iy,iz) -> (qx,iy,iz) -> (qx,qy,iz) -> (qx,qy,qz)
    double uq[3];
    for (int c = 0; c < 3; ++c) {
        if (on) {
            double s0 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s0 = fma(sB[tx][k], U[lc][c][k + Q * (ty + Q * tz)], s0);
            A[lc][t] = s0;
        }
        cell_sync<TPC>();
        if (on) {
            double s1 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s1 = fma(sB[ty][k], A[lc][tx + Q * (k + Q * tz)], s1);
            Bq[lc][t] = s1;
        }
        cell_sync<TPC>();
        if (on) {
            double s2 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s2 = fma(sB[tz][k], Bq[lc][tx + Q * (ty + Q * k)], s2);
            uq[c] = s2;
        }
    }
    cell_sync<TPC>();  // every point has read the nodal values of its cell
    if (on)
        for (int c = 0; c < 3; ++c) U[lc][c][t] = uq[c];
    cell_sync<TPC>();
    // gradients at the point by the collocation derivative along each axis
    double gr[3][3];
    if (on) {
        for (int c = 0; c < 3; ++c) {
            double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                gx = fma(sG[0][tx][k], U[lc][c][k + Q * (ty + Q * tz)], gx);
                gy = fma(sG[1][ty][k], U[lc][c][tx + Q * (k + Q * tz)], gy);
                gz = fma(sG[2][tz][k], U[lc][c][tx + Q * (ty + Q * k)], gz);
            }
            gr[c][0] = gx;
            gr[c][1] = gy;
            gr[c][2] = gz;
        }
    }
    // weighted stress at the point: F[c][j] = w detJ (lam tr(eps) delta_cj + 2 mu eps_cj)
    double F[3][3];
    if (on) {
        const double w = sW[tx] * sW[ty] * sW[tz] * T.detJ;
        const double ltr = T.lam * (gr[0][0] + gr[1][1] + gr[2][2]);
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j) F[c][j] = w * (T.mu * (gr[c][j] + gr[j][c]) + (c == j ? ltr : 0.0));
    }
    double out[3];
    for (int c = 0; c < 3; ++c) {
        cell_sync<TPC>();  // the previous readers of U and A are done
        if (on)
            for (int j = 0; j < 3; ++j) U[lc][j][t] = F[c][j];
        cell_sync<TPC>();
        if (on) {  // transposed collocation derivative: point values of component c's force
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                v = fma(sG[0][k][tx], U[lc][0][k + Q * (ty + Q * tz)], v);
                v = fma(sG[1][k][ty], U[lc][1][tx + Q * (k + Q * tz)], v);
                v = fma(sG[2][k][tz], U[lc][2][tx + Q * (ty + Q * k)], v);
            }
            A[lc][t] = v;
        }
        cell_sync<TPC>();
        if (on) {  // z^T: (qx, qy, iz)
            double s2 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s2 = fma(sB[k][tz], A[lc][tx + Q * (ty + Q * k)], s2);
            Bq[lc][t] = s2;
        }
        cell_sync<TPC>();
        if (on) {  // y^T: (qx, iy, iz)
            double s1 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s1 = fma(sB[k][ty], Bq[lc][tx + Q * (k + Q * tz)], s1);
            A[lc][t] = s1;
        }
        cell_sync<TPC>();
        if (on) {  // x^T: nodal force (ix, iy, iz)
            double o = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) o = fma(sB[k][tx], A[lc][k + Q * (ty + Q * tz)], o);
            out[c] = o;
        }
    }
    if (on)
        for (int c = 0; c < 3; ++c)
            if (mask[3 * node + c]) y[3 * node + c] += out[c];
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
void k_launch(const Grid3 &g, const double *x, double *y, const uint8_t *mask, const double *elem, const KCells &kc,
              const int *done, cudaStream_t s, const KStreams &ks)
{
    constexpr int NE = 3 * (P + 1) * (P + 1) * (P + 1);
    constexpr int CPC = 256 / round32((P + 1) * (P + 1) * (P + 1));
    for (int c = 0; c < 8; ++c) {
        const int nu = kc.uncut_off[c + 1] - kc.uncut_off[c];
        const int nc = kc.cut_off[c + 1] - kc.cut_off[c];
        // cut and uncut cells of one colour share no DOF: the cut cells may run beside the uncut ones
        const bool fork = ks.side && nu > 0 && nc > 0;
        if (fork) {
            cudaEventRecord(ks.fork, s);
            cudaStreamWaitEvent(ks.side, ks.fork, 0);
        }
        if (nc > 0)
            ebe_apply_kernel<P><<<nc, threads_for(NE), 0, fork ? ks.side : s>>>(x, y, mask, elem, kc.cut + kc.cut_off[c],
                                                                               g, done);
        if (nu > 0)
            sf_apply_kernel<P><<<(nu + CPC - 1) / CPC, 256, 0, s>>>(x, y, mask, kc.uncut + kc.uncut_off[c], nu, g, kc.sf,
                                                                   done);
        if (fork) {
            cudaEventRecord(ks.join, ks.side);
            cudaStreamWaitEvent(s, ks.join, 0);
        }
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_k_apply(int p, const Grid3 &g, const double *x, double *y, const uint8_t *mask, const double *elem,
                    const KCells &kc, const int *done, cudaStream_t s, const KStreams &ks)
{
    switch (p) {
    case 1: k_launch<1>(g, x, y, mask, elem, kc, done, s, ks); break;
    case 2: k_launch<2>(g, x, y, mask, elem, kc, done, s, ks); break;
    case 3: k_launch<3>(g, x, y, mask, elem, kc, done, s, ks); break;
    case 4: k_launch<4>(g, x, y, mask, elem, kc, done, s, ks); break;
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
