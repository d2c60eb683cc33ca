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

// y += K_ref x_e for uncut cells of one colour, without the matrix: the
// displacement gradients at the (p+1)^3 Gauss points are obtained by
// one-dimensional contractions along x, y, z (sum factorisation), the
// weighted stress sigma = lam tr(eps) I + 2 mu eps is formed per point, and the
// transposed contractions give the nodal forces.  Exact for the uncut
// integrand (degree <= 2p per axis), so it equals K_ref x_e up to rounding
// with (p+1)^3 * 24 * ... ~ 2.7x fewer FP64 multiply-adds than the dense
// product at p = 3 and no matrix traffic.  Threads of a cell: one per point.
template <int P>
__global__ void __launch_bounds__(256)
    sf_apply_kernel(const double *__restrict__ x, double *__restrict__ y, const uint8_t *__restrict__ mask,
                    const int *__restrict__ cells, int ncells, Grid3 g, SfTables T, const int *__restrict__ done)
{
    constexpr int Q = P + 1, Q3 = Q * Q * Q, TPC = round32(Q3), CPC = 256 / TPC;
    if (done && *done) return;
    __shared__ double sB[Q][Q], sD[3][Q][Q], sW[Q];
    __shared__ double U[CPC][3][Q3];
    __shared__ double S0[CPC][Q3], S1[CPC][Q3], S2[CPC][Q3];
    __shared__ double R0[CPC][Q3], R1[CPC][Q3], R2[CPC][Q3];
    for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) {
        const int q = t / Q, i = t % Q;
        sB[q][i] = T.B[q][i];
        for (int a = 0; a < 3; ++a) sD[a][q][i] = T.D[a][q][i];
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
    double gr[3][3];
    for (int c = 0; c < 3; ++c) {
        if (on) {  // x: S0 = B u, S1 = D_x u at (qx, iy, iz)
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const double u = U[lc][c][k + Q * (ty + Q * tz)];
                s0 = fma(sB[tx][k], u, s0);
                s1 = fma(sD[0][tx][k], u, s1);
            }
            S0[lc][t] = s0;
            S1[lc][t] = s1;
        }
        __syncthreads();
        if (on) {  // y: R0 = B S0, R1 = D_y S0, R2 = B S1 at (qx, qy, iz)
            double r0 = 0.0, r1 = 0.0, r2 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int id = tx + Q * (k + Q * tz);
                const double a = S0[lc][id], b = S1[lc][id];
                r0 = fma(sB[ty][k], a, r0);
                r1 = fma(sD[1][ty][k], a, r1);
                r2 = fma(sB[ty][k], b, r2);
            }
            R0[lc][t] = r0;
            R1[lc][t] = r1;
            R2[lc][t] = r2;
        }
        __syncthreads();
        if (on) {  // z: gradient of u_c at the point (qx, qy, qz)
            double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int id = tx + Q * (ty + Q * k);
                gx = fma(sB[tz][k], R2[lc][id], gx);
                gy = fma(sB[tz][k], R1[lc][id], gy);
                gz = fma(sD[2][tz][k], R0[lc][id], gz);
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
        __syncthreads();
        if (on) {
            R0[lc][t] = F[c][0];
            R1[lc][t] = F[c][1];
            R2[lc][t] = F[c][2];
        }
        __syncthreads();
        if (on) {  // z^T: (qx, qy, iz)
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int id = tx + Q * (ty + Q * k);
                s0 = fma(sB[k][tz], R0[lc][id], s0);
                s1 = fma(sB[k][tz], R1[lc][id], s1);
                s2 = fma(sD[2][k][tz], R2[lc][id], s2);
            }
            S0[lc][t] = s0;
            S1[lc][t] = s1;
            S2[lc][t] = s2;
        }
        __syncthreads();
        if (on) {  // y^T: (qx, iy, iz)
            double r0 = 0.0, r1 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int id = tx + Q * (k + Q * tz);
                r0 = fma(sB[k][ty], S0[lc][id], r0);
                r1 = fma(sD[1][k][ty], S1[lc][id], r1);
                r1 = fma(sB[k][ty], S2[lc][id], r1);
            }
            R0[lc][t] = r0;
            R1[lc][t] = r1;
        }
        __syncthreads();
        if (on) {  // x^T: nodal force (ix, iy, iz)
            double o = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int id = k + Q * (ty + Q * tz);
                o = fma(sD[0][k][tx], R0[lc][id], o);
                o = fma(sB[k][tx], R1[lc][id], o);
            }
            out[c] = o;
        }
    }
    if (on)
        for (int c = 0; c < 3; ++c)
            if (mask[3 * node + c]) y[3 * node + c] += out[c];
}

// Work kinds of the Schwarz apply, stored in bits 8.. of a batch's .y (bits 0..7: patch count).
enum { kF32Shared = 0, kF32Single = 1, kF64Shared = 2, kF64Single = 3 };

// z += F r_B for the `count` patches of one batch, which share the stored
// factor F (shared batches, up to G patches) or have their own (G = 1).  F is
// the dense symmetric pseudo inverse over the patch box (zero rows/columns
// for box DOFs outside the block), stored in T = double or float.  Each
// thread owns rows of the box; one load of F[j][t] feeds G multiply-adds, so
// a shared factor is read once per batch instead of once per patch.  The
// gathered residuals sit in shared memory as rbT[j][g], so one vector load
// returns the G values a row step needs.  UNROLL sets the loads in flight
// per thread (cut patches stream their factor from DRAM and are latency-bound).
template <int P, int G, typename T, int UNROLL>
__device__ __forceinline__ void apply_batch(const double *__restrict__ r, double *__restrict__ z,
                                            const T *__restrict__ pool, const PatchRec *__restrict__ patches,
                                            int first, int count, const Grid3 &g, unsigned char *smem)
{
    constexpr int W = 2 * P - 1, NB = 3 * W * W * W;
    T(*rbT)[G] = reinterpret_cast<T(*)[G]>(smem);
    int *vtx = reinterpret_cast<int *>(smem + sizeof(T) * NB * G);
    const int nvx = g.n[0] + 1, nvy = g.n[1] + 1;
    const PatchRec p0 = patches[first];
    if (threadIdx.x < G) vtx[threadIdx.x] = (int)threadIdx.x < count ? patches[first + threadIdx.x].v : -1;
    // the patches of a batch share the factor, hence the box shape; the origin differs
    int d[3];
    {
        const int v[3] = {p0.v % nvx, (p0.v / nvx) % nvy, p0.v / (nvx * nvy)};
        for (int a = 0; a < 3; ++a) {
            const int lo = max(0, P * v[a] - (P - 1));
            d[a] = min(g.M[a] - 1, P * v[a] + (P - 1)) - lo + 1;
        }
    }
    const int n = 3 * d[0] * d[1] * d[2];
    __syncthreads();
    auto gidx = [&](int vv, int t) -> int64_t {
        const int v0 = vv % nvx, v1 = (vv / nvx) % nvy, v2 = vv / (nvx * nvy);
        const int l0 = max(0, P * v0 - (P - 1)), l1 = max(0, P * v1 - (P - 1)), l2 = max(0, P * v2 - (P - 1));
        const int nl = t / 3;
        const int ix = nl % d[0], iy = (nl / d[0]) % d[1], iz = nl / (d[0] * d[1]);
        return 3 * ((l0 + ix) + (int64_t)g.M[0] * ((l1 + iy) + (int64_t)g.M[1] * (l2 + iz))) + t % 3;
    };
    for (int e = threadIdx.x; e < n * G; e += blockDim.x) {
        const int t = e / G, k = e % G;
        const int vv = vtx[k];
        rbT[t][k] = vv >= 0 ? (T)r[gidx(vv, t)] : (T)0;
    }
    __syncthreads();
    const T *__restrict__ F = pool + p0.off;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        T acc[G];
#pragma unroll
        for (int k = 0; k < G; ++k) acc[k] = (T)0;
#pragma unroll UNROLL
        for (int j = 0; j < n; ++j) {
            const T f = __ldg(F + (size_t)j * n + t);
#pragma unroll
            for (int k = 0; k < G; ++k) acc[k] = fma(f, rbT[j][k], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < G; ++k)
            if (vtx[k] >= 0) z[gidx(vtx[k], t)] += (double)acc[k];
    }
}

// Several right-hand sides (nr <= 8, vectors nlat apart): z_k += F r_k,B for each patch of
// the work item, one patch after the other; one load of F[j][t] feeds nr multiply-adds.
template <int P, typename T, int UNROLL>
__device__ __forceinline__ void apply_multi(const double *__restrict__ r, double *__restrict__ z, int64_t nlat, int nr,
                                            const T *__restrict__ pool, const PatchRec *__restrict__ patches,
                                            int first, int count, const Grid3 &g, unsigned char *smem)
{
    constexpr int W = 2 * P - 1, NB = 3 * W * W * W, MR = 8;
    T(*rbT)[MR] = reinterpret_cast<T(*)[MR]>(smem);
    const int nvx = g.n[0] + 1, nvy = g.n[1] + 1;
    for (int b = 0; b < count; ++b) {
        const PatchRec pr = patches[first + b];
        const int v[3] = {pr.v % nvx, (pr.v / nvx) % nvy, pr.v / (nvx * nvy)};
        int lo[3], d[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = max(0, P * v[a] - (P - 1));
            d[a] = min(g.M[a] - 1, P * v[a] + (P - 1)) - lo[a] + 1;
        }
        const int n = 3 * d[0] * d[1] * d[2];
        auto gidx = [&](int t) -> int64_t {
            const int nl = t / 3;
            const int ix = nl % d[0], iy = (nl / d[0]) % d[1], iz = nl / (d[0] * d[1]);
            return 3 * ((lo[0] + ix) + (int64_t)g.M[0] * ((lo[1] + iy) + (int64_t)g.M[1] * (lo[2] + iz))) + t % 3;
        };
        __syncthreads();
        for (int e = threadIdx.x; e < n * MR; e += blockDim.x) {
            const int t = e / MR, k = e % MR;
            rbT[t][k] = k < nr ? (T)r[(int64_t)k * nlat + gidx(t)] : (T)0;
        }
        __syncthreads();
        const T *__restrict__ F = pool + pr.off;
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            T acc[MR];
#pragma unroll
            for (int k = 0; k < MR; ++k) acc[k] = (T)0;
#pragma unroll UNROLL
            for (int j = 0; j < n; ++j) {
                const T f = __ldg(F + (size_t)j * n + t);
#pragma unroll
                for (int k = 0; k < MR; ++k) acc[k] = fma(f, rbT[j][k], acc[k]);
            }
            const int64_t gi = gidx(t);
            for (int k = 0; k < nr; ++k) z[(int64_t)k * nlat + gi] += (double)acc[k];
        }
    }
}

// One colour of the Schwarz apply for nr right-hand sides at once (multi-RHS solves).
template <int P>
__global__ void __launch_bounds__(threads_for(3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1)))
    schwarz_multi_kernel(const double *__restrict__ r, double *__restrict__ z, int64_t nlat, int nr,
                         const double *__restrict__ f64, const float *__restrict__ f32,
                         const PatchRec *__restrict__ patches, const int2 *__restrict__ batches, Grid3 g,
                         const int *__restrict__ done)
{
    constexpr int W = 2 * P - 1, NB = 3 * W * W * W;
    __shared__ __align__(16) unsigned char smem[NB * 8 * (P == 4 ? 4 : 8)];
    if (done && *done) return;
    const int2 bt = batches[blockIdx.x];
    const int count = bt.y & 255, kind = bt.y >> 8;
    if (kind == kF32Shared || kind == kF32Single)
        apply_multi<P, float, 8>(r, z, nlat, nr, f32, patches, bt.x, count, g, smem);
    else if (P < 4)
        apply_multi<P, double, 8>(r, z, nlat, nr, f64, patches, bt.x, count, g, smem);
}

// One colour of the Schwarz apply (Sec. 3.1 Eq. (5)): each CTA takes one work
// item (a shared-factor batch or a single patch, FP32 or FP64 factor).  The
// patches of one colour are DOF-disjoint, so the scatter needs no atomics.
template <int P>
__global__ void __launch_bounds__(threads_for(3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1)))
    schwarz_colour_kernel(const double *__restrict__ r, double *__restrict__ z, const double *__restrict__ f64,
                          const float *__restrict__ f32, const PatchRec *__restrict__ patches,
                          const int2 *__restrict__ batches, Grid3 g, const int *__restrict__ done)
{
    constexpr int W = 2 * P - 1, NB = 3 * W * W * W, GD = (P == 4 ? 4 : 8);
    constexpr int ROW = (GD * 8 > 8 * 4 ? GD * 8 : 8 * 4);  // bytes of one rbT row, largest variant
    __shared__ __align__(16) unsigned char smem[NB * ROW + 64];
    if (done && *done) return;
    const int2 bt = batches[blockIdx.x];
    const int count = bt.y & 255, kind = bt.y >> 8;
    switch (kind) {
    case kF32Shared: apply_batch<P, 8, float, 4>(r, z, f32, patches, bt.x, count, g, smem); break;
    case kF32Single: apply_batch<P, 1, float, 16>(r, z, f32, patches, bt.x, count, g, smem); break;
    case kF64Shared: apply_batch<P, GD, double, 4>(r, z, f64, patches, bt.x, count, g, smem); break;
    default: apply_batch<P, 1, double, 16>(r, z, f64, patches, bt.x, count, g, smem); break;
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
void k_launch(const Grid3 &g, const double *x, double *y, const uint8_t *mask, const double *elem, const KCells &kc,
              const int *done, cudaStream_t s)
{
    constexpr int NE = 3 * (P + 1) * (P + 1) * (P + 1);
    constexpr int CPC = 256 / round32((P + 1) * (P + 1) * (P + 1));
    for (int c = 0; c < 8; ++c) {
        const int nu = kc.uncut_off[c + 1] - kc.uncut_off[c];
        if (nu > 0)
            sf_apply_kernel<P><<<(nu + CPC - 1) / CPC, 256, 0, s>>>(x, y, mask, kc.uncut + kc.uncut_off[c], nu, g, kc.sf,
                                                                   done);
        const int nc = kc.cut_off[c + 1] - kc.cut_off[c];
        if (nc > 0) ebe_apply_kernel<P><<<nc, threads_for(NE), 0, s>>>(x, y, mask, elem, kc.cut + kc.cut_off[c], g, done);
    }
}

template <int P>
void schwarz_launch(const Grid3 &g, const double *r, double *z, const double *f64, const float *f32,
                    const SchwarzPlan &plan, const int *done, cudaStream_t s)
{
    constexpr int NB = 3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1);
    for (int i = 0; i < plan.nseg; ++i) {
        const SchwarzSeg &sg = plan.seg[i];
        if (sg.count > 0)
            schwarz_colour_kernel<P><<<sg.count, threads_for(NB), 0, s>>>(r, z, f64, f32, plan.patches,
                                                                         plan.batches + sg.first, g, done);
    }
}

template <int P>
void schwarz_multi_launch(const Grid3 &g, const double *r, double *z, int64_t nlat, int nr, const double *f64,
                          const float *f32, const SchwarzPlan &plan, const int *done, cudaStream_t s)
{
    constexpr int NB = 3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1);
    for (int i = 0; i < plan.nseg; ++i) {
        const SchwarzSeg &sg = plan.seg[i];
        if (sg.count > 0)
            schwarz_multi_kernel<P><<<sg.count, threads_for(NB), 0, s>>>(r, z, nlat, nr, f64, f32, plan.patches,
                                                                        plan.batches + sg.first, g, done);
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
                    const KCells &kc, const int *done, cudaStream_t s)
{
    switch (p) {
    case 1: k_launch<1>(g, x, y, mask, elem, kc, done, s); break;
    case 2: k_launch<2>(g, x, y, mask, elem, kc, done, s); break;
    case 3: k_launch<3>(g, x, y, mask, elem, kc, done, s); break;
    case 4: k_launch<4>(g, x, y, mask, elem, kc, done, s); break;
    default: break;
    }
}

void launch_schwarz_apply(int p, const Grid3 &g, const double *r, double *z, const double *f64, const float *f32,
                          const SchwarzPlan &plan, const int *done, cudaStream_t s)
{
    switch (p) {
    case 1: schwarz_launch<1>(g, r, z, f64, f32, plan, done, s); break;
    case 2: schwarz_launch<2>(g, r, z, f64, f32, plan, done, s); break;
    case 3: schwarz_launch<3>(g, r, z, f64, f32, plan, done, s); break;
    case 4: schwarz_launch<4>(g, r, z, f64, f32, plan, done, s); break;
    default: break;
    }
}

void launch_schwarz_apply_multi(int p, const Grid3 &g, const double *r, double *z, int64_t nlat, int nr,
                                const double *f64, const float *f32, const SchwarzPlan &plan, const int *done,
                                cudaStream_t s)
{
    switch (p) {
    case 1: schwarz_multi_launch<1>(g, r, z, nlat, nr, f64, f32, plan, done, s); break;
    case 2: schwarz_multi_launch<2>(g, r, z, nlat, nr, f64, f32, plan, done, s); break;
    case 3: schwarz_multi_launch<3>(g, r, z, nlat, nr, f64, f32, plan, done, s); break;
    case 4: schwarz_multi_launch<4>(g, r, z, nlat, nr, f64, f32, plan, done, s); break;
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
