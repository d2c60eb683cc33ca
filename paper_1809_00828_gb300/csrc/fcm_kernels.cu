// Hot kernels of the finite cell Schwarz-PCG on sm_103a:
//  * element-by-element stiffness apply y = K x (Sec. 2.1 Eq. (1)), one CTA
//    per active cell, cells processed in 8 parity colours so that cells of one
//    launch share no lattice DOF and the scatter needs no atomics;
//  * Additive-Schwarz apply z = D r + sum_B R_B^T A_B+^-1 R_B r (Sec. 3.1
//    Eq. (5), Algorithm 1): diagonal part D for the DOFs in no block, then
//    gather r over the block box, dense symmetric block apply, scatter into z,
//    blocks (vertex patches or element blocks) processed in 8 parity colours
//    (blocks of one colour are DOF-disjoint).
#include <cuda_runtime.h>

#include <algorithm>

#include "fcm_device.cuh"

namespace fcm {

namespace {

__host__ __device__ constexpr int round32(int v) { return (v + 31) / 32 * 32; }
// One thread per row up to 512 rows; larger blocks loop over rows.
__host__ __device__ constexpr int threads_for(int rows) { return round32(rows) < 512 ? round32(rows) : 512; }

// Lattice width of the largest block box: vertex patches span 2p - 1 nodes per axis, element
// blocks p + 1 (the wider of the two at p = 1).
__host__ __device__ constexpr int box_width(int P) { return 2 * P - 1 > P + 1 ? 2 * P - 1 : P + 1; }

// Threads of a Schwarz CTA: one per row of the largest block of the rule.
__host__ __device__ constexpr int schwarz_threads(int P, int rule)
{
    return rule == 3 ? threads_for(3 * (P + 1) * (P + 1) * (P + 1)) : threads_for(3 * (2 * P - 1) * (2 * P - 1) * (2 * P - 1));
}

// Lattice box of block `id`: rule 0, the vertex patch of vertex id, [p v - (p-1), p v + (p-1)]
// clipped to the lattice; rule 3, the element block of cell id, [p c, p c + p].
__device__ __forceinline__ void block_box(int rule, int P, const Grid3 &g, int id, int lo[3], int d[3])
{
    if (rule == 3) {
        const int c[3] = {id % g.n[0], (id / g.n[0]) % g.n[1], id / (g.n[0] * g.n[1])};
        for (int a = 0; a < 3; ++a) {
            lo[a] = P * c[a];
            d[a] = P + 1;
        }
    } else {
        const int nvx = g.n[0] + 1, nvy = g.n[1] + 1;
        const int v[3] = {id % nvx, (id / nvx) % nvy, id / (nvx * nvy)};
        for (int a = 0; a < 3; ++a) {
            lo[a] = max(0, P * v[a] - (P - 1));
            d[a] = min(g.M[a] - 1, P * v[a] + (P - 1)) - lo[a] + 1;
        }
    }
}

// 16-byte vectors of float (4) or double (2): load type, dot-accumulate, element access.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float dot(float4 a, float4 b, float c)
    {
        return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, c))));
    }
    __device__ static float get(float4 a, int e) { return e == 0 ? a.x : e == 1 ? a.y : e == 2 ? a.z : a.w; }
};
template <> struct Vec16<double> {
    using type = double2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double dot(double2 a, double2 b, double c) { return fma(a.y, b.y, fma(a.x, b.x, c)); }
    __device__ static double get(double2 a, int e) { return e == 0 ? a.x : a.y; }
};

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
        __syncthreads();
        if (on) {
            double s1 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s1 = fma(sB[ty][k], A[lc][tx + Q * (k + Q * tz)], s1);
            Bq[lc][t] = s1;
        }
        __syncthreads();
        if (on) {
            double s2 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s2 = fma(sB[tz][k], Bq[lc][tx + Q * (ty + Q * k)], s2);
            uq[c] = s2;
        }
    }
    __syncthreads();  // every point has read the nodal values of its cell
    if (on)
        for (int c = 0; c < 3; ++c) U[lc][c][t] = uq[c];
    __syncthreads();
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
        __syncthreads();  // the previous readers of U and A are done
        if (on)
            for (int j = 0; j < 3; ++j) U[lc][j][t] = F[c][j];
        __syncthreads();
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
        __syncthreads();
        if (on) {  // z^T: (qx, qy, iz)
            double s2 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s2 = fma(sB[k][tz], A[lc][tx + Q * (ty + Q * k)], s2);
            Bq[lc][t] = s2;
        }
        __syncthreads();
        if (on) {  // y^T: (qx, iy, iz)
            double s1 = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s1 = fma(sB[k][ty], Bq[lc][tx + Q * (k + Q * tz)], s1);
            A[lc][t] = s1;
        }
        __syncthreads();
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

// Work kinds of the Schwarz apply, stored in bits 8.. of a work item's .y.  Bits 0..7 hold the
// block count of a shared-factor batch, or the row tile index of a block with its own factor.
enum { kF32Shared = 0, kF32Single = 1, kF64Shared = 2, kF64Single = 3 };

// z += F r_B for the `count` blocks of one batch, which share the stored factor F
// (up to G blocks).  F is the dense symmetric pseudo inverse over the block box (zero
// rows/columns for box DOFs outside the block), stored in T = double or float.  Each
// thread owns rows of the box; one load of F[j][t] feeds G multiply-adds, so a shared
// factor is read once per batch instead of once per block.  The gathered residuals sit in
// shared memory as rbT[j][g], so one vector load returns the G values a row step needs.
// The blocks of a batch have the same box shape, so a box entry's lattice index is the
// block's base plus an offset common to the batch: both are tabulated once per CTA.
template <int P, int G, typename T, int UNROLL>
__device__ __forceinline__ void apply_batch(const double *__restrict__ r, double *__restrict__ z,
                                            const T *__restrict__ pool, const PatchRec *__restrict__ patches,
                                            int first, int count, const Grid3 &g, int rule, unsigned char *smem)
{
    constexpr int W = box_width(P), NB = 3 * W * W * W;
    T(*rbT)[G] = reinterpret_cast<T(*)[G]>(smem);
    // G entries, -1: no block; 16-byte aligned after rbT (4 NB bytes for one FP32 block)
    int64_t *base = reinterpret_cast<int64_t *>(smem + (sizeof(T) * NB * G + 15) / 16 * 16);
    int *rel = reinterpret_cast<int *>(base + G);  // NB entries
    const PatchRec p0 = patches[first];
    int lo0[3], d[3];
    block_box(rule, P, g, p0.v, lo0, d);
    const int n = 3 * d[0] * d[1] * d[2];
    if (threadIdx.x < G) {
        int64_t b = -1;
        if ((int)threadIdx.x < count) {
            int l[3], dd[3];
            block_box(rule, P, g, patches[first + threadIdx.x].v, l, dd);
            b = 3 * (l[0] + (int64_t)g.M[0] * (l[1] + (int64_t)g.M[1] * l[2]));
        }
        base[threadIdx.x] = b;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int nl = t / 3;
        const int ix = nl % d[0], iy = (nl / d[0]) % d[1], iz = nl / (d[0] * d[1]);
        rel[t] = 3 * (ix + g.M[0] * (iy + g.M[1] * iz)) + t % 3;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * G; e += blockDim.x) {
        const int t = e / G, k = e % G;
        const int64_t b = base[k];
        rbT[t][k] = b >= 0 ? (T)r[b + rel[t]] : (T)0;
    }
    __syncthreads();
    const T *__restrict__ F = pool + p0.off;
    const int ld = factor_ld<T>(n);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        T acc[G];
#pragma unroll
        for (int k = 0; k < G; ++k) acc[k] = (T)0;
#pragma unroll UNROLL
        for (int j = 0; j < n; ++j) {
            const T f = __ldg(F + (size_t)j * ld + t);
#pragma unroll
            for (int k = 0; k < G; ++k) acc[k] = fma(f, rbT[j][k], acc[k]);
        }
        const int rt = rel[t];
#pragma unroll
        for (int k = 0; k < G; ++k)
            if (base[k] >= 0) z[base[k] + rt] += (double)acc[k];
    }
}

// ---- bulk copies (cp.async.bulk, global -> shared) completed on an mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the single arrival of the barrier's phase, announcing `bytes` of bulk copies
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// dst, src and bytes multiples of 16
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier; gives up (false) after a bounded number of tries.
constexpr int kWaitTries = 1 << 21;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (int i = 0; i < kWaitTries; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Bytes in front of the factor tile in the Schwarz kernel's dynamic shared memory: the
// mbarrier (16) and the gathered residual r_B in T, padded to the factor's row length.
template <int P>
__host__ __device__ constexpr int rows_tile_offset()
{
    return 16 + (factor_ld<double>(3 * box_width(P) * box_width(P) * box_width(P)) * 8 + 15) / 16 * 16;
}

// Small blocks (p <= 2: 81 DOFs at most) are applied whole, one item each, with each thread
// streaming its row straight from the factor pool: their few kilobytes do not amortise a staged
// bulk copy.  Larger blocks go through row tiles.
template <int P>
__host__ __device__ constexpr bool direct_singles()
{
    return P <= 2;
}

// Blocks per FP32 shared-factor batch: each load of a factor entry (from L2: shared factors are
// few) feeds that many multiply-adds.  (16 measured slower than 8 at p = 3: more registers, no
// less time.)
template <int P>
__host__ __device__ constexpr int f32_batch_cap()
{
    return 8;
}

// Row tiles of a block with its own factor (cut blocks stream their factor from DRAM): rows
// [row0, row0 + rows) of z_B += F r_B.  The rows of a tile are contiguous in the factor pool (the
// factor is symmetric, rows padded to 16 bytes), so one thread starts them on their way into
// shared memory as bulk copies completed on an mbarrier (tile_issue); the CTA gathers r_B
// meanwhile (tile_gather), waits, and applies the rows (tile_apply): each warp takes 4 (FP32)
// or 2 (FP64) rows at a time, its lanes split a row into 16-byte vectors (r_B's vectors stay in
// registers across rows), and warp shuffles finish the sums.

struct TileGeom {
    int lo[3], d[3], n, ld, row1;
};

template <int P, typename T>
__device__ __forceinline__ TileGeom tile_geom(const PatchRec &pr, int row0, int rows, const Grid3 &g, int rule)
{
    TileGeom t;
    block_box(rule, P, g, pr.v, t.lo, t.d);
    t.n = 3 * t.d[0] * t.d[1] * t.d[2];
    t.ld = factor_ld<T>(t.n);
    t.row1 = min(t.n, row0 + rows);
    return t;
}

__device__ __forceinline__ int64_t tile_gidx(const TileGeom &tg, const Grid3 &g, int t)
{
    const int nl = t / 3;
    const int ix = nl % tg.d[0], iy = (nl / tg.d[0]) % tg.d[1], iz = nl / (tg.d[0] * tg.d[1]);
    return 3 * ((tg.lo[0] + ix) + (int64_t)g.M[0] * ((tg.lo[1] + iy) + (int64_t)g.M[1] * (tg.lo[2] + iz))) + t % 3;
}

// One thread: announce and start the bulk copies of the tile's rows into `tile`.
template <int P, typename T>
__device__ __forceinline__ void tile_issue(const T *__restrict__ pool, const PatchRec &pr, int row0, const TileGeom &tg,
                                           unsigned char *tile, uint64_t *bar)
{
    const uint32_t bytes = (uint32_t)((tg.row1 - row0) * tg.ld * (int)sizeof(T));
    const char *src = reinterpret_cast<const char *>(pool + pr.off + (size_t)row0 * tg.ld);
    mbar_expect(bar, bytes);
    constexpr uint32_t kChunk = 16384;
    for (uint32_t o = 0; o < bytes; o += kChunk)
        bulk_load(tile + o, src + o, bytes - o < kChunk ? bytes - o : kChunk, bar);
}

// All threads: r_B into rb, zero-padded to the row length.
template <typename T>
__device__ __forceinline__ void tile_gather(const double *__restrict__ r, const TileGeom &tg, const Grid3 &g, T *rb)
{
    for (int t = threadIdx.x; t < tg.ld; t += blockDim.x) rb[t] = t < tg.n ? (T)r[tile_gidx(tg, g, t)] : (T)0;
}

// All threads, once the tile has landed: z_B[rows] += F[rows, :] r_B.
template <int P, typename T>
__device__ __forceinline__ void tile_apply(double *__restrict__ z, const TileGeom &tg, const Grid3 &g, int row0,
                                           const T *rb, const T *tile)
{
    using VT = typename Vec16<T>::type;
    constexpr int W = box_width(P), NB = 3 * W * W * W, V = 16 / (int)sizeof(T);
    constexpr int KV = (factor_ld<T>(NB) / V + 31) / 32;  // 16-byte vectors per lane and row
    constexpr int RPW = sizeof(T) == 8 ? 2 : 4;          // rows per warp and pass
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nv = tg.ld / V, row1 = tg.row1, ld = tg.ld;
    const VT *rbv = reinterpret_cast<const VT *>(rb);
    VT xr[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) xr[k] = lane + 32 * k < nv ? rbv[lane + 32 * k] : Vec16<T>::zero();
    for (int t = row0 + RPW * w; t < row1; t += RPW * nw) {
        T a[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            // rows past row1 repeat the last row (in bounds) and are not written
            const VT *fr = reinterpret_cast<const VT *>(tile + (size_t)(min(t + q, row1 - 1) - row0) * ld);
            T acc = (T)0;
#pragma unroll
            for (int k = 0; k < KV; ++k)
                if (lane + 32 * k < nv) acc = Vec16<T>::dot(fr[lane + 32 * k], xr[k], acc);
            a[q] = acc;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < RPW; ++q) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
        if (lane < RPW && t + lane < row1) {
            T v = a[0];
#pragma unroll
            for (int q = 1; q < RPW; ++q)
                if (lane == q) v = a[q];
            z[tile_gidx(tg, g, t + lane)] += (double)v;
        }
    }
}

// One row tile as one work item of a CTA: issue, gather while the copies fly, wait, apply.  A
// wait that runs out sets *err and the CTA returns without writing.
template <int P, typename T>
__device__ __forceinline__ void apply_rows(const double *__restrict__ r, double *__restrict__ z,
                                           const T *__restrict__ pool, const PatchRec *__restrict__ patches,
                                           int first, int row0, int rows, const Grid3 &g, int rule,
                                           unsigned char *smem, int *err)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *rb = reinterpret_cast<T *>(smem + 16);
    unsigned char *tile = smem + rows_tile_offset<P>();
    const PatchRec pr = patches[first];
    const TileGeom tg = tile_geom<P, T>(pr, row0, rows, g, rule);
    if (threadIdx.x == 0) {
        mbar_init(bar);
        tile_issue<P, T>(pool, pr, row0, tg, tile, bar);
    }
    tile_gather<T>(r, tg, g, rb);
    __syncthreads();  // r_B gathered; the barrier is initialised
    if (!__syncthreads_and(mbar_wait(bar, 0))) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            mbar_wait(bar, 0);  // let the copies still in flight land before the CTA leaves
        }
        __syncthreads();
        return;
    }
    tile_apply<P, T>(z, tg, g, row0, rb, reinterpret_cast<const T *>(tile));
}

// Rows [row0, row0 + rows) of z_k,B += F r_k,B for nr <= 8 right-hand sides (vectors nlat
// apart) of a block with its own factor: warp-per-row as in apply_rows, two rows at a time,
// each lane holding nr partial sums per row; one load of F feeds nr multiply-adds.  A lane
// visits the same 16-byte vectors of a row in the same order as apply_rows, so each
// right-hand side gets exactly the single-vector result.
template <int P, typename T>
__device__ __forceinline__ void apply_multi_rows(const double *__restrict__ r, double *__restrict__ z, int64_t nlat,
                                                 int nr, const T *__restrict__ pool,
                                                 const PatchRec *__restrict__ patches, int first, int row0, int rows,
                                                 const Grid3 &g, int rule, unsigned char *smem)
{
    using VT = typename Vec16<T>::type;
    constexpr int MR = 8, V = 16 / (int)sizeof(T);
    T(*rbT)[MR] = reinterpret_cast<T(*)[MR]>(smem);
    const PatchRec pr = patches[first];
    int lo[3], d[3];
    block_box(rule, P, g, pr.v, lo, d);
    const int n = 3 * d[0] * d[1] * d[2], ld = factor_ld<T>(n);
    auto gidx = [&](int t) -> int64_t {
        const int nl = t / 3;
        const int ix = nl % d[0], iy = (nl / d[0]) % d[1], iz = nl / (d[0] * d[1]);
        return 3 * ((lo[0] + ix) + (int64_t)g.M[0] * ((lo[1] + iy) + (int64_t)g.M[1] * (lo[2] + iz))) + t % 3;
    };
    for (int e = threadIdx.x; e < ld * MR; e += blockDim.x) {
        const int t = e / MR, k = e % MR;
        rbT[t][k] = (k < nr && t < n) ? (T)r[(int64_t)k * nlat + gidx(t)] : (T)0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int row1 = min(n, row0 + rows), nv = ld / V;
    const T *__restrict__ F = pool + pr.off;
    for (int t = row0 + 2 * w; t < row1; t += 2 * nw) {
        const VT *f0 = reinterpret_cast<const VT *>(F + (size_t)t * ld);
        const VT *f1 = reinterpret_cast<const VT *>(F + (size_t)min(t + 1, row1 - 1) * ld);
        T a[2][MR];
#pragma unroll
        for (int k = 0; k < MR; ++k) a[0][k] = a[1][k] = (T)0;
        for (int c = lane; c < nv; c += 32) {
            const VT g0 = __ldg(f0 + c), g1 = __ldg(f1 + c);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int j = c * V + e;
                const T v0 = Vec16<T>::get(g0, e), v1 = Vec16<T>::get(g1, e);
#pragma unroll
                for (int k = 0; k < MR; ++k) {
                    a[0][k] = fma(v0, rbT[j][k], a[0][k]);
                    a[1][k] = fma(v1, rbT[j][k], a[1][k]);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < MR; ++k) {
                a[0][k] += __shfl_xor_sync(0xffffffffu, a[0][k], o);
                a[1][k] += __shfl_xor_sync(0xffffffffu, a[1][k], o);
            }
        // lane 8 h + k writes row t + h, right-hand side k
        const int h = lane >> 3, k = lane & 7;
        if (h < 2 && k < nr && t + h < row1) {
            T v = (T)0;
#pragma unroll
            for (int kk = 0; kk < MR; ++kk)
                if (kk == k) v = h == 0 ? a[0][kk] : a[1][kk];
            z[(int64_t)k * nlat + gidx(t + h)] += (double)v;
        }
    }
}

// Several right-hand sides (nr <= 8, vectors nlat apart): z_k += F r_k,B for each block of a
// shared-factor batch, one block after the other; one load of F[j][t] feeds nr multiply-adds.
template <int P, typename T, int UNROLL>
__device__ __forceinline__ void apply_multi(const double *__restrict__ r, double *__restrict__ z, int64_t nlat, int nr,
                                            const T *__restrict__ pool, const PatchRec *__restrict__ patches,
                                            int first, int count, const Grid3 &g, int rule, unsigned char *smem)
{
    constexpr int MR = 8;
    T(*rbT)[MR] = reinterpret_cast<T(*)[MR]>(smem);
    for (int b = 0; b < count; ++b) {
        const PatchRec pr = patches[first + b];
        int lo[3], d[3];
        block_box(rule, P, g, pr.v, lo, d);
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
        const int ld = factor_ld<T>(n);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            T acc[MR];
#pragma unroll
            for (int k = 0; k < MR; ++k) acc[k] = (T)0;
#pragma unroll UNROLL
            for (int j = 0; j < n; ++j) {
                const T f = __ldg(F + (size_t)j * ld + t);
#pragma unroll
                for (int k = 0; k < MR; ++k) acc[k] = fma(f, rbT[j][k], acc[k]);
            }
            const int64_t gi = gidx(t);
#pragma unroll
            for (int k = 0; k < MR; ++k)
                if (k < nr) z[(int64_t)k * nlat + gi] += (double)acc[k];
        }
    }
}

// One colour of the Schwarz apply for nr right-hand sides at once (multi-RHS solves).
template <int P>
__global__ void __launch_bounds__(threads_for(3 * box_width(P) * box_width(P) * box_width(P)))
    schwarz_multi_kernel(const double *__restrict__ r, double *__restrict__ z, int64_t nlat, int nr,
                         const double *__restrict__ f64, const float *__restrict__ f32,
                         const PatchRec *__restrict__ patches, const int2 *__restrict__ batches, Grid3 g, int rule,
                         int rows32, int rows64, const int *__restrict__ done)
{
    constexpr int W = box_width(P), NB = 3 * W * W * W;
    __shared__ __align__(16) unsigned char smem[factor_ld<double>(NB) * 8 * (P == 4 ? 4 : 8)];
    if (done && *done) return;
    const int2 bt = batches[blockIdx.x];
    const int count = bt.y & 255, kind = bt.y >> 8;
    // single-factor items carry a row tile index in place of the block count (small blocks: one
    // item each, in the order of the direct single-vector path)
    if (direct_singles<P>() && kind == kF32Single)
        apply_multi<P, float, 8>(r, z, nlat, nr, f32, patches, bt.x, 1, g, rule, smem);
    else if (direct_singles<P>() && kind == kF64Single)
        apply_multi<P, double, 8>(r, z, nlat, nr, f64, patches, bt.x, 1, g, rule, smem);
    else if (kind == kF32Single)
        apply_multi_rows<P, float>(r, z, nlat, nr, f32, patches, bt.x, count * rows32, rows32, g, rule, smem);
    else if (kind == kF64Single && P < 4)
        apply_multi_rows<P, double>(r, z, nlat, nr, f64, patches, bt.x, count * rows64, rows64, g, rule, smem);
    else if (kind == kF32Shared)
        apply_multi<P, float, 8>(r, z, nlat, nr, f32, patches, bt.x, count, g, rule, smem);
    else if (P < 4)
        apply_multi<P, double, 8>(r, z, nlat, nr, f64, patches, bt.x, count, g, rule, smem);
}

// One colour of the Schwarz apply (Sec. 3.1 Eq. (5)): each CTA takes one work item (a
// shared-factor batch, or a row tile of a block with its own factor; FP32 or FP64 factor).
// The blocks of one colour are DOF-disjoint, so the scatter needs no atomics.  Dynamic shared
// memory: schwarz_smem_bytes(P, rows32, rows64).
template <int P>
__global__ void __launch_bounds__(threads_for(3 * box_width(P) * box_width(P) * box_width(P)), P == 3 ? 3 : 1)
    schwarz_colour_kernel(const double *__restrict__ r, double *__restrict__ z, const double *__restrict__ f64,
                          const float *__restrict__ f32, const PatchRec *__restrict__ patches,
                          const int2 *__restrict__ batches, Grid3 g, int rule, int rows32, int rows64, int *err,
                          const int *__restrict__ done)
{
    constexpr int GD = (P == 4 ? 4 : 8);
    extern __shared__ __align__(128) unsigned char smem[];
    if (done && *done) return;
    const int2 bt = batches[blockIdx.x];
    const int count = bt.y & 255, kind = bt.y >> 8;
    switch (kind) {
    case kF32Shared: apply_batch<P, f32_batch_cap<P>(), float, 16>(r, z, f32, patches, bt.x, count, g, rule, smem); break;
    case kF64Shared: apply_batch<P, GD, double, 4>(r, z, f64, patches, bt.x, count, g, rule, smem); break;
    // single-factor items carry a row tile index in place of the block count; small blocks (p <= 2)
    // are one item each, applied with direct loads (no staging pays off for them)
    case kF32Single:
        if (direct_singles<P>()) apply_batch<P, 1, float, 16>(r, z, f32, patches, bt.x, 1, g, rule, smem);
        else apply_rows<P, float>(r, z, f32, patches, bt.x, count * rows32, rows32, g, rule, smem, err);
        break;
    default:
        if (direct_singles<P>()) apply_batch<P, 1, double, 16>(r, z, f64, patches, bt.x, 1, g, rule, smem);
        else apply_rows<P, double>(r, z, f64, patches, bt.x, count * rows64, rows64, g, rule, smem, err);
        break;
    }
}

// One colour of the Schwarz apply as a persistent launch: CTA b takes work items b, b + G,
// b + 2G, ... (G = gridDim.x) and pipelines the row tiles of cut blocks through two shared-memory
// stages: while it works on item i, the bulk copies of its next row tile (item i + G) are already
// in flight, so the gather, compute and scatter phases of one tile overlap the DRAM transfer of
// the next and the CTAs of a launch do not fall into step.  Shared-factor batches use a separate
// area.  Each stage's mbarrier flips phase on every use.  The arithmetic is tile_apply /
// apply_batch, so S r is bit-identical to schwarz_colour_kernel's.  Dynamic shared memory:
// rows_tile_offset + 2 tile_bytes + the batch area (schwarz_persistent_smem_bytes).
template <int P>
__global__ void __launch_bounds__(threads_for(3 * box_width(P) * box_width(P) * box_width(P)), P == 3 ? 3 : 1)
    schwarz_persistent_kernel(const double *__restrict__ r, double *__restrict__ z, const double *__restrict__ f64,
                              const float *__restrict__ f32, const PatchRec *__restrict__ patches,
                              const int2 *__restrict__ items, int nitems, Grid3 g, int rule, int rows32, int rows64,
                              int tile_bytes, int *err, const int *__restrict__ done)
{
    constexpr int GD = (P == 4 ? 4 : 8);
    extern __shared__ __align__(128) unsigned char smem[];
    if (done && *done) return;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // bar[0], bar[1]
    unsigned char *rb = smem + 16;
    unsigned char *tiles = smem + rows_tile_offset<P>();
    unsigned char *area = tiles + 2 * (size_t)tile_bytes;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
    }
    __syncthreads();
    auto single = [&](int i) {
        const int k = items[i].y >> 8;
        return !direct_singles<P>() && (k == kF32Single || k == kF64Single);
    };
    int issued = 0, used = 0;
    unsigned phase = 0u;  // bit s: parity of the next completion of stage s
    auto issue = [&](int i) {
        if (threadIdx.x == 0) {
            const int2 it = items[i];
            const int kind = it.y >> 8, tile = it.y & 255;
            unsigned char *dst = tiles + (size_t)(issued & 1) * tile_bytes;
            uint64_t *b = &bar[issued & 1];
            const PatchRec pr = patches[it.x];
            // the stage was last read through the generic proxy; order those reads before the copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (kind == kF32Single)
                tile_issue<P, float>(f32, pr, tile * rows32, tile_geom<P, float>(pr, tile * rows32, rows32, g, rule), dst, b);
            else
                tile_issue<P, double>(f64, pr, tile * rows64, tile_geom<P, double>(pr, tile * rows64, rows64, g, rule), dst, b);
        }
        ++issued;
    };
    int i = blockIdx.x;
    if (i < nitems && single(i)) issue(i);
    for (; i < nitems; i += gridDim.x) {
        // a CTA that gave up on a copy has flagged the apply as failed: stop early
        if (__syncthreads_or(*reinterpret_cast<volatile int *>(err) != 0)) {
            if (threadIdx.x == 0 && issued > used) mbar_wait(&bar[used & 1], (phase >> (used & 1)) & 1u);
            __syncthreads();
            return;
        }
        const int nx = i + gridDim.x;
        if (nx < nitems && single(nx)) issue(nx);
        const int2 it = items[i];
        const int kind = it.y >> 8, count = it.y & 255;
        if (kind == kF32Shared) {
            apply_batch<P, f32_batch_cap<P>(), float, 16>(r, z, f32, patches, it.x, count, g, rule, area);
        } else if (kind == kF64Shared) {
            apply_batch<P, GD, double, 4>(r, z, f64, patches, it.x, count, g, rule, area);
        } else if (direct_singles<P>() && kind == kF32Single) {
            apply_batch<P, 1, float, 16>(r, z, f32, patches, it.x, 1, g, rule, area);
        } else if (direct_singles<P>()) {
            apply_batch<P, 1, double, 16>(r, z, f64, patches, it.x, 1, g, rule, area);
        } else {
            const int s = used & 1;
            ++used;
            const PatchRec pr = patches[it.x];
            const bool f = kind == kF32Single;
            const int rows = f ? rows32 : rows64, row0 = count * rows;
            const TileGeom tg = f ? tile_geom<P, float>(pr, row0, rows, g, rule) : tile_geom<P, double>(pr, row0, rows, g, rule);
            if (f)
                tile_gather<float>(r, tg, g, reinterpret_cast<float *>(rb));
            else
                tile_gather<double>(r, tg, g, reinterpret_cast<double *>(rb));
            __syncthreads();
            const bool ok = __syncthreads_and(mbar_wait(&bar[s], (phase >> s) & 1u));
            phase ^= 1u << s;
            if (!ok) {
                if (threadIdx.x == 0) {
                    atomicExch(err, 1);
                    mbar_wait(&bar[s], (phase >> s) & 1u ^ 1u);  // the copies still in flight land first
                    if (issued > used) mbar_wait(&bar[s ^ 1], (phase >> (s ^ 1)) & 1u);
                }
                __syncthreads();
                return;
            }
            if (f)
                tile_apply<P, float>(z, tg, g, row0, reinterpret_cast<const float *>(rb),
                                     reinterpret_cast<const float *>(tiles + (size_t)s * tile_bytes));
            else
                tile_apply<P, double>(z, tg, g, row0, reinterpret_cast<const double *>(rb),
                                      reinterpret_cast<const double *>(tiles + (size_t)s * tile_bytes));
        }
        __syncthreads();  // the item's shared memory is free again
    }
}

// Start of z = S r for nr vectors nlat apart: z = D r with D = 1 / K_ll for the DOFs in no
// block (Algorithm 1's diagonal part) and 0 elsewhere, or z = 0 when the blocks cover every
// free DOF (jac == nullptr).
__global__ void schwarz_init_kernel(const double *__restrict__ r, double *__restrict__ z,
                                    const double *__restrict__ jac, int64_t nlat, int64_t n,
                                    const int *__restrict__ done)
{
    if (done && *done) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = jac ? jac[i % nlat] * r[i] : 0.0;
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
    const int threads = schwarz_threads(P, plan.rule);
    for (int i = 0; i < plan.nseg; ++i) {
        const SchwarzSeg &sg = plan.seg[i];
        if (sg.count > 0 && plan.persistent)
            schwarz_persistent_kernel<P><<<std::min(sg.count, plan.grid_cap), threads, plan.smem, s>>>(
                r, z, f64, f32, plan.patches, plan.batches + sg.first, sg.count, g, plan.rule, plan.rows, plan.rows64,
                plan.tile_bytes, plan.err, done);
        else if (sg.count > 0)
            schwarz_colour_kernel<P><<<sg.count, threads, plan.smem, s>>>(
                r, z, f64, f32, plan.patches, plan.batches + sg.first, g, plan.rule, plan.rows, plan.rows64, plan.err, done);
    }
}

template <int P>
void schwarz_multi_launch(const Grid3 &g, const double *r, double *z, int64_t nlat, int nr, const double *f64,
                          const float *f32, const SchwarzPlan &plan, const int *done, cudaStream_t s)
{
    const int threads = schwarz_threads(P, plan.rule);
    for (int i = 0; i < plan.nseg; ++i) {
        const SchwarzSeg &sg = plan.seg[i];
        if (sg.count > 0)
            schwarz_multi_kernel<P><<<sg.count, threads, 0, s>>>(r, z, nlat, nr, f64, f32, plan.patches,
                                                                 plan.batches + sg.first, g, plan.rule, plan.rows, plan.rows64, done);
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

namespace {

// Batches: rbT, then the block bases and box offsets; row tiles: mbarrier, r_B, the tile.
template <int P>
int smem_bytes_p(int rows32, int rows64)
{
    constexpr int W = box_width(P), NB = 3 * W * W * W, GD = (P == 4 ? 4 : 8), ROW = (GD * 8 > 32 ? GD * 8 : 32);
    // rbT, the block bases (16-byte aligned) and the box offsets, for the largest batch of either precision
    const int batch = std::max(NB * ROW + 16 + 64 + 4 * NB, NB * f32_batch_cap<P>() * 4 + 16 + 8 * f32_batch_cap<P>() + 4 * NB);
    static_assert(f32_batch_cap<P>() <= 16, "the batch's block bases take 8 bytes each after rbT");
    if (direct_singles<P>()) return batch;  // no row tiles
    const int t32 = rows_tile_offset<P>() + rows32 * factor_ld<float>(NB) * 4;
    const int t64 = rows_tile_offset<P>() + rows64 * factor_ld<double>(NB) * 8;
    return std::max(batch, std::max(t32, t64));
}

template <int P>
cudaError_t prepare_p(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(schwarz_colour_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(schwarz_colour_kernel<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

}  // namespace

void schwarz_default_rows(int p, int rule, int *rows32, int *rows64)
{
    // 4 (FP32) or 2 (FP64) rows per warp of the launch, as long as a tile stays within kTileBudget bytes
    const int nb = 3 * box_width(p) * box_width(p) * box_width(p);
    const int nw = schwarz_threads(p, rule) / 32;
    const int cap32 = kTileBudget / (factor_ld<float>(nb) * 4), cap64 = kTileBudget / (factor_ld<double>(nb) * 8);
    *rows32 = std::max(4, std::min(4 * nw, cap32) / 4 * 4);
    *rows64 = std::max(2, std::min(2 * nw, cap64) / 2 * 2);
}

int schwarz_smem_bytes(int p, int rows32, int rows64)
{
    switch (p) {
    case 1: return smem_bytes_p<1>(rows32, rows64);
    case 2: return smem_bytes_p<2>(rows32, rows64);
    case 3: return smem_bytes_p<3>(rows32, rows64);
    default: return smem_bytes_p<4>(rows32, rows64);
    }
}

namespace {

template <int P>
int persistent_smem_p(int rows32, int rows64, int *tile_bytes)
{
    constexpr int W = box_width(P), NB = 3 * W * W * W, GD = (P == 4 ? 4 : 8), ROW = (GD * 8 > 32 ? GD * 8 : 32);
    const int tb = direct_singles<P>() ? 0
                                       : (std::max(rows32 * factor_ld<float>(NB) * 4, rows64 * factor_ld<double>(NB) * 8) + 15) / 16 * 16;
    *tile_bytes = tb;
    return rows_tile_offset<P>() + 2 * tb + NB * ROW + 16 + 64 + 4 * NB;
}

template <int P>
cudaError_t persistent_grid_p(int threads, int smem, int *grid)
{
    cudaError_t e = cudaFuncSetAttribute(schwarz_persistent_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(schwarz_persistent_kernel<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, schwarz_persistent_kernel<P>, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *grid = std::max(1, per_sm) * std::max(1, sms);
    return e;
}

}  // namespace

int schwarz_persistent_smem_bytes(int p, int rows32, int rows64, int *tile_bytes)
{
    switch (p) {
    case 1: return persistent_smem_p<1>(rows32, rows64, tile_bytes);
    case 2: return persistent_smem_p<2>(rows32, rows64, tile_bytes);
    case 3: return persistent_smem_p<3>(rows32, rows64, tile_bytes);
    default: return persistent_smem_p<4>(rows32, rows64, tile_bytes);
    }
}

cudaError_t schwarz_persistent_grid(int p, int rule, int smem, int *grid)
{
    const int threads = schwarz_threads(p, rule);
    switch (p) {
    case 1: return persistent_grid_p<1>(threads, smem, grid);
    case 2: return persistent_grid_p<2>(threads, smem, grid);
    case 3: return persistent_grid_p<3>(threads, smem, grid);
    default: return persistent_grid_p<4>(threads, smem, grid);
    }
}

bool schwarz_direct_singles(int p) { return p <= 2 ? direct_singles<2>() : direct_singles<3>(); }

int schwarz_f32_batch_cap(int p) { return p == 4 ? f32_batch_cap<4>() : f32_batch_cap<3>(); }

cudaError_t schwarz_prepare(int p, int smem_bytes)
{
    switch (p) {
    case 1: return prepare_p<1>(smem_bytes);
    case 2: return prepare_p<2>(smem_bytes);
    case 3: return prepare_p<3>(smem_bytes);
    default: return prepare_p<4>(smem_bytes);
    }
}

void launch_schwarz_apply(int p, const Grid3 &g, const double *r, double *z, const double *f64, const float *f32,
                          const SchwarzPlan &plan, const int *done, cudaStream_t s)
{
    const int64_t nlat = 3 * (int64_t)g.M[0] * g.M[1] * g.M[2];
    schwarz_init_kernel<<<grid_for(nlat, 256), 256, 0, s>>>(r, z, plan.jac, nlat, nlat, done);
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
    schwarz_init_kernel<<<grid_for(nlat * nr, 256), 256, 0, s>>>(r, z, plan.jac, nlat, nlat * nr, done);
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
