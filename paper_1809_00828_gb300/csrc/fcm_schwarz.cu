// Additive-Schwarz apply z = D r + sum_B R_B^T F_B R_B r on sm_103a (Sec. 3.1 Eq. (5), Algorithm 1;
// F_B the eigenvalue-filtered pseudo inverse of Sec. 3.2 Eqs. (11)-(13), D Algorithm 1's diagonal
// scaling of the DOFs in no block).
//
// Two phases, so that no block waits for another:
//   1. block products Zb[B] = F_B r_B for every block at once, each written to its own slot of a
//      buffer (no scatter, no colours):
//        - blocks with their own factor (cut blocks) stream the factor from HBM once; a work item is
//          a tile of rows of one block (schwarz_rows_kernel: a warp per row, the lanes split the row
//          into 16-byte vectors; schwarz_cols_kernel: a thread per row, for small blocks and for
//          several right-hand sides);
//        - blocks that share a factor (uncut patches with equal boundary patterns) form a dense
//          product F [r_B1 ... r_Bm]: schwarz_gemm_kernel stages the factor through shared memory
//          by bulk copies (cp.async.bulk, completed on mbarriers, double-buffered) and keeps an
//          8 x 8 register tile of outputs per thread, so one shared-memory read of a factor entry
//          feeds 8 multiply-adds;
//   2. schwarz_sum_kernel: z_l = D_l r_l + the Zb rows of the blocks that contain DOF l, summed in
//      a fixed order of the blocks: deterministic, and every launch shape gives the same bits.
//
// Factor storage per block: FP64; FP32; or "double-float" (each FP64 entry f stored as the float
// pair hi = fl32(f), lo = fl32(f - hi), relative error 2^-48) for the ill-conditioned blocks of
// the mixed form.  Double-float products run on the FP32 pipe with error-free transformations
// (Dekker's product by FMA, Knuth's TwoSum; Ogita, Rump & Oishi's compensated dot product), which
// GB300's FP64 pipe (2 fused multiply-adds per clock per SM) could not do at HBM rate.
#include <cuda_runtime.h>

#include <algorithm>

#include "fcm_device.cuh"
#include "fcm_ff.cuh"

namespace fcm {

namespace {

__host__ __device__ constexpr int sbox_width(int P) { return 2 * P - 1 > P + 1 ? 2 * P - 1 : P + 1; }
// rows of the largest block box of either rule
__host__ __device__ constexpr int sbox_max(int P) { return 3 * sbox_width(P) * sbox_width(P) * sbox_width(P); }
__host__ __device__ constexpr int rnd32(int v) { return (v + 31) / 32 * 32; }

struct SBox {
    int lo[3], d[3], n;
};

// Lattice box of block `id`: rule 0, the vertex patch of vertex id, [p v - (p-1), p v + (p-1)] clipped to
// the lattice; rule 3, the element block of cell id, [p c, p c + p].
__device__ __forceinline__ SBox sbox(int rule, int P, const Grid3 &g, int id)
{
    SBox b;
    if (rule == 3) {
        const int c[3] = {id % g.n[0], (id / g.n[0]) % g.n[1], id / (g.n[0] * g.n[1])};
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = P * c[a];
            b.d[a] = P + 1;
        }
    } else {
        const int nvx = g.n[0] + 1, nvy = g.n[1] + 1;
        const int v[3] = {id % nvx, (id / nvx) % nvy, id / (nvx * nvy)};
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = max(0, P * v[a] - (P - 1));
            b.d[a] = min(g.M[a] - 1, P * v[a] + (P - 1)) - b.lo[a] + 1;
        }
    }
    b.n = 3 * b.d[0] * b.d[1] * b.d[2];
    return b;
}

// offset of box entry t from the box's first lattice DOF
__device__ __forceinline__ int box_rel(const SBox &b, const Grid3 &g, int t)
{
    const int nl = t / 3;
    const int ix = nl % b.d[0], iy = (nl / b.d[0]) % b.d[1], iz = nl / (b.d[0] * b.d[1]);
    return 3 * (ix + g.M[0] * (iy + g.M[1] * iz)) + t % 3;
}

__device__ __forceinline__ int64_t box_base(const SBox &b, const Grid3 &g)
{
    return 3 * (b.lo[0] + (int64_t)g.M[0] * (b.lo[1] + (int64_t)g.M[1] * b.lo[2]));
}

// Block products Zb: nslots * zs entries of 8 bytes per right-hand side, slot by slot.  With `pairs`
// (the mixed forms) a slot of an FP32 factor holds its rows as floats (the first half of the slot's
// bytes), any other slot as float pairs (hi, lo) whose sum is the value: double-float results (S, C),
// FP64 results split by split_bits<23>; the sum kernel adds them on the FP32 pipe.  Otherwise (FP64
// form) a slot holds FP64 values.  `zslot` points at the slot's first entry.
__device__ __forceinline__ void put_f32(double *zslot, int row, float v, bool pairs)
{
    if (pairs) reinterpret_cast<float *>(zslot)[row] = v;
    else zslot[row] = f2d(v);
}
__device__ __forceinline__ void put_ff(double *zslot, int row, float s, float c, bool pairs)
{
    if (pairs) reinterpret_cast<float2 *>(zslot)[row] = make_float2(s, c);
    else zslot[row] = f2d(s) + f2d(c);
}
__device__ __forceinline__ void put_f64(double *zslot, int row, double v, bool pairs)
{
    if (pairs) {
        float h, l;
        split_bits<23>(v, h, l);
        reinterpret_cast<float2 *>(zslot)[row] = make_float2(h, l);
    } else {
        zslot[row] = v;
    }
}
__device__ __forceinline__ void put_val(double *zslot, int row, float v, bool pairs) { put_f32(zslot, row, v, pairs); }
__device__ __forceinline__ void put_val(double *zslot, int row, double v, bool pairs) { put_f64(zslot, row, v, pairs); }

// slot_of entries of FP32 slots in the pair format carry this flag
constexpr int kSlotF32 = 1 << 30;

// 16-byte vectors of float (4) or double (2)
template <typename T> struct V16;
template <> struct V16<float> {
    using type = float4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float dot(float4 a, float4 b, float c)
    {
        return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, c))));
    }
};
template <> struct V16<double> {
    using type = double2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double dot(double2 a, double2 b, double c) { return fma(a.y, b.y, fma(a.x, b.x, c)); }
};

// ---- phase 1a: own factors, a warp per row (blocks of p = 3, one right-hand side)

constexpr int kRowsThreads = 256;

// rows [row0, row0 + rows) of Zb = F r_B, F in T (FP32 or FP64), rows of ld entries padded to 16 bytes
template <int P, typename T>
__device__ __forceinline__ void rows_plain(const double *__restrict__ r, const T *__restrict__ F, const SBox &b,
                                           const Grid3 &g, int row0, int rows, double *__restrict__ zout,
                                           bool pairs, unsigned char *smem)
{
    using VT = typename V16<T>::type;
    constexpr int V = 16 / (int)sizeof(T);
    constexpr int KV = (factor_ld<T>(sbox_max(P)) / V + 31) / 32;  // 16-byte vectors per lane and row
    constexpr int RPW = sizeof(T) == 8 ? 2 : 4;                     // rows per warp and pass
    T *rb = reinterpret_cast<T *>(smem);
    const int n = b.n, ld = factor_ld<T>(n), nv = ld / V;
    const int64_t base = box_base(b, g);
    for (int t = threadIdx.x; t < ld; t += blockDim.x) rb[t] = t < n ? gathered<T>(r[base + box_rel(b, g, t)]) : (T)0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    VT xr[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) xr[k] = lane + 32 * k < nv ? reinterpret_cast<const VT *>(rb)[lane + 32 * k] : V16<T>::zero();
    const int row1 = min(n, row0 + rows);
    for (int t = row0 + RPW * w; t < row1; t += RPW * nw) {
        VT fv[RPW][KV];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            // rows past row1 repeat the last row (in bounds) and are not written
            const VT *fr = reinterpret_cast<const VT *>(F + (size_t)min(t + q, row1 - 1) * ld);
#pragma unroll
            for (int k = 0; k < KV; ++k) fv[q][k] = lane + 32 * k < nv ? __ldcs(fr + lane + 32 * k) : V16<T>::zero();
        }
        T a[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            a[q] = (T)0;
#pragma unroll
            for (int k = 0; k < KV; ++k) a[q] = V16<T>::dot(fv[q][k], xr[k], a[q]);
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
            put_val(zout, t + lane, v, pairs);
        }
    }
}

// the same for a double-float factor: entry j of a row is the float pair at 2j, 2j+1
template <int P>
__device__ __forceinline__ void rows_ff(const double *__restrict__ r, const float *__restrict__ F, const SBox &b,
                                        const Grid3 &g, int row0, int rows, double *__restrict__ zout, bool pairs,
                                        unsigned char *smem)
{
    constexpr int KV = (factor_ld<double>(sbox_max(P)) / 2 + 31) / 32;  // float4 = two entries
    constexpr int RPW = 2;
    float2 *rb = reinterpret_cast<float2 *>(smem);
    const int n = b.n, ld = factor_ld<double>(n), nv = ld / 2;
    const int64_t base = box_base(b, g);
    for (int t = threadIdx.x; t < ld; t += blockDim.x)
        rb[t] = t < n ? split_ff(r[base + box_rel(b, g, t)]) : make_float2(0.f, 0.f);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float4 xr[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k)
        xr[k] = lane + 32 * k < nv ? reinterpret_cast<const float4 *>(rb)[lane + 32 * k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int row1 = min(n, row0 + rows);
    for (int t = row0 + RPW * w; t < row1; t += RPW * nw) {
        float4 fv[RPW][KV];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const float4 *fr = reinterpret_cast<const float4 *>(F + (size_t)min(t + q, row1 - 1) * 2 * ld);
#pragma unroll
            for (int k = 0; k < KV; ++k)
                fv[q][k] = lane + 32 * k < nv ? __ldcs(fr + lane + 32 * k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float S[RPW], C[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            S[q] = 0.f;
            C[q] = 0.f;
#pragma unroll
            for (int k = 0; k < KV; ++k) {
                ff_fma(fv[q][k].x, fv[q][k].y, xr[k].x, xr[k].y, S[q], C[q]);
                ff_fma(fv[q][k].z, fv[q][k].w, xr[k].z, xr[k].w, S[q], C[q]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const float s2 = __shfl_xor_sync(0xffffffffu, S[q], o), c2 = __shfl_xor_sync(0xffffffffu, C[q], o);
                ff_add(S[q], C[q], s2, c2);
            }
        if (lane < RPW && t + lane < row1) {
            float s = S[0], c = C[0];
#pragma unroll
            for (int q = 1; q < RPW; ++q)
                if (lane == q) {
                    s = S[q];
                    c = C[q];
                }
            put_ff(zout, t + lane, s, c, pairs);
        }
    }
}

// One work item per CTA: (slot, first row) of a block with its own factor; the slot's record
// gives the factor's offset and storage (0 FP64, 1 FP32, 2 double-float).
template <int P>
__global__ void __launch_bounds__(kRowsThreads)
    schwarz_rows_kernel(const double *__restrict__ r, const double *__restrict__ f64, const float *__restrict__ f32,
                        const PatchRec *__restrict__ slots, const int2 *__restrict__ items, int rows, Grid3 g, int rule,
                        double *__restrict__ zb, int zs, int pairs, const int *__restrict__ done)
{
    __shared__ __align__(16) double smem_d[factor_ld<double>(sbox_max(P))];
    if (done && *done) return;
    unsigned char *smem = reinterpret_cast<unsigned char *>(smem_d);
    const int2 it = items[blockIdx.x];
    const PatchRec pr = slots[it.x];
    const SBox b = sbox(rule, P, g, pr.v);
    double *zout = zb + (size_t)it.x * zs;
    if (pr.prec == 1) rows_plain<P, float>(r, f32 + pr.off, b, g, it.y, rows, zout, pairs, smem);
    else if (pr.prec == 2) rows_ff<P>(r, f32 + pr.off, b, g, it.y, rows, zout, pairs, smem);
    else rows_plain<P, double>(r, f64 + pr.off, b, g, it.y, rows, zout, pairs, smem);
}

// ---- phase 1b: own factors, a thread per row (small blocks; several right-hand sides)
//
// Thread t of the item owns row row0 + t and walks the columns j: F[j][row] = F[row][j] (F is
// symmetric) is read coalesced across the threads, and the NR residual entries r_k,B[j] are one
// broadcast shared-memory read for the whole CTA.  nr <= NR right-hand sides are nlat apart in r, and
// zsize apart in Zb.

__host__ __device__ constexpr int cols_threads(int P) { return P >= 3 ? 128 : rnd32(sbox_max(P)); }

template <int P, int NR, typename T>
__device__ __forceinline__ void cols_plain(const double *__restrict__ r, int64_t nlat, int nr, const T *__restrict__ F,
                                           const SBox &b, const Grid3 &g, int row0, double *__restrict__ zout,
                                           int64_t zsize, bool pairs, unsigned char *smem)
{
    T(*rbT)[NR] = reinterpret_cast<T(*)[NR]>(smem);
    const int n = b.n, ld = factor_ld<T>(n);
    const int64_t base = box_base(b, g);
    for (int e = threadIdx.x; e < n * NR; e += blockDim.x) {
        const int t = e / NR, k = e % NR;
        rbT[t][k] = k < nr ? gathered<T>(r[(int64_t)k * nlat + base + box_rel(b, g, t)]) : (T)0;
    }
    __syncthreads();
    const int row = row0 + threadIdx.x;
    if (row >= n) return;
    T acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = (T)0;
    const T *__restrict__ col = F + row;
#pragma unroll 8
    for (int j = 0; j < n; ++j) {
        const T f = __ldcs(col + (size_t)j * ld);
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = fma(f, rbT[j][k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k)
        if (k < nr) put_val(zout + (int64_t)k * zsize, row, acc[k], pairs);
}

template <int P, int NR>
__device__ __forceinline__ void cols_ff(const double *__restrict__ r, int64_t nlat, int nr, const float *__restrict__ F,
                                        const SBox &b, const Grid3 &g, int row0, double *__restrict__ zout, int64_t zsize,
                                        bool pairs, unsigned char *smem)
{
    float2(*rbT)[NR] = reinterpret_cast<float2(*)[NR]>(smem);
    const int n = b.n, ld = factor_ld<double>(n);
    const int64_t base = box_base(b, g);
    for (int e = threadIdx.x; e < n * NR; e += blockDim.x) {
        const int t = e / NR, k = e % NR;
        rbT[t][k] = k < nr ? split_ff(r[(int64_t)k * nlat + base + box_rel(b, g, t)]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int row = row0 + threadIdx.x;
    if (row >= n) return;
    float S[NR], C[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) S[k] = C[k] = 0.f;
    const float2 *__restrict__ col = reinterpret_cast<const float2 *>(F) + row;
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
        const float2 f = __ldcs(col + (size_t)j * ld);
#pragma unroll
        for (int k = 0; k < NR; ++k)
            if (k < nr) ff_fma(f.x, f.y, rbT[j][k].x, rbT[j][k].y, S[k], C[k]);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k)
        if (k < nr) put_ff(zout + (int64_t)k * zsize, row, S[k], C[k], pairs);
}

template <int P, int NR>
__global__ void __launch_bounds__(cols_threads(P))
    schwarz_cols_kernel(const double *__restrict__ r, int64_t nlat, int nr, const double *__restrict__ f64,
                        const float *__restrict__ f32, const PatchRec *__restrict__ slots,
                        const int2 *__restrict__ items, Grid3 g, int rule, double *__restrict__ zb, int zs,
                        int64_t zsize, int pairs, const int *__restrict__ done)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    if (done && *done) return;
    const int2 it = items[blockIdx.x];
    const PatchRec pr = slots[it.x];
    const SBox b = sbox(rule, P, g, pr.v);
    double *zout = zb + (size_t)it.x * zs;
    if (pr.prec == 1) cols_plain<P, NR, float>(r, nlat, nr, f32 + pr.off, b, g, it.y, zout, zsize, pairs, smem);
    else if (pr.prec == 2) cols_ff<P, NR>(r, nlat, nr, f32 + pr.off, b, g, it.y, zout, zsize, pairs, smem);
    else cols_plain<P, NR, double>(r, nlat, nr, f64 + pr.off, b, g, it.y, zout, zsize, pairs, smem);
}

// ---- phase 1c: blocks sharing a factor, Zb[B_1 .. B_m] = F [r_B1 .. r_Bm] (m = count of the tile)
//
// Columns of the tile are (block, right-hand side) pairs, NC per group; the residual panel R[k][col]
// (the gathered r_B, converted to T) sits in shared memory for the whole group.  The factor streams
// through two shared-memory stages of KC rows: F[k0 .. k0 + KC)[0 .. ld) is one contiguous bulk copy
// (F is symmetric, so these rows are the columns k0 .. k0 + KC of the product).  Thread (rg, cg)
// accumulates rows 8 rg .. 8 rg + 7 for 8 columns (NC/8): two 16-byte reads of the stage and two of
// the panel feed 64 multiply-adds.  Blocks with more rows than 8 x (threads / 8) take several passes
// over the factor.

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// dst, src and bytes multiples of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier, giving up (false) after `tries` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int tries)
{
    for (int i = 0; i < tries; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Polls of the wait that lets copies still in flight land before a CTA that gave up leaves.
constexpr int kDrainTries = 1 << 22;

// m consecutive values from shared memory at a pointer aligned to min(16, m sizeof(T)) bytes, in
// 16-byte (or 8-byte) vector reads
template <typename T, int m>
__device__ __forceinline__ void load_vec(const T *p, T *out)
{
    if constexpr (sizeof(T) * m % 16 == 0) {
        using VT = typename V16<T>::type;
        constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
        for (int i = 0; i < m / V; ++i) {
            const VT v = reinterpret_cast<const VT *>(p)[i];
            if constexpr (V == 4) {
                out[4 * i] = v.x;
                out[4 * i + 1] = v.y;
                out[4 * i + 2] = v.z;
                out[4 * i + 3] = v.w;
            } else {
                out[2 * i] = v.x;
                out[2 * i + 1] = v.y;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < m; ++i) out[i] = p[i];
    }
}

__host__ __device__ constexpr int gemm_threads(int P)
{
    return 8 * ((sbox_max(P) + 7) / 8) < 512 ? rnd32(8 * ((sbox_max(P) + 7) / 8)) : 512;
}
template <typename T, int P> struct GemmCfg {
    static constexpr int NC = sizeof(T) == 4 ? (P == 4 ? 32 : 64) : (P == 4 ? 16 : 32);  // columns per group
    static constexpr int KC = (sizeof(T) == 4 ? 16 : 8) / (P == 4 ? 2 : 1);            // factor rows per stage
};

// shared memory: 2 mbarriers | column sources and destinations | box offsets | panel | 2 stages
template <int P, typename T>
__host__ __device__ constexpr int gemm_stage_elems()
{
    return (GemmCfg<T, P>::KC * factor_ld<T>(sbox_max(P)) + 8 + 15) / 16 * 16;
}
template <int P, typename T>
__host__ __device__ constexpr int gemm_panel_off()
{
    return (16 + 16 * GemmCfg<T, P>::NC + 4 * sbox_max(P) + 127) / 128 * 128;
}
template <int P, typename T>
__host__ __device__ constexpr int gemm_smem_bytes()
{
    return gemm_panel_off<P, T>() + (int)sizeof(T) * (sbox_max(P) * GemmCfg<T, P>::NC + 2 * gemm_stage_elems<P, T>());
}

template <int P, typename T>
__global__ void __launch_bounds__(gemm_threads(P))
    schwarz_gemm_kernel(const double *__restrict__ r, int64_t nlat, int nr, const T *__restrict__ pool,
                        const PatchRec *__restrict__ slots, const int2 *__restrict__ tiles, Grid3 g, int rule,
                        double *__restrict__ zb, int zs, int64_t zsize, int pairs, int *err, int wait_tries,
                        const int *__restrict__ done)
{
    constexpr int NC = GemmCfg<T, P>::NC, KC = GemmCfg<T, P>::KC, CPT = NC / 8, HALF = CPT / 2;
    constexpr int SE = gemm_stage_elems<P, T>();
    extern __shared__ __align__(1024) unsigned char smem[];
    if (done && *done) return;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int64_t *src = reinterpret_cast<int64_t *>(smem + 16);   // NC: first lattice DOF of the column's r_B, -1 none
    int64_t *dst = src + NC;                                  // NC: the column's Zb row 0, -1 none
    int *rel = reinterpret_cast<int *>(smem + 16 + 16 * NC);  // box offsets
    T *panel = reinterpret_cast<T *>(smem + gemm_panel_off<P, T>());
    T *stage = panel + sbox_max(P) * NC;
    const int2 tl = tiles[blockIdx.x];
    const int first = tl.x, count = tl.y;
    const PatchRec p0 = slots[first];
    const SBox b0 = sbox(rule, P, g, p0.v);
    const int n = b0.n, ld = factor_ld<T>(n);
    const T *F = pool + p0.off;
    const int tid = threadIdx.x, rg = tid >> 3, cg = tid & 7, nrg = blockDim.x >> 3;
    const int per_group = NC / nr;                               // blocks per column group
    const int groups = (count + per_group - 1) / per_group;
    const int passes = (n + 8 * nrg - 1) / (8 * nrg);
    const int nch = (n + KC - 1) / KC;
    const int Q = groups * passes * nch;                         // factor chunks streamed by this CTA
    for (int t = tid; t < n; t += blockDim.x) rel[t] = box_rel(b0, g, t);
    if (tid == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
    }
    __syncthreads();
    auto issue = [&](int q) {  // thread 0: chunk q into stage q & 1
        const int c = q % nch, k0 = c * KC, kc = min(KC, n - k0);
        const uint32_t bytes = (uint32_t)(kc * ld * (int)sizeof(T));
        unsigned char *d = reinterpret_cast<unsigned char *>(stage + (size_t)(q & 1) * SE);
        const unsigned char *s = reinterpret_cast<const unsigned char *>(F + (size_t)k0 * ld);
        // the stage was last read through the generic proxy: order those reads before the copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect(&bar[q & 1], bytes);
        for (uint32_t o = 0; o < bytes; o += 16384u) bulk_g2s(d + o, s + o, min(16384u, bytes - o), &bar[q & 1]);
    };
    if (tid == 0) {
        issue(0);
        if (Q > 1) issue(1);
    }
    int q = 0;
    for (int grp = 0; grp < groups; ++grp) {
        // columns of this group and their gathered residuals
        for (int c = tid; c < NC; c += blockDim.x) {
            const int pj = grp * per_group + c / nr, k = c % nr;
            int64_t s = -1, d = -1;
            if (c < per_group * nr && pj < count) {
                const PatchRec pr = slots[first + pj];
                s = (int64_t)k * nlat + box_base(sbox(rule, P, g, pr.v), g);
                d = (int64_t)k * zsize + (int64_t)(first + pj) * zs;
            }
            src[c] = s;
            dst[c] = d;
        }
        __syncthreads();
        for (int e = tid; e < n * NC; e += blockDim.x) {
            const int t = e / NC, c = e % NC;
            const int64_t s = src[c];
            panel[e] = s >= 0 ? gathered<T>(r[s + rel[t]]) : (T)0;
        }
        __syncthreads();
        for (int pass = 0; pass < passes; ++pass) {
            const int row0 = pass * 8 * nrg + 8 * rg;
            T acc[8][CPT];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < CPT; ++j) acc[i][j] = (T)0;
            for (int c = 0; c < nch; ++c, ++q) {
                const int s = q & 1;
                const bool ok = __syncthreads_and(mbar_wait(&bar[s], (q >> 1) & 1, wait_tries));
                if (!ok) {
                    // flag the apply as failed; the copies still in flight land before the CTA leaves
                    if (tid == 0) {
                        atomicExch(err, 1);
                        mbar_wait(&bar[s], (q >> 1) & 1, kDrainTries);
                        if (q + 1 < Q) mbar_wait(&bar[s ^ 1], ((q + 1) >> 1) & 1, kDrainTries);
                    }
                    __syncthreads();
                    return;
                }
                const int k0 = c * KC, kc = min(KC, n - k0);
                if (row0 < n) {
                    const T *fs = stage + (size_t)s * SE + row0;
                    const T *pk = panel + (size_t)k0 * NC + cg * HALF;
                    for (int kk = 0; kk < kc; ++kk) {
                        T fv[8], rv[CPT];
                        load_vec<T, 8>(fs + (size_t)kk * ld, fv);
                        load_vec<T, HALF>(pk + (size_t)kk * NC, rv);
                        load_vec<T, HALF>(pk + (size_t)kk * NC + NC / 2, rv + HALF);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
#pragma unroll
                            for (int j = 0; j < CPT; ++j) acc[i][j] = fma(fv[i], rv[j], acc[i][j]);
                    }
                }
                __syncthreads();  // every thread is done with stage s
                if (tid == 0 && q + 2 < Q) issue(q + 2);
            }
            if (row0 < n) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    const int c = j < HALF ? cg * HALF + j : NC / 2 + cg * HALF + (j - HALF);
                    const int64_t d = dst[c];
                    if (d < 0) continue;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (row0 + i < n) put_val(zb + d, row0 + i, acc[i][j], pairs);
                }
            }
        }
        __syncthreads();  // the next group overwrites the columns and the panel
    }
}

// ---- phase 2: z = D r + sum over the blocks containing each DOF of their Zb rows

// Along one axis, the blocks whose box contains lattice index i (at most two, ascending), with i's
// offset in the box and the box width: vertex patches [P v - (P-1), P v + (P-1)] clipped (the vertex
// i / P itself when i is a vertex node, else both vertices of the cell), element boxes [P c, P c + P]
// (at a vertex node the cells on both sides that exist).
struct AxisCand {
    int id[2], loc[2], dim[2];
    bool on[2];
};

template <int P>
__device__ __forceinline__ AxisCand axis_cand(int rule, int i, int ncell, int M)
{
    AxisCand a;
    const int c = i / P, s = i - P * c;
    if (rule == 3) {
        a.on[0] = s == 0 && c >= 1;
        a.id[0] = c - 1;
        a.loc[0] = i - P * (c - 1);
        a.on[1] = c < ncell;
        a.id[1] = c;
        a.loc[1] = s;
        a.dim[0] = a.dim[1] = P + 1;
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int v = c + k, lo = max(0, P * v - (P - 1)), hi = min(M - 1, P * v + (P - 1));
            a.id[k] = v;
            a.loc[k] = i - lo;
            a.dim[k] = hi - lo + 1;
        }
        a.on[0] = true;
        a.on[1] = s != 0;
    }
    return a;
}

// One thread per lattice node: blockDim (32, 8), grid (ceil(M0 / 32), ceil(M1 / 8), M2), so a warp is 32
// consecutive nodes along x with the same y and z (coalesced Zb rows, warp-uniform y/z candidates).
template <int P, bool PAIRS>
__global__ void __launch_bounds__(256)
    schwarz_sum_kernel(const double *__restrict__ r, double *__restrict__ z, const double *__restrict__ jac,
                       const double *__restrict__ zb, const int *__restrict__ slot_of, Grid3 g, int rule, int zs,
                       int64_t zsize, int64_t nlat, int nr, const int *__restrict__ done)
{
    if (done && *done) return;
    const int nid0 = rule == 3 ? g.n[0] : g.n[0] + 1, nid1 = rule == 3 ? g.n[1] : g.n[1] + 1;
    const int i0 = blockIdx.x * 32 + threadIdx.x, i1 = blockIdx.y * 8 + threadIdx.y, i2 = blockIdx.z;
    if (i0 < g.M[0] && i1 < g.M[1]) {
        const int64_t node = i0 + (int64_t)g.M[0] * (i1 + (int64_t)g.M[1] * i2);
        const AxisCand ax = axis_cand<P>(rule, i0, g.n[0], g.M[0]);
        const AxisCand ay = axis_cand<P>(rule, i1, g.n[1], g.M[1]);
        const AxisCand az = axis_cand<P>(rule, i2, g.n[2], g.M[2]);
        // the (up to 8) blocks in a fixed order: the node's first entry in the block's slot (entries of
        // 8 bytes from the start of Zb; nslots * zs < 2^31), -1 for none, and the slot's format
        int ent[8];
        bool f32[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int kx = q & 1, ky = (q >> 1) & 1, kz = q >> 2;
            int sv = -1;
            if (ax.on[kx] && ay.on[ky] && az.on[kz]) sv = slot_of[ax.id[kx] + nid0 * (ay.id[ky] + nid1 * az.id[kz])];
            f32[q] = sv >= 0 && (sv & kSlotF32);
            ent[q] = sv < 0 ? -1 : (sv & (kSlotF32 - 1)) * zs;
            // within the slot: FP32 slots count floats, the others 8-byte entries
            const int loc = 3 * (ax.loc[kx] + ax.dim[kx] * (ay.loc[ky] + ay.dim[ky] * az.loc[kz]));
            ent[q] = sv < 0 ? -1 : 2 * ent[q] + (f32[q] ? loc : 2 * loc);  // in floats
        }
        for (int k = 0; k < nr; ++k) {
            const int64_t gi = (int64_t)k * nlat + 3 * node;
            const float *zk = reinterpret_cast<const float *>(zb + (int64_t)k * zsize);
            // FP64 entries: FP64 sums.  Pair format: FP32 results summed in FP32 (they carry FP32 accuracy),
            // float pairs by TwoSum; one FP64 add per DOF at the end.
            double acc[3] = {0.0, 0.0, 0.0};
            float S[3] = {0.f, 0.f, 0.f}, C[3] = {0.f, 0.f, 0.f}, F[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (ent[q] < 0) continue;
                const float *zf = zk + ent[q];
                if constexpr (PAIRS) {
                    if (f32[q]) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) F[c] = __fadd_rn(F[c], zf[c]);
                    } else {
                        const float2 *zp = reinterpret_cast<const float2 *>(zf);
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float2 v = zp[c];
                            ff_add(S[c], C[c], v.x, v.y);
                        }
                    }
                } else {
                    const double *zd = reinterpret_cast<const double *>(zf);
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[c] += zd[c];
                }
            }
            if constexpr (PAIRS) {
#pragma unroll
                for (int c = 0; c < 3; ++c) ff_add(S[c], C[c], F[c], 0.f);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double v = PAIRS ? f2d(S[c]) + f2d(C[c]) : acc[c];
                if (jac) v = fma(jac[3 * node + c], r[gi + c], v);
                z[gi + c] = v;
            }
        }
    }
}

// ---- phase 1c on the tensor cores: tcgen05 products for the FP32 shared factors (p = 2, 3; one
// right-hand side)
//
// D[m][i] = sum_k R[m][k] F[i][k] for the 128 columns m of a tile (blocks sharing the factor F) and
// the rows i of F, as tcgen05.mma kind::tf32 with M = 128 columns, N = the factor's rows (pieces of
// at most 256) and K = 8 per instruction, the accumulators in tensor memory (TMEM).  TF32 keeps 10
// mantissa bits, so each operand is split, x = hi + lo with hi = x with its low 13 bits cleared
// (exact in TF32) and lo = x - hi rounded to TF32, and the products hi*hi + hi*lo + lo*hi are
// accumulated in FP32: about 2^-22 relative, which the shared (uncut, well-conditioned) factors
// tolerate.
//
// Operands in shared memory use the tensor core's canonical K-major layout without swizzle: 8 rows x
// 16 bytes per core matrix, core matrices 128 B apart along K and 512 B apart along M or N, in chunks
// of 16 K values.  The factor's hi/lo tiles are built once at fcm_precond_build (tc_factor_kernel) in
// that layout, so a chunk of them is one run of bytes, moved by bulk copies completed on the stage's
// mbarrier.  The residual panel is gathered from r by eight producer warps straight into the stage
// (FP64 -> hi/lo), each thread one column and 8 K values, loading the next chunk while it stores the
// current one.  One thread issues the copies and the MMAs; tcgen05.commit on a stage's `empty`
// barrier hands the stage back to the producers and the copy engine.  The producer warps then read
// the accumulators (tcgen05.ld) and write the rows to Zb through a shared-memory transpose, so that
// each store covers consecutive rows of one block.

template <int P> struct TcCfg {
    static constexpr int NRP = (sbox_max(P) + 15) / 16 * 16;          // factor rows, padded (384 at p = 3)
    static constexpr int NPIECE = NRP > 256 ? NRP / 2 : NRP;         // N of one MMA (192 or 96)
    static constexpr int NPIECES = NRP / NPIECE;
    static constexpr int TMEM_COLS = NRP > 256 ? 512 : NRP > 128 ? 256 : 128;
    static constexpr int A_BYTES = 2 * 128 * 16 * 4;                 // hi and lo of 128 columns x 16 K
    static constexpr int B_BYTES = 2 * NRP * 16 * 4;                 // hi and lo of NRP rows x 16 K
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = 3;
    static constexpr int HEAD = 4096;                                // barriers, TMEM address, column bases, box offsets
    static constexpr int SMEM = HEAD + STAGES * STAGE;
    static constexpr int THREADS = 32 * 9;                           // warp 0: copies and MMAs; warps 1-8: producers
    static constexpr int CTAS_PER_SM = 2 * SMEM <= 227 * 1024 ? 2 : 1;
};
static_assert(TcCfg<3>::NPIECE % 16 == 0 && TcCfg<3>::NPIECE <= 256 && TcCfg<2>::NPIECE % 16 == 0, "MMA N");
static_assert(TcCfg<3>::SMEM <= 227 * 1024 && TcCfg<2>::SMEM <= 227 * 1024, "tensor-core tile exceeds shared memory");
static_assert((TcCfg<3>::NRP / 2) % 16 == 0 && (TcCfg<2>::NRP / 2) % 16 == 0, "epilogue column split");

// float offset of element (row, kk) (kk < 16) in one hi or lo part of a chunk, canonical K-major layout
__host__ __device__ __forceinline__ int tc_off(int row, int kk)
{
    return (row >> 3) * 128 + (kk >> 2) * 32 + (row & 7) * 4 + (kk & 3);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// x rounded to the nearest TF32 value (ties away from zero), so that the tensor core's reading of the
// low part drops nothing
__device__ __forceinline__ float tf32_rn(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

// 64-bit shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init_count(uint64_t *bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Factor tiles of one shared factor (built once): chunk c = [hi | lo], NRP rows x 16 K each.
template <int P>
__global__ void tc_factor_kernel(const double *__restrict__ F, int n, float *__restrict__ ft)
{
    using Cfg = TcCfg<P>;
    const int ld = factor_ld<double>(n), nch = (n + 15) / 16;
    const int64_t total = (int64_t)nch * Cfg::NRP * 16;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / (Cfg::NRP * 16)), rem = (int)(e % (Cfg::NRP * 16));
        const int row = rem / 16, kk = rem % 16, k = 16 * c + kk;
        const double x = row < n && k < n ? F[(size_t)row * ld + k] : 0.0;
        const float h = tf32_hi((float)x);
        float *hi = ft + (int64_t)c * 2 * Cfg::NRP * 16;
        hi[tc_off(row, kk)] = h;
        hi[Cfg::NRP * 16 + tc_off(row, kk)] = tf32_rn((float)(x - (double)h));
    }
}

template <int P>
__global__ void __launch_bounds__(TcCfg<P>::THREADS, TcCfg<P>::CTAS_PER_SM)
    tc_gemm_kernel(const double *__restrict__ r, const PatchRec *__restrict__ slots, const TcTile *__restrict__ tiles,
                   Grid3 g, int rule, const float *__restrict__ ft, double *__restrict__ zb, int zs, int pairs,
                   int *err, int wait_tries, const int *__restrict__ done)
{
    using Cfg = TcCfg<P>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ __align__(1024) unsigned char smem[];
    if (done && *done) return;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);   // S: panel written and factor chunk landed
    uint64_t *empty = full + S;                            // S: the stage's MMAs completed
    uint64_t *fin = empty + S;                             // every MMA completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    int *flag = reinterpret_cast<int *>(tmem_slot + 1);    // a producer gave up waiting
    int64_t *base = reinterpret_cast<int64_t *>(smem + 128);  // 128 column bases (-1: no block)
    int *rel = reinterpret_cast<int *>(smem + 128 + 1024);     // box offsets, NRP entries
    unsigned char *stages = smem + Cfg::HEAD;
    const TcTile tl = tiles[blockIdx.x];
    const SBox b0 = sbox(rule, P, g, slots[tl.first].v);
    const int n = b0.n, nch = tl.nch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < 128; t += blockDim.x)
        base[t] = t < tl.count ? box_base(sbox(rule, P, g, slots[tl.first + t].v), g) : -1;
    for (int t = threadIdx.x; t < Cfg::NRP; t += blockDim.x) rel[t] = t < n ? box_rel(b0, g, t) : -1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init_count(&full[i], 256 + 1);  // 256 producer arrivals + the copy's expect_tx
            mbar_init(&empty[i]);
        }
        mbar_init(fin);
        *flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool failed = false;
    if (warp == 0) {
        if (lane == 0) {
            const char *bsrc = reinterpret_cast<const char *>(ft + tl.ft_off);
            auto issue = [&](int c) {  // factor chunk c into stage c % S
                unsigned char *st = stages + (size_t)(c % S) * Cfg::STAGE + Cfg::A_BYTES;
                mbar_expect(&full[c % S], (uint32_t)Cfg::B_BYTES);
                for (int o = 0; o < Cfg::B_BYTES; o += 16384)
                    bulk_g2s(st + o, bsrc + (size_t)c * Cfg::B_BYTES + o, min(16384, Cfg::B_BYTES - o), &full[c % S]);
            };
            int issued = 0;
            for (; issued < min(S, nch); ++issued) issue(issued);
            constexpr uint32_t idesc = tc_idesc(128, Cfg::NPIECE);
            int c = 0;
            for (; c < nch; ++c) {
                const int s = c % S;
                if (!mbar_wait(&full[s], (c / S) & 1, wait_tries)) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a_hi = smem_u32(stages + (size_t)s * Cfg::STAGE), a_lo = a_hi + 128 * 16 * 4;
                const uint32_t b_hi = a_hi + Cfg::A_BYTES, b_lo = b_hi + Cfg::NRP * 16 * 4;
                for (int ks = 0; ks < 2; ++ks)
                    for (int h = 0; h < Cfg::NPIECES; ++h) {
                        const uint32_t d = tmem + h * Cfg::NPIECE;
                        const uint32_t bo = h * (Cfg::NPIECE / 8) * 512 + ks * 256;
                        const uint64_t ah = smem_desc(a_hi + ks * 256, 128, 512), al = smem_desc(a_lo + ks * 256, 128, 512);
                        const uint64_t bh = smem_desc(b_hi + bo, 128, 512), bl = smem_desc(b_lo + bo, 128, 512);
                        tc_mma(d, ah, bh, idesc, (c | ks) != 0);
                        tc_mma(d, ah, bl, idesc, 1);
                        tc_mma(d, al, bh, idesc, 1);
                    }
                tc_commit(&empty[s]);
                // refill the stage of the previous chunk once its MMAs are done (this chunk's are queued)
                if (c >= 1 && issued < nch) {
                    const int sp = (c - 1) % S;
                    if (!mbar_wait(&empty[sp], ((c - 1) / S) & 1, wait_tries)) {
                        failed = true;
                        ++c;
                        break;
                    }
                    issue(issued++);
                }
            }
            tc_commit(fin);  // arrives once every MMA issued above has completed
            if (failed) {
                // factor copies issued but not consumed land before the CTA leaves
                for (int q = c; q < issued; ++q) mbar_wait(&full[q % S], (q / S) & 1, kDrainTries);
            }
        }
    } else {
        // producers: column m, K values 8 kh .. 8 kh + 7 of each chunk
        const int p = threadIdx.x - 32, m = p & 127, kh = p >> 7;
        const int64_t bm = base[m];
        double cur[8], nxt[8];
        auto load = [&](int c, double *v) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = 16 * c + 8 * kh + i;
                const int rk = k < Cfg::NRP ? rel[k] : -1;
                v[i] = (bm >= 0 && rk >= 0) ? r[bm + rk] : 0.0;
            }
        };
        load(0, cur);
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) load(c + 1, nxt);
            const int s = c % S;
            if (c >= S && !mbar_wait(&empty[s], ((c / S) - 1) & 1, wait_tries)) {
                failed = true;
                break;
            }
            float *hi = reinterpret_cast<float *>(stages + (size_t)s * Cfg::STAGE), *lo = hi + 128 * 16;
#pragma unroll
            for (int q = 0; q < 2; ++q) {  // two groups of 4 K values: one 16-byte store each
                float4 vh, vl;
                float *ph = &vh.x, *pl = &vl.x;
#pragma unroll
                for (int i = 0; i < 4; ++i) split_bits<10>(cur[4 * q + i], ph[i], pl[i]);
                const int o = tc_off(m, 8 * kh + 4 * q);
                *reinterpret_cast<float4 *>(hi + o) = vh;
                *reinterpret_cast<float4 *>(lo + o) = vl;
            }
            // the tensor core reads the panel through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
#pragma unroll
            for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
        }
        if (failed) atomicExch(flag, 1);
    }
    __syncthreads();
    const bool ok = mbar_wait(fin, 0, kDrainTries);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    failed = __syncthreads_or(failed || !ok || *reinterpret_cast<volatile int *>(flag));
    if (failed) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else if (warp >= 1) {
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (columns m) and half (w - 1) / 4 of the rows, 16 at
        // a time, and writes them through a 32 x 17 transpose buffer: each store covers 16 rows of a block
        const int q4 = warp & 3, half = (warp - 1) >> 2;
        float *tb = reinterpret_cast<float *>(stages) + (warp - 1) * 32 * 17;
        const int m = 32 * q4 + lane;
        for (int j0 = half * (Cfg::NRP / 2); j0 < (half + 1) * (Cfg::NRP / 2); j0 += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + j0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
                "%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) tb[lane * 17 + i] = __uint_as_float(v[i]);
            __syncwarp();
            for (int i = 0; i < 16; ++i) {  // columns 2 i, 2 i + 1: 16 rows each
                const int ml = 2 * i + (lane >> 4), row = j0 + (lane & 15), mm = 32 * q4 + ml;
                if (mm < tl.count && row < n)
                    put_f32(zb + (int64_t)(tl.first + mm) * zs, row, tb[ml * 17 + (lane & 15)], pairs);
            }
            __syncwarp();
        }
        (void)m;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS) : "memory");
}

dim3 sum_grid(const Grid3 &g) { return dim3((g.M[0] + 31) / 32, (g.M[1] + 7) / 8, g.M[2]); }

template <int P>
void gemm_launch(const double *r, int64_t nlat, int nr, const double *f64, const float *f32, const SchwarzPlan &pl,
                 double *zb, int64_t zsize, const int *done, cudaStream_t s)
{
    const Grid3 &g = pl.g;
    // one right-hand side: the FP32 shared factors that have tensor-core tiles go through tcgen05
    const bool tc = nr == 1 && pl.n_tc_tiles > 0;
    if constexpr (P == 2 || P == 3) {
        if (tc)
            tc_gemm_kernel<P><<<pl.n_tc_tiles, TcCfg<P>::THREADS, TcCfg<P>::SMEM, s>>>(
                r, pl.slots, pl.tc_tiles, g, pl.rule, pl.tc_ft, zb, pl.zs, pl.pairs, pl.err, pl.wait_tries, done);
    }
    const int n32 = tc ? pl.n_tiles32_plain : pl.n_tiles32;
    if (n32 > 0)
        schwarz_gemm_kernel<P, float><<<n32, gemm_threads(P), gemm_smem_bytes<P, float>(), s>>>(
            r, nlat, nr, f32, pl.slots, pl.tiles, g, pl.rule, zb, pl.zs, zsize, pl.pairs, pl.err, pl.wait_tries, done);
    if (pl.n_tiles64 > 0)
        schwarz_gemm_kernel<P, double><<<pl.n_tiles64, gemm_threads(P), gemm_smem_bytes<P, double>(), s>>>(
            r, nlat, nr, f64, pl.slots, pl.tiles + pl.n_tiles32, g, pl.rule, zb, pl.zs, zsize, pl.pairs, pl.err,
            pl.wait_tries, done);
}

template <int P, int NR>
void cols_launch(const double *r, int64_t nlat, int nr, const double *f64, const float *f32, const SchwarzPlan &pl,
                 double *zb, int64_t zsize, const int *done, cudaStream_t s)
{
    const int smem = factor_ld<double>(sbox_max(P)) * NR * 8;
    schwarz_cols_kernel<P, NR><<<pl.n_col_items, cols_threads(P), smem, s>>>(
        r, nlat, nr, f64, f32, pl.slots, pl.col_items, pl.g, pl.rule, zb, pl.zs, zsize, pl.pairs, done);
}

template <int P>
void apply_p(const double *r, double *z, int64_t nlat, int nr, const double *f64, const float *f32,
             const SchwarzPlan &pl, double *zb, const int *done, cudaStream_t s)
{
    const int64_t zsize = (int64_t)pl.nslots * pl.zs;
    const bool gemm = pl.n_tiles32 + pl.n_tiles64 + (nr == 1 ? pl.n_tc_tiles : 0) > 0;
    const bool own = nr == 1 && P == 3 ? pl.n_row_items > 0 : pl.n_col_items > 0;
    const bool side = pl.concurrent && gemm && own && pl.side;
    if (side) {
        // the shared-factor products on the second stream, beside the streamed factors
        cudaEventRecord(pl.ev_fork, s);
        cudaStreamWaitEvent(pl.side, pl.ev_fork, 0);
        gemm_launch<P>(r, nlat, nr, f64, f32, pl, zb, zsize, done, pl.side);
        cudaEventRecord(pl.ev_join, pl.side);
    } else if (gemm) {
        gemm_launch<P>(r, nlat, nr, f64, f32, pl, zb, zsize, done, s);
    }
    if (own) {
        if constexpr (P == 3) {
            if (nr == 1)
                schwarz_rows_kernel<P><<<pl.n_row_items, kRowsThreads, 0, s>>>(
                    r, f64, f32, pl.slots, pl.row_items, pl.rows, pl.g, pl.rule, zb, pl.zs, pl.pairs, done);
            else
                cols_launch<P, 8>(r, nlat, nr, f64, f32, pl, zb, zsize, done, s);
        } else if (nr == 1)
            cols_launch<P, 1>(r, nlat, nr, f64, f32, pl, zb, zsize, done, s);
        else
            cols_launch<P, 8>(r, nlat, nr, f64, f32, pl, zb, zsize, done, s);
    }
    if (side) cudaStreamWaitEvent(s, pl.ev_join, 0);
    if (pl.pairs)
        schwarz_sum_kernel<P, true><<<sum_grid(pl.g), dim3(32, 8), 0, s>>>(r, z, pl.jac, zb, pl.slot_of, pl.g, pl.rule,
                                                                       pl.zs, zsize, nlat, nr, done);
    else
        schwarz_sum_kernel<P, false><<<sum_grid(pl.g), dim3(32, 8), 0, s>>>(r, z, pl.jac, zb, pl.slot_of, pl.g, pl.rule,
                                                                        pl.zs, zsize, nlat, nr, done);
}

template <int P>
cudaError_t prepare_p()
{
    cudaError_t e = cudaFuncSetAttribute(schwarz_gemm_kernel<P, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         gemm_smem_bytes<P, float>());
    if constexpr (P == 2 || P == 3)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tc_gemm_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<P>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(schwarz_gemm_kernel<P, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gemm_smem_bytes<P, double>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(schwarz_cols_kernel<P, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 factor_ld<double>(sbox_max(P)) * 8 * 8);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(schwarz_cols_kernel<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 factor_ld<double>(sbox_max(P)) * 8);
    return e;
}

static_assert(gemm_smem_bytes<3, float>() <= 227 * 1024, "GEMM tile exceeds shared memory");
static_assert(gemm_smem_bytes<3, double>() <= 227 * 1024, "GEMM tile exceeds shared memory");
static_assert(gemm_smem_bytes<4, float>() <= 227 * 1024, "GEMM tile exceeds shared memory");
static_assert(gemm_smem_bytes<4, double>() <= 227 * 1024, "GEMM tile exceeds shared memory");
static_assert(factor_ld<double>(sbox_max(4)) * 8 * 8 <= 227 * 1024, "multi-RHS panel exceeds shared memory");

}  // namespace

int schwarz_gemm_cols(int p, int prec)
{
    switch (p) {
    case 1: return prec == 1 ? GemmCfg<float, 1>::NC : GemmCfg<double, 1>::NC;
    case 2: return prec == 1 ? GemmCfg<float, 2>::NC : GemmCfg<double, 2>::NC;
    case 3: return prec == 1 ? GemmCfg<float, 3>::NC : GemmCfg<double, 3>::NC;
    default: return prec == 1 ? GemmCfg<float, 4>::NC : GemmCfg<double, 4>::NC;
    }
}

int schwarz_col_rows(int p)
{
    switch (p) {
    case 1: return cols_threads(1);
    case 2: return cols_threads(2);
    case 3: return cols_threads(3);
    default: return cols_threads(4);
    }
}

bool schwarz_uses_rows_kernel(int p) { return p == 3; }

bool schwarz_tc_supported(int p) { return p == 2 || p == 3; }

int64_t schwarz_tc_factor_floats(int p, int n)
{
    const int nrp = p == 3 ? TcCfg<3>::NRP : TcCfg<2>::NRP;
    return (int64_t)((n + 15) / 16) * 2 * nrp * 16;
}

cudaError_t schwarz_tc_factor(int p, const double *F, int n, float *ft, cudaStream_t s)
{
    const int64_t total = schwarz_tc_factor_floats(p, n) / 2;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 1024);
    if (p == 3) tc_factor_kernel<3><<<grid, 256, 0, s>>>(F, n, ft);
    else if (p == 2) tc_factor_kernel<2><<<grid, 256, 0, s>>>(F, n, ft);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int schwarz_rows_threads() { return kRowsThreads; }

cudaError_t schwarz_prepare(int p)
{
    switch (p) {
    case 1: return prepare_p<1>();
    case 2: return prepare_p<2>();
    case 3: return prepare_p<3>();
    default: return prepare_p<4>();
    }
}

void launch_schwarz_apply_multi(int p, const double *r, double *z, int64_t nlat, int nr, const double *f64,
                                const float *f32, const SchwarzPlan &plan, double *zb, const int *done, cudaStream_t s)
{
    switch (p) {
    case 1: apply_p<1>(r, z, nlat, nr, f64, f32, plan, zb, done, s); break;
    case 2: apply_p<2>(r, z, nlat, nr, f64, f32, plan, zb, done, s); break;
    case 3: apply_p<3>(r, z, nlat, nr, f64, f32, plan, zb, done, s); break;
    case 4: apply_p<4>(r, z, nlat, nr, f64, f32, plan, zb, done, s); break;
    default: break;
    }
}

void launch_schwarz_apply(int p, const Grid3 &g, const double *r, double *z, const double *f64, const float *f32,
                          const SchwarzPlan &plan, const int *done, cudaStream_t s)
{
    const int64_t nlat = 3 * (int64_t)g.M[0] * g.M[1] * g.M[2];
    launch_schwarz_apply_multi(p, r, z, nlat, 1, f64, f32, plan, plan.zb, done, s);
}

}  // namespace fcm
