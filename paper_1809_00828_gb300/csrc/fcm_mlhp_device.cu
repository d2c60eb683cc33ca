// The multi-level hp system on the GPU (Sec. 2.2 overlays, Sec. 3.2 leaf blocks, Sec. 5 PCG).
//
// The host plan assembles K over the free DOFs (CSR) and the Schwarz factors of the leaf blocks
// (fcm_mlhp.cpp); this file uploads them and runs:
//   - K x: one warp per CSR row;
//   - S r (Eq. (5)) in two launches, as on the uniform grid: every block's product Zb = A_B^+ r_B goes
//     into a slot of its own (one CTA per 32 rows of a block: gather r_B into shared memory, a warp per
//     row reading the factor row coalesced), then one thread per DOF adds the diagonal part and the
//     slots of the blocks containing it, in block order (no colours, no atomics, a fixed order);
//   - K values and factors are stored as float pairs (8 B, as FP64) and both products run in
//     double-float arithmetic on the FP32 pipe, each result within ~2^-44 of the sum of the products'
//     magnitudes, leaving the FP64 pipe one add per row;
//   - PCG with x0 = 0, stopped on ||S r_i|| / ||S b|| <= tol (Eq. (14)), with the uniform grid's fused
//     CG kernels: every scalar stays on the device (deterministic two-level reductions), eight
//     iterations are captured in one CUDA graph, and the host polls the scalars once per graph.
// Every index the kernels use is checked on the host before the upload.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fcm_device.cuh"
#include "fcm_ff.cuh"

namespace fcm {

namespace {

constexpr int kThreads = 256;

// (S, C) summed over the warp, every lane holding the result (ff_add is symmetric in its operands)
__device__ __forceinline__ void ff_warp_sum(float &S, float &C)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float S2 = __shfl_xor_sync(0xffffffffu, S, o), C2 = __shfl_xor_sync(0xffffffffu, C, o);
        ff_add(S, C, S2, C2);
    }
}

// x2 = x as float pairs (split by integer operations), once per product instead of once per nonzero
__global__ void __launch_bounds__(kThreads) mlhp_split_kernel(int n, const double *__restrict__ x,
                                                              float2 *__restrict__ x2, const int *done)
{
    if (done && *done) return;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) x2[i] = split_ff(x[i]);
}

// y = K x, a warp per CSR row.  The values are stored as float pairs (hi, lo; |v - hi - lo| <= 2^-48 |v|),
// x arrives split (mlhp_split_kernel), and every product and sum runs in double-float arithmetic on the
// FP32 pipe (GB300's FP64 pipe does 2 operations per clock per SM; a FP64 multiply-add per nonzero plus
// the row reductions kept it busy 77 % of the time).  One FP64 add per row.
__global__ void __launch_bounds__(kThreads) mlhp_spmv_kernel(int n, const int64_t *__restrict__ rowptr,
                                                             const int *__restrict__ cols,
                                                             const float2 *__restrict__ vals,
                                                             const float2 *__restrict__ x, double *__restrict__ y,
                                                             const int *done)
{
    if (done && *done) return;
    const int row = (int)((blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;  // uniform across the warp
    float S = 0.f, C = 0.f;
    const int64_t e1 = rowptr[row + 1];
#pragma unroll 4
    for (int64_t e = rowptr[row] + lane; e < e1; e += 32) {
        const float2 v = __ldcs(vals + e);
        const float2 xv = x[cols[e]];
        ff_fma(v.x, v.y, xv.x, xv.y, S, C);
    }
    ff_warp_sum(S, C);
    if (lane == 0) y[row] = ff_to_double(ff_norm(S, C));
}

// Zb[o_B + i] = (A_B^+ r_B)_i for the rows i of item (block, first row): a CTA per 32 rows of a block.
// Factors as float pairs, r_B split once into shared memory, double-float products and sums.
constexpr int kRowsPerCta = 32;

// Blocks with `prec` 1 keep FP32 factors (retained condition number <= 1e7, the uniform grid's rule):
// half the bytes, and plain FP32 products and sums (the factor's own rounding, 2^-24, already bounds the
// accuracy; about (m / 32 + 8) 2^-24 of sum |F_ij r_j| per row).  fptr: offset in the block's own pool.
template <class T>
__device__ __forceinline__ void row_fma(const T *p, float2 rj, float &S, float &C);
template <>
__device__ __forceinline__ void row_fma<float2>(const float2 *p, float2 rj, float &S, float &C)
{
    const float2 f = __ldcs(p);
    ff_fma(f.x, f.y, rj.x, rj.y, S, C);
}
template <>
__device__ __forceinline__ void row_fma<float>(const float *p, float2 rj, float &S, float &)
{
    S = __fmaf_rn(__ldcs(p), __fadd_rn(rj.x, rj.y), S);
}

template <class T>
__device__ __forceinline__ void block_rows(const T *__restrict__ F, int m, int row0, const float2 *rb, int64_t o,
                                           double *__restrict__ zb)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the warp's four rows row0 + warp + 8 t at once: four independent streams of factor loads in flight
    constexpr int kRowsPerWarp = kRowsPerCta / (kThreads / 32);
    const int row_end = min(m, row0 + kRowsPerCta);
    const T *Fi[kRowsPerWarp];
    bool on[kRowsPerWarp];
#pragma unroll
    for (int t = 0; t < kRowsPerWarp; ++t) {
        const int i = row0 + warp + t * (kThreads / 32);
        on[t] = i < row_end;  // warp-uniform
        Fi[t] = F + (int64_t)(on[t] ? i : row0) * m;
    }
    float S[kRowsPerWarp] = {}, C[kRowsPerWarp] = {};
#pragma unroll 2
    for (int j = lane; j < m; j += 32) {
        const float2 rj = rb[j];
#pragma unroll
        for (int t = 0; t < kRowsPerWarp; ++t)
            if (on[t]) row_fma<T>(Fi[t] + j, rj, S[t], C[t]);
    }
#pragma unroll
    for (int t = 0; t < kRowsPerWarp; ++t) {
        double v;
        if constexpr (sizeof(T) == sizeof(float)) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) S[t] = __fadd_rn(S[t], __shfl_xor_sync(0xffffffffu, S[t], off));
            v = f2d(S[t]);
        } else {
            ff_warp_sum(S[t], C[t]);
            v = ff_to_double(ff_norm(S[t], C[t]));
        }
        if (on[t] && lane == 0) zb[o + row0 + warp + t * (kThreads / 32)] = v;
    }
}

__global__ void __launch_bounds__(kThreads) mlhp_block_rows_kernel(const int2 *__restrict__ items,
                                                                   const int64_t *__restrict__ bptr,
                                                                   const int *__restrict__ bdofs,
                                                                   const int64_t *__restrict__ fptr,
                                                                   const uint8_t *__restrict__ prec,
                                                                   const float2 *__restrict__ fac,
                                                                   const float *__restrict__ fac32,
                                                                   const double *__restrict__ r,
                                                                   double *__restrict__ zb, const int *done)
{
    if (done && *done) return;
    extern __shared__ float2 rb[];
    const int2 it = items[blockIdx.x];
    const int64_t o = bptr[it.x];
    const int m = (int)(bptr[it.x + 1] - o);
    for (int j = threadIdx.x; j < m; j += kThreads) rb[j] = split_ff(r[bdofs[o + j]]);
    __syncthreads();
    if (prec[it.x])  // CTA-uniform
        block_rows<float>(fac32 + fptr[it.x], m, it.y, rb, o, zb);
    else
        block_rows<float2>(fac + fptr[it.x], m, it.y, rb, o, zb);
}

// z_d = jac_d r_d + sum of the slots of the blocks containing d, in block order
__global__ void __launch_bounds__(kThreads) mlhp_sum_kernel(int n, const int64_t *__restrict__ occ_ptr,
                                                            const int *__restrict__ occ, const double *__restrict__ zb,
                                                            const double *__restrict__ jac, const double *__restrict__ r,
                                                            double *__restrict__ z, const int *done)
{
    if (done && *done) return;
    for (int d = blockIdx.x * kThreads + threadIdx.x; d < n; d += gridDim.x * kThreads) {
        double s = jac[d] * r[d];
        for (int64_t k = occ_ptr[d]; k < occ_ptr[d + 1]; ++k) s += zb[occ[k]];
        z[d] = s;
    }
}

template <class T>
cudaError_t upload(T **d, const T *h, size_t count, cudaStream_t st)
{
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(d), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (count) e = cudaMemcpyAsync(*d, h, count * sizeof(T), cudaMemcpyHostToDevice, st);
    return e;
}

}  // namespace

constexpr int kChunk = 8;  // PCG iterations per captured graph

struct MlhpDevice {
    cudaStream_t st = nullptr;    // the caller's stream (applies; the solve is ordered after it)
    cudaStream_t own = nullptr;   // the solve's stream (capturable)
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int n = 0, max_block = 0, nitems = 0;
    int64_t nslots = 0;
    int64_t *rowptr = nullptr, *bptr = nullptr, *fptr = nullptr, *occ_ptr = nullptr;
    int *cols = nullptr, *bdofs = nullptr, *occ = nullptr;
    int2 *items = nullptr;
    float2 *vals = nullptr, *fac = nullptr;  // K values and factors as float pairs
    float *fac32 = nullptr;                  // FP32 factors (mixed precision)
    uint8_t *prec = nullptr;                 // per block: 1 when its factor is in fac32
    int64_t n_fp32 = 0, factor_bytes = 0;
    float2 *x2 = nullptr;                    // the K apply's input as float pairs
    double *jac = nullptr, *zb = nullptr;
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b = nullptr, *partial = nullptr;
    unsigned *counter = nullptr;
    CgScalars *s = nullptr, *hs = nullptr;  // device scalars, pinned host copy
    int grid_n = 1, red_blocks = 1;
    cudaGraphExec_t graph = nullptr;
};

void mlhp_device_destroy(MlhpDevice *d)
{
    if (!d) return;
    if (d->graph) cudaGraphExecDestroy(d->graph);
    for (void *ptr : {(void *)d->rowptr, (void *)d->bptr, (void *)d->fptr, (void *)d->occ_ptr, (void *)d->cols,
                      (void *)d->bdofs, (void *)d->occ, (void *)d->items, (void *)d->vals, (void *)d->fac,
                      (void *)d->jac, (void *)d->zb, (void *)d->x, (void *)d->r, (void *)d->z, (void *)d->p,
                      (void *)d->q, (void *)d->b, (void *)d->partial, (void *)d->counter, (void *)d->s,
                      (void *)d->x2, (void *)d->fac32, (void *)d->prec})
        if (ptr) cudaFree(ptr);
    if (d->hs) cudaFreeHost(d->hs);
    if (d->ev_a) cudaEventDestroy(d->ev_a);
    if (d->ev_b) cudaEventDestroy(d->ev_b);
    if (d->own) cudaStreamDestroy(d->own);
    delete d;
}

#define MLHP_CUDA(call)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return std::string(#call) + ": " + cudaGetErrorString(e_);          \
    } while (0)

std::string mlhp_device_create(void *stream, int64_t n, const int64_t *rowptr, const int64_t *cols, const double *vals,
                               int64_t nblocks, const int64_t *bptr, const int64_t *bdofs, const int64_t *fptr,
                               const double *fac, int ncolours, const int64_t *cptr, const double *jac,
                               const double *fac_cond, MlhpDevice **out)
{
    *out = nullptr;
    // every index the kernels will use, checked here
    if (n < 1 || n > ((int64_t)1 << 30)) return "system size out of range";  // 32-bit grid-stride indices stay valid
    if (rowptr[0] != 0) return "bad CSR row pointer";
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return "bad CSR row pointer";
    const int64_t nnz = rowptr[n];
    for (int64_t e = 0; e < nnz; ++e)
        if (cols[e] < 0 || cols[e] >= n) return "CSR column out of range";
    if (nblocks < 0 || nblocks > ((int64_t)1 << 30) || bptr[0] != 0 || fptr[0] != 0) return "bad block pointers";
    int max_block = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t m = bptr[b + 1] - bptr[b];
        if (m < 1 || m > 4096 || fptr[b + 1] - fptr[b] != m * m) return "bad block pointers";
        max_block = std::max(max_block, (int)m);
    }
    const int64_t nslots = bptr[nblocks];
    if (nslots >= ((int64_t)1 << 31)) return "too many block rows";
    for (int64_t k = 0; k < nslots; ++k)
        if (bdofs[k] < 0 || bdofs[k] >= n) return "block DOF out of range";
    if (ncolours < 0 || cptr[0] != 0 || cptr[ncolours] != nblocks) return "bad colour pointers";
    for (int c = 0; c < ncolours; ++c)
        if (cptr[c + 1] < cptr[c]) return "bad colour pointers";
    // work items (block, first row) and, per DOF, its slots in block order
    std::vector<int2> items;
    for (int64_t b = 0; b < nblocks; ++b)
        for (int64_t i = 0; i < bptr[b + 1] - bptr[b]; i += kRowsPerCta) items.push_back(make_int2((int)b, (int)i));
    std::vector<int64_t> occ_ptr(n + 1, 0);
    for (int64_t k = 0; k < nslots; ++k) occ_ptr[bdofs[k] + 1] += 1;
    for (int64_t i = 0; i < n; ++i) occ_ptr[i + 1] += occ_ptr[i];
    std::vector<int> occ(nslots), fill(occ_ptr.begin(), occ_ptr.end() - 1);
    for (int64_t k = 0; k < nslots; ++k) occ[fill[bdofs[k]]++] = (int)k;  // k grows with the block index
    MlhpDevice *d = new MlhpDevice;
    d->st = static_cast<cudaStream_t>(stream);
    d->n = (int)n;
    d->max_block = max_block;
    d->nitems = (int)items.size();
    d->nslots = nslots;
    d->grid_n = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 8 * 152);
    d->red_blocks = d->grid_n;
    std::vector<int> cols32(cols, cols + nnz), bdofs32(bdofs, bdofs + nslots);
    auto fail = [&](const std::string &m) {
        mlhp_device_destroy(d);
        return m;
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaStreamCreateWithFlags(&d->own, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&d->ev_a, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&d->ev_b, cudaEventDisableTiming)) != cudaSuccess)
        return fail(std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    // float pairs: hi = fl32(v), lo = fl32(v - hi), so |v - hi - lo| <= 2^-48 |v|
    auto pairs = [](const double *v, int64_t cnt) {
        std::vector<float2> out((size_t)cnt);
        for (int64_t i = 0; i < cnt; ++i) {
            const float h = (float)v[i];
            out[(size_t)i] = make_float2(h, (float)(v[i] - (double)h));
        }
        return out;
    };
    const std::vector<float2> vals2 = pairs(vals, nnz);
    // factors: FP32 for the blocks whose retained condition number is at most 1e7 (when fac_cond is
    // given), float pairs for the others; each block's offset is into its own pool
    std::vector<float2> fac2;
    std::vector<float> fac32;
    std::vector<int64_t> foff(nblocks + 1, 0);
    std::vector<uint8_t> prec(std::max<int64_t>(nblocks, 1), 0);
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t cnt = fptr[b + 1] - fptr[b];
        const bool f32 = fac_cond && fac_cond[b] <= 1e7;
        prec[b] = f32 ? 1 : 0;
        if (f32) {
            foff[b] = (int64_t)fac32.size();
            for (int64_t k = 0; k < cnt; ++k) fac32.push_back((float)fac[fptr[b] + k]);
            d->n_fp32 += 1;
        } else {
            foff[b] = (int64_t)fac2.size();
            const std::vector<float2> pb = pairs(fac + fptr[b], cnt);
            fac2.insert(fac2.end(), pb.begin(), pb.end());
        }
    }
    d->factor_bytes = (int64_t)(fac2.size() * sizeof(float2) + fac32.size() * sizeof(float));
    if ((e = upload(&d->rowptr, rowptr, (size_t)n + 1, d->st)) != cudaSuccess ||
        (e = upload(&d->cols, cols32.data(), cols32.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->vals, vals2.data(), vals2.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->bptr, bptr, (size_t)nblocks + 1, d->st)) != cudaSuccess ||
        (e = upload(&d->bdofs, bdofs32.data(), bdofs32.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->fptr, foff.data(), (size_t)nblocks + 1, d->st)) != cudaSuccess ||
        (e = upload(&d->fac, fac2.data(), fac2.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->fac32, fac32.data(), fac32.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->prec, prec.data(), prec.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->jac, jac, (size_t)n, d->st)) != cudaSuccess ||
        (e = upload(&d->items, items.data(), items.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->occ_ptr, occ_ptr.data(), occ_ptr.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->occ, occ.data(), occ.size(), d->st)) != cudaSuccess)
        return fail(std::string("upload: ") + cudaGetErrorString(e));
    if ((e = cudaMalloc(reinterpret_cast<void **>(&d->x2), (size_t)n * sizeof(float2))) != cudaSuccess)
        return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    if ((e = cudaMalloc(reinterpret_cast<void **>(&d->zb), std::max<int64_t>(nslots, 1) * sizeof(double))) != cudaSuccess)
        return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    for (double **v : {&d->x, &d->r, &d->z, &d->p, &d->q, &d->b})
        if ((e = cudaMalloc(reinterpret_cast<void **>(v), (size_t)n * sizeof(double))) != cudaSuccess)
            return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    if ((e = cudaMalloc(reinterpret_cast<void **>(&d->partial), 2 * (size_t)d->red_blocks * sizeof(double))) !=
            cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d->counter), sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d->s), sizeof(CgScalars))) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void **>(&d->hs), sizeof(CgScalars))) != cudaSuccess)
        return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    if ((e = cudaMemsetAsync(d->counter, 0, sizeof(unsigned), d->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d->s, 0, sizeof(CgScalars), d->st)) != cudaSuccess)
        return fail(std::string("cudaMemset: ") + cudaGetErrorString(e));
    // the host copies above come from pageable memory owned by the caller: finish them before returning
    if ((e = cudaStreamSynchronize(d->st)) != cudaSuccess) return fail(std::string("upload: ") + cudaGetErrorString(e));
    *out = d;
    return std::string();
}

namespace {

void apply_K(MlhpDevice *d, const double *x, double *y, const int *done, cudaStream_t st)
{
    const int64_t warps_per_cta = kThreads / 32;
    const unsigned grid = (unsigned)((d->n + warps_per_cta - 1) / warps_per_cta);
    mlhp_split_kernel<<<d->grid_n, kThreads, 0, st>>>(d->n, x, d->x2, done);
    mlhp_spmv_kernel<<<grid, kThreads, 0, st>>>(d->n, d->rowptr, d->cols, d->vals, d->x2, y, done);
}

void apply_S(MlhpDevice *d, const double *r, double *z, const int *done, cudaStream_t st)
{
    if (d->nitems > 0)
        mlhp_block_rows_kernel<<<d->nitems, kThreads, (size_t)d->max_block * sizeof(float2), st>>>(
            d->items, d->bptr, d->bdofs, d->fptr, d->prec, d->fac, d->fac32, r, d->zb, done);
    mlhp_sum_kernel<<<d->grid_n, kThreads, 0, st>>>(d->n, d->occ_ptr, d->occ, d->zb, d->jac, r, z, done);
}

CgWork work_of(MlhpDevice *d)
{
    CgWork w;
    w.x = d->x;
    w.r = d->r;
    w.z = d->z;
    w.p = d->p;
    w.q = d->q;
    w.b = d->b;
    w.partial = d->partial;
    w.counter = d->counter;
    w.s = d->s;
    w.n = d->n;
    w.red_blocks = d->red_blocks;
    return w;
}

const int *done_flag(MlhpDevice *d)
{
    return reinterpret_cast<const int *>(reinterpret_cast<const char *>(d->s) + offsetof(CgScalars, done));
}

}  // namespace

void mlhp_device_info(const MlhpDevice *d, int64_t *n_fp32_blocks, int64_t *factor_bytes)
{
    *n_fp32_blocks = d->n_fp32;
    *factor_bytes = d->factor_bytes;
}

std::string mlhp_device_apply_K(MlhpDevice *d, const double *x, double *y)
{
    apply_K(d, x, y, nullptr, d->st);
    MLHP_CUDA(cudaGetLastError());
    return std::string();
}

std::string mlhp_device_apply_S(MlhpDevice *d, const double *r, double *z)
{
    apply_S(d, r, z, nullptr, d->st);
    MLHP_CUDA(cudaGetLastError());
    return std::string();
}

// status: 0 converged, 1 not converged within maxit, 2 breakdown (p.Kp <= 0 or a non-finite scalar).
std::string mlhp_device_pcg(MlhpDevice *d, const double *b, double tol, int maxit, double *u, int *its, double *relres,
                            int *status)
{
    cudaStream_t st = d->own;
    const CgWork w = work_of(d);
    const size_t bytes = (size_t)d->n * sizeof(double);
    // ordered after the caller's stream, and the caller's stream after the solve
    MLHP_CUDA(cudaEventRecord(d->ev_a, d->st));
    MLHP_CUDA(cudaStreamWaitEvent(st, d->ev_a, 0));
    CgScalars &h = *d->hs;
    std::memset(&h, 0, sizeof h);
    h.tol = tol;
    h.maxit = std::max(maxit, 1);
    MLHP_CUDA(cudaMemcpyAsync(d->s, &h, sizeof h, cudaMemcpyHostToDevice, st));
    MLHP_CUDA(cudaMemcpyAsync(d->b, b, bytes, cudaMemcpyDeviceToDevice, st));
    cg_init_kernels(w, st);
    apply_S(d, d->r, d->z, nullptr, st);
    cg_after_first_S(w, st);
    MLHP_CUDA(cudaGetLastError());
    MLHP_CUDA(cudaMemcpyAsync(&h, d->s, sizeof h, cudaMemcpyDeviceToHost, st));
    MLHP_CUDA(cudaStreamSynchronize(st));
    if (!h.done && maxit > 0) {
        if (!d->graph) {
            MLHP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int *done = done_flag(d);
            for (int i = 0; i < kChunk; ++i) {
                apply_K(d, d->p, d->q, done, st);
                cg_after_K(w, st);
                apply_S(d, d->r, d->z, done, st);
                cg_after_S(w, st);
            }
            cudaGraph_t g = nullptr;
            MLHP_CUDA(cudaStreamEndCapture(st, &g));
            const cudaError_t e = cudaGraphInstantiate(&d->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                d->graph = nullptr;
                return std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
            }
        }
        while (!h.done) {
            MLHP_CUDA(cudaGraphLaunch(d->graph, st));
            MLHP_CUDA(cudaMemcpyAsync(&h, d->s, sizeof h, cudaMemcpyDeviceToHost, st));
            MLHP_CUDA(cudaStreamSynchronize(st));
        }
    }
    MLHP_CUDA(cudaMemcpyAsync(u, d->x, bytes, cudaMemcpyDeviceToDevice, st));
    MLHP_CUDA(cudaEventRecord(d->ev_b, st));
    MLHP_CUDA(cudaStreamWaitEvent(d->st, d->ev_b, 0));
    MLHP_CUDA(cudaStreamSynchronize(st));
    *its = h.it;
    *relres = h.relres;
    if (!h.done) {  // maxit == 0 and not converged at the start
        *status = 1;
    } else {
        *status = h.status == FCM_OK ? 0 : h.status == FCM_ENOTCONV ? 1 : 2;
    }
    return std::string();
}

}  // namespace fcm

// ---- pseudo inverses of the leaf blocks on the device (fcm_mlhp_factorize_device) ----
namespace fcm {

namespace {

// per block (one CTA): U(:, k) = V(:, k) / lambda_k for lambda_k > eps lambda_max, else 0 (V column-major, the
// eigenvectors from syev), and the retained condition number lambda_max / lambda_min
__global__ void __launch_bounds__(kThreads) mlhp_pinv_scale_kernel(const double *__restrict__ V,
                                                                   const double *__restrict__ W, int m, double eps,
                                                                   double *__restrict__ U, double *__restrict__ cond)
{
    const double *v = V + (size_t)blockIdx.x * m * m;
    const double *w = W + (size_t)blockIdx.x * m;
    double *u = U + (size_t)blockIdx.x * m * m;
    __shared__ double lmax_s, lmin_s;
    if (threadIdx.x == 0) {
        double lmax = 0.0;
        for (int k = 0; k < m; ++k) lmax = fmax(lmax, w[k]);
        double lmin = lmax;
        for (int k = 0; k < m; ++k)
            if (w[k] > eps * lmax) lmin = fmin(lmin, w[k]);
        lmax_s = lmax;
        lmin_s = lmin;
        cond[blockIdx.x] = lmin > 0.0 ? lmax / lmin : 1.0;
    }
    __syncthreads();
    const double cut = eps * lmax_s;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int k = t / m;  // column
        u[t] = w[k] > cut ? v[t] / w[k] : 0.0;
    }
}

}  // namespace

#define PINV_CUDA(call)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return std::string(#call) + ": " + cudaGetErrorString(e_);          \
    } while (0)
#define PINV_SOLVER(call)                                                                          \
    do {                                                                                           \
        cusolverStatus_t e_ = (call);                                                              \
        if (e_ != CUSOLVER_STATUS_SUCCESS) return std::string(#call) + ": cusolver status " + std::to_string((int)e_); \
    } while (0)
#define PINV_BLAS(call)                                                                            \
    do {                                                                                           \
        cublasStatus_t e_ = (call);                                                                \
        if (e_ != CUBLAS_STATUS_SUCCESS) return std::string(#call) + ": cublas status " + std::to_string((int)e_); \
    } while (0)

std::string mlhp_device_pinv(void *stream, int64_t nblocks, const int64_t *fac_ptr, const double *A, double eps,
                             double *F, double *cond)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // blocks by size: one batched eigensolve per size (and per chunk of at most ~1 GB of work arrays)
    std::map<int, std::vector<int64_t>> groups;
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t n2 = fac_ptr[b + 1] - fac_ptr[b];
        const int m = (int)std::llround(std::sqrt((double)n2));
        if ((int64_t)m * m != n2 || m < 1) return "factor sizes are not squares";
        groups[m].push_back(b);
    }
    struct Res {
        std::vector<void *> p;
        cusolverDnHandle_t s = nullptr;
        cublasHandle_t b = nullptr;
        cusolverDnParams_t q = nullptr;
        ~Res()
        {
            for (void *x : p) cudaFree(x);
            if (q) cusolverDnDestroyParams(q);
            if (s) cusolverDnDestroy(s);
            if (b) cublasDestroy(b);
        }
    } res;
    PINV_SOLVER(cusolverDnCreate(&res.s));
    PINV_SOLVER(cusolverDnCreateParams(&res.q));
    PINV_SOLVER(cusolverDnSetStream(res.s, st));
    PINV_BLAS(cublasCreate(&res.b));
    PINV_BLAS(cublasSetStream(res.b, st));
    for (auto &kv : groups) {
        const int m = kv.first;
        const std::vector<int64_t> &ids = kv.second;
        const size_t m2 = (size_t)m * m;
        const int chunk = (int)std::max<size_t>(1, std::min<size_t>(ids.size(), (size_t)(1ull << 30) / (3 * m2 * 8)));
        double *dA = nullptr, *dU = nullptr, *dC = nullptr, *dW = nullptr, *dcond = nullptr;
        int *dinfo = nullptr;
        PINV_CUDA(cudaMalloc(&dA, sizeof(double) * m2 * chunk));
        res.p.push_back(dA);
        PINV_CUDA(cudaMalloc(&dU, sizeof(double) * m2 * chunk));
        res.p.push_back(dU);
        PINV_CUDA(cudaMalloc(&dC, sizeof(double) * m2 * chunk));
        res.p.push_back(dC);
        PINV_CUDA(cudaMalloc(&dW, sizeof(double) * m * chunk));
        res.p.push_back(dW);
        PINV_CUDA(cudaMalloc(&dcond, sizeof(double) * chunk));
        res.p.push_back(dcond);
        PINV_CUDA(cudaMalloc(&dinfo, sizeof(int) * chunk));
        res.p.push_back(dinfo);
        bool batched = true;
        size_t dws = 0, hws = 0;
        if (cusolverDnXsyevBatched_bufferSize(res.s, res.q, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m,
                                              CUDA_R_64F, dA, m, CUDA_R_64F, dW, CUDA_R_64F, &dws, &hws,
                                              chunk) != CUSOLVER_STATUS_SUCCESS)
            batched = false;
        if (!batched)
            PINV_SOLVER(cusolverDnXsyevd_bufferSize(res.s, res.q, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m,
                                                    CUDA_R_64F, dA, m, CUDA_R_64F, dW, CUDA_R_64F, &dws, &hws));
        void *dwork = nullptr;
        PINV_CUDA(cudaMalloc(&dwork, std::max<size_t>(dws, 16)));
        res.p.push_back(dwork);
        std::vector<char> hwork(std::max<size_t>(hws, 1));
        std::vector<double> stage(m2 * chunk), hcond(chunk);
        std::vector<int> hinfo(chunk);
        for (size_t s0 = 0; s0 < ids.size(); s0 += chunk) {
            const int B = (int)std::min<size_t>(chunk, ids.size() - s0);
            // the blocks are symmetric, so row-major host storage is their column-major form
            for (int b = 0; b < B; ++b)
                std::copy(A + fac_ptr[ids[s0 + b]], A + fac_ptr[ids[s0 + b]] + m2, stage.begin() + (size_t)b * m2);
            PINV_CUDA(cudaMemcpyAsync(dA, stage.data(), sizeof(double) * m2 * B, cudaMemcpyHostToDevice, st));
            if (batched) {
                PINV_SOLVER(cusolverDnXsyevBatched(res.s, res.q, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m,
                                                   CUDA_R_64F, dA, m, CUDA_R_64F, dW, CUDA_R_64F, dwork, dws,
                                                   hwork.data(), hws, dinfo, B));
            } else {
                for (int b = 0; b < B; ++b)
                    PINV_SOLVER(cusolverDnXsyevd(res.s, res.q, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m,
                                                 CUDA_R_64F, dA + m2 * b, m, CUDA_R_64F, dW + (size_t)m * b, CUDA_R_64F,
                                                 dwork, dws, hwork.data(), hws, dinfo + b));
            }
            mlhp_pinv_scale_kernel<<<B, kThreads, 0, st>>>(dA, dW, m, eps, dU, dcond);
            PINV_CUDA(cudaGetLastError());
            const double one = 1.0, zero = 0.0;
            // C = U V^T: C(i, j) = sum_k V(i, k) V(j, k) / lambda_k, symmetric
            PINV_BLAS(cublasDgemmStridedBatched(res.b, CUBLAS_OP_N, CUBLAS_OP_T, m, m, m, &one, dU, m, (long long)m2, dA,
                                                m, (long long)m2, &zero, dC, m, (long long)m2, B));
            PINV_CUDA(cudaMemcpyAsync(stage.data(), dC, sizeof(double) * m2 * B, cudaMemcpyDeviceToHost, st));
            PINV_CUDA(cudaMemcpyAsync(hcond.data(), dcond, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
            PINV_CUDA(cudaMemcpyAsync(hinfo.data(), dinfo, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
            PINV_CUDA(cudaStreamSynchronize(st));
            for (int b = 0; b < B; ++b) {
                if (hinfo[b] != 0) return "eigensolver failed for a block (info " + std::to_string(hinfo[b]) + ")";
                const int64_t id = ids[s0 + b];
                // exact symmetry, as the host path makes it: the mean of C and its transpose
                const double *c = stage.data() + (size_t)b * m2;
                double *f = F + fac_ptr[id];
                for (int i = 0; i < m; ++i)
                    for (int j = 0; j < m; ++j) f[(size_t)i * m + j] = 0.5 * (c[(size_t)i * m + j] + c[(size_t)j * m + i]);
                cond[id] = hcond[b];
            }
        }
    }
    return std::string();
}

}  // namespace fcm
