// The multi-level hp system on the GPU (Sec. 2.2 overlays, Sec. 3.2 leaf blocks, Sec. 5 PCG).
//
// The host plan assembles K over the free DOFs (CSR) and the Schwarz factors of the leaf blocks
// (fcm_mlhp.cpp); this file uploads them and runs:
//   - K x: one warp per CSR row;
//   - S r (Eq. (5)): z = D r for the DOFs in no block, then one launch per colour, each block's rows split
//     over a few CTAs: gather r_B into shared memory, z_B += A_B^+ r_B with a warp per row, scatter (the
//     blocks of one colour share no DOF, so no atomics);
//   - PCG with x0 = 0, stopped on ||S r_i|| / ||S b|| <= tol (Eq. (14)): the dot products are two-level
//     reductions in a fixed order (deterministic), the scalars go to the host each iteration.
// Every index the kernels use is checked on the host before the upload.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fcm_internal.h"

namespace fcm {

namespace {

constexpr int kDotGrid = 304;  // 2 CTAs per SM of a 152-SM GB300
constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kThreads) mlhp_spmv_kernel(int n, const int64_t *__restrict__ rowptr,
                                                             const int *__restrict__ cols,
                                                             const double *__restrict__ vals,
                                                             const double *__restrict__ x, double *__restrict__ y)
{
    const int row = (int)((blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;  // uniform across the warp
    double s = 0.0;
    for (int64_t e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) s += vals[e] * x[cols[e]];
    s = warp_sum(s);
    if (lane == 0) y[row] = s;
}

__global__ void __launch_bounds__(kThreads) mlhp_diag_kernel(int n, const double *__restrict__ jac,
                                                             const double *__restrict__ r, double *__restrict__ z)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) z[i] = jac[i] * r[i];
}

// z_B += A_B^+ r_B for the blocks of one colour.  A block's rows are split over `splits` CTAs of
// kRowsPerCta rows (more CTAs in flight than blocks in a colour); every CTA gathers r_B into shared memory,
// then each warp takes one row at a time and reads it coalesced, lanes striding over the columns.
constexpr int kRowsPerCta = 32;

__global__ void __launch_bounds__(kThreads) mlhp_block_kernel(int64_t first, int splits, const int64_t *__restrict__ bptr,
                                                              const int *__restrict__ bdofs,
                                                              const int64_t *__restrict__ fptr,
                                                              const double *__restrict__ fac,
                                                              const double *__restrict__ r, double *__restrict__ z)
{
    extern __shared__ double rb[];
    const int64_t b = first + blockIdx.x / splits;
    const int row0 = (int)(blockIdx.x % splits) * kRowsPerCta;
    const int64_t o = bptr[b];
    const int m = (int)(bptr[b + 1] - o);
    if (row0 >= m) return;  // uniform across the CTA, before any barrier
    const double *F = fac + fptr[b];
    for (int j = threadIdx.x; j < m; j += kThreads) rb[j] = r[bdofs[o + j]];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row_end = min(m, row0 + kRowsPerCta);
    for (int i = row0 + warp; i < row_end; i += kThreads / 32) {  // warp-uniform bounds
        const double *Fi = F + (int64_t)i * m;
        double s = 0.0;
        for (int j = lane; j < m; j += 32) s += Fi[j] * rb[j];
        s = warp_sum(s);
        if (lane == 0) z[bdofs[o + i]] += s;
    }
}

__global__ void __launch_bounds__(kThreads) mlhp_dot_partial_kernel(int n, const double *__restrict__ a,
                                                                    const double *__restrict__ b,
                                                                    double *__restrict__ partial)
{
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) s += a[i] * b[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

__global__ void mlhp_dot_final_kernel(int g, const double *__restrict__ partial, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < g; ++i) s += partial[i];
        *out = s;
    }
}

__global__ void __launch_bounds__(kThreads) mlhp_xr_kernel(int n, double a, const double *__restrict__ p,
                                                           const double *__restrict__ q, double *__restrict__ x,
                                                           double *__restrict__ r)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        x[i] += a * p[i];
        r[i] -= a * q[i];
    }
}

__global__ void __launch_bounds__(kThreads) mlhp_p_kernel(int n, double beta, const double *__restrict__ z,
                                                          double *__restrict__ p)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) p[i] = z[i] + beta * p[i];
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

struct MlhpDevice {
    cudaStream_t st = nullptr;
    int n = 0, ncolours = 0, max_block = 0;
    std::vector<int64_t> colour_ptr;
    int64_t *rowptr = nullptr, *bptr = nullptr, *fptr = nullptr;
    int *cols = nullptr, *bdofs = nullptr;
    double *vals = nullptr, *fac = nullptr, *jac = nullptr;
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *partial = nullptr, *scalar = nullptr;
    int grid_n = 1;
};

void mlhp_device_destroy(MlhpDevice *d)
{
    if (!d) return;
    for (void *ptr : {(void *)d->rowptr, (void *)d->bptr, (void *)d->fptr, (void *)d->cols, (void *)d->bdofs,
                      (void *)d->vals, (void *)d->fac, (void *)d->jac, (void *)d->x, (void *)d->r, (void *)d->z,
                      (void *)d->p, (void *)d->q, (void *)d->partial, (void *)d->scalar})
        if (ptr) cudaFree(ptr);
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
                               MlhpDevice **out)
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
    if (nblocks < 0 || bptr[0] != 0 || fptr[0] != 0) return "bad block pointers";
    int max_block = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t m = bptr[b + 1] - bptr[b];
        if (m < 1 || m > 4096 || fptr[b + 1] - fptr[b] != m * m) return "bad block pointers";
        max_block = std::max(max_block, (int)m);
    }
    for (int64_t k = 0; k < bptr[nblocks]; ++k)
        if (bdofs[k] < 0 || bdofs[k] >= n) return "block DOF out of range";
    if (ncolours < 0 || cptr[0] != 0 || cptr[ncolours] != nblocks) return "bad colour pointers";
    for (int c = 0; c < ncolours; ++c)
        if (cptr[c + 1] < cptr[c]) return "bad colour pointers";
    {  // blocks of one colour share no DOF
        std::vector<int> seen(n, -1);
        for (int c = 0; c < ncolours; ++c)
            for (int64_t b = cptr[c]; b < cptr[c + 1]; ++b)
                for (int64_t k = bptr[b]; k < bptr[b + 1]; ++k) {
                    if (seen[bdofs[k]] == c) return "blocks of one colour share a DOF";
                    seen[bdofs[k]] = c;
                }
    }
    MlhpDevice *d = new MlhpDevice;
    d->st = static_cast<cudaStream_t>(stream);
    d->n = (int)n;
    d->ncolours = ncolours;
    d->max_block = max_block;
    d->colour_ptr.assign(cptr, cptr + ncolours + 1);
    d->grid_n = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 8 * 152);
    std::vector<int> cols32(cols, cols + nnz), bdofs32(bdofs, bdofs + bptr[nblocks]);
    auto fail = [&](const std::string &m) {
        mlhp_device_destroy(d);
        return m;
    };
    cudaError_t e = cudaSuccess;
    if ((e = upload(&d->rowptr, rowptr, (size_t)n + 1, d->st)) != cudaSuccess ||
        (e = upload(&d->cols, cols32.data(), cols32.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->vals, vals, (size_t)nnz, d->st)) != cudaSuccess ||
        (e = upload(&d->bptr, bptr, (size_t)nblocks + 1, d->st)) != cudaSuccess ||
        (e = upload(&d->bdofs, bdofs32.data(), bdofs32.size(), d->st)) != cudaSuccess ||
        (e = upload(&d->fptr, fptr, (size_t)nblocks + 1, d->st)) != cudaSuccess ||
        (e = upload(&d->fac, fac, (size_t)fptr[nblocks], d->st)) != cudaSuccess ||
        (e = upload(&d->jac, jac, (size_t)n, d->st)) != cudaSuccess)
        return fail(std::string("upload: ") + cudaGetErrorString(e));
    for (double **v : {&d->x, &d->r, &d->z, &d->p, &d->q})
        if ((e = cudaMalloc(reinterpret_cast<void **>(v), (size_t)n * sizeof(double))) != cudaSuccess)
            return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    if ((e = cudaMalloc(reinterpret_cast<void **>(&d->partial), kDotGrid * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void **>(&d->scalar), sizeof(double))) != cudaSuccess)
        return fail(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    // the host copies above come from pageable memory owned by the caller: finish them before returning
    if ((e = cudaStreamSynchronize(d->st)) != cudaSuccess) return fail(std::string("upload: ") + cudaGetErrorString(e));
    *out = d;
    return std::string();
}

std::string mlhp_device_apply_K(MlhpDevice *d, const double *x, double *y)
{
    const int64_t warps_per_cta = kThreads / 32;
    const unsigned grid = (unsigned)((d->n + warps_per_cta - 1) / warps_per_cta);
    mlhp_spmv_kernel<<<grid, kThreads, 0, d->st>>>(d->n, d->rowptr, d->cols, d->vals, x, y);
    MLHP_CUDA(cudaGetLastError());
    return std::string();
}

std::string mlhp_device_apply_S(MlhpDevice *d, const double *r, double *z)
{
    mlhp_diag_kernel<<<d->grid_n, kThreads, 0, d->st>>>(d->n, d->jac, r, z);
    MLHP_CUDA(cudaGetLastError());
    const size_t smem = (size_t)d->max_block * sizeof(double);
    const int splits = (d->max_block + kRowsPerCta - 1) / kRowsPerCta;
    for (int c = 0; c < d->ncolours; ++c) {
        const int64_t nb = d->colour_ptr[c + 1] - d->colour_ptr[c];
        if (nb == 0) continue;
        mlhp_block_kernel<<<(unsigned)(nb * splits), kThreads, smem, d->st>>>(d->colour_ptr[c], splits, d->bptr, d->bdofs,
                                                                            d->fptr, d->fac, r, z);
        MLHP_CUDA(cudaGetLastError());
    }
    return std::string();
}

namespace {

std::string dot(MlhpDevice *d, const double *a, const double *b, double *out)
{
    mlhp_dot_partial_kernel<<<kDotGrid, kThreads, 0, d->st>>>(d->n, a, b, d->partial);
    MLHP_CUDA(cudaGetLastError());
    mlhp_dot_final_kernel<<<1, 32, 0, d->st>>>(kDotGrid, d->partial, d->scalar);
    MLHP_CUDA(cudaGetLastError());
    MLHP_CUDA(cudaMemcpyAsync(out, d->scalar, sizeof(double), cudaMemcpyDeviceToHost, d->st));
    MLHP_CUDA(cudaStreamSynchronize(d->st));
    return std::string();
}

}  // namespace

// status: 0 converged, 1 not converged within maxit, 2 breakdown (p.Kp <= 0 or a non-finite scalar).
std::string mlhp_device_pcg(MlhpDevice *d, const double *b, double tol, int maxit, double *u, int *its, double *relres,
                            int *status)
{
    std::string err;
    const size_t bytes = (size_t)d->n * sizeof(double);
    MLHP_CUDA(cudaMemsetAsync(d->x, 0, bytes, d->st));
    MLHP_CUDA(cudaMemcpyAsync(d->r, b, bytes, cudaMemcpyDeviceToDevice, d->st));
    if (!(err = mlhp_device_apply_S(d, d->r, d->z)).empty()) return err;
    MLHP_CUDA(cudaMemcpyAsync(d->p, d->z, bytes, cudaMemcpyDeviceToDevice, d->st));
    double rz = 0.0, zz = 0.0;
    if (!(err = dot(d, d->r, d->z, &rz)).empty()) return err;
    if (!(err = dot(d, d->z, d->z, &zz)).empty()) return err;
    const double zn0 = std::sqrt(zz);
    *its = 0;
    *relres = 1.0;
    *status = 1;
    if (zn0 == 0.0) {
        *status = 0;
        *relres = 0.0;
    }
    for (int it = 1; it <= maxit && *status == 1; ++it) {
        if (!(err = mlhp_device_apply_K(d, d->p, d->q)).empty()) return err;
        double pq = 0.0;
        if (!(err = dot(d, d->p, d->q, &pq)).empty()) return err;
        *its = it;
        if (!(pq > 0.0)) {
            *status = 2;
            break;
        }
        const double a = rz / pq;
        mlhp_xr_kernel<<<d->grid_n, kThreads, 0, d->st>>>(d->n, a, d->p, d->q, d->x, d->r);
        MLHP_CUDA(cudaGetLastError());
        if (!(err = mlhp_device_apply_S(d, d->r, d->z)).empty()) return err;
        double rz_new = 0.0;
        if (!(err = dot(d, d->r, d->z, &rz_new)).empty()) return err;
        if (!(err = dot(d, d->z, d->z, &zz)).empty()) return err;
        const double rel = std::sqrt(zz) / zn0;
        *relres = rel;
        if (!std::isfinite(rel) || !std::isfinite(rz_new)) {
            *status = 2;
            break;
        }
        if (rel <= tol) {
            *status = 0;
            break;
        }
        mlhp_p_kernel<<<d->grid_n, kThreads, 0, d->st>>>(d->n, rz_new / rz, d->z, d->p);
        MLHP_CUDA(cudaGetLastError());
        rz = rz_new;
    }
    MLHP_CUDA(cudaMemcpyAsync(u, d->x, bytes, cudaMemcpyDeviceToDevice, d->st));
    MLHP_CUDA(cudaStreamSynchronize(d->st));
    return std::string();
}

}  // namespace fcm
