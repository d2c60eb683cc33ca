// Additive-Schwarz preconditioner set-up (Algorithm 1 of Jomo et al.,
// arXiv:1809.00828): getBlocks -> extractSubMatrix -> computePseudoInverse ->
// store, with the eigenvalue filter of Sec. 3.2 Eqs. (11)-(13).
//
// Two block rules.  Vertex patches (rule 0): for grid vertex v the free
// functions carried by v and by the edges, faces and cells whose closure
// contains v; in lattice terms the box [p v - (p-1), p v + (p-1)] per axis
// (clipped at the domain).  Element blocks (rule 3, the paper's rule, Sec. 3.2
// "Optimizing the number of blocks"): for each active cell with volume
// fraction eta_T <= eta_bar, every function supported on the cell, the box
// [p c, p c + p]; the free DOFs in no block get Algorithm 1's diagonal
// scaling 1 / K_ll.  A block is stored densely over its box, with zero rows
// and columns for box DOFs that are not free.  Blocks whose contributing cells
// are all uncut (or inactive, or outside the grid) in the same pattern have
// identical matrices and share one stored factor.
//
// Device pipeline per group of equal-size blocks: assemble A_B from the element
// matrices of the cells around the block (8 for a patch, 27 for an element block), pad the diagonal of non-free rows
// with max_i A_ii (which leaves lambda_max and the filtered set unchanged),
// batched symmetric eigensolve (cuSOLVER), filter/invert the eigenvalues,
// F = V diag(lambda+^-1) V^T (cuBLAS batched GEMM), symmetrise, zero the
// non-free rows/columns.  Mixed precision keeps factors whose retained
// condition number exceeds cond_fp64 in FP64 and stores the rest in FP32.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "fcm_device.cuh"

namespace fcm {

namespace {

#define PC_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return std::string(#call) + ": " + cudaGetErrorString(e_);              \
    } while (0)
#define PC_SOLVER(call)                                                                                \
    do {                                                                                               \
        cusolverStatus_t e_ = (call);                                                                  \
        if (e_ != CUSOLVER_STATUS_SUCCESS) return std::string(#call) + ": cusolver status " + std::to_string((int)e_); \
    } while (0)
#define PC_BLAS(call)                                                                                  \
    do {                                                                                               \
        cublasStatus_t e_ = (call);                                                                    \
        if (e_ != CUBLAS_STATUS_SUCCESS) return std::string(#call) + ": cublas status " + std::to_string((int)e_); \
    } while (0)

struct BoxInfo {
    int lo[3], d[3], n;
    int clo[3], chi[3];  // cells whose element matrices contribute to K[B,B]
};

__host__ __device__ inline BoxInfo patch_box(int p, const Grid3 &g, int vx, int vy, int vz)
{
    BoxInfo b;
    const int v[3] = {vx, vy, vz};
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = v[a] * p - (p - 1);
        if (b.lo[a] < 0) b.lo[a] = 0;
        int hi = v[a] * p + (p - 1);
        if (hi > g.M[a] - 1) hi = g.M[a] - 1;
        b.d[a] = hi - b.lo[a] + 1;
    }
    b.n = 3 * b.d[0] * b.d[1] * b.d[2];
    for (int a = 0; a < 3; ++a) {
        b.clo[a] = v[a] - 1;
        b.chi[a] = v[a];
    }
    return b;
}

// Element block of cell (cx, cy, cz): the box [p c, p c + p]; its DOFs on the cell's faces are
// shared with the neighbours, so the 27 cells around contribute to K[B,B].
__host__ __device__ inline BoxInfo element_box(int p, int cx, int cy, int cz)
{
    BoxInfo b;
    const int c[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = p * c[a];
        b.d[a] = p + 1;
        b.clo[a] = c[a] - 1;
        b.chi[a] = c[a] + 1;
    }
    b.n = 3 * (p + 1) * (p + 1) * (p + 1);
    return b;
}

__host__ __device__ inline BoxInfo block_box_of(int rule, int p, const Grid3 &g, int id)
{
    if (rule == FCM_BLOCKS_ELEMENT)
        return element_box(p, id % g.n[0], (id / g.n[0]) % g.n[1], id / (g.n[0] * g.n[1]));
    const int nv0 = g.n[0] + 1, nv1 = g.n[1] + 1;
    return patch_box(p, g, id % nv0, (id / nv0) % nv1, id / (nv0 * nv1));
}

// A_B[i][j] = K[g_i][g_j] summed over the active cells around the block (0 if i or j is not free).
__global__ void assemble_kernel(int p, Grid3 g, int rule, const int *__restrict__ rep, int n, double *__restrict__ A,
                                const double *__restrict__ elem, const int32_t *__restrict__ cell_elem,
                                const uint8_t *__restrict__ mask)
{
    const int b = blockIdx.y;
    const BoxInfo bx = block_box_of(rule, p, g, rep[b]);
    const int q = p + 1, ne = 3 * q * q * q;
    double *Ab = A + (size_t)b * n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        int Li[3], Lj[3];
        const int ni = i / 3, nj = j / 3, ci = i % 3, cj = j % 3;
        Li[0] = bx.lo[0] + ni % bx.d[0];
        Li[1] = bx.lo[1] + (ni / bx.d[0]) % bx.d[1];
        Li[2] = bx.lo[2] + ni / (bx.d[0] * bx.d[1]);
        Lj[0] = bx.lo[0] + nj % bx.d[0];
        Lj[1] = bx.lo[1] + (nj / bx.d[0]) % bx.d[1];
        Lj[2] = bx.lo[2] + nj / (bx.d[0] * bx.d[1]);
        const int64_t gi = 3 * (Li[0] + (int64_t)g.M[0] * (Li[1] + (int64_t)g.M[1] * Li[2])) + ci;
        const int64_t gj = 3 * (Lj[0] + (int64_t)g.M[0] * (Lj[1] + (int64_t)g.M[1] * Lj[2])) + cj;
        double s = 0.0;
        if (mask[gi] && mask[gj]) {
            const int w0 = bx.chi[0] - bx.clo[0] + 1, w1 = bx.chi[1] - bx.clo[1] + 1, w2 = bx.chi[2] - bx.clo[2] + 1;
            for (int t = 0; t < w0 * w1 * w2; ++t) {
                int c[3] = {bx.clo[0] + t % w0, bx.clo[1] + (t / w0) % w1, bx.clo[2] + t / (w0 * w1)};
                if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= g.n[0] || c[1] >= g.n[1] || c[2] >= g.n[2]) continue;
                const int el = cell_elem[c[0] + (int64_t)g.n[0] * (c[1] + (int64_t)g.n[1] * c[2])];
                if (el < 0) continue;
                int li[3], lj[3];
                bool in = true;
                for (int a = 0; a < 3; ++a) {
                    li[a] = Li[a] - p * c[a];
                    lj[a] = Lj[a] - p * c[a];
                    in = in && li[a] >= 0 && li[a] <= p && lj[a] >= 0 && lj[a] <= p;
                }
                if (!in) continue;
                const int Ii = li[0] + q * (li[1] + q * li[2]), Ij = lj[0] + q * (lj[1] + q * lj[2]);
                s += elem[(size_t)el * ne * ne + (size_t)(3 * Ii + ci) * ne + 3 * Ij + cj];
            }
        }
        Ab[e] = s;
    }
}

// Non-free diagonal entries get max_i A_ii: decoupled eigenpairs that neither
// raise lambda_max nor fall under the filter; removed again in finalize.
__global__ void pad_kernel(double *A, int n)
{
    double *Ab = A + (size_t)blockIdx.x * n * n;
    __shared__ double smax[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, Ab[(size_t)i * n + i]);
    smax[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        __syncthreads();
    }
    const double d = smax[0] > 0.0 ? smax[0] : 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bool zero_row = true;
        for (int j = 0; j < n && zero_row; ++j) zero_row = Ab[(size_t)i * n + j] == 0.0;
        if (zero_row) Ab[(size_t)i * n + i] = d;
    }
}

// U = V diag(lambda+^-1), lambda+^-1 = 1/lambda for lambda > eps * lambda_max, else 0
// (eps < 0: every nonzero eigenvalue inverted, the unstabilised inverse).
__global__ void invert_kernel(const double *V, const double *W, double *U, int n, double eps, double *cond,
                              int *nfilt)
{
    const int b = blockIdx.x;
    const double *w = W + (size_t)b * n;
    const double lmax = w[n - 1];  // ascending order
    const double thr = eps * lmax;
    __shared__ double smin[256];
    __shared__ int sfilt[256];
    double lmin = INFINITY;
    int filt = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        if (eps < 0.0 || w[k] > thr) {
            if (w[k] > 0.0) lmin = fmin(lmin, w[k]);
        } else {
            ++filt;
        }
    }
    smin[threadIdx.x] = lmin;
    sfilt[threadIdx.x] = filt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            sfilt[threadIdx.x] += sfilt[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cond[b] = lmax / smin[0];
        nfilt[b] = sfilt[0];
    }
    const double *Vb = V + (size_t)b * n * n;
    double *Ub = U + (size_t)b * n * n;
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        const int k = (int)(e / n);  // column-major: e = i + k n
        const double lk = w[k];
        double inv = 0.0;
        if (eps < 0.0) inv = lk != 0.0 ? 1.0 / lk : 0.0;
        else if (lk > thr) inv = 1.0 / lk;
        Ub[e] = Vb[e] * inv;
    }
}

// F = sym(C) on free rows/columns, 0 elsewhere; written to the FP64 pool.
__global__ void finalize_kernel(const double *C, int n, const int *rep, const int64_t *off, double *pool, int p,
                                Grid3 g, int rule, const uint8_t *mask)
{
    const int b = blockIdx.y;
    const BoxInfo bx = block_box_of(rule, p, g, rep[b]);
    const double *Cb = C + (size_t)b * n * n;
    double *F = pool + off[b];
    const int ld = factor_ld<double>(n);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * ld; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ld), j = (int)(e % ld);
        if (j >= n) {
            F[e] = 0.0;  // row padding
            continue;
        }
        auto gidx = [&](int t) {
            const int nl = t / 3;
            const int x = bx.lo[0] + nl % bx.d[0], y = bx.lo[1] + (nl / bx.d[0]) % bx.d[1], z = bx.lo[2] + nl / (bx.d[0] * bx.d[1]);
            return 3 * (x + (int64_t)g.M[0] * (y + (int64_t)g.M[1] * z)) + t % 3;
        };
        const bool on = mask[gidx(i)] && mask[gidx(j)];
        F[e] = on ? 0.5 * (Cb[(size_t)i + (size_t)j * n] + Cb[(size_t)j + (size_t)i * n]) : 0.0;
    }
}

// FP64 factor (rows padded to factor_ld<double>) -> FP32 factor (rows padded to factor_ld<float>)
__global__ void to_f32_kernel(const double *in, float *out, int n)
{
    const int ldi = factor_ld<double>(n), ldo = factor_ld<float>(n);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * ldo; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldo), j = (int)(e % ldo);
        out[e] = j < n ? (float)in[(size_t)i * ldi + j] : 0.f;
    }
}

// FP64 factor -> double-float pairs: entry j of row i at floats 2 (i ld + j) (hi) and +1 (lo),
// hi = fl32(f), lo = fl32(f - hi); rows of ld = factor_ld<double>(n) entries, padding zero
__global__ void to_ff_kernel(const double *in, float *out, int n)
{
    const int ld = factor_ld<double>(n);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * ld; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % ld);
        const double x = j < n ? in[e] : 0.0;
        const float h = __double2float_rn(x);
        out[2 * e] = h;
        out[2 * e + 1] = __double2float_rn(x - (double)h);
    }
}

// A factor shared by at least this many blocks is applied as a dense product over its blocks
// (GEMM tiles); factors with fewer blocks stream once per block.
constexpr int kGemmMinBlocks = 8;

// Largest retained condition number of an FP32 shared factor applied by the tensor cores (TF32
// three-pass products, ~2^-22 relative): the perturbation stays below ~1e-1 of the smallest retained
// eigenvalue.  Shared factors belong to uncut patches, whose condition numbers are far below it.
constexpr double kTcCondMax = 1e5;

struct FactorInfo {
    int rep;      // representative vertex
    int n;        // box size
    int64_t off;  // offset in the FP64 staging pool (16-byte aligned, rows padded to factor_ld<double>)
    double cond;
    int nfilt;
};

}  // namespace

std::string build_preconditioner(fcm_ctx *C, const fcm_precond_opts &o)
{
    auto t0 = std::chrono::steady_clock::now();
    const HostProblem &hp = C->hp;
    const int p = C->p;
    const Grid3 g = C->g;
    const int nv[3] = {g.n[0] + 1, g.n[1] + 1, g.n[2] + 1};
    const int rule = o.block_rule;
    if (rule != FCM_BLOCKS_VERTEX && rule != FCM_BLOCKS_ELEMENT) return "unknown block rule";
    // block ids: vertices (rule 0) or cells (rule 3)
    const int nid[3] = {rule == FCM_BLOCKS_ELEMENT ? g.n[0] : nv[0], rule == FCM_BLOCKS_ELEMENT ? g.n[1] : nv[1],
                        rule == FCM_BLOCKS_ELEMENT ? g.n[2] : nv[2]};
    const int64_t npatch = (int64_t)nid[0] * nid[1] * nid[2];
    cudaStream_t st = C->stream;
    auto box_has_free = [&](const BoxInfo &bx) {
        for (int t = 0; t < bx.n; ++t) {
            const int nl = t / 3;
            const int x = bx.lo[0] + nl % bx.d[0], y = bx.lo[1] + (nl / bx.d[0]) % bx.d[1], z = bx.lo[2] + nl / (bx.d[0] * bx.d[1]);
            if (hp.mask[3 * (x + (int64_t)g.M[0] * (y + (int64_t)g.M[1] * z)) + t % 3]) return true;
        }
        return false;
    };

    // ---- getBlocks, deduplicated by signature
    std::vector<int> patch_factor(npatch, -1);
    std::vector<FactorInfo> fac;
    std::map<uint64_t, int> regular;
    if (rule == FCM_BLOCKS_ELEMENT) {
        for (int cz = 0; cz < g.n[2]; ++cz)
            for (int cy = 0; cy < g.n[1]; ++cy)
                for (int cx = 0; cx < g.n[0]; ++cx) {
                    const int c = cx + g.n[0] * (cy + g.n[1] * cz);
                    // eta_T is a volume fraction: clamped to 1 against the rounding of its quadrature
                    if (hp.cell_elem[c] < 0 || !(std::min(hp.eta[c], 1.0) <= o.eta_bar)) continue;
                    const BoxInfo bx = element_box(p, cx, cy, cz);
                    if (!box_has_free(bx)) continue;
                    // 2 bits per contributing cell: 0 outside the grid, 1 inactive, 2 uncut; any cut
                    // cell makes the block unique
                    bool cut = false;
                    uint64_t key = 0;
                    for (int t = 0; t < 27; ++t) {
                        const int n3[3] = {cx - 1 + t % 3, cy - 1 + (t / 3) % 3, cz - 1 + t / 9};
                        uint64_t code = 0;
                        if (n3[0] >= 0 && n3[1] >= 0 && n3[2] >= 0 && n3[0] < g.n[0] && n3[1] < g.n[1] && n3[2] < g.n[2]) {
                            const int el = hp.cell_elem[n3[0] + (int64_t)g.n[0] * (n3[1] + (int64_t)g.n[1] * n3[2])];
                            if (el > 0) cut = true;
                            code = el < 0 ? 1 : 2;
                        }
                        key |= code << (2 * t);
                    }
                    int fid;
                    if (!cut) {
                        auto it = regular.find(key);
                        if (it != regular.end()) {
                            patch_factor[c] = it->second;
                            continue;
                        }
                        fid = (int)fac.size();
                        regular[key] = fid;
                    } else {
                        fid = (int)fac.size();
                    }
                    fac.push_back({c, bx.n, 0, 0.0, 0});
                    patch_factor[c] = fid;
                }
    } else
    for (int vz = 0; vz < nv[2]; ++vz)
        for (int vy = 0; vy < nv[1]; ++vy)
            for (int vx = 0; vx < nv[0]; ++vx) {
                const int v = vx + nv[0] * (vy + nv[1] * vz);
                const BoxInfo bx = patch_box(p, g, vx, vy, vz);
                if (!box_has_free(bx)) continue;
                bool cut = false;
                uint64_t key = 0;
                for (int t = 0; t < 8; ++t) {
                    const int c[3] = {vx - 1 + (t & 1), vy - 1 + ((t >> 1) & 1), vz - 1 + ((t >> 2) & 1)};
                    int el = -2;
                    if (c[0] >= 0 && c[1] >= 0 && c[2] >= 0 && c[0] < g.n[0] && c[1] < g.n[1] && c[2] < g.n[2])
                        el = hp.cell_elem[c[0] + (int64_t)g.n[0] * (c[1] + (int64_t)g.n[1] * c[2])];
                    if (el > 0) cut = true;
                    key |= (uint64_t)(el == 0) << t;
                }
                int fid;
                if (!cut) {
                    const int cl[3] = {(vx == 0) + 2 * (vx == g.n[0]), (vy == 0) + 2 * (vy == g.n[1]), (vz == 0) + 2 * (vz == g.n[2])};
                    key |= (uint64_t)(cl[0] + 4 * cl[1] + 16 * cl[2]) << 8;
                    auto it = regular.find(key);
                    if (it != regular.end()) {
                        patch_factor[v] = it->second;
                        continue;
                    }
                    fid = (int)fac.size();
                    regular[key] = fid;
                } else {
                    fid = (int)fac.size();
                }
                fac.push_back({v, bx.n, 0, 0.0, 0});
                patch_factor[v] = fid;
            }

    // ---- group by size, staging offsets
    std::map<int, std::vector<int>> groups;
    for (int f = 0; f < (int)fac.size(); ++f) groups[fac[f].n].push_back(f);
    int64_t total = 0;
    int maxn = 0;
    for (auto &kv : groups)
        for (int f : kv.second) {
            total = (total + 1) / 2 * 2;  // 16-byte alignment
            fac[f].off = total;
            total += (int64_t)kv.first * factor_ld<double>(kv.first);
            maxn = std::max(maxn, kv.first);
        }

    double *stage = nullptr;
    PC_CUDA(cudaMalloc(&stage, sizeof(double) * std::max<int64_t>(total, 1)));
    struct Guard {
        std::vector<void *> ptrs;
        ~Guard()
        {
            for (void *q : ptrs) cudaFree(q);
        }
    } guard;
    guard.ptrs.push_back(stage);

    cusolverDnHandle_t sh = nullptr;
    cublasHandle_t bh = nullptr;
    cusolverDnParams_t params = nullptr;
    PC_SOLVER(cusolverDnCreate(&sh));
    struct HGuard {
        cusolverDnHandle_t s;
        cublasHandle_t b;
        cusolverDnParams_t p;
        ~HGuard()
        {
            if (p) cusolverDnDestroyParams(p);
            if (s) cusolverDnDestroy(s);
            if (b) cublasDestroy(b);
        }
    } hguard{sh, nullptr, nullptr};
    PC_BLAS(cublasCreate(&bh));
    hguard.b = bh;
    PC_SOLVER(cusolverDnCreateParams(&params));
    hguard.p = params;
    PC_SOLVER(cusolverDnSetStream(sh, st));
    PC_BLAS(cublasSetStream(bh, st));

    for (auto &kv : groups) {
        const int n = kv.first;
        const std::vector<int> &ids = kv.second;
        const size_t n2 = (size_t)n * n;
        int chunk = (int)std::max<size_t>(1, std::min<size_t>(ids.size(), (size_t)(1536ull << 20) / (3 * n2 * sizeof(double))));
        double *dA = nullptr, *dU = nullptr, *dC = nullptr, *dW = nullptr, *dcond = nullptr;
        int *dinfo = nullptr, *drep = nullptr, *dfilt = nullptr;
        int64_t *doff = nullptr;
        PC_CUDA(cudaMalloc(&dA, sizeof(double) * n2 * chunk));
        guard.ptrs.push_back(dA);
        PC_CUDA(cudaMalloc(&dU, sizeof(double) * n2 * chunk));
        guard.ptrs.push_back(dU);
        PC_CUDA(cudaMalloc(&dC, sizeof(double) * n2 * chunk));
        guard.ptrs.push_back(dC);
        PC_CUDA(cudaMalloc(&dW, sizeof(double) * n * chunk));
        guard.ptrs.push_back(dW);
        PC_CUDA(cudaMalloc(&dcond, sizeof(double) * chunk));
        guard.ptrs.push_back(dcond);
        PC_CUDA(cudaMalloc(&dinfo, sizeof(int) * chunk));
        guard.ptrs.push_back(dinfo);
        PC_CUDA(cudaMalloc(&dfilt, sizeof(int) * chunk));
        guard.ptrs.push_back(dfilt);
        PC_CUDA(cudaMalloc(&drep, sizeof(int) * chunk));
        guard.ptrs.push_back(drep);
        PC_CUDA(cudaMalloc(&doff, sizeof(int64_t) * chunk));
        guard.ptrs.push_back(doff);

        // eigen workspace: batched API if it accepts this size, else one matrix at a time
        bool batched = true;
        size_t dws = 0, hws = 0;
        if (cusolverDnXsyevBatched_bufferSize(sh, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F,
                                              dA, n, CUDA_R_64F, dW, CUDA_R_64F, &dws, &hws, chunk) != CUSOLVER_STATUS_SUCCESS)
            batched = false;
        if (!batched) {
            PC_SOLVER(cusolverDnXsyevd_bufferSize(sh, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F,
                                                  dA, n, CUDA_R_64F, dW, CUDA_R_64F, &dws, &hws));
        }
        void *dwork = nullptr;
        std::vector<char> hwork(std::max<size_t>(hws, 1));
        PC_CUDA(cudaMalloc(&dwork, std::max<size_t>(dws, 16)));
        guard.ptrs.push_back(dwork);

        std::vector<int> hrep(chunk), hinfo(chunk), hfilt(chunk);
        std::vector<int64_t> hoff(chunk);
        std::vector<double> hcond(chunk);
        for (size_t s0 = 0; s0 < ids.size(); s0 += chunk) {
            const int B = (int)std::min<size_t>(chunk, ids.size() - s0);
            for (int b = 0; b < B; ++b) {
                hrep[b] = fac[ids[s0 + b]].rep;
                hoff[b] = fac[ids[s0 + b]].off;
            }
            PC_CUDA(cudaMemcpyAsync(drep, hrep.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
            PC_CUDA(cudaMemcpyAsync(doff, hoff.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, st));
            const int gx = (int)std::min<int64_t>(((int64_t)n2 + 255) / 256, 64);
            assemble_kernel<<<dim3(gx, B), 256, 0, st>>>(p, g, rule, drep, n, dA, C->d_elem, C->d_cell_elem, C->d_mask);
            pad_kernel<<<B, 256, 0, st>>>(dA, n);
            PC_CUDA(cudaGetLastError());
            if (batched) {
                PC_SOLVER(cusolverDnXsyevBatched(sh, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, dA,
                                                 n, CUDA_R_64F, dW, CUDA_R_64F, dwork, dws, hwork.data(), hws, dinfo, B));
            } else {
                for (int b = 0; b < B; ++b)
                    PC_SOLVER(cusolverDnXsyevd(sh, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F,
                                               dA + n2 * b, n, CUDA_R_64F, dW + (size_t)n * b, CUDA_R_64F, dwork, dws,
                                               hwork.data(), hws, dinfo + b));
            }
            invert_kernel<<<B, 256, 0, st>>>(dA, dW, dU, n, o.eps, dcond, dfilt);
            PC_CUDA(cudaGetLastError());
            const double one = 1.0, zero = 0.0;
            // C = U V^T (column-major): C(i,j) = sum_k U(i,k) V(j,k)
            PC_BLAS(cublasDgemmStridedBatched(bh, CUBLAS_OP_N, CUBLAS_OP_T, n, n, n, &one, dU, n, (long long)n2, dA, n,
                                              (long long)n2, &zero, dC, n, (long long)n2, B));
            finalize_kernel<<<dim3(gx, B), 256, 0, st>>>(dC, n, drep, doff, stage, p, g, rule, C->d_mask);
            PC_CUDA(cudaGetLastError());
            PC_CUDA(cudaMemcpyAsync(hinfo.data(), dinfo, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
            PC_CUDA(cudaMemcpyAsync(hcond.data(), dcond, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
            PC_CUDA(cudaMemcpyAsync(hfilt.data(), dfilt, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
            PC_CUDA(cudaStreamSynchronize(st));
            for (int b = 0; b < B; ++b) {
                if (hinfo[b] != 0) return "eigensolver failed for a block (info " + std::to_string(hinfo[b]) + ")";
                fac[ids[s0 + b]].cond = hcond[b];
                fac[ids[s0 + b]].nfilt = hfilt[b];
            }
        }
    }

    // ---- blocks of each factor, in vertex (or cell) order
    std::vector<std::vector<int>> blocks_of(fac.size());
    for (int64_t v = 0; v < npatch; ++v)
        if (patch_factor[v] >= 0) blocks_of[patch_factor[v]].push_back((int)v);
    std::vector<char> shared(fac.size(), 0);
    for (size_t f = 0; f < fac.size(); ++f) shared[f] = (int)blocks_of[f].size() >= kGemmMinBlocks;

    // ---- final pools.  FP64 form: every factor FP64 (the staging layout is final).  Mixed forms: FP32
    // where the retained condition number is at most cond_fp64; above it double-float pairs (FCM_PREC_MIXED)
    // or FP64 (FCM_PREC_MIXED_FP64); a shared factor above it stays FP64 (the dense product runs in FP32
    // or FP64).  prec: 0 FP64, 1 FP32, 2 double-float.
    const bool mixed = o.precision != FCM_PREC_FP64;
    std::vector<int> prec(fac.size(), 0);
    std::vector<int64_t> off(fac.size(), 0);
    int64_t n64 = 0, n32 = 0, alg_bytes = 0;
    for (size_t f = 0; f < fac.size(); ++f) {
        const int n = fac[f].n;
        if (mixed) prec[f] = fac[f].cond <= o.cond_fp64 ? 1 : (o.precision == FCM_PREC_MIXED && !shared[f] ? 2 : 0);
        if (prec[f] == 1) {
            n32 = (n32 + 3) / 4 * 4;
            off[f] = n32;
            n32 += (int64_t)n * factor_ld<float>(n);
            alg_bytes += (int64_t)n * n * 4;
        } else if (prec[f] == 2) {
            n32 = (n32 + 3) / 4 * 4;
            off[f] = n32;
            n32 += 2 * (int64_t)n * factor_ld<double>(n);
            alg_bytes += (int64_t)n * n * 8;
        } else {
            n64 = (n64 + 1) / 2 * 2;
            off[f] = n64;
            n64 += (int64_t)n * factor_ld<double>(n);
            alg_bytes += (int64_t)n * n * 8;
        }
    }
    if (C->d_f64) cudaFree(C->d_f64);
    if (C->d_f32) cudaFree(C->d_f32);
    C->d_f64 = nullptr;
    C->d_f32 = nullptr;
    if (!mixed) {
        C->d_f64 = stage;  // staging layout is final
        guard.ptrs.erase(std::find(guard.ptrs.begin(), guard.ptrs.end(), (void *)stage));
        for (size_t f = 0; f < fac.size(); ++f) off[f] = fac[f].off;
    } else {
        if (n64 > 0) PC_CUDA(cudaMalloc(&C->d_f64, sizeof(double) * n64));
        if (n32 > 0) PC_CUDA(cudaMalloc(&C->d_f32, sizeof(float) * n32));
        for (size_t f = 0; f < fac.size(); ++f) {
            const int64_t sz = (int64_t)fac[f].n * factor_ld<double>(fac[f].n);
            const int grid = (int)std::min<int64_t>((sz + 255) / 256, 1024);
            if (prec[f] == 1)
                to_f32_kernel<<<grid, 256, 0, st>>>(stage + fac[f].off, C->d_f32 + off[f], fac[f].n);
            else if (prec[f] == 2)
                to_ff_kernel<<<grid, 256, 0, st>>>(stage + fac[f].off, C->d_f32 + off[f], fac[f].n);
            else
                PC_CUDA(cudaMemcpyAsync(C->d_f64 + off[f], stage + fac[f].off, sizeof(double) * sz, cudaMemcpyDeviceToDevice, st));
        }
        PC_CUDA(cudaGetLastError());
        PC_CUDA(cudaStreamSynchronize(st));
    }

    // ---- slots: the blocks of shared factors first (FP32 factors without, then with tensor-core tiles,
    // then FP64), consecutive per factor, then the blocks streaming their own factor.  FP32 shared factors
    // of the mixed form with a retained condition number up to kTcCondMax also get tensor-core tiles
    // (TF32 three-pass products, about 2^-22 relative); the SIMT tiles of the same blocks serve the
    // multi-RHS applies.
    std::vector<char> tc(fac.size(), 0);
    for (size_t f = 0; f < fac.size(); ++f)
        tc[f] = mixed && !o.simt_shared && shared[f] && prec[f] == 1 && schwarz_tc_supported(p) &&
                fac[f].cond <= kTcCondMax;
    std::vector<PatchRec> slots;
    std::vector<int> slot_of(npatch, -1);
    std::vector<int2> tiles32, tiles64;
    std::vector<TcTile> tc_tiles;
    std::vector<int64_t> ft_off(fac.size(), -1);
    int64_t gemm_blocks = 0, ft_floats = 0;
    int n_tiles32_plain = 0;
    for (int pass = 0; pass < 3; ++pass) {
        const int want = pass < 2 ? 1 : 0;
        for (size_t f = 0; f < fac.size(); ++f) {
            if (!shared[f] || prec[f] != want || (want == 1 && tc[f] != (pass == 1))) continue;
            const int nc = schwarz_gemm_cols(p, want);
            const int first = (int)slots.size();
            for (int v : blocks_of[f]) {
                slot_of[v] = (int)slots.size();
                slots.push_back({off[f], v, prec[f]});
            }
            const int cnt = (int)blocks_of[f].size();
            for (int s0 = 0; s0 < cnt; s0 += nc) (want == 1 ? tiles32 : tiles64).push_back(make_int2(first + s0, std::min(nc, cnt - s0)));
            gemm_blocks += cnt;
            if (pass == 1) {
                ft_off[f] = ft_floats;
                ft_floats += schwarz_tc_factor_floats(p, fac[f].n);
                const int nch = (fac[f].n + 15) / 16;
                for (int s0 = 0; s0 < cnt; s0 += 128) tc_tiles.push_back({first + s0, std::min(128, cnt - s0), ft_off[f], nch, 0});
            }
        }
        if (pass == 0) n_tiles32_plain = (int)tiles32.size();
    }
    // factor tiles of the tensor-core products, from the FP64 staging copy
    if (C->d_tc_ft) cudaFree(C->d_tc_ft);
    if (C->d_tc_tiles) cudaFree(C->d_tc_tiles);
    C->d_tc_ft = nullptr;
    C->d_tc_tiles = nullptr;
    if (!tc_tiles.empty()) {
        PC_CUDA(cudaMalloc(&C->d_tc_ft, sizeof(float) * ft_floats));
        PC_CUDA(cudaMalloc(&C->d_tc_tiles, sizeof(TcTile) * tc_tiles.size()));
        PC_CUDA(cudaMemcpyAsync(C->d_tc_tiles, tc_tiles.data(), sizeof(TcTile) * tc_tiles.size(), cudaMemcpyHostToDevice, st));
        for (size_t f = 0; f < fac.size(); ++f)
            if (ft_off[f] >= 0) PC_CUDA(schwarz_tc_factor(p, stage + fac[f].off, fac[f].n, C->d_tc_ft + ft_off[f], st));
        PC_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<int> own_slots[3];  // by storage
    for (size_t f = 0; f < fac.size(); ++f) {
        if (shared[f]) continue;
        for (int v : blocks_of[f]) {
            slot_of[v] = (int)slots.size();
            own_slots[prec[f]].push_back((int)slots.size());
            slots.push_back({off[f], v, prec[f]});
        }
    }
    C->n_blocks = 0;
    C->sapply_fmas = 0;
    for (size_t f = 0; f < fac.size(); ++f) {
        C->n_blocks += (int64_t)blocks_of[f].size();
        C->sapply_fmas += (int64_t)blocks_of[f].size() * fac[f].n * fac[f].n;
    }
    // work items of the streamed factors, (slot, first row): the three storages interleaved by relative
    // position, so that every part of a launch mixes FP64-pipe, FP32-pipe and DRAM-bound work
    auto make_items = [&](int rows, std::vector<int2> &items) {
        std::vector<int2> lists[3];
        for (int k = 0; k < 3; ++k)
            for (int sl : own_slots[k])
                for (int r0 = 0; r0 < fac[patch_factor[slots[sl].v]].n; r0 += rows) lists[k].push_back(make_int2(sl, r0));
        items.clear();
        size_t pos[3] = {0, 0, 0};
        for (;;) {
            int best = -1;
            double key = 2.0;
            for (int l = 0; l < 3; ++l)
                if (pos[l] < lists[l].size()) {
                    const double k = (pos[l] + 0.5) / (double)lists[l].size();
                    if (k < key) {
                        key = k;
                        best = l;
                    }
                }
            if (best < 0) break;
            items.push_back(lists[best][pos[best]++]);
        }
    };
    const bool rows_kernel = schwarz_uses_rows_kernel(p);
    std::vector<int2> col_items;
    make_items(schwarz_col_rows(p), col_items);
    // candidates: rows per row item (p = 3: 64, 128, the whole block), each with the shared-factor products
    // after the streamed factors or beside them on a second stream
    struct Cand {
        int rows, conc;
    };
    std::vector<Cand> cand;
    const int whole = (maxn + 31) / 32 * 32;
    std::vector<int> row_opts = rows_kernel ? std::vector<int>{128, 64, whole} : std::vector<int>{0};
    if (o.fixed_tiles == 1 || o.fixed_tiles == 2) {
        cand.push_back({row_opts[0], o.fixed_tiles - 1});
    } else {
        for (int conc = 0; conc < 2; ++conc)
            for (int ro : row_opts) cand.push_back({ro, conc});
    }
    std::vector<int2> row_items;
    size_t max_rows_items = 0;
    for (const auto &c2 : cand)
        if (rows_kernel) {
            make_items(c2.rows, row_items);
            max_rows_items = std::max(max_rows_items, row_items.size());
        }

    // ---- device arrays: slots, slot_of, [row items | column items | tiles], Zb
    auto reup = [&](auto **d, size_t count) -> cudaError_t {
        if (*d) cudaFree(*d);
        *d = nullptr;
        return cudaMalloc((void **)d, sizeof(**d) * std::max<size_t>(count, 1));
    };
    PC_CUDA(reup(&C->d_slots, slots.size()));
    PC_CUDA(reup(&C->d_slot_of, slot_of.size()));
    const size_t n_tiles = tiles32.size() + tiles64.size();
    PC_CUDA(reup(&C->d_items, max_rows_items + col_items.size() + n_tiles));
    const int zs = (maxn + 7) / 8 * 8;
    // the sum kernel addresses Zb in 32-bit float offsets
    if (2 * (int64_t)slots.size() * zs >= ((int64_t)1 << 31)) return "too many blocks for the block-product buffer";
    PC_CUDA(reup(&C->d_zb, (size_t)slots.size() * zs));
    PC_CUDA(cudaMemcpyAsync(C->d_slots, slots.data(), sizeof(PatchRec) * slots.size(), cudaMemcpyHostToDevice, st));
    // the pair format stores FP32 slots as floats: their slot_of entries carry the flag the sum kernel reads
    if (mixed)
        for (int64_t v = 0; v < npatch; ++v)
            if (slot_of[v] >= 0 && slots[slot_of[v]].prec == 1) slot_of[v] |= 1 << 30;
    PC_CUDA(cudaMemcpyAsync(C->d_slot_of, slot_of.data(), sizeof(int) * slot_of.size(), cudaMemcpyHostToDevice, st));
    int2 *d_col = C->d_items + max_rows_items, *d_tiles = d_col + col_items.size();
    PC_CUDA(cudaMemcpyAsync(d_col, col_items.data(), sizeof(int2) * col_items.size(), cudaMemcpyHostToDevice, st));
    std::vector<int2> tiles(tiles32);
    tiles.insert(tiles.end(), tiles64.begin(), tiles64.end());
    PC_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st));
    if (!C->d_err) PC_CUDA(cudaMalloc(&C->d_err, sizeof(int)));
    PC_CUDA(cudaMemsetAsync(C->d_err, 0, sizeof(int), st));
    if (!C->side) {
        PC_CUDA(cudaStreamCreateWithFlags(&C->side, cudaStreamNonBlocking));
        PC_CUDA(cudaEventCreateWithFlags(&C->ev_fork, cudaEventDisableTiming));
        PC_CUDA(cudaEventCreateWithFlags(&C->ev_join, cudaEventDisableTiming));
    }
    PC_CUDA(schwarz_prepare(p));
    if (C->d_mzb) cudaFree(C->d_mzb);  // multi-RHS products: sized again by the next multi-RHS solve
    C->d_mzb = nullptr;
    C->m_nr = 0;

    SchwarzPlan plan = {};
    plan.g = g;
    plan.rule = rule;
    plan.zs = zs;
    plan.nslots = (int64_t)slots.size();
    plan.slots = C->d_slots;
    plan.slot_of = C->d_slot_of;
    plan.row_items = C->d_items;
    plan.col_items = d_col;
    plan.n_col_items = (int)col_items.size();
    plan.tiles = d_tiles;
    plan.n_tiles32 = (int)tiles32.size();
    plan.n_tiles64 = (int)tiles64.size();
    plan.n_tiles32_plain = n_tiles32_plain;
    plan.tc_tiles = C->d_tc_tiles;
    plan.n_tc_tiles = (int)tc_tiles.size();
    plan.tc_ft = C->d_tc_ft;
    plan.zb = C->d_zb;
    plan.pairs = mixed ? 1 : 0;
    plan.err = C->d_err;
    plan.wait_tries = C->wait_tries;
    plan.side = C->side;
    plan.ev_fork = C->ev_fork;
    plan.ev_join = C->ev_join;
    plan.jac = nullptr;  // set below, with the diagonal part
    auto configure = [&](const Cand &c2) -> cudaError_t {
        plan.concurrent = c2.conc;
        plan.rows = c2.rows;
        plan.n_row_items = 0;
        if (rows_kernel) {
            make_items(c2.rows, row_items);
            plan.n_row_items = (int)row_items.size();
            return cudaMemcpyAsync(C->d_items, row_items.data(), sizeof(int2) * row_items.size(), cudaMemcpyHostToDevice, st);
        }
        return cudaSuccess;
    };
    // ---- Algorithm 1's diagonal part: 1 / K_ll for the free DOFs in no block
    std::vector<uint8_t> covered(hp.nlat, 0);
    for (int64_t v = 0; v < npatch; ++v) {
        if (patch_factor[v] < 0) continue;
        const BoxInfo bx = block_box_of(rule, p, g, (int)v);
        for (int t = 0; t < bx.n; ++t) {
            const int nl = t / 3;
            const int x = bx.lo[0] + nl % bx.d[0], y = bx.lo[1] + (nl / bx.d[0]) % bx.d[1], z = bx.lo[2] + nl / (bx.d[0] * bx.d[1]);
            covered[3 * (x + (int64_t)g.M[0] * (y + (int64_t)g.M[1] * z)) + t % 3] = 1;
        }
    }
    int64_t nuncovered = 0;
    for (int64_t l = 0; l < hp.nlat; ++l) nuncovered += hp.mask[l] && !covered[l];
    if (C->d_jac) cudaFree(C->d_jac);
    C->d_jac = nullptr;
    C->n_jacobi = nuncovered;
    if (nuncovered > 0) {
        const std::vector<double> &diag = hp.kdiag;  // K_ll, tabulated at set-up
        std::vector<double> jac(hp.nlat, 0.0);
        for (int64_t l = 0; l < hp.nlat; ++l)
            if (hp.mask[l] && !covered[l] && diag[l] > 0.0) jac[l] = 1.0 / diag[l];
        PC_CUDA(cudaMalloc(&C->d_jac, sizeof(double) * hp.nlat));
        PC_CUDA(cudaMemcpyAsync(C->d_jac, jac.data(), sizeof(double) * hp.nlat, cudaMemcpyHostToDevice, st));
        PC_CUDA(cudaStreamSynchronize(st));
    }
    plan.jac = C->d_jac;

    // ---- autotuner: S applied to the load vector (a field with the problem's own structure) into the z
    // work vector, 2 warm-up and 5 timed applies per candidate on the context's stream; S r does not depend
    // on the choice
    for (int k = 0; k < 8; ++k) C->tune_seconds[k] = 0.0;
    size_t best_k = 0;
    if (cand.size() > 1) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        PC_CUDA(cudaEventCreate(&e0));
        PC_CUDA(cudaEventCreate(&e1));
        double best = 1e300;
        std::string fail;
        for (size_t k = 0; k < cand.size() && k < 8; ++k) {
            if (configure(cand[k]) != cudaSuccess) {
                fail = "autotune upload";
                break;
            }
            for (int w = 0; w < 2; ++w) launch_schwarz_apply(p, g, C->d_rhs, C->d_z, C->d_f64, C->d_f32, plan, nullptr, st);
            cudaEventRecord(e0, st);
            for (int w = 0; w < 5; ++w) launch_schwarz_apply(p, g, C->d_rhs, C->d_z, C->d_f64, C->d_f32, plan, nullptr, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                fail = "autotune run";
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            C->tune_seconds[k] = ms / 5e3;
            if (C->tune_seconds[k] < best) {
                best = C->tune_seconds[k];
                best_k = k;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!fail.empty()) return fail + ": " + cudaGetErrorString(cudaGetLastError());
    }
    PC_CUDA(configure(cand[best_k]));
    PC_CUDA(cudaStreamSynchronize(st));
    C->plan = plan;
    C->n_ff_factors = 0;
    for (size_t f = 0; f < fac.size(); ++f) C->n_ff_factors += prec[f] == 2;
    C->n_gemm_blocks = gemm_blocks;
    C->n_factors = (int64_t)fac.size();
    C->factor_bytes = alg_bytes;  // n^2 entries per factor (the stored rows carry < 16 bytes of padding)
    C->max_block = maxn;
    C->n_fp32_factors = 0;
    C->max_cond = 0.0;
    for (size_t f = 0; f < fac.size(); ++f) {
        C->n_fp32_factors += prec[f] == 1;
        if (std::isfinite(fac[f].cond)) C->max_cond = std::max(C->max_cond, fac[f].cond);
    }
    C->have_precond = true;
    C->precond_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return std::string();
}

}  // namespace fcm
