// Learned coarse correction: a 3D U-Net on the cell grid with hand-written
// CUDA kernels for inference and training (BF16 weights, FP32 activations
// and accumulation), the restriction / prolongation between lattice DOFs
// and cells, and Adam.  The paper's Additive-Schwarz preconditioner has no
// coarse space (Sec. 6 lists this as a limitation of local preconditioners);
// this network supplies one, used by fcm_fpcg_solve.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "fcm_device.cuh"

namespace fcm {
namespace {

constexpr int kConvThreads = 128;
constexpr int kCiChunk = 16;

// out[b][co][p] = bias[co] + sum_{ci, tap} w[co][ci][tap] in[b][ci][p + off(tap)], zero padding.
// One thread per output voxel and COB output channels; a chunk of weights is staged in shared memory.
template <int COB>
__global__ void __launch_bounds__(kConvThreads)
    conv3_fwd_kernel(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
                     float *__restrict__ out, int Cin, int Cout, int nx, int ny, int nz)
{
    __shared__ float ws[COB][kCiChunk][27];
    const int S = nx * ny * nz;
    const int b = blockIdx.z;
    const int co0 = blockIdx.y * COB;
    const int p = blockIdx.x * kConvThreads + threadIdx.x;
    const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
    float acc[COB];
#pragma unroll
    for (int k = 0; k < COB; ++k) acc[k] = (bias && co0 + k < Cout) ? bias[co0 + k] : 0.f;
    const float *inb = in + (size_t)b * Cin * S;
    for (int ci0 = 0; ci0 < Cin; ci0 += kCiChunk) {
        const int nci = min(kCiChunk, Cin - ci0);
        __syncthreads();
        for (int e = threadIdx.x; e < COB * kCiChunk * 27; e += kConvThreads) {
            const int k = e / (kCiChunk * 27), r = e % (kCiChunk * 27), ci = r / 27, t = r % 27;
            ws[k][ci][t] = (co0 + k < Cout && ci < nci) ? __bfloat162float(w[((size_t)(co0 + k) * Cin + ci0 + ci) * 27 + t]) : 0.f;
        }
        __syncthreads();
        if (p < S) {
            for (int ci = 0; ci < nci; ++ci) {
                const float *src = inb + (size_t)(ci0 + ci) * S;
                for (int dz = -1; dz <= 1; ++dz) {
                    const int zz = z + dz;
                    if (zz < 0 || zz >= nz) continue;
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int yy = y + dy;
                        if (yy < 0 || yy >= ny) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int xx = x + dx;
                            if (xx < 0 || xx >= nx) continue;
                            const float v = src[(zz * ny + yy) * nx + xx];
                            const int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
#pragma unroll
                            for (int k = 0; k < COB; ++k) acc[k] = fmaf(ws[k][ci][t], v, acc[k]);
                        }
                    }
                }
            }
        }
    }
    if (p < S)
#pragma unroll
        for (int k = 0; k < COB; ++k)
            if (co0 + k < Cout) out[((size_t)b * Cout + co0 + k) * S + p] = acc[k];
}

// gw[co][ci][tap] += sum_{b,p} gout[b][co][p] in[b][ci][p + off(tap)];  gb[co] += sum gout (ci == 0 block).
// One block per (ci, co); fixed-order block reduction (deterministic).
__global__ void __launch_bounds__(256)
    conv3_wgrad_kernel(const float *__restrict__ in, const float *__restrict__ gout, int Cin, int Cout, int B, int nx,
                       int ny, int nz, float *__restrict__ gw, float *__restrict__ gb)
{
    __shared__ float red[28][256];
    const int ci = blockIdx.x, co = blockIdx.y;
    const int S = nx * ny * nz;
    float acc[28];
#pragma unroll
    for (int t = 0; t < 28; ++t) acc[t] = 0.f;
    for (int b = 0; b < B; ++b) {
        const float *src = in + ((size_t)b * Cin + ci) * S;
        const float *go = gout + ((size_t)b * Cout + co) * S;
        for (int p = threadIdx.x; p < S; p += blockDim.x) {
            const float g = go[p];
            const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
            acc[27] += g;
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int zz = z + dz, yy = y + dy, xx = x + dx;
                        const bool ok = zz >= 0 && zz < nz && yy >= 0 && yy < ny && xx >= 0 && xx < nx;
                        const float v = ok ? src[(zz * ny + yy) * nx + xx] : 0.f;
                        acc[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = fmaf(g, v, acc[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]);
                    }
        }
    }
#pragma unroll
    for (int t = 0; t < 28; ++t) red[t][threadIdx.x] = acc[t];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int t = 0; t < 28; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 27) gw[((size_t)co * Cin + ci) * 27 + threadIdx.x] += red[threadIdx.x][0];
    if (threadIdx.x == 27 && ci == 0) gb[co] += red[27][0];
}

// wt[ci][co][26 - t] = w[co][ci][t] (the weights of the data-gradient convolution)
__global__ void transpose_flip_kernel(const __nv_bfloat16 *w, __nv_bfloat16 *wt, int Cin, int Cout)
{
    const int64_t n = (int64_t)Cin * Cout * 27;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e % 27);
        const int64_t r = e / 27;
        const int ci = (int)(r % Cin), co = (int)(r / Cin);
        wt[((int64_t)ci * Cout + co) * 27 + (26 - t)] = w[e];
    }
}

__global__ void relu_fwd_kernel(const float *a, float *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = fmaxf(a[i], 0.f);
}

__global__ void relu_bwd_kernel(const float *pre, const float *g, float *gpre, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gpre[i] = pre[i] > 0.f ? g[i] : 0.f;
}

// coarse[bc][Z][Y][X] = mean of the 8 children (2x average pooling); bc = batch * channels
__global__ void pool_fwd_kernel(const float *fine, float *coarse, int64_t bc, int nx, int ny, int nz)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int64_t n = bc * cx * cy * cz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(e % cx), Y = (int)((e / cx) % cy), Z = (int)((e / ((int64_t)cx * cy)) % cz);
        const int64_t c = e / ((int64_t)cx * cy * cz);
        const float *f = fine + c * (int64_t)nx * ny * nz;
        float s = 0.f;
        for (int k = 0; k < 8; ++k) s += f[((2 * Z + (k >> 2)) * ny + 2 * Y + ((k >> 1) & 1)) * nx + 2 * X + (k & 1)];
        coarse[e] = 0.125f * s;
    }
}

// gfine += gcoarse / 8 at every child
__global__ void pool_bwd_kernel(const float *gcoarse, float *gfine, int64_t bc, int nx, int ny, int nz)
{
    const int64_t n = bc * (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % nx), y = (int)((e / nx) % ny), z = (int)((e / ((int64_t)nx * ny)) % nz);
        const int64_t c = e / ((int64_t)nx * ny * nz);
        gfine[e] += 0.125f * gcoarse[((c * (nz / 2) + z / 2) * (ny / 2) + y / 2) * (nx / 2) + x / 2];
    }
}

// dst[b][c0 + c][p] = nearest-upsampled src[b][c][p/2]  (src at half resolution, C channels)
__global__ void up_fwd_kernel(const float *src, float *dst, int B, int C, int Cdst, int c0, int nx, int ny, int nz)
{
    const int64_t S = (int64_t)nx * ny * nz, n = (int64_t)B * C * S;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % S, bc = e / S;
        const int c = (int)(bc % C), b = (int)(bc / C);
        const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((int64_t)nx * ny));
        dst[((int64_t)b * Cdst + c0 + c) * S + p] =
            src[(((int64_t)b * C + c) * (nz / 2) + z / 2) * (ny / 2) * (nx / 2) + (y / 2) * (nx / 2) + x / 2];
    }
}

// gsrc[b][c][P] (=|+=) sum over the 8 children of gdst[b][c0 + c][.]
__global__ void up_bwd_kernel(const float *gdst, float *gsrc, int B, int C, int Cdst, int c0, int nx, int ny, int nz,
                              int accumulate)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int64_t S = (int64_t)nx * ny * nz, Sc = (int64_t)cx * cy * cz, n = (int64_t)B * C * Sc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t P = e % Sc, bc = e / Sc;
        const int c = (int)(bc % C), b = (int)(bc / C);
        const int X = (int)(P % cx), Y = (int)((P / cx) % cy), Z = (int)(P / ((int64_t)cx * cy));
        const float *g = gdst + ((int64_t)b * Cdst + c0 + c) * S;
        float s = 0.f;
        for (int k = 0; k < 8; ++k) s += g[((2 * Z + (k >> 2)) * ny + 2 * Y + ((k >> 1) & 1)) * nx + 2 * X + (k & 1)];
        gsrc[e] = accumulate ? gsrc[e] + s : s;
    }
}

// dst[b][c0 + c][p] (=|+=) src[b][cs0 + c][p] for c < C
__global__ void chan_copy_kernel(const float *src, int Csrc, int cs0, float *dst, int Cdst, int c0, int B, int C,
                                 int64_t S, int accumulate)
{
    const int64_t n = (int64_t)B * C * S;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % S, bc = e / S;
        const int c = (int)(bc % C), b = (int)(bc / C);
        const float v = src[((int64_t)b * Csrc + cs0 + c) * S + p];
        float &d = dst[((int64_t)b * Cdst + c0 + c) * S + p];
        d = accumulate ? d + v : v;
    }
}

__global__ void fill_kernel(float *a, int64_t n, float v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

__global__ void to_bf16_kernel(const float *a, __nv_bfloat16 *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// Adam (Kingma & Ba, 2015) with bias correction.
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int blocks_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

}  // namespace
}  // namespace fcm

using namespace fcm;

struct UConv {
    int cin, cout;
    int64_t woff, boff;  // offsets in the parameter arrays
};

struct fcm_unet {
    cudaStream_t stream = nullptr;
    int in_ch = 0, out_ch = 0, base = 0, levels = 0;
    std::vector<UConv> conv;  // enc (2 per level), dec (2 per level above the bottom, top-down), out
    int64_t nparam = 0, max_w = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *w16 = nullptr, *wt16 = nullptr;
    // activations for the current shape
    int B = 0, n[3] = {0, 0, 0};
    std::vector<float *> act;  // owned buffers
    const float *input = nullptr;
    float *output = nullptr;
    // per level l
    std::vector<float *> xin, ea, eA, eb, eB, cat, da, dA, db, dB;
    std::vector<float *> gxin, gea, geA, geb, geB, gcat, gda, gdA, gdb, gdB;
    std::vector<int64_t> S;   // voxels per level
    std::vector<int> dim;     // nx >> l etc. (cube not required: stored per axis below)
    std::vector<int> lx, ly, lz;
    // identity of this network and of its activation buffers, for graphs that captured its launches
    uint64_t serial = 0, act_gen = 0;
    int ch(int l) const { return std::min(base << l, 4 * base); }
    int enc_a(int l) const { return 2 * l; }
    int enc_b(int l) const { return 2 * l + 1; }
    int dec_a(int l) const { return 2 * levels + 2 * (levels - 2 - l); }
    int dec_b(int l) const { return dec_a(l) + 1; }
    int out_layer() const { return (int)conv.size() - 1; }
};

namespace {

void free_acts(fcm_unet *N)
{
    for (float *p : N->act) cudaFree(p);
    N->act.clear();
    N->B = 0;
}

cudaError_t falloc(fcm_unet *N, float **p, int64_t count)
{
    cudaError_t e = cudaMalloc((void **)p, sizeof(float) * std::max<int64_t>(count, 1));
    if (e == cudaSuccess) N->act.push_back(*p);
    return e;
}

cudaError_t ensure_shape(fcm_unet *N, int B, int nx, int ny, int nz)
{
    if (N->B == B && N->n[0] == nx && N->n[1] == ny && N->n[2] == nz) return cudaSuccess;
    free_acts(N);
    ++N->act_gen;
    const int L = N->levels;
    auto resize = [&](std::vector<float *> &v) { v.assign(L, nullptr); };
    for (auto *v : {&N->xin, &N->ea, &N->eA, &N->eb, &N->eB, &N->cat, &N->da, &N->dA, &N->db, &N->dB, &N->gxin, &N->gea,
                    &N->geA, &N->geb, &N->geB, &N->gcat, &N->gda, &N->gdA, &N->gdb, &N->gdB})
        resize(*v);
    N->S.assign(L, 0);
    N->lx.assign(L, 0);
    N->ly.assign(L, 0);
    N->lz.assign(L, 0);
    cudaError_t e;
    for (int l = 0; l < L; ++l) {
        N->lx[l] = nx >> l;
        N->ly[l] = ny >> l;
        N->lz[l] = nz >> l;
        const int64_t S = (int64_t)N->lx[l] * N->ly[l] * N->lz[l];
        N->S[l] = S;
        const int c = N->ch(l);
        const int64_t bs = (int64_t)B * c * S;
        if (l > 0) {
            if ((e = falloc(N, &N->xin[l], (int64_t)B * N->ch(l - 1) * S)) != cudaSuccess) return e;
            if ((e = falloc(N, &N->gxin[l], (int64_t)B * N->ch(l - 1) * S)) != cudaSuccess) return e;
        }
        for (auto pr : {std::make_pair(&N->ea, &N->gea), std::make_pair(&N->eA, &N->geA), std::make_pair(&N->eb, &N->geb),
                        std::make_pair(&N->eB, &N->geB)}) {
            if ((e = falloc(N, &(*pr.first)[l], bs)) != cudaSuccess) return e;
            if ((e = falloc(N, &(*pr.second)[l], bs)) != cudaSuccess) return e;
        }
        if (l <= L - 2) {
            const int64_t cs = (int64_t)B * (N->ch(l + 1) + c) * S;
            if ((e = falloc(N, &N->cat[l], cs)) != cudaSuccess) return e;
            if ((e = falloc(N, &N->gcat[l], cs)) != cudaSuccess) return e;
            for (auto pr : {std::make_pair(&N->da, &N->gda), std::make_pair(&N->dA, &N->gdA), std::make_pair(&N->db, &N->gdb),
                            std::make_pair(&N->dB, &N->gdB)}) {
                if ((e = falloc(N, &(*pr.first)[l], bs)) != cudaSuccess) return e;
                if ((e = falloc(N, &(*pr.second)[l], bs)) != cudaSuccess) return e;
            }
        }
    }
    N->B = B;
    N->n[0] = nx;
    N->n[1] = ny;
    N->n[2] = nz;
    return cudaSuccess;
}

void conv_fwd(fcm_unet *N, int layer, const float *in, float *out, int l)
{
    const UConv &c = N->conv[layer];
    const int64_t S = N->S[l];
    const dim3 blk(kConvThreads);
    if (c.cout <= 4) {
        const dim3 grid((unsigned)((S + kConvThreads - 1) / kConvThreads), (c.cout + 3) / 4, N->B);
        conv3_fwd_kernel<4><<<grid, blk, 0, N->stream>>>(in, N->w16 + c.woff, N->w + c.boff, out, c.cin, c.cout, N->lx[l],
                                                         N->ly[l], N->lz[l]);
    } else {
        const dim3 grid((unsigned)((S + kConvThreads - 1) / kConvThreads), (c.cout + 15) / 16, N->B);
        conv3_fwd_kernel<16><<<grid, blk, 0, N->stream>>>(in, N->w16 + c.woff, N->w + c.boff, out, c.cin, c.cout,
                                                          N->lx[l], N->ly[l], N->lz[l]);
    }
}

// weight gradients of `layer` and, if gin != NULL, the data gradient (overwritten)
void conv_bwd(fcm_unet *N, int layer, const float *in, const float *gout, float *gin, int l)
{
    const UConv &c = N->conv[layer];
    conv3_wgrad_kernel<<<dim3(c.cin, c.cout), 256, 0, N->stream>>>(in, gout, c.cin, c.cout, N->B, N->lx[l], N->ly[l],
                                                                     N->lz[l], N->g + c.woff, N->g + c.boff);
    if (!gin) return;
    const int64_t nw = (int64_t)c.cin * c.cout * 27;
    transpose_flip_kernel<<<blocks_for(nw), 256, 0, N->stream>>>(N->w16 + c.woff, N->wt16, c.cin, c.cout);
    const int64_t S = N->S[l];
    const dim3 grid((unsigned)((S + kConvThreads - 1) / kConvThreads), (c.cin + 15) / 16, N->B);
    if (c.cin <= 4) {
        const dim3 g4((unsigned)((S + kConvThreads - 1) / kConvThreads), (c.cin + 3) / 4, N->B);
        conv3_fwd_kernel<4><<<g4, kConvThreads, 0, N->stream>>>(gout, N->wt16, nullptr, gin, c.cout, c.cin, N->lx[l],
                                                                N->ly[l], N->lz[l]);
    } else {
        conv3_fwd_kernel<16><<<grid, kConvThreads, 0, N->stream>>>(gout, N->wt16, nullptr, gin, c.cout, c.cin, N->lx[l],
                                                                   N->ly[l], N->lz[l]);
    }
}

void relu_f(fcm_unet *N, const float *a, float *b, int64_t n) { relu_fwd_kernel<<<blocks_for(n), 256, 0, N->stream>>>(a, b, n); }
void relu_b(fcm_unet *N, const float *pre, const float *g, float *gp, int64_t n)
{
    relu_bwd_kernel<<<blocks_for(n), 256, 0, N->stream>>>(pre, g, gp, n);
}

uint64_t splitmix(uint64_t &s)
{
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}


}  // namespace


namespace fcm {
void unet_identity(const fcm_unet *N, uint64_t *serial, uint64_t *gen)
{
    *serial = N ? N->serial : 0;
    *gen = N ? N->act_gen : 0;
}

cudaStream_t unet_set_stream(fcm_unet *N, cudaStream_t s)
{
    cudaStream_t old = N->stream;
    N->stream = s;
    return old;
}
}  // namespace fcm

#define UN_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            fcm_unet_last_error() = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return e_ == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;                  \
        }                                                                                     \
    } while (0)

extern "C" {

fcm_status fcm_unet_create(const fcm_unet_desc *d, void *cuda_stream, fcm_unet **out)
{
    if (!d || !out || d->in_ch < 1 || d->out_ch < 1 || d->base < 1 || d->base > 256 || d->levels < 1 ||
        d->levels > 6) {
        fcm_unet_last_error() = "fcm_unet_create: invalid description";
        return FCM_EINVAL;
    }
    *out = nullptr;
    fcm_unet *N = new fcm_unet();
    static std::atomic<uint64_t> next_serial{1};
    N->serial = next_serial++;
    N->stream = (cudaStream_t)cuda_stream;
    N->in_ch = d->in_ch;
    N->out_ch = d->out_ch;
    N->base = d->base;
    N->levels = d->levels;
    const int L = d->levels;
    for (int l = 0; l < L; ++l) {
        N->conv.push_back({l == 0 ? d->in_ch : N->ch(l - 1), N->ch(l), 0, 0});
        N->conv.push_back({N->ch(l), N->ch(l), 0, 0});
    }
    for (int l = L - 2; l >= 0; --l) {
        N->conv.push_back({N->ch(l + 1) + N->ch(l), N->ch(l), 0, 0});
        N->conv.push_back({N->ch(l), N->ch(l), 0, 0});
    }
    N->conv.push_back({N->ch(0), d->out_ch, 0, 0});
    int64_t off = 0;
    for (UConv &c : N->conv) {
        c.woff = off;
        off += (int64_t)c.cout * c.cin * 27;
        c.boff = off;
        off += c.cout;
        N->max_w = std::max<int64_t>(N->max_w, (int64_t)c.cout * c.cin * 27);
    }
    N->nparam = off;
    // Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases; the output layer 10x smaller
    std::vector<float> h(off, 0.f);
    uint64_t s = d->seed;
    for (size_t k = 0; k < N->conv.size(); ++k) {
        const UConv &c = N->conv[k];
        float bound = std::sqrt(6.0f / (c.cin * 27.0f));
        if ((int)k == N->out_layer()) bound *= 0.1f;
        for (int64_t i = 0; i < (int64_t)c.cout * c.cin * 27; ++i) {
            const double u = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
            h[c.woff + i] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    auto fail = [&](cudaError_t e) {
        fcm_unet_last_error() = std::string("fcm_unet_create: ") + cudaGetErrorString(e);
        fcm_unet_destroy(N);
        return e == cudaErrorMemoryAllocation ? FCM_ENOMEM : FCM_ECUDA;
    };
    cudaError_t e;
    float **arrs[] = {&N->w, &N->g, &N->m, &N->v};
    for (float **a : arrs) {
        if ((e = cudaMalloc((void **)a, sizeof(float) * off)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(*a, 0, sizeof(float) * off, N->stream)) != cudaSuccess) return fail(e);
    }
    if ((e = cudaMalloc((void **)&N->w16, sizeof(__nv_bfloat16) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc((void **)&N->wt16, sizeof(__nv_bfloat16) * N->max_w)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(N->w, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice, N->stream)) != cudaSuccess)
        return fail(e);
    to_bf16_kernel<<<blocks_for(off), 256, 0, N->stream>>>(N->w, N->w16, off);
    if ((e = cudaStreamSynchronize(N->stream)) != cudaSuccess) return fail(e);
    *out = N;
    return FCM_OK;
}

fcm_status fcm_unet_params(const fcm_unet *N, int64_t *count)
{
    if (!N || !count) return FCM_EINVAL;
    *count = N->nparam;
    return FCM_OK;
}

fcm_status fcm_unet_get(fcm_unet *N, float *w_host, float *g_host)
{
    if (!N || !w_host) return FCM_EINVAL;
    UN_CUDA(cudaMemcpyAsync(w_host, N->w, sizeof(float) * N->nparam, cudaMemcpyDeviceToHost, N->stream));
    if (g_host) UN_CUDA(cudaMemcpyAsync(g_host, N->g, sizeof(float) * N->nparam, cudaMemcpyDeviceToHost, N->stream));
    UN_CUDA(cudaStreamSynchronize(N->stream));
    return FCM_OK;
}

fcm_status fcm_unet_set(fcm_unet *N, const float *w_host)
{
    if (!N || !w_host) return FCM_EINVAL;
    UN_CUDA(cudaMemcpyAsync(N->w, w_host, sizeof(float) * N->nparam, cudaMemcpyHostToDevice, N->stream));
    to_bf16_kernel<<<blocks_for(N->nparam), 256, 0, N->stream>>>(N->w, N->w16, N->nparam);
    UN_CUDA(cudaStreamSynchronize(N->stream));
    return FCM_OK;
}

fcm_status fcm_unet_forward(fcm_unet *N, const float *in, int B, int nx, int ny, int nz, float *out)
{
    if (!N || !in || !out || B < 1) return FCM_EINVAL;
    const int div = 1 << (N->levels - 1);
    if (nx < div || ny < div || nz < div || nx % div || ny % div || nz % div) {
        fcm_unet_last_error() = "fcm_unet_forward: spatial sizes must be positive multiples of 2^(levels-1)";
        return FCM_EINVAL;
    }
    UN_CUDA(ensure_shape(N, B, nx, ny, nz));
    const int L = N->levels;
    N->input = in;
    N->output = out;
    for (int l = 0; l < L; ++l) {
        const int64_t bs = (int64_t)B * N->ch(l) * N->S[l];
        if (l > 0)
            pool_fwd_kernel<<<blocks_for((int64_t)B * N->ch(l - 1) * N->S[l]), 256, 0, N->stream>>>(
                N->eB[l - 1], N->xin[l], (int64_t)B * N->ch(l - 1), N->lx[l - 1], N->ly[l - 1], N->lz[l - 1]);
        conv_fwd(N, N->enc_a(l), l == 0 ? in : N->xin[l], N->ea[l], l);
        relu_f(N, N->ea[l], N->eA[l], bs);
        conv_fwd(N, N->enc_b(l), N->eA[l], N->eb[l], l);
        relu_f(N, N->eb[l], N->eB[l], bs);
    }
    const float *prev = N->eB[L - 1];
    for (int l = L - 2; l >= 0; --l) {
        const int cu = N->ch(l + 1), cs = N->ch(l), cc = cu + cs;
        const int64_t S = N->S[l];
        up_fwd_kernel<<<blocks_for((int64_t)B * cu * S), 256, 0, N->stream>>>(prev, N->cat[l], B, cu, cc, 0, N->lx[l],
                                                                             N->ly[l], N->lz[l]);
        chan_copy_kernel<<<blocks_for((int64_t)B * cs * S), 256, 0, N->stream>>>(N->eB[l], cs, 0, N->cat[l], cc, cu, B, cs,
                                                                                S, 0);
        const int64_t bs = (int64_t)B * cs * S;
        conv_fwd(N, N->dec_a(l), N->cat[l], N->da[l], l);
        relu_f(N, N->da[l], N->dA[l], bs);
        conv_fwd(N, N->dec_b(l), N->dA[l], N->db[l], l);
        relu_f(N, N->db[l], N->dB[l], bs);
        prev = N->dB[l];
    }
    conv_fwd(N, N->out_layer(), prev, out, 0);
    UN_CUDA(cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_unet_backward(fcm_unet *N, const float *gout, float *gin)
{
    if (!N || !gout || N->B == 0 || !N->input) {
        fcm_unet_last_error() = "fcm_unet_backward: call fcm_unet_forward first";
        return N ? FCM_ESTATE : FCM_EINVAL;
    }
    const int L = N->levels, B = N->B;
    // skip/encoder-output gradients accumulate from two consumers
    for (int l = 0; l < L; ++l) {
        const int64_t bs = (int64_t)B * N->ch(l) * N->S[l];
        fill_kernel<<<blocks_for(bs), 256, 0, N->stream>>>(N->geB[l], bs, 0.f);
    }
    float *gtop = (L >= 2) ? N->gdB[0] : N->geB[0];
    const float *top = (L >= 2) ? N->dB[0] : N->eB[0];
    conv_bwd(N, N->out_layer(), top, gout, gtop, 0);
    for (int l = 0; l <= L - 2; ++l) {
        const int cu = N->ch(l + 1), cs = N->ch(l), cc = cu + cs;
        const int64_t S = N->S[l], bs = (int64_t)B * cs * S;
        relu_b(N, N->db[l], N->gdB[l], N->gdb[l], bs);
        conv_bwd(N, N->dec_b(l), N->dA[l], N->gdb[l], N->gdA[l], l);
        relu_b(N, N->da[l], N->gdA[l], N->gda[l], bs);
        conv_bwd(N, N->dec_a(l), N->cat[l], N->gda[l], N->gcat[l], l);
        // skip part -> encoder output of level l
        chan_copy_kernel<<<blocks_for(bs), 256, 0, N->stream>>>(N->gcat[l], cc, cu, N->geB[l], cs, 0, B, cs, S, 1);
        // upsampled part -> the level below
        float *gprev = (l + 1 == L - 1) ? N->geB[L - 1] : N->gdB[l + 1];
        const int acc = (l + 1 == L - 1) ? 1 : 0;
        up_bwd_kernel<<<blocks_for((int64_t)B * cu * N->S[l + 1]), 256, 0, N->stream>>>(
            N->gcat[l], gprev, B, cu, cc, 0, N->lx[l], N->ly[l], N->lz[l], acc);
    }
    for (int l = L - 1; l >= 0; --l) {
        const int64_t bs = (int64_t)B * N->ch(l) * N->S[l];
        relu_b(N, N->eb[l], N->geB[l], N->geb[l], bs);
        conv_bwd(N, N->enc_b(l), N->eA[l], N->geb[l], N->geA[l], l);
        relu_b(N, N->ea[l], N->geA[l], N->gea[l], bs);
        if (l > 0) {
            conv_bwd(N, N->enc_a(l), N->xin[l], N->gea[l], N->gxin[l], l);
            pool_bwd_kernel<<<blocks_for((int64_t)B * N->ch(l - 1) * N->S[l - 1]), 256, 0, N->stream>>>(
                N->gxin[l], N->geB[l - 1], (int64_t)B * N->ch(l - 1), N->lx[l - 1], N->ly[l - 1], N->lz[l - 1]);
        } else {
            conv_bwd(N, N->enc_a(0), N->input, N->gea[0], gin, 0);
        }
    }
    UN_CUDA(cudaGetLastError());
    return FCM_OK;
}

fcm_status fcm_unet_zero_grad(fcm_unet *N)
{
    if (!N) return FCM_EINVAL;
    UN_CUDA(cudaMemsetAsync(N->g, 0, sizeof(float) * N->nparam, N->stream));
    return FCM_OK;
}

fcm_status fcm_unet_adam(fcm_unet *N, float lr, float b1, float b2, float eps, int step)
{
    if (!N || step < 1) return FCM_EINVAL;
    const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
    adam_kernel<<<blocks_for(N->nparam), 256, 0, N->stream>>>(N->w, N->g, N->m, N->v, N->nparam, lr, b1, b2, eps, c1, c2);
    to_bf16_kernel<<<blocks_for(N->nparam), 256, 0, N->stream>>>(N->w, N->w16, N->nparam);
    UN_CUDA(cudaGetLastError());
    return FCM_OK;
}

void fcm_unet_destroy(fcm_unet *N)
{
    if (!N) return;
    if (N->stream) cudaStreamSynchronize(N->stream);
    free_acts(N);
    void *ptrs[] = {N->w, N->g, N->m, N->v, N->w16, N->wt16};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete N;
}

}  // extern "C"
