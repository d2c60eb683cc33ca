// Stiffness apply y += K x (Sec. 2.1 Eq. (1)) in double-float arithmetic on the FP32 pipe.
//
// The same two kernels as fcm_kernels.cu -- matrix-free sum factorisation for uncut cells, the
// cell's own dense element matrix for cut cells, 8 parity colours without atomics -- with every
// FP64 multiply-add replaced by a compensated double-float one (fcm_ff.cuh): values and tables are
// float pairs (hi, lo), a product is Dekker's exact product by FMA plus the cross terms, sums run by
// TwoSum.  Each contraction of Q terms is accurate to about 2^-46 relative, so K x agrees with the
// FP64 kernels to ~1e-13, while GB300's FP32 pipe (128 lanes per SM) replaces its FP64 pipe (2
// multiply-adds per clock per SM).  x is read and split by integer operations; the result is added
// into the FP64 vector y, the only FP64 arithmetic left (two adds per DOF and cell).
#include <cuda_runtime.h>

#include "fcm_device.cuh"
#include "fcm_ff.cuh"

namespace fcm {

namespace {

__host__ __device__ constexpr int rnd32k(int v) { return (v + 31) / 32 * 32; }
__host__ __device__ constexpr int ebe_threads(int rows) { return rnd32k(rows) < 512 ? rnd32k(rows) : 512; }

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

// S + C += sum over k < n of a_k b_k for double-float operands
struct FFAcc {
    float S = 0.f, C = 0.f;
    __device__ __forceinline__ void add(float2 a, float2 b) { ff_fma(a.x, a.y, b.x, b.y, S, C); }
    __device__ __forceinline__ float2 get() const { return ff_norm(S, C); }
};

// y += K_e x_e over the cut cells of one colour, K_e stored as double-float pairs (symmetric; column t
// read as row t); rows that are not free stay untouched.
template <int P>
__global__ void __launch_bounds__(ebe_threads(3 * (P + 1) * (P + 1) * (P + 1)))
    ebe_apply_ff_kernel(const double *__restrict__ x, double *__restrict__ y, const uint8_t *__restrict__ mask,
                        const float2 *__restrict__ elem, const int2 *__restrict__ cells, Grid3 g,
                        const int *__restrict__ done)
{
    constexpr int Q = P + 1, NL = Q * Q * Q, NE = 3 * NL;
    if (done && *done) return;
    __shared__ float2 xe[NE];
    __shared__ int64_t node[NL];
    const int2 ce = cells[blockIdx.x];
    const int cx = ce.x % g.n[0], cy = (ce.x / g.n[0]) % g.n[1], cz = ce.x / (g.n[0] * g.n[1]);
    for (int t = threadIdx.x; t < NL; t += blockDim.x) {
        const int ix = t % Q, iy = (t / Q) % Q, iz = t / (Q * Q);
        node[t] = (P * cx + ix) + (int64_t)g.M[0] * ((P * cy + iy) + (int64_t)g.M[1] * (P * cz + iz));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NE; t += blockDim.x) xe[t] = split_ff(x[3 * node[t / 3] + t % 3]);
    __syncthreads();
    const float2 *__restrict__ K = elem + (size_t)ce.y * NE * NE;
    for (int t = threadIdx.x; t < NE; t += blockDim.x) {
        FFAcc s;
#pragma unroll 8
        for (int j = 0; j < NE; ++j) s.add(__ldcs(K + (size_t)j * NE + t), xe[j]);
        const int64_t gi = 3 * node[t / 3] + t % 3;
        if (mask[gi]) y[gi] += ff_to_double(s.get());
    }
}

// y += K_ref x_e for the uncut cells of one colour, matrix-free: the steps of sf_apply_kernel
// (interpolation to the Gauss points by 1D contractions, collocation derivative, weighted stress,
// transposed steps) in double-float arithmetic.  One thread per point (and node) of a cell.
template <int P>
__global__ void __launch_bounds__(256)
    sf_apply_ff_kernel(const double *__restrict__ x, double *__restrict__ y, const uint8_t *__restrict__ mask,
                       const int *__restrict__ cells, int ncells, Grid3 g, SfTablesFF T, const int *__restrict__ done)
{
    constexpr int Q = P + 1, Q3 = Q * Q * Q, TPC = rnd32k(Q3), CPC = 256 / TPC;
    if (done && *done) return;
    __shared__ float2 sB[Q][Q], sG[3][Q][Q], sW[Q];
    __shared__ float2 U[CPC][3][Q3];  // nodal values; then the point values per component
    __shared__ float2 A[CPC][Q3], Bq[CPC][Q3];
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
        for (int c = 0; c < 3; ++c) U[lc][c][t] = split_ff(x[3 * node + c]);
    }
    __syncthreads();
    // interpolation to the points: (ix,iy,iz) -> (qx,iy,iz) -> (qx,qy,iz) -> (qx,qy,qz)
    float2 uq[3];
    for (int c = 0; c < 3; ++c) {
        if (on) {
            FFAcc s;
#pragma unroll
            for (int k = 0; k < Q; ++k) s.add(sB[tx][k], U[lc][c][k + Q * (ty + Q * tz)]);
            A[lc][t] = s.get();
        }
        cell_sync<TPC>();
        if (on) {
            FFAcc s;
#pragma unroll
            for (int k = 0; k < Q; ++k) s.add(sB[ty][k], A[lc][tx + Q * (k + Q * tz)]);
            Bq[lc][t] = s.get();
        }
        cell_sync<TPC>();
        if (on) {
            FFAcc s;
#pragma unroll
            for (int k = 0; k < Q; ++k) s.add(sB[tz][k], Bq[lc][tx + Q * (ty + Q * k)]);
            uq[c] = s.get();
        }
    }
    cell_sync<TPC>();  // every point has read the nodal values of its cell
    if (on)
        for (int c = 0; c < 3; ++c) U[lc][c][t] = uq[c];
    cell_sync<TPC>();
    // gradients at the point by the collocation derivative along each axis
    float2 gr[3][3];
    if (on) {
        for (int c = 0; c < 3; ++c) {
            FFAcc gx, gy, gz;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                gx.add(sG[0][tx][k], U[lc][c][k + Q * (ty + Q * tz)]);
                gy.add(sG[1][ty][k], U[lc][c][tx + Q * (k + Q * tz)]);
                gz.add(sG[2][tz][k], U[lc][c][tx + Q * (ty + Q * k)]);
            }
            gr[c][0] = gx.get();
            gr[c][1] = gy.get();
            gr[c][2] = gz.get();
        }
    }
    // weighted stress at the point: F[c][j] = w detJ (lam tr(eps) delta_cj + mu (g_cj + g_jc))
    float2 F[3][3];
    if (on) {
        const float2 w = ff_mul(ff_mul(ff_mul(sW[tx], sW[ty]), sW[tz]), T.detJ);
        const float2 ltr = ff_mul(T.lam, ff_addv(ff_addv(gr[0][0], gr[1][1]), gr[2][2]));
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j) {
                float2 v = ff_mul(T.mu, ff_addv(gr[c][j], gr[j][c]));
                if (c == j) v = ff_addv(v, ltr);
                F[c][j] = ff_mul(w, v);
            }
    }
    float2 out[3];
    for (int c = 0; c < 3; ++c) {
        cell_sync<TPC>();  // the previous readers of U and A are done
        if (on)
            for (int j = 0; j < 3; ++j) U[lc][j][t] = F[c][j];
        cell_sync<TPC>();
        if (on) {  // transposed collocation derivative: point values of component c's force
            FFAcc v;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                v.add(sG[0][k][tx], U[lc][0][k + Q * (ty + Q * tz)]);
                v.add(sG[1][k][ty], U[lc][1][tx + Q * (k + Q * tz)]);
                v.add(sG[2][k][tz], U[lc][2][tx + Q * (ty + Q * k)]);
            }
            A[lc][t] = v.get();
        }
        cell_sync<TPC>();
        if (on) {  // z^T: (qx, qy, iz)
            FFAcc s;
#pragma unroll
            for (int k = 0; k < Q; ++k) s.add(sB[k][tz], A[lc][tx + Q * (ty + Q * k)]);
            Bq[lc][t] = s.get();
        }
        cell_sync<TPC>();
        if (on) {  // y^T: (qx, iy, iz)
            FFAcc s;
#pragma unroll
            for (int k = 0; k < Q; ++k) s.add(sB[k][ty], Bq[lc][tx + Q * (k + Q * tz)]);
            A[lc][t] = s.get();
        }
        cell_sync<TPC>();
        if (on) {  // x^T: nodal force (ix, iy, iz)
            FFAcc s;
#pragma unroll
            for (int k = 0; k < Q; ++k) s.add(sB[k][tx], A[lc][k + Q * (ty + Q * tz)]);
            out[c] = s.get();
        }
    }
    if (on)
        for (int c = 0; c < 3; ++c)
            if (mask[3 * node + c]) y[3 * node + c] += ff_to_double(out[c]);
}

template <int P>
void k_launch_ff(const Grid3 &g, const double *x, double *y, const uint8_t *mask, const float2 *elem,
                 const KCells &kc, const int *done, cudaStream_t s, const KStreams &ks)
{
    constexpr int NE = 3 * (P + 1) * (P + 1) * (P + 1);
    constexpr int CPC = 256 / rnd32k((P + 1) * (P + 1) * (P + 1));
    for (int c = 0; c < 8; ++c) {
        const int nu = kc.uncut_off[c + 1] - kc.uncut_off[c];
        const int nc = kc.cut_off[c + 1] - kc.cut_off[c];
        // cut and uncut cells of one colour share no DOF: the cut cells (HBM-bound) run beside the uncut
        // ones (FP32-pipe and latency bound)
        const bool fork = ks.side && nu > 0 && nc > 0;
        if (fork) {
            cudaEventRecord(ks.fork, s);
            cudaStreamWaitEvent(ks.side, ks.fork, 0);
        }
        if (nc > 0)
            ebe_apply_ff_kernel<P><<<nc, ebe_threads(NE), 0, fork ? ks.side : s>>>(x, y, mask, elem,
                                                                                  kc.cut + kc.cut_off[c], g, done);
        if (nu > 0)
            sf_apply_ff_kernel<P><<<(nu + CPC - 1) / CPC, 256, 0, s>>>(x, y, mask, kc.uncut + kc.uncut_off[c], nu, g,
                                                                      kc.sff, done);
        if (fork) {
            cudaEventRecord(ks.join, ks.side);
            cudaStreamWaitEvent(s, ks.join, 0);
        }
    }
}

// FP64 element matrices -> double-float pairs
__global__ void to_ff_pairs_kernel(const double *__restrict__ in, float2 *__restrict__ out, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = split_ff(in[e]);
}

}  // namespace

void launch_k_apply_ff(int p, const Grid3 &g, const double *x, double *y, const uint8_t *mask, const float2 *elem,
                       const KCells &kc, const int *done, cudaStream_t s, const KStreams &ks)
{
    switch (p) {
    case 1: k_launch_ff<1>(g, x, y, mask, elem, kc, done, s, ks); break;
    case 2: k_launch_ff<2>(g, x, y, mask, elem, kc, done, s, ks); break;
    case 3: k_launch_ff<3>(g, x, y, mask, elem, kc, done, s, ks); break;
    case 4: k_launch_ff<4>(g, x, y, mask, elem, kc, done, s, ks); break;
    default: break;
    }
}

void launch_to_ff_pairs(const double *in, float2 *out, int64_t n, cudaStream_t s)
{
    const int64_t b = (n + 255) / 256;
    to_ff_pairs_kernel<<<(int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16), 256, 0, s>>>(in, out, n);
}

void make_sf_tables_ff(const SfTables &T, SfTablesFF &F)
{
    auto sp = [](double v) {
        const float h = (float)v;
        return make_float2(h, (float)(v - (double)h));
    };
    for (int q = 0; q < 5; ++q) {
        F.W[q] = sp(T.W[q]);
        for (int i = 0; i < 5; ++i) {
            F.B[q][i] = sp(T.B[q][i]);
            for (int a = 0; a < 3; ++a) F.G[a][q][i] = sp(T.G[a][q][i]);
        }
    }
    F.detJ = sp(T.detJ);
    F.lam = sp(T.lam);
    F.mu = sp(T.mu);
}

}  // namespace fcm
