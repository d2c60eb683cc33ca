// Device-side context and kernel launchers of libfcm (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "fcm_internal.h"

struct fcm_ctx;

namespace fcm {

// One Schwarz block as seen by the block-apply kernel.
struct PatchRec {
    int64_t off;   // element offset of the block factor in the factor pool
    int32_t v;     // vertex patches: linear vertex index v_x + (n_x+1)(v_y + (n_y+1) v_z);
                   // element blocks: linear cell index c_x + n_x (c_y + n_y c_z)
    int32_t prec;  // 0: factor stored in FP64, 1: FP32
};

// Leading dimension of a stored block factor with n rows: rows are padded to a multiple of 16
// bytes (zeros), so a row, or a run of rows, can be moved by one bulk copy and read as 16-byte
// vectors.  Factor offsets in a pool are multiples of 16 bytes too.
template <typename T>
__host__ __device__ constexpr int factor_ld(int n)
{
    return (n + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T));
}

// CG scalars kept on the device for the whole solve (no host round trip per iteration).
struct CgScalars {
    double rz, pq, zz, zz0, alpha, beta, relres, tol;
    int it, maxit, done, status;
};

struct Grid3 {
    int n[3];   // cells
    int M[3];   // lattice nodes per axis
};

// The sum-factorisation tables as double-float pairs (hi = fl32(v), lo = fl32(v - hi)).
struct SfTablesFF {
    float2 B[5][5], G[3][5][5], W[5];
    float2 detJ, lam, mu;
};
void make_sf_tables_ff(const SfTables &T, SfTablesFF &F);

// Active cells of the K apply, grouped by parity colour: uncut cells (matrix-free,
// sum-factorised) and cut cells (their own dense element matrix).
struct KCells {
    const int *uncut;     // cell ids
    const int2 *cut;      // (cell id, element id)
    int uncut_off[9];
    int cut_off[9];
    SfTables sf;
    SfTablesFF sff;
};

// Launch plan of the Schwarz apply (fcm_schwarz.cu).  Every block has a slot: its record
// (factor offset, vertex or cell id, storage: 0 FP64, 1 FP32, 2 double-float) and nslots * zs
// doubles of Zb for its product.  Slots of blocks that share a factor are consecutive (GEMM tiles
// of up to NC blocks: (first slot, count), the FP32 tiles first); the other blocks stream their
// own factor in row tiles ((slot, first row) work items), with a warp per row (row_items, `rows`
// rows each; p = 3, one right-hand side) or a thread per row (col_items, schwarz_col_rows(p) rows
// each).  slot_of maps a vertex (or cell) id to its slot, -1 when the block has no free DOF.
// A tile of the tensor-core product: 128 consecutive slots (`count` used) sharing one FP32 factor, its
// factor tiles at ft_off (floats), nch chunks of 16 K values.
struct TcTile {
    int first, count;
    int64_t ft_off;
    int nch, pad;
};

struct SchwarzPlan {
    Grid3 g;
    int rule;                 // 0 vertex patches, 3 element blocks (FCM_BLOCKS_*)
    int zs;                   // Zb rows per slot (largest block, rounded up to 8)
    int64_t nslots;
    const PatchRec *slots;
    const int *slot_of;
    const int2 *row_items;
    int n_row_items, rows;
    const int2 *col_items;
    int n_col_items;
    const int2 *tiles;        // n_tiles32 FP32 tiles, then n_tiles64 FP64 tiles
    int n_tiles32, n_tiles64;
    int n_tiles32_plain;      // FP32 tiles of the factors without tensor-core tiles (listed first)
    const TcTile *tc_tiles;   // tensor-core tiles (one right-hand side), same blocks as the rest of the FP32 tiles
    int n_tc_tiles;
    const float *tc_ft;       // factor tiles (hi, lo) in the tensor core's layout
    double *zb;               // Zb for one right-hand side
    int pairs;                // 1: Zb entries are float pairs (mixed forms), 0: FP64 values
    const double *jac;        // 1 / K_ll for the free DOFs in no block, 0 elsewhere (lattice); null if none
    int *err;                 // device flag, set to 1 by a bulk-copy wait that ran out
    int wait_tries;           // polls of a bulk-copy wait before it gives up
    int concurrent;           // 1: the GEMM tiles run on `side` beside the streamed factors
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
};

// Second stream of the K apply: per colour, the cut cells run on `side` beside the uncut cells on the
// main stream (the two sets are DOF-disjoint within a colour); null side: one stream.
struct KStreams {
    cudaStream_t side;
    cudaEvent_t fork, join;
};

// Launchers (all asynchronous on `s`).  `done` may be null.  The Schwarz launchers overwrite z
// with S r.  The multi-RHS form takes nr <= 8 vectors nlat apart and a Zb of nr * nslots * zs doubles.
void launch_k_apply(int p, const Grid3 &g, const double *x, double *y, const uint8_t *mask, const double *elem,
                    const KCells &kc, const int *done, cudaStream_t s, const KStreams &ks);
// the same in double-float arithmetic on the FP32 pipe (fcm_kapply_ff.cu); elem: the element matrices as
// float pairs
void launch_k_apply_ff(int p, const Grid3 &g, const double *x, double *y, const uint8_t *mask, const float2 *elem,
                       const KCells &kc, const int *done, cudaStream_t s, const KStreams &ks);
void launch_to_ff_pairs(const double *in, float2 *out, int64_t n, cudaStream_t s);
void launch_schwarz_apply(int p, const Grid3 &g, const double *r, double *z, const double *fpool64,
                          const float *fpool32, const SchwarzPlan &plan, const int *done, cudaStream_t s);
void launch_schwarz_apply_multi(int p, const double *r, double *z, int64_t nlat, int nr, const double *f64,
                                const float *f32, const SchwarzPlan &plan, double *zb, const int *done,
                                cudaStream_t s);
// columns of a GEMM tile for FP32 (prec 1) or FP64 (prec 0) factors; rows per col_items work item;
// whether single right-hand sides stream through row_items; threads of a row_items CTA
int schwarz_gemm_cols(int p, int prec);
int schwarz_col_rows(int p);
bool schwarz_uses_rows_kernel(int p);
// tensor-core products (p = 2, 3): floats of one factor's tiles, and the kernel that builds them from an
// FP64 factor (rows padded to factor_ld<double>(n))
bool schwarz_tc_supported(int p);
int64_t schwarz_tc_factor_floats(int p, int n);
cudaError_t schwarz_tc_factor(int p, const double *F, int n, float *ft, cudaStream_t s);
int schwarz_rows_threads();
// kernel attributes (dynamic shared memory); host call, outside stream capture
cudaError_t schwarz_prepare(int p);
// polls of a bulk-copy wait before it gives up (default)
constexpr int kWaitTries = 1 << 21;
void launch_mask_copy(const double *in, double *out, const uint8_t *mask, int64_t n, cudaStream_t s);
// fcm_noalloc.cu: device address of the static scratch of fcm_apply_S_noalloc on the current device
cudaError_t noalloc_scratch_address(double **out);
void launch_zero(double *v, int64_t n, const int *done, cudaStream_t s);

// CG building blocks (fcm_solver.cu)
struct CgWork {
    double *x, *r, *z, *p, *q, *b;
    double *partial;      // reduction partials
    unsigned *counter;    // last-block ticket
    CgScalars *s;         // device scalars
    int64_t n;
    int red_blocks;
};
void cg_init_kernels(const CgWork &w, cudaStream_t s);                  // x=0, r=b
void cg_after_first_S(const CgWork &w, cudaStream_t s);                 // rz, zz0, p = z
void cg_after_K(const CgWork &w, cudaStream_t s);                       // pq, alpha, x, r
void cg_after_S(const CgWork &w, cudaStream_t s);                       // rz, zz, convergence, beta, p
void cg_residual_norms(const CgWork &w, const double *res, const double *b, double *out2, cudaStream_t s);

// fcm_precond.cu
std::string build_preconditioner(fcm_ctx *C, const fcm_precond_opts &o);

// fcm_capi.cu: operators and the plain PCG on a context's own work stream
void ctx_apply_K(fcm_ctx *C, const double *x, double *y);
void ctx_apply_S(fcm_ctx *C, const double *r, double *z);
// the same, skipped on the device while *stop != 0 (stop may be null)
void ctx_apply_K_flag(fcm_ctx *C, const double *x, double *y, const int *stop);
void ctx_apply_S_flag(fcm_ctx *C, const double *r, double *z, const int *stop);
fcm_status ctx_solve_one(fcm_ctx *C, const double *rhs, double tol, int maxit, double *u, fcm_solve_info &info);

// fcm_unet.cu: redirect a network's launches to stream s; returns the previous stream
cudaStream_t unet_set_stream(fcm_unet *N, cudaStream_t s);
// identity of a network and of its current activation buffers (changes when they are reallocated)
void unet_identity(const fcm_unet *N, uint64_t *serial, uint64_t *gen);

// fcm_coarse_op.cu: Galerkin coarse operator K_H = P^T K P on the cell grid
struct CoarseOp;
fcm_status coarse_ensure(fcm_ctx *C);
void coarse_free(CoarseOp *op);
// start: 0 from zero, 1 from the given y, 2 from the given y scaled by the energy-minimising step
// st: the stream to run on (null: the context's work stream)
void coarse_solve(fcm_ctx *C, const float *f, float *y, int iters, int start, const int *stop,
                  cudaStream_t st = nullptr);
void coarse_apply(fcm_ctx *C, const float *x, float *y);
double coarse_seconds(const CoarseOp *op);

// fcm_coarse.cu: workspace and captured graph of the flexible PCG, kept between solves
struct FcgState;
void fcg_free(FcgState *f);
// drop the captured flexible-CG graph (it holds the addresses of the Schwarz plan and factors)
void fcg_forget_graph(FcgState *f);

}  // namespace fcm

std::string &fcm_unet_last_error();

struct fcm_ctx {
    std::string err;
    cudaStream_t ustream = nullptr;  // caller's stream (ordering with the caller)
    cudaStream_t stream = nullptr;   // the library's own work stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaEvent_t ev_f0 = nullptr, ev_f1 = nullptr;  // start and end of a flexible solve (ev_t0/ev_t1 time its inner plain solve)
    fcm::HostProblem hp;
    fcm::Grid3 g;
    int p = 0, ne = 0;
    int64_t nlat = 0;
    // problem on the device
    double *d_elem = nullptr;        // [Kref | Kcut_1 | ...], ne*ne each, row-major (symmetric)
    float2 *d_elem_ff = nullptr;     // the same as double-float pairs (allocated by fcm_set_k_precision)
    int k_ff = 0;                    // 1: K applied in double-float arithmetic
    int32_t *d_cell_elem = nullptr;  // per cell
    uint8_t *d_mask = nullptr;       // per lattice DOF
    double *d_rhs = nullptr;         // load case 0
    float *d_eta = nullptr;          // volume fraction per cell
    int2 *d_cells = nullptr;         // cut cells by colour: (cell, element id)
    int *d_uncut = nullptr;          // uncut cells by colour
    fcm::KCells kc = {};
    int64_t element_bytes = 0;
    double setup_seconds = 0.0;
    // preconditioner
    bool have_precond = false;
    double *d_f64 = nullptr;         // FP64 factor pool
    float *d_f32 = nullptr;          // FP32 factor pool (mixed precision)
    fcm::PatchRec *d_slots = nullptr;
    int *d_slot_of = nullptr;
    int2 *d_items = nullptr;         // row items, column items, GEMM tiles
    fcm::TcTile *d_tc_tiles = nullptr;
    float *d_tc_ft = nullptr;        // tensor-core factor tiles
    double *d_zb = nullptr;          // block products of one S apply
    cudaStream_t side = nullptr;     // second stream of the Schwarz apply (shared-factor products)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    fcm::KStreams ks{};              // second stream of the K apply (cut cells beside uncut ones)
    int64_t n_ff_factors = 0;        // factors stored as double-float pairs
    int64_t n_gemm_blocks = 0;       // blocks applied by the shared-factor GEMM
    double *d_jac = nullptr;         // diagonal part of S (element blocks), lattice; null if none
    int *d_err = nullptr;            // set by a Schwarz CTA whose bulk-copy wait ran out
    double *noalloc_scratch = nullptr;  // device address of fcm_apply_S_noalloc's static scratch
    std::string noalloc_err;            // why it is null (problem too large, or the lookup failed)
    int device = 0;                     // CUDA device current at fcm_setup
    int fcg_window = 100;            // stall window of the flexible CG (fcm_fpcg_set_stall_window)
    double tune_seconds[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // S-apply times of the launch shapes tried
    int wait_tries = fcm::kWaitTries;  // fcm_set_wait_limit
    int64_t n_jacobi = 0;
    fcm::SchwarzPlan plan = {};
    int64_t n_factors = 0, factor_bytes = 0, n_fp32_factors = 0;
    double max_cond = 0.0;
    int64_t n_blocks = 0, sapply_fmas = 0;
    int max_block = 0;
    double precond_seconds = 0.0;
    // solver workspace
    double *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_b = nullptr,
           *d_t = nullptr;
    double *d_partial = nullptr;
    unsigned *d_counter = nullptr;
    fcm::CgScalars *d_s = nullptr;
    fcm::CgScalars *h_s = nullptr;   // pinned
    int *h_err = nullptr;            // pinned copy of d_err, read with the scalars
    double *d_out2 = nullptr;
    int red_blocks = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    fcm_solve_info last = {};
    // multi-RHS workspace: x, r, z, p, q, b for m_nr right-hand sides, and their CG scalars
    double *d_m = nullptr;
    fcm::CgScalars *d_ms = nullptr, *h_ms = nullptr;
    double *d_mzb = nullptr;         // block products of the multi-RHS Schwarz apply
    int m_nr = 0;
    // coarse operator of the learned correction (built on first use)
    fcm::CoarseOp *coarse = nullptr;
    int coarse_prec = FCM_COARSE_JACOBI;  // fcm_coarse_set_preconditioner
    int coarse_half = 0;                  // fcm_coarse_set_storage
    fcm::FcgState *fcg = nullptr;
};
