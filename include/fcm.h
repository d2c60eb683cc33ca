/*
 * fcm.h -- C ABI of the GB300 finite cell Schwarz-PCG solver (libfcm.so).
 *
 * The library solves the finite cell stiffness system of 3D linear elasticity
 * (Jomo et al., arXiv:1809.00828, Sec. 2.1 Eq. (1)) on a Cartesian grid with an
 * integrated-Legendre basis of order p, cut cells integrated by octree
 * partitioning (Sec. 5.1 setup) and a fictitious-domain stiffness alpha, by
 * conjugate gradients preconditioned with the overlapping Additive-Schwarz
 * operator S = sum_B R_B^T A_B+^-1 R_B (Sec. 3.1 Eq. (5)) built from
 * eigenvalue-filtered pseudo inverses (Sec. 3.2 Eqs. (11)-(13), Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Vectors (right-hand sides, solutions, K/S inputs and outputs) are FP64
 * arrays of length fcm_info.n_lattice in "lattice" layout:
 *   M_a = p * n[a] + 1 lattice nodes per axis, node (i,j,k) -> i + M_0 (j + M_1 k),
 *   DOF = 3 * node + component (components interleaved).
 * Along an axis, cell c owns lattice indices p*c .. p*c+p: p*c is its left
 * grid vertex, p*c+p its right one, p*c+a (0<a<p) the integrated Legendre
 * function phi_{a+1} = (P_{a+1} - P_{a-1}) / sqrt(2(2a+1)) of that cell.
 * Entries that are not free (on no active cell, or Dirichlet-fixed) are
 * ignored on input and written as 0 on output.
 *
 * Pointers named *_dev are CUDA device pointers on the current device; the
 * caller owns them.  Everything reachable from an fcm_ctx is owned by the
 * library and released by fcm_destroy.  No C++ exception crosses this ABI.
 * All device work is ordered on the stream passed to fcm_setup; functions
 * that return results to host memory synchronise that stream.
 * On error a function returns a nonzero fcm_status and leaves a message in
 * fcm_last_error(ctx) (or fcm_last_error(NULL) when no context exists).
 */
#ifndef FCM_H
#define FCM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcm_ctx fcm_ctx;

typedef enum {
    FCM_OK = 0,
    FCM_EINVAL = 1,      /* invalid argument (sizes, NaN inputs, null pointers)      */
    FCM_ENOMEM = 2,      /* device or host allocation failed                         */
    FCM_ECUDA = 3,       /* a CUDA / cuSOLVER / cuBLAS call failed                   */
    FCM_ENOTCONV = 4,    /* maxit reached; the last iterate is returned              */
    FCM_EBREAKDOWN = 5,  /* p^T K p <= 0 or a non-finite scalar in CG                */
    FCM_ETIMEOUT = 6,    /* a bounded device wait gave up                            */
    FCM_ESTATE = 7       /* call out of order (e.g. solve before fcm_precond_build)  */
} fcm_status;

/* Cartesian grid: n[a] cells on [lo[a], hi[a]] per axis. */
typedef struct {
    int n[3];
    double lo[3], hi[3];
} fcm_grid;

enum { FCM_GEOM_SPHERE_VOIDS = 0, FCM_GEOM_VOXELS = 1, FCM_GEOM_HALFSPACE = 2 };

/* Physical domain Omega_phys (Sec. 2.1).  Host arrays, copied by fcm_setup.
 *   kind 0: the grid box minus the union of open balls sph[4*s..4*s+3] = (cx, cy, cz, r)
 *   kind 1: voxel image vox (vdim[0] fastest) over the grid box; solid where vox != 0
 *   kind 2: half-space {x : plane[0] x + plane[1] y + plane[2] z < plane[3]}
 * octree_depth: partition depth of cut cells relative to the cell size (Sec. 5.1). */
typedef struct {
    int kind;
    int nsph;
    const double *sph;
    int vdim[3];
    const unsigned char *vox;
    double plane[4];
    int octree_depth;
} fcm_geometry;

enum { FCM_BC_NONE = -1, FCM_BC_CLAMP_ZLO = 0, FCM_BC_ROLLERS = 1 };

/* Material and boundary conditions.  bc: FCM_BC_CLAMP_ZLO fixes every
 * component on the face z = lo[2]; FCM_BC_ROLLERS fixes u_x on x = lo[0],
 * u_y on y = lo[1], u_z on z = lo[2]; FCM_BC_NONE fixes nothing (K then has
 * the rigid-body modes in its null space).  Dirichlet data is homogeneous and
 * imposed strongly on the grid-aligned faces.  traction: surface load on the
 * face z = hi[2] where it lies in Omega_phys (load case 0). */
typedef struct {
    double E, nu;
    int bc;
    double traction[3];
} fcm_bc;

/* Sizes of a set-up problem. */
typedef struct {
    int64_t n_lattice;        /* length of every vector, 3 * prod(M_a)                 */
    int64_t n_free;           /* free DOFs                                             */
    int64_t n_cells_active;   /* cells with eta_T > 0                                  */
    int64_t n_cells_cut;      /* active cells with their own element matrix            */
    int64_t n_patches;        /* vertex patches (blocks), (n0+1)(n1+1)(n2+1)           */
    int64_t n_factors;        /* distinct stored block factors after deduplication     */
    int64_t factor_bytes;     /* device bytes of the stored block factors              */
    int64_t element_bytes;    /* device bytes of the stored element matrices           */
    int max_block;            /* largest block, 3 (2p-1)^3                              */
    int p;
    double setup_seconds;     /* host+device time of fcm_setup                         */
    double precond_seconds;   /* time of the last fcm_precond_build                    */
    int64_t n_blocks;         /* blocks (patches or elements) with at least one free DOF */
    int64_t n_blocks_fp32;    /* of the stored factors, those kept in FP32             */
    int64_t kapply_fmas;      /* multiply-adds of one K apply (sum over active cells)  */
    int64_t sapply_fmas;      /* multiply-adds of one S apply (sum of block box sizes^2) */
    double max_block_cond;    /* largest retained condition number of a block          */
    double coarse_seconds;    /* assembly time of the coarse operator K_H (0 until built) */
    int64_t n_jacobi;         /* free DOFs in no block (diagonal part of S), last build   */
    int stream_rows;          /* rows per work item of a block that streams its own factor (p = 3) */
    int schwarz_concurrent;   /* 1: shared-factor products run on a second stream beside the
                                 streamed factors; 0: after them                          */
    double tune_seconds[8];   /* S-apply time of each tried launch shape (0: not tried)  */
    int device_error;         /* 1 if a Schwarz kernel gave up waiting for its factor copy
                                 since the last fcm_precond_build or solve (its output is then wrong) */
    int64_t n_factors_ff;     /* factors stored as double-float pairs (FCM_PREC_MIXED, cond > cond_fp64) */
    int64_t n_gemm_blocks;    /* blocks applied by the shared-factor dense product        */
    int k_double_float;       /* 1: K applied in double-float arithmetic (fcm_set_k_precision) */
    int s_apply_launches;     /* kernel launches of one fcm_apply_S (one right-hand side, masked copy excluded) */
    int k_apply_launches;     /* kernel launches of one fcm_apply_K (masked copy excluded)  */
} fcm_info_t;

enum { FCM_PREC_FP64 = 0, FCM_PREC_MIXED = 1, FCM_PREC_MIXED_FP64 = 2 };

enum { FCM_BLOCKS_VERTEX = 0, FCM_BLOCKS_ELEMENT = 3 };

/* Preconditioner options (Algorithm 1).
 *   eps: pseudo-inverse threshold, eigenvalues <= eps * lambda_max are dropped
 *        (Sec. 3.2 Eq. (13); the paper uses 1e-13).  eps < 0 gives the
 *        unstabilised inverse S* (every nonzero eigenvalue inverted).
 *   precision: FCM_PREC_FP64 stores and applies every factor in FP64;
 *        FCM_PREC_MIXED stores factors in FP32 except blocks whose retained
 *        condition number exceeds cond_fp64: those keep their FP64 values as
 *        double-float pairs (hi = fl32(f), lo = fl32(f - hi), 2^-48 relative)
 *        applied with error-free FP32 transformations (compensated products
 *        and sums; ~1e-14 relative per dot product), or in FP64 when the factor
 *        is shared by many blocks; FCM_PREC_MIXED_FP64 is the same with FP64
 *        storage and arithmetic for every factor above the threshold.
 *   cond_fp64: threshold for FCM_PREC_MIXED (default 1e7).
 *   block_rule: FCM_BLOCKS_VERTEX (0, default): one block per grid vertex,
 *        the free functions carried by the vertex and by the edges, faces and
 *        cells whose closure contains it (every free DOF is covered).
 *        FCM_BLOCKS_ELEMENT (3): the paper's element blocks (Sec. 3.2,
 *        "Optimizing the number of blocks"): for every active cell with volume
 *        fraction eta_T <= eta_bar, all functions supported on the cell; the free
 *        DOFs in no block get Algorithm 1's diagonal scaling 1 / K_ll.
 *        eta_bar = 0 gives pure Jacobi; eta_bar = 1 blocks every active cell
 *        (Sec. 5.2's end points; eta_T is clamped to 1 against rounding).
 *   eta_bar: threshold of FCM_BLOCKS_ELEMENT (ignored by FCM_BLOCKS_VERTEX).
 *   fixed_tiles: 0 (default) lets the build time the Schwarz apply for up to
 *        six launch shapes (three row-tile sizes of the blocks that stream their
 *        own factor, each with the shared-factor products after the streamed
 *        factors or beside them on a second stream) and keep the fastest; 1 keeps
 *        the default tile, products after the streamed factors; 2 the default
 *        tile, both at once.  S r does not depend on the choice.
 *   simt_shared: 0 (default) applies the FP32 shared factors of the mixed
 *        forms (p = 2, 3; one right-hand side) on the tensor cores (tcgen05,
 *        TF32 three-pass products, ~2^-22 relative); 1 applies them on the
 *        CUDA cores in FP32.
 * A zero-initialised struct with eps, precision and cond_fp64 set selects
 * vertex patches and the autotuned tiles. */
typedef struct {
    double eps;
    int precision;
    double cond_fp64;
    int block_rule;
    double eta_bar;
    int fixed_tiles;
    int simt_shared;
} fcm_precond_opts;

/* Solver result details. */
typedef struct {
    int iterations;            /* K applications performed                          */
    double relres;             /* ||S r_i|| / ||S b||, Eq. (14)                      */
    double true_relres;        /* ||b - K x_i|| / ||b|| recomputed at exit           */
    int status;                /* fcm_status of the solve                           */
    double seconds;            /* device time of the solve                          */
    int flexible_iterations;   /* fcm_fpcg_solve: iterations with the learned term  */
    int fallback;              /* fcm_fpcg_solve: 1 if it fell back to plain PCG    */
} fcm_solve_info;

/* Set up the problem: classify cells by octree quadrature, compute eta_T,
 * the element matrices, the free-DOF mask and the load (Sec. 2.1 Eq. (1),
 * Sec. 5.1).  p in [1, 4].  alpha in (0, 1].  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) used for every later call on this context.
 * Returns FCM_EINVAL for bad sizes, FCM_ECUDA/FCM_ENOMEM for device failures. */
fcm_status fcm_setup(const fcm_grid *grid, const fcm_geometry *geom, int p, double alpha,
                     const fcm_bc *bc, void *cuda_stream, fcm_ctx **out);

/* Copy the problem sizes into *out. */
fcm_status fcm_info(const fcm_ctx *ctx, fcm_info_t *out);

/* Write load case load_case into b_dev (n_lattice FP64, device).
 *   0: traction of fcm_bc on the top face (Sec. 2.1 Eq. (1), Neumann term).
 *   1..6: unit-strain load cases b_k(v) = -int alpha eps(v) : C : E_k dOmega, E_k the
 *         Voigt unit strains xx, yy, zz, yz, xz, xy (engineering shears), i.e. the load
 *         that a prescribed uniform strain E_k exerts through the alpha-weighted
 *         stiffness of Eq. (1) (equal to -K u_k for the linear field u_k = E_k x). */
fcm_status fcm_rhs(const fcm_ctx *ctx, int load_case, double *b_dev);

/* Build the Additive-Schwarz preconditioner (Algorithm 1) with the blocks of
 * opts->block_rule (vertex patches by default, or the paper's element blocks
 * with the eta_bar threshold and diagonal scaling of uncovered DOFs).
 * Extracts A_B = K[B,B], computes its eigendecomposition, keeps
 * lambda_k > eps * max lambda and stores A_B+^-1.  Identical blocks (blocks of
 * uncut cells with the same boundary pattern) share one stored factor.  opts
 * may be NULL (eps 1e-13, FP64, vertex patches).  Returns FCM_EINVAL for an
 * unknown rule or precision or a negative or NaN eta_bar.  Invalidates the
 * captured solver graphs of the context (they are captured again by the next
 * solve). */
fcm_status fcm_precond_build(fcm_ctx *ctx, const fcm_precond_opts *opts);

/* Preconditioned CG, x0 = 0, stopping when ||S r_i|| / ||S b|| <= tol
 * (Sec. 5 Eq. (14)) or after maxit iterations.  rhs_dev / u_dev: nrhs
 * vectors of n_lattice FP64 each, stored one after another (device).
 * iterations / final_relres may be NULL; with nrhs > 1 they receive the
 * largest count and residual over the right-hand sides.
 * Returns FCM_ESTATE before fcm_precond_build, FCM_EINVAL for a non-finite
 * rhs, FCM_ENOTCONV after maxit (u_dev holds the last iterate),
 * FCM_EBREAKDOWN when p^T K p <= 0 or a scalar becomes non-finite. */
fcm_status fcm_pcg_solve(fcm_ctx *ctx, const double *rhs_dev, int nrhs, double tol, int maxit,
                         double *u_dev, int *iterations, double *final_relres);

/* Same as fcm_pcg_solve with host buffers: rhs_host is copied to the device,
 * solved, and the solution copied back into u_host before returning. */
fcm_status fcm_pcg_solve_host(fcm_ctx *ctx, const double *rhs_host, int nrhs, double tol, int maxit,
                              double *u_host, int *iterations, double *final_relres);

/* Details of the last solve (all right-hand sides folded as in fcm_pcg_solve). */
fcm_status fcm_last_solve(const fcm_ctx *ctx, fcm_solve_info *out);

/* y_dev = K x_dev (Sec. 2.1 Eq. (1), left-hand side), lattice layout, device. */
fcm_status fcm_apply_K(fcm_ctx *ctx, const double *x_dev, double *y_dev);

/* z_dev = S r_dev, S = sum_B R_B^T A_B+^-1 R_B (Sec. 3.1 Eq. (5)); device.
 * FCM_ESTATE before fcm_precond_build. */
fcm_status fcm_apply_S(fcm_ctx *ctx, const double *r_dev, double *z_dev);

enum { FCM_K_FP64 = 0, FCM_K_DOUBLE_FLOAT = 1 };

/* Arithmetic of K x (Eq. (1); every K apply of the context, solves included).
 * FCM_K_FP64 (default): FP64 multiply-adds.  FCM_K_DOUBLE_FLOAT: the same
 * steps with double-float values (float pairs) and compensated products and
 * sums on the FP32 pipe, about 2^-46 relative per contraction (K x within
 * ~1e-13 of the FP64 result); GB300's FP32 pipe is 64 times wider than its
 * FP64 pipe.  The first switch to double-float stores a float-pair copy of
 * the element matrices (fcm_info.element_bytes more device memory).  Captured
 * solver graphs are dropped.  FCM_EINVAL for another mode. */
fcm_status fcm_set_k_precision(fcm_ctx *ctx, int mode);

/* z_dev = S r_dev for nrhs (1..8) vectors stored n_lattice apart (device);
 * the block factors are read once for all of them.  Column k equals
 * fcm_apply_S of column k.  FCM_EINVAL for nrhs outside 1..8. */
fcm_status fcm_apply_S_many(fcm_ctx *ctx, const double *r_dev, int nrhs, double *z_dev);

/* Failure detection: polls of the bounded mbarrier wait with which a Schwarz
 * kernel waits for a bulk copy of a shared factor into shared memory (default
 * 2^21).  A wait that runs out lets the copies in flight land, marks the apply
 * as failed and returns; the solves then stop with FCM_ETIMEOUT (and
 * fcm_info.device_error reports it after fcm_apply_S).  tries = 0 gives up at
 * the first poll (for tests); tries < 0 restores the default.  Captured solver
 * graphs are dropped (captured again by the next solve). */
fcm_status fcm_set_wait_limit(fcm_ctx *ctx, int tries);

/* ------------------------------------------------------------------------ */
/* Learned coarse correction (not in the paper: the paper's preconditioner   */
/* has no coarse space, Sec. 6; this adds one, learned).                     */
/* ------------------------------------------------------------------------ */

/* 3D U-Net on the cell grid: `levels` resolution levels with channels
 * base * 2^l capped at 4 * base, two 3x3x3 convolutions + ReLU per level and
 * decoder stage, average pooling, nearest upsampling with skip
 * concatenation, and a final 3x3x3 convolution to out_ch channels.
 * Weights are stored in BF16 for the forward pass (FP32 master copy and
 * Adam moments for training); activations and accumulation are FP32.
 * Tensors are float, layout [batch][channel][z][y][x] (x fastest), device.
 * Spatial sizes must be divisible by 2^(levels-1). */
typedef struct fcm_unet fcm_unet;
typedef struct {
    int in_ch, out_ch, base, levels;
    uint64_t seed;            /* SplitMix64 seed of the Kaiming-uniform initial weights */
} fcm_unet_desc;

fcm_status fcm_unet_create(const fcm_unet_desc *desc, void *cuda_stream, fcm_unet **out);
/* Number of parameters (all weights then all biases, layer by layer). */
fcm_status fcm_unet_params(const fcm_unet *net, int64_t *count);
/* Copy the FP32 master parameters (and, if g_host != NULL, their gradients) to host memory. */
fcm_status fcm_unet_get(fcm_unet *net, float *w_host, float *g_host);
/* Replace the FP32 master parameters from host memory (BF16 copies are refreshed). */
fcm_status fcm_unet_set(fcm_unet *net, const float *w_host);
/* out_dev[batch][out_ch][nz][ny][nx] = U-Net(in_dev[batch][in_ch][nz][ny][nx]); keeps the activations
 * for a following fcm_unet_backward. */
fcm_status fcm_unet_forward(fcm_unet *net, const float *in_dev, int batch, int nx, int ny, int nz, float *out_dev);
/* Back-propagates dL/d(out) of the last forward: accumulates parameter gradients; writes
 * dL/d(in) to din_dev unless it is NULL. */
fcm_status fcm_unet_backward(fcm_unet *net, const float *dout_dev, float *din_dev);
fcm_status fcm_unet_zero_grad(fcm_unet *net);
/* One Adam step (Kingma & Ba 2015) on the FP32 master parameters; step counts from 1. */
fcm_status fcm_unet_adam(fcm_unet *net, float lr, float beta1, float beta2, float eps, int step);
void fcm_unet_destroy(fcm_unet *net);

/* Restriction of a lattice vector to the cell grid: cells_dev[c][cell] = s * mean of
 * v at the (up to 8) vertex nodes of the cell, component c (3 x n_cells floats, cell
 * index x fastest).  With eta_channel != 0 a 4th channel receives eta_T of each cell.
 * The transpose of fcm_coarse_prolong up to the factor s. */
fcm_status fcm_coarse_restrict(fcm_ctx *ctx, const double *v_dev, float s, int eta_channel, float *cells_dev);
/* Prolongation: y_dev (lattice) = s * P cells_dev, where P puts on each free vertex DOF
 * 1/8 of the sum of the cell values of the cells that contain the vertex; higher-order
 * DOFs get 0. */
fcm_status fcm_coarse_prolong(fcm_ctx *ctx, const float *cells_dev, double s, double *y_dev);

/* Galerkin coarse operator on the cell grid: y_cells = K_H x_cells with
 * K_H = P^T K P (P as in fcm_coarse_prolong, K the FCM stiffness of Sec. 2).
 * Cell vectors are 3 * n_cells floats, component-major (a * n_cells + cell).
 * K_H is assembled on the first call by probing K with 375 coloured cell
 * vectors (each cell couples with the cells of its 5x5x5 neighbourhood) and
 * is kept in FP32 on the context (n_cells * 125 * 9 floats).  Returns
 * FCM_ENOMEM if it does not fit. */
fcm_status fcm_coarse_apply(fcm_ctx *ctx, const float *x_cells_dev, float *y_cells_dev);

/* Flexible PCG with a coarse correction: z = S r + P y, S the Additive-Schwarz
 * operator (Eq. (5)) and y an approximation of K_H^-1 R r.  y starts from the
 * U-Net's prediction gamma sigma N(R r / sigma, eta) (sigma the RMS of R r;
 * zero when net is NULL) and is refined by coarse_iters steps of CG on K_H,
 * preconditioned as fcm_coarse_set_preconditioner chose (block Jacobi by
 * default, or the cell-grid multigrid cycle) (coarse_iters = 0: the prediction
 * alone; net == NULL needs coarse_iters >= 1).  Without a network, and where
 * K_H exceeds the 129 MB L2, R r and the coarse solve run on a second stream
 * beside the Schwarz apply.  Since z depends nonlinearly on r, every new direction
 * is K-orthogonalised against the previous four (truncated flexible CG,
 * FCG(4), Notay 2000).  Convergence is tested on the plain Schwarz residual
 * ||S r|| / ||S b|| <= tol (Eq. (14)).  When the stopping residual grows
 * 100-fold over its best value, has not halved within the stall window
 * (100 iterations unless set by fcm_fpcg_set_stall_window), or a
 * scalar breaks down, the solve falls back to plain Schwarz-PCG on the
 * remaining residual, from the current iterate (fcm_last_solve reports it).
 * iterations counts K applications of both phases on the fine lattice.
 * Returns FCM_EINVAL on bad arguments, FCM_ESTATE before fcm_precond_build,
 * FCM_ENOTCONV when maxit is reached. */
fcm_status fcm_fpcg_solve(fcm_ctx *ctx, fcm_unet *net, double gamma, int coarse_iters, const double *rhs_dev,
                          double tol, int maxit, double *u_dev, int *iterations, double *final_relres);

/* Stall window of fcm_fpcg_solve: the flexible phase gives way to plain
 * Schwarz-PCG when the stopping residual has not halved within this many
 * iterations (default 100).  The stopping residual of CG is not monotone, so on
 * slowly converging problems a longer window keeps the coarse correction in
 * use through plateaus.  Returns FCM_EINVAL for window < 1. */
fcm_status fcm_fpcg_set_stall_window(fcm_ctx *ctx, int window);

/* Preconditioner of the coarse CG inside fcm_fpcg_solve.
 *   FCM_COARSE_JACOBI (the default): the inverses of the 3x3 diagonal blocks of K_H.
 *   FCM_COARSE_VCYCLE: one V-cycle of a geometric multigrid hierarchy on the cell grid.  Level l+1
 *     halves the cells of level l along every axis with more than one cell (n' = (n + 1) / 2); the
 *     interpolation P2 is cell-centred trilinear (3/4 from the coarse cell containing the fine one,
 *     1/4 from its neighbour on the fine cell's side, all of it at the boundary); K_{l+1} =
 *     P2^T K_l P2, assembled on the device by probing like K_H; one block-Jacobi step damped by
 *     4 / (3.3 lambda_max(D^-1 K_l)) before and one after the coarse correction; the coarsest level
 *     (at most 512 cells) by its dense pseudo-inverse (eigenvalues below 1e-12 of the largest
 *     dropped).  The cycle is a fixed symmetric linear operator, so the coarse CG stays a
 *     preconditioned CG.  Not part of the paper's method: a coarse space for its Sec. 6 limitation.
 *   FCM_COARSE_HYBRID: the same hierarchy, but on the finest cell grid (level 0) the damped block-Jacobi
 *     step and the coarse correction are added, x = omega D^-1 f + P2 V_1(P2^T f), V_1 the V-cycle of
 *     the levels below: symmetric and linear too, and it applies K_H itself no more (the level-0
 *     apply is the costly one when K_H streams from HBM).
 * The hierarchy is built on the first coarse solve after the choice (FCM_ENOMEM if it does not fit).
 * Changing the choice drops the flexible CG's captured graph.  FCM_EINVAL for another kind. */
#define FCM_COARSE_JACOBI 0
#define FCM_COARSE_VCYCLE 1
#define FCM_COARSE_HYBRID 2
fcm_status fcm_coarse_set_preconditioner(fcm_ctx *ctx, int kind);

/* Storage of K_H on its own cell grid, used by every K_H product (fcm_coarse_apply, the coarse CG and
 * the finest level of the cycles; the coarser levels are built from the FP32 operator and stay FP32):
 *   FCM_COARSE_STORE_FP32 (the default): the 63 stored 3x3 blocks per cell in FP32, 2,268 B per cell;
 *   FCM_COARSE_STORE_FP16: symmetrically scaled, K~_cj = s_c K_cj s_j with s_c = (tr K_cc / 3)^(-1/2),
 *     in FP16 rounded to nearest, 1,134 B per cell (+ 4 B for s).  For the positive semi-definite K_H
 *     every scaled entry is at most 3 in magnitude, so FP16 keeps 11 significant bits of each entry
 *     above 6e-5 and an absolute 3e-8 below: a perturbation of K_H of relative size ~5e-4 in the scaled
 *     norm, which the coarse part of the flexible CG's preconditioner tolerates; the copy halves the
 *     bytes of each product where K_H streams from HBM.
 *   FCM_COARSE_STORE_FP16_CYCLES: the FP16 copy only in the V-cycle's residual and smoothing products on
 *     the finest cell grid; the coarse CG's own products and fcm_coarse_apply stay FP32.
 * The FP16 copy is made on the next coarse call (FCM_ENOMEM if it does not fit); changing the storage
 * drops the flexible CG's captured graph.  FCM_EINVAL for another value. */
#define FCM_COARSE_STORE_FP32 0
#define FCM_COARSE_STORE_FP16 1
#define FCM_COARSE_STORE_FP16_CYCLES 2
fcm_status fcm_coarse_set_storage(fcm_ctx *ctx, int storage);

/* The multigrid hierarchy after it is built: *levels (0 before), the cell grid of each level in
 * dims[3 * l + axis] (room for 3 * 12 ints, may be null), the smoother's lambda_max estimate per
 * level but the last in lambdas (room for 12, may be null) and the build time in *seconds (may be
 * null). */
fcm_status fcm_coarse_levels(fcm_ctx *ctx, int *levels, int *dims, double *lambdas, double *seconds);

/* x_cells_dev = one cycle of that hierarchy, kind FCM_COARSE_VCYCLE or FCM_COARSE_HYBRID, applied to
 * f_cells_dev (cell vectors, 3 * n_cells floats, component-major, distinct device buffers), whatever
 * the coarse preconditioner in use; builds K_H and the hierarchy if needed.  Ordered on the caller's
 * stream like fcm_coarse_apply.  A fixed symmetric linear operator: on a grid of at most 512 cells it
 * is the pseudo-inverse of K_H.  FCM_EINVAL for another kind. */
fcm_status fcm_coarse_vcycle(fcm_ctx *ctx, int kind, const float *f_cells_dev, float *x_cells_dev);

/* Same as fcm_fpcg_solve with host buffers: rhs_host (n_lattice doubles) is
 * copied to the device, solved, and the solution copied back into u_host
 * before returning (pinned host memory makes the copies asynchronous DMA). */
fcm_status fcm_fpcg_solve_host(fcm_ctx *ctx, fcm_unet *net, double gamma, int coarse_iters, const double *rhs_host,
                               double tol, int maxit, double *u_host, int *iterations, double *final_relres);

/* Largest n_lattice that fcm_apply_S_noalloc accepts (8 MiB of FP64 scratch). */
#define FCM_NOALLOC_MAX_LATTICE 1048576

/* Same result as fcm_apply_S, for callers that must not allocate device
 * memory once they are running (an application whose device memory belongs
 * to its own pool allocator, or a real-time loop that forbids allocation
 * after start-up).  This call allocates nothing: its scratch vector is a
 * fixed static device array of FCM_NOALLOC_MAX_LATTICE doubles, held by
 * every GPU that loads the library until the process exits.  The paper has
 * no counterpart; it is an interface convenience.
 *   - Returns FCM_EINVAL when n_lattice > FCM_NOALLOC_MAX_LATTICE, FCM_ESTATE
 *     before fcm_precond_build.
 *   - All calls on a device share the one array; calls that overlap on the
 *     GPU (different streams or contexts) race on it.  Each call overwrites
 *     every entry it reads, so nothing needs clearing between calls.
 *   - fcm_precond_build looks the array's device address up
 *     (cudaGetSymbolAddress, with the context's device current, outside any
 *     capture) and keeps it in the context; this call only launches work.
 *     FCM_ECUDA if that lookup failed. */
fcm_status fcm_apply_S_noalloc(fcm_ctx *ctx, const double *r_dev, double *z_dev);

/* ---- Multi-level hp overlays (Sec. 2.2) and their leaf blocks (Sec. 3.2) -------------------------------
 *
 * A base grid (grid->n cells on [grid->lo, grid->hi]) refined k times toward the boundary of geom: a level-l
 * cell that the boundary crosses carries an overlay of its 8 children on level l + 1.  Crossing: spheres,
 * min distance < r < max distance from the centre; voxels (an image spanning the grid box), the voxels the
 * cell overlaps are not all equal; half space, min a.x < d < max a.x over the cell.  Every level has its own integrated-
 * Legendre basis of order p, one set of modes per topological component.  A level-l component is active iff
 * every in-domain level-l cell position around it exists (homogeneous Dirichlet conditions on the overlay's
 * boundary) and at least one of them is a leaf (covered components are deactivated).
 *
 * Blocks are per leaf cell (Sec. 3.2 "Selecting suitable blocks"):
 *   kind 0, full: every active scalar function supported on the leaf;
 *   kind 1, truncated: the leaf's own-level functions plus, for each corner whose own-level vertex function
 *           is inactive, the vertex function of the highest coarser level at which the corner point is an
 *           active vertex.  No scalar function is in more than 2^3 truncated blocks.
 * Scalar function f carries 3 displacement DOFs.  Orders: functions level by level, components (doubled
 * coordinates: even = on a grid plane, odd = inside a cell interval) sorted by (z, y, x), modes with the
 * bubble index of the lowest odd axis slowest; leaves by level, then (x, y, z) lexicographically.
 *
 * The plan, the assembled system and the factors live in host memory; fcm_mlhp_device_setup adds a device
 * copy for the K and S applies and the PCG.  The library owns everything until fcm_mlhp_destroy.  Device
 * calls return FCM_ECUDA when a CUDA call fails. */
typedef struct fcm_mlhp fcm_mlhp;
typedef struct {
    int levels;                 /* levels of the hierarchy, 1 = the base grid only */
    int64_t n_leaves;           /* leaf cells over all levels */
    int64_t n_functions;        /* active scalar functions, full tensor-product modes */
    int64_t n_functions_trunk;  /* the same in the trunk space (face and cell bubble indices sum to <= p) */
    int n_max_full;             /* most full blocks one scalar function belongs to (over all leaves) */
    int n_max_truncated;        /* the same for truncated blocks */
    int max_block_full;         /* most scalar functions in one full block */
    int max_block_truncated;    /* the same for truncated blocks */
} fcm_mlhp_info;

/* Build the plan.  1 <= p <= 4, 0 <= k <= 10, grid->n[a] << k < 2^20.  FCM_EINVAL on bad arguments,
 * FCM_ENOMEM when host memory runs out. */
fcm_status fcm_mlhp_create(const fcm_grid *grid, const fcm_geometry *geom, int p, int k, fcm_mlhp **out);
fcm_status fcm_mlhp_get_info(const fcm_mlhp *plan, fcm_mlhp_info *info);
/* Level and cell index (on the level's grid of n * 2^level cells) of leaf `leaf`. */
fcm_status fcm_mlhp_leaf(const fcm_mlhp *plan, int64_t leaf, int *level, int cell[3]);
/* Level, component (doubled coordinates on the level's grid) and mode of scalar function f: mode[a] is 0
 * on an axis where the component is a vertex coordinate (linear factor), else the bubble index 2..p. */
fcm_status fcm_mlhp_function(const fcm_mlhp *plan, int64_t f, int *level, int comp[3], int mode[3]);
/* Scalar functions of leaf `leaf`'s block (kind 0 full, 1 truncated) into fids[0 .. *count).  *count is
 * always set; FCM_EINVAL (nothing copied) when it exceeds cap. */
fcm_status fcm_mlhp_block(const fcm_mlhp *plan, int64_t leaf, int kind, int64_t *fids, int cap, int *count);
/* Colour classes of the leaf blocks (kind 0 full, 1 truncated): colour[n_leaves] such that two leaves of one
 * colour share no scalar function, so a launch per colour can scatter without atomics.  Greedy in leaf
 * order.  Truncated blocks take about 13 colours on refined hierarchies (8 on a uniform grid); full blocks
 * need at least n_max_full colours, and FCM_EINVAL is returned beyond 64. */
fcm_status fcm_mlhp_colour(const fcm_mlhp *plan, int kind, int *colour, int *n_colours);
/* Function f restricted to leaf `leaf` (f must be supported there: FCM_EINVAL otherwise) is the tensor
 * product over the axes a of sum_j coef[a (p+1) + j] b_j(t_a), with b = (N0, N1, phi_2 .. phi_p) the
 * leaf's own 1D shape functions in its local coordinate t_a in [-1, 1]. */
fcm_status fcm_mlhp_restriction(const fcm_mlhp *plan, int64_t leaf, int64_t f, double *coef);
/* Assemble the elasticity system of Eq. (1) on the hierarchy (host memory), with the plan's geometry
 * (alpha in the void) and its octree_depth, material and conditions from bc (FCM_BC_* as for
 * fcm_setup; Dirichlet DOFs are removed: a function is fixed in component a when its component lies on the
 * plane of that condition), and the traction bc->traction on the top face z = hi[2].  Each leaf with eta > 0
 * contributes C K_cell C^T, with K_cell the cell matrix of the leaf's box (the same moment quadrature as
 * fcm_setup, octree depth counted from the leaf) and C the restriction above; a function is kept when some
 * leaf in its support has eta > 0.  FCM_EINVAL on bad arguments (alpha in (0, 1]). */
fcm_status fcm_mlhp_assemble(fcm_mlhp *plan, double alpha, const fcm_bc *bc);
/* Sizes of the assembled system: free DOFs and CSR nonzeros.  FCM_ESTATE before fcm_mlhp_assemble. */
fcm_status fcm_mlhp_system_size(const fcm_mlhp *plan, int64_t *n_free, int64_t *nnz);
/* Copy the assembled system to caller-owned host arrays (any may be NULL): free_dofs[n_free] (3 f + comp,
 * ascending), the CSR rowptr[n_free + 1], cols[nnz], vals[nnz] over the free DOFs, the load rhs[n_free] and
 * the volume fraction of every leaf leaf_eta[n_leaves]. */
fcm_status fcm_mlhp_system(const fcm_mlhp *plan, int64_t *free_dofs, int64_t *rowptr, int64_t *cols, double *vals,
                           double *rhs, double *leaf_eta);
/* Schwarz factors of the assembled system (Sec. 3.2, Algorithm 1), on the host: one block per leaf with
 * 0 < eta_T <= eta_bar (eta_T clamped to 1; eta_bar in [0, 1], 1 = every leaf), holding the free DOFs of the
 * leaf's functions (kind 0 full, 1 truncated); its pseudo inverse A_B^+ (eigenpairs with lambda > eps
 * lambda_max of the block, Eq. (13); cyclic Jacobi eigen-decomposition); and 1 / K_ll for free DOFs in no
 * block.  Blocks are coloured greedily (no two blocks of one colour share a DOF) and stored
 * colour by colour.  Host time grows as the cube of the block size: meant for truncated blocks.
 * FCM_ESTATE before fcm_mlhp_assemble. */
fcm_status fcm_mlhp_factorize(fcm_mlhp *plan, int kind, double eps, double eta_bar);
/* fcm_mlhp_factorize with the blocks' eigensolves on the current CUDA device: the blocks are formed on the
 * host as there, then solved by batched FP64 eigensolves (cuSOLVER, one batch per block size) on
 * cuda_stream, with the same Eq. (13) cut-off and the same pseudo inverse up to the two eigensolvers'
 * rounding; the factors land in host memory as with fcm_mlhp_factorize.  FCM_ECUDA (message in
 * fcm_mlhp_last_error) when a device call fails, FCM_ENOMEM when memory runs out. */
fcm_status fcm_mlhp_factorize_device(fcm_mlhp *plan, int kind, double eps, double eta_bar, void *cuda_stream);
fcm_status fcm_mlhp_factor_info(const fcm_mlhp *plan, int *n_blocks, int *n_colours, int64_t *factor_entries);
/* Copy the factors to caller-owned host arrays (any may be NULL): blk_ptr[n_blocks + 1] and blk_dofs (free
 * DOF indices of block b in blk_dofs[blk_ptr[b] .. blk_ptr[b+1]), ascending), fac_ptr[n_blocks + 1] and
 * factors (A_B^+ of block b, row-major, at factors[fac_ptr[b]]), colour_ptr[n_colours + 1] (blocks of colour
 * c are colour_ptr[c] .. colour_ptr[c+1]) and jacobi[n_free] (0 on DOFs inside blocks). */
fcm_status fcm_mlhp_factors(const fcm_mlhp *plan, int64_t *blk_ptr, int64_t *blk_dofs, int64_t *fac_ptr, double *factors,
                            int64_t *colour_ptr, double *jacobi);
/* Upload the assembled system and the factors to the current device (after fcm_mlhp_factorize, else
 * FCM_ESTATE); every index is checked on the host first (FCM_EINVAL).  The device arrays belong to the plan
 * until fcm_mlhp_destroy or the next assemble / factorize.  Work is queued on cuda_stream. */
fcm_status fcm_mlhp_device_setup(fcm_mlhp *plan, void *cuda_stream);
/* Factor storage of the next fcm_mlhp_device_setup: FCM_PREC_FP64 (the default; every factor as a float
 * pair, FP64 accuracy) or FCM_PREC_MIXED (FP32 for the blocks whose retained condition number
 * lambda_max / lambda_min is at most 1e7, as on the uniform grid: half the bytes, products within 2^-24 of
 * the factor's magnitude; float pairs for the others).  FCM_EINVAL for another value. */
fcm_status fcm_mlhp_set_precision(fcm_mlhp *plan, int precision);
/* After fcm_mlhp_device_setup (else FCM_ESTATE): blocks stored in FP32 and the device factor bytes. */
fcm_status fcm_mlhp_device_info(const fcm_mlhp *plan, int64_t *n_fp32_blocks, int64_t *factor_bytes);
/* y_dev = K x_dev over the free DOFs (device arrays of n_free doubles): x split into float pairs, then one
 * warp per CSR row in double-float arithmetic (values stored as float pairs, 2^-48 relative), each entry
 * of y within 2^-43 (|K| |x|) of the exact product.  x_dev and y_dev must differ (FCM_EINVAL): warps
 * write y while others still read x. */
fcm_status fcm_mlhp_apply_K(fcm_mlhp *plan, const double *x_dev, double *y_dev);
/* z_dev = S r_dev (Eq. (5)) in two launches: every block's product A_B^+ r_B into a slot of its own
 * (double-float arithmetic on float-pair factors), then per DOF the diagonal part plus the slots of the
 * blocks containing it in block order (deterministic, no atomics).  r_dev and z_dev must differ. */
fcm_status fcm_mlhp_apply_S(fcm_mlhp *plan, const double *r_dev, double *z_dev);
/* PCG on K u = b (x0 = 0), stopped when ||S r_i|| / ||S b|| <= tol (Eq. (14)) or after maxit iterations;
 * *iterations counts the K applications.  The scalars stay on the device (deterministic reductions);
 * eight iterations per captured CUDA graph on the plan's own stream, ordered after cuda_stream of
 * fcm_mlhp_device_setup.  FCM_OK, FCM_ENOTCONV (u = the last iterate), FCM_EBREAKDOWN (p.Kp <= 0 or a
 * non-finite scalar).  Synchronises the stream. */
fcm_status fcm_mlhp_pcg_solve(fcm_mlhp *plan, const double *b_dev, double tol, int maxit, double *u_dev, int *iterations,
                              double *relres);
/* Message of the last failed device call on the plan (fcm_mlhp_device_setup, the applies, the PCG): the
 * CUDA error or the rejected input; "" when none.  Device set-up returns FCM_ENOMEM when an allocation
 * fails, FCM_ECUDA for other CUDA failures and FCM_EINVAL for a rejected index. */
const char *fcm_mlhp_last_error(const fcm_mlhp *plan);
void fcm_mlhp_destroy(fcm_mlhp *plan);

/* Message of the last failure on ctx (ctx may be NULL for setup failures). */
const char *fcm_last_error(const fcm_ctx *ctx);

/* Release every device and host resource of ctx (NULL is a no-op). */
void fcm_destroy(fcm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FCM_H */
