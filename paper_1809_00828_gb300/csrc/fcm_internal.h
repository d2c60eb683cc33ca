// Internal declarations of libfcm (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fcm.h"

namespace fcm {

// Host-side description of a set-up finite cell problem.  Produced by
// build_host_problem() from the ABI inputs; uploaded to the device by the
// context.  Lattice layout as documented in fcm.h.
struct HostProblem {
    // grid, order, material
    int n[3];
    double lo[3], hi[3], h[3];
    int p;
    double alpha;
    double E, nu;
    int bc;
    double traction[3];
    // geometry
    int gkind;
    std::vector<double> sph;       // 4 per sphere
    int vdim[3];
    std::vector<uint8_t> vox;
    double plane[4];
    int depth;
    // sizes
    int M[3];
    int64_t nnodes, nlat;
    int ne;                         // 3 (p+1)^3, rows of an element matrix
    int64_t ncells;
    // results
    std::vector<int32_t> cell_elem; // -1 inactive, 0 uncut (reference matrix), 1+k k-th cut cell
    std::vector<double> eta;        // volume fraction per cell
    std::vector<double> Kref;       // ne x ne
    std::vector<double> Kcut;       // ncut x ne x ne (released once uploaded)
    std::vector<double> kdiag;      // diagonal of K per lattice DOF (sum over the active cells)
    int64_t ncut = 0;
    int64_t nactive = 0;
    std::vector<uint8_t> mask;      // per lattice DOF: 1 = free
    int64_t nfree = 0;
    std::vector<double> rhs;        // load case 0, lattice layout
    std::vector<double> rhs_strain; // load cases 1..6 (unit Voigt strains), 6 x nlat
};

// 1D tables for the sum-factorised stiffness apply of an uncut cell: shape
// functions and their physical derivatives at the p+1 Gauss points of each
// axis (exact for the uncut integrand, whose degree is <= 2p per axis).
struct SfTables {
    double B[5][5];     // B[q][i] = f_i(xi_q)
    double D[3][5][5];  // D[a][q][i] = f_i'(xi_q) * 2 / h_a
    double G[3][5][5];  // G[a][q][k] = l_k'(xi_q) * 2 / h_a, l_k the Lagrange polynomials through the Gauss points
    double W[5];        // Gauss weights on [-1, 1]
    double detJ;        // h_0 h_1 h_2 / 8
    double lam, mu;     // Lame parameters
};
void make_sf_tables(const HostProblem &P, SfTables &T);

// Builds everything on the host.  Returns an empty string on success, else
// the error message.  nthreads <= 0 uses the hardware concurrency.
std::string build_host_problem(const fcm_grid &grid, const fcm_geometry &geom, int p, double alpha,
                               const fcm_bc &bc, HostProblem &out, int nthreads = 0);

// One cell on the box [clo, chi] with the grid cells' moment quadrature (octree depth counted from the
// cell): alpha-weighted element matrix K (3 (p+1)^3 square, lattice order), volume fraction eta and, if
// face != nullptr, the solid-part integrals face[i1 (p+1) + i0] of N_i0 N_i1 over the top face z = chi[2].
// Voxel images span the domain box [dlo, dhi].
void box_cell_setup(const fcm_geometry &geom, const double *dlo, const double *dhi, int p, double alpha, double E,
                    double nu, const double *clo, const double *chi, double *K, double *eta, double *face);

// The multi-level system on the device (fcm_mlhp_device.cu): CSR K over the free DOFs, the Schwarz blocks
// (free-DOF lists, row-major pseudo inverses, colour ranges) and the diagonal part.  create() checks every
// index on the host, uploads and synchronises; the vectors of the other calls are device arrays of n.
struct MlhpDevice;
// fac_cond (may be null): the blocks whose retained condition number is at most 1e7 keep FP32 factors.
std::string mlhp_device_create(void *stream, int64_t n, const int64_t *rowptr, const int64_t *cols, const double *vals,
                               int64_t nblocks, const int64_t *bptr, const int64_t *bdofs, const int64_t *fptr,
                               const double *fac, int ncolours, const int64_t *cptr, const double *jac,
                               const double *fac_cond, MlhpDevice **out);
void mlhp_device_info(const MlhpDevice *d, int64_t *n_fp32_blocks, int64_t *factor_bytes);
// Pseudo inverses of nblocks symmetric blocks (A: row-major m_b x m_b at fac_ptr[b]) by batched eigensolves
// on the device (stream), eigenvalues below eps * lambda_max dropped (Eq. (13)); F as A, cond[b] the retained
// condition number.  "" on success, else the failure.
std::string mlhp_device_pinv(void *stream, int64_t nblocks, const int64_t *fac_ptr, const double *A, double eps,
                             double *F, double *cond);
void mlhp_device_destroy(MlhpDevice *d);
std::string mlhp_device_apply_K(MlhpDevice *d, const double *x, double *y);
std::string mlhp_device_apply_S(MlhpDevice *d, const double *r, double *z);
// status: 0 converged, 1 not converged within maxit, 2 breakdown.
std::string mlhp_device_pcg(MlhpDevice *d, const double *b, double tol, int maxit, double *u, int *its, double *relres,
                            int *status);

// Gauss-Legendre rule with n points on [-1, 1].
void gauss_legendre(int n, double *x, double *w);

}  // namespace fcm
