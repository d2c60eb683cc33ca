/*
 * fcm_oracle.c -- plain FP64 CPU oracle for the finite cell Additive-Schwarz PCG.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU baseline may load this library.  It shares no code with the GPU path.
 *
 * What it computes (Jomo et al., "Robust and parallel scalable iterative
 * solutions for large-scale finite cell analyses", arXiv:1809.00828):
 *   - Sec. 2.1, Eq. (1): the finite cell weak form of linear elasticity with the
 *     indicator alpha (1 in the physical domain, 0 < alpha << 1 outside).
 *   - Sec. 3.2 (footnote on the full tensor product space): integrated
 *     Legendre shape functions of order p, (p+1)^3 per cell and component.
 *   - Sec. 5.1 problem setup: octree partitioning of cut cells to a fixed
 *     depth relative to the cell size for the numerical integration.
 *   - Sec. 3.2 Eq. (10): the volume fraction eta_T of a cell.
 *   - Sec. 3.1 Eq. (5): the Additive-Schwarz operator S = sum_B R_B^T A_B^-1 R_B.
 *   - Sec. 3.2 Eqs. (11)-(13): the eigenvalue-filtered pseudo inverse with
 *     lambda_tres = eps * max_k lambda_k.
 *   - Algorithm 1: blocks, extraction, pseudo inverse, prolongation, and the
 *     diagonal (Jacobi) scaling of functions that are in no block.
 *   - Sec. 5, Eq. (14): the relative preconditioned residual ||S r_i|| / ||S b||
 *     as the stopping measure; Eq. (15): the relative energy-norm error.
 *
 * Readings where the paper is silent (binding for both paths):
 *   - A (sub)cell is cut when the geometry boundary crosses it; cut boxes are
 *     split into 8 until the octree depth; every leaf (cut or not) gets a
 *     (p+1)^3 Gauss-Legendre rule with alpha evaluated at each point.
 *   - A cell is active iff eta_T > 0; inactive cells are removed.
 *   - phi_j = (P_j - P_{j-2}) / sqrt(2(2j-1)), j = 2..p (integrated Legendre).
 *   - Vertex-patch blocks: the functions carried by the vertex v and by every
 *     edge, face and cell whose closure contains v.
 *   - Dirichlet conditions are imposed strongly on the grid-aligned faces.
 *   - The traction acts on the top face (z = hi) of the active cells where it
 *     lies in the physical domain, integrated by a quadtree of the same depth.
 *
 * Numbering: lattice nodes (i,j,k), i,j,k = 0..p*n, i along x fastest;
 * DOF = 3*node + component.  Along an axis, cell c owns lattice indices
 * p*c .. p*c+p: p*c is its left vertex (N0), p*c+p its right vertex (N1),
 * p*c+a (1 <= a <= p-1) the integrated Legendre function phi_{a+1}.
 * The oracle numbers its free DOFs in increasing lattice DOF order.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n[3];
    double lo[3], hi[3];
    int p;
    int depth;
    double alpha, E, nu;
    int bc;              /* -1 none, 0 clamp all components on z=lo, 1 rollers on x=lo,y=lo,z=lo */
    double traction[3];
    int gkind;           /* 0 spherical voids, 1 voxels, 2 half-space */
    int nsph;
    const double *sph;   /* nsph x (cx, cy, cz, r) */
    int vdim[3];
    const unsigned char *vox; /* vdim[0] fastest */
    double plane[4];     /* solid iff a x + b y + c z < d */
} ora_desc;

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1] by Newton iteration on P_n.           */
/* ------------------------------------------------------------------ */
static void legendre_and_derivative(int n, double x, double *pn, double *dpn)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    *pn = p1;
    /* (x^2 - 1) P_n'(x) = n (x P_n - P_{n-1}) */
    *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

int ora_gauss(int n, double *x, double *w)
{
    if (n < 1 || n > 64) return -1;
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, dpn;
            legendre_and_derivative(n, t, &pn, &dpn);
            double dt = pn / dpn;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double pn, dpn;
        legendre_and_derivative(n, t, &pn, &dpn);
        x[n - 1 - i] = t;
        w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dpn * dpn);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 1D shape functions in lattice order: f_0 = N0, f_p = N1, f_a = phi_{a+1}. */
/* ------------------------------------------------------------------ */
void ora_shape1d(int p, double xi, double *f, double *df)
{
    double P[32], dP[32];
    P[0] = 1.0; dP[0] = 0.0;
    P[1] = xi;  dP[1] = 1.0;
    for (int k = 2; k <= p; ++k) {
        P[k] = ((2.0 * k - 1.0) * xi * P[k - 1] - (k - 1.0) * P[k - 2]) / k;
        dP[k] = dP[k - 2] + (2.0 * k - 1.0) * P[k - 1];
    }
    f[0] = 0.5 * (1.0 - xi); df[0] = -0.5;
    f[p] = 0.5 * (1.0 + xi); df[p] = 0.5;
    for (int a = 1; a <= p - 1; ++a) {
        int j = a + 1;
        double s = 1.0 / sqrt(2.0 * (2.0 * j - 1.0));
        f[a] = (P[j] - P[j - 2]) * s;
        df[a] = (dP[j] - dP[j - 2]) * s;
    }
}

/* ------------------------------------------------------------------ */
/* Geometry: pointwise indicator and the "boundary crosses box" test.  */
/* ------------------------------------------------------------------ */
static int vox_index(const ora_desc *d, int ax, double x)
{
    double t = (x - d->lo[ax]) / (d->hi[ax] - d->lo[ax]) * d->vdim[ax];
    int i = (int)floor(t);
    if (i < 0) i = 0;
    if (i >= d->vdim[ax]) i = d->vdim[ax] - 1;
    return i;
}

int ora_solid_at(const ora_desc *d, const double *x)
{
    if (d->gkind == 0) {
        for (int s = 0; s < d->nsph; ++s) {
            const double *c = d->sph + 4 * s;
            double dx = x[0] - c[0], dy = x[1] - c[1], dz = x[2] - c[2];
            if (dx * dx + dy * dy + dz * dz < c[3] * c[3]) return 0;
        }
        return 1;
    } else if (d->gkind == 1) {
        int i = vox_index(d, 0, x[0]), j = vox_index(d, 1, x[1]), k = vox_index(d, 2, x[2]);
        return d->vox[i + (size_t)d->vdim[0] * (j + (size_t)d->vdim[1] * k)] != 0;
    } else {
        return d->plane[0] * x[0] + d->plane[1] * x[1] + d->plane[2] * x[2] < d->plane[3];
    }
}

int ora_box_cut(const ora_desc *d, const double *blo, const double *bhi)
{
    if (d->gkind == 0) {
        for (int s = 0; s < d->nsph; ++s) {
            const double *c = d->sph + 4 * s;
            double dmin2 = 0.0, dmax2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double e = 0.0;
                if (c[a] < blo[a]) e = blo[a] - c[a];
                else if (c[a] > bhi[a]) e = c[a] - bhi[a];
                dmin2 += e * e;
                double f = fmax(fabs(c[a] - blo[a]), fabs(c[a] - bhi[a]));
                dmax2 += f * f;
            }
            double r2 = c[3] * c[3];
            if (dmin2 < r2 && r2 < dmax2) return 1;
        }
        return 0;
    } else if (d->gkind == 1) {
        int i0[3], i1[3];
        for (int a = 0; a < 3; ++a) {
            double h = (d->hi[a] - d->lo[a]) / d->vdim[a];
            i0[a] = (int)floor((blo[a] - d->lo[a]) / h);
            i1[a] = (int)ceil((bhi[a] - d->lo[a]) / h) - 1;
            if (i1[a] < i0[a]) i1[a] = i0[a];
            if (i0[a] < 0) i0[a] = 0;
            if (i1[a] > d->vdim[a] - 1) i1[a] = d->vdim[a] - 1;
            if (i0[a] > d->vdim[a] - 1) i0[a] = d->vdim[a] - 1;
        }
        int first = -1;
        for (int k = i0[2]; k <= i1[2]; ++k)
            for (int j = i0[1]; j <= i1[1]; ++j)
                for (int i = i0[0]; i <= i1[0]; ++i) {
                    int v = d->vox[i + (size_t)d->vdim[0] * (j + (size_t)d->vdim[1] * k)] != 0;
                    if (first < 0) first = v;
                    else if (v != first) return 1;
                }
        return 0;
    } else {
        double mn = 0.0, mx = 0.0;
        for (int a = 0; a < 3; ++a) {
            double u = d->plane[a] * blo[a], v = d->plane[a] * bhi[a];
            mn += fmin(u, v);
            mx += fmax(u, v);
        }
        return mn < d->plane[3] && d->plane[3] < mx;
    }
}

/* ------------------------------------------------------------------ */
/* Element stiffness of one cell by octree quadrature:                 */
/*   K_e = sum_q w_q alpha(x_q) B_q^T D B_q,  eta_T = sum_q w_q [solid] / |T|. */
/* ------------------------------------------------------------------ */
typedef struct {
    const ora_desc *d;
    double clo[3], h[3];
    int nloc, ndof;
    double gx[64], gw[64];
    double D[6][6];
    double *K;          /* ndof x ndof, or NULL */
    double *Fs;         /* 6 x ndof unit-strain loads, or NULL */
    double solid_vol;
    /* scratch */
    double *B;          /* 6 x ndof */
    double *DB;         /* 6 x ndof */
} cell_integrator;

static void material_D(double E, double nu, double D[6][6])
{
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = E / (2.0 * (1.0 + nu));
    memset(D, 0, sizeof(double) * 36);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i][j] = lam;
    for (int i = 0; i < 3; ++i) D[i][i] = lam + 2.0 * mu;
    for (int i = 3; i < 6; ++i) D[i][i] = mu;
}

static void leaf_quadrature(cell_integrator *ci, const double *blo, const double *bhi)
{
    const ora_desc *d = ci->d;
    int p = d->p, q = p + 1;
    double vol = (bhi[0] - blo[0]) * (bhi[1] - blo[1]) * (bhi[2] - blo[2]);
    double f[3][32], df[3][32];
    for (int kz = 0; kz < q; ++kz)
        for (int ky = 0; ky < q; ++ky)
            for (int kx = 0; kx < q; ++kx) {
                double x[3], xi[3];
                int k3[3] = {kx, ky, kz};
                for (int a = 0; a < 3; ++a) {
                    x[a] = blo[a] + 0.5 * (bhi[a] - blo[a]) * (ci->gx[k3[a]] + 1.0);
                    xi[a] = 2.0 * (x[a] - ci->clo[a]) / ci->h[a] - 1.0;
                }
                double w = ci->gw[kx] * ci->gw[ky] * ci->gw[kz] * vol / 8.0;
                int solid = ora_solid_at(d, x);
                ci->solid_vol += w * solid;
                if (!ci->K && !ci->Fs) continue;
                double al = solid ? 1.0 : d->alpha;
                for (int a = 0; a < 3; ++a) ora_shape1d(p, xi[a], f[a], df[a]);
                /* B: 6 x ndof, Voigt order xx, yy, zz, yz, xz, xy (engineering shears) */
                memset(ci->B, 0, sizeof(double) * 6 * ci->ndof);
                for (int iz = 0; iz <= p; ++iz)
                    for (int iy = 0; iy <= p; ++iy)
                        for (int ix = 0; ix <= p; ++ix) {
                            int I = ix + q * (iy + q * iz);
                            double gxv = df[0][ix] * (2.0 / ci->h[0]) * f[1][iy] * f[2][iz];
                            double gyv = f[0][ix] * df[1][iy] * (2.0 / ci->h[1]) * f[2][iz];
                            double gzv = f[0][ix] * f[1][iy] * df[2][iz] * (2.0 / ci->h[2]);
                            int cx = 3 * I, cy = 3 * I + 1, cz = 3 * I + 2;
                            int n = ci->ndof;
                            ci->B[0 * n + cx] = gxv;
                            ci->B[1 * n + cy] = gyv;
                            ci->B[2 * n + cz] = gzv;
                            ci->B[3 * n + cy] = gzv; ci->B[3 * n + cz] = gyv;
                            ci->B[4 * n + cx] = gzv; ci->B[4 * n + cz] = gxv;
                            ci->B[5 * n + cx] = gyv; ci->B[5 * n + cy] = gxv;
                        }
                int n = ci->ndof;
                for (int r = 0; r < 6; ++r)
                    for (int j = 0; j < n; ++j) {
                        double s = 0.0;
                        for (int t = 0; t < 6; ++t) s += ci->D[r][t] * ci->B[t * n + j];
                        ci->DB[r * n + j] = s;
                    }
                double wa = w * al;
                /* unit-strain load k: -(B^T D e_k) = -(D B)[k][.] since D is symmetric */
                if (ci->Fs)
                    for (int k = 0; k < 6; ++k)
                        for (int i = 0; i < n; ++i) ci->Fs[k * n + i] -= wa * ci->DB[k * n + i];
                if (!ci->K) continue;
                for (int i = 0; i < n; ++i)
                    for (int j = i; j < n; ++j) {
                        double s = 0.0;
                        for (int t = 0; t < 6; ++t) s += ci->B[t * n + i] * ci->DB[t * n + j];
                        ci->K[(size_t)i * n + j] += wa * s;
                    }
            }
}

static void octree(cell_integrator *ci, const double *blo, const double *bhi, int level)
{
    if (level < ci->d->depth && ora_box_cut(ci->d, blo, bhi)) {
        double mid[3];
        for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (blo[a] + bhi[a]);
        for (int c = 0; c < 8; ++c) {
            double lo2[3], hi2[3];
            for (int a = 0; a < 3; ++a) {
                int up = (c >> a) & 1;
                lo2[a] = up ? mid[a] : blo[a];
                hi2[a] = up ? bhi[a] : mid[a];
            }
            octree(ci, lo2, hi2, level + 1);
        }
    } else {
        leaf_quadrature(ci, blo, bhi);
    }
}

static void cell_box(const ora_desc *d, const int *c, double *clo, double *chi, double *h)
{
    for (int a = 0; a < 3; ++a) {
        h[a] = (d->hi[a] - d->lo[a]) / d->n[a];
        clo[a] = d->lo[a] + c[a] * h[a];
        chi[a] = (c[a] + 1 == d->n[a]) ? d->hi[a] : d->lo[a] + (c[a] + 1) * h[a];
    }
}

/* Element matrix (3(p+1)^3 square, row-major, local DOF = 3*I + comp with
 * I = ix + (p+1)(iy + (p+1) iz)), the six unit-strain loads of the cell
 * Fs[k][i] = -int alpha (B^T D e_k)_i (e_k the k-th Voigt unit strain, engineering
 * shears) and the volume fraction of cell c.  Ke and Fs may be NULL. */
int ora_cell_matrix_ex(const ora_desc *d, const int *c, double *Ke, double *Fs, double *eta);

int ora_cell_matrix(const ora_desc *d, const int *c, double *Ke, double *eta)
{
    return ora_cell_matrix_ex(d, c, Ke, NULL, eta);
}

int ora_cell_matrix_ex(const ora_desc *d, const int *c, double *Ke, double *Fs, double *eta)
{
    cell_integrator ci;
    memset(&ci, 0, sizeof ci);
    ci.d = d;
    double chi[3];
    cell_box(d, c, ci.clo, chi, ci.h);
    int q = d->p + 1;
    ci.nloc = q * q * q;
    ci.ndof = 3 * ci.nloc;
    ora_gauss(q, ci.gx, ci.gw);
    material_D(d->E, d->nu, ci.D);
    ci.K = Ke;
    ci.Fs = Fs;
    if (Ke) memset(Ke, 0, sizeof(double) * ci.ndof * ci.ndof);
    if (Fs) memset(Fs, 0, sizeof(double) * 6 * ci.ndof);
    if (Ke || Fs) {
        ci.B = malloc(sizeof(double) * 6 * ci.ndof);
        ci.DB = malloc(sizeof(double) * 6 * ci.ndof);
    }
    octree(&ci, ci.clo, chi, 0);
    if (Ke)
        for (int i = 0; i < ci.ndof; ++i)
            for (int j = 0; j < i; ++j) Ke[(size_t)i * ci.ndof + j] = Ke[(size_t)j * ci.ndof + i];
    free(ci.B);
    free(ci.DB);
    if (eta) *eta = ci.solid_vol / ((chi[0] - ci.clo[0]) * (chi[1] - ci.clo[1]) * (chi[2] - ci.clo[2]));
    return ci.ndof;
}

/* ------------------------------------------------------------------ */
/* Traction load on the top face of one cell (quadtree of the same depth). */
/* ------------------------------------------------------------------ */
static void face_rec(const ora_desc *d, const double *clo, const double *h, const double *flo,
                     const double *fhi, int level, const double *gx, const double *gw, double *be)
{
    double blo[3] = {flo[0], flo[1], d->hi[2]}, bhi[3] = {fhi[0], fhi[1], d->hi[2]};
    if (level < d->depth && ora_box_cut(d, blo, bhi)) {
        double mid[2] = {0.5 * (flo[0] + fhi[0]), 0.5 * (flo[1] + fhi[1])};
        for (int c = 0; c < 4; ++c) {
            double lo2[2], hi2[2];
            for (int a = 0; a < 2; ++a) {
                int up = (c >> a) & 1;
                lo2[a] = up ? mid[a] : flo[a];
                hi2[a] = up ? fhi[a] : mid[a];
            }
            face_rec(d, clo, h, lo2, hi2, level + 1, gx, gw, be);
        }
        return;
    }
    int p = d->p, q = p + 1;
    double area = (fhi[0] - flo[0]) * (fhi[1] - flo[1]);
    double fx[32], dfx[32], fy[32], dfy[32];
    for (int ky = 0; ky < q; ++ky)
        for (int kx = 0; kx < q; ++kx) {
            double x[3];
            x[0] = flo[0] + 0.5 * (fhi[0] - flo[0]) * (gx[kx] + 1.0);
            x[1] = flo[1] + 0.5 * (fhi[1] - flo[1]) * (gx[ky] + 1.0);
            x[2] = d->hi[2];
            if (!ora_solid_at(d, x)) continue;
            double w = gw[kx] * gw[ky] * area / 4.0;
            ora_shape1d(p, 2.0 * (x[0] - clo[0]) / h[0] - 1.0, fx, dfx);
            ora_shape1d(p, 2.0 * (x[1] - clo[1]) / h[1] - 1.0, fy, dfy);
            /* on z = hi only the local functions with iz = p (N1 in z, value 1) are nonzero */
            for (int iy = 0; iy <= p; ++iy)
                for (int ix = 0; ix <= p; ++ix) {
                    int I = ix + q * (iy + q * p);
                    double v = w * fx[ix] * fy[iy];
                    for (int a = 0; a < 3; ++a) be[3 * I + a] += v * d->traction[a];
                }
        }
}

int ora_cell_traction(const ora_desc *d, const int *c, double *be)
{
    double clo[3], chi[3], h[3];
    cell_box(d, c, clo, chi, h);
    int q = d->p + 1, ndof = 3 * q * q * q;
    memset(be, 0, sizeof(double) * ndof);
    if (c[2] != d->n[2] - 1) return ndof;
    double gx[64], gw[64];
    ora_gauss(q, gx, gw);
    double flo[2] = {clo[0], clo[1]}, fhi[2] = {chi[0], chi[1]};
    face_rec(d, clo, h, flo, fhi, 0, gx, gw, be);
    return ndof;
}

/* ------------------------------------------------------------------ */
/* Global problem: active cells, free DOFs, sparse K (CSR), load b.    */
/* ------------------------------------------------------------------ */
typedef struct {
    int n, bs;           /* block count and rows of one block */
    int *idx;            /* n_B global (free) indices */
    double *F;           /* n_B x n_B pseudo inverse, row-major */
    double cond;         /* lambda_max / smallest retained lambda */
    int nneg;            /* eigenvalues <= 0 */
    int nfilt;           /* eigenvalues filtered out */
} ora_block;

typedef struct {
    ora_desc d;
    double *sph_copy;
    unsigned char *vox_copy;
    int M[3];
    int64_t nlat;           /* lattice DOFs */
    int ncells;
    double *eta;            /* per cell */
    unsigned char *active;  /* per cell */
    int64_t nfree;
    int64_t *free_lat;      /* free index -> lattice DOF */
    int64_t *lat_free;      /* lattice DOF -> free index or -1 */
    int64_t *rowptr;
    int64_t *col;
    double *val;
    double *b;
    double *bs[6];          /* unit-strain load cases 1..6 (per free DOF) */
    /* preconditioner */
    int nblocks;
    ora_block *blocks;
    double *jac;            /* per free DOF: 1/K_ll for DOFs in no block, else 0 */
    unsigned char *covered;
} ora_problem;

typedef struct { int64_t key; double v; } coo_entry;

static int coo_cmp(const void *a, const void *b)
{
    int64_t x = ((const coo_entry *)a)->key, y = ((const coo_entry *)b)->key;
    return (x > y) - (x < y);
}

static int node_fixed(const ora_desc *d, int i, int j, int k, int comp)
{
    if (d->bc == 0) return k == 0;
    if (d->bc == 1) return (comp == 0 && i == 0) || (comp == 1 && j == 0) || (comp == 2 && k == 0);
    return 0;
}

ora_problem *ora_problem_build(const ora_desc *din)
{
    ora_problem *P = calloc(1, sizeof *P);
    P->d = *din;
    if (din->gkind == 0 && din->nsph > 0) {
        P->sph_copy = malloc(sizeof(double) * 4 * din->nsph);
        memcpy(P->sph_copy, din->sph, sizeof(double) * 4 * din->nsph);
        P->d.sph = P->sph_copy;
    }
    if (din->gkind == 1) {
        size_t nv = (size_t)din->vdim[0] * din->vdim[1] * din->vdim[2];
        P->vox_copy = malloc(nv);
        memcpy(P->vox_copy, din->vox, nv);
        P->d.vox = P->vox_copy;
    }
    const ora_desc *d = &P->d;
    int p = d->p, q = p + 1, nloc = q * q * q, ndof = 3 * nloc;
    for (int a = 0; a < 3; ++a) P->M[a] = p * d->n[a] + 1;
    int64_t nnodes = (int64_t)P->M[0] * P->M[1] * P->M[2];
    P->nlat = 3 * nnodes;
    P->ncells = d->n[0] * d->n[1] * d->n[2];
    P->eta = calloc(P->ncells, sizeof(double));
    P->active = calloc(P->ncells, 1);
    double **Ke = calloc(P->ncells, sizeof(double *));
    double **Fcell = calloc(P->ncells, sizeof(double *));
    for (int cz = 0; cz < d->n[2]; ++cz)
        for (int cy = 0; cy < d->n[1]; ++cy)
            for (int cx = 0; cx < d->n[0]; ++cx) {
                int c[3] = {cx, cy, cz};
                int ci = cx + d->n[0] * (cy + d->n[1] * cz);
                double *K = malloc(sizeof(double) * ndof * ndof);
                double *Fs = malloc(sizeof(double) * 6 * ndof);
                ora_cell_matrix_ex(d, c, K, Fs, &P->eta[ci]);
                Fcell[ci] = Fs;
                P->active[ci] = P->eta[ci] > 0.0;
                if (P->active[ci]) Ke[ci] = K;
                else free(K);
            }
    /* free DOFs: nodes in the closure of an active cell, minus the Dirichlet ones */
    unsigned char *node_on = calloc(nnodes, 1);
    for (int cz = 0; cz < d->n[2]; ++cz)
        for (int cy = 0; cy < d->n[1]; ++cy)
            for (int cx = 0; cx < d->n[0]; ++cx) {
                int ci = cx + d->n[0] * (cy + d->n[1] * cz);
                if (!P->active[ci]) continue;
                for (int iz = 0; iz <= p; ++iz)
                    for (int iy = 0; iy <= p; ++iy)
                        for (int ix = 0; ix <= p; ++ix)
                            node_on[(p * cx + ix) + (int64_t)P->M[0] * ((p * cy + iy) + (int64_t)P->M[1] * (p * cz + iz))] = 1;
            }
    P->lat_free = malloc(sizeof(int64_t) * P->nlat);
    P->free_lat = malloc(sizeof(int64_t) * P->nlat);
    P->nfree = 0;
    for (int k = 0; k < P->M[2]; ++k)
        for (int j = 0; j < P->M[1]; ++j)
            for (int i = 0; i < P->M[0]; ++i) {
                int64_t node = i + (int64_t)P->M[0] * (j + (int64_t)P->M[1] * k);
                for (int comp = 0; comp < 3; ++comp) {
                    int64_t L = 3 * node + comp;
                    if (node_on[node] && !node_fixed(d, i, j, k, comp)) {
                        P->lat_free[L] = P->nfree;
                        P->free_lat[P->nfree++] = L;
                    } else {
                        P->lat_free[L] = -1;
                    }
                }
            }
    free(node_on);
    /* assemble K from the element matrices (COO, sort, merge) and b from the tractions */
    int64_t cap = 0;
    for (int ci = 0; ci < P->ncells; ++ci) if (P->active[ci]) cap += (int64_t)ndof * ndof;
    coo_entry *coo = malloc(sizeof(coo_entry) * (cap > 0 ? cap : 1));
    int64_t nz = 0;
    P->b = calloc(P->nfree > 0 ? P->nfree : 1, sizeof(double));
    for (int k = 0; k < 6; ++k) P->bs[k] = calloc(P->nfree > 0 ? P->nfree : 1, sizeof(double));
    int64_t *g = malloc(sizeof(int64_t) * ndof);
    double *be = malloc(sizeof(double) * ndof);
    for (int cz = 0; cz < d->n[2]; ++cz)
        for (int cy = 0; cy < d->n[1]; ++cy)
            for (int cx = 0; cx < d->n[0]; ++cx) {
                int ci = cx + d->n[0] * (cy + d->n[1] * cz);
                if (!P->active[ci]) continue;
                for (int iz = 0; iz <= p; ++iz)
                    for (int iy = 0; iy <= p; ++iy)
                        for (int ix = 0; ix <= p; ++ix) {
                            int I = ix + q * (iy + q * iz);
                            int64_t node = (p * cx + ix) + (int64_t)P->M[0] * ((p * cy + iy) + (int64_t)P->M[1] * (p * cz + iz));
                            for (int comp = 0; comp < 3; ++comp) g[3 * I + comp] = P->lat_free[3 * node + comp];
                        }
                const double *K = Ke[ci];
                for (int i = 0; i < ndof; ++i) {
                    if (g[i] < 0) continue;
                    for (int j = 0; j < ndof; ++j) {
                        if (g[j] < 0) continue;
                        coo[nz].key = g[i] * P->nfree + g[j];
                        coo[nz].v = K[(size_t)i * ndof + j];
                        ++nz;
                    }
                }
                int c[3] = {cx, cy, cz};
                ora_cell_traction(d, c, be);
                for (int i = 0; i < ndof; ++i)
                    if (g[i] >= 0) P->b[g[i]] += be[i];
                for (int k = 0; k < 6; ++k)
                    for (int i = 0; i < ndof; ++i)
                        if (g[i] >= 0) P->bs[k][g[i]] += Fcell[ci][k * ndof + i];
            }
    free(g);
    free(be);
    for (int ci = 0; ci < P->ncells; ++ci) {
        free(Ke[ci]);
        free(Fcell[ci]);
    }
    free(Ke);
    free(Fcell);
    qsort(coo, nz, sizeof(coo_entry), coo_cmp);
    P->rowptr = calloc(P->nfree + 1, sizeof(int64_t));
    P->col = malloc(sizeof(int64_t) * (nz > 0 ? nz : 1));
    P->val = malloc(sizeof(double) * (nz > 0 ? nz : 1));
    int64_t m = 0;
    for (int64_t e = 0; e < nz;) {
        int64_t key = coo[e].key;
        double s = 0.0;
        while (e < nz && coo[e].key == key) s += coo[e++].v;
        int64_t r = key / P->nfree, cc = key % P->nfree;
        P->col[m] = cc;
        P->val[m] = s;
        P->rowptr[r + 1]++;
        ++m;
    }
    for (int64_t r = 0; r < P->nfree; ++r) P->rowptr[r + 1] += P->rowptr[r];
    free(coo);
    return P;
}

void ora_problem_free(ora_problem *P)
{
    if (!P) return;
    for (int b = 0; b < P->nblocks; ++b) { free(P->blocks[b].idx); free(P->blocks[b].F); }
    free(P->blocks); free(P->jac); free(P->covered);
    free(P->eta); free(P->active); free(P->free_lat); free(P->lat_free);
    free(P->rowptr); free(P->col); free(P->val); free(P->b);
    for (int k = 0; k < 6; ++k) free(P->bs[k]);
    free(P->sph_copy); free(P->vox_copy);
    free(P);
}

int64_t ora_nfree(const ora_problem *P) { return P->nfree; }
int64_t ora_nnz(const ora_problem *P) { return P->rowptr[P->nfree]; }
int64_t ora_nlat(const ora_problem *P) { return P->nlat; }
int ora_ncells(const ora_problem *P) { return P->ncells; }
void ora_get_free_lat(const ora_problem *P, int64_t *out) { memcpy(out, P->free_lat, sizeof(int64_t) * P->nfree); }
void ora_get_rhs(const ora_problem *P, double *out) { memcpy(out, P->b, sizeof(double) * P->nfree); }
/* load case 0: traction; 1..6: unit Voigt strains (xx, yy, zz, yz, xz, xy) */
int ora_get_load(const ora_problem *P, int load_case, double *out)
{
    if (load_case == 0) { memcpy(out, P->b, sizeof(double) * P->nfree); return 0; }
    if (load_case < 1 || load_case > 6) return -1;
    memcpy(out, P->bs[load_case - 1], sizeof(double) * P->nfree);
    return 0;
}
void ora_get_eta(const ora_problem *P, double *out) { memcpy(out, P->eta, sizeof(double) * P->ncells); }
void ora_get_csr(const ora_problem *P, int64_t *rowptr, int64_t *col, double *val)
{
    memcpy(rowptr, P->rowptr, sizeof(int64_t) * (P->nfree + 1));
    memcpy(col, P->col, sizeof(int64_t) * P->rowptr[P->nfree]);
    memcpy(val, P->val, sizeof(double) * P->rowptr[P->nfree]);
}

void ora_apply_K(const ora_problem *P, const double *x, double *y)
{
    for (int64_t r = 0; r < P->nfree; ++r) {
        double s = 0.0;
        for (int64_t e = P->rowptr[r]; e < P->rowptr[r + 1]; ++e) s += P->val[e] * x[P->col[e]];
        y[r] = s;
    }
}

static double K_entry(const ora_problem *P, int64_t r, int64_t c)
{
    int64_t lo = P->rowptr[r], hi = P->rowptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (P->col[mid] == c) return P->val[mid];
        if (P->col[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* Symmetric eigendecomposition by the cyclic Jacobi method            */
/* (Golub & Van Loan, Matrix Computations, Sec. 8.5).  A is overwritten; */
/* eigenvalues on the diagonal, eigenvectors in the columns of V.       */
/* ------------------------------------------------------------------ */
int ora_jacobi_eig(int n, double *A, double *V, double *lam)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j);
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                if (apq == 0.0) continue;
                if (fabs(apq) <= 2.2e-16 * sqrt(fabs(app) * fabs(aqq))) {
                    A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
                    continue;
                }
                rotated = 1;
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        if (!rotated) break;
    }
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
    return sweep;
}

/* Pseudo inverse of a symmetric matrix, Sec. 3.2 Eqs. (11)-(13):
 *   lambda_k^-1 kept iff lambda_k > eps * max_k lambda_k.
 * eps < 0 selects the unstabilised inverse S* (every nonzero eigenvalue inverted). */
void ora_pseudo_inverse(int n, const double *A, double eps, double *F, double *cond, int *nneg, int *nfilt)
{
    double *W = malloc(sizeof(double) * n * n), *V = malloc(sizeof(double) * n * n), *lam = malloc(sizeof(double) * n);
    memcpy(W, A, sizeof(double) * n * n);
    ora_jacobi_eig(n, W, V, lam);
    double lmax = 0.0;
    for (int k = 0; k < n; ++k) if (lam[k] > lmax) lmax = lam[k];
    double thr = eps * lmax;
    double lmin_kept = INFINITY;
    int neg = 0, filt = 0;
    double *inv = malloc(sizeof(double) * n);
    for (int k = 0; k < n; ++k) {
        if (lam[k] <= 0.0) ++neg;
        if (eps < 0.0) {
            inv[k] = lam[k] != 0.0 ? 1.0 / lam[k] : 0.0;
        } else if (lam[k] > thr) {
            inv[k] = 1.0 / lam[k];
            if (lam[k] < lmin_kept) lmin_kept = lam[k];
        } else {
            inv[k] = 0.0;
            ++filt;
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += V[(size_t)i * n + k] * inv[k] * V[(size_t)j * n + k];
            F[(size_t)i * n + j] = s;
        }
    if (cond) *cond = (lmin_kept < INFINITY && lmin_kept > 0.0) ? lmax / lmin_kept : INFINITY;
    if (nneg) *nneg = neg;
    if (nfilt) *nfilt = filt;
    free(W); free(V); free(lam); free(inv);
}

/* Does the entity carrying lattice index i (along one axis) contain vertex v in its closure? */
static int entity_touches_vertex(int p, int i, int v)
{
    if (i % p == 0) return i / p == v;     /* a vertex: only itself */
    int c = i / p;                          /* interior of the 1D cell c = [c, c+1] */
    return c == v || c + 1 == v;
}

static int add_block(ora_problem *P, int *cap, int n, int *idx)
{
    if (n == 0) return 0;
    if (P->nblocks == *cap) {
        *cap = *cap ? 2 * *cap : 64;
        P->blocks = realloc(P->blocks, sizeof(ora_block) * *cap);
    }
    ora_block *B = &P->blocks[P->nblocks++];
    memset(B, 0, sizeof *B);
    B->n = n;
    B->idx = malloc(sizeof(int) * n);
    memcpy(B->idx, idx, sizeof(int) * n);
    return 1;
}

/* Blocks of Algorithm 1, then pseudo inverses and the diagonal scaling.
 *   rule 0: vertex patches (one block per grid vertex)
 *   rule 1: one block with every free DOF (S = A^-1, Sec. 3.1)
 *   rule 2: no blocks (pure diagonal scaling, i.e. Jacobi)
 *   rule 3: element blocks (all functions supported on a cell) for active
 *           cells with eta_T <= eta_bar (Sec. 3.2 "Optimizing the number of
 *           blocks"; the study of Sec. 5.2 fixes the end points: eta_bar = 1
 *           gives a block for every element, eta_bar = 0 pure diagonal
 *           scaling).  eta_T is a volume fraction, so it is clamped to 1
 *           against the rounding of its quadrature. */
int ora_precond_build(ora_problem *P, int rule, double eps, double eta_bar)
{
    const ora_desc *d = &P->d;
    int p = d->p;
    for (int b = 0; b < P->nblocks; ++b) { free(P->blocks[b].idx); free(P->blocks[b].F); }
    free(P->blocks); P->blocks = NULL; P->nblocks = 0;
    int cap = 0;
    int *idx = malloc(sizeof(int) * (P->nfree > 0 ? P->nfree : 1));
    if (rule == 0) {
        for (int vz = 0; vz <= d->n[2]; ++vz)
            for (int vy = 0; vy <= d->n[1]; ++vy)
                for (int vx = 0; vx <= d->n[0]; ++vx) {
                    int n = 0;
                    for (int64_t f = 0; f < P->nfree; ++f) {
                        int64_t node = P->free_lat[f] / 3;
                        int i = (int)(node % P->M[0]);
                        int j = (int)((node / P->M[0]) % P->M[1]);
                        int k = (int)(node / ((int64_t)P->M[0] * P->M[1]));
                        if (entity_touches_vertex(p, i, vx) && entity_touches_vertex(p, j, vy) &&
                            entity_touches_vertex(p, k, vz))
                            idx[n++] = (int)f;
                    }
                    add_block(P, &cap, n, idx);
                }
    } else if (rule == 1) {
        for (int64_t f = 0; f < P->nfree; ++f) idx[f] = (int)f;
        add_block(P, &cap, (int)P->nfree, idx);
    } else if (rule == 3) {
        for (int cz = 0; cz < d->n[2]; ++cz)
            for (int cy = 0; cy < d->n[1]; ++cy)
                for (int cx = 0; cx < d->n[0]; ++cx) {
                    int ci = cx + d->n[0] * (cy + d->n[1] * cz);
                    if (!P->active[ci] || !((P->eta[ci] < 1.0 ? P->eta[ci] : 1.0) <= eta_bar)) continue;
                    int n = 0;
                    for (int iz = 0; iz <= p; ++iz)
                        for (int iy = 0; iy <= p; ++iy)
                            for (int ix = 0; ix <= p; ++ix) {
                                int64_t node = (p * cx + ix) + (int64_t)P->M[0] * ((p * cy + iy) + (int64_t)P->M[1] * (p * cz + iz));
                                for (int comp = 0; comp < 3; ++comp) {
                                    int64_t f = P->lat_free[3 * node + comp];
                                    if (f >= 0) idx[n++] = (int)f;
                                }
                            }
                    /* keep the block's indices sorted by free index */
                    for (int a = 1; a < n; ++a) {
                        int v = idx[a], b = a - 1;
                        while (b >= 0 && idx[b] > v) { idx[b + 1] = idx[b]; --b; }
                        idx[b + 1] = v;
                    }
                    add_block(P, &cap, n, idx);
                }
    }
    free(idx);
    free(P->covered);
    free(P->jac);
    P->covered = calloc(P->nfree > 0 ? P->nfree : 1, 1);
    P->jac = calloc(P->nfree > 0 ? P->nfree : 1, sizeof(double));
    for (int b = 0; b < P->nblocks; ++b) {
        ora_block *B = &P->blocks[b];
        int n = B->n;
        double *A = malloc(sizeof(double) * n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = K_entry(P, B->idx[i], B->idx[j]);
        B->F = malloc(sizeof(double) * n * n);
        ora_pseudo_inverse(n, A, eps, B->F, &B->cond, &B->nneg, &B->nfilt);
        free(A);
        for (int i = 0; i < n; ++i) P->covered[B->idx[i]] = 1;
    }
    /* Algorithm 1, diagonal scaling: functions in no block get 1 / A(l,l) */
    for (int64_t l = 0; l < P->nfree; ++l)
        if (!P->covered[l]) P->jac[l] = 1.0 / K_entry(P, l, l);
    return P->nblocks;
}

int ora_nblocks(const ora_problem *P) { return P->nblocks; }
int ora_block_size(const ora_problem *P, int b) { return P->blocks[b].n; }
void ora_block_get(const ora_problem *P, int b, int *idx, double *F, double *info)
{
    const ora_block *B = &P->blocks[b];
    if (idx) memcpy(idx, B->idx, sizeof(int) * B->n);
    if (F) memcpy(F, B->F, sizeof(double) * B->n * B->n);
    if (info) { info[0] = B->cond; info[1] = B->nneg; info[2] = B->nfilt; }
}

/* z = S r = sum_B R_B^T A_B+^-1 R_B r + D_jac r  (Eq. (5) with Algorithm 1's diagonal part) */
void ora_apply_S(const ora_problem *P, const double *r, double *z)
{
    for (int64_t l = 0; l < P->nfree; ++l) z[l] = P->jac[l] * r[l];
    double *rb = NULL;
    int cap = 0;
    for (int b = 0; b < P->nblocks; ++b) {
        const ora_block *B = &P->blocks[b];
        if (B->n > cap) { cap = B->n; rb = realloc(rb, sizeof(double) * cap); }
        for (int i = 0; i < B->n; ++i) rb[i] = r[B->idx[i]];
        for (int i = 0; i < B->n; ++i) {
            double s = 0.0;
            for (int j = 0; j < B->n; ++j) s += B->F[(size_t)i * B->n + j] * rb[j];
            z[B->idx[i]] += s;
        }
    }
    free(rb);
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Preconditioned CG (x0 = 0), stopping on ||S r_i|| / ||S b|| <= tol (Eq. (14)).
 * Returns the iteration count (number of K applications), -1 on breakdown,
 * and maxit + 1 when not converged.  hist[i] = ||S r_i|| / ||S b|| for i = 0..its. */
int ora_pcg(const ora_problem *P, const double *b, double tol, int maxit, double *x, double *hist)
{
    int64_t n = P->nfree;
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *pv = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    ora_apply_S(P, r, z);
    memcpy(pv, z, sizeof(double) * n);
    double rz = dot(n, r, z);
    double zn0 = sqrt(dot(n, z, z));
    if (hist) hist[0] = 1.0;
    int it = 0, status = maxit + 1;
    if (zn0 == 0.0) { status = 0; goto done; }
    for (it = 1; it <= maxit; ++it) {
        ora_apply_K(P, pv, q);
        double pq = dot(n, pv, q);
        if (!(pq > 0.0)) { status = -1; break; }
        double a = rz / pq;
        for (int64_t i = 0; i < n; ++i) { x[i] += a * pv[i]; r[i] -= a * q[i]; }
        ora_apply_S(P, r, z);
        double rz_new = dot(n, r, z);
        double rel = sqrt(dot(n, z, z)) / zn0;
        if (hist) hist[it] = rel;
        if (!(rel == rel)) { status = -1; break; }
        if (rel <= tol) { status = it; break; }
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) pv[i] = z[i] + beta * pv[i];
    }
done:
    free(r); free(z); free(pv); free(q);
    return status;
}

/* Relative energy-norm error of Eq. (15). */
double ora_energy_error(const ora_problem *P, const double *xref, const double *x)
{
    int64_t n = P->nfree;
    double *e = malloc(sizeof(double) * n), *Ke = malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) e[i] = xref[i] - x[i];
    ora_apply_K(P, e, Ke);
    double num = dot(n, e, Ke);
    ora_apply_K(P, xref, Ke);
    double den = dot(n, xref, Ke);
    free(e); free(Ke);
    return sqrt(fabs(num) / den);
}

/* ------------------------------------------------------------------ */
/* Local (sampled) quantities for full-size checks: one vertex-patch   */
/* block assembled from the cells around the vertex alone.             */
/* ------------------------------------------------------------------ */
/* Fills lat (lattice DOFs of the block, ascending) and F (pseudo inverse);
 * returns the block size.  lat/F must hold 3(2p-1)^3 and its square. */
int ora_patch_factor(const ora_desc *d, const int *v, double eps, int64_t *lat, double *F, double *cond)
{
    int p = d->p, q = p + 1, ndof = 3 * q * q * q;
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = p * d->n[a] + 1;
    /* cells around v and their element matrices */
    double *Ke[8] = {0};
    int cc[8][3], act[8] = {0};
    for (int t = 0; t < 8; ++t) {
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
            cc[t][a] = v[a] - 1 + ((t >> a) & 1);
            if (cc[t][a] < 0 || cc[t][a] >= d->n[a]) ok = 0;
        }
        if (!ok) continue;
        double eta;
        Ke[t] = malloc(sizeof(double) * ndof * ndof);
        ora_cell_matrix(d, cc[t], Ke[t], &eta);
        act[t] = eta > 0.0;
    }
    /* block members: nodes whose entity contains v, on an active cell of the patch, not fixed */
    int nb = 0;
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int64_t)p * v[a] - (p - 1); if (lo[a] < 0) lo[a] = 0;
        hi[a] = (int64_t)p * v[a] + (p - 1); if (hi[a] > M[a] - 1) hi[a] = M[a] - 1;
    }
    for (int64_t k = lo[2]; k <= hi[2]; ++k)
        for (int64_t j = lo[1]; j <= hi[1]; ++j)
            for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                if (!entity_touches_vertex(p, (int)i, v[0]) || !entity_touches_vertex(p, (int)j, v[1]) ||
                    !entity_touches_vertex(p, (int)k, v[2]))
                    continue;
                int on = 0;
                for (int t = 0; t < 8; ++t) {
                    if (!act[t]) continue;
                    if (i >= (int64_t)p * cc[t][0] && i <= (int64_t)p * cc[t][0] + p &&
                        j >= (int64_t)p * cc[t][1] && j <= (int64_t)p * cc[t][1] + p &&
                        k >= (int64_t)p * cc[t][2] && k <= (int64_t)p * cc[t][2] + p)
                        on = 1;
                }
                if (!on) continue;
                for (int comp = 0; comp < 3; ++comp)
                    if (!node_fixed(d, (int)i, (int)j, (int)k, comp))
                        lat[nb++] = 3 * (i + (int64_t)M[0] * (j + (int64_t)M[1] * k)) + comp;
            }
    double *A = calloc((size_t)nb * nb, sizeof(double));
    for (int t = 0; t < 8; ++t) {
        if (!act[t]) continue;
        for (int r = 0; r < nb; ++r)
            for (int s = 0; s < nb; ++s) {
                int64_t nr = lat[r] / 3, ns = lat[s] / 3;
                int lr[3] = {(int)(nr % M[0]) - p * cc[t][0], (int)((nr / M[0]) % M[1]) - p * cc[t][1],
                             (int)(nr / ((int64_t)M[0] * M[1])) - p * cc[t][2]};
                int ls[3] = {(int)(ns % M[0]) - p * cc[t][0], (int)((ns / M[0]) % M[1]) - p * cc[t][1],
                             (int)(ns / ((int64_t)M[0] * M[1])) - p * cc[t][2]};
                int in = 1;
                for (int a = 0; a < 3; ++a)
                    if (lr[a] < 0 || lr[a] > p || ls[a] < 0 || ls[a] > p) in = 0;
                if (!in) continue;
                int ir = 3 * (lr[0] + q * (lr[1] + q * lr[2])) + (int)(lat[r] % 3);
                int is = 3 * (ls[0] + q * (ls[1] + q * ls[2])) + (int)(lat[s] % 3);
                A[(size_t)r * nb + s] += Ke[t][(size_t)ir * ndof + is];
            }
    }
    if (nb > 0) ora_pseudo_inverse(nb, A, eps, F, cond, NULL, NULL);
    free(A);
    for (int t = 0; t < 8; ++t) free(Ke[t]);
    return nb;
}

/* Sampled rows of K: y_l = (K x)_l for the lattice DOFs `rows`, using only the
 * cells around each row's node.  x is a full lattice vector (inactive and
 * fixed entries are ignored). Returns 0, or -1 when a row is not free. */
int ora_sample_Kx(const ora_desc *d, int nrows, const int64_t *rows, const double *x, double *y)
{
    int p = d->p, q = p + 1, ndof = 3 * q * q * q;
    int M[3];
    for (int a = 0; a < 3; ++a) M[a] = p * d->n[a] + 1;
    double *Ke = malloc(sizeof(double) * ndof * ndof);
    int status = 0;
    for (int s = 0; s < nrows; ++s) {
        int64_t L = rows[s], node = L / 3;
        int comp = (int)(L % 3);
        int nd[3] = {(int)(node % M[0]), (int)((node / M[0]) % M[1]), (int)(node / ((int64_t)M[0] * M[1]))};
        double acc = 0.0;
        int any_active = 0;
        /* candidate cells: those whose lattice box contains the node */
        int c0[3], c1[3];
        for (int a = 0; a < 3; ++a) {
            c0[a] = (nd[a] % p == 0) ? nd[a] / p - 1 : nd[a] / p;
            c1[a] = nd[a] / p;
            if (c0[a] < 0) c0[a] = 0;
            if (c1[a] > d->n[a] - 1) c1[a] = d->n[a] - 1;
        }
        for (int cz = c0[2]; cz <= c1[2]; ++cz)
            for (int cy = c0[1]; cy <= c1[1]; ++cy)
                for (int cx = c0[0]; cx <= c1[0]; ++cx) {
                    int c[3] = {cx, cy, cz};
                    double eta;
                    ora_cell_matrix(d, c, Ke, &eta);
                    if (!(eta > 0.0)) continue;
                    any_active = 1;
                    int li[3] = {nd[0] - p * cx, nd[1] - p * cy, nd[2] - p * cz};
                    int row = 3 * (li[0] + q * (li[1] + q * li[2])) + comp;
                    for (int iz = 0; iz <= p; ++iz)
                        for (int iy = 0; iy <= p; ++iy)
                            for (int ix = 0; ix <= p; ++ix) {
                                int64_t nn = (p * cx + ix) + (int64_t)M[0] * ((p * cy + iy) + (int64_t)M[1] * (p * cz + iz));
                                for (int cj = 0; cj < 3; ++cj) {
                                    if (node_fixed(d, p * cx + ix, p * cy + iy, p * cz + iz, cj)) continue;
                                    int col = 3 * (ix + q * (iy + q * iz)) + cj;
                                    acc += Ke[(size_t)row * ndof + col] * x[3 * nn + cj];
                                }
                            }
                }
        if (!any_active || node_fixed(d, nd[0], nd[1], nd[2], comp)) status = -1;
        y[s] = acc;
    }
    free(Ke);
    return status;
}
