// Host-side problem set-up of libfcm: geometry classification, Legendre
// moments of the physical part of every cut cell, element stiffness matrices
// by sum factorisation of those moments, free-DOF mask and traction load.
//
// Method (Jomo et al., arXiv:1809.00828):
//  * Sec. 2.1, Eq. (1): a(v,u) = int alpha eps(v):C:eps(u) dOmega with alpha = 1
//    in Omega_phys and the fictitious stiffness alpha outside.
//  * Sec. 5.1 setup: cut cells are integrated on an octree partition of fixed
//    depth relative to the cell size.
//  * Sec. 3.2, Eq. (10): eta_T = |T cap Omega_phys| / |T|; cells with eta_T = 0
//    are removed (the usual preprocessing of Sec. 5.2).
//
// Instead of summing B^T D B over every quadrature point, this file integrates
// the Legendre moments mu_abc = int_{T cap Omega_phys} P_a(xi) P_b(eta) P_c(zeta)
// (a, b, c <= 2p) once per cut cell and obtains every entry of the element
// matrix from them: each integrand d_j N_I d_l N_J is a tensor product of 1D
// polynomials of degree <= 2p, whose Legendre coefficients are tabulated once.
// Leaves of the octree that the boundary does not cross contribute their
// moments in closed form; crossed leaves at full depth use a (p+1)^3
// Gauss-Legendre rule with the indicator evaluated at each point.  Both are
// exact for the polynomial integrand wherever the indicator is constant, so
// the result equals point-wise octree quadrature up to rounding.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "fcm_internal.h"

namespace fcm {

namespace {

constexpr int kMaxP = 4;
constexpr int kMaxQ = kMaxP + 1;
constexpr int kMaxL = 2 * kMaxP + 1;

// P_0..P_m at x by the three-term recurrence.
inline void legendre_values(int m, double x, double *P)
{
    P[0] = 1.0;
    if (m >= 1) P[1] = x;
    for (int k = 2; k <= m; ++k) P[k] = ((2 * k - 1) * x * P[k - 1] - (k - 1) * P[k - 2]) / k;
}

// int_a^b P_m(t) dt for m < L, from (2m+1) P_m = (P_{m+1} - P_{m-1})'.
inline void legendre_integrals(int L, double a, double b, double *out)
{
    double Pa[kMaxL + 2], Pb[kMaxL + 2];
    legendre_values(L, a, Pa);
    legendre_values(L, b, Pb);
    out[0] = b - a;
    for (int m = 1; m < L; ++m) out[m] = ((Pb[m + 1] - Pb[m - 1]) - (Pa[m + 1] - Pa[m - 1])) / (2 * m + 1);
}

// 1D shape functions in lattice order with xi-derivatives:
// f_0 = (1-xi)/2, f_p = (1+xi)/2, f_a = phi_{a+1} = (P_{a+1} - P_{a-1}) / sqrt(2(2a+1)),
// phi_j' = (2j-1) P_{j-1} / sqrt(2(2j-1)).
inline void shape_1d(int p, double xi, double *f, double *df)
{
    double P[kMaxL + 2];
    legendre_values(p, xi, P);
    f[0] = 0.5 * (1.0 - xi);
    df[0] = -0.5;
    f[p] = 0.5 * (1.0 + xi);
    df[p] = 0.5;
    for (int a = 1; a < p; ++a) {
        const int j = a + 1;
        const double c = 1.0 / std::sqrt(4.0 * j - 2.0);
        f[a] = (P[j] - P[j - 2]) * c;
        df[a] = (2.0 * j - 1.0) * P[j - 1] * c;
    }
}

struct Geometry {
    int kind;
    const double *sph;
    int nsph;
    const uint8_t *vox;
    int vdim[3];
    double lo[3], hi[3];
    double plane[4];

    bool solid(const double *x) const
    {
        if (kind == FCM_GEOM_SPHERE_VOIDS) {
            for (int s = 0; s < nsph; ++s) {
                const double *c = sph + 4 * s;
                const double d0 = x[0] - c[0], d1 = x[1] - c[1], d2 = x[2] - c[2];
                if (d0 * d0 + d1 * d1 + d2 * d2 < c[3] * c[3]) return false;
            }
            return true;
        }
        if (kind == FCM_GEOM_VOXELS) {
            int idx[3];
            for (int a = 0; a < 3; ++a) {
                int i = (int)std::floor((x[a] - lo[a]) / (hi[a] - lo[a]) * vdim[a]);
                idx[a] = std::min(std::max(i, 0), vdim[a] - 1);
            }
            return vox[idx[0] + (size_t)vdim[0] * (idx[1] + (size_t)vdim[1] * idx[2])] != 0;
        }
        return plane[0] * x[0] + plane[1] * x[1] + plane[2] * x[2] < plane[3];
    }

    // True when the geometry boundary may cross the box.  Deliberately
    // generous: flagging an uncrossed box only costs extra subdivision (the
    // quadrature of an uncrossed box is exact either way), while missing a
    // crossed one would change the integral.
    bool crossed(const double *blo, const double *bhi) const
    {
        if (kind == FCM_GEOM_SPHERE_VOIDS) {
            for (int s = 0; s < nsph; ++s) {
                const double *c = sph + 4 * s;
                double near2 = 0.0, far2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double e = std::max(0.0, std::max(blo[a] - c[a], c[a] - bhi[a]));
                    near2 += e * e;
                    double f = std::max(std::fabs(c[a] - blo[a]), std::fabs(c[a] - bhi[a]));
                    far2 += f * f;
                }
                const double r2 = c[3] * c[3], slack = 1e-12 * r2;
                if (near2 < r2 + slack && far2 > r2 - slack) return true;
            }
            return false;
        }
        if (kind == FCM_GEOM_VOXELS) {
            int i0[3], i1[3];
            for (int a = 0; a < 3; ++a) {
                const double t0 = (blo[a] - lo[a]) / (hi[a] - lo[a]) * vdim[a];
                const double t1 = (bhi[a] - lo[a]) / (hi[a] - lo[a]) * vdim[a];
                i0[a] = std::max(0, (int)std::floor(t0 - 1e-9));
                i1[a] = std::min(vdim[a] - 1, (int)std::floor(t1 + 1e-9));
                if (i1[a] < i0[a]) i1[a] = i0[a];
            }
            const uint8_t first = vox[i0[0] + (size_t)vdim[0] * (i0[1] + (size_t)vdim[1] * i0[2])] != 0;
            for (int k = i0[2]; k <= i1[2]; ++k)
                for (int j = i0[1]; j <= i1[1]; ++j)
                    for (int i = i0[0]; i <= i1[0]; ++i)
                        if ((vox[i + (size_t)vdim[0] * (j + (size_t)vdim[1] * k)] != 0) != first) return true;
            return false;
        }
        double mn = 0.0, mx = 0.0;
        for (int a = 0; a < 3; ++a) {
            mn += std::min(plane[a] * blo[a], plane[a] * bhi[a]);
            mx += std::max(plane[a] * blo[a], plane[a] * bhi[a]);
        }
        const double slack = 1e-12 * (std::fabs(plane[3]) + std::fabs(mn) + std::fabs(mx));
        return mn < plane[3] + slack && plane[3] - slack < mx;
    }
};

struct Tables {
    int p, q, L;
    double gx[kMaxQ], gw[kMaxQ];
    // coef[dd][a][b][m]: Legendre coefficient m of f_a^(da) f_b^(db), dd = da + 2 db
    double coef[4][kMaxQ][kMaxQ][kMaxL];
    // face[a][m]: Legendre coefficient m of f_a
    double face[kMaxQ][kMaxL];
    // dface[a][m]: Legendre coefficient m of f_a'
    double dface[kMaxQ][kMaxL];
};

void make_tables(int p, Tables &T)
{
    T.p = p;
    T.q = p + 1;
    T.L = 2 * p + 1;
    gauss_legendre(T.q, T.gx, T.gw);
    const int ng = 2 * p + 2;
    double x[2 * kMaxP + 2], w[2 * kMaxP + 2];
    gauss_legendre(ng, x, w);
    std::memset(T.coef, 0, sizeof T.coef);
    std::memset(T.face, 0, sizeof T.face);
    std::memset(T.dface, 0, sizeof T.dface);
    for (int g = 0; g < ng; ++g) {
        double f[kMaxQ], df[kMaxQ], P[kMaxL + 2];
        shape_1d(p, x[g], f, df);
        legendre_values(T.L, x[g], P);
        for (int m = 0; m < T.L; ++m) {
            const double s = w[g] * P[m] * (2 * m + 1) * 0.5;
            for (int a = 0; a <= p; ++a) {
                T.face[a][m] += s * f[a];
                T.dface[a][m] += s * df[a];
                for (int b = 0; b <= p; ++b) {
                    T.coef[0][a][b][m] += s * f[a] * f[b];
                    T.coef[1][a][b][m] += s * df[a] * f[b];
                    T.coef[2][a][b][m] += s * f[a] * df[b];
                    T.coef[3][a][b][m] += s * df[a] * df[b];
                }
            }
        }
    }
}

struct Setup {
    const HostProblem *P;
    Geometry geo;
    Tables T;
};

void cell_box(const HostProblem &P, const int *c, double *clo, double *chi)
{
    for (int a = 0; a < 3; ++a) {
        clo[a] = P.lo[a] + c[a] * P.h[a];
        chi[a] = (c[a] + 1 == P.n[a]) ? P.hi[a] : P.lo[a] + (c[a] + 1) * P.h[a];
    }
}

// Solid-part Legendre moments of one cell (reference cube measure dxi deta dzeta).
void cell_moments_rec(const Setup &S, const double *clo, const double *blo, const double *bhi, int level,
                      double *mu, bool &crossed_any)
{
    const HostProblem &P = *S.P;
    const int L = S.T.L, q = S.T.q;
    const bool crossed = S.geo.crossed(blo, bhi);
    if (crossed) crossed_any = true;
    if (crossed && level < P.depth) {
        double mid[3];
        for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (blo[a] + bhi[a]);
        for (int c = 0; c < 8; ++c) {
            double lo2[3], hi2[3];
            for (int a = 0; a < 3; ++a) {
                const bool up = (c >> a) & 1;
                lo2[a] = up ? mid[a] : blo[a];
                hi2[a] = up ? bhi[a] : mid[a];
            }
            cell_moments_rec(S, clo, lo2, hi2, level + 1, mu, crossed_any);
        }
        return;
    }
    if (!crossed) {
        double ctr[3];
        for (int a = 0; a < 3; ++a) ctr[a] = 0.5 * (blo[a] + bhi[a]);
        if (!S.geo.solid(ctr)) return;
        double I[3][kMaxL];
        for (int a = 0; a < 3; ++a)
            legendre_integrals(L, 2.0 * (blo[a] - clo[a]) / P.h[a] - 1.0, 2.0 * (bhi[a] - clo[a]) / P.h[a] - 1.0, I[a]);
        for (int m0 = 0; m0 < L; ++m0)
            for (int m1 = 0; m1 < L; ++m1) {
                const double s = I[0][m0] * I[1][m1];
                for (int m2 = 0; m2 < L; ++m2) mu[(m0 * L + m1) * L + m2] += s * I[2][m2];
            }
        return;
    }
    // crossed leaf at full depth: Gauss-Legendre points, indicator per point
    double wscale = 1.0;
    for (int a = 0; a < 3; ++a) wscale *= (bhi[a] - blo[a]) / P.h[a];
    for (int kz = 0; kz < q; ++kz)
        for (int ky = 0; ky < q; ++ky)
            for (int kx = 0; kx < q; ++kx) {
                const int k3[3] = {kx, ky, kz};
                double x[3], Pm[3][kMaxL + 2];
                for (int a = 0; a < 3; ++a) {
                    x[a] = blo[a] + 0.5 * (bhi[a] - blo[a]) * (S.T.gx[k3[a]] + 1.0);
                    legendre_values(L - 1, 2.0 * (x[a] - clo[a]) / P.h[a] - 1.0, Pm[a]);
                }
                if (!S.geo.solid(x)) continue;
                const double w = S.T.gw[kx] * S.T.gw[ky] * S.T.gw[kz] * wscale;
                for (int m0 = 0; m0 < L; ++m0)
                    for (int m1 = 0; m1 < L; ++m1) {
                        const double s = w * Pm[0][m0] * Pm[1][m1];
                        for (int m2 = 0; m2 < L; ++m2) mu[(m0 * L + m1) * L + m2] += s * Pm[2][m2];
                    }
            }
}

// Element stiffness from moments mu (of the alpha-weighted measure):
// G_jl[I,J] = int d_j N_I d_l N_J, K[(I,a),(J,b)] = lam G_ab + mu G_ba + delta_ab mu tr G.
void element_from_moments(const Setup &S, const double *mu, double *K)
{
    const HostProblem &P = *S.P;
    const int q = S.T.q, L = S.T.L, nl = q * q * q, ne = 3 * nl;
    const double lam = P.E * P.nu / ((1.0 + P.nu) * (1.0 - 2.0 * P.nu));
    const double mus = P.E / (2.0 * (1.0 + P.nu));
    const double vol = P.h[0] * P.h[1] * P.h[2] / 8.0;
    std::vector<double> G(9 * (size_t)nl * nl);
    std::vector<double> T1((size_t)L * L * q * q), T2((size_t)L * q * q * q * q);
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
            int dd[3];
            double scale = vol;
            for (int a = 0; a < 3; ++a) {
                dd[a] = (j == a) + 2 * (l == a);
                if (j == a) scale *= 2.0 / P.h[a];
                if (l == a) scale *= 2.0 / P.h[a];
            }
            // T1[m0][m1][i2][j2] = sum_m2 C2[i2][j2][m2] mu[m0][m1][m2]
            for (int m0 = 0; m0 < L; ++m0)
                for (int m1 = 0; m1 < L; ++m1)
                    for (int i2 = 0; i2 < q; ++i2)
                        for (int j2 = 0; j2 < q; ++j2) {
                            double s = 0.0;
                            for (int m2 = 0; m2 < L; ++m2) s += S.T.coef[dd[2]][i2][j2][m2] * mu[(m0 * L + m1) * L + m2];
                            T1[((m0 * L + m1) * q + i2) * q + j2] = s;
                        }
            // T2[m0][i1][j1][i2][j2] = sum_m1 C1[i1][j1][m1] T1[m0][m1][i2][j2]
            for (int m0 = 0; m0 < L; ++m0)
                for (int i1 = 0; i1 < q; ++i1)
                    for (int j1 = 0; j1 < q; ++j1)
                        for (int i2 = 0; i2 < q; ++i2)
                            for (int j2 = 0; j2 < q; ++j2) {
                                double s = 0.0;
                                for (int m1 = 0; m1 < L; ++m1)
                                    s += S.T.coef[dd[1]][i1][j1][m1] * T1[((m0 * L + m1) * q + i2) * q + j2];
                                T2[(((m0 * q + i1) * q + j1) * q + i2) * q + j2] = s;
                            }
            double *Gjl = G.data() + (size_t)(3 * j + l) * nl * nl;
            for (int i2 = 0; i2 < q; ++i2)
                for (int i1 = 0; i1 < q; ++i1)
                    for (int i0 = 0; i0 < q; ++i0)
                        for (int j2 = 0; j2 < q; ++j2)
                            for (int j1 = 0; j1 < q; ++j1)
                                for (int j0 = 0; j0 < q; ++j0) {
                                    double s = 0.0;
                                    for (int m0 = 0; m0 < L; ++m0)
                                        s += S.T.coef[dd[0]][i0][j0][m0] * T2[(((m0 * q + i1) * q + j1) * q + i2) * q + j2];
                                    const int I = i0 + q * (i1 + q * i2), J = j0 + q * (j1 + q * j2);
                                    Gjl[(size_t)I * nl + J] = scale * s;
                                }
        }
    for (int I = 0; I < nl; ++I)
        for (int J = 0; J < nl; ++J) {
            const size_t e = (size_t)I * nl + J;
            const double tr = G[0 * nl * nl + e] + G[4 * (size_t)nl * nl + e] + G[8 * (size_t)nl * nl + e];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double v = lam * G[(size_t)(3 * a + b) * nl * nl + e] + mus * G[(size_t)(3 * b + a) * nl * nl + e];
                    if (a == b) v += mus * tr;
                    K[(size_t)(3 * I + a) * ne + 3 * J + b] = v;
                }
        }
    // exact symmetry (the contraction is symmetric up to rounding)
    for (int r = 0; r < ne; ++r)
        for (int c = r + 1; c < ne; ++c) {
            const double v = 0.5 * (K[(size_t)r * ne + c] + K[(size_t)c * ne + r]);
            K[(size_t)r * ne + c] = v;
            K[(size_t)c * ne + r] = v;
        }
}

// Unit-strain loads of one cell from the moments of the alpha-weighted measure:
// G1[j][I] = int alpha d_j N_I, and load case k (Voigt unit strain e_k, engineering
// shears) gives be[k][3I + a] = -sum_j sigma_k[a][j] G1[j][I] with sigma_k = C : E_k.
void strain_loads_from_moments(const Setup &S, const double *mu, double *be)
{
    const HostProblem &P = *S.P;
    const int q = S.T.q, L = S.T.L, nl = q * q * q, ne = 3 * nl;
    const double vol = P.h[0] * P.h[1] * P.h[2] / 8.0;
    const double lam = P.E * P.nu / ((1.0 + P.nu) * (1.0 - 2.0 * P.nu));
    const double mus = P.E / (2.0 * (1.0 + P.nu));
    std::vector<double> G1(3 * (size_t)nl);
    for (int j = 0; j < 3; ++j)
        for (int i2 = 0; i2 < q; ++i2)
            for (int i1 = 0; i1 < q; ++i1)
                for (int i0 = 0; i0 < q; ++i0) {
                    const double *e0 = j == 0 ? S.T.dface[i0] : S.T.face[i0];
                    const double *e1 = j == 1 ? S.T.dface[i1] : S.T.face[i1];
                    const double *e2 = j == 2 ? S.T.dface[i2] : S.T.face[i2];
                    double s = 0.0;
                    for (int m0 = 0; m0 < L; ++m0)
                        for (int m1 = 0; m1 < L; ++m1) {
                            const double t = e0[m0] * e1[m1];
                            for (int m2 = 0; m2 < L; ++m2) s += t * e2[m2] * mu[(m0 * L + m1) * L + m2];
                        }
                    G1[(size_t)j * nl + i0 + q * (i1 + q * i2)] = vol * (2.0 / P.h[j]) * s;
                }
    static const int voigt[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    for (int k = 0; k < 6; ++k) {
        double sig[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const int a0 = voigt[k][0], b0 = voigt[k][1];
        if (a0 == b0) {
            for (int a = 0; a < 3; ++a) sig[a][a] = lam;
            sig[a0][a0] += 2.0 * mus;
        } else {
            sig[a0][b0] = sig[b0][a0] = mus;  // engineering shear strain 1
        }
        for (int I = 0; I < nl; ++I)
            for (int a = 0; a < 3; ++a) {
                double v = 0.0;
                for (int j = 0; j < 3; ++j) v += sig[a][j] * G1[(size_t)j * nl + I];
                be[(size_t)k * ne + 3 * I + a] = -v;
            }
    }
}

// Solid-part 2D Legendre moments of the top face of a cell (reference square measure).
void face_moments_rec(const Setup &S, const double *clo, const double *flo, const double *fhi, int level,
                      double *nu)
{
    const HostProblem &P = *S.P;
    const int L = S.T.L, q = S.T.q;
    const double blo[3] = {flo[0], flo[1], P.hi[2]}, bhi[3] = {fhi[0], fhi[1], P.hi[2]};
    const bool crossed = S.geo.crossed(blo, bhi);
    if (crossed && level < P.depth) {
        const double mid[2] = {0.5 * (flo[0] + fhi[0]), 0.5 * (flo[1] + fhi[1])};
        for (int c = 0; c < 4; ++c) {
            double lo2[2], hi2[2];
            for (int a = 0; a < 2; ++a) {
                const bool up = (c >> a) & 1;
                lo2[a] = up ? mid[a] : flo[a];
                hi2[a] = up ? fhi[a] : mid[a];
            }
            face_moments_rec(S, clo, lo2, hi2, level + 1, nu);
        }
        return;
    }
    if (!crossed) {
        const double ctr[3] = {0.5 * (flo[0] + fhi[0]), 0.5 * (flo[1] + fhi[1]), P.hi[2]};
        if (!S.geo.solid(ctr)) return;
        double I[2][kMaxL];
        for (int a = 0; a < 2; ++a)
            legendre_integrals(L, 2.0 * (flo[a] - clo[a]) / P.h[a] - 1.0, 2.0 * (fhi[a] - clo[a]) / P.h[a] - 1.0, I[a]);
        for (int m0 = 0; m0 < L; ++m0)
            for (int m1 = 0; m1 < L; ++m1) nu[m0 * L + m1] += I[0][m0] * I[1][m1];
        return;
    }
    const double wscale = (fhi[0] - flo[0]) / P.h[0] * (fhi[1] - flo[1]) / P.h[1];
    for (int ky = 0; ky < q; ++ky)
        for (int kx = 0; kx < q; ++kx) {
            double x[3], Pm[2][kMaxL + 2];
            x[0] = flo[0] + 0.5 * (fhi[0] - flo[0]) * (S.T.gx[kx] + 1.0);
            x[1] = flo[1] + 0.5 * (fhi[1] - flo[1]) * (S.T.gx[ky] + 1.0);
            x[2] = P.hi[2];
            if (!S.geo.solid(x)) continue;
            legendre_values(L - 1, 2.0 * (x[0] - clo[0]) / P.h[0] - 1.0, Pm[0]);
            legendre_values(L - 1, 2.0 * (x[1] - clo[1]) / P.h[1] - 1.0, Pm[1]);
            const double w = S.T.gw[kx] * S.T.gw[ky] * wscale;
            for (int m0 = 0; m0 < L; ++m0)
                for (int m1 = 0; m1 < L; ++m1) nu[m0 * L + m1] += w * Pm[0][m0] * Pm[1][m1];
        }
}

template <class F>
void parallel_for(int64_t n, int nthreads, F &&fn)
{
    if (nthreads <= 1 || n < 2) {
        for (int64_t i = 0; i < n; ++i) fn(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back([&]() {
            for (;;) {
                const int64_t i = next.fetch_add(1);
                if (i >= n) break;
                fn(i);
            }
        });
    for (auto &th : pool) th.join();
}

}  // namespace

void gauss_legendre(int n, double *x, double *w)
{
    // Newton iteration on P_n from the Chebyshev-like initial guess
    // cos(pi (k - 1/4) / (n + 1/2)); P_n' from (1 - t^2) P_n' = n (P_{n-1} - t P_n).
    for (int k = 1; k <= n; ++k) {
        double t = std::cos(M_PI * (k - 0.25) / (n + 0.5));
        double pn = 0.0, pm = 0.0;
        for (int it = 0; it < 60; ++it) {
            double a = 1.0, b = t;
            for (int j = 2; j <= n; ++j) {
                const double c = ((2 * j - 1) * t * b - (j - 1) * a) / j;
                a = b;
                b = c;
            }
            pn = (n == 1) ? t : b;
            pm = (n == 1) ? 1.0 : a;
            const double dp = n * (pm - t * pn) / (1.0 - t * t);
            const double step = pn / dp;
            t -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double a = 1.0, b = t;
        for (int j = 2; j <= n; ++j) {
            const double c = ((2 * j - 1) * t * b - (j - 1) * a) / j;
            a = b;
            b = c;
        }
        pn = (n == 1) ? t : b;
        pm = (n == 1) ? 1.0 : a;
        const double dp = n * (pm - t * pn) / (1.0 - t * t);
        x[n - k] = t;
        w[n - k] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

void make_sf_tables(const HostProblem &P, SfTables &T)
{
    std::memset(&T, 0, sizeof T);
    const int q = P.p + 1;
    double x[kMaxQ], w[kMaxQ];
    gauss_legendre(q, x, w);
    for (int k = 0; k < q; ++k) {
        double f[kMaxQ], df[kMaxQ];
        shape_1d(P.p, x[k], f, df);
        T.W[k] = w[k];
        for (int i = 0; i < q; ++i) {
            T.B[k][i] = f[i];
            for (int a = 0; a < 3; ++a) T.D[a][k][i] = df[i] * 2.0 / P.h[a];
        }
    }
    // collocation derivative on the Gauss points (barycentric form): for a polynomial of degree
    // <= p per axis, its values at the p+1 points give its derivative there exactly
    double lam_b[kMaxQ];
    for (int k = 0; k < q; ++k) {
        lam_b[k] = 1.0;
        for (int m = 0; m < q; ++m)
            if (m != k) lam_b[k] /= (x[k] - x[m]);
    }
    for (int i = 0; i < q; ++i) {
        double diag = 0.0;
        for (int k = 0; k < q; ++k) {
            if (k == i) continue;
            const double v = (lam_b[k] / lam_b[i]) / (x[i] - x[k]);
            diag -= v;
            for (int a = 0; a < 3; ++a) T.G[a][i][k] = v * 2.0 / P.h[a];
        }
        for (int a = 0; a < 3; ++a) T.G[a][i][i] = diag * 2.0 / P.h[a];
    }
    T.detJ = P.h[0] * P.h[1] * P.h[2] / 8.0;
    T.lam = P.E * P.nu / ((1.0 + P.nu) * (1.0 - 2.0 * P.nu));
    T.mu = P.E / (2.0 * (1.0 + P.nu));
}

std::string build_host_problem(const fcm_grid &grid, const fcm_geometry &geom, int p, double alpha,
                               const fcm_bc &bc, HostProblem &P, int nthreads)
{
    if (p < 1 || p > kMaxP) return "p must be in [1, 4]";
    if (!(alpha > 0.0 && alpha <= 1.0)) return "alpha must be in (0, 1]";
    if (!(bc.E > 0.0) || !(bc.nu > -1.0 && bc.nu < 0.5)) return "invalid material (E > 0, -1 < nu < 0.5)";
    if (bc.bc < -1 || bc.bc > 1) return "invalid boundary condition kind";
    if (geom.octree_depth < 0 || geom.octree_depth > 12) return "octree_depth must be in [0, 12]";
    for (int a = 0; a < 3; ++a) {
        if (grid.n[a] < 1 || grid.n[a] > 4096) return "grid cells per axis must be in [1, 4096]";
        if (!(grid.hi[a] > grid.lo[a])) return "grid box must have hi > lo";
        if (!std::isfinite(bc.traction[a])) return "traction must be finite";
    }
    P.p = p;
    P.alpha = alpha;
    P.E = bc.E;
    P.nu = bc.nu;
    P.bc = bc.bc;
    for (int a = 0; a < 3; ++a) {
        P.n[a] = grid.n[a];
        P.lo[a] = grid.lo[a];
        P.hi[a] = grid.hi[a];
        P.h[a] = (grid.hi[a] - grid.lo[a]) / grid.n[a];
        P.traction[a] = bc.traction[a];
        P.M[a] = p * grid.n[a] + 1;
    }
    P.gkind = geom.kind;
    P.depth = geom.octree_depth;
    std::memcpy(P.plane, geom.plane, sizeof P.plane);
    if (geom.kind == FCM_GEOM_SPHERE_VOIDS) {
        if (geom.nsph < 0 || (geom.nsph > 0 && !geom.sph)) return "sphere list missing";
        P.sph.assign(geom.sph, geom.sph + 4 * (size_t)geom.nsph);
        for (double v : P.sph)
            if (!std::isfinite(v)) return "non-finite sphere data";
    } else if (geom.kind == FCM_GEOM_VOXELS) {
        if (!geom.vox) return "voxel image missing";
        size_t nv = 1;
        for (int a = 0; a < 3; ++a) {
            if (geom.vdim[a] < 1) return "voxel dimensions must be positive";
            nv *= (size_t)geom.vdim[a];
            P.vdim[a] = geom.vdim[a];
        }
        P.vox.assign(geom.vox, geom.vox + nv);
    } else if (geom.kind != FCM_GEOM_HALFSPACE) {
        return "unknown geometry kind";
    }
    P.nnodes = (int64_t)P.M[0] * P.M[1] * P.M[2];
    P.nlat = 3 * P.nnodes;
    const int q = p + 1, nl = q * q * q;
    P.ne = 3 * nl;
    P.ncells = (int64_t)P.n[0] * P.n[1] * P.n[2];
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());

    Setup S;
    S.P = &P;
    S.geo.kind = P.gkind;
    S.geo.sph = P.sph.data();
    S.geo.nsph = (int)(P.sph.size() / 4);
    S.geo.vox = P.vox.data();
    for (int a = 0; a < 3; ++a) {
        S.geo.vdim[a] = P.vdim[a];
        S.geo.lo[a] = P.lo[a];
        S.geo.hi[a] = P.hi[a];
    }
    std::memcpy(S.geo.plane, P.plane, sizeof P.plane);
    make_tables(p, S.T);
    const int L = S.T.L, L3 = L * L * L;

    // 1. classify every cell; keep the solid moments of crossed cells
    P.cell_elem.assign(P.ncells, -1);
    P.eta.assign(P.ncells, 0.0);
    std::vector<uint8_t> kind(P.ncells, 0);  // 0 void, 1 uncrossed solid, 2 crossed
    std::vector<std::vector<double>> moments(P.ncells);
    parallel_for(P.ncells, nthreads, [&](int64_t ci) {
        const int c[3] = {(int)(ci % P.n[0]), (int)((ci / P.n[0]) % P.n[1]), (int)(ci / ((int64_t)P.n[0] * P.n[1]))};
        double clo[3], chi[3];
        cell_box(P, c, clo, chi);
        if (!S.geo.crossed(clo, chi)) {
            double ctr[3];
            for (int a = 0; a < 3; ++a) ctr[a] = 0.5 * (clo[a] + chi[a]);
            if (S.geo.solid(ctr)) {
                kind[ci] = 1;
                P.eta[ci] = 1.0;
            }
            return;
        }
        std::vector<double> mu(L3, 0.0);
        bool any = false;
        cell_moments_rec(S, clo, clo, chi, 0, mu.data(), any);
        const double eta = mu[0] / 8.0;
        P.eta[ci] = eta;
        if (eta > 0.0) {
            kind[ci] = 2;
            moments[ci].swap(mu);
        }
    });
    int64_t ncut = 0, nact = 0;
    for (int64_t ci = 0; ci < P.ncells; ++ci) {
        if (kind[ci] == 1) P.cell_elem[ci] = 0;
        if (kind[ci] == 2) P.cell_elem[ci] = (int32_t)(1 + ncut++);
        nact += kind[ci] != 0;
    }
    P.ncut = ncut;
    P.nactive = nact;

    // 2. element matrices: the uncut reference and one per crossed cell
    const size_t ne2 = (size_t)P.ne * P.ne;
    P.Kref.assign(ne2, 0.0);
    std::vector<double> be_ref;
    {
        std::vector<double> mu(L3, 0.0);
        mu[0] = 8.0;
        element_from_moments(S, mu.data(), P.Kref.data());
        be_ref.assign(6 * (size_t)P.ne, 0.0);
        strain_loads_from_moments(S, mu.data(), be_ref.data());
    }
    P.Kcut.assign(ne2 * ncut, 0.0);
    std::vector<int64_t> cut_cells;
    cut_cells.reserve(ncut);
    for (int64_t ci = 0; ci < P.ncells; ++ci)
        if (kind[ci] == 2) cut_cells.push_back(ci);
    std::vector<double> be_cut(6 * (size_t)P.ne * ncut);
    parallel_for(ncut, nthreads, [&](int64_t k) {
        const int64_t ci = cut_cells[k];
        std::vector<double> mu(moments[ci]);
        for (int m = 0; m < L3; ++m) mu[m] *= (1.0 - P.alpha);
        mu[0] += 8.0 * P.alpha;
        element_from_moments(S, mu.data(), P.Kcut.data() + ne2 * k);
        strain_loads_from_moments(S, mu.data(), be_cut.data() + 6 * (size_t)P.ne * k);
        std::vector<double>().swap(moments[ci]);
    });

    // 3. free DOFs: nodes on an active cell, minus the Dirichlet ones
    std::vector<uint8_t> node_on(P.nnodes, 0);
    for (int64_t ci = 0; ci < P.ncells; ++ci) {
        if (P.cell_elem[ci] < 0) continue;
        const int c[3] = {(int)(ci % P.n[0]), (int)((ci / P.n[0]) % P.n[1]), (int)(ci / ((int64_t)P.n[0] * P.n[1]))};
        for (int iz = 0; iz <= p; ++iz)
            for (int iy = 0; iy <= p; ++iy)
                for (int ix = 0; ix <= p; ++ix)
                    node_on[(p * c[0] + ix) + (int64_t)P.M[0] * ((p * c[1] + iy) + (int64_t)P.M[1] * (p * c[2] + iz))] = 1;
    }
    P.mask.assign(P.nlat, 0);
    P.nfree = 0;
    for (int64_t node = 0; node < P.nnodes; ++node) {
        if (!node_on[node]) continue;
        const int i = (int)(node % P.M[0]), j = (int)((node / P.M[0]) % P.M[1]), k = (int)(node / ((int64_t)P.M[0] * P.M[1]));
        for (int comp = 0; comp < 3; ++comp) {
            bool fixed = false;
            if (P.bc == FCM_BC_CLAMP_ZLO) fixed = (k == 0);
            if (P.bc == FCM_BC_ROLLERS) fixed = (comp == 0 && i == 0) || (comp == 1 && j == 0) || (comp == 2 && k == 0);
            if (!fixed) {
                P.mask[3 * node + comp] = 1;
                ++P.nfree;
            }
        }
    }

    // 4a. unit-strain load cases 1..6
    P.rhs_strain.assign(6 * (size_t)P.nlat, 0.0);
    for (int64_t ci = 0; ci < P.ncells; ++ci) {
        const int32_t el = P.cell_elem[ci];
        if (el < 0) continue;
        const double *be = el == 0 ? be_ref.data() : be_cut.data() + 6 * (size_t)P.ne * (el - 1);
        const int c[3] = {(int)(ci % P.n[0]), (int)((ci / P.n[0]) % P.n[1]), (int)(ci / ((int64_t)P.n[0] * P.n[1]))};
        for (int iz = 0; iz <= p; ++iz)
            for (int iy = 0; iy <= p; ++iy)
                for (int ix = 0; ix <= p; ++ix) {
                    const int I = ix + q * (iy + q * iz);
                    const int64_t node = (p * c[0] + ix) + (int64_t)P.M[0] * ((p * c[1] + iy) + (int64_t)P.M[1] * (p * c[2] + iz));
                    for (int a = 0; a < 3; ++a) {
                        if (!P.mask[3 * node + a]) continue;
                        for (int k = 0; k < 6; ++k) P.rhs_strain[(size_t)k * P.nlat + 3 * node + a] += be[(size_t)k * P.ne + 3 * I + a];
                    }
                }
    }

    // 4. traction on the top faces of active top-layer cells
    P.rhs.assign(P.nlat, 0.0);
    const int64_t ntop = (int64_t)P.n[0] * P.n[1];
    std::vector<std::vector<double>> face(ntop);
    parallel_for(ntop, nthreads, [&](int64_t t) {
        const int c[3] = {(int)(t % P.n[0]), (int)(t / P.n[0]), P.n[2] - 1};
        const int64_t ci = c[0] + (int64_t)P.n[0] * (c[1] + (int64_t)P.n[1] * c[2]);
        if (P.cell_elem[ci] < 0) return;
        double clo[3], chi[3];
        cell_box(P, c, clo, chi);
        std::vector<double> nu(L * L, 0.0);
        const double flo[2] = {clo[0], clo[1]}, fhi[2] = {chi[0], chi[1]};
        face_moments_rec(S, clo, flo, fhi, 0, nu.data());
        face[t].swap(nu);
    });
    const double area = P.h[0] * P.h[1] / 4.0;
    for (int64_t t = 0; t < ntop; ++t) {
        if (face[t].empty()) continue;
        const int c[3] = {(int)(t % P.n[0]), (int)(t / P.n[0]), P.n[2] - 1};
        for (int i1 = 0; i1 <= p; ++i1)
            for (int i0 = 0; i0 <= p; ++i0) {
                double s = 0.0;
                for (int m0 = 0; m0 < L; ++m0)
                    for (int m1 = 0; m1 < L; ++m1) s += S.T.face[i0][m0] * S.T.face[i1][m1] * face[t][m0 * L + m1];
                const int64_t node = (p * c[0] + i0) + (int64_t)P.M[0] * ((p * c[1] + i1) + (int64_t)P.M[1] * (P.M[2] - 1));
                for (int a = 0; a < 3; ++a)
                    if (P.mask[3 * node + a]) P.rhs[3 * node + a] += area * s * P.traction[a];
            }
    }
    return std::string();
}

}  // namespace fcm

namespace fcm {

// One cell on the box [clo, chi]: its alpha-weighted element matrix (lattice order, 3 (p+1)^3 rows), its
// volume fraction eta, and, if face != nullptr, the solid-part integrals face[i1 (p+1) + i0] of
// N_i0(x) N_i1(y) over its top face z = chi[2] (physical area).  The same moment quadrature as the grid's
// cells, with the octree depth counted from this cell.  Voxel images span the domain box [dlo, dhi].
void box_cell_setup(const fcm_geometry &geom, const double *dlo, const double *dhi, int p, double alpha, double E,
                    double nu, const double *clo, const double *chi, double *K, double *eta, double *face)
{
    HostProblem P;
    P.p = p;
    P.alpha = alpha;
    P.E = E;
    P.nu = nu;
    P.bc = FCM_BC_NONE;
    for (int a = 0; a < 3; ++a) {
        P.n[a] = 1;
        P.lo[a] = clo[a];
        P.hi[a] = chi[a];
        P.h[a] = chi[a] - clo[a];
        P.M[a] = p + 1;
        P.traction[a] = 0.0;
    }
    P.gkind = geom.kind;
    P.depth = geom.octree_depth;
    std::memcpy(P.plane, geom.plane, sizeof P.plane);
    Setup S;
    S.P = &P;
    S.geo.kind = geom.kind;
    S.geo.sph = geom.sph;
    S.geo.nsph = geom.kind == FCM_GEOM_SPHERE_VOIDS ? geom.nsph : 0;
    S.geo.vox = geom.vox;
    for (int a = 0; a < 3; ++a) {
        S.geo.vdim[a] = geom.vdim[a];
        S.geo.lo[a] = dlo[a];
        S.geo.hi[a] = dhi[a];
    }
    std::memcpy(S.geo.plane, geom.plane, sizeof S.geo.plane);
    make_tables(p, S.T);
    const int L = S.T.L, L3 = L * L * L;
    std::vector<double> mu(L3, 0.0);
    if (!S.geo.crossed(clo, chi)) {
        double ctr[3];
        for (int a = 0; a < 3; ++a) ctr[a] = 0.5 * (clo[a] + chi[a]);
        const bool solid = S.geo.solid(ctr);
        *eta = solid ? 1.0 : 0.0;
        mu[0] = solid ? 8.0 : 8.0 * alpha;
    } else {
        bool any = false;
        cell_moments_rec(S, clo, clo, chi, 0, mu.data(), any);
        *eta = mu[0] / 8.0;
        for (int m = 0; m < L3; ++m) mu[m] *= (1.0 - alpha);
        mu[0] += 8.0 * alpha;
    }
    element_from_moments(S, mu.data(), K);
    if (face) {
        std::vector<double> fm(L * L, 0.0);
        const double flo[2] = {clo[0], clo[1]}, fhi[2] = {chi[0], chi[1]};
        face_moments_rec(S, clo, flo, fhi, 0, fm.data());
        const double area = P.h[0] * P.h[1] / 4.0;
        for (int i1 = 0; i1 <= p; ++i1)
            for (int i0 = 0; i0 <= p; ++i0) {
                double s = 0.0;
                for (int m0 = 0; m0 < L; ++m0)
                    for (int m1 = 0; m1 < L; ++m1) s += S.T.face[i0][m0] * S.T.face[i1][m1] * fm[m0 * L + m1];
                face[i1 * (p + 1) + i0] = area * s;
            }
    }
}

}  // namespace fcm
