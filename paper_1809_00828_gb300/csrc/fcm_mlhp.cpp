// Multi-level hp hierarchy and its leaf blocks: the host-side plan (Sec. 2.2, Sec. 3.2).
//
// A base grid of cells is refined toward the domain boundary (sphere surfaces, a voxel image's solid-void
// interfaces or a plane) by superposed overlays: level l + 1 holds the 8
// children of every refined level-l cell.  Every level carries its own integrated-Legendre basis, one
// set of modes per topological component (vertex, edge, face, cell) of the level's grid.  A level-l
// component is active iff every in-domain level-l cell position around it exists (the overlay's
// homogeneous Dirichlet boundary, Sec. 2.2) and at least one of them is a leaf (components a finer
// overlay covers are deactivated for linear independence).
//
// Blocks are per leaf (Sec. 3.2 "Selecting suitable blocks"): the full block holds every active function
// supported on the leaf; the truncated block holds the leaf's own-level functions plus, for each leaf
// corner whose own-level vertex function is inactive, the vertex function of the highest coarser level
// at which the corner point is a vertex and is active (the 1D rule of Sec. 3.2 applied to the trilinear
// functions).
//
// A level-l function restricted to a level-L leaf is a polynomial of the leaf's own tensor-product space:
// fcm_mlhp_restriction gives its 1D coefficients per axis in the leaf's basis (N0, N1, phi_2..phi_p), so
// a leaf's stiffness is C K_leaf C^T with the leaf's standard element matrix K_leaf.
//
// Enumeration orders (binding for callers that compare with other implementations): functions level by
// level, components sorted by (z, y, x), modes with the bubble index of the lowest odd axis slowest;
// leaves by level, then by (x, y, z) lexicographically; a leaf's full block level by level from 0, the
// components of the ancestor's closure with x fastest.
#include "fcm.h"
#include "fcm_internal.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <array>
#include <cmath>
#include <cstdint>
#include <new>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

using I3 = std::array<int, 3>;

uint64_t key3(const I3 &c) { return (uint64_t)c[0] | ((uint64_t)c[1] << 21) | ((uint64_t)c[2] << 42); }

// 1D shape functions on [-1, 1] in the order N0, N1, phi_2..phi_p (Sec. 2.1 integrated Legendre).
void shape1d(int p, double xi, double *f)
{
    double P[6];
    P[0] = 1.0;
    P[1] = xi;
    for (int k = 1; k < p; ++k) P[k + 1] = ((2 * k + 1) * xi * P[k] - k * P[k - 1]) / (k + 1);
    f[0] = 0.5 * (1.0 - xi);
    f[1] = 0.5 * (1.0 + xi);
    for (int j = 2; j <= p; ++j) f[j] = (P[j] - P[j - 2]) / std::sqrt(2.0 * (2 * j - 1));
}

// Eigen-decomposition of a symmetric n x n matrix by cyclic Jacobi rotations (Golub & Van Loan,
// Matrix Computations, Sec. 8.5): A (row-major) is overwritten, lam[k] and column k of V (row-major) are the
// eigenpairs.  Sweeps until the off-diagonal part is below 1e-15 of the Frobenius norm (at most 100).
void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &lam, std::vector<double> &V)
{
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double v : A) fro += v * v;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += 2.0 * A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (off <= 1e-30 * fro) break;
        for (int pp = 0; pp < n - 1; ++pp)
            for (int qq = pp + 1; qq < n; ++qq) {
                const double apq = A[(size_t)pp * n + qq];
                if (apq == 0.0) continue;
                const double app = A[(size_t)pp * n + pp], aqq = A[(size_t)qq * n + qq];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns pp, qq of A
                    const double akp = A[(size_t)k * n + pp], akq = A[(size_t)k * n + qq];
                    A[(size_t)k * n + pp] = c * akp - s * akq;
                    A[(size_t)k * n + qq] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows pp, qq of A
                    const double apk = A[(size_t)pp * n + k], aqk = A[(size_t)qq * n + k];
                    A[(size_t)pp * n + k] = c * apk - s * aqk;
                    A[(size_t)qq * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // columns pp, qq of V
                    const double vkp = V[(size_t)k * n + pp], vkq = V[(size_t)k * n + qq];
                    V[(size_t)k * n + pp] = c * vkp - s * vkq;
                    V[(size_t)k * n + qq] = s * vkp + c * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

}  // namespace

struct fcm_mlhp {
    std::string err;  // message of the last failed device call (fcm_mlhp_last_error)
    int n[3] = {0, 0, 0};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int p = 0, levels = 0;
    std::vector<std::unordered_set<uint64_t>> cells, refined;
    std::vector<std::pair<int, I3>> leaves;
    // functions: level, component (doubled coordinates), mode (0 on vertex axes, 2..p on bubble axes)
    std::vector<int> f_level;
    std::vector<I3> f_comp, f_mode;
    std::vector<std::unordered_map<uint64_t, int64_t>> first;  // per level: component -> its first function
    int64_t n_trunk = 0;
    int nmax_full = 0, nmax_trunc = 0, maxb_full = 0, maxb_trunc = 0;
    // geometry of the refinement, kept for the assembly
    // the physical domain: spheres (kind 0), a voxel image over the box (kind 1) or a half space (kind 2)
    int gkind = 0;
    std::vector<double> sph;
    std::vector<uint8_t> vox;
    int vdim[3] = {1, 1, 1};
    double plane[4] = {0.0, 0.0, 1.0, 2.0};
    int depth = 0;

    // The boundary crosses the closed box [blo, bhi] (the refinement test): spheres, min distance < r < max
    // distance from the centre; voxels, the voxels the box overlaps are not all equal; half space,
    // min a.x < d < max a.x over the box.
    bool crossed(const double *blo, const double *bhi) const
    {
        if (gkind == FCM_GEOM_SPHERE_VOIDS) {
            for (size_t s4 = 0; s4 + 3 < sph.size(); s4 += 4) {
                double dn = 0.0, df = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double c = sph[s4 + a];
                    const double nr = std::min(std::max(c, blo[a]), bhi[a]);
                    const double fr = std::fabs(c - blo[a]) > std::fabs(c - bhi[a]) ? blo[a] : bhi[a];
                    dn += (c - nr) * (c - nr);
                    df += (c - fr) * (c - fr);
                }
                if (std::sqrt(dn) < sph[s4 + 3] && sph[s4 + 3] < std::sqrt(df)) return true;
            }
            return false;
        }
        if (gkind == FCM_GEOM_VOXELS) {
            int i0[3], i1[3];
            for (int a = 0; a < 3; ++a) {
                const double h = (hi[a] - lo[a]) / vdim[a];
                i0[a] = (int)std::floor((blo[a] - lo[a]) / h);
                i1[a] = (int)std::ceil((bhi[a] - lo[a]) / h) - 1;
                if (i1[a] < i0[a]) i1[a] = i0[a];
                i0[a] = std::min(std::max(i0[a], 0), vdim[a] - 1);
                i1[a] = std::min(std::max(i1[a], 0), vdim[a] - 1);
            }
            int first = -1;
            for (int z = i0[2]; z <= i1[2]; ++z)
                for (int y = i0[1]; y <= i1[1]; ++y)
                    for (int x = i0[0]; x <= i1[0]; ++x) {
                        const int v = vox[x + (size_t)vdim[0] * (y + (size_t)vdim[1] * z)] != 0;
                        if (first < 0) first = v;
                        else if (v != first) return true;
                    }
            return false;
        }
        double mn = 0.0, mx = 0.0;
        for (int a = 0; a < 3; ++a) {
            mn += std::min(plane[a] * blo[a], plane[a] * bhi[a]);
            mx += std::max(plane[a] * blo[a], plane[a] * bhi[a]);
        }
        return mn < plane[3] && plane[3] < mx;
    }
    // assembled system (fcm_mlhp_assemble): free DOFs 3 f + comp ascending, CSR over them, load
    bool assembled = false;
    std::vector<double> leaf_eta;
    std::vector<int64_t> free_dofs, rowptr, cols;
    std::vector<double> vals, rhs;
    // Schwarz factors (fcm_mlhp_factorize): blocks over free DOFs in colour order, their pseudo inverses
    // (row-major, one after the other), the colour ranges of blocks, and 1 / K_ll for free DOFs in no block
    bool factorized = false;
    // device copy (fcm_mlhp_device_setup)
    fcm::MlhpDevice *dev = nullptr;

    ~fcm_mlhp() { fcm::mlhp_device_destroy(dev); }
    std::vector<int64_t> blk_ptr, blk_dofs, fac_ptr, colour_ptr;
    std::vector<double> factors, jacobi;
    std::vector<double> fac_cond;  // retained condition number lambda_max / lambda_min of each block
    int precision = FCM_PREC_FP64;  // fcm_mlhp_set_precision: factor storage of the next device set-up

    int ext(int l, int a) const { return n[a] << l; }

    bool has(int l, const I3 &c) const { return cells[l].count(key3(c)) != 0; }
    bool is_refined(int l, const I3 &c) const { return refined[l].count(key3(c)) != 0; }

    bool active(int l, const I3 &q) const
    {
        int lists[3][2], cnt[3];
        for (int a = 0; a < 3; ++a) {
            cnt[a] = 0;
            if (q[a] % 2) {
                lists[a][cnt[a]++] = (q[a] - 1) / 2;
            } else {
                for (int i : {q[a] / 2 - 1, q[a] / 2})
                    if (i >= 0 && i < ext(l, a)) lists[a][cnt[a]++] = i;
            }
        }
        bool any_leaf = false;
        for (int i = 0; i < cnt[0]; ++i)
            for (int j = 0; j < cnt[1]; ++j)
                for (int k = 0; k < cnt[2]; ++k) {
                    const I3 c = {lists[0][i], lists[1][j], lists[2][k]};
                    if (!has(l, c)) return false;
                    if (!is_refined(l, c)) any_leaf = true;
                }
        return any_leaf;
    }

    int64_t nmodes(const I3 &q) const
    {
        int64_t m = 1;
        for (int a = 0; a < 3; ++a)
            if (q[a] & 1) m *= p - 1;
        return m;
    }

    // append the functions of active component q of level l
    void append_component(int l, const I3 &q, std::vector<int64_t> &out) const
    {
        const auto it = first[l].find(key3(q));
        const int64_t m = nmodes(q);
        for (int64_t i = 0; i < m; ++i) out.push_back(it->second + i);
    }

    static std::array<I3, 27> closure(const I3 &c)
    {
        std::array<I3, 27> out;
        int t = 0;
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) out[t++] = {2 * c[0] + i, 2 * c[1] + j, 2 * c[2] + k};
        return out;
    }

    void full_block(int L, const I3 &c, std::vector<int64_t> &out) const
    {
        for (int l = 0; l <= L; ++l) {
            const I3 A = {c[0] >> (L - l), c[1] >> (L - l), c[2] >> (L - l)};
            for (const I3 &q : closure(A))
                if (active(l, q)) append_component(l, q, out);
        }
    }

    void truncated_block(int L, const I3 &c, std::vector<int64_t> &out) const
    {
        for (const I3 &q : closure(c))
            if (active(L, q)) append_component(L, q, out);
        for (int cx : {0, 2})
            for (int cy : {0, 2})
                for (int cz : {0, 2}) {
                    const I3 q = {2 * c[0] + cx, 2 * c[1] + cy, 2 * c[2] + cz};
                    if (active(L, q)) continue;
                    for (int l = L - 1; l >= 0; --l) {
                        const int s = 1 << (L - l);
                        if (q[0] % (2 * s) || q[1] % (2 * s) || q[2] % (2 * s)) break;  // not a vertex of level l
                        const I3 ql = {q[0] / s, q[1] / s, q[2] / s};
                        if (active(l, ql)) {
                            out.push_back(first[l].find(key3(ql))->second);
                            break;
                        }
                    }
                }
    }

    void build(int k)
    {
        std::unordered_set<uint64_t> base;
        for (int z = 0; z < n[2]; ++z)
            for (int y = 0; y < n[1]; ++y)
                for (int x = 0; x < n[0]; ++x) base.insert(key3({x, y, z}));
        cells.push_back(base);
        for (int l = 0; l < k; ++l) {
            std::unordered_set<uint64_t> R, next;
            double h[3];
            for (int a = 0; a < 3; ++a) h[a] = (hi[a] - lo[a]) / (double)(n[a] << l);
            for (uint64_t key : cells[l]) {
                const I3 c = {(int)(key & 0x1fffff), (int)((key >> 21) & 0x1fffff), (int)(key >> 42)};
                double blo[3], bhi[3];
                for (int a = 0; a < 3; ++a) {
                    blo[a] = lo[a] + c[a] * h[a];
                    bhi[a] = lo[a] + (c[a] + 1) * h[a];
                }
                if (!crossed(blo, bhi)) continue;
                R.insert(key);
                for (int i = 0; i < 8; ++i)
                    next.insert(key3({2 * c[0] + (i & 1), 2 * c[1] + ((i >> 1) & 1), 2 * c[2] + (i >> 2)}));
            }
            refined.push_back(R);
            if (R.empty()) break;
            cells.push_back(next);
        }
        while (refined.size() < cells.size()) refined.emplace_back();
        levels = (int)cells.size();
        // leaves, by level and then (x, y, z) lexicographically
        for (int l = 0; l < levels; ++l) {
            std::vector<I3> lv;
            for (uint64_t key : cells[l])
                if (!refined[l].count(key))
                    lv.push_back({(int)(key & 0x1fffff), (int)((key >> 21) & 0x1fffff), (int)(key >> 42)});
            std::sort(lv.begin(), lv.end());
            for (const I3 &c : lv) leaves.push_back({l, c});
        }
        // functions, level by level, components sorted by (z, y, x)
        first.resize(levels);
        for (int l = 0; l < levels; ++l) {
            std::unordered_set<uint64_t> seen;
            std::vector<I3> comps;
            for (uint64_t key : cells[l]) {
                const I3 c = {(int)(key & 0x1fffff), (int)((key >> 21) & 0x1fffff), (int)(key >> 42)};
                for (const I3 &q : closure(c))
                    if (seen.insert(key3(q)).second) comps.push_back(q);
            }
            std::sort(comps.begin(), comps.end(), [](const I3 &a, const I3 &b) {
                return std::make_tuple(a[2], a[1], a[0]) < std::make_tuple(b[2], b[1], b[0]);
            });
            for (const I3 &q : comps) {
                if (!active(l, q)) continue;
                first[l][key3(q)] = (int64_t)f_level.size();
                int odd[3], no = 0;
                for (int a = 0; a < 3; ++a)
                    if (q[a] & 1) odd[no++] = a;
                const int64_t m = nmodes(q);
                for (int64_t i = 0; i < m; ++i) {
                    I3 mode = {0, 0, 0};
                    int64_t r = i;
                    for (int t = no - 1; t >= 0; --t) {  // lowest odd axis slowest
                        mode[odd[t]] = 2 + (int)(r % (p - 1));
                        r /= p - 1;
                    }
                    f_level.push_back(l);
                    f_comp.push_back(q);
                    f_mode.push_back(mode);
                }
                // trunk space: the bubble indices of a face or cell sum to at most p
                if (no <= 1) {
                    n_trunk += m;
                } else {
                    for (int64_t i = 0; i < m; ++i) {
                        int64_t r = i, sum = 0;
                        for (int t = 0; t < no; ++t) {
                            sum += 2 + r % (p - 1);
                            r /= p - 1;
                        }
                        if (sum <= p) ++n_trunk;
                    }
                }
            }
        }
        // block overlap and sizes over all leaves
        std::vector<int> cf(f_level.size(), 0), ct(f_level.size(), 0);
        std::vector<int64_t> b;
        for (const auto &lf : leaves) {
            b.clear();
            full_block(lf.first, lf.second, b);
            maxb_full = std::max(maxb_full, (int)b.size());
            for (int64_t f : b) ++cf[f];
            b.clear();
            truncated_block(lf.first, lf.second, b);
            maxb_trunc = std::max(maxb_trunc, (int)b.size());
            for (int64_t f : b) ++ct[f];
        }
        for (size_t f = 0; f < cf.size(); ++f) {
            nmax_full = std::max(nmax_full, cf[f]);
            nmax_trunc = std::max(nmax_trunc, ct[f]);
        }
    }

    // Eq. (1) on the leaves: K = sum over leaves with eta > 0 of C K_cell C^T, C the restriction of the
    // leaf's functions to its own lattice-ordered basis and K_cell the cell matrix of the leaf's box; the
    // traction on the top face z = hi[2] the same way.  Returns an error message or "".
    std::string assemble(double alpha, const fcm_bc &bc)
    {
        const int q = p + 1, nl = q * q * q, ne = 3 * nl;
        fcm_geometry g;
        std::memset(&g, 0, sizeof g);
        g.kind = gkind;
        g.nsph = (int)(sph.size() / 4);
        g.sph = sph.data();
        g.vox = vox.data();
        for (int a = 0; a < 3; ++a) g.vdim[a] = vdim[a];
        for (int a = 0; a < 4; ++a) g.plane[a] = plane[a];
        g.octree_depth = depth;
        const int64_t nleaf = (int64_t)leaves.size();
        leaf_eta.assign(nleaf, 0.0);
        std::vector<std::vector<double>> Kc(nleaf), face(nleaf);
        std::atomic<int64_t> next(0);
        auto work = [&]() {
            for (int64_t i = next++; i < nleaf; i = next++) {
                const int L = leaves[i].first;
                const I3 &c = leaves[i].second;
                double clo[3], chi[3];
                for (int a = 0; a < 3; ++a) {
                    const double h = (hi[a] - lo[a]) / (double)(n[a] << L);
                    clo[a] = lo[a] + c[a] * h;
                    chi[a] = clo[a] + h;
                }
                const bool top = c[2] == ext(L, 2) - 1;
                Kc[i].assign((size_t)ne * ne, 0.0);
                if (top) face[i].assign((size_t)q * q, 0.0);
                fcm::box_cell_setup(g, lo, hi, p, alpha, bc.E, bc.nu, clo, chi, Kc[i].data(), &leaf_eta[i],
                                    top ? face[i].data() : nullptr);
                if (!(leaf_eta[i] > 0.0)) {
                    std::vector<double>().swap(Kc[i]);
                    std::vector<double>().swap(face[i]);
                }
            }
        };
        const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(work);
        work();
        for (auto &t : pool) t.join();
        // kept functions (some active leaf in their support) and free DOFs
        const int64_t nf = (int64_t)f_level.size();
        std::vector<uint8_t> kept(nf, 0);
        std::vector<std::vector<int64_t>> blocks(nleaf);
        for (int64_t i = 0; i < nleaf; ++i) {
            if (!(leaf_eta[i] > 0.0)) continue;
            full_block(leaves[i].first, leaves[i].second, blocks[i]);
            for (int64_t f : blocks[i]) kept[f] = 1;
        }
        std::vector<int64_t> pos(3 * nf, -1);
        free_dofs.clear();
        for (int64_t f = 0; f < nf; ++f) {
            if (!kept[f]) continue;
            for (int a = 0; a < 3; ++a) {
                bool fixed = false;
                if (bc.bc == FCM_BC_CLAMP_ZLO) fixed = f_comp[f][2] == 0;
                if (bc.bc == FCM_BC_ROLLERS) fixed = f_comp[f][a] == 0;
                if (!fixed) {
                    pos[3 * f + a] = (int64_t)free_dofs.size();
                    free_dofs.push_back(3 * f + a);
                }
            }
        }
        const int64_t nfree = (int64_t)free_dofs.size();
        // leaf matrices through the restriction, gathered as (row, col, value)
        std::vector<std::vector<std::pair<int64_t, double>>> rows(nfree);
        rhs.assign(nfree, 0.0);
        std::vector<double> coef(3 * q), C, T;
        for (int64_t i = 0; i < nleaf; ++i) {
            if (!(leaf_eta[i] > 0.0)) continue;
            const std::vector<int64_t> &fb = blocks[i];
            const int m = (int)fb.size();
            C.assign((size_t)m * nl, 0.0);
            std::vector<double> ztop(m, 0.0);
            for (int r = 0; r < m; ++r) {
                restriction(i, fb[r], coef.data());
                double cl[3][5];  // lattice order (N0, phi_2 .. phi_p, N1) from (N0, N1, phi_2 .. phi_p)
                for (int a = 0; a < 3; ++a)
                    for (int j = 0; j < q; ++j) cl[a][j] = coef[a * q + (j == p ? 1 : (j == 0 ? 0 : j + 1))];
                for (int iz = 0; iz < q; ++iz)
                    for (int iy = 0; iy < q; ++iy)
                        for (int ix = 0; ix < q; ++ix)
                            C[(size_t)r * nl + ix + q * (iy + q * iz)] = cl[0][ix] * cl[1][iy] * cl[2][iz];
                if (!face[i].empty()) {
                    double s = 0.0;
                    for (int iy = 0; iy < q; ++iy)
                        for (int ix = 0; ix < q; ++ix) s += cl[0][ix] * cl[1][iy] * face[i][iy * q + ix];
                    ztop[r] = s * cl[2][p];  // only N1 is nonzero on the top face
                }
            }
            // T[(I,a)][(g,b)] = sum_J K_cell[(I,a)][(J,b)] C[g][J]
            T.assign((size_t)ne * 3 * m, 0.0);
            for (int I3i = 0; I3i < ne; ++I3i)
                for (int gI = 0; gI < m; ++gI)
                    for (int b = 0; b < 3; ++b) {
                        double s = 0.0;
                        const double *krow = Kc[i].data() + (size_t)I3i * ne;
                        const double *cg = C.data() + (size_t)gI * nl;
                        for (int J = 0; J < nl; ++J) s += krow[3 * J + b] * cg[J];
                        T[(size_t)I3i * 3 * m + 3 * gI + b] = s;
                    }
            for (int fI = 0; fI < m; ++fI)
                for (int a = 0; a < 3; ++a) {
                    const int64_t r = pos[3 * fb[fI] + a];
                    if (r < 0) continue;
                    if (!face[i].empty()) rhs[r] += bc.traction[a] * ztop[fI];
                    const double *cf = C.data() + (size_t)fI * nl;
                    for (int gI = 0; gI < m; ++gI)
                        for (int b = 0; b < 3; ++b) {
                            const int64_t col = pos[3 * fb[gI] + b];
                            if (col < 0) continue;
                            double s = 0.0;
                            for (int I = 0; I < nl; ++I) s += cf[I] * T[(size_t)(3 * I + a) * 3 * m + 3 * gI + b];
                            rows[r].push_back({col, s});
                        }
                }
        }
        rowptr.assign(nfree + 1, 0);
        cols.clear();
        vals.clear();
        for (int64_t r = 0; r < nfree; ++r) {
            auto &v = rows[r];
            std::sort(v.begin(), v.end(), [](const std::pair<int64_t, double> &x, const std::pair<int64_t, double> &y) {
                return x.first < y.first;
            });
            for (size_t k = 0; k < v.size(); ++k) {
                if (!cols.empty() && (int64_t)cols.size() > rowptr[r] && cols.back() == v[k].first) {
                    vals.back() += v[k].second;
                } else {
                    cols.push_back(v[k].first);
                    vals.push_back(v[k].second);
                }
            }
            std::vector<std::pair<int64_t, double>>().swap(v);
            rowptr[r + 1] = (int64_t)cols.size();
        }
        assembled = true;
        return std::string();
    }

    // Sec. 3.2 / Algorithm 1 on the assembled system: a block per leaf with 0 < eta <= eta_bar (its full or
    // truncated functions, the free DOFs among them), A_B^+ = V diag(1/lambda, lambda > eps lambda_max) V^T, and the
    // diagonal part for free DOFs in no block.  Blocks are coloured greedily (no two blocks of one colour
    // share a DOF) and stored colour by colour.
    // on_device: the blocks' eigensolves run batched on the current CUDA device (stream); the result is the
    // same pseudo inverse up to the two eigensolvers' rounding.  Returns "" or the device failure.
    std::string factorize(int kind, double eps, double eta_bar, bool on_device = false, void *stream = nullptr)
    {
        const int64_t nfree = (int64_t)free_dofs.size();
        std::vector<int64_t> pos(3 * f_level.size(), -1);
        for (int64_t i = 0; i < nfree; ++i) pos[free_dofs[i]] = i;
        std::vector<std::vector<int64_t>> blocks;
        std::vector<int64_t> fb;
        for (size_t i = 0; i < leaves.size(); ++i) {
            if (!(leaf_eta[i] > 0.0) || std::min(leaf_eta[i], 1.0) > eta_bar) continue;  // Sec. 3.2 threshold
            fb.clear();
            if (kind == 0) full_block(leaves[i].first, leaves[i].second, fb);
            else truncated_block(leaves[i].first, leaves[i].second, fb);
            std::vector<int64_t> loc;
            for (int64_t f : fb)
                for (int a = 0; a < 3; ++a)
                    if (pos[3 * f + a] >= 0) loc.push_back(pos[3 * f + a]);
            std::sort(loc.begin(), loc.end());
            loc.erase(std::unique(loc.begin(), loc.end()), loc.end());
            if (!loc.empty()) blocks.push_back(std::move(loc));
        }
        // greedy colours over free DOFs
        std::vector<int> colour(blocks.size(), 0);
        std::vector<std::vector<uint8_t>> used;
        int nc = 0;
        for (size_t b = 0; b < blocks.size(); ++b) {
            int c = 0;
            for (;; ++c) {
                if (c >= nc) break;
                bool clash = false;
                for (int64_t d : blocks[b])
                    if (used[c][d]) {
                        clash = true;
                        break;
                    }
                if (!clash) break;
            }
            if (c == nc) {
                used.emplace_back(nfree, 0);
                ++nc;
            }
            colour[b] = c;
            for (int64_t d : blocks[b]) used[c][d] = 1;
        }
        std::vector<size_t> order(blocks.size());
        for (size_t b = 0; b < order.size(); ++b) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return colour[x] < colour[y]; });
        colour_ptr.assign(nc + 1, 0);
        for (size_t b = 0; b < blocks.size(); ++b) ++colour_ptr[colour[b] + 1];
        for (int c = 0; c < nc; ++c) colour_ptr[c + 1] += colour_ptr[c];
        blk_ptr.assign(1, 0);
        blk_dofs.clear();
        fac_ptr.assign(1, 0);
        for (size_t b : order) {
            blk_dofs.insert(blk_dofs.end(), blocks[b].begin(), blocks[b].end());
            blk_ptr.push_back((int64_t)blk_dofs.size());
            fac_ptr.push_back(fac_ptr.back() + (int64_t)blocks[b].size() * (int64_t)blocks[b].size());
        }
        factors.assign(fac_ptr.back(), 0.0);
        fac_cond.assign(order.size(), 1.0);
        std::vector<double> dense;  // the blocks themselves, for the device eigensolves
        if (on_device) dense.assign(fac_ptr.back(), 0.0);
        // pseudo inverses (or, on_device, the dense blocks), in parallel over blocks
        std::atomic<size_t> next(0);
        auto work = [&]() {
            std::vector<int64_t> where(nfree, -1);
            std::vector<double> A, lam, V;
            for (size_t k = next++; k < order.size(); k = next++) {
                const int64_t *B = blk_dofs.data() + blk_ptr[k];
                const int m = (int)(blk_ptr[k + 1] - blk_ptr[k]);
                for (int i = 0; i < m; ++i) where[B[i]] = i;
                A.assign((size_t)m * m, 0.0);
                for (int i = 0; i < m; ++i)
                    for (int64_t e = rowptr[B[i]]; e < rowptr[B[i] + 1]; ++e)
                        if (where[cols[e]] >= 0) A[(size_t)i * m + where[cols[e]]] = vals[e];
                for (int i = 0; i < m; ++i) where[B[i]] = -1;
                for (int i = 0; i < m; ++i)  // exact symmetry
                    for (int j = i + 1; j < m; ++j) {
                        const double v = 0.5 * (A[(size_t)i * m + j] + A[(size_t)j * m + i]);
                        A[(size_t)i * m + j] = A[(size_t)j * m + i] = v;
                    }
                if (on_device) {
                    std::copy(A.begin(), A.end(), dense.begin() + fac_ptr[k]);
                    continue;
                }
                jacobi_eigen(m, A, lam, V);
                double lmax = 0.0;
                for (double l : lam) lmax = std::max(lmax, l);
                double lmin = lmax;
                for (double l : lam)
                    if (l > eps * lmax) lmin = std::min(lmin, l);
                fac_cond[k] = lmin > 0.0 ? lmax / lmin : 1.0;
                double *F = factors.data() + fac_ptr[k];
                for (int t = 0; t < m; ++t) {
                    if (!(lam[t] > eps * lmax)) continue;
                    const double inv = 1.0 / lam[t];
                    for (int i = 0; i < m; ++i) {
                        const double vi = V[(size_t)i * m + t] * inv;
                        for (int j = 0; j < m; ++j) F[(size_t)i * m + j] += vi * V[(size_t)j * m + t];
                    }
                }
            }
        };
        const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(work);
        work();
        for (auto &t : pool) t.join();
        if (on_device) {
            const std::string e = fcm::mlhp_device_pinv(stream, (int64_t)order.size(), fac_ptr.data(), dense.data(), eps,
                                                        factors.data(), fac_cond.data());
            if (!e.empty()) return e;
        }
        // diagonal part for free DOFs in no block
        std::vector<uint8_t> covered(nfree, 0);
        for (int64_t d : blk_dofs) covered[d] = 1;
        jacobi.assign(nfree, 0.0);
        for (int64_t i = 0; i < nfree; ++i) {
            if (covered[i]) continue;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
                if (cols[e] == i) jacobi[i] = 1.0 / vals[e];
        }
        factorized = true;
        return std::string();
    }

    // 1D factor of function f along axis a on leaf (L, c), as coefficients in the leaf's 1D basis
    bool restriction(int64_t leaf, int64_t f, double *coef) const
    {
        const int L = leaves[leaf].first;
        const I3 &c = leaves[leaf].second;
        const int l = f_level[f];
        if (l > L) return false;
        const int s = 1 << (L - l);
        const I3 A = {c[0] >> (L - l), c[1] >> (L - l), c[2] >> (L - l)};
        const I3 &q = f_comp[f];
        for (int a = 0; a < 3; ++a) {  // supported on the leaf: q in the closure of the ancestor
            if (q[a] < 2 * A[a] || q[a] > 2 * A[a] + 2) return false;
        }
        const int np = p + 1;
        for (int a = 0; a < 3; ++a) {
            const int off = c[a] - A[a] * s;
            // collocation at p + 1 equispaced leaf points: V coef = g(xi(t))
            double V[5][6];
            for (int k = 0; k < np; ++k) {
                const double t = -1.0 + 2.0 * k / p;
                shape1d(p, t, V[k]);
                double g[5];
                shape1d(p, -1.0 + (2 * off + 1 + t) / s, g);
                const int which = (q[a] & 1) ? f_mode[f][a] : (q[a] / 2 == A[a] ? 0 : 1);
                V[k][np] = g[which];
            }
            for (int col = 0; col < np; ++col) {  // Gaussian elimination with partial pivoting
                int piv = col;
                for (int r = col + 1; r < np; ++r)
                    if (std::fabs(V[r][col]) > std::fabs(V[piv][col])) piv = r;
                for (int j = 0; j <= np; ++j) std::swap(V[col][j], V[piv][j]);
                for (int r = 0; r < np; ++r) {
                    if (r == col) continue;
                    const double m = V[r][col] / V[col][col];
                    for (int j = col; j <= np; ++j) V[r][j] -= m * V[col][j];
                }
            }
            for (int j = 0; j < np; ++j) coef[a * np + j] = V[j][np] / V[j][j];
        }
        return true;
    }
};

extern "C" {

fcm_status fcm_mlhp_create(const fcm_grid *grid, const fcm_geometry *geom, int p, int k, fcm_mlhp **out)
{
    if (!out) return FCM_EINVAL;
    *out = nullptr;
    if (!grid || !geom || p < 1 || p > 4 || k < 0 || k > 10 || geom->octree_depth < 0 || geom->octree_depth > 12)
        return FCM_EINVAL;
    if (geom->kind == FCM_GEOM_SPHERE_VOIDS) {
        if (geom->nsph < 0 || (geom->nsph > 0 && !geom->sph)) return FCM_EINVAL;
    } else if (geom->kind == FCM_GEOM_VOXELS) {
        if (!geom->vox || geom->vdim[0] < 1 || geom->vdim[1] < 1 || geom->vdim[2] < 1) return FCM_EINVAL;
    } else if (geom->kind != FCM_GEOM_HALFSPACE) {
        return FCM_EINVAL;
    }
    for (int a = 0; a < 3; ++a) {
        if (grid->n[a] < 1 || ((int64_t)grid->n[a] << k) >= (1 << 20) || !(grid->hi[a] > grid->lo[a])) return FCM_EINVAL;
    }
    fcm_mlhp *h = new (std::nothrow) fcm_mlhp;
    if (!h) return FCM_ENOMEM;
    try {
        for (int a = 0; a < 3; ++a) {
            h->n[a] = grid->n[a];
            h->lo[a] = grid->lo[a];
            h->hi[a] = grid->hi[a];
        }
        h->p = p;
        h->gkind = geom->kind;
        if (geom->kind == FCM_GEOM_SPHERE_VOIDS) h->sph.assign(geom->sph, geom->sph + 4 * (size_t)geom->nsph);
        if (geom->kind == FCM_GEOM_VOXELS) {
            for (int a = 0; a < 3; ++a) h->vdim[a] = geom->vdim[a];
            h->vox.assign(geom->vox, geom->vox + (size_t)geom->vdim[0] * geom->vdim[1] * geom->vdim[2]);
        }
        for (int a = 0; a < 4; ++a) h->plane[a] = geom->plane[a];
        h->depth = geom->octree_depth;
        h->build(k);
    } catch (...) {
        delete h;
        return FCM_ENOMEM;
    }
    *out = h;
    return FCM_OK;
}

fcm_status fcm_mlhp_get_info(const fcm_mlhp *h, fcm_mlhp_info *info)
{
    if (!h || !info) return FCM_EINVAL;
    info->levels = h->levels;
    info->n_leaves = (int64_t)h->leaves.size();
    info->n_functions = (int64_t)h->f_level.size();
    info->n_functions_trunk = h->n_trunk;
    info->n_max_full = h->nmax_full;
    info->n_max_truncated = h->nmax_trunc;
    info->max_block_full = h->maxb_full;
    info->max_block_truncated = h->maxb_trunc;
    return FCM_OK;
}

fcm_status fcm_mlhp_leaf(const fcm_mlhp *h, int64_t leaf, int *level, int cell[3])
{
    if (!h || !level || !cell || leaf < 0 || leaf >= (int64_t)h->leaves.size()) return FCM_EINVAL;
    *level = h->leaves[leaf].first;
    for (int a = 0; a < 3; ++a) cell[a] = h->leaves[leaf].second[a];
    return FCM_OK;
}

fcm_status fcm_mlhp_function(const fcm_mlhp *h, int64_t f, int *level, int comp[3], int mode[3])
{
    if (!h || !level || !comp || !mode || f < 0 || f >= (int64_t)h->f_level.size()) return FCM_EINVAL;
    *level = h->f_level[f];
    for (int a = 0; a < 3; ++a) {
        comp[a] = h->f_comp[f][a];
        mode[a] = h->f_mode[f][a];
    }
    return FCM_OK;
}

fcm_status fcm_mlhp_block(const fcm_mlhp *h, int64_t leaf, int kind, int64_t *fids, int cap, int *count)
{
    if (!h || !count || leaf < 0 || leaf >= (int64_t)h->leaves.size() || (kind != 0 && kind != 1) || cap < 0 ||
        (cap > 0 && !fids))
        return FCM_EINVAL;
    std::vector<int64_t> b;
    try {
        if (kind == 0) h->full_block(h->leaves[leaf].first, h->leaves[leaf].second, b);
        else h->truncated_block(h->leaves[leaf].first, h->leaves[leaf].second, b);
    } catch (...) {
        return FCM_ENOMEM;
    }
    *count = (int)b.size();
    if ((int)b.size() > cap) return FCM_EINVAL;
    std::copy(b.begin(), b.end(), fids);
    return FCM_OK;
}

fcm_status fcm_mlhp_colour(const fcm_mlhp *h, int kind, int *colour, int *n_colours)
{
    if (!h || !colour || !n_colours || (kind != 0 && kind != 1)) return FCM_EINVAL;
    // greedy, leaves in plan order: the lowest colour that no block sharing a function already has
    std::vector<uint64_t> used;
    try {
        used.assign(h->f_level.size(), 0);
        std::vector<int64_t> b;
        int nc = 0;
        for (size_t i = 0; i < h->leaves.size(); ++i) {
            b.clear();
            if (kind == 0) h->full_block(h->leaves[i].first, h->leaves[i].second, b);
            else h->truncated_block(h->leaves[i].first, h->leaves[i].second, b);
            uint64_t taken = 0;
            for (int64_t f : b) taken |= used[f];
            if (taken == ~0ull) return FCM_EINVAL;  // more than 64 colours
            int c = 0;
            while (taken >> c & 1ull) ++c;
            colour[i] = c;
            nc = std::max(nc, c + 1);
            for (int64_t f : b) used[f] |= 1ull << c;
        }
        *n_colours = nc;
    } catch (...) {
        return FCM_ENOMEM;
    }
    return FCM_OK;
}

fcm_status fcm_mlhp_restriction(const fcm_mlhp *h, int64_t leaf, int64_t f, double *coef)
{
    if (!h || !coef || leaf < 0 || leaf >= (int64_t)h->leaves.size() || f < 0 || f >= (int64_t)h->f_level.size())
        return FCM_EINVAL;
    return h->restriction(leaf, f, coef) ? FCM_OK : FCM_EINVAL;
}

fcm_status fcm_mlhp_assemble(fcm_mlhp *h, double alpha, const fcm_bc *bc)
{
    if (!h || !bc || !(alpha > 0.0 && alpha <= 1.0) || !(bc->E > 0.0) || !(bc->nu > -1.0 && bc->nu < 0.5) ||
        bc->bc < FCM_BC_NONE || bc->bc > FCM_BC_ROLLERS)
        return FCM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(bc->traction[a])) return FCM_EINVAL;
    try {
        h->assembled = false;
        h->factorized = false;
        fcm::mlhp_device_destroy(h->dev);
        h->dev = nullptr;
        if (!h->assemble(alpha, *bc).empty()) return FCM_EINVAL;
    } catch (const std::bad_alloc &) {
        return FCM_ENOMEM;
    } catch (...) {  // e.g. std::system_error from thread creation: no exception crosses the C ABI
        return FCM_ENOMEM;
    }
    return FCM_OK;
}

fcm_status fcm_mlhp_system_size(const fcm_mlhp *h, int64_t *n_free, int64_t *nnz)
{
    if (!h || !n_free || !nnz) return FCM_EINVAL;
    if (!h->assembled) return FCM_ESTATE;
    *n_free = (int64_t)h->free_dofs.size();
    *nnz = (int64_t)h->cols.size();
    return FCM_OK;
}

fcm_status fcm_mlhp_system(const fcm_mlhp *h, int64_t *free_dofs, int64_t *rowptr, int64_t *cols, double *vals,
                           double *rhs, double *leaf_eta)
{
    if (!h) return FCM_EINVAL;
    if (!h->assembled) return FCM_ESTATE;
    if (free_dofs) std::copy(h->free_dofs.begin(), h->free_dofs.end(), free_dofs);
    if (rowptr) std::copy(h->rowptr.begin(), h->rowptr.end(), rowptr);
    if (cols) std::copy(h->cols.begin(), h->cols.end(), cols);
    if (vals) std::copy(h->vals.begin(), h->vals.end(), vals);
    if (rhs) std::copy(h->rhs.begin(), h->rhs.end(), rhs);
    if (leaf_eta) std::copy(h->leaf_eta.begin(), h->leaf_eta.end(), leaf_eta);
    return FCM_OK;
}

fcm_status fcm_mlhp_factorize(fcm_mlhp *h, int kind, double eps, double eta_bar)
{
    if (!h || (kind != 0 && kind != 1) || !(eps < 1.0) || !(eta_bar >= 0.0 && eta_bar <= 1.0)) return FCM_EINVAL;
    if (!h->assembled) return FCM_ESTATE;
    try {
        h->factorized = false;
        fcm::mlhp_device_destroy(h->dev);
        h->dev = nullptr;
        h->factorize(kind, eps, eta_bar);
    } catch (...) {
        return FCM_ENOMEM;
    }
    return FCM_OK;
}

fcm_status fcm_mlhp_factorize_device(fcm_mlhp *h, int kind, double eps, double eta_bar, void *cuda_stream)
{
    if (!h || (kind != 0 && kind != 1) || !(eps < 1.0) || !(eta_bar >= 0.0 && eta_bar <= 1.0)) return FCM_EINVAL;
    if (!h->assembled) return FCM_ESTATE;
    h->err.clear();
    try {
        h->factorized = false;
        fcm::mlhp_device_destroy(h->dev);
        h->dev = nullptr;
        const std::string e = h->factorize(kind, eps, eta_bar, true, cuda_stream);
        if (!e.empty()) {
            h->err = "fcm_mlhp_factorize_device: " + e;
            return e.find("out of memory") != std::string::npos ? FCM_ENOMEM : FCM_ECUDA;
        }
    } catch (...) {
        return FCM_ENOMEM;
    }
    return FCM_OK;
}

fcm_status fcm_mlhp_factor_info(const fcm_mlhp *h, int *n_blocks, int *n_colours, int64_t *factor_entries)
{
    if (!h || !n_blocks || !n_colours || !factor_entries) return FCM_EINVAL;
    if (!h->factorized) return FCM_ESTATE;
    *n_blocks = (int)(h->blk_ptr.size() - 1);
    *n_colours = (int)(h->colour_ptr.size() - 1);
    *factor_entries = h->fac_ptr.back();
    return FCM_OK;
}

fcm_status fcm_mlhp_factors(const fcm_mlhp *h, int64_t *blk_ptr, int64_t *blk_dofs, int64_t *fac_ptr, double *factors,
                            int64_t *colour_ptr, double *jacobi)
{
    if (!h) return FCM_EINVAL;
    if (!h->factorized) return FCM_ESTATE;
    if (blk_ptr) std::copy(h->blk_ptr.begin(), h->blk_ptr.end(), blk_ptr);
    if (blk_dofs) std::copy(h->blk_dofs.begin(), h->blk_dofs.end(), blk_dofs);
    if (fac_ptr) std::copy(h->fac_ptr.begin(), h->fac_ptr.end(), fac_ptr);
    if (factors) std::copy(h->factors.begin(), h->factors.end(), factors);
    if (colour_ptr) std::copy(h->colour_ptr.begin(), h->colour_ptr.end(), colour_ptr);
    if (jacobi) std::copy(h->jacobi.begin(), h->jacobi.end(), jacobi);
    return FCM_OK;
}

fcm_status fcm_mlhp_device_setup(fcm_mlhp *h, void *cuda_stream)
{
    if (!h) return FCM_EINVAL;
    h->err.clear();
    if (!h->factorized) {
        h->err = "fcm_mlhp_device_setup: call fcm_mlhp_factorize first";
        return FCM_ESTATE;
    }
    fcm::mlhp_device_destroy(h->dev);
    h->dev = nullptr;
    try {
        const std::string e = fcm::mlhp_device_create(
            cuda_stream, (int64_t)h->free_dofs.size(), h->rowptr.data(), h->cols.data(), h->vals.data(),
            (int64_t)h->blk_ptr.size() - 1, h->blk_ptr.data(), h->blk_dofs.data(), h->fac_ptr.data(), h->factors.data(),
            (int)h->colour_ptr.size() - 1, h->colour_ptr.data(), h->jacobi.data(),
            h->precision == FCM_PREC_MIXED ? h->fac_cond.data() : nullptr, &h->dev);
        if (!e.empty()) {
            h->err = "fcm_mlhp_device_setup: " + e;
            // CUDA failures carry the call's name in front; an allocation failure reads "out of memory"
            if (e.find("out of memory") != std::string::npos) return FCM_ENOMEM;
            return e.rfind("upload", 0) == 0 || e.rfind("cuda", 0) == 0 ? FCM_ECUDA : FCM_EINVAL;
        }
    } catch (const std::bad_alloc &) {
        h->err = "fcm_mlhp_device_setup: out of host memory";
        return FCM_ENOMEM;
    } catch (...) {
        h->err = "fcm_mlhp_device_setup: host failure";
        return FCM_ECUDA;
    }
    return FCM_OK;
}

fcm_status fcm_mlhp_apply_K(fcm_mlhp *h, const double *x_dev, double *y_dev)
{
    if (!h || !x_dev || !y_dev) return FCM_EINVAL;
    if (x_dev == y_dev) {
        h->err = "fcm_mlhp_apply_K: x_dev and y_dev must differ";
        return FCM_EINVAL;
    }
    if (!h->dev) return FCM_ESTATE;
    const std::string e = fcm::mlhp_device_apply_K(h->dev, x_dev, y_dev);
    if (!e.empty()) h->err = "fcm_mlhp_apply_K: " + e;
    return e.empty() ? FCM_OK : FCM_ECUDA;
}

fcm_status fcm_mlhp_apply_S(fcm_mlhp *h, const double *r_dev, double *z_dev)
{
    if (!h || !r_dev || !z_dev) return FCM_EINVAL;
    if (r_dev == z_dev) {
        h->err = "fcm_mlhp_apply_S: r_dev and z_dev must differ";
        return FCM_EINVAL;
    }
    if (!h->dev) return FCM_ESTATE;
    const std::string e = fcm::mlhp_device_apply_S(h->dev, r_dev, z_dev);
    if (!e.empty()) h->err = "fcm_mlhp_apply_S: " + e;
    return e.empty() ? FCM_OK : FCM_ECUDA;
}

fcm_status fcm_mlhp_pcg_solve(fcm_mlhp *h, const double *b_dev, double tol, int maxit, double *u_dev, int *iterations,
                              double *relres)
{
    if (!h || !b_dev || !u_dev || !iterations || !relres || maxit < 0 || !(tol >= 0.0)) return FCM_EINVAL;
    if (!h->dev) return FCM_ESTATE;
    int status = 0;
    const std::string e = fcm::mlhp_device_pcg(h->dev, b_dev, tol, maxit, u_dev, iterations, relres, &status);
    if (!e.empty()) {
        h->err = "fcm_mlhp_pcg_solve: " + e;
        return FCM_ECUDA;
    }
    return status == 0 ? FCM_OK : status == 1 ? FCM_ENOTCONV : FCM_EBREAKDOWN;
}

fcm_status fcm_mlhp_set_precision(fcm_mlhp *h, int precision)
{
    if (!h) return FCM_EINVAL;
    if (precision != FCM_PREC_FP64 && precision != FCM_PREC_MIXED) {
        h->err = "fcm_mlhp_set_precision: precision must be FCM_PREC_FP64 or FCM_PREC_MIXED";
        return FCM_EINVAL;
    }
    h->precision = precision;
    return FCM_OK;
}

fcm_status fcm_mlhp_device_info(const fcm_mlhp *h, int64_t *n_fp32_blocks, int64_t *factor_bytes)
{
    if (!h || !n_fp32_blocks || !factor_bytes) return FCM_EINVAL;
    if (!h->dev) return FCM_ESTATE;
    fcm::mlhp_device_info(h->dev, n_fp32_blocks, factor_bytes);
    return FCM_OK;
}

const char *fcm_mlhp_last_error(const fcm_mlhp *h) { return h ? h->err.c_str() : ""; }

void fcm_mlhp_destroy(fcm_mlhp *h) { delete h; }

}  // extern "C"
