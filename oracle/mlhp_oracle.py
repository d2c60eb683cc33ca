"""Multi-level hp finite cell discretisation and its Additive-Schwarz blocks: plain FP64 numpy.

TEST INFRASTRUCTURE ONLY: imported by the tests.  The product path never loads it.

What it computes, following the paper:
- Sec. 2.2 (multi-level hp): a base grid of cells is refined by superposing overlay grids.  Level l + 1
  holds the 8 children of every refined level-l cell.  Each level carries its own integrated-Legendre
  basis (Sec. 2.1 shape functions, one per topological component: vertex, edge, face, cell).
  Homogeneous Dirichlet conditions on the boundary of each overlay, and the deactivation of components
  that a finer overlay covers, make the sum continuous and linearly independent.
- Sec. 2.1 / Eq. (1): the stiffness is integrated on leaf cells (cells with no overlay) with the octree
  rule and the fictitious stiffness alpha in the void.
- Sec. 3.2 "Selecting suitable blocks": one Additive-Schwarz block per leaf cell.  The full block holds
  every basis function supported on the leaf.  The truncated block holds the leaf's own-level functions
  plus, for each leaf corner without an own-level vertex function, the vertex function found by
  traversing down the element hierarchy.
- Sec. 3.1 Eq. (5) with the pseudo inverse of Sec. 3.2 (cut-off eps relative to the largest eigenvalue),
  the Jacobi fill of Algorithm 1 for functions in no block, and PCG with the Eq. (14) stopping test.

Readings where the paper is silent (each is binding for any implementation compared with this one):
- Activation.  A level-l component is active iff every in-domain cell position around it exists at
  level l and at least one of them is a leaf.  The first condition is the overlay's homogeneous
  Dirichlet boundary; it applies only where the overlay borders unrefined cells, not on the domain
  boundary.  The second deactivates components that finer overlays cover.  In 1D this keeps, on a leaf
  at the domain end, both vertex functions on the finest level, as the paper's Fig. 4 discussion says.
- Refinement toward a surface: a level-l cell is refined (l < k) when the domain boundary crosses its
  closed box, the octree's cut test (Shape.cut: sphere surfaces, voxel interfaces or a plane).
- Truncation in 3D: the paper states the 1D rule (p - 1 higher-order functions of the leaf and two
  linear functions, the missing one found by traversing down the hierarchy) and says 3D follows by
  the tensor product.  Read here: every non-vertex function comes from the leaf's own level; only
  vertex (trilinear) functions are looked up on coarser levels, at the leaf corner's point.
- Discarded functions: a function is kept iff some leaf in its support has eta > 0 (as cells with
  eta = 0 are dropped on the uniform grid).
"""
from __future__ import annotations

import itertools

import numpy as np
import numpy.polynomial.legendre as npleg
import scipy.sparse as sp

__all__ = ["Shape", "Hierarchy", "refine_toward_spheres", "Basis", "MLProblem", "count_dofs", "shape1d"]


# ----------------------------------------------------------------------------- 1D basis (Sec. 2.1)
def shape1d(p, xi):
    """Integrated-Legendre shape functions on [-1, 1] and their derivatives, for an array xi.

    Row 0: N0 = (1 - xi)/2 (left vertex), row 1: N1 = (1 + xi)/2 (right vertex), row j >= 2:
    phi_j = (P_j - P_{j-2}) / sqrt(2 (2j - 1)), whose derivative is sqrt((2j - 1)/2) P_{j-1}.
    """
    xi = np.asarray(xi, dtype=np.float64)
    P = [np.ones_like(xi), xi.copy()]
    for k in range(1, p):
        P.append(((2 * k + 1) * xi * P[k] - k * P[k - 1]) / (k + 1))
    f = np.zeros((p + 1,) + xi.shape)
    d = np.zeros((p + 1,) + xi.shape)
    f[0], d[0] = 0.5 * (1.0 - xi), -0.5
    f[1], d[1] = 0.5 * (1.0 + xi), 0.5
    for j in range(2, p + 1):
        f[j] = (P[j] - P[j - 2]) / np.sqrt(2.0 * (2 * j - 1))
        d[j] = np.sqrt((2 * j - 1) / 2.0) * P[j - 1]
    return f, d


# ----------------------------------------------------------------------------- geometry
class Shape:
    """The physical domain, as for the uniform grid: the box minus sphere voids (kind 0), the solid voxels of
    an image spanning the box (kind 1, array [z][y][x]), or the half space a.x < d (kind 2).

    void(x): the fictitious domain at points x (m, 3).  cut(lo, hi): the boundary crosses the closed box:
    spheres, min distance < r < max distance from the centre; voxels, the voxels the box overlaps are not all
    equal; half space, min a.x < d < max a.x over the box."""

    def __init__(self, kind=0, spheres=(), voxels=None, plane=(0.0, 0.0, 1.0, 2.0), lo=(0, 0, 0), hi=(1, 1, 1)):
        self.kind = int(kind)
        self.spheres = [tuple(float(v) for v in s) for s in spheres]
        self.voxels = None if voxels is None else np.asarray(voxels, dtype=np.uint8)
        self.plane = tuple(float(v) for v in plane)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)

    @classmethod
    def of(cls, geometry, lo=(0, 0, 0), hi=(1, 1, 1)):
        """From a sphere list (cx, cy, cz, r) or an object with kind, spheres, voxels, plane."""
        if isinstance(geometry, Shape):
            return geometry
        if hasattr(geometry, "kind"):
            sph = geometry.spheres if geometry.spheres is not None else ()
            return cls(geometry.kind, sph, geometry.voxels, geometry.plane, lo, hi)
        return cls(0, geometry, lo=lo, hi=hi)

    def _vox_index(self, x):
        dims = np.array(self.voxels.shape[::-1])
        t = (x - self.lo) / (self.hi - self.lo) * dims
        return np.clip(np.floor(t).astype(np.int64), 0, dims - 1)

    def void(self, x):
        x = np.atleast_2d(x)
        if self.kind == 0:
            out = np.zeros(len(x), dtype=bool)
            for c0, c1, c2, r in self.spheres:
                out |= (x[:, 0] - c0) ** 2 + (x[:, 1] - c1) ** 2 + (x[:, 2] - c2) ** 2 < r * r
            return out
        if self.kind == 1:
            i = self._vox_index(x)
            return self.voxels[i[:, 2], i[:, 1], i[:, 0]] == 0
        a = np.array(self.plane[:3])
        return ~(x @ a < self.plane[3])

    def cut(self, lo, hi):
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        if self.kind == 0:
            for c0, c1, c2, r in self.spheres:
                c = np.array([c0, c1, c2])
                near = np.clip(c, lo, hi)
                far = np.where(np.abs(c - lo) > np.abs(c - hi), lo, hi)
                if np.linalg.norm(c - near) < r < np.linalg.norm(c - far):
                    return True
            return False
        if self.kind == 1:
            dims = np.array(self.voxels.shape[::-1])
            h = (self.hi - self.lo) / dims
            i0 = np.floor((lo - self.lo) / h).astype(np.int64)
            i1 = np.ceil((hi - self.lo) / h).astype(np.int64) - 1
            i1 = np.maximum(i1, i0)
            i0 = np.clip(i0, 0, dims - 1)
            i1 = np.clip(i1, 0, dims - 1)
            sub = self.voxels[i0[2]:i1[2] + 1, i0[1]:i1[1] + 1, i0[0]:i1[0] + 1] != 0
            return bool(sub.any() and not sub.all())
        a = np.array(self.plane[:3])
        mn = np.sum(np.minimum(a * lo, a * hi))
        mx = np.sum(np.maximum(a * lo, a * hi))
        return bool(mn < self.plane[3] < mx)


def _void(shape, x):
    return shape.void(x)


def _box_cut(shape, lo, hi):
    return shape.cut(lo, hi)


# ----------------------------------------------------------------------------- the hierarchy
class Hierarchy:
    """Base grid of n cells on [lo, hi] and the refined cells of each level (Sec. 2.2).

    Cells of level l are integer triples on the grid of n * 2^l cells.  `refined[l]` is the set of
    level-l cells that carry an overlay (their 8 children form part of level l + 1).
    """

    def __init__(self, n, lo, hi, refined):
        self.n = tuple(int(v) for v in n)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        base = set(itertools.product(*[range(v) for v in self.n]))
        self.cells = [base]
        self.refined = []
        for l, R in enumerate(refined):
            R = set(tuple(int(v) for v in c) for c in R)
            assert R <= self.cells[l], "only existing cells can be refined"
            self.refined.append(R)
            if not R:
                break
            self.cells.append({(2 * a + i, 2 * b + j, 2 * c + k) for (a, b, c) in R
                               for i in (0, 1) for j in (0, 1) for k in (0, 1)})
        while len(self.refined) < len(self.cells):
            self.refined.append(set())
        self.levels = len(self.cells)
        self.leaves = [(l, c) for l in range(self.levels) for c in sorted(self.cells[l] - self.refined[l])]

    def extent(self, l):
        return tuple(v << l for v in self.n)

    def h(self, l):
        return (self.hi - self.lo) / np.array(self.extent(l), dtype=np.float64)

    def box(self, l, c):
        h = self.h(l)
        lo = self.lo + np.array(c) * h
        return lo, lo + h

    def around(self, l, q):
        """In-domain level-l cell positions whose closure holds component q (doubled coordinates)."""
        ext = self.extent(l)
        axes = []
        for a in range(3):
            if q[a] % 2:
                axes.append([(q[a] - 1) // 2])
            else:
                axes.append([i for i in (q[a] // 2 - 1, q[a] // 2) if 0 <= i < ext[a]])
        return list(itertools.product(*axes))

    def active(self, l, q):
        """Activation reading: every in-domain position around q exists at level l (q is not on the
        overlay's Dirichlet boundary) and at least one of them is a leaf (no finer overlay covers q)."""
        pos = self.around(l, q)
        return all(c in self.cells[l] for c in pos) and any(c not in self.refined[l] for c in pos)


def refine_toward_spheres(n, lo, hi, spheres, k):
    """Hierarchy refined k times toward the boundary of the domain (cells the boundary crosses); `spheres` is
    a sphere list or a geometry (see Shape.of)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    spheres = Shape.of(spheres, lo, hi)
    refined = []
    cells = set(itertools.product(*[range(v) for v in n]))
    for l in range(k):
        h = (hi - lo) / (np.array(n) * 2 ** l)
        R = {c for c in cells if _box_cut(spheres, lo + np.array(c) * h, lo + (np.array(c) + 1) * h)}
        refined.append(R)
        cells = {(2 * a + i, 2 * b + j, 2 * c + kk) for (a, b, c) in R
                 for i in (0, 1) for j in (0, 1) for kk in (0, 1)}
    return Hierarchy(n, lo, hi, refined)


def _closure(c):
    return [(2 * c[0] + i, 2 * c[1] + j, 2 * c[2] + k) for k in range(3) for j in range(3) for i in range(3)]


def _modes(q, p, space):
    """Mode indices of component q: per axis 0 where q is a vertex coordinate (the linear factor),
    j = 2..p where q spans the cell interval (the bubble phi_j).  'full': the tensor product;
    'trunk': the trunk space, where the bubble indices of a face or cell sum to at most p."""
    odd = [a for a in range(3) if q[a] % 2]
    out = []
    for js in itertools.product(range(2, p + 1), repeat=len(odd)):
        if space == "trunk" and len(odd) >= 2 and sum(js) > p:
            continue
        m = [0, 0, 0]
        for a, j in zip(odd, js):
            m[a] = j
        out.append(tuple(m))
    return out


def count_dofs(H, p, space="full", components=3):
    """Number of basis functions of the hierarchy, before any are discarded or constrained."""
    total = 0
    for l in range(H.levels):
        comps = set()
        for c in H.cells[l]:
            comps.update(_closure(c))
        total += sum(len(_modes(q, p, space)) for q in comps if H.active(l, q))
    return components * total


# ----------------------------------------------------------------------------- the problem
class Basis:
    """The active scalar basis functions of a hierarchy: (level, component, mode), level by level in
    lattice order, and the functions each leaf supports (Sec. 2.2, Sec. 3.2)."""

    def __init__(self, H, p):
        self.H, self.p = H, int(p)
        self.funcs, self.index = [], {}
        for l in range(H.levels):
            comps = set()
            for c in H.cells[l]:
                comps.update(_closure(c))
            for q in sorted(comps, key=lambda t: (t[2], t[1], t[0])):
                if H.active(l, q):
                    for m in _modes(q, self.p, "full"):
                        self.index[(l, q, m)] = len(self.funcs)
                        self.funcs.append((l, q, m))

    def leaf_functions(self, L, c):
        """Indices of the active scalar functions supported on leaf (L, c): on each level l <= L the
        components in the closure of the leaf's level-l ancestor (the full block's functions)."""
        out = []
        for l in range(L + 1):
            A = tuple(v >> (L - l) for v in c)
            for q in _closure(A):
                if self.H.active(l, q):
                    out.extend(self.index[(l, q, m)] for m in _modes(q, self.p, "full"))
        return out

    def truncated_functions(self, L, c):
        """Truncated block of a leaf (reading above): own-level functions, then for each corner whose
        own-level vertex function is inactive, the vertex function of the highest coarser level at
        which the corner point is a vertex of the leaf's ancestor and is active."""
        out = []
        for q in _closure(c):
            if self.H.active(L, q):
                out.extend(self.index[(L, q, m)] for m in _modes(q, self.p, "full"))
        for corner in itertools.product((0, 2), repeat=3):
            q = tuple(2 * c[a] + corner[a] for a in range(3))
            if self.H.active(L, q):
                continue
            for l in range(L - 1, -1, -1):
                s = 1 << (L - l)
                if any(q[a] % (2 * s) for a in range(3)):  # the point is not a vertex of level l
                    break
                ql = tuple(v // s for v in q)
                if self.H.active(l, ql):
                    out.append(self.index[(l, ql, (0, 0, 0))])
                    break
        return out

    def span_functions(self, L, c):
        """The alternative reading of 3D truncation, kept for comparison: the leaf's own-level functions,
        then coarser levels in order, each function kept when its restriction to the leaf is linearly
        independent of those kept (rank test at (p+1)^3 Gauss points), until the block spans the
        leaf's (p+1)^3-dimensional local space."""
        g = npleg.leggauss(self.p + 1)[0]
        t = np.array(list(itertools.product(g, g, g)))
        out, rows = [], np.zeros((0, len(t)))
        for l in range(L, -1, -1):
            A = tuple(v >> (L - l) for v in c)
            lev = [self.index[(l, q, m)] for q in _closure(A) if self.H.active(l, q)
                   for m in _modes(q, self.p, "full")]
            val, _ = self.eval_on_leaf(L, c, lev, t)
            for r, f in enumerate(lev):
                if len(out) == len(t):
                    return out
                cand = np.vstack([rows, val[r]])
                if np.linalg.matrix_rank(cand, tol=1e-9) > len(rows):
                    rows = cand
                    out.append(f)
        return out

    def block_functions(self, kind, L, c):
        if kind == "full":
            return self.leaf_functions(L, c)
        if kind == "truncated":
            return self.truncated_functions(L, c)
        assert kind == "span"
        return self.span_functions(L, c)

    def overlap(self, kind, leaves=None):
        """Largest number of blocks (one per leaf) that one scalar function belongs to: n_max."""
        cnt = np.zeros(len(self.funcs), dtype=np.int64)
        for lc in (self.H.leaves if leaves is None else leaves):
            cnt[np.unique(np.array(self.block_functions(kind, *lc), dtype=np.int64))] += 1
        return int(cnt.max())

    def eval_on_leaf(self, L, c, fids, t):
        """Values (nf, m) and physical gradients (nf, m, 3) of functions `fids` at leaf-local points t:
        a level-l function is evaluated through the leaf's level-l ancestor, whose local coordinate is
        xi = -1 + (2 offset + 1 + t) / 2^(L - l) along each axis."""
        nf, m = len(fids), len(t)
        val = np.ones((nf, m))
        grad = np.ones((nf, m, 3))
        for r, f in enumerate(fids):
            l, q, mode = self.funcs[f]
            s = 1 << (L - l)
            A = [v >> (L - l) for v in c]
            h = self.H.h(l)
            for a in range(3):
                off = c[a] - A[a] * s
                xi = -1.0 + (2 * off + 1 + t[:, a]) / s
                F, D = shape1d(self.p, xi)
                if q[a] % 2:
                    fa, da = F[mode[a]], D[mode[a]]
                elif q[a] // 2 == A[a]:
                    fa, da = F[0], D[0]
                else:
                    assert q[a] // 2 == A[a] + 1
                    fa, da = F[1], D[1]
                da = da * 2.0 / h[a]
                val[r] *= fa
                for b in range(3):
                    grad[r, :, b] *= da if b == a else fa
        return val, grad


class MLProblem:
    """Linear elasticity on a multi-level hp hierarchy with cut cells (Eq. (1), alpha in the void).

    bc 'clamp': all components fixed on z = lo_z (strong, functions whose component lies on the plane
    are removed), traction on z = hi_z.  bc 'roller': component a fixed on x_a = lo_a, traction on
    z = hi_z (the patch test's set-up).
    """

    def __init__(self, H, p, spheres=(), alpha=1e-8, depth=2, E=1.0, nu=0.3, traction=(0.0, 0.0, -1.0),
                 bc="clamp"):
        """spheres: the voids (cx, cy, cz, r), or any geometry Shape.of accepts."""
        self.H, self.p, self.depth = H, int(p), int(depth)
        self.spheres = Shape.of(spheres, H.lo, H.hi)
        self.alpha = float(alpha)
        self.lam = E * nu / ((1 + nu) * (1 - nu * 2))
        self.mu = E / (2 * (1 + nu))
        self.traction = np.asarray(traction, dtype=np.float64)
        self.basis = Basis(H, p)
        self.funcs = self.basis.funcs
        self.leaf_functions = self.basis.leaf_functions
        self.eval_on_leaf = self.basis.eval_on_leaf
        # quadrature and eta per leaf (octree of `depth` levels relative to the leaf)
        self.quad = {}
        self.eta = {}
        for (l, c) in H.leaves:
            t, w, a, eta = self._leaf_rule(l, c)
            self.quad[(l, c)] = (t, w, a)
            self.eta[(l, c)] = eta
        self.active_leaves = [lc for lc in H.leaves if self.eta[lc] > 0.0]
        kept = set()
        for lc in self.active_leaves:
            kept.update(self.leaf_functions(*lc))
        # displacement DOFs: 3 per kept scalar function, minus the Dirichlet ones
        fixed = set()
        for f in kept:
            q = self.funcs[f][1]
            for comp in range(3):
                if (bc == "clamp" and q[2] == 0) or (bc == "roller" and q[comp] == 0):
                    fixed.add(3 * f + comp)
        self.free = np.array(sorted(3 * f + comp for f in kept for comp in range(3) if 3 * f + comp not in fixed),
                             dtype=np.int64)
        self.pos = -np.ones(3 * len(self.funcs), dtype=np.int64)
        self.pos[self.free] = np.arange(len(self.free))
        self.n = len(self.free)
        self.K = self._assemble()
        self.b = self._traction_rhs()
        self.blocks = None

    # -- quadrature (octree, Sec. 5.1 "relative to the local element size") -----------------------
    def _leaf_rule(self, l, c):
        lo, hi = self.H.box(l, c)
        g, gw = npleg.leggauss(self.p + 1)
        pts, wts = [], []

        def rec(blo, bhi, d):  # blo, bhi in leaf-local coordinates [-1, 1]^3
            plo = lo + (blo + 1) * 0.5 * (hi - lo)
            phi = lo + (bhi + 1) * 0.5 * (hi - lo)
            if d < self.depth and _box_cut(self.spheres, plo, phi):
                mid = 0.5 * (blo + bhi)
                for o in itertools.product((0, 1), repeat=3):
                    o = np.array(o)
                    rec(np.where(o, mid, blo), np.where(o, bhi, mid), d + 1)
                return
            half = 0.5 * (bhi - blo)
            for i, j, k in itertools.product(range(self.p + 1), repeat=3):
                pts.append(0.5 * (blo + bhi) + half * np.array([g[i], g[j], g[k]]))
                wts.append(gw[i] * gw[j] * gw[k] * np.prod(half))

        rec(-np.ones(3), np.ones(3), 0)
        t = np.array(pts)
        jac = np.prod(0.5 * (hi - lo))
        w = np.array(wts) * jac
        x = lo + (t + 1) * 0.5 * (hi - lo)
        void = _void(self.spheres, x)
        a = np.where(void, self.alpha, 1.0)
        eta = float(np.sum(w[~void]) / np.prod(hi - lo))
        return t, w, a, eta

    # -- Eq. (1): stiffness and traction --------------------------------------------------------------
    def leaf_matrix(self, L, c):
        fids = self.leaf_functions(L, c)
        t, w, a = self.quad[(L, c)]
        _, G = self.eval_on_leaf(L, c, fids, t)
        wa = w * a
        M = np.einsum("q,fqa,gqb->abfg", wa, G, G)  # M[a, b] = sum_q w alpha d_a s_f d_b s_g
        nf = len(fids)
        Ke = np.zeros((nf, 3, nf, 3))
        tr = M[0, 0] + M[1, 1] + M[2, 2]
        for i in range(3):
            for k in range(3):
                blk = self.lam * M[i, k] + self.mu * M[k, i]
                if i == k:
                    blk = blk + self.mu * tr
                Ke[:, i, :, k] = blk
        dofs = (3 * np.array(fids)[:, None] + np.arange(3)[None, :]).reshape(-1)
        return dofs, Ke.reshape(3 * nf, 3 * nf)

    def _assemble(self):
        rows, cols, vals = [], [], []
        for (L, c) in self.active_leaves:
            dofs, Ke = self.leaf_matrix(L, c)
            loc = self.pos[dofs]
            keep = loc >= 0
            ii, jj = np.meshgrid(loc[keep], loc[keep], indexing="ij")
            rows.append(ii.ravel())
            cols.append(jj.ravel())
            vals.append(Ke[np.ix_(keep, keep)].ravel())
        K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n)).tocsr()
        K.sum_duplicates()
        return K

    def _traction_rhs(self):
        """Traction on the top face intersected with the physical domain: quadtree of `depth` levels
        on each leaf's top face, (p+1)^2 Gauss points per square, solid points only."""
        b = np.zeros(self.n)
        g, gw = npleg.leggauss(self.p + 1)
        for (L, c) in self.active_leaves:
            if c[2] != self.H.extent(L)[2] - 1:
                continue
            lo, hi = self.H.box(L, c)
            pts, wts = [], []

            def rec(blo, bhi, d):  # face-local coordinates [-1, 1]^2
                plo = np.append(lo[:2] + (blo + 1) * 0.5 * (hi[:2] - lo[:2]), hi[2])
                phi = np.append(lo[:2] + (bhi + 1) * 0.5 * (hi[:2] - lo[:2]), hi[2])
                if d < self.depth and _box_cut(self.spheres, plo, phi):
                    mid = 0.5 * (blo + bhi)
                    for o in itertools.product((0, 1), repeat=2):
                        o = np.array(o)
                        rec(np.where(o, mid, blo), np.where(o, bhi, mid), d + 1)
                    return
                half = 0.5 * (bhi - blo)
                for i, j in itertools.product(range(self.p + 1), repeat=2):
                    pts.append(0.5 * (blo + bhi) + half * np.array([g[i], g[j]]))
                    wts.append(gw[i] * gw[j] * np.prod(half))

            rec(-np.ones(2), np.ones(2), 0)
            t2 = np.array(pts)
            w = np.array(wts) * 0.25 * (hi[0] - lo[0]) * (hi[1] - lo[1])
            t = np.column_stack([t2, np.ones(len(t2))])
            x = lo + (t + 1) * 0.5 * (hi - lo)
            w = np.where(_void(self.spheres, x), 0.0, w)
            fids = self.leaf_functions(L, c)
            val, _ = self.eval_on_leaf(L, c, fids, t)
            for r, f in enumerate(fids):
                for comp in range(3):
                    k = self.pos[3 * f + comp]
                    if k >= 0:
                        b[k] += self.traction[comp] * np.dot(w, val[r])
        return b

    # -- Sec. 3.2: blocks on leaves --------------------------------------------------------------------
    def build_blocks(self, kind="truncated", eps=1e-13, eta_bar=1.0):
        """Blocks (free DOF index arrays, one per leaf with 0 < eta_T <= eta_bar, Sec. 3.2 "Optimizing the
        number of blocks", eta_T clamped to 1) and their pseudo inverses; the diagonal part of Algorithm 1
        (1 / K_ll) for free DOFs in no block.  kind: 'full', 'truncated' or 'span'."""
        blocks = []
        for (L, c) in self.active_leaves:
            if min(self.eta[(L, c)], 1.0) > eta_bar:
                continue
            fids = self.basis.block_functions(kind, L, c)
            dofs = (3 * np.array(sorted(set(fids)))[:, None] + np.arange(3)[None, :]).reshape(-1)
            loc = self.pos[dofs]
            loc = np.sort(loc[loc >= 0])
            if len(loc):
                blocks.append(loc)
        factors = [_pseudo_inverse(self.K[B][:, B].toarray(), eps) for B in blocks]
        covered = np.zeros(self.n, dtype=bool)
        for B in blocks:
            covered[B] = True
        self.jacobi = np.where(covered, 0.0, 1.0 / np.where(covered, 1.0, self.K.diagonal()))
        self.blocks, self.factors = blocks, factors
        return blocks

    def membership(self):
        """Number of blocks each free DOF belongs to."""
        cnt = np.zeros(self.n, dtype=np.int64)
        for B in self.blocks:
            cnt[B] += 1
        return cnt

    def apply_S(self, r):
        """Sec. 3.1 Eq. (5): z = sum_B R_B^T A_B^+ R_B r, plus the diagonal part."""
        z = self.jacobi * r
        for B, F in zip(self.blocks, self.factors):
            z[B] += F @ r[B]
        return z

    def pcg(self, tol=1e-8, maxit=10000, b=None):
        """PCG from x = 0, stopped when ||S r|| / ||S b|| <= tol (Eq. (14))."""
        b = self.b if b is None else b
        x = np.zeros(self.n)
        r = b.copy()
        z = self.apply_S(r)
        ref = np.linalg.norm(self.apply_S(b))
        p = z.copy()
        rz = r @ z
        for it in range(1, maxit + 1):
            q = self.K @ p
            a = rz / (p @ q)
            x += a * p
            r -= a * q
            z = self.apply_S(r)
            if np.linalg.norm(z) <= tol * ref:
                return x, it
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, maxit

    def energy_error(self, xref, x):
        d = xref - x
        return float(np.sqrt(abs(d @ (self.K @ d)) / (xref @ (self.K @ xref))))

    def displacement(self, x, pts):
        """u at physical points `pts` (m, 3) from the free-DOF vector x."""
        full = np.zeros(3 * len(self.funcs))
        full[self.free] = x
        out = np.zeros((len(pts), 3))
        H = self.H
        for i, X in enumerate(pts):
            for (L, c) in H.leaves:
                lo, hi = H.box(L, c)
                if np.all(X >= lo) and np.all(X <= hi):
                    t = (2 * (X - lo) / (hi - lo) - 1)[None, :]
                    fids = self.leaf_functions(L, c)
                    val, _ = self.eval_on_leaf(L, c, fids, t)
                    for r, f in enumerate(fids):
                        out[i] += val[r, 0] * full[3 * f:3 * f + 3]
                    break
        return out


def _pseudo_inverse(A, eps):
    """Sec. 3.2: A^+ = V diag(1/lambda, lambda > eps * lambda_max) V^T (numpy's symmetric eigensolver)."""
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    keep = lam > eps * lam.max()
    return (V[:, keep] / lam[keep]) @ V[:, keep].T
