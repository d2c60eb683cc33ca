"""Pins of the multi-level hp oracle (Sec. 2.2 overlays, Sec. 3.2 full and truncated leaf blocks).

Each test checks the oracle against something other than itself: the paper's DOF table for the
refined cube, the uniform-grid oracle in C (a different implementation) on the grid that a uniform
refinement or the finest level produces, a brute-force dimension count of the continuous leafwise-Q_p
space, the exact patch-test solution, the paper's block-overlap table and the Additive-Schwarz
lemma's consequence stated in Sec. 3.2.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import mlhp_oracle as M
from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I

BALL = [(0.5, 0.5, 0.5, 0.01)]


def _golden_dofs():
    rows = [line.split() for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_sec5_1_dofs.txt"))
            if line.strip() and not line.startswith("#")]
    return {int(k): int(v) for k, v in rows}


def test_paper_dof_table_of_the_refined_cube():
    # Sec. 5.1: 8^3 base cells, p = 3, refined toward the surface of a sphere of radius 0.01 at the cube's
    # centre, k = 0..4 levels.  The table counts the trunk space (reading 1); every level adds the same
    # 690 DOFs, which the activation rule reproduces exactly.
    table = _golden_dofs()
    for k, dofs in table.items():
        H = M.refine_toward_spheres((8, 8, 8), (0, 0, 0), (1, 1, 1), BALL, k)
        assert [len(r) for r in H.refined[:k]] == [8] * k
        assert M.count_dofs(H, 3, "trunk") == dofs


def test_uniform_refinement_is_the_uniform_grid_of_the_c_oracle():
    # Every base cell refined once: all level-0 components are covered, the level-1 overlay is the
    # uniform grid of 2N cells with no Dirichlet boundary, so K and b must equal those of the uniform-grid
    # oracle (C) on 2N cells, cut cells and alpha included, up to the DOF order.
    p, N, depth = 2, 2, 2
    g = I.random_sphere_voids(9, 3, 0.15, 0.3, octree_depth=depth)
    P = O.Problem.from_workload(I.Workload("u", (2 * N,) * 3, p, 1e-3, g, 1e-9))
    H = M.Hierarchy((N,) * 3, (0, 0, 0), (1, 1, 1), [set(itertools.product(range(N), repeat=3))])
    Q = M.MLProblem(H, p, g.sphere_array(), alpha=1e-3, depth=depth)
    assert Q.n == len(P.free_lat)
    Mx = p * 2 * N + 1
    lat = []
    for d in Q.free:
        f, comp = divmod(int(d), 3)
        l, q, m = Q.funcs[f]
        assert l == 1
        L = [p * (q[a] // 2) if q[a] % 2 == 0 else p * ((q[a] - 1) // 2) + m[a] - 1 for a in range(3)]
        lat.append(3 * (L[0] + Mx * (L[1] + Mx * L[2])) + comp)
    where = {int(v): i for i, v in enumerate(P.free_lat)}
    perm = np.array([where[v] for v in lat])
    K = P.csr()[perm][:, perm]
    assert abs(K - Q.K).max() <= 1e-13 * abs(Q.K).max()
    assert np.abs(P.rhs()[perm] - Q.b).max() <= 1e-13 * np.abs(Q.b).max()


def _fine_lattice_coefficients(B, p):
    """Coefficients of every multi-level scalar function in the finest uniform grid's lattice basis
    (the C oracle's shape functions), from values at the finest lattice points; also the largest
    disagreement between leaves that share a point (continuity)."""
    H = B.H
    Mc = H.n[0] << (H.levels - 1)
    nl = p * Mc + 1
    xs = np.arange(nl) / (p * Mc)
    E = np.zeros((nl, nl))
    h = 1.0 / Mc
    for k, x in enumerate(xs):
        i = min(int(x / h), Mc - 1)
        f, _ = O.shape1d(p, 2 * (x - i * h) / h - 1)
        E[k, p * i: p * i + p + 1] = f
    Ei = np.linalg.inv(E)
    Phi = np.full((nl, nl, nl, len(B.funcs)), np.nan)
    jump = 0.0
    for (L, c) in H.leaves:
        lo, hi = H.box(L, c)
        idx = [np.flatnonzero((xs >= lo[a] - 1e-12) & (xs <= hi[a] + 1e-12)) for a in range(3)]
        ijk = [(i, j, k) for k in idx[2] for j in idx[1] for i in idx[0]]
        pts = np.array([(xs[i], xs[j], xs[k]) for (i, j, k) in ijk])
        fids = B.leaf_functions(L, c)
        val, _ = B.eval_on_leaf(L, c, fids, 2 * (pts - lo) / (hi - lo) - 1)
        row = np.zeros((len(pts), len(B.funcs)))
        row[:, fids] = val.T
        for r, (i, j, k) in enumerate(ijk):
            if not np.isnan(Phi[k, j, i, 0]):
                jump = max(jump, np.abs(Phi[k, j, i] - row[r]).max())
            Phi[k, j, i] = row[r]
    T = np.einsum("zc,yb,xa,cbaf->zyxf", Ei, Ei, Ei, Phi).reshape(nl ** 3, -1)
    T[np.abs(T) < 1e-14] = 0.0
    return T, jump, Mc


def test_overlay_stiffness_is_the_finest_grid_stiffness_on_the_subspace():
    # Three levels (a corner cell refined, then its child at the domain centre), uncut: every multi-level
    # function is continuous and piecewise Q_p on the finest grid, so it has coefficients T in that grid's
    # basis, and the multi-level stiffness must be T^T K_fine T with K_fine from the C oracle.
    p = 2
    H = M.Hierarchy((2, 2, 2), (0, 0, 0), (1, 1, 1), [{(0, 0, 0)}, {(1, 1, 1)}])
    Q = M.MLProblem(H, p, (), alpha=1.0, depth=0)
    T, jump, Mc = _fine_lattice_coefficients(Q.basis, p)
    assert jump == 0.0
    assert np.linalg.matrix_rank(T) == len(Q.funcs)          # linearly independent
    P = O.Problem.from_workload(I.Workload("fine", (Mc,) * 3, p, 1.0, I.uncut(), 1e-9))
    where = {int(v): i for i, v in enumerate(P.free_lat)}
    rows, cols, vals = [], [], []
    for j, d in enumerate(Q.free):
        f, comp = divmod(int(d), 3)
        for s in np.flatnonzero(T[:, f]):
            assert 3 * s + comp in where                        # no clamped fine DOF is used
            rows.append(where[3 * s + comp])
            cols.append(j)
            vals.append(T[s, f])
    T3 = sp.csr_matrix((vals, (rows, cols)), shape=(len(P.free_lat), Q.n))
    Kc = T3.T @ P.csr() @ T3
    assert abs(Kc - Q.K).max() <= 1e-13 * abs(Q.K).max()
    assert np.abs(T3.T @ P.rhs() - Q.b).max() <= 1e-13 * np.abs(Q.b).max()


def _dim_continuous_leafwise_qp(H, p):
    """Brute force: functions that are Q_p on every leaf and continuous, parametrised by their values at
    the union U of the leaves' own equispaced nodes, constrained by Q_p interpolation inside each leaf."""
    F = H.levels - 1
    own, U = {}, set()
    for (L, c) in H.leaves:
        s = 1 << (F - L)
        own[(L, c)] = [tuple((c[a] * p + i[a]) * s for a in range(3)) for i in itertools.product(range(p + 1), repeat=3)]
        U.update(own[(L, c)])
    U = sorted(U)
    pos = {u: i for i, u in enumerate(U)}
    Ua = np.array(U)
    tn = np.arange(p + 1, dtype=float)
    rows = []
    for (L, c) in H.leaves:
        s = 1 << (F - L)
        lo = np.array(c) * p * s
        mine = set(own[(L, c)])
        for i in np.flatnonzero(np.all((Ua >= lo) & (Ua <= lo + p * s), axis=1)):
            if U[i] in mine:
                continue
            t = (np.array(U[i]) - lo) / s
            lag = [np.array([np.prod([(t[a] - tn[m]) / (tn[k] - tn[m]) for m in range(p + 1) if m != k])
                             for k in range(p + 1)]) for a in range(3)]
            row = np.zeros(len(U))
            row[i] = 1.0
            for idx in itertools.product(range(p + 1), repeat=3):
                row[pos[tuple(lo[a] + idx[a] * s for a in range(3))]] -= lag[0][idx[0]] * lag[1][idx[1]] * lag[2][idx[2]]
            rows.append(row)
    return len(U) - (np.linalg.matrix_rank(np.array(rows)) if rows else 0)


@pytest.mark.parametrize("p,refined", [
    (2, [{(0, 0, 0)}, {(1, 1, 1)}]),
    (3, [{(0, 0, 0), (1, 0, 0)}, {(1, 1, 1)}, {(2, 2, 2)}]),
    (2, [{(0, 0, 0), (1, 1, 1)}]),                 # refined cells meeting at one vertex only
    (1, [{(0, 0, 0)}, {(0, 0, 0)}]),               # refinement into a domain corner, two levels
])
def test_basis_spans_exactly_the_continuous_leafwise_qp_space(p, refined):
    # Sec. 2.2: the overlay Dirichlet boundaries enforce continuity and the deactivation keeps the sum
    # linearly independent.  Too many active components would make the basis dependent, too few would
    # lose part of the space: the count must equal the brute-force dimension.
    H = M.Hierarchy((2, 2, 2), (0, 0, 0), (1, 1, 1), refined)
    assert len(M.Basis(H, p).funcs) == _dim_continuous_leafwise_qp(H, p)


def test_patch_test_on_three_levels_is_exact():
    # Uniaxial stress (traction -1 on z = 1, rollers on x = 0, y = 0, z = 0): the exact solution
    # u = (nu x, nu y, -z) / E lies in the space, so the Galerkin solution reproduces it at any point.
    H = M.Hierarchy((2, 2, 2), (0, 0, 0), (1, 1, 1), [{(0, 0, 0)}, {(1, 1, 1)}, {(2, 2, 2)}])
    Q = M.MLProblem(H, 2, (), alpha=1.0, depth=0, bc="roller")
    assert abs(Q.K - Q.K.T).max() <= 1e-15 * abs(Q.K).max()
    x = spla.spsolve(Q.K.tocsc(), Q.b)
    pts = np.random.default_rng(0).random((20, 3))
    pts[:8] *= 0.3                                             # inside the refined corner
    u = Q.displacement(x, pts)
    exact = np.column_stack([0.3 * pts[:, 0], 0.3 * pts[:, 1], -pts[:, 2]])
    assert np.abs(u - exact).max() < 1e-12


def test_truncated_blocks_keep_the_overlap_at_eight_full_blocks_do_not():
    # Sec. 3.2 / Sec. 5.3 table of n_max: truncated blocks keep every function in at most 2^d = 8 blocks
    # at every refinement depth; full blocks (all functions supported on the leaf) take the coarse linear
    # functions into more and more blocks as k grows.
    full = []
    for k in range(4):
        H = M.refine_toward_spheres((8, 8, 8), (0, 0, 0), (1, 1, 1), BALL, k)
        B = M.Basis(H, 3)
        assert B.overlap("truncated") == 8
        full.append(B.overlap("full"))
    assert full[0] == 8 and all(b > a for a, b in zip(full, full[1:]))


def test_overlap_is_a_lower_bound_of_the_largest_eigenvalue():
    # Sec. 3.2: a function in n blocks has e_k^T S^-1 e_k <= A_kk / n (the Additive-Schwarz lemma of
    # Sec. 3.1 with v_B = e_k / n), so lambda_max(S A) >= n.  Uncut (alpha = 1, every block nonsingular),
    # two levels toward a sphere.
    H = M.refine_toward_spheres((2, 2, 2), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.2)], 2)
    Q = M.MLProblem(H, 2, (), alpha=1.0, depth=0)
    A = Q.K.toarray()
    lam = {}
    for kind in ("full", "truncated"):
        Q.build_blocks(kind)
        S = np.diag(Q.jacobi)
        for B, F in zip(Q.blocks, Q.factors):
            S[np.ix_(B, B)] += F
        lam[kind] = np.linalg.eigvals(S @ A).real.max()
        assert lam[kind] >= Q.membership().max()
    assert Q.membership().max() == 8
    assert lam["full"] > 2 * lam["truncated"]


def test_span_reading_fills_every_block_but_breaks_the_overlap_bound():
    # The alternative reading of 3D truncation (complete each block to the leaf's (p+1)^3 local space from
    # coarser levels) gives every leaf a full-size block but takes coarse functions into more than 2^d
    # blocks, against the paper's n_max table: the corner reading is the one that keeps n_max = 8.
    H = M.refine_toward_spheres((4, 4, 4), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.1)], 1)
    B = M.Basis(H, 2)
    assert all(len(B.span_functions(*lc)) == 27 for lc in H.leaves)
    assert B.overlap("span") > 8 == B.overlap("truncated")
    assert any(len(B.truncated_functions(*lc)) < 27 for lc in H.leaves)


def test_truncated_blocks_converge_faster_than_full_blocks_under_refinement():
    # Sec. 5.1: the cube with a small spherical cavity at its centre, refined toward the cavity's surface.
    # With full blocks the iteration count grows with the depth k much faster than with truncated blocks.
    # The paper's set-up scaled to a 4^3 base grid (r / h = 0.08 as for r = 0.01 on 8^3), p = 2,
    # alpha = 1e-8, k = 0..3.
    its = {}
    ball = [(0.5, 0.5, 0.5, 0.02)]
    for k in range(4):
        H = M.refine_toward_spheres((4, 4, 4), (0, 0, 0), (1, 1, 1), ball, k)
        Q = M.MLProblem(H, 2, ball, alpha=1e-8, depth=3)
        for kind in ("full", "truncated"):
            Q.build_blocks(kind)
            its[kind, k] = Q.pcg(tol=1e-8, maxit=3000)[1]
    assert its["full", 0] == its["truncated", 0]               # no overlay: the blocks coincide
    for k in (1, 2, 3):
        assert its["truncated", k] < its["full", k]
    assert its["full", 3] > 2.5 * its["full", 0]
    assert its["truncated", 3] < 1.6 * its["truncated", 0]
