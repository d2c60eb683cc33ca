"""The library's multi-level hp plan (host side of Sec. 2.2 / Sec. 3.2) against the multi-level oracle.

The plan is host memory only, so these run without a GPU: DOF counts against the paper's table,
and the hierarchy, the basis, every leaf's full and truncated block and the restriction of functions
to leaves against `oracle/mlhp_oracle.py`, element by element.
"""
import os

import numpy as np
import pytest

from oracle import mlhp_oracle as M

fcm = pytest.importorskip("paper_1809_00828_gb300.fcm")
if not os.path.exists(fcm.LIB_PATH):
    pytest.skip("libfcm.so is not built", allow_module_level=True)

CASES = [
    ((8, 8, 8), [(0.5, 0.5, 0.5, 0.01)], 3, 2),            # the Sec. 5.1 cube, two levels
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.1)], 2, 3),             # a cavity that cuts many cells per level
    ((3, 2, 4), [(0.2, 0.3, 0.4, 0.25), (0.9, 0.1, 0.7, 0.3)], 4, 2),  # odd grid, two spheres, p = 4
    ((2, 2, 2), [(0.0, 0.0, 0.0, 0.3)], 1, 3),             # refinement into a domain corner, p = 1
]


def test_paper_dof_table_from_the_library_plan():
    rows = [line.split() for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_sec5_1_dofs.txt"))
            if line.strip() and not line.startswith("#")]
    for k, dofs in ((int(a), int(b)) for a, b in rows):
        P = fcm.MLHPPlan((8, 8, 8), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.01)], 3, k)
        assert 3 * P.info["n_functions_trunk"] == dofs
        assert P.info["n_max_truncated"] == 8
        P.close()


@pytest.mark.parametrize("n,spheres,p,k", CASES)
def test_plan_matches_the_oracle_hierarchy_basis_and_blocks(n, spheres, p, k):
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), spheres, p, k)
    H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), spheres, k)
    B = M.Basis(H, p)
    assert P.info["levels"] == H.levels
    assert P.info["n_leaves"] == len(H.leaves)
    assert [P.leaf(i) for i in range(len(H.leaves))] == [(l, tuple(c)) for l, c in H.leaves]
    assert P.info["n_functions"] == len(B.funcs)
    assert [P.function(f) for f in range(len(B.funcs))] == [(l, tuple(q), tuple(m)) for l, q, m in B.funcs]
    assert 3 * P.info["n_functions_trunk"] == M.count_dofs(H, p, "trunk")
    for i, (L, c) in enumerate(H.leaves):
        assert P.block(i, "full").tolist() == B.leaf_functions(L, c)
        assert P.block(i, "truncated").tolist() == B.truncated_functions(L, c)
    assert P.info["n_max_full"] == B.overlap("full")
    assert P.info["n_max_truncated"] == B.overlap("truncated") <= 8
    P.close()


@pytest.mark.parametrize("n,spheres,p,k", CASES[1:])
def test_restriction_reproduces_the_function_on_the_leaf(n, spheres, p, k):
    # fcm_mlhp_restriction: the tensor product of the 1D coefficients in the leaf's own basis must give
    # the values the oracle evaluates through the leaf's ancestors, at random points of the leaf.
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), spheres, p, k)
    H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), spheres, k)
    B = M.Basis(H, p)
    rng = np.random.default_rng(4)
    t = rng.uniform(-1, 1, (12, 3))
    leaves = [i for i, (L, _) in enumerate(H.leaves) if L == H.levels - 1][:6] + list(range(3))
    for i in leaves:
        L, c = H.leaves[i]
        fids = B.leaf_functions(L, c)
        ref, _ = B.eval_on_leaf(L, c, fids, t)
        for r, f in enumerate(fids):
            coef = P.restriction(i, f)
            val = np.ones(len(t))
            for a in range(3):
                F, _ = M.shape1d(p, t[:, a])
                val *= coef[a] @ F
            assert np.abs(val - ref[r]).max() < 1e-13
    # a function not supported on the leaf is refused
    L, c = H.leaves[0]
    outside = sorted(set(range(len(B.funcs))) - set(B.leaf_functions(L, c)))
    with pytest.raises(fcm.FcmError):
        P.restriction(0, outside[0])
    P.close()


def test_plan_rejects_bad_arguments():
    with pytest.raises(fcm.FcmError):
        fcm.MLHPPlan((2, 2, 2), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.1)], 5, 1)
    with pytest.raises(fcm.FcmError):
        fcm.MLHPPlan((0, 2, 2), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.1)], 2, 1)
    with pytest.raises(fcm.FcmError):
        fcm.MLHPPlan((2, 2, 2), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.1)], 2, -1)


def test_leaf_stiffness_is_the_standard_cell_matrix_through_the_restriction():
    # The multi-level path's K apply per leaf: gather the leaf's functions, map them with the plan's
    # restriction C onto the leaf's own basis, apply the standard element matrix of a cell of the leaf's
    # size (the uniform-grid C oracle's, cut cells included), map back.  C K_cell C^T must be the
    # multi-level oracle's leaf matrix.
    from oracle import oracle as O
    from paper_1809_00828_gb300 import inputs as I
    p, k, depth, alpha = 2, 2, 2, 1e-6
    sph = np.array([[0.5, 0.5, 0.5, 0.1]])
    P = fcm.MLHPPlan((4, 4, 4), (0, 0, 0), (1, 1, 1), sph, p, k)
    H = M.refine_toward_spheres((4, 4, 4), (0, 0, 0), (1, 1, 1), sph, k)
    Q = M.MLProblem(H, p, sph, alpha=alpha, depth=depth)
    g = I.Geometry(I.GEOM_SPHERE_VOIDS, spheres=sph, octree_depth=depth)
    order = [0] + list(range(2, p + 1)) + [1]          # plan's (N0, N1, phi_2..) -> lattice order within a cell
    descs = {}
    checked = cut = 0
    for i, (L, c) in enumerate(H.leaves):
        if Q.eta[(L, c)] == 0.0 or (i % 7 and L < H.levels - 1):
            continue
        if L not in descs:
            descs[L] = O.make_desc([4 << L] * 3, p, alpha, g)
        Kc, eta = O.cell_matrix(descs[L][0], c)
        assert abs(eta - Q.eta[(L, c)]) < 1e-13
        fids = P.block(i, "full")
        C = np.zeros((len(fids), (p + 1) ** 3))
        for r, f in enumerate(fids):
            cf = P.restriction(i, int(f))[:, order]
            C[r] = np.einsum("z,y,x->zyx", cf[2], cf[1], cf[0]).reshape(-1)
        C3 = np.kron(C, np.eye(3))
        Kml = C3 @ Kc @ C3.T
        _, Kref = Q.leaf_matrix(L, c)
        assert np.abs(Kml - Kref).max() <= 1e-12 * np.abs(Kref).max()
        checked += 1
        cut += 0.0 < eta < 1.0
    assert checked >= 20 and cut >= 5
    P.close()


@pytest.mark.parametrize("n,spheres,p,k,depth,alpha,bc", [
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.1)], 2, 2, 2, 1e-6, "clamp"),
    ((3, 2, 2), [(0.2, 0.3, 0.4, 0.25), (0.9, 0.1, 0.97, 0.3)], 3, 1, 2, 1e-3, "roller"),  # a void through z = 1
    ((2, 2, 2), [(0.0, 0.0, 0.0, 0.3)], 1, 3, 3, 1e-8, "clamp"),
])
def test_assembled_system_matches_the_oracle(n, spheres, p, k, depth, alpha, bc):
    # fcm_mlhp_assemble (moment quadrature per leaf box, C K_cell C^T, quadtree traction) against the
    # oracle's point-wise assembly on the same hierarchy: same free DOFs, K and b to rounding.
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), spheres, p, k, octree_depth=depth)
    free, K, rhs, eta = P.assemble(alpha, bc)
    H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), spheres, k)
    Q = M.MLProblem(H, p, spheres, alpha=alpha, depth=depth, bc=bc)
    assert np.array_equal(free, Q.free)
    assert abs(K - Q.K).max() <= 1e-13 * abs(Q.K).max()
    assert np.abs(rhs - Q.b).max() <= 1e-13 * np.abs(Q.b).max()
    assert max(abs(eta[i] - Q.eta[lc]) for i, lc in enumerate(H.leaves)) < 1e-13
    P.close()


def test_truncated_block_colours_share_no_function():
    # fcm_mlhp_colour: blocks of one colour are disjoint in their functions (one launch per colour can
    # scatter without atomics); the uniform grid needs the 8 parity colours.
    for n, spheres, p, k in CASES[:3]:
        P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), spheres, p, k)
        colour, nc = P.colour("truncated")
        assert nc == colour.max() + 1 <= 16
        for c in range(nc):
            seen = set()
            for i in np.flatnonzero(colour == c):
                f = set(P.block(int(i), "truncated").tolist())
                assert not (f & seen)
                seen |= f
        P.close()
    P = fcm.MLHPPlan((4, 4, 4), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.1)], 2, 0)
    assert P.colour("truncated")[1] == P.colour("full")[1] == 8
    P.close()


@pytest.mark.parametrize("n,spheres,p,k,depth,alpha,kind,eta_bar", [
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.1)], 2, 2, 2, 1e-6, "truncated", 1.0),
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.1)], 2, 2, 2, 1e-6, "truncated", 0.5),   # blocks on the cut leaves only
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.1)], 2, 1, 2, 1e-6, "full", 1.0),
    ((2, 2, 2), [(0.0, 0.0, 0.0, 0.3)], 3, 2, 2, 1e-8, "truncated", 1.0),
])
def test_schwarz_factors_match_the_oracle_blocks_and_pseudo_inverses(n, spheres, p, k, depth, alpha, kind, eta_bar):
    # fcm_mlhp_factorize: the same blocks as the oracle (as sets of free DOFs), colour classes without a
    # shared DOF, and each factor the pseudo inverse of its block (numpy's eigensolver on the assembled K):
    # two eigensolvers agree on A_B^+ to about cond(A_B) times the rounding unit.
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), spheres, p, k, octree_depth=depth)
    free, K, rhs, eta = P.assemble(alpha, "clamp")
    blocks, F, cptr, jac = P.factorize(kind, eta_bar=eta_bar)
    H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), spheres, k)
    Q = M.MLProblem(H, p, spheres, alpha=alpha, depth=depth)
    Q.build_blocks(kind, eta_bar=eta_bar)
    assert sorted(tuple(b) for b in blocks) == sorted(tuple(b) for b in Q.blocks)
    assert np.array_equal(jac == 0.0, Q.jacobi == 0.0)
    assert np.abs(jac - Q.jacobi).max() <= 1e-13 * np.abs(Q.jacobi).max(initial=1.0)
    for c in range(len(cptr) - 1):
        members = np.concatenate([blocks[b] for b in range(cptr[c], cptr[c + 1])])
        assert len(members) == len(np.unique(members))
    for B, Fb in zip(blocks, F):
        lam, V = np.linalg.eigh(K[B][:, B].toarray())
        keep = lam > 1e-13 * lam.max()
        Fn = (V[:, keep] / lam[keep]) @ V[:, keep].T
        cond = lam.max() / lam[keep].min()
        assert np.abs(Fb - Fn).max() <= max(1e-12, 64 * cond * 2.2e-16) * np.abs(Fn).max()
    P.close()


def test_eta_bar_zero_leaves_only_the_diagonal_part():
    # eta_bar = 0: no leaf gets a block (Sec. 3.2, "eta_bar = 0 results in a Jacobi preconditioner"), so S is
    # 1 / K_ll on every free DOF.
    P = fcm.MLHPPlan((4, 4, 4), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.1)], 2, 1, octree_depth=2)
    free, K, rhs, eta = P.assemble(1e-6, "clamp")
    blocks, F, cptr, jac = P.factorize("truncated", eta_bar=0.0)
    assert blocks == [] and len(cptr) == 1
    assert np.array_equal(jac, 1.0 / K.diagonal())
    P.close()


def test_porous_hierarchy_overlap_grows_like_the_paper_table_for_full_blocks_only():
    # Sec. 5.3 table of n_max (gearbox, refined toward internal pores, k = 0..3): full blocks 8, 64, 274, 810;
    # truncated blocks 8 at every depth.  A porous cube (40 voids, 8^3 base, p = 3) refined toward the void
    # surfaces shows the same pattern: 8, 57, 323, 1450 for full blocks, 8 for truncated ones.
    from paper_1809_00828_gb300 import inputs as I
    sph = I.random_sphere_voids(11, 40, 0.02, 0.08).sphere_array()
    full = []
    for k in range(4):
        P = fcm.MLHPPlan((8, 8, 8), (0, 0, 0), (1, 1, 1), sph, 3, k)
        assert P.info["n_max_truncated"] == 8
        full.append(P.info["n_max_full"])
        P.close()
    assert full[0] == 8
    assert all(b > 2.5 * a for a, b in zip(full, full[1:]))


@pytest.mark.parametrize("which", ["voxels", "halfspace"])
def test_voxel_and_halfspace_hierarchies_match_the_oracle(which):
    # The plan refines toward any boundary the uniform grid supports: a voxel image's solid-void interfaces
    # (a 16^3 Gaussian random field, as for the trabecular workloads) or a tilted plane.  Hierarchy, blocks
    # and the assembled system against the oracle.
    from paper_1809_00828_gb300 import inputs as I
    if which == "voxels":
        g = I.gaussian_random_field_voxels(3, m=16, corr_len=0.15, solid_fraction=0.5, octree_depth=2)
        n, k = (4, 4, 4), 2
    else:
        g = I.halfspace(1.0, 0.3, 0.2, 0.81, octree_depth=2)
        n, k = (3, 3, 3), 1
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), None, 2, k, octree_depth=2, geometry=g)
    H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), g, k)
    assert all(len(r) > 0 for r in H.refined[:k])
    B = M.Basis(H, 2)
    assert [P.leaf(i) for i in range(len(H.leaves))] == [(l, tuple(c)) for l, c in H.leaves]
    for i, (L, c) in enumerate(H.leaves):
        assert P.block(i, "truncated").tolist() == B.truncated_functions(L, c)
    assert P.info["n_max_truncated"] <= 8
    free, K, rhs, eta = P.assemble(1e-6, "clamp")
    Q = M.MLProblem(H, 2, g, alpha=1e-6, depth=2)
    assert np.array_equal(free, Q.free)
    assert abs(K - Q.K).max() <= 1e-13 * abs(Q.K).max()
    assert np.abs(rhs - Q.b).max() <= 1e-13 * np.abs(Q.b).max()
    assert max(abs(eta[i] - Q.eta[lc]) for i, lc in enumerate(H.leaves)) < 1e-13
    P.close()


def test_random_hierarchies_match_the_oracle():
    # Seeded random cases: boxes that are not cubes, spheres that cross the domain boundary, p = 1..4,
    # k = 0..3.  Leaves, functions, every full and truncated block, and n_max against the oracle.
    rng = np.random.default_rng(123)
    for _ in range(25):
        n = tuple(int(v) for v in rng.integers(1, 4, 3))
        p = int(rng.integers(1, 5))
        k = int(rng.integers(0, 4))
        sph = [tuple(float(v) for v in (*rng.uniform(-0.2, 1.2, 3), rng.uniform(0.05, 0.5)))
               for _ in range(int(rng.integers(1, 4)))]
        hi = tuple(float(v) for v in rng.uniform(0.5, 2.0, 3))
        P = fcm.MLHPPlan(n, (0, 0, 0), hi, sph, p, k)
        H = M.refine_toward_spheres(n, (0, 0, 0), hi, sph, k)
        B = M.Basis(H, p)
        assert [P.leaf(i) for i in range(P.info["n_leaves"])] == [(l, tuple(c)) for l, c in H.leaves]
        assert P.info["n_functions"] == len(B.funcs)
        for i, (L, c) in enumerate(H.leaves):
            assert P.block(i, "full").tolist() == B.leaf_functions(L, c)
            assert P.block(i, "truncated").tolist() == B.truncated_functions(L, c)
        assert P.info["n_max_truncated"] == B.overlap("truncated") <= 8
        P.close()
