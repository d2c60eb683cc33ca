"""Full-size parity on the porous workloads: porous40_32_p3 (the bench workload: 32^3 cells, p = 3, 40 voids,
2.7M free DOFs), porous40_64_p2 (64^3 cells, 6.3M) and porous300_80_p2 (80^3 cells, 300 voids, 11.4M), in the
launch configuration bench.py times (the autotuned Schwarz launch): sampled outputs of K x and S r, each
recomputed on its own by the oracle from the cells around it.

- K x: rows at random free DOFs and at the vertex nodes of cut patches; the oracle integrates the element
  matrices of the cells around each row (octree quadrature of depth 4) and forms the row.  FP64 against FP64
  (sum factorisation against dense element matrices): 1e-9 of the row plus 1e-11 of the largest |y|.
- S r: at a vertex node, a DOF belongs to exactly one vertex patch (overlap 1), so (S r)_i is one row of that
  patch's pseudo inverse times r on the patch: the oracle assembles the patch block and inverts it with its
  own eigensolver (cyclic Jacobi).  Two eigensolvers agree on F to about cond(A_B) * 1e-16 relative, so the
  bound is max(1e-9, 1e-15 cond) of sum_j |F_ij r_j|; FP32 factors (mixed precision, cond <= 1e7) add
  5e-5 of the same scale.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["porous40_32_p3", "porous40_64_p2", "porous300_80_p2"])
def bench_problem(request):
    from paper_1809_00828_gb300 import fcm
    w = I.WORKLOADS[request.param]()
    s = fcm.Solver(w)
    d, keep = O.desc_for(w)
    yield w, s, d, keep
    s.close()


def _lattice_index(w, node, comp):
    M = [w.p * n + 1 for n in w.n]
    return 3 * (node[0] + M[0] * (node[1] + M[1] * node[2])) + comp


def _patch_vertices(w, cut, count, seed=5):
    """Interior vertices (0 < v_z) whose 8 cells a sphere surface crosses (cut) or no sphere touches
    (uncut), `count` of them picked at random from all such vertices."""
    h = np.array([(w.hi[a] - w.lo[a]) / w.n[a] for a in range(3)])
    sph = w.geometry.sphere_array()
    g = np.stack(np.meshgrid(*[np.arange(1, w.n[a]) for a in range(3)], indexing="ij"), axis=-1).reshape(-1, 3)
    lo = np.array(w.lo) + (g - 1) * h                       # (V, 3) box of the 8 cells around each vertex
    hi = lo + 2 * h
    c = sph[None, :, :3]                                    # (1, S, 3)
    near = np.clip(c, lo[:, None, :], hi[:, None, :])
    far = np.where(np.abs(c - lo[:, None, :]) > np.abs(c - hi[:, None, :]), lo[:, None, :], hi[:, None, :])
    dmin = np.linalg.norm(c - near, axis=2)
    dmax = np.linalg.norm(c - far, axis=2)
    r = sph[None, :, 3]
    crossed = np.any((dmin < r) & (r < dmax), axis=1)
    touched = np.any(dmin < r, axis=1)
    pick = np.flatnonzero(crossed if cut else ~touched)
    assert len(pick) >= count
    chosen = np.random.default_rng(seed).choice(pick, count, replace=False)
    return [tuple(int(t) for t in g[k]) for k in chosen]


def test_K_apply_sampled_rows_match_the_oracle(bench_problem):
    w, s, d, _ = bench_problem
    x = I.random_vector(21, s.n)
    y = s.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    rng = np.random.default_rng(3)
    rows = [int(i) for i in rng.choice(np.flatnonzero(y), 8, replace=False)]
    for v in _patch_vertices(w, True, 1):  # the vertex node of a cut patch: free, next to a void
        rows += [_lattice_index(w, [w.p * v[0], w.p * v[1], w.p * v[2]], c) for c in range(3)]
    rows = np.array(rows, dtype=np.int64)
    ref, st = O.sample_Kx(d, rows, x)
    assert st == 0
    # rows next to a void mix entries of size 1 and alpha = 1e-10; the bound is relative to the row and
    # to the largest entry of y
    assert np.all(np.abs(y[rows] - ref) <= 1e-9 * np.abs(ref) + 1e-11 * np.abs(y).max())


_FACTORS = {}


def _oracle_factor(w, d, v):
    # the oracle's cut-patch blocks take ~20 s each at p = 3 (depth-4 octree quadrature): computed once
    key = (w.name, v)
    if key not in _FACTORS:
        _FACTORS[key] = O.patch_factor(d, v)
    return _FACTORS[key]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_S_apply_sampled_vertex_rows_match_the_oracle(bench_problem, precision):
    w, s, d, _ = bench_problem
    s.precond_build(precision=precision)
    r = I.random_vector(22, s.n)
    z = s.apply_S(torch.from_numpy(r).cuda()).cpu().numpy()
    checked = 0
    for cut in (True, False):
        # (a cut vertex may still have every cell inside the union of voids: no block, skipped)
        for v in _patch_vertices(w, cut, 3 if cut else 1):
            lat, F, cond = _oracle_factor(w, d, v)
            pos = {int(l): k for k, l in enumerate(lat)}
            for c in range(3):
                i = _lattice_index(w, [w.p * v[0], w.p * v[1], w.p * v[2]], c)
                if i not in pos:
                    continue
                row = F[pos[i]]
                ref = row @ r[lat]
                scale = np.abs(row) @ np.abs(r[lat])
                tol = max(1e-9, 1e-15 * cond)
                if precision == "mixed" and cond <= 1e7:
                    tol += 5e-5
                assert abs(z[i] - ref) <= tol * scale, (v, c, z[i], ref, cond)
                checked += 1
    assert checked >= 6
    assert s.get_info()["device_error"] == 0
