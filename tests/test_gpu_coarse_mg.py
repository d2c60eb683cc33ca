"""GPU tests of the cell-grid multigrid V-cycle that can precondition the coarse CG of the flexible
PCG (fcm_coarse_set_preconditioner, fcm_coarse_vcycle).  Not part of the paper's method: a coarse
space for the iteration growth its Sec. 6 names.

The reference is the V-cycle written out here from its definition with scipy, on the Galerkin
product K_H = P^T K P of the oracle's assembled stiffness:
  levels halve the cells per axis (n' = (n + 1) / 2), P2 cell-centred trilinear (3/4 and 1/4, all of
  it at the boundary), K_{l+1} = P2^T K_l P2, the 3x3 diagonal blocks inverted, one block-Jacobi step
  damped by omega = 4 / (3.3 lambda) before and after the coarse correction (lambda the device's
  power-iteration estimate, reported by fcm_coarse_levels and checked against eigs here), the last
  level (at most 512 cells) by its pseudo-inverse (eigenvalues below 1e-12 of the largest dropped).

The device stores K_H and the levels in FP32 and computes in FP32; a pseudo-inverse amplifies such
perturbations by up to the condition number of the coarsest operator, so the bound on the
difference in the K_H energy norm is 64 * 2^-24 * cond(K_L) + 1e-5.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _prolongation(w, free_lat):
    """Explicit P: cell value (component-major) -> lattice DOFs (1/8 at the 8 vertex nodes), free rows."""
    nx, ny, nz = w.n
    p = w.p
    M = [p * n + 1 for n in w.n]
    nc = nx * ny * nz
    rows, cols = [], []
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                c = cx + nx * (cy + ny * cz)
                for k in range(8):
                    node = p * (cx + (k & 1)) + M[0] * (p * (cy + ((k >> 1) & 1)) + M[1] * p * (cz + (k >> 2)))
                    for a in range(3):
                        rows.append(3 * node + a)
                        cols.append(a * nc + c)
    nlat = 3 * M[0] * M[1] * M[2]
    Pl = sp.csr_matrix((np.full(len(rows), 0.125), (rows, cols)), shape=(nlat, 3 * nc))
    return Pl[free_lat, :]


def _p1d(nf):
    """1-D cell-centred interpolation from (nf + 1) // 2 coarse cells to nf fine cells."""
    if nf == 1:
        return sp.identity(1, format="csr")
    nc = (nf + 1) // 2
    rows, cols, vals = [], [], []
    for i in range(nf):
        c = i // 2
        o = c + 1 if i % 2 else c - 1
        if 0 <= o < nc:
            rows += [i, i]
            cols += [c, o]
            vals += [0.75, 0.25]
        else:
            rows.append(i)
            cols.append(c)
            vals.append(1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def _p2(n):
    """P2 for component-major cell vectors of grid n = (nx, ny, nz) (cell index x fastest)."""
    Px, Py, Pz = (_p1d(m) for m in n)
    P1 = sp.kron(Pz, sp.kron(Py, Px)).tocsr()
    return sp.block_diag([P1, P1, P1]).tocsr(), tuple(m if m == 1 else (m + 1) // 2 for m in n)


def _block_dinv(A, nc):
    """Inverses of the 3x3 blocks {c, nc + c, 2 nc + c} of A (0 where singular, as on the device)."""
    A = A.tocsr()
    rows, cols, vals = [], [], []
    for c in range(nc):
        idx = [c, nc + c, 2 * nc + c]
        B = A[idx, :][:, idx].toarray()
        tr = abs(B[0, 0]) + abs(B[1, 1]) + abs(B[2, 2])
        det = np.linalg.det(B)
        if tr == 0.0 or not abs(det) > 1e-30 * tr ** 3:
            continue
        Bi = np.linalg.inv(B)
        for a in range(3):
            for b in range(3):
                rows.append(idx[a])
                cols.append(idx[b])
                vals.append(Bi[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=A.shape)


def _reference_vcycle(KH, n, lambdas):
    """The V-cycle as a function f -> x; returns (fn, level grids, cond of the last level, levels)."""
    mats, P2s, dims = [KH.tocsr()], [], [tuple(n)]
    while int(np.prod(dims[-1])) > 512:
        P2, nc = _p2(dims[-1])
        mats.append((P2.T @ mats[-1] @ P2).tocsr())
        P2s.append(P2)
        dims.append(nc)
    last = mats[-1].toarray()
    last = 0.5 * (last + last.T)
    ev, V = np.linalg.eigh(last)
    keep = ev > 1e-12 * ev.max()
    pinv = (V[:, keep] / ev[keep]) @ V[:, keep].T
    cond = ev[keep].max() / ev[keep].min()
    levels = []
    for l in range(len(P2s)):
        nc = int(np.prod(dims[l]))
        om = float(np.float32(4.0 / (3.0 * 1.1 * lambdas[l])))
        levels.append((mats[l], P2s[l], _block_dinv(mats[l], nc), om))

    def vc(f, l=0):
        if l == len(levels):
            return pinv @ f
        A, P2, Di, om = levels[l]
        x = om * (Di @ f)
        r = f - A @ x
        x = x + P2 @ vc(P2.T @ r, l + 1)
        return x + om * (Di @ (f - A @ x))

    def hybrid(f):
        if not levels:
            return pinv @ f
        _, P2, Di, om = levels[0]
        return om * (Di @ f) + P2 @ vc(P2.T @ f, 1)

    return {"vcycle": vc, "hybrid": hybrid}, dims, cond, levels


def _workload(kind):
    if kind == "odd":
        geo = I.random_sphere_voids(21, 4, 0.05, 0.12, octree_depth=2)
        return I.Workload("porous_18x12x9_p1", (18, 12, 9), 1, 1e-3, geo, 1e-8)
    geo = I.random_sphere_voids(22, 6, 0.05, 0.12, octree_depth=2)
    return I.Workload("porous_24_p1", (24, 24, 24), 1, 1e-3, geo, 1e-8)


@pytest.mark.parametrize("cycle", ["vcycle", "hybrid"])
@pytest.mark.parametrize("kind,levels", [("odd", 2), ("cube", 3)])
def test_vcycle_matches_its_definition(kind, levels, cycle):
    from paper_1809_00828_gb300 import fcm
    w = _workload(kind)
    P = O.Problem.from_workload(w)
    s = fcm.Solver(w)
    try:
        s.precond_build()
        nc = int(np.prod(w.n))
        rng = np.random.default_rng(5)
        f = rng.standard_normal(3 * nc).astype(np.float32)
        x_dev = s.coarse_vcycle(torch.from_numpy(f).cuda(), kind=cycle).cpu().numpy().astype(np.float64)
        info = s.coarse_levels()
        assert info["levels"] == levels
        Pf = _prolongation(w, P.free_lat)
        KH = (Pf.T @ P.csr() @ Pf).tocsr()
        cycles, dims, cond, lv = _reference_vcycle(KH, w.n, info["lambda_max"])
        vc = cycles[cycle]
        assert [tuple(d) for d in info["dims"]] == dims
        # the smoother's lambda: 15 power steps approach lambda_max(Dinv K_l) from below
        for l, (A, _, Di, _) in enumerate(lv):
            lam = abs(spla.eigs(Di @ A, k=1, which="LM", return_eigenvectors=False, tol=1e-6)[0])
            # (|| Dinv K v || / || v || of a non-normal Dinv K may overshoot its spectral radius a little)
            assert 0.7 * lam <= info["lambda_max"][l] <= 1.5 * lam, (l, info["lambda_max"][l], lam)
        x_ref = vc(f.astype(np.float64))
        e = x_dev - x_ref
        err = np.sqrt(e @ (KH @ e)) / np.sqrt(x_ref @ (KH @ x_ref))
        bound = 64 * 2.0 ** -24 * cond + 1e-5
        print(f"{kind} {cycle}: levels {dims}, cond(K_L) {cond:.3g}, energy difference {err:.3g} (bound {bound:.3g})")
        assert err <= bound
        # a symmetric positive semi-definite operator, as the coarse CG needs
        g = rng.standard_normal(3 * nc).astype(np.float32)
        y_dev = s.coarse_vcycle(torch.from_numpy(g).cuda(), kind=cycle).cpu().numpy().astype(np.float64)
        a, b = g.astype(np.float64) @ x_dev, f.astype(np.float64) @ y_dev
        assert abs(a - b) <= max(1e-4, bound) * max(abs(a), abs(b))
        assert f.astype(np.float64) @ x_dev > 0.0
    finally:
        s.close()


def test_vcycle_on_one_level_is_the_pseudo_inverse():
    from paper_1809_00828_gb300 import fcm
    w = I.workload_porous(5, 8, 2, 6, 1e-3, 3, 1e-9)
    P = O.Problem.from_workload(w)
    s = fcm.Solver(w)
    try:
        s.precond_build()
        nc = int(np.prod(w.n))
        Pf = _prolongation(w, P.free_lat)
        KH = (Pf.T @ P.csr() @ Pf).tocsr()
        f = (KH @ np.random.default_rng(2).standard_normal(3 * nc)).astype(np.float32)  # in the range of K_H
        x = s.coarse_vcycle(torch.from_numpy(f).cuda()).cpu().numpy().astype(np.float64)
        assert s.coarse_levels()["levels"] == 1
        ev = np.linalg.eigvalsh(KH.toarray())
        ev = ev[ev > 1e-12 * ev.max()]
        cond = ev.max() / ev.min()
        r = KH @ x - f
        # FP32 K_H and FP32 pseudo-inverse entries: relative residual ~ cond * 2^-24
        assert np.linalg.norm(r) <= (64 * 2.0 ** -24 * cond + 1e-5) * np.linalg.norm(f)
    finally:
        s.close()


def test_fpcg_with_vcycle_coarse_cg():
    """Flexible PCG whose coarse CG is preconditioned by the V-cycle: the same solution as the
    direct solve, in fewer iterations than with block-Jacobi coarse steps."""
    from paper_1809_00828_gb300 import fcm
    w = _workload("cube")
    P = O.Problem.from_workload(w)
    s = fcm.Solver(w)
    try:
        s.precond_build()
        b = s.rhs()
        _, its_j, _, st_j = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=2)
        s.set_coarse_preconditioner("vcycle")
        u, its_v, rel, st = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=2)
        assert st == 0 and st_j == 0 and rel <= w.tol * 1.0001
        assert s.last_solve()["fallback"] == 0
        x_ref = spla.spsolve(P.csr().tocsc(), P.rhs())
        assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
        assert its_v < its_j
        s.set_coarse_preconditioner("hybrid")
        u, its_h, rel, st = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=2)
        assert st == 0 and rel <= w.tol * 1.0001
        assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
        print(f"flexible PCG, 2 coarse steps: block Jacobi {its_j} iterations, V-cycle {its_v}, hybrid {its_h}")
        # back to block Jacobi: the captured iteration is rebuilt and gives the first count again
        s.set_coarse_preconditioner("jacobi")
        _, its_j2, _, _ = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=2)
        assert its_j2 == its_j
        with pytest.raises(ValueError):
            s.set_coarse_preconditioner("amg")
    finally:
        s.close()


def test_fp16_storage_of_the_coarse_operator():
    """K_H stored as K~ = s K s in FP16 (s_c = (tr K_cc / 3)^-1/2).  Each stored entry is rounded once to
    FP16: relative error <= 2^-11 above FP16's normal range, absolute <= 2^-25 (half the subnormal spacing)
    below it, i.e. |K'_cj - K_cj| <= 2^-11 |K_cj| + 2^-25 / (s_c s_j); FP32 scaling and accumulation add
    ~1e-6 relative.  So per cell row |y - K_H x| <= (2^-11 + 1e-5) (|K_H| |x|) + 2^-25 / s_c (B (|x| / s))
    with B the block pattern.  Then the flexible PCG with the FP16 operator reaches the direct solution."""
    from paper_1809_00828_gb300 import fcm
    w = _workload("cube")
    P = O.Problem.from_workload(w)
    s = fcm.Solver(w)
    try:
        s.precond_build()
        nc = int(np.prod(w.n))
        Pf = _prolongation(w, P.free_lat)
        KH = (Pf.T @ P.csr() @ Pf).tocsr()
        d = KH.diagonal()
        tr = d[:nc] + d[nc:2 * nc] + d[2 * nc:]
        sc = np.where(tr > 0, 1.0 / np.sqrt(np.maximum(tr, 1e-300) / 3.0), 0.0)
        s3 = np.concatenate([sc, sc, sc])
        s.set_coarse_storage("fp16")
        rng = np.random.default_rng(8)
        for trial in range(2):
            x = rng.standard_normal(3 * nc).astype(np.float32)
            y = s.coarse_apply(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
            xd = x.astype(np.float64)
            ref = KH @ xd
            absK = abs(KH)
            pattern = (absK > 0).astype(np.float64)
            inv_s = np.where(s3 > 0, 1.0 / np.where(s3 > 0, s3, 1.0), 0.0)
            bound = (2.0 ** -11 + 1e-5) * (absK @ np.abs(xd)) + 2.0 ** -25 * inv_s * (pattern @ (np.abs(xd) * inv_s))
            assert (np.abs(y - ref) <= bound + 1e-30).all(), float(np.max(np.abs(y - ref) / (bound + 1e-30)))
            # and FP16 is not FP32: the products do differ (the copy is in use)
            if trial == 0:
                s.set_coarse_storage("fp32")
                y32 = s.coarse_apply(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
                assert np.abs(y32 - ref).max() <= 1e-5 * np.abs(ref).max()
                assert np.abs(y - y32).max() > 0.0
                s.set_coarse_storage("fp16")
        s.set_coarse_preconditioner("vcycle")
        b = s.rhs()
        u, its, rel, st = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=2)
        assert st == 0 and rel <= w.tol * 1.0001
        x_ref = spla.spsolve(P.csr().tocsc(), P.rhs())
        assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
        print(f"flexible PCG, 2 V-cycle steps, FP16 K_H: {its} iterations")
        with pytest.raises(ValueError):
            s.set_coarse_storage("bf16")
    finally:
        s.close()
