"""Parity of the multi-level GPU path (fcm_mlhp_device_setup / apply_K / apply_S / pcg_solve) with the
multi-level oracle.  The inputs are a cavity cube refined toward the cavity's surface (Sec. 5.1 set-up,
scaled to a 4^3 base grid) and a larger cavity that cuts many leaves.

- K x: the device CSR product against the oracle's assembled K.  The device stores the values as float
  pairs (2^-48 relative) and sums double-float products (2^-46 relative each, TwoSum accumulation), so
  per row |y - Kx| <= 2^-43 (|K| |x|), which also covers the two assemblies' rounding.
- S r: against the same factors applied on the host, per DOF 2^-43 sum_B (|A_B^+| |r_B|) for the same
  reason (float-pair factors, double-float products and sums).  Against
  the oracle's own pseudo inverses per DOF: two backward-stable eigensolvers agree on A_B^+ to
  c n eps (cond(A_B) + 1) ||A_B^+|| (cond over the retained spectrum), so a DOF may differ by the sum of
  that times ||r_B|| over the blocks containing it (c = 10); sliver leaves reach cond ~ 1e10 and loosen
  the bound on their own DOFs only.
- PCG with truncated blocks: iterations within 5 % of the oracle's (its factors come from another
  eigensolver), energy error below 1e-6 against a sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import mlhp_oracle as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.02)], 2, 3, 3, 1e-8),   # the Sec. 5.1 cavity scaled to a 4^3 base grid
    ((4, 4, 4), [(0.5, 0.5, 0.5, 0.1)], 2, 2, 2, 1e-6),    # a cavity that cuts many leaves into slivers
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def case(request):
    from paper_1809_00828_gb300 import fcm
    n, sph, p, k, depth, alpha = CASES[request.param]
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), sph, p, k, octree_depth=depth)
    free, K, b, eta = P.assemble(alpha, "clamp")
    blocks, F, cptr, jac = P.factorize("truncated")
    P.device_setup()
    H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), sph, k)
    Q = M.MLProblem(H, p, sph, alpha=alpha, depth=depth)
    Q.build_blocks("truncated")
    assert np.array_equal(free, Q.free)
    yield fcm, P, b, blocks, F, jac, Q
    P.close()


def test_mlhp_apply_K_matches_the_oracle(case):
    fcm, P, b, blocks, F, jac, Q = case
    x = np.random.default_rng(2).standard_normal(Q.n)
    y = P.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = Q.K @ x
    bound = 2.0 ** -43 * (abs(Q.K) @ np.abs(x))
    assert (np.abs(y - ref) <= bound).all(), float(np.max(np.abs(y - ref) / bound))


def test_mlhp_apply_S_matches_the_factors_and_the_oracle(case):
    fcm, P, b, blocks, F, jac, Q = case
    r = np.random.default_rng(3).standard_normal(Q.n)
    z = P.apply_S(torch.from_numpy(r).cuda()).cpu().numpy()
    zh = jac * r
    mag = np.abs(jac * r) * 2.0 ** -50
    for B, Fb in zip(blocks, F):
        zh[B] += Fb @ r[B]
        mag[B] += 2.0 ** -43 * (np.abs(Fb) @ np.abs(r[B]))
    assert (np.abs(z - zh) <= mag).all(), float(np.max(np.abs(z - zh) / mag))
    zo = Q.apply_S(r)
    bound = np.zeros(Q.n)
    for B in Q.blocks:
        lam = np.linalg.eigvalsh(Q.K[B][:, B].toarray())
        keep = lam[lam > 1e-13 * lam.max()]
        cond = keep.max() / keep.min()
        bound[B] += 10.0 * len(B) * 2.0 ** -52 * (cond + 1.0) / keep.min() * np.linalg.norm(r[B])
    bound += np.abs(jac * r) * 2.0 ** -52 * 4  # the diagonal part, rounding only
    assert (np.abs(z - zo) <= bound).all(), float(np.max(np.abs(z - zo) / np.maximum(bound, 1e-300)))


def test_mlhp_pcg_matches_the_oracle(case):
    fcm, P, b, blocks, F, jac, Q = case
    _, its_o = Q.pcg(tol=1e-8, maxit=5000)
    u, its, rel, st = P.pcg_solve(torch.from_numpy(b).cuda(), 1e-8, 5000)
    assert st == fcm.FCM_OK and rel <= 1e-8
    # the factors come from two eigensolvers (cond-level differences on sliver leaves): iterations within 5 %
    assert abs(its - its_o) <= max(3, 0.05 * its_o)
    xref = spla.spsolve(Q.K.tocsc(), Q.b)
    assert Q.energy_error(xref, u.cpu().numpy()) < 1e-6


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_mlhp_mixed_precision_factors(ci):
    """FP32 factors for the blocks whose retained condition number is at most 1e7 (fcm_mlhp_set_precision):
    the blocks so stored are those; their products run in FP32 (factor, r_B, products and the row sum each
    rounded: (m / 32 + 8) 2^-24 of sum_j |F_ij r_j| for a row of m entries, 32 lanes), so S r stays within
    that, summed over the blocks containing a DOF, of the FP64 factors; and PCG reaches the direct
    solution in the oracle's iteration count within 5 %."""
    from paper_1809_00828_gb300 import fcm
    n, sph, p, k, depth, alpha = CASES[ci]
    P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), sph, p, k, octree_depth=depth)
    try:
        free, K, b, eta = P.assemble(alpha, "clamp")
        blocks, F, cptr, jac = P.factorize("truncated")
        P.device_setup(precision="mixed")
        n32, fbytes = P.device_info()
        conds = []
        for B in blocks:
            lam = np.linalg.eigvalsh(K[B][:, B].toarray())
            keep = lam[lam > 1e-13 * lam.max()]
            conds.append(keep.max() / keep.min())
        conds = np.array(conds)
        sizes = np.array([len(B) for B in blocks])
        sure32 = conds <= 0.99e7
        sure64 = conds > 1.01e7
        assert sure32.sum() <= n32 <= len(blocks) - sure64.sum()
        assert 4 * (sizes[sure32] ** 2).sum() + 8 * (sizes[sure64] ** 2).sum() <= fbytes
        assert fbytes <= 4 * (sizes[~sure64] ** 2).sum() + 8 * (sizes[~sure32] ** 2).sum()
        r = np.random.default_rng(4).standard_normal(len(free))
        z = P.apply_S(torch.from_numpy(r).cuda()).cpu().numpy()
        zh = jac * r
        mag = np.abs(jac * r) * 2.0 ** -50
        for B, Fb in zip(blocks, F):
            zh[B] += Fb @ r[B]
            mag[B] += ((len(B) / 32 + 8) * 2.0 ** -24 + 2.0 ** -43) * (np.abs(Fb) @ np.abs(r[B]))
        assert (np.abs(z - zh) <= mag).all(), float(np.max(np.abs(z - zh) / mag))
        H = M.refine_toward_spheres(n, (0, 0, 0), (1, 1, 1), sph, k)
        Q = M.MLProblem(H, p, sph, alpha=alpha, depth=depth)
        Q.build_blocks("truncated")
        _, its_o = Q.pcg(tol=1e-8, maxit=5000)
        u, its, rel, st = P.pcg_solve(torch.from_numpy(b).cuda(), 1e-8, 5000)
        assert st == fcm.FCM_OK and rel <= 1e-8
        assert abs(its - its_o) <= max(3, 0.05 * its_o)
        xref = spla.spsolve(Q.K.tocsc(), Q.b)
        assert Q.energy_error(xref, u.cpu().numpy()) < 1e-6
        print(f"case {ci}: {n32} of {len(blocks)} blocks in FP32, {fbytes} factor bytes, {its} iterations")
    finally:
        P.close()


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_mlhp_device_factorisation_matches_the_host(ci):
    """fcm_mlhp_factorize_device (batched cuSOLVER eigensolves) against the host's cyclic-Jacobi factors: the
    same blocks, and per block ||F_dev - F_host||_2 <= 10 m eps (cond(A_B) + 1) ||F_host||_2, the bound two
    backward-stable eigensolvers satisfy when they keep the same eigenvalues; then the PCG on the device
    factors takes the host factors' iteration count within 2 and reaches the direct solution."""
    from paper_1809_00828_gb300 import fcm
    n, sph, p, k, depth, alpha = CASES[ci]
    P1 = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), sph, p, k, octree_depth=depth)
    P2 = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), sph, p, k, octree_depth=depth)
    try:
        free, K, b, eta = P1.assemble(alpha, "clamp")
        P2.assemble(alpha, "clamp")
        blocks_h, F_h, _, jac_h = P1.factorize("truncated")
        blocks_d, F_d, _, jac_d = P2.factorize("truncated", device=True)
        assert len(blocks_h) == len(blocks_d)
        assert all(np.array_equal(x, y) for x, y in zip(blocks_h, blocks_d))
        assert np.array_equal(jac_h, jac_d)
        worst = 0.0
        for B, Fh, Fd in zip(blocks_h, F_h, F_d):
            lam = np.linalg.eigvalsh(K[B][:, B].toarray())
            keep = lam[lam > 1e-13 * lam.max()]
            cond = keep.max() / keep.min()
            bound = 10 * len(B) * 2.0 ** -52 * (cond + 1.0) * np.linalg.norm(Fh, 2)
            err = np.linalg.norm(Fd - Fh, 2)
            worst = max(worst, err / bound)
            assert err <= bound, (len(B), cond, err, bound)
        bd = torch.from_numpy(b).cuda()
        P1.device_setup(precision="fp64")
        P2.device_setup(precision="fp64")
        _, its_h, _, st_h = P1.pcg_solve(bd, 1e-8, 5000)
        u, its_d, rel, st_d = P2.pcg_solve(bd, 1e-8, 5000)
        assert st_h == fcm.FCM_OK and st_d == fcm.FCM_OK and rel <= 1e-8
        assert abs(its_d - its_h) <= 2
        xref = spla.spsolve(K.tocsc(), b)
        e = u.cpu().numpy() - xref
        assert np.sqrt(e @ (K @ e) / (xref @ (K @ xref))) < 1e-6
        print(f"case {ci}: worst factor difference {worst:.2g} of its bound; PCG {its_h} (host), {its_d} (device)")
    finally:
        P1.close()
        P2.close()
