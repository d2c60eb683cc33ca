"""GPU parity of the multi-RHS Schwarz apply and PCG at p = 3 (the order and the six unit-strain load
cases of the trabecular workload), against the CPU oracle.

A porous 4^3-cell cube with 3 voids: cut patches stream their own factors (FP32 and, in the mixed
build, double-float pairs), uncut interior patches share factors and go through the dense product,
and 375-row blocks cross several row tiles with a ragged tail.  Bounds: S r per DOF by the
eigensolver perturbation of the blocks that contain it (tests/schwarz_bounds.py; FP32 factors add
their storage rounding, 2^-24, and the tensor-core products of shared factors theirs, ~2^-22: 2^-20
covers both), and 1e-9 (FP64) or 1e-5 (FP32 factors) in the energy norm of K; the
PCG solutions within 1e-8 of a sparse direct solve in the energy norm (Eq. (15)), iteration counts
within 2 of the oracle's PCG on each load case.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I
from schwarz_bounds import dof_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def porous4():
    w = I.workload_porous(13, 4, 3, 3, 1e-10, 3, 1e-10)
    P = O.Problem.from_workload(w)
    P.precond_build(0)
    return w, P


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_rhs_S_columns_match_oracle(porous4, precision):
    from paper_1809_00828_gb300 import fcm
    w, P = porous4
    s = fcm.Solver(w)
    # mixed: a low threshold (1e3) so that this small cube also has double-float factors
    s.precond_build(precision=precision, cond_fp64=1e3)
    assert s.info["n_gemm_blocks"] > 0
    if precision == "mixed":
        assert s.info["n_factors_ff"] > 0 and s.info["n_blocks_fp32"] > 0
    R = np.concatenate([I.random_vector(40 + k, s.n) for k in range(6)])
    Z = s.apply_S(torch.from_numpy(R).cuda()).cpu().numpy()
    K = P.csr()
    # FP32 factors round to 2^-24; the tensor-core products of shared factors (TF32, three passes) to ~2^-22
    u = 2.0 ** -20 if precision == "mixed" else 0.0
    for k in range(6):
        rk = R[k * s.n:(k + 1) * s.n]
        zk = Z[k * s.n:(k + 1) * s.n]
        z_ref = P.apply_S(rk[P.free_lat])
        d = zk[P.free_lat] - z_ref
        e = np.sqrt(abs(d @ (K @ d)) / (z_ref @ (K @ z_ref)))
        assert e < (1e-5 if precision == "mixed" else 1e-9), (k, e)
        assert np.all(np.abs(d) <= dof_bound(P, rk[P.free_lat], u_factor=u)), k
        # the non-free entries stay zero
        mask = np.zeros(s.n, dtype=bool)
        mask[P.free_lat] = True
        assert not zk[~mask].any()
        # column k of the multi-vector apply against the single-vector apply
        z1 = s.apply_S(torch.from_numpy(rk).cuda()).cpu().numpy()
        assert np.all(np.abs(zk - z1)[P.free_lat] <= dof_bound(P, rk[P.free_lat], u_factor=u))
    s.close()


def test_multi_rhs_pcg_p3_matches_oracle(porous4):
    import scipy.sparse.linalg as spla
    from paper_1809_00828_gb300 import fcm
    w, P = porous4
    s = fcm.Solver(w)
    s.precond_build()
    B = torch.cat([s.rhs(k) for k in range(1, 7)])
    U, its, rel, st = s.pcg_solve(B, w.tol, 3000)
    K = P.csr().tocsc()
    solve = spla.factorized(K)
    worst = 0
    for k in range(6):
        bk = P.load(k + 1)
        x_direct = solve(bk)
        uk = U[k * s.n:(k + 1) * s.n].cpu().numpy()[P.free_lat]
        assert P.energy_error(x_direct, uk) < 1e-8, k
        _, its_o, _ = P.pcg(b=bk, tol=w.tol, maxit=3000)
        _, its_1, _, _ = s.pcg_solve(s.rhs(k + 1), w.tol, 3000)
        assert abs(its_1 - its_o) <= 2, (k, its_1, its_o)
        worst = max(worst, its_o)
    assert rel <= w.tol and abs(its - worst) <= 2
    s.close()
