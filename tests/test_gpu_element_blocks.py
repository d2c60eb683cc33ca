"""GPU parity of the paper's element-block rule (Sec. 3.2, "Optimizing the number of
blocks"; Algorithm 1): element blocks for the active cells with eta_T <= eta_bar and
diagonal scaling 1 / K_ll for the free DOFs in no block, against the oracle's rule 3.

Tolerances as in test_gpu_parity.py: the block pseudo-inverses come from different
eigensolvers, so S r is compared in the energy norm of K (1e-9); the diagonal part
alone (eta_bar = 0, no blocks) is exact up to the rounding of K_ll, compared at 1e-13.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lat(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def porous8():
    from paper_1809_00828_gb300 import fcm
    w = I.workload_porous(5, 8, 2, 6, 1e-8, 3, 1e-9)
    P = O.Problem.from_workload(w)
    s = fcm.Solver(w)
    yield w, P, s
    s.close()


def _energy_rel(P, z, z_ref):
    K = P.csr()
    d = z - z_ref
    return np.sqrt(abs(d @ (K @ d)) / (z_ref @ (K @ z_ref)))


def test_eta_bar_zero_is_the_oracles_jacobi(porous8):
    w, P, s = porous8
    s.precond_build(blocks="element", eta_bar=0.0)
    assert s.info["n_blocks"] == 0 and s.info["n_jacobi"] == P.nfree
    P.precond_build(2)
    r = I.random_vector(303, s.n)
    z = s.apply_S(_lat(r)).cpu().numpy()[P.free_lat]
    z_ref = P.apply_S(r[P.free_lat])
    assert np.abs(z - z_ref).max() <= 1e-13 * np.abs(z_ref).max()


@pytest.mark.parametrize("eta_bar", [0.65, 0.999, 1.0])
def test_element_blocks_apply_S_matches_oracle(porous8, eta_bar):
    w, P, s = porous8
    s.precond_build(blocks="element", eta_bar=eta_bar)
    nb = P.precond_build(3, 1e-13, eta_bar)
    assert s.info["n_blocks"] == nb
    if eta_bar == 1.0:
        # every active cell is a block (Sec. 5.2): nothing is left to the diagonal part, and the
        # uncut interior cells share factors
        assert s.info["n_jacobi"] == 0 and s.info["n_factors"] < nb
    else:
        assert s.info["n_jacobi"] > 0
    r = I.random_vector(404, s.n)
    z = s.apply_S(_lat(r)).cpu().numpy()[P.free_lat]
    z_ref = P.apply_S(r[P.free_lat])
    assert _energy_rel(P, z, z_ref) < 1e-9


def test_element_blocks_pcg_matches_oracle(porous8):
    w, P, s = porous8
    eta_bar = 0.65
    s.precond_build(blocks="element", eta_bar=eta_bar)
    P.precond_build(3, 1e-13, eta_bar)
    b = s.rhs()
    u, its, rel, st = s.pcg_solve(b, w.tol, 5000)
    assert st == 0 and rel <= w.tol
    _, its_ref, _ = P.pcg(tol=w.tol, maxit=5000)
    assert abs(its - its_ref) <= 2
    import scipy.sparse.linalg as spla
    x_ref = spla.spsolve(P.csr().tocsc(), P.rhs())
    assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6


def test_element_blocks_mixed_multi_rhs_and_coarse(porous8):
    w, P, s = porous8
    s.precond_build(blocks="element", eta_bar=0.65, precision="mixed")
    b = torch.cat([s.rhs(1), s.rhs(4)])
    n = s.n
    u, its, rel, st = s.pcg_solve(b, w.tol, 5000)
    assert st == 0
    for k in range(2):
        uk, _, _, stk = s.pcg_solve(b[k * n:(k + 1) * n].clone(), w.tol, 5000)
        assert stk == 0
        d = (u[k * n:(k + 1) * n] - uk).cpu().numpy()[P.free_lat]
        x = uk.cpu().numpy()[P.free_lat]
        K = P.csr()
        assert np.sqrt(abs(d @ (K @ d)) / (x @ (K @ x))) < 1e-7
    # the coarse-corrected flexible CG works on top of any Schwarz operator
    u2, its2, rel2, st2 = s.fpcg_solve(None, 0.0, s.rhs(), w.tol, 5000, coarse_iters=20)
    assert st2 == 0 and rel2 <= w.tol
