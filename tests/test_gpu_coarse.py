"""GPU tests of the Galerkin coarse operator K_H = P^T K P and the flexible PCG that
uses it as the coarse part of the preconditioner.

K_H is checked against the product P^T K P formed here from the oracle's assembled
stiffness (scipy sparse) and an explicit P (1/8 at the 8 vertex DOFs of each cell,
free DOFs only).  The grid has more than 5 cells per axis, so the 5-periodic probing
that assembles K_H on the device is exercised with cells of one class that are
5 apart.  The device stores K_H in FP32 and accumulates in FP32: products agree to
~1e-6 of the largest entry; the bound leaves a factor 10 or more.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _prolongation(w, p, free_lat):
    """Explicit P: cell value (component-major) -> lattice DOFs, restricted to the free DOFs."""
    nx, ny, nz = w.n
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


@pytest.fixture(scope="module")
def porous8():
    from paper_1809_00828_gb300 import fcm
    w = I.workload_porous(5, 8, 2, 6, 1e-8, 3, 1e-9)
    s = fcm.Solver(w)
    s.precond_build()
    P = O.Problem.from_workload(w)
    yield w, s, P
    s.close()


def test_coarse_operator_is_the_galerkin_product(porous8):
    w, s, P = porous8
    K = P.csr()
    Pf = _prolongation(w, w.p, P.free_lat)
    KH = (Pf.T @ K @ Pf).tocsr()
    nc = int(np.prod(w.n))
    rng = np.random.default_rng(3)
    for trial in range(3):
        x = rng.standard_normal(3 * nc).astype(np.float32)
        if trial == 2:  # a single cell: one column of K_H
            x[:] = 0.0
            x[1 * nc + 37] = 1.0
        y = s.coarse_apply(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
        ref = KH @ x.astype(np.float64)
        assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()
    # symmetric positive semi-definite, as P^T K P must be
    a = rng.standard_normal(3 * nc).astype(np.float32)
    b = rng.standard_normal(3 * nc).astype(np.float32)
    ya = s.coarse_apply(torch.from_numpy(a).cuda()).cpu().numpy().astype(np.float64)
    yb = s.coarse_apply(torch.from_numpy(b).cuda()).cpu().numpy().astype(np.float64)
    assert abs(b @ ya - a @ yb) <= 1e-5 * max(abs(b @ ya), 1e-30)
    assert a @ ya > 0.0


def test_fpcg_with_coarse_cg_converges_faster_than_pcg(porous8):
    w, s, P = porous8
    b = s.rhs()
    _, its_pcg, _, _ = s.pcg_solve(b, w.tol, 4000)
    u, its, rel, st = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=20)
    info = s.last_solve()
    assert st == 0 and rel <= w.tol and info["fallback"] == 0
    assert its < its_pcg
    x_ref = spla.spsolve(P.csr().tocsc(), P.rhs())
    assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6


def test_fpcg_network_start_plus_coarse_cg(porous8):
    from paper_1809_00828_gb300 import fcm
    w, s, P = porous8
    net = fcm.UNet(in_ch=4, out_ch=3, base=4, levels=2, seed=9)
    b = s.rhs()
    u, its, rel, st = s.fpcg_solve(net, 0.1, b, w.tol, 4000, coarse_iters=5)
    assert st == 0 and rel <= w.tol * 1.0001
    x_ref = spla.spsolve(P.csr().tocsc(), P.rhs())
    assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
    net.close()
    # a second network of another depth: the solver's captured iteration must be rebuilt for it
    net2 = fcm.UNet(in_ch=4, out_ch=3, base=3, levels=3, seed=10)
    u2, its2, rel2, st2 = s.fpcg_solve(net2, 1.0, b, w.tol, 4000, coarse_iters=5)
    assert st2 == 0 and rel2 <= w.tol * 1.0001
    assert P.energy_error(x_ref, u2.cpu().numpy()[P.free_lat]) < 1e-6
    net2.close()
    # and back to no network, same coarse steps
    u3, its3, rel3, st3 = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=5)
    assert st3 == 0 and P.energy_error(x_ref, u3.cpu().numpy()[P.free_lat]) < 1e-6


def test_fpcg_after_the_preconditioner_is_rebuilt(porous8):
    # the flexible CG iteration is captured once and reused; rebuilding the Schwarz blocks
    # (new factor pools and plan) must make the next solve capture it again
    w, s, P = porous8
    b = s.rhs()
    x_ref = spla.spsolve(P.csr().tocsc(), P.rhs())
    _, its0, _, st0 = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=5)
    assert st0 == 0
    for prec in ("mixed", "fp64"):
        s.precond_build(precision=prec)
        u, its, rel, st = s.fpcg_solve(None, 0.0, b, w.tol, 4000, coarse_iters=5)
        assert st == 0 and rel <= w.tol * 1.0001
        assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
    assert its == its0


def test_fpcg_rejects_no_network_and_no_coarse_steps(porous8):
    from paper_1809_00828_gb300 import fcm
    w, s, P = porous8
    b = s.rhs()
    _, _, _, st = s.fpcg_solve(None, 0.0, b, w.tol, 10, check=False)
    assert st == fcm.FCM_EINVAL
