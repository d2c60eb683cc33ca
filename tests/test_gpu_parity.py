"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * K x: the element matrices of both sides integrate the same polynomials
    on the same octree leaves; they differ by rounding only, so entries agree
    to ~1e-13 of max|K_e| and K x to 1e-12 relative (max-norm).
  * S r: each block factor is a pseudo inverse computed by a different
    eigensolver.  Perturbation theory bounds the change of a pseudo inverse by
    ~ n eps_mach cond(A_B) ||F||; the comparison is made in the energy norm of
    K (directions with small eigenvalues, where S is large, weigh little),
    bounded by 1e-9, and per DOF by the sum of that perturbation over the
    blocks containing the DOF (tests/schwarz_bounds.py).
  * PCG: the relative energy-norm error against the oracle's dense solve
    (Eq. (15)) must be below 1e-6 (1e-8 where the tolerance allows), and the
    iteration count must equal the oracle's within 2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I
from schwarz_bounds import dof_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(w):
    from paper_1809_00828_gb300 import fcm
    return fcm.Solver(w)


def _lat(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def single():
    w = I.workload_single_void(0)
    P = O.Problem.from_workload(w)
    P.precond_build(0)
    s = _solver(w)
    s.precond_build()
    yield w, P, s
    s.close()


def test_rhs_and_free_dofs_match(single):
    w, P, s = single
    b = s.rhs().cpu().numpy()
    assert s.info["n_free"] == P.nfree == 1944
    nz = np.zeros(s.n, dtype=bool)
    nz[P.free_lat] = True
    assert not b[~nz].any()
    assert np.abs(b[P.free_lat] - P.rhs()).max() <= 1e-14 * np.abs(P.rhs()).max()


def test_apply_K_matches_oracle(single):
    w, P, s = single
    x = I.random_vector(101, s.n)
    y = s.apply_K(_lat(x)).cpu().numpy()
    y_ref = P.apply_K(x[P.free_lat])
    assert np.abs(y[P.free_lat] - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    mask = np.zeros(s.n, dtype=bool)
    mask[P.free_lat] = True
    assert not y[~mask].any()


def test_apply_S_matches_oracle(single):
    w, P, s = single
    r = I.random_vector(202, s.n)
    z = s.apply_S(_lat(r)).cpu().numpy()[P.free_lat]
    z_ref = P.apply_S(r[P.free_lat])
    K = P.csr()
    d = z - z_ref
    e_energy = np.sqrt(abs(d @ (K @ d)) / (z_ref @ (K @ z_ref)))
    assert e_energy < 1e-9
    # per DOF: the eigensolver perturbation of the blocks that contain it (tests/schwarz_bounds.py)
    assert np.all(np.abs(d) <= dof_bound(P, r[P.free_lat]))


def test_pcg_matches_oracle_and_dense_solve(single):
    w, P, s = single
    b = s.rhs()
    u, its, rel, st = s.pcg_solve(b, w.tol, 2000)
    x = u.cpu().numpy()[P.free_lat]
    x_dense = np.linalg.solve(P.csr().toarray(), P.rhs())
    assert rel <= w.tol
    assert P.energy_error(x_dense, x) < 1e-8
    _, its_ref, _ = P.pcg(tol=w.tol, maxit=2000)
    assert abs(its - its_ref) <= 2
    info = s.last_solve()
    assert info["status"] == 0 and info["true_relres"] < 1e-8


def test_pcg_host_buffers_match_device(single):
    w, P, s = single
    b = s.rhs()
    u_dev, its_d, _, _ = s.pcg_solve(b, w.tol, 2000)
    u_host, its_h, _ = s.pcg_solve_host(b.cpu().numpy(), w.tol, 2000)
    assert its_h == its_d
    assert np.array_equal(u_host, u_dev.cpu().numpy())


def test_solve_is_deterministic(single):
    w, P, s = single
    b = s.rhs()
    u1, i1, r1, _ = s.pcg_solve(b, w.tol, 2000)
    u2, i2, r2, _ = s.pcg_solve(b, w.tol, 2000)
    assert i1 == i2 and r1 == r2 and torch.equal(u1, u2)


def test_error_statuses(single):
    from paper_1809_00828_gb300 import fcm
    w, P, s = single
    b = s.rhs()
    bad = b.clone()
    bad[int(P.free_lat[5])] = float("nan")
    _, _, _, st = s.pcg_solve(bad, w.tol, 100, check=False)
    assert st == fcm.FCM_EINVAL
    u, its, rel, st = s.pcg_solve(b, w.tol, 3, check=False)
    assert st == fcm.FCM_ENOTCONV and its == 3 and rel > w.tol
    assert torch.isfinite(u).all() and u.abs().max() > 0
    fresh = _solver(w)
    _, _, _, st = fresh.pcg_solve(b, w.tol, 10, check=False)
    assert st == fcm.FCM_ESTATE
    fresh.close()


@pytest.mark.parametrize("p,n", [(1, (3, 2, 2)), (3, (2, 2, 3)), (4, (2, 1, 2))])
def test_apply_K_and_S_other_orders(p, n):
    g = I.random_sphere_voids(9, 3, 0.15, 0.3, octree_depth=2)
    w = I.Workload("orders", n, p, 1e-6, g, 1e-9, hi=(0.3 * n[0], 0.25 * n[1], 0.2 * n[2]))
    P = O.Problem.from_workload(w)
    P.precond_build(0)
    s = _solver(w)
    s.precond_build()
    x = I.random_vector(7 + p, s.n)
    y = s.apply_K(_lat(x)).cpu().numpy()[P.free_lat]
    y_ref = P.apply_K(x[P.free_lat])
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    z = s.apply_S(_lat(x)).cpu().numpy()[P.free_lat]
    z_ref = P.apply_S(x[P.free_lat])
    K = P.csr()
    d = z - z_ref
    assert np.sqrt(abs(d @ (K @ d)) / (z_ref @ (K @ z_ref))) < 1e-9
    u, its, rel, st = s.pcg_solve(s.rhs(), 1e-9, 3000)
    x_dense = np.linalg.solve(K.toarray(), P.rhs())
    assert P.energy_error(x_dense, u.cpu().numpy()[P.free_lat]) < 1e-7
    s.close()


@pytest.fixture(scope="module")
def porous8():
    # 8^3 cells, p=2, 40 voids, alpha 1e-10: a small member of the porous family
    w = I.workload_porous(12, 8, 2, 40, 1e-10, 3, 1e-8)
    P = O.Problem.from_workload(w)
    P.precond_build(0)
    x_ref, _, _ = P.pcg(tol=1e-12, maxit=5000)
    _, its_o, _ = P.pcg(tol=w.tol, maxit=5000)
    return w, P, x_ref, its_o


def test_porous_8_cells_iterations_and_energy_error(porous8):
    w, P, x_ref, its_o = porous8
    s = _solver(w)
    s.precond_build()
    u, its, rel, st = s.pcg_solve(s.rhs(), w.tol, 5000)
    assert abs(its - its_o) <= 2
    assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
    s.close()


def test_mixed_precision_factors_keep_energy_error_below_1e6(single):
    # FP32 block factors (FP64 for blocks with retained condition number > 1e7)
    w, P, s0 = single
    s = _solver(w)
    s.precond_build(precision="mixed")
    assert s.info["n_blocks_fp32"] > 0
    u, its, rel, st = s.pcg_solve(s.rhs(), w.tol, 2000)
    x_dense = np.linalg.solve(P.csr().toarray(), P.rhs())
    assert P.energy_error(x_dense, u.cpu().numpy()[P.free_lat]) < 1e-6
    _, its64, _, _ = s0.pcg_solve(s0.rhs(), w.tol, 2000)
    assert its <= its64 * 1.2 + 5
    s.close()


def test_mixed_precision_porous_8_cells(porous8):
    w, P, x_ref, _ = porous8
    s = _solver(w)
    s.precond_build(precision="mixed", cond_fp64=1e7)
    u, its, rel, st = s.pcg_solve(s.rhs(), w.tol, 5000)
    assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
    s.close()


def test_unit_strain_loads_match_oracle(single):
    w, P, s = single
    for k in range(1, 7):
        b = s.rhs(k).cpu().numpy()
        ref = P.load(k)
        assert np.abs(b[P.free_lat] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_multi_rhs_solve_matches_separate_solves(single):
    # six unit-strain load cases in one call: the recurrences share every Schwarz launch
    w, P, s = single
    B = torch.cat([s.rhs(k) for k in range(1, 7)])
    U, its, rel, st = s.pcg_solve(B, 1e-10, 3000)
    K = P.csr().toarray()
    its_each = []
    for k in range(6):
        u1, i1, r1, _ = s.pcg_solve(s.rhs(k + 1), 1e-10, 3000)
        its_each.append(i1)
        uk = U[k * s.n:(k + 1) * s.n]
        assert torch.allclose(uk, u1, rtol=0, atol=1e-12 * float(u1.abs().max()))
        x_dense = np.linalg.solve(K, P.load(k + 1))
        assert P.energy_error(x_dense, uk.cpu().numpy()[P.free_lat]) < 1e-8
    assert its == max(its_each) and rel <= 1e-10


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_launch_shapes_leave_S_unchanged(precision):
    # p = 3 porous cube: cut patches stream their own factors in row tiles (FP32 and double-float in the
    # mixed build), uncut patches go through the shared-factor product; the tile size and the stream
    # arrangement that the build picks by timing must not change S r by a bit
    w = I.workload_porous(11, 6, 3, 10, 1e-10, 3, 1e-8)
    s = _solver(w)
    x = _lat(I.random_vector(5, s.n))
    # a low threshold sends this cube's cut-patch factors with cond > 1e3 to double-float storage
    cond = 1e3 if precision == "mixed" else 1e7
    s.precond_build(precision=precision, autotune=False, cond_fp64=cond)
    z0 = s.apply_S(x).clone()
    info0 = s.get_info()
    assert info0["n_gemm_blocks"] > 0 and info0["n_gemm_blocks"] < info0["n_blocks"]
    if precision == "mixed":
        assert info0["n_factors_ff"] > 0
    s.precond_build(precision=precision, cond_fp64=cond)
    z1 = s.apply_S(x)
    info1 = s.get_info()
    assert torch.equal(z0, z1)
    assert info0["tune_seconds"] == [0.0] * 8 and sum(t > 0 for t in info1["tune_seconds"]) >= 2
    assert info0["device_error"] == 0 and info1["device_error"] == 0
    # the shared-factor products on a second stream, beside the streamed factors
    s.precond_build(precision=precision, launch="concurrent", cond_fp64=cond)
    info2 = s.get_info()
    assert info2["schwarz_concurrent"] == 1 and info0["schwarz_concurrent"] == 0
    z2 = s.apply_S(x)
    assert torch.equal(z0, z2) and s.get_info()["device_error"] == 0
    # and inside a solve, where the launches sit in the captured graph
    u1, its1, _, _ = s.pcg_solve(s.rhs(), w.tol, 5000)
    s.precond_build(precision=precision, launch="serial", cond_fp64=cond)
    u0, its0, _, _ = s.pcg_solve(s.rhs(), w.tol, 5000)
    assert its0 == its1 and torch.equal(u0, u1)
    s.close()


@pytest.mark.parametrize("p,n", [(1, (3, 2, 2)), (2, (4, 4, 4)), (3, (2, 2, 3)), (4, (2, 1, 2))])
def test_apply_K_double_float_matches_oracle(p, n):
    # K x in double-float arithmetic on the FP32 pipe: every contraction to ~2^-46, so the result agrees
    # with the oracle's FP64 K x to the same 1e-12 (max norm) as the FP64 kernels
    g = I.random_sphere_voids(9, 3, 0.15, 0.3, octree_depth=2)
    w = I.Workload("orders_ff", n, p, 1e-6, g, 1e-9, hi=(0.3 * n[0], 0.25 * n[1], 0.2 * n[2]))
    P = O.Problem.from_workload(w)
    s = _solver(w)
    s.set_k_precision("double_float")
    assert s.info["k_double_float"] == 1
    for seed in (7, 8):
        x = I.random_vector(seed + p, s.n)
        y = s.apply_K(_lat(x)).cpu().numpy()
        y_ref = P.apply_K(x[P.free_lat])
        assert np.abs(y[P.free_lat] - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
        mask = np.zeros(s.n, dtype=bool)
        mask[P.free_lat] = True
        assert not y[~mask].any()
    s.close()


def test_pcg_with_double_float_K(porous8):
    w, P, x_ref, its_o = porous8
    s = _solver(w)
    s.set_k_precision("double_float")
    s.precond_build()
    u, its, rel, st = s.pcg_solve(s.rhs(), w.tol, 5000)
    assert abs(its - its_o) <= 2
    assert P.energy_error(x_ref, u.cpu().numpy()[P.free_lat]) < 1e-6
    # back to FP64 K: the graphs are captured again
    s.set_k_precision("fp64")
    u2, its2, _, _ = s.pcg_solve(s.rhs(), w.tol, 5000)
    assert abs(its2 - its_o) <= 2 and s.get_info()["k_double_float"] == 0
    s.close()
