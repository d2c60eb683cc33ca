"""GPU tests of the learned coarse correction: U-Net kernels against the numpy oracle,
Adam against its formula, restriction/prolongation adjointness, and the flexible PCG.

Tolerances: the GPU accumulates in FP32 (weights in BF16, as the oracle models), so
forward outputs agree to ~1e-5 relative and gradients, sums over up to 8^3 x 2
voxels, to ~1e-4; the bounds below leave a factor 10.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import unet_oracle as U
from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


# the last case is the network of the learned correction's workload (4 levels, channels 16/32/64/64):
# its inner levels have Cin = 32, 64 and 128 (decoder concatenation), beyond one 16-channel chunk of
# the conv kernels' input loop
@pytest.mark.parametrize("levels,base,shape", [(3, 4, (8, 8, 8)), (2, 3, (4, 6, 2)), (1, 2, (3, 2, 5)),
                                               (4, 16, (16, 16, 16))])
def test_unet_forward_backward_match_oracle(levels, base, shape):
    from paper_1809_00828_gb300 import fcm
    net = fcm.UNet(in_ch=4, out_ch=3, base=base, levels=levels, seed=7)
    rng = np.random.default_rng(11)
    Z, Y, X = shape
    x = rng.standard_normal((2, 4, Z, Y, X)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    out = net.forward(xt).cpu().numpy()
    ref = U.UNetOracle(net.get(), 4, 3, base, levels)
    out_ref = ref.forward(x.astype(np.float64))
    assert _rel(out, out_ref) < 1e-4
    gout = rng.standard_normal(out.shape).astype(np.float32)
    net.zero_grad()
    din = net.backward(torch.from_numpy(gout).cuda(), want_din=True).cpu().numpy()
    _, g = net.get(with_grad=True)
    din_ref, g_ref = ref.backward(gout.astype(np.float64))
    assert _rel(din, din_ref) < 1e-3
    assert _rel(g, g_ref) < 1e-3
    net.close()


def test_adam_step_matches_formula():
    from paper_1809_00828_gb300 import fcm
    net = fcm.UNet(in_ch=4, out_ch=3, base=2, levels=2, seed=3)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((1, 4, 4, 4, 4)).astype(np.float32)).cuda()
    out = net.forward(x)
    net.zero_grad()
    net.backward(torch.ones_like(out))
    w0, g = net.get(with_grad=True)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    net.adam(lr, 1, b1, b2, eps)
    w1 = net.get()
    m = (1 - b1) * g.astype(np.float64)
    v = (1 - b2) * g.astype(np.float64) ** 2
    want = w0 - lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps)
    assert np.abs(w1 - want).max() < 1e-5 * max(1.0, np.abs(w0).max())
    net.close()


@pytest.fixture(scope="module")
def single():
    from paper_1809_00828_gb300 import fcm
    w = I.workload_single_void(0)
    s = fcm.Solver(w)
    s.precond_build()
    P = O.Problem.from_workload(w)
    yield w, s, P
    s.close()


def test_restriction_and_prolongation_are_adjoint(single):
    w, s, P = single
    nc = 4 * 4 * 4
    v = torch.from_numpy(I.random_vector(5, s.n)).cuda()
    c = torch.from_numpy(I.random_vector(6, 3 * nc).astype(np.float32)).cuda()
    Rv = s.coarse_restrict(v, 1.0, eta_channel=True)
    Pc = s.coarse_prolong(c, 1.0)
    mask = np.zeros(s.n, dtype=bool)
    mask[P.free_lat] = True
    vm = v.cpu().numpy() * mask
    lhs = float(np.dot(Rv[: 3 * nc].cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)))
    rhs = float(np.dot(vm, Pc.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1e-12)
    # the 4th channel is eta_T, which the oracle integrates independently
    assert np.allclose(Rv[3 * nc:].cpu().numpy(), P.eta(), atol=1e-6)
    # prolongation of a unit cell value reaches exactly the free vertex DOFs of that cell
    e = torch.zeros(3 * nc, dtype=torch.float32, device="cuda")
    e[0 * nc + 21] = 8.0
    y = s.coarse_prolong(e, 1.0).cpu().numpy()
    assert set(np.nonzero(y)[0]) <= set(P.free_lat) and np.allclose(y[np.nonzero(y)], 1.0)


def test_fpcg_with_zero_correction_reproduces_pcg(single):
    from paper_1809_00828_gb300 import fcm
    w, s, P = single
    net = fcm.UNet(in_ch=4, out_ch=3, base=4, levels=3, seed=1)
    b = s.rhs()
    u0, its0, _, _ = s.pcg_solve(b, w.tol, 2000)
    u1, its1, rel1, st = s.fpcg_solve(net, 0.0, b, w.tol, 2000)
    assert st == fcm.FCM_OK and rel1 <= w.tol
    assert abs(its1 - its0) <= 2
    x_dense = np.linalg.solve(P.csr().toarray(), P.rhs())
    assert P.energy_error(x_dense, u1.cpu().numpy()[P.free_lat]) < 1e-8
    info = s.last_solve()
    assert info["fallback"] == 0 and info["flexible_iterations"] == its1
    net.close()


def test_fpcg_falls_back_to_plain_pcg_on_a_harmful_correction(single):
    from paper_1809_00828_gb300 import fcm
    w, s, P = single
    net = fcm.UNet(in_ch=4, out_ch=3, base=4, levels=3, seed=2)
    b = s.rhs()
    u, its, rel, st = s.fpcg_solve(net, -1e9, b, w.tol, 4000)
    info = s.last_solve()
    x_dense = np.linalg.solve(P.csr().toarray(), P.rhs())
    assert st == fcm.FCM_OK and rel <= w.tol * 1.0001
    assert P.energy_error(x_dense, u.cpu().numpy()[P.free_lat]) < 1e-7
    assert info["true_relres"] < 1e-7
    net.close()
