"""Failure detection on the GPU without a fault: the statuses FCM_ETIMEOUT and FCM_EBREAKDOWN.

FCM_ETIMEOUT: the shared-factor product waits for bulk copies of the factor on mbarriers, a bounded
number of polls.  fcm_set_wait_limit(ctx, 0) makes the first poll give up: the CTA marks the apply
as failed, lets the copies already in flight land and returns, the GPU stays usable, and the solve
returns FCM_ETIMEOUT.  Restoring the default limit gives a normal solve again.

FCM_EBREAKDOWN: a right-hand side made on the host, b = c e_l with c^2 finite but c^2 S_ll beyond
the FP64 range, so r.z (or p.Kp) overflows in the first iteration and alpha is not finite.  The
overflow is checked on the oracle's S first.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_wait_limit_zero_gives_timeout_status_and_the_context_recovers():
    from paper_1809_00828_gb300 import fcm
    # an uncut 6^3 cube: the interior patches share one factor (dense product with bulk-copy waits)
    w = I.Workload("uncut6", (6, 6, 6), 2, 1.0, I.uncut(), 1e-8)
    s = fcm.Solver(w)
    s.precond_build()
    assert s.info["n_gemm_blocks"] > 0
    b = s.rhs()
    u_ref, its_ref, _, st = s.pcg_solve(b, w.tol, 2000)
    assert st == fcm.FCM_OK
    s.set_wait_limit(0)
    _, _, _, st = s.pcg_solve(b, w.tol, 2000, check=False)
    assert st == fcm.FCM_ETIMEOUT
    assert s.last_solve()["status"] == fcm.FCM_ETIMEOUT
    z = s.apply_S(b)
    torch.cuda.synchronize()
    assert s.get_info()["device_error"] == 1
    s.set_wait_limit(-1)
    u, its, _, st = s.pcg_solve(b, w.tol, 2000)
    assert st == fcm.FCM_OK and its == its_ref and torch.equal(u, u_ref)
    assert s.get_info()["device_error"] == 0
    s.close()


def test_overflowing_rhs_gives_breakdown_status():
    from paper_1809_00828_gb300 import fcm
    w = I.workload_single_void(0)
    P = O.Problem.from_workload(w)
    P.precond_build(0)
    s = fcm.Solver(w)
    s.precond_build()
    # the free DOF with the largest diagonal entry of S
    diag = np.zeros(P.nfree)
    for bidx in range(P.nblocks()):
        idx, F, _ = P.block(bidx)
        diag[idx] += np.diag(F)
    l = int(np.argmax(diag))
    c = 1.2e154
    # ||b||^2 = c^2 finite, b.Sb = c^2 S_ll beyond the FP64 range (1.8e308) by a wide margin
    assert np.isfinite(c * c) and 2 * np.log10(c) + np.log10(diag[l]) > 309.5
    b = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    b[int(P.free_lat[l])] = c
    _, its, _, st = s.pcg_solve(b, 1e-8, 100, check=False)
    assert st == fcm.FCM_EBREAKDOWN and its <= 1
    # the context stays usable
    _, _, rel, st = s.pcg_solve(s.rhs(), w.tol, 2000)
    assert st == fcm.FCM_OK and rel <= w.tol
    s.close()
