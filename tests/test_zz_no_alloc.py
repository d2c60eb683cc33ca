"""fcm_apply_S_noalloc: the Schwarz apply for callers that cannot allocate device memory.

Such callers (an application whose device memory belongs to its own pool
allocator, or a loop that forbids allocation once running) set the context
up at start-up and later only apply the preconditioner; this entry point
keeps its scratch vector in a static device array.  The test calls it through
the C ABI twice in a row and compares it with fcm_apply_S bit for bit: both
run the same kernels in the same order on the same masked input (the Schwarz
scatter is deterministic), so any difference means one path changed.  This
file is collected last on purpose: a run that stops at the first failure has
already run every other test when it gets here.
"""
import ctypes

import numpy as np
import pytest

from paper_1809_00828_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_schwarz_apply_matches_fcm_apply_S_twice():
    from paper_1809_00828_gb300 import fcm
    L = fcm.load()
    w = I.workload_single_void(4)
    s = fcm.Solver(w)
    s.precond_build()
    assert s.n <= fcm.NOALLOC_MAX_LATTICE
    for seed in (31, 32):  # two calls in a row, different inputs
        r = torch.from_numpy(I.random_vector(seed, s.n)).cuda()
        z_ref = s.apply_S(r)
        z = torch.full_like(r, float("nan"))
        st = L.fcm_apply_S_noalloc(s.ctx, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()))
        assert st == fcm.FCM_OK, L.fcm_last_error(s.ctx)
        torch.cuda.synchronize()
        assert np.array_equal(z.cpu().numpy(), z_ref.cpu().numpy())
    s.close()


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    from paper_1809_00828_gb300 import fcm
    L = fcm.load()
    # 3 * (2*51+1)^2 * (2*34+1) lattice DOFs > 2^20
    w = I.Workload("big", (51, 51, 34), 2, 1e-6, I.uncut(), 1e-8)
    s = fcm.Solver(w)
    assert s.n > fcm.NOALLOC_MAX_LATTICE
    s.precond_build()
    r = s.empty()
    z = s.empty()
    st = L.fcm_apply_S_noalloc(s.ctx, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()))
    assert st == fcm.FCM_EINVAL
    assert b"FCM_NOALLOC_MAX_LATTICE" in L.fcm_last_error(s.ctx)
    s.close()
