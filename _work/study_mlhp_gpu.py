"""Timing of the multi-level GPU path on the Sec. 5.1 cube (8^3 base cells, p = 3, cavity r = 0.01 at the
centre, refined k times toward its surface, alpha = 1e-8, truncated blocks).

Not a test: run it on a GPU with `python tests/study_mlhp_gpu.py [k ...]` (default 0 1 2 3).  For each k it
prints one JSON
line: host set-up times, the device K and S applies (CUDA events on the plan's stream, median of 20 after 3
warm-ups) with their algorithmic bytes and bandwidth, and the PCG solve (tol 1e-8).  Algorithmic bytes:
K x reads 12 B per CSR nonzero (value and column) plus the row pointers and writes y; S r reads every
factor entry once (8 B) plus the gathers and the read-modify-write of z on the block DOFs.
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch  # noqa: E402

from paper_1809_00828_gb300 import fcm  # noqa: E402


def timed(fn, reps=20, warm=3):
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    return float(np.median(ts))


def run(k):
    t0 = time.time()
    P = fcm.MLHPPlan((8, 8, 8), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.01)], 3, k, octree_depth=3)
    free, K, b, eta = P.assemble(1e-8, "clamp")
    t1 = time.time()
    blocks, F, cptr, jac = P.factorize("truncated")
    t2 = time.time()
    P.device_setup()
    n = len(free)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(n)).cuda()
    y = torch.empty_like(x)
    tk = timed(lambda: P.apply_K(x, y))
    ts = timed(lambda: P.apply_S(x, y))
    bk = 12 * K.nnz + 8 * (n + 1) + 16 * n
    nb_dofs = sum(len(B) for B in blocks)
    bs = 8 * sum(len(B) ** 2 for B in blocks) + 4 * nb_dofs + 8 * nb_dofs * 3 + 24 * n
    bd = torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    t3 = time.time()
    u, its, rel, st = P.pcg_solve(bd, 1e-8, 20000, check=False)
    torch.cuda.synchronize()
    t4 = time.time()
    line = {"k": k, "dofs": n, "nnz": int(K.nnz), "blocks": len(blocks), "colours": len(cptr) - 1,
            "assemble_s": round(t1 - t0, 2), "factorize_s": round(t2 - t1, 2),
            "apply_K_ms": round(tk * 1e3, 4), "apply_K_GBs": round(bk / tk * 1e-9, 1),
            "apply_S_ms": round(ts * 1e3, 4), "apply_S_GBs": round(bs / ts * 1e-9, 1),
            "pcg_iterations": its, "pcg_status": st, "pcg_s": round(t4 - t3, 4)}
    print(json.dumps(line), flush=True)
    P.close()


if __name__ == "__main__":
    for k in [int(a) for a in sys.argv[1:]] or [0, 1, 2, 3]:
        run(k)
