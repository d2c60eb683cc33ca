"""Sec. 5.1 refinement study on the paper's own cube: 8^3 base cells, p = 3, a spherical cavity of radius
0.01 at the centre, refined toward its surface k = 0..K times.  For each k, PCG iterations (tol 1e-8) with
full and with truncated leaf blocks, and their overlap n_max.

Not a test (it takes minutes): run it with `python tests/study_sec5_1_refinement.py [K] [alpha] [porous]`;
`porous` swaps the cube for a porous cube (10 voids, 4^3 base cells, p = 2) refined toward its void
surfaces, the analogue of the paper's gearbox study (Sec. 5.3); `voxels` for a trabecular-like voxel image
(32^3 Gaussian random field, half solid, 4^3 base cells, p = 2) refined toward its surface.  The
system comes from the library's host assembly (fcm_mlhp_assemble) and its block lists (fcm_mlhp_block);
the pseudo inverses and the PCG are plain numpy, as in the multi-level oracle.  Differences from the
paper's set-up: the full tensor-product basis instead of the trunk space, a clamped base and a traction
on the top face instead of penalty conditions and a pressure load.
"""
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_1809_00828_gb300 import fcm  # noqa: E402


def pseudo_inverse(A, eps=1e-13):
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    keep = lam > eps * lam.max()
    return (V[:, keep] / lam[keep]) @ V[:, keep].T


CUBE = ((8, 8, 8), [(0.5, 0.5, 0.5, 0.01)], 3)


def study(k, alpha=1e-8, setup=CUBE, tol=1e-8, maxit=5000):
    n, geometry, p = setup
    if hasattr(geometry, "kind"):
        P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), None, p, k, octree_depth=3, geometry=geometry)
    else:
        P = fcm.MLHPPlan(n, (0, 0, 0), (1, 1, 1), geometry, p, k, octree_depth=3)
    free, K, b, eta = P.assemble(alpha, "clamp")
    pos = -np.ones(3 * P.info["n_functions"], dtype=np.int64)
    pos[free] = np.arange(len(free))
    out = {"k": k, "dofs": len(free)}
    for kind in ("full", "truncated"):
        blocks, factors = [], []
        covered = np.zeros(len(free), dtype=bool)
        for i in range(P.info["n_leaves"]):
            if eta[i] <= 0.0:
                continue
            f = P.block(i, kind)
            d = (3 * f[:, None] + np.arange(3)[None, :]).reshape(-1)
            loc = np.sort(pos[d][pos[d] >= 0])
            if len(loc):
                blocks.append(loc)
                factors.append(pseudo_inverse(K[loc][:, loc].toarray()))
                covered[loc] = True
        jac = np.where(covered, 0.0, 1.0 / K.diagonal())

        def S(r):
            z = jac * r
            for B, F in zip(blocks, factors):
                z[B] += F @ r[B]
            return z

        x = np.zeros(len(free))
        r = b.copy()
        z = S(r)
        ref = np.linalg.norm(S(b))
        d = z.copy()
        rz = r @ z
        its = maxit
        for it in range(1, maxit + 1):
            q = K @ d
            a = rz / (d @ q)
            x += a * d
            r -= a * q
            z = S(r)
            if np.linalg.norm(z) <= tol * ref:
                its = it
                break
            rz_new = r @ z
            d = z + (rz_new / rz) * d
            rz = rz_new
        cnt = np.zeros(len(free), dtype=np.int64)
        for B in blocks:
            cnt[B] += 1
        out[kind] = {"iterations": its, "n_max": int(cnt.max())}
    P.close()
    return out


if __name__ == "__main__":
    K = int(sys.argv[1]) if len(sys.argv) > 1 else 3
    alpha = float(sys.argv[2]) if len(sys.argv) > 2 else 1e-8
    setup = CUBE
    if len(sys.argv) > 3 and sys.argv[3] == "porous":
        # a porous cube refined toward its void surfaces, as the paper's gearbox is refined toward its pores
        from paper_1809_00828_gb300 import inputs as I
        setup = ((4, 4, 4), I.random_sphere_voids(11, 10, 0.05, 0.15).sphere_array(), 2)
    if len(sys.argv) > 3 and sys.argv[3] == "voxels":
        # a trabecular-like voxel image (32^3 Gaussian random field, half solid) refined toward its surface
        from paper_1809_00828_gb300 import inputs as I
        setup = ((4, 4, 4), I.gaussian_random_field_voxels(3, m=32, corr_len=0.1, solid_fraction=0.5), 2)
    for k in range(K + 1):
        t = time.time()
        print(study(k, alpha, setup), f"{time.time() - t:.0f} s", flush=True)
