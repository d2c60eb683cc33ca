"""Per-DOF bounds for comparing a Schwarz apply z = S r against the oracle's.

The two sides compute each block's pseudo inverse with different eigensolvers
(cuSOLVER on the GPU, cyclic Jacobi in the oracle).  A backward-stable
eigensolver returns the exact eigen-decomposition of A_B + dA with
||dA|| <= c n eps ||A_B||; when the retained eigenvalue set is the same, the
pseudo inverse then moves by F dA F, so ||dF|| <= c n eps cond(A_B) ||F||
(cond over the retained spectrum, ||F|| ||A_B|| = cond).  Forming
V diag(1/lambda) V^T and applying F add n eps ||F|| more.  A DOF l receives
the contributions of the blocks that contain it, so

    |z_l - z_ref,l| <= sum_{B contains l} (c n eps (cond_B + 1) ||F_B||_2 + u_F ||F_B||_2) ||r_B||_2,

with u_F the storage rounding of the factor (2^-24 for FP32 factors, 0 for
FP64) and c a small constant (10 below).  Ill-conditioned blocks loosen the
bound only on their own DOFs.
"""
import numpy as np

EPS64 = 2.0 ** -52


def dof_bound(P, r_free, c=10.0, u_factor=0.0):
    """Bound per free DOF of the oracle problem P (its blocks must be built) for input r_free."""
    bound = np.zeros(P.nfree)
    for b in range(P.nblocks()):
        idx, F, info = P.block(b)
        n = len(idx)
        if n == 0:
            continue
        cond = info[0] if np.isfinite(info[0]) else 1e300
        fn = np.linalg.norm(F, 2)
        rn = np.linalg.norm(r_free[idx])
        bound[idx] += (c * n * EPS64 * (cond + 1.0) + u_factor) * fn * rn
    return bound
