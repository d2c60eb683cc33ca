"""Slab decomposition of the Schwarz-PCG (Sec. 4.2 ghost layers, Sec. 5.3.3 distributed scaling) on
CPU ranks: two to four gloo processes run the partitioned PCG of paper_1809_00828_gb300/slabs.py with the
oracle's operators cut to each slab (the K rows of the owned DOFs, the vertex-patch blocks of the
owned vertices) and reproduce the single-domain oracle PCG: the same iteration count, the same first
residual history steps and the same solution, up to the order of the summations.

Only the host logic is tested here: one GPU per run, so no NCCL rank runs on hardware.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1809_00828_gb300 import inputs as I  # noqa: E402
from paper_1809_00828_gb300.slabs import SlabPlan  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(name):
    if name == "single_void":
        return I.workload_single_void(0)
    return I.workload_porous(12, 4, 2, 8, 1e-10, 3, 1e-8)


def _slab_operators(P, w, plan):
    """The oracle's K rows and blocks, restricted to one slab, as functions of local vectors."""
    import scipy.sparse as sp
    p = w.p
    lo = plan.lo * plan.plane
    free_lat = np.asarray(P.free_lat)
    node = free_lat // 3
    ijk = np.stack([node % plan.M[0], (node // plan.M[0]) % plan.M[1], node // (plan.M[0] * plan.M[1])], 1)
    own = (ijk[:, 2] >= plan.own_lo) & (ijk[:, 2] < plan.own_hi)
    K = P.csr()
    rows = np.nonzero(own)[0]
    Kown = K[rows, :].tocoo()
    cols_local = free_lat[Kown.col] - lo
    assert cols_local.min() >= 0 and cols_local.max() < plan.size, "K row reaches beyond the ghost planes"
    Kloc = sp.csr_matrix((Kown.data, (Kown.row, cols_local)), shape=(len(rows), plan.size))
    rows_local = free_lat[rows] - lo
    # vertex-patch blocks in the oracle's order (vertices z, y, x; empty patches skipped)
    blocks = []
    b = 0
    for vz in range(w.n[2] + 1):
        inz = np.abs(ijk[:, 2] - p * vz) <= p - 1
        for vy in range(w.n[1] + 1):
            iny = inz & (np.abs(ijk[:, 1] - p * vy) <= p - 1)
            for vx in range(w.n[0] + 1):
                members = np.nonzero(iny & (np.abs(ijk[:, 0] - p * vx) <= p - 1))[0]
                if members.size == 0:
                    continue
                idx, F, _ = P.block(b)
                assert np.array_equal(np.sort(idx), members)
                b += 1
                if plan.owns_vertex(vz):
                    loc = free_lat[idx] - lo
                    assert loc.min() >= 0 and loc.max() < plan.size, "block reaches beyond the ghost planes"
                    blocks.append((loc, F))
    assert b == P.nblocks()

    def apply_K(x):
        y = np.zeros(plan.size)
        y[rows_local] = Kloc @ x.numpy()
        return torch.from_numpy(y)

    def apply_S(r):
        rn = r.numpy()
        z = np.zeros(plan.size)
        for loc, F in blocks:
            z[loc] += F @ rn[loc]
        return torch.from_numpy(z)

    return apply_K, apply_S, rows_local, rows


def _worker(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_1809_00828_gb300 import slabs
        w = _workload(name)
        P = O.Problem.from_workload(w)
        P.precond_build(0)
        plan = SlabPlan(w.n, w.p, rank, world)
        apply_K, apply_S, rows_local, rows = _slab_operators(P, w, plan)
        b = np.zeros(plan.size)
        b[rows_local] = P.rhs()[rows]
        x, its, hist = slabs.distributed_pcg(plan, apply_K, apply_S, torch.from_numpy(b), dist, w.tol, 5000)
        x_ref, its_ref, hist_ref = P.pcg(tol=w.tol, maxit=5000)
        # the distributed solution, gathered over the ranks, in the energy norm of K (Eq. 15)
        xg = torch.zeros(P.nlat, dtype=torch.float64)
        xg[plan.own_lo * plan.plane:plan.own_hi * plan.plane] = plan.owned(x)
        dist.all_reduce(xg)
        e_energy = P.energy_error(x_ref, xg.numpy()[np.asarray(P.free_lat)])
        h, hr = np.asarray(hist), hist_ref[:len(hist)]
        # the first iterations agree to rounding; later the sums' different order (owned partial dots,
        # then an all-reduce) is amplified by CG's loss of orthogonality, as any reordering would be,
        # so the later history is compared loosely and the end point exactly
        out.put((rank, its, its_ref, float(np.abs(x.numpy()[rows_local] - x_ref[rows]).max()),
                 float(np.abs(x_ref).max()), float((np.abs(h - hr)[:8] / hr[:8]).max()),
                 float((np.abs(h - hr) / hr).max()), e_energy))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("single_void", 2), ("porous4", 2), ("porous4", 3), ("porous4", 4)])
def test_slab_ranks_reproduce_the_single_domain_pcg(name, world):
    # world 4 on 4 cell layers: every rank owns one layer, so every halo and reverse addition crosses ranks
    # (the plan test below covers the ghost planes of p = 1, 3 and 4)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, its, its_ref, dx, xmax, dh, dh_all, e_energy in res:
        assert its == its_ref, (rank, its, its_ref)
        assert e_energy <= 1e-9, (rank, e_energy)  # both iterates stop at ||S r|| / ||S b|| <= 1e-8
        assert dx <= 1e-8 * xmax, (rank, dx, xmax)
        assert dh <= 1e-10, (rank, dh)  # relative, the first 8 iterations
        assert dh_all <= 0.5, (rank, dh_all)


@pytest.mark.parametrize("nz,p,world", [(4, 2, 2), (5, 3, 2), (7, 1, 3), (8, 4, 4), (3, 2, 3)])
def test_slab_plan_owns_every_plane_and_vertex_once_and_covers_the_stencils(nz, p, world):
    n = (3, 2, nz)
    plans = [SlabPlan(n, p, r, world) for r in range(world)]
    M2 = p * nz + 1
    owner = np.zeros(M2, dtype=int)
    vown = np.zeros(nz + 1, dtype=int)
    for pl in plans:
        owner[pl.own_lo:pl.own_hi] += 1
        vown[pl.v_lo:pl.v_hi] += 1
        # the K rows of owned planes reach the cells touching them: planes [p (cz0 - 1), p cz1]
        assert pl.lo <= max(0, p * (pl.cz0 - 1)) and pl.hi >= min(M2, p * pl.cz1 + 1)
        # the boxes of owned vertices, [p v - (p - 1), p v + (p - 1)] clipped, stay inside the local planes
        for vz in range(pl.v_lo, pl.v_hi):
            assert pl.lo <= max(0, p * vz - (p - 1)) and min(M2 - 1, p * vz + (p - 1)) < pl.hi
        # ghost planes: owned by the neighbours
        assert pl.lo == (plans[pl.rank - 1].own_hi - p if pl.rank > 0 else 0)
    assert (owner == 1).all() and (vown == 1).all()
    with pytest.raises(ValueError):
        SlabPlan((2, 2, world - 1), p, 0, world)
