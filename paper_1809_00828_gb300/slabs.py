"""Slab decomposition of the Schwarz-PCG over ranks (one process per GPU).

The distributed-memory design of Jomo et al. (Sec. 4.2: each process owns a part of the mesh plus
ghost layers, so that the rows of K and the Schwarz blocks of its part need no set-up
communication; Sec. 5.3.3 scales it to many nodes) restated for a Cartesian grid split along z:

* rank r owns the cells with z in [cz0, cz1) (cz_r = r nz / world) and the lattice node planes
  [p cz0, p cz1) (the last rank also the top plane); a DOF belongs to the rank owning its plane;
* its local vectors cover planes [p (cz0 - 1), p cz1] (clipped): the owned planes, p ghost planes
  below and one above -- every column of the K rows of owned DOFs (cells cz0 - 1 .. cz1 - 1);
* it applies the vertex-patch blocks of the vertices on its owned planes (v_z in [cz0, cz1), the
  last rank also nz); their boxes reach p - 1 planes below the owned range, whose contributions
  belong to rank r - 1;
* per PCG iteration: one forward halo exchange of p before K (1 plane down, p planes up), one of r
  before S, one reverse addition of the S contributions on the ghost planes below, and two
  all-reduces of partial dot products (p.q; r.z with z.z), as in the plain PCG of Sec. 5 with the
  stopping rule ||S r|| / ||S b|| <= tol (Eq. 14).

The operators are callables supplied by the caller (local K rows and local blocks), so the same
driver runs on CPU ranks (gloo) and on GPU ranks (NCCL, tensors on the device).  Vectors are 1-D
torch tensors in the local lattice layout (3 components interleaved, node index x fastest).
"""
from __future__ import annotations

import math


class SlabPlan:
    """Ownership and halo planes of rank `rank` of `world` for a grid of n = (nx, ny, nz) cells of
    order p.  Needs nz >= world (every rank owns at least one cell layer, i.e. p node planes)."""

    def __init__(self, n, p, rank, world):
        if n[2] < world:
            raise ValueError(f"{n[2]} cell layers cannot be split over {world} ranks")
        self.n, self.p, self.rank, self.world = tuple(n), p, rank, world
        M = [p * n[a] + 1 for a in range(3)]
        self.M = M
        self.plane = 3 * M[0] * M[1]  # DOFs per node plane
        cz = [(r * n[2]) // world for r in range(world + 1)]
        self.cz0, self.cz1 = cz[rank], cz[rank + 1]
        self.own_lo = p * self.cz0
        self.own_hi = p * self.cz1 if rank < world - 1 else M[2]
        self.lo = p * (self.cz0 - 1) if rank > 0 else 0
        self.hi = p * self.cz1 + 1 if rank < world - 1 else M[2]
        # vertex planes whose patches this rank applies
        self.v_lo = self.cz0
        self.v_hi = self.cz1 if rank < world - 1 else n[2] + 1

    @property
    def size(self):
        """Length of a local vector."""
        return (self.hi - self.lo) * self.plane

    def owned(self, v):
        """The owned part of local vector v (a view)."""
        return v[(self.own_lo - self.lo) * self.plane:(self.own_hi - self.lo) * self.plane]

    def planes(self, v, a, b):
        """Planes [a, b) (global plane indices) of local vector v (a view)."""
        return v[(a - self.lo) * self.plane:(b - self.lo) * self.plane]

    def global_index(self, local):
        """Global lattice index of local index `local`."""
        return local + self.lo * self.plane

    def owns_vertex(self, vz):
        return self.v_lo <= vz < self.v_hi


def exchange_halo(plan, v, dist):
    """Fill the ghost planes of local vector v from the neighbours' owned planes: rank r - 1 needs
    plane own_lo of rank r (its ghost above), rank r + 1 the top p owned planes of rank r (its
    ghosts below)."""
    reqs = []
    r, W, p = plan.rank, plan.world, plan.p
    if r > 0:
        reqs.append(dist.isend(plan.planes(v, plan.own_lo, plan.own_lo + 1).contiguous(), r - 1))
        below = v.new_empty((plan.own_lo - plan.lo) * plan.plane)
        reqs.append(dist.irecv(below, r - 1))
    if r < W - 1:
        reqs.append(dist.isend(plan.planes(v, plan.own_hi - p, plan.own_hi).contiguous(), r + 1))
        above = v.new_empty((plan.hi - plan.own_hi) * plan.plane)
        reqs.append(dist.irecv(above, r + 1))
    for q in reqs:
        q.wait()
    if r > 0:
        plan.planes(v, plan.lo, plan.own_lo).copy_(below)
    if r < W - 1:
        plan.planes(v, plan.own_hi, plan.hi).copy_(above)


def reverse_add(plan, z, dist):
    """Add the contributions that the local blocks put on the ghost planes below to their owner
    (rank r - 1, its top p owned planes), and receive rank r + 1's onto ours; ghost planes are
    then cleared."""
    reqs = []
    r, W, p = plan.rank, plan.world, plan.p
    if r > 0:
        reqs.append(dist.isend(plan.planes(z, plan.lo, plan.own_lo).contiguous(), r - 1))
    if r < W - 1:
        got = z.new_empty(p * plan.plane)
        reqs.append(dist.irecv(got, r + 1))
    for q in reqs:
        q.wait()
    if r < W - 1:
        plan.planes(z, plan.own_hi - p, plan.own_hi).add_(got)
    plan.planes(z, plan.lo, plan.own_lo).zero_()
    plan.planes(z, plan.own_hi, plan.hi).zero_()


def _allreduce(vals, dist, like):
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=like.device)
    dist.all_reduce(t)
    return t.tolist()


def distributed_pcg(plan, apply_K_local, apply_S_local, b, dist, tol, maxit):
    """Plain Schwarz-PCG over the slab ranks; x0 = 0.

    apply_K_local(x) -> y: y (local vector) holds K x on the owned DOFs (ghost planes of x current);
    apply_S_local(r) -> z: z holds the contributions of this rank's blocks on owned and ghost-below
    planes (ghost planes of r current).  b: local vector, owned part set.  Returns (x, iterations,
    relative preconditioned residuals ||S r_i|| / ||S b||).
    """
    def dot(a, c):
        return float((plan.owned(a) * plan.owned(c)).sum())

    x = b.new_zeros(plan.size)
    r = b.clone()
    plan.planes(r, plan.lo, plan.own_lo).zero_()
    plan.planes(r, plan.own_hi, plan.hi).zero_()

    def precond(rv):
        exchange_halo(plan, rv, dist)
        z = apply_S_local(rv)
        reverse_add(plan, z, dist)
        return z

    z = precond(r)
    rz, zz0 = _allreduce([dot(r, z), dot(z, z)], dist, b)
    hist = [1.0]
    if zz0 == 0.0:
        return x, 0, hist
    pv = z.clone()
    it = 0
    while it < maxit:
        exchange_halo(plan, pv, dist)
        q = apply_K_local(pv)
        (pq,) = _allreduce([dot(pv, q)], dist, b)
        if not (pq > 0.0) or not math.isfinite(rz / pq):
            raise FloatingPointError("CG breakdown: p.Kp <= 0 or a non-finite scalar")
        alpha = rz / pq
        plan.owned(x).add_(plan.owned(pv), alpha=alpha)
        plan.owned(r).add_(plan.owned(q), alpha=-alpha)
        z = precond(r)
        rz_new, zz = _allreduce([dot(r, z), dot(z, z)], dist, b)
        it += 1
        rel = math.sqrt(zz / zz0)
        hist.append(rel)
        if rel <= tol:
            break
        beta = rz_new / rz
        rz = rz_new
        pv = z + beta * pv
        plan.planes(pv, plan.lo, plan.own_lo).zero_()
        plan.planes(pv, plan.own_hi, plan.hi).zero_()
    return x, it, hist
