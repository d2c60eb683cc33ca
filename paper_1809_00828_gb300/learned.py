"""Training and use of the learned coarse correction (U-Net on the cell grid).

The paper's Additive-Schwarz preconditioner (Sec. 3) is local: it has no
coarse space, so the iteration count grows with the grid (Sec. 6 names this
limitation of the approach).  The learned correction adds a coarse term to
the preconditioner, used inside flexible PCG (fcm_fpcg_solve):

    z = S r + gamma * sigma * P N(R r / sigma, eta)

R averages a lattice vector to the cell grid (vertex nodes), P = R^T,
sigma = RMS of R r, eta the cell volume fractions, N the U-Net.

Training data are (residual, error) pairs of plain FP64 Schwarz-PCG runs on
seeded porous cubes: snapshots x_k of the iteration, r_k = b - K x_k,
e_k = x_ref - x_k.  The loss of one pair is the relative energy-norm error
left after adding the correction c to x_k:

    ||e_k - c||_K^2 / ||e_k||_K^2 = 1 + (c.Kc - 2 c.r_k) / (e_k.r_k),

which uses K e_k = r_k, so each step needs one K application per sample.
Its gradient with respect to the network output is
(2 gamma sigma / e_k.r_k) R (K c - r_k).

Everything that computes runs in libfcm's kernels (K, S, R, P, the U-Net
forward/backward and Adam); this module only orchestrates the calls and a
few vector differences and dot products of the training loop.
"""
from __future__ import annotations

import dataclasses
import math
import struct
import time

import numpy as np

from . import fcm, inputs

SNAPSHOTS = (3, 6, 12, 25, 50, 100, 200, 400)


@dataclasses.dataclass
class Sample:
    solver: "fcm.Solver"
    r: object            # lattice residual (cuda float64)
    cells: object        # R r (3 channels) + eta (1 channel), cuda float32, unnormalised
    sigma: float         # RMS of R r
    energy: float        # e.r = e^T K e
    ratio: float         # RMS(R e) / RMS(R r)


def training_workloads(seeds, n=32, p=2, count=40, alpha=1e-10, depth=3):
    return [inputs.workload_porous(s, n, p, count, alpha, depth, 1e-8) for s in seeds]


def generate(workloads, snapshots=SNAPSHOTS, tol_ref=1e-10, maxit=20000, log=print):
    """Plain FP64 Schwarz-PCG runs; returns (samples, solvers, gamma)."""
    import torch

    samples, solvers = [], []
    for w in workloads:
        t0 = time.perf_counter()
        s = fcm.Solver(w)
        s.precond_build()
        b = s.rhs()
        x_ref, its, _, _ = s.pcg_solve(b, tol_ref, maxit)
        nc = w.n[0] * w.n[1] * w.n[2]
        for k in snapshots:
            if k >= its:
                break
            xk, _, _, _ = s.pcg_solve(b, tol_ref, k, check=False)
            rk = b - s.apply_K(xk)
            ek = x_ref - xk
            energy = float(torch.dot(ek, rk))
            if not energy > 0:
                continue
            cells = s.coarse_restrict(rk, 1.0, eta_channel=True)
            re = s.coarse_restrict(ek, 1.0, eta_channel=False)
            sig_r = float(cells[: 3 * nc].double().pow(2).mean().sqrt())
            sig_e = float(re.double().pow(2).mean().sqrt())
            if sig_r > 0:
                samples.append(Sample(s, rk, cells, sig_r, energy, sig_e / sig_r))
        solvers.append(s)
        if log:
            log(f"  {w.name}: {its} iterations to {tol_ref:g}, {time.perf_counter() - t0:.1f} s")
    gamma = float(np.median([smp.ratio for smp in samples]))
    return samples, solvers, gamma


def _batch_input(samples, idx, grid):
    import torch

    nx, ny, nz = grid
    nc = nx * ny * nz
    x = torch.empty((len(idx), 4, nz, ny, nx), dtype=torch.float32, device="cuda")
    for j, i in enumerate(idx):
        smp = samples[i]
        x[j, :3] = (smp.cells[: 3 * nc] / smp.sigma).view(3, nz, ny, nx)
        x[j, 3] = smp.cells[3 * nc:].view(nz, ny, nx)
    return x


def loss_and_grad(net, samples, idx, gamma, grid):
    """Mean relative energy-norm loss over the batch and its gradient w.r.t. the network output."""
    import torch

    nx, ny, nz = grid
    x = _batch_input(samples, idx, grid)
    out = net.forward(x)
    gout = torch.empty_like(out)
    losses = []
    for j, i in enumerate(idx):
        smp = samples[i]
        a = gamma * smp.sigma
        c = smp.solver.coarse_prolong(out[j].reshape(-1), a)
        kc = smp.solver.apply_K(c)
        losses.append(1.0 + float(torch.dot(c, kc) - 2.0 * torch.dot(c, smp.r)) / smp.energy)
        g = smp.solver.coarse_restrict(kc - smp.r, 2.0 * a / smp.energy / len(idx), eta_channel=False)
        gout[j] = g.view(3, nz, ny, nx)
    return float(np.mean(losses)), gout


def train(net, samples, gamma, steps=400, batch=4, lr=1e-3, seed=0, log=print, log_every=50):
    grid = samples[0].solver.workload.n
    rng = np.random.default_rng(seed)
    history = []
    for step in range(1, steps + 1):
        idx = rng.choice(len(samples), size=min(batch, len(samples)), replace=False)
        loss, gout = loss_and_grad(net, samples, idx, gamma, grid)
        net.zero_grad()
        net.backward(gout)
        net.adam(lr * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / steps)), step)
        history.append(loss)
        if log and (step % log_every == 0 or step == 1):
            log(f"  step {step:5d}  loss {np.mean(history[-log_every:]):.4f}")
    return history


def evaluate(net, samples, gamma):
    """Mean loss over all samples (no update)."""
    grid = samples[0].solver.workload.n
    return float(np.mean([loss_and_grad(net, samples, [i], gamma, grid)[0] for i in range(len(samples))]))


MAGIC = b"FCMUNET1"


def save(path, net, gamma):
    """Checkpoint: magic, in/out channels, base, levels, gamma, then the FP32 parameters."""
    w = net.get()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<4id", *net.desc, gamma))
        f.write(w.astype("<f4").tobytes())


def load(path, seed=0):
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a U-Net checkpoint")
        in_ch, out_ch, base, levels, gamma = struct.unpack("<4id", f.read(24))
        w = np.frombuffer(f.read(), dtype="<f4").astype(np.float32)
    net = fcm.UNet(in_ch, out_ch, base, levels, seed)
    net.set(w)
    return net, gamma
