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


def train_cubes(net, seeds, n=32, p=2, count=40, group=8, steps_per_group=100, batch=4, lr=1e-3,
                snapshots=SNAPSHOTS, log=print):
    """Train on many seeded porous cubes, `group` cubes at a time: their snapshots are generated (one
    FP64 Schwarz-PCG per cube), the network takes `steps_per_group` Adam steps on them, and the group's
    contexts are released before the next group.  gamma is the median RMS(R e) / RMS(R r) of the first
    group.  Returns (gamma, loss history)."""
    gamma = None
    history = []
    seeds = list(seeds)
    for g0 in range(0, len(seeds), group):
        ws = training_workloads(seeds[g0:g0 + group], n=n, p=p, count=count)
        samples, solvers, g = generate(ws, snapshots, log=None)
        if gamma is None:
            gamma = g
        history += train(net, samples, gamma, steps=steps_per_group, batch=batch, lr=lr, seed=g0, log=None)
        for s in solvers:
            s.close()
        if log:
            log(f"  cubes {g0}..{g0 + len(ws) - 1}: {len(samples)} pairs, mean loss {np.mean(history[-steps_per_group:]):.4f}")
    return gamma, history


def solve_gain(net, gamma, workload, coarse_iters, tol=None, maxit=20000):
    """Flexible PCG on `workload` with the network's start and without it (zero start), the same coarse
    steps: (iterations with, iterations without, seconds with, seconds without)."""
    s = fcm.Solver(workload)
    s.set_k_precision("double_float")
    s.precond_build(precision="mixed")
    b = s.rhs()
    tol = tol or workload.tol
    out = []
    for nn in (net, None):
        if nn is None and coarse_iters == 0:
            _, its, _, _ = s.pcg_solve(b, tol, maxit)
        else:
            _, its, _, _ = s.fpcg_solve(nn, gamma if nn is not None else 0.0, b, tol, maxit, coarse_iters=coarse_iters)
        out.append((its, s.last_solve()["seconds"]))
    s.close()
    return out[0][0], out[1][0], out[0][1], out[1][1]


def main(argv=None):
    """python -m paper_1809_00828_gb300.learned train|gain ...

    train: the configured training set (seeded 32^3, p = 2 porous cubes with 40 voids; seeds 1000..1199 by
    default), a 4-level U-Net (channels 16/32/64/64), checkpoint to --out.
    gain: flexible PCG on a held-out workload with the checkpoint's start and without it.
    """
    import argparse
    ap = argparse.ArgumentParser(prog="python -m paper_1809_00828_gb300.learned")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--seeds", default="1000-1199", help="first-last seed of the training cubes")
    t.add_argument("--n", type=int, default=32)
    t.add_argument("--p", type=int, default=2)
    t.add_argument("--count", type=int, default=40)
    t.add_argument("--group", type=int, default=8)
    t.add_argument("--steps-per-group", type=int, default=100)
    t.add_argument("--batch", type=int, default=4)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--base", type=int, default=16)
    t.add_argument("--levels", type=int, default=4)
    t.add_argument("--out", required=True)
    g = sub.add_parser("gain")
    g.add_argument("--net", required=True)
    g.add_argument("--workload", default="porous300_80_p2")
    g.add_argument("--coarse-iters", type=int, default=10)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        lo, hi = (int(v) for v in a.seeds.split("-"))
        net = fcm.UNet(in_ch=4, out_ch=3, base=a.base, levels=a.levels, seed=0)
        t0 = time.perf_counter()
        gamma, hist = train_cubes(net, range(lo, hi + 1), n=a.n, p=a.p, count=a.count, group=a.group,
                                  steps_per_group=a.steps_per_group, batch=a.batch, lr=a.lr)
        save(a.out, net, gamma)
        print(f"trained on seeds {lo}..{hi} in {time.perf_counter() - t0:.0f} s, gamma {gamma:.4f}, "
              f"final mean loss {np.mean(hist[-a.steps_per_group:]):.4f} -> {a.out}")
        net.close()
    else:
        net, gamma = load(a.net)
        w = inputs.WORKLOADS[a.workload]()
        iw, io, sw, so = solve_gain(net, gamma, w, a.coarse_iters)
        print(f"{w.name}, {a.coarse_iters} coarse steps: with the network {iw} iterations {sw:.3f} s, "
              f"without {io} iterations {so:.3f} s")
        net.close()


if __name__ == "__main__":
    main()
