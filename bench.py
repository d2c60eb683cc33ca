"""Benchmark: PCG time-to-solution of the finite cell Schwarz-PCG on one GB300.

A step is one complete preconditioned CG solve (x0 = 0 to ||S r|| / ||S b|| <=
tol) of the default workload, the 80^3-cell, p=2 porous cube with 300 seeded
spherical voids (alpha 1e-10, octree depth 3, 11.4M free DOFs; the largest
configuration that fits one GPU), with the set-up, the preconditioner and the
coarse operator built once beforehand.  Forms:

  coarse (default): flexible CG, z = S r + P y with y from `--coarse-iters`
                    coarse CG steps on K_H = P^T K P, preconditioned by block
                    Jacobi or by a V-cycle of the cell-grid multigrid hierarchy
                    (`--coarse-prec`; both defaults per workload), optionally
                    started from a trained U-Net (`--net`); FP32 / double-float
                    block factors (`--precision`)
  pcg:              plain Schwarz-PCG

The same run also times plain FP64 Schwarz-PCG and reports the energy-norm
error of this form against it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fcm|reference]
                  [--workload NAME] [--form coarse|pcg] [--precision fp64|mixed]
                  [--coarse-iters K] [--coarse-prec jacobi|vcycle] [--net CHECKPOINT]
                  [--loads traction|strain6] [--mlhp-k K]
                  [--blocks vertex|element] [--eta-bar X]

N > 1 runs independent replicas (one per GPU, launched by torchrun); the
solve has no data-path collective.  `--impl reference` times the CPU oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time-to-solution (s) and GB/s vs HBM roofline at 1e-8, learned/mixed vs plain FP64"
DEFAULT_WORKLOAD = "porous300_80_p2"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 pipe of one SM: 2 fused multiply-adds per clock (64x below the 128 FP32
# lanes), i.e. 152 SMs x 2070 MHz x 4 flop = 1.26 TFLOP/s, the nominal GB300 FP64 rate.
FP64_FLOP_PER_CLK_PER_SM = 4
N_SM = 152


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "schwarz_apply_traffic_porous300_80_p2.md")

# Coarse CG of the flexible PCG per workload (preconditioner, steps), the fastest measured: while K_H fits
# the 129 MB L2 (32^3 cells: 74 MB) block-Jacobi steps are cheap and 20 of them solve the coarse grid
# well; at 80^3 cells K_H (1.16 GB) streams from HBM and two V-cycle-preconditioned steps win (3.2 s
# against 6.4 s for 10 block-Jacobi steps, which stall into the plain-PCG fallback).
COARSE_DEFAULTS = {"porous40_32_p3": ("jacobi", 20, "fp32"), "porous40_32_p2": ("jacobi", 20, "fp32"),
                   "porous300_80_p2": ("vcycle", 2, "fp32")}


def _schwarz_traffic(workload_name, precision):
    """DRAM bytes of one S apply from the committed ncu capture, or None.

    The capture (dram__bytes_read.sum + dram__bytes_write.sum over the 8 colour launches of one S
    apply) holds for the kernel source it was taken with: the profile records the SHA-256 of
    fcm_schwarz.cu, and any other source gives None.
    """
    import hashlib
    import re
    if workload_name != DEFAULT_WORKLOAD or precision != "mixed" or not os.path.exists(TRAFFIC_PROFILE):
        return None
    text = open(TRAFFIC_PROFILE).read()
    m_b = re.search(r"traffic_bytes_per_s_apply:\s*([0-9.eE+]+)", text)
    m_h = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    if not m_b or not m_h:
        return None
    src = os.path.join(ROOT, "paper_1809_00828_gb300", "csrc", "fcm_schwarz.cu")
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != m_h.group(1):
        return None
    return float(m_b.group(1))


def fp64_peak_tflops(sm_mhz):
    return N_SM * sm_mhz * 1e6 * FP64_FLOP_PER_CLK_PER_SM / 1e12


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload(name):
    from paper_1809_00828_gb300 import inputs
    return inputs.WORKLOADS[name]()


def oracle_sample(w, gpu_iterations, sapply_fmas, kapply_fmas, min_seconds=10.0):
    """Time the CPU oracle's PCG on a bounded window of the same workload and scale it.

    The window is the 2x2x2-cell corner [0, 2h]^3 of the same geometry, order,
    alpha and octree depth (27 vertex patches).  The oracle's per-iteration time
    is scaled by the ratio of per-iteration multiply-adds (K entries + sum of
    block sizes squared) of the full workload to the window, times the full
    workload's iteration count.
    """
    from oracle import oracle as O
    from paper_1809_00828_gb300 import inputs
    h = [(w.hi[a] - w.lo[a]) / w.n[a] for a in range(3)]
    win = inputs.Workload(w.name + "_window", (2, 2, 2), w.p, w.alpha, w.geometry, w.tol, E=w.E, nu=w.nu,
                          traction=w.traction, bc=w.bc, lo=w.lo,
                          hi=tuple(w.lo[a] + 2 * h[a] for a in range(3)))
    P = O.Problem.from_workload(win)
    P.precond_build(0)
    # work measure shared by window and full problem: active cells x ne^2 + sum of block sizes^2
    ne = 3 * (w.p + 1) ** 3
    nnz = int((P.eta() > 0).sum()) * ne * ne
    blocks = sum(P.block(b)[0].size ** 2 for b in range(P.nblocks()))
    per_iter = []
    t_total = 0.0
    while t_total < min_seconds:
        t0 = time.perf_counter()
        _, its, _ = P.pcg(tol=w.tol, maxit=20000)
        dt = time.perf_counter() - t0
        t_total += dt
        per_iter.append(dt / max(its, 1))
    t_iter = statistics.median(per_iter)
    scale = (kapply_fmas + sapply_fmas) / float(nnz + blocks)
    value = t_iter * scale * gpu_iterations
    sample = (f"oracle PCG on the 2x2x2-cell corner window of {w.name} ({P.nfree} DOFs, {P.nblocks()} blocks), "
              f"{len(per_iter)} solves in {t_total:.1f} s; {t_iter * 1e3:.3f} ms/iteration scaled by per-iteration multiply-adds x{scale:.1f} "
              f"and {gpu_iterations} iterations")
    return value, sample, t_total


# iterations of plain FP64 Schwarz-PCG (the oracle's algorithm) measured on the GPU for these workloads
REF_ITERATIONS = {"porous40_32_p3": 877, "porous300_80_p2": 2706}

MODEL_NOTE = ("model: the oracle's measured per-iteration time on the corner window, scaled by multiply-adds to "
              "the whole workload; full_solve_measured is a complete oracle solve, measured")

FULL_SOLVE_WORKLOAD = ("porous40_8_p2", 11, 8, 2, 40, 1e-10, 3, 1e-8)


def full_solve_comparison(fcm=None, repeats=3):
    """A complete solve the oracle finishes in seconds, timed on the host and on the GPU.

    The 8^3-cell, p = 2 member of the porous family (40 seeded voids, seed 11, 13,872 free DOFs): the
    oracle's plain FP64 Schwarz-PCG (one thread, as it stands; set-up and preconditioner timed apart,
    solve only, median of `repeats`) beside this library's plain FP64 Schwarz-PCG on the same problem
    (device time of fcm_pcg_solve, median of `repeats`), when `fcm` is given.
    """
    from oracle import oracle as O
    from paper_1809_00828_gb300 import inputs
    name, seed, nc, p, cnt, alpha, depth, tol = FULL_SOLVE_WORKLOAD
    w = inputs.workload_porous(seed, nc, p, cnt, alpha, depth, tol)
    t0 = time.perf_counter()
    P = O.Problem.from_workload(w)
    t1 = time.perf_counter()
    P.precond_build(0)
    t2 = time.perf_counter()
    times, its = [], 0
    for _ in range(repeats):
        ts = time.perf_counter()
        _, its, _ = P.pcg(tol=tol, maxit=20000)
        times.append(time.perf_counter() - ts)
    out = {"workload": f"{name}: {nc}^3 cells, p={p}, {cnt} spherical voids (seed {seed}), alpha={alpha:g}, "
                       f"octree depth {depth}, tol {tol:g}, {P.nfree} free DOFs",
           "oracle_threads": 1, "oracle_setup_s": t1 - t0, "oracle_precond_s": t2 - t1,
           "oracle_solve_s": statistics.median(times), "oracle_iterations": its}
    if fcm is not None:
        s = fcm.Solver(w)
        s.precond_build(precision="fp64")
        b = s.rhs()
        gt = []
        for _ in range(repeats + 1):
            _, gits, _, _ = s.pcg_solve(b, tol, 20000)
            gt.append(s.last_solve()["seconds"])
        out.update({"gpu_solve_s": statistics.median(gt[1:]), "gpu_iterations": gits,
                    "solve_speedup": statistics.median(times) / statistics.median(gt[1:])})
        s.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = _workload(args.workload)
    # per-iteration work is counted on the host from the problem sizes; the iteration count that
    # scales the per-iteration time is --ref-iterations (a full oracle solve at this size would
    # take hours)
    gpu_like_iters = args.ref_iterations
    kf, sf = _host_work_counts(w)
    steps, walls = [], []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, sample, wall = oracle_sample(w, gpu_like_iters, sf, kf, min_seconds=1.0 if i < args.warmup else 5.0)
        if i >= args.warmup:
            steps.append(v)
            walls.append(wall)
    value = statistics.median(steps)
    # a step is a bounded sample (the corner window) whose per-iteration time is scaled to the whole
    # workload; ms_per_step is the wall time a sample actually took
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(walls) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _describe(w, args), "precision": "fp64",
                       "value_kind": "time-to-solution of the whole workload, scaled from each step's sample"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                             "value_kind": MODEL_NOTE, "full_solve_measured": full_solve_comparison(None)},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _host_work_counts(w):
    """Per-iteration multiply-adds of K (active cells x ne^2) and S (sum of box sizes^2), counted on the host."""
    p = w.p
    ne = 3 * (p + 1) ** 3
    ncells = w.n[0] * w.n[1] * w.n[2]
    kf = ncells * ne * ne
    sf = 0
    dims = []
    for a in range(3):
        M = p * w.n[a] + 1
        d = []
        for v in range(w.n[a] + 1):
            lo = max(0, p * v - (p - 1))
            hi = min(M - 1, p * v + (p - 1))
            d.append(hi - lo + 1)
        dims.append(np.array(d, dtype=np.int64))
    box = 3 * dims[0][None, None, :] * dims[1][None, :, None] * dims[2][:, None, None]
    sf = int((box.astype(np.int64) ** 2).sum())
    return kf, sf


def _describe(w, args):
    g = w.geometry
    shape = (f"{len(g.spheres)} spherical voids" if g.spheres is not None else
             f"voxel image {'x'.join(str(v) for v in g.voxels.shape)} (solid fraction {g.voxels.mean():.2f})"
             if g.voxels is not None else "no voids")
    return (f"{w.name}: {w.n[0]}x{w.n[1]}x{w.n[2]} cells, p={w.p}, alpha={w.alpha:g}, {shape}, "
            f"octree depth {w.geometry.octree_depth}, tol {w.tol:g}, E={w.E:g}, nu={w.nu:g}, z=0 clamped, "
            f"{'unit traction on z=1' if args.loads == 'traction' else 'six unit-strain load cases'}, "
            f"{_blocks(args)}, eps=1e-13")


def _blocks(args):
    if args.blocks == "element":
        return (f"element blocks for the cells with eta_T <= {args.eta_bar:g} and diagonal scaling of the DOFs "
                f"in no block")
    return "vertex-patch blocks"


def _form(args, net):
    if args.form == "pcg":
        return "plain Schwarz-PCG"
    start = "trained U-Net prediction scaled by the coarse line search" if net is not None else "zero"
    prec = {"jacobi": "block-Jacobi",
            "vcycle": "V-cycle-preconditioned (cell-grid multigrid, Galerkin levels, damped block-Jacobi "
                      "smoothing, dense coarsest level)",
            "hybrid": "hybrid-V-cycle-preconditioned (cell-grid multigrid, additive block Jacobi on the finest "
                      "cell grid, V-cycle below)"}[args.coarse_prec]
    return (f"flexible CG(4), z = S r + P y, y from {args.coarse_iters} {prec} CG steps on the Galerkin "
            f"coarse operator K_H = P^T K P ({args.coarse_storage} storage) starting from {start}")


def _launches_per_solve(args, info, its, flex_its, net, mg_levels=0):
    """Kernels of one solve (device-side loop, so the count follows the iterations): K and S applies
    from the library's own counts, plus the CG vector kernels, the coarse solve and the network."""
    k_apply, s_apply = info["k_apply_launches"], info["s_apply_launches"]
    plain = k_apply + 2 + s_apply + 2                   # K, pq, xr, S, rz, p
    start = 3 + 1 + s_apply + 1 + k_apply + 2           # mask copy, norms, init, first S, first kernel, true residual
    if args.form == "pcg":
        return start + its * plain
    k = args.coarse_iters
    coarse = 1 + (1 + 2 * k) + 1                        # restrict, coarse start + 2 per step, prolong
    if args.coarse_prec == "vcycle" and k > 0:
        # a V-cycle (5 launches per level above the last, 1 for the last) and r.z, once per step
        coarse += k * (5 * (mg_levels - 1) + 1 + 1)
    elif args.coarse_prec == "hybrid" and k > 0:
        # level 0: Jacobi, restrict, interpolate; 5 per level between; 1 for the last; r.z
        coarse += k * ((3 + 5 * (mg_levels - 2) if mg_levels > 1 else 0) + 1 + 1)
    if net is not None:
        coarse += 2 + 1 + 2 + _unet_launches(net)       # sigma, prep, post, start apply + line search
    flex = k_apply + 2 + s_apply + 1 + coarse + 2       # pq, xr, conv, dots, newp
    return start + coarse + flex_its * flex + (its - flex_its) * plain


def _unet_launches(net):
    L = net.desc[3]
    # per level: pool (l > 0), 2 x (conv, relu); per decoder level: up, copy, 2 x (conv, relu); output conv
    return (L - 1) + 4 * L + 6 * (L - 1) + 1


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (the job ends with its slowest replica); `value` itself
    without a process group."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_fcm(args, rank, world, local_rank):
    import torch
    from paper_1809_00828_gb300 import fcm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = _workload(args.workload)
    s = fcm.Solver(w)
    k_prec = args.k_precision if args.precision != "fp64" else "fp64"
    s.set_k_precision(k_prec)
    if args.profile_apply == "KH":
        # the coarse operator alone (no preconditioner on the device): K_H products between
        # cudaProfilerStart / Stop, after its assembly and 3 warm-up products
        nc = w.n[0] * w.n[1] * w.n[2]
        xc = torch.ones(3 * nc, dtype=torch.float32, device="cuda")
        yc = torch.empty_like(xc)
        for _ in range(3):
            s.coarse_apply(xc, out=yc)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.profile_reps):
            s.coarse_apply(xc, out=yc)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profiled {args.profile_reps} K_H applies of {w.name}")
        s.close()
        return 0
    s.precond_build(precision=args.precision, blocks=args.blocks, eta_bar=args.eta_bar)
    n = s.n
    # load cases: 0 = traction on z = 1; 1..6 = unit Voigt strains (one solve of all six)
    cases = [0] if args.loads == "traction" else [1, 2, 3, 4, 5, 6]
    nrhs = len(cases)
    b = torch.cat([s.rhs(k) for k in cases])
    u = s.empty(nrhs)
    stream = torch.cuda.current_stream()
    net, gamma = None, 0.0
    if args.form == "coarse":
        s.set_stall_window(args.stall_window)
        s.set_coarse_preconditioner(args.coarse_prec)
        s.set_coarse_storage(args.coarse_storage)
    if args.form == "coarse" and args.net:
        from paper_1809_00828_gb300 import learned
        net, gamma = learned.load(args.net)

    def solve(out):
        """One step: every right-hand side solved; returns the largest iteration count and residual."""
        if args.form == "coarse":
            its, rel = 0, 0.0
            for k in range(nrhs):
                _, i, r, _ = s.fpcg_solve(net, gamma, b[k * n:(k + 1) * n], w.tol, args.maxit,
                                          out=out[k * n:(k + 1) * n], coarse_iters=args.coarse_iters)
                its, rel = max(its, i), max(rel, r)
        else:
            _, its, rel, _ = s.pcg_solve(b, w.tol, args.maxit, out=out)
        return its, rel

    if args.profile_apply:
        # apply S (or K) a few times between cudaProfilerStart / Stop, after 3 warm-up applies, for
        # `ncu --profile-from-start off`; no JSON line
        r = b[:n].clone()
        z = s.empty()
        op = s.apply_S if args.profile_apply == "S" else s.apply_K
        for _ in range(3):
            op(r, out=z)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.profile_reps):
            op(r, out=z)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profiled {args.profile_reps} {args.profile_apply} applies of {w.name}")
        s.close()
        return 0
    for _ in range(args.warmup):
        its, rel = solve(u)
    if args.profile_one_step:
        # one step between cudaProfilerStart / Stop, for `ncu --profile-from-start off`; no JSON line
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        its, rel = solve(u)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profiled one step: {its} iterations, relres {rel:.3e}")
        s.close()
        return 0
    info = s.get_info()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = []
    for _ in range(args.steps):
        its, rel = solve(u)
        iters.append(its)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    ms_per_step = elapsed / args.steps * 1e3
    last = s.last_solve()

    # the Schwarz apply (all its launches, block products and sum) and the K apply, timed live on the stream
    r = b[:n].clone()
    z = s.empty()
    for _ in range(3):
        s.apply_S(r, out=z)
    torch.cuda.synchronize()
    reps = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.apply_S(r, out=z)
    e1.record(stream)
    torch.cuda.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3 / reps
    e0.record(stream)
    for _ in range(reps):
        s.apply_K(r, out=z)
    e1.record(stream)
    torch.cuda.synchronize()
    t_k = e0.elapsed_time(e1) / 1e3 / reps

    peaks, peak_kind = _peaks()
    s_flops = 2.0 * info["sapply_fmas"]
    # algorithmic HBM bytes of one S apply: distinct stored factors + gather of r + read-modify-write of z
    s_bytes = info["factor_bytes"] + 8.0 * n * 3
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = fp64_peak_tflops(sm_mhz)
    achieved_tf = s_flops / t_s / 1e12
    achieved_gbs = s_bytes / t_s / 1e9
    shared = (f"tc_gemm_kernel<{w.p}> (tcgen05, shared factors)" if args.precision != "fp64" and w.p in (2, 3)
              else f"schwarz_gemm_kernel<{w.p}> (shared factors)")
    kernel = (f"S apply, {info['s_apply_launches']} launches: {shared} + "
              f"{'schwarz_rows_kernel' if w.p == 3 else 'schwarz_cols_kernel'}<{w.p}> (streamed factors) + "
              f"schwarz_sum_kernel<{w.p}>, shared-factor products "
              f"{'beside' if info['schwarz_concurrent'] else 'before'} the streamed ones (the shape the build's "
              f"autotuner kept)")
    if args.precision == "fp64":
        # FP64 factors: one FP64 multiply-add per 8-byte entry; the FP64 pipe saturates first
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved_tf / fp64_peak, "traffic": None, "kernel": kernel,
                    "peak_source": f"derived FP64 peak: {N_SM} SMs x {FP64_FLOP_PER_CLK_PER_SM} flop/clk x median "
                                   f"SM clock {sm_mhz:.0f} MHz",
                    "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                    "hbm_frac": achieved_gbs / peaks["hbm_gbs"]}
    else:
        # FP32 factors stream from HBM (shared factors from L2); FP64 only for the ill-conditioned blocks
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved_gbs / peaks["hbm_gbs"], "traffic": _schwarz_traffic(args.workload, args.precision),
                    "traffic_source": os.path.relpath(TRAFFIC_PROFILE, ROOT), "kernel": kernel,
                    "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "fp64_tflops_equivalent": achieved_tf, "fp64_peak_tflops": fp64_peak}
    if args.form == "coarse":
        # the coarse operator apply (one kh_kernel launch), timed live; algorithmic bytes: the
        # stored half of K_H once plus the input and output cell vectors
        nc = w.n[0] * w.n[1] * w.n[2]
        xc = torch.ones(3 * nc, dtype=torch.float32, device="cuda")
        yc = torch.empty_like(xc)
        for _ in range(3):
            s.coarse_apply(xc, out=yc)
        e0.record(stream)
        for _ in range(reps):
            s.coarse_apply(xc, out=yc)
        e1.record(stream)
        torch.cuda.synchronize()
        t_h = e0.elapsed_time(e1) / 1e3 / reps
        kh_bytes = nc * (63 * 9 * 4 + 2 * 3 * 4)
        roofline.update({"kh_apply_us": t_h * 1e6, "kh_algorithmic_bytes": kh_bytes,
                         "kh_achieved_gbs": kh_bytes / t_h / 1e9,
                         "kh_note": f"K_H ({nc * 63 * 9 * 4 / 1e6:.0f} MB) "
                                    + ("stays in L2 (129 MB) across a coarse solve, so this rate can exceed the "
                                       "HBM copy peak" if nc * 63 * 9 * 4 < 100e6 else "streams from HBM")})
    roofline.update({"s_apply_ms": t_s * 1e3, "k_apply_ms": t_k * 1e3, "k_precision": k_prec,
                     "k_apply_multiply_adds_per_s": info["kapply_fmas"] / t_k,
                     "k_apply_fp64_frac": 2.0 * info["kapply_fmas"] / t_k / 1e12 / fp64_peak,
                     "algorithmic_bytes_per_s_apply": s_bytes})

    # end to end through the host-buffer entry point (pinned buffers, copies inside the timed region)
    b_host = torch.empty(n * nrhs, dtype=torch.float64, pin_memory=True)
    b_host.copy_(b)
    u_host = torch.empty(n * nrhs, dtype=torch.float64, pin_memory=True)
    bh = b_host.numpy()
    uh = u_host.numpy()
    def solve_host():
        if args.form == "coarse":
            for k in range(nrhs):
                s.fpcg_solve_host(net, gamma, bh[k * n:(k + 1) * n], w.tol, args.maxit,
                                  out=uh[k * n:(k + 1) * n], coarse_iters=args.coarse_iters)
        else:
            s.pcg_solve_host(bh, w.tol, args.maxit, out=uh)

    solve_host()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        solve_host()
    e2e = (time.perf_counter() - t0) / e2e_steps

    its_med = int(statistics.median(iters))
    flex_its = last["flexible_iterations"] if args.form == "coarse" else 0
    mg = s.coarse_levels() if args.form == "coarse" else {"levels": 0, "dims": [], "seconds": 0.0}
    launches_per_solve = (_launches_per_solve(args, info, its_med, flex_its, net, mg["levels"]) *
                          (nrhs if args.form == "coarse" else 1))
    line = {"metric": METRIC, "value": ms_per_step / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
            "config": {"workload": _describe(w, args), "loads": args.loads, "form": _form(args, net),
                       "precision": args.precision, "k_precision": k_prec, "n_free": info["n_free"],
                       "iterations": its_med, "relres": rel, "true_relres": last["true_relres"],
                       "fell_back_to_plain_pcg": bool(last["fallback"]) if args.form == "coarse" else None,
                       "flexible_iterations": last["flexible_iterations"] if args.form == "coarse" else None,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"inputs larger than L2: factor pool {info['factor_bytes'] / 2**30:.2f} GiB, "
                             f"element matrices {info['element_bytes'] / 2**30:.2f} GiB",
                       "n_blocks": info["n_blocks"], "n_factors": info["n_factors"],
                       "n_factors_fp32": info["n_blocks_fp32"], "n_jacobi_dofs": info["n_jacobi"],
                       "n_factors_double_float": info["n_factors_ff"], "n_gemm_blocks": info["n_gemm_blocks"],
                       "schwarz_launch": {"stream_rows": info["stream_rows"],
                                          "concurrent": bool(info["schwarz_concurrent"]),
                                          "autotune_ms": [round(t * 1e3, 4) for t in info["tune_seconds"] if t > 0]},
                       "setup_s": info["setup_seconds"], "precond_s": info["precond_seconds"],
                       "coarse_operator_s": info["coarse_seconds"],
                       "coarse_multigrid": ({"levels": mg["dims"], "build_s": mg["seconds"]}
                                            if mg["levels"] else None),
                       "load_cases": cases},
            "roofline": roofline,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 8 * n * nrhs, "d2h_bytes_per_step": 8 * n * nrhs},
            "gpu_launches": launches_per_solve * args.steps,
            "clocks": clk}
    its64 = its_med
    if args.form != "pcg" or args.precision != "fp64":
        # plain Schwarz-PCG on the same GPU (mixed factors, then FP64 factors): their times-to-solution
        # for the comparison the metric names, and the relative energy-norm error (Eq. (15)) of this
        # form against the plain FP64 solve
        x = u.clone()
        nrep = max(1, min(args.steps, 3))
        if args.form != "pcg" and args.precision == "mixed":
            s.pcg_solve(b, w.tol, args.maxit)
            tm = []
            for _ in range(nrep):
                _, itsm, _, _ = s.pcg_solve(b, w.tol, args.maxit)
                tm.append(s.last_solve()["seconds"])  # device time of the call (all right-hand sides)
            line["config"]["plain_mixed"] = {"seconds": statistics.median(tm), "iterations": itsm,
                                             "speedup_of_this_form": statistics.median(tm) / (ms_per_step / 1e3)}
        s.set_k_precision("fp64")
        s.precond_build(precision="fp64", blocks=args.blocks, eta_bar=args.eta_bar)
        x64, its64, _, _ = s.pcg_solve(b, w.tol, args.maxit)
        t64 = []
        for _ in range(nrep):
            s.pcg_solve(b, w.tol, args.maxit, out=x64)
            t64.append(s.last_solve()["seconds"])
        errs = []
        for k in range(nrhs):
            e = x[k * n:(k + 1) * n] - x64[k * n:(k + 1) * n]
            num = torch.dot(e, s.apply_K(e)).item()
            den = torch.dot(x64[k * n:(k + 1) * n], s.apply_K(x64[k * n:(k + 1) * n])).item()
            errs.append((abs(num) / den) ** 0.5)
        line["config"]["energy_error_vs_fp64"] = max(errs)
        line["config"]["plain_fp64"] = {"seconds": statistics.median(t64), "iterations": its64,
                                        "speedup_of_this_form": statistics.median(t64) / (ms_per_step / 1e3)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs plain FP64 Schwarz-PCG: scaled to that method's iteration count
        kf = info["n_cells_active"] * (3 * (w.p + 1) ** 3) ** 2
        sf = info["sapply_fmas"]
        v, sample, _ = oracle_sample(w, its64, sf, kf)
        if nrhs > 1:
            v *= nrhs
            sample += f"; times {nrhs} right-hand sides"
        line["cpu_baseline"] = {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                                "value_kind": MODEL_NOTE, "full_solve_measured": full_solve_comparison(fcm)}
    if net is not None:
        net.close()
    s.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_mlhp(args):
    """Multi-level hp path on the Sec. 5.1 cube: 8^3 base cells, p = 3, a cavity of radius 0.01 at the
    centre refined `args.mlhp_k` times toward its surface, alpha = 1e-8, truncated blocks.  One JSON line:
    host set-up times, the device K and S applies (CUDA events on the plan's stream, median of 20 after 3
    warm-ups) with their algorithmic bytes and bandwidth, and the PCG solve to 1e-8.  Algorithmic bytes: K x
    reads 12 B per CSR nonzero plus the row pointers and writes y; S r reads every stored factor byte once
    (8 B per entry as a float pair, 4 B in FP32) plus the gathers and the block-row sums."""
    import numpy as np
    import torch
    from paper_1809_00828_gb300 import fcm

    t0 = time.time()
    P = fcm.MLHPPlan((8, 8, 8), (0, 0, 0), (1, 1, 1), [(0.5, 0.5, 0.5, 0.01)], 3, args.mlhp_k, octree_depth=3)
    free, K, b, eta = P.assemble(1e-8, "clamp")
    t1 = time.time()
    blocks, F, cptr, jac = P.factorize("truncated", device=args.mlhp_factorize == "device")
    torch.cuda.synchronize()
    t2 = time.time()
    P.device_setup(precision=args.mlhp_precision)
    n32, fbytes = P.device_info()
    n = len(free)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(n)).cuda()
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()

    def timed(fn, reps=20, warm=3):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return float(np.median(ts))

    tk = timed(lambda: P.apply_K(x, y))
    ts = timed(lambda: P.apply_S(x, y))
    bk = 12 * K.nnz + 8 * (n + 1) + 16 * n
    nb_dofs = sum(len(B) for B in blocks)
    bs = fbytes + 4 * nb_dofs + 8 * nb_dofs * 3 + 24 * n
    bd = torch.from_numpy(b).cuda()
    P.pcg_solve(bd, 1e-8, 20000, check=False)  # warm-up: captures the iteration graph
    torch.cuda.synchronize()
    t3 = time.time()
    _, its, _, status = P.pcg_solve(bd, 1e-8, 20000, check=False)
    torch.cuda.synchronize()
    t4 = time.time()
    hbm = _peaks()[0]["hbm_gbs"]
    print(json.dumps({"workload": f"mlhp cube: 8^3 base cells, p=3, cavity r=0.01, k={args.mlhp_k}, truncated blocks",
                      "dofs": n, "nnz": int(K.nnz), "blocks": len(blocks), "colours": len(cptr) - 1,
                      "precision": args.mlhp_precision, "fp32_blocks": n32, "factor_bytes": fbytes,
                      "assemble_s": round(t1 - t0, 2), "factorize_s": round(t2 - t1, 2),
                      "factorize_on": args.mlhp_factorize,
                      "apply_K_ms": round(tk * 1e3, 4), "apply_K_GBs": round(bk / tk * 1e-9, 1),
                      "apply_K_frac": round(bk / tk * 1e-9 / hbm, 3),
                      "apply_S_ms": round(ts * 1e3, 4), "apply_S_GBs": round(bs / ts * 1e-9, 1),
                      "apply_S_frac": round(bs / ts * 1e-9 / hbm, 3),
                      "pcg_iterations": its, "pcg_status": status, "pcg_s": round(t4 - t3, 4)}))
    P.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fcm", choices=["fcm", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed_fp64"],
                    help="mixed: FP32 block factors, double-float pairs for cond > 1e7 (mixed_fp64: FP64 there), "
                         "compared with plain FP64 in the same run")
    ap.add_argument("--form", default="coarse", choices=["coarse", "pcg"],
                    help="coarse: flexible CG with the Galerkin coarse correction; pcg: plain Schwarz-PCG")
    ap.add_argument("--coarse-iters", type=int, default=None,
                    help="coarse CG steps per preconditioner apply (default: per workload, COARSE_DEFAULTS)")
    ap.add_argument("--coarse-storage", default=None, choices=["fp32", "fp16", "fp16_cycles"],
                    help="storage of K_H: FP32, or symmetrically scaled FP16 (default: per workload)")
    ap.add_argument("--coarse-prec", default=None, choices=["jacobi", "vcycle", "hybrid"],
                    help="preconditioner of the coarse CG: 3x3 diagonal blocks of K_H, or one V-cycle of the "
                         "cell-grid multigrid hierarchy (default: per workload, COARSE_DEFAULTS)")
    ap.add_argument("--k-precision", default="double_float", choices=["double_float", "fp64"],
                    help="arithmetic of K x in the forms with FP32 factors (plain FP64 always uses FP64 K)")
    ap.add_argument("--stall-window", type=int, default=100,
                    help="iterations without halving after which the flexible CG falls back to plain PCG")
    ap.add_argument("--net", default=None, help="U-Net checkpoint whose prediction starts the coarse solve")
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--loads", default="traction", choices=["traction", "strain6"],
                    help="traction: the z = 1 traction load; strain6: the six unit-strain load cases in one step")
    ap.add_argument("--blocks", default="vertex", choices=["vertex", "element"],
                    help="Schwarz blocks: vertex patches, or the paper's element blocks with --eta-bar")
    ap.add_argument("--eta-bar", type=float, default=1.0,
                    help="element blocks for the cells with volume fraction at most this (1: every cell); "
                         "the DOFs in no block diagonal")
    ap.add_argument("--ref-iterations", type=int, default=None,
                    help="iteration count that scales the reference arm's per-iteration time (default: the plain "
                         "FP64 Schwarz-PCG count measured on the GPU for the workload, which the oracle's "
                         "algorithm shares)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-apply", default=None, choices=["S", "K", "KH"],
                    help="apply S, K or the coarse operator K_H (KH: without building the preconditioner) "
                         "--profile-reps times between cudaProfilerStart/Stop and exit (for ncu)")
    ap.add_argument("--profile-reps", type=int, default=3)
    ap.add_argument("--profile-one-step", action="store_true",
                    help="after the warm-up, run one step between cudaProfilerStart/Stop and exit (for ncu)")
    ap.add_argument("--mlhp-factorize", default="device", choices=["host", "device"],
                    help="eigensolves of the multi-level blocks: host threads or batched on the GPU")
    ap.add_argument("--mlhp-precision", default="mixed", choices=["fp64", "mixed"],
                    help="factor storage of the multi-level path (mixed: FP32 where cond <= 1e7)")
    ap.add_argument("--mlhp-k", type=int, default=None,
                    help="instead of the bench line: time the multi-level hp path on the Sec. 5.1 cube refined k times")
    args = ap.parse_args()
    prec, iters, storage = COARSE_DEFAULTS.get(args.workload, ("vcycle", 2, "fp32"))
    args.coarse_prec = args.coarse_prec or prec
    args.coarse_storage = args.coarse_storage or storage
    args.coarse_iters = iters if args.coarse_iters is None else args.coarse_iters
    if args.mlhp_k is not None:
        return run_mlhp(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.ref_iterations is None and args.workload not in REF_ITERATIONS:
            print(json.dumps({"impl": "reference", "unavailable": f"no plain FP64 iteration count recorded for "
                                                                  f"{args.workload}; pass --ref-iterations"}))
            return 0
        if args.ref_iterations is None:
            args.ref_iterations = REF_ITERATIONS[args.workload]
        return run_reference(args, rank, world)
    return run_fcm(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
