"""Benchmark: 4-D phase-space point-updates/s of the periodic two-body Wigner
2-RDM Lawson step on GB300, FP64 results (the sliced FP64 path, held to the
FP64 oracle at 1e-10), 64^4 double-well workload; the FP64-pipe path and the
precision, batching and learned forms are reported beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl w2|reference]

One JSON line on rank 0.  "value" is whole-job throughput (all ranks) with
the state resident in HBM; "e2e" goes through the public C ABI with the state
copied from pinned host memory and the observables read back every step (the
copy of the next step's input staged during the current step).
Each rank advances its own independent replica (the step has no exchange
between replicas), so scaling is weak and there is no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4-D phase-space point-updates/s vs plain FP64 GPU path at fixed rel-L2 error"
UNIT = "point-updates/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, dist_mod, device):
    """Maximum of a per-rank float over all ranks (the job's time is that of
    the slowest replica)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, steps, world_size, max_ms):
    """Point-updates per second of all replicas together (weak scaling)."""
    return points_per_rank * steps * world_size / (max_ms / 1e3)


def _workload_desc(prob):
    return {"workload": f"double-well 2-RDM Wigner step, {prob.nx}^2 x {prob.nk}^2 grid, L={prob.L:g}, "
                        f"dt={prob.dt:g}, soft-Coulomb pair gamma={prob.gamma:g}, Hartree c_H={prob.c_hartree:g}, "
                        f"capped well min(0.05(x^2-16)^2,20)",
            "nx": prob.nx, "nk": prob.nk, "points": prob.points,
            "l2": "inputs larger than L2: four 134 MB FP64 phase-space arrays are streamed every step",
            "parallelism": "replicas"}


def _oracle_sample(prob_full, min_seconds):
    """Time the FP64 oracle on a bounded sample of the workload: whole Lawson
    steps of the same 64^4 problem, as many as fit in min_seconds (>= 1)."""
    import oracle
    from paper_2511_11354_gb300 import inputs
    prob, f0 = inputs.workload_dwell(nx=prob_full.nx, nk=prob_full.nk)
    o = oracle.Oracle(prob)
    steps, t0 = 0, time.perf_counter()
    f = f0
    while True:
        f = o.step(f, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return {"value": prob.points * steps / el, "unit": UNIT, "cores": oracle.Oracle.threads(), "kind": "oracle",
            "sample": f"{steps} oracle Lawson step(s) of the full {prob.nx}^2 x {prob.nk}^2 workload "
                      f"from its initial state, {el:.1f} s"}


class ClockSampler:
    def __init__(self, index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"w2_clocks_{os.getpid()}.csv")
        if shutil.which("nvidia-smi") is None:
            return
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                      "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


def _pipe_peaks():
    """Live peaks of the FP64 tensor path (DMMA), of DFMA and of BF16 mma.sync
    (register-only loops of the committed probe)."""
    src = os.path.join(ROOT, "bench_pipe_peaks.cu")
    exe = os.path.join(ROOT, "_build", "bench_pipe_peaks")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip().splitlines()[-1]
    return json.loads(out)


# DRAM bytes (read + write) per k_theta_s launch on the 64^4 workload, the mean
# of the predictor and the corrector of one ncu capture
# (profiles/k_theta_s_dwell_64x64.md), keyed by the hash of the kernel's
# sources (w2_f64s.cu, w2_slice.cuh) it was taken on: any change reports null.
THETA_TRAFFIC = {"0b8020afffd5fb75": 0.5 * ((134.501888e6 + 94.811392e6) + (268.730112e6 + 92.352000e6))}


def _theta_traffic():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2511_11354_gb300", "csrc")
    blob = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("w2_f64s.cu", "w2_slice.cuh"))
    h = hashlib.sha256(blob).hexdigest()[:16]
    return THETA_TRAFFIC.get(h)


def theta_flops_per_point(nk):
    """Algorithmic FP64 flops of one pseudo-difference operator per phase-space
    point: 2 nk multiply-adds for the one-body shifts along p1 and p2 plus the
    mean anti-diagonal length (sum_s len(s)^2 / nk^2) for the pair shift."""
    lens = [min(s + 1, 2 * nk - 1 - s) for s in range(2 * nk - 1)]
    diag = sum(l * l for l in lens) / (nk * nk)
    return 2.0 * (2 * nk + diag)


def bench_forms(args, barrier):
    """The precision and batching forms on their own workloads (rank-local)."""
    import torch

    from paper_2511_11354_gb300 import inputs, w2
    stream = torch.cuda.current_stream()
    forms = {}

    def timed(step, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        step(k)
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1)

    k = args.form_steps
    precisions = [("precision_tf32x3", w2.W2_F32_TF32X3), ("precision_bf16x3", w2.W2_F32_BF16X3)]
    for key, prec in ([] if args.no_precision else precisions):
        # precision form: 128^4, double-well physics, FP32 state, split contractions
        prob, _ = inputs.workload_dwell(nx=128, nk=128)
        f0 = inputs.initial_state_chunked(prob, centres=inputs.draw_centres(2), seed=2, dtype=np.float32)
        ctx = w2.Context.from_problem(prob, precision=prec)
        ctx.set_state(torch.from_numpy(f0).cuda())
        del f0
        ctx.step(args.warmup)
        k = args.form_steps
        ms = timed(ctx.step, k)
        kp = ctx.step_profile(min(k, 10))
        theta_ms = 0.5 * (kp[2] + kp[7])
        method = theta_flops_per_point(prob.nk) * prob.points
        theta_gbs = 24.0 * prob.points / ((kp[2] + kp[7]) * 1e-3) / 1e9   # 8 B/point predictor, 16 corrector
        if prec == w2.W2_F32_TF32X3:
            kname = "k_theta32 (TF32 split contractions, mma.sync m16n8k8)"
            flops = 4 * theta_mma_per_block(prob.nk) * 2048.0 * prob.nx * prob.nx  # 4 products, 2048 flop per mma
            peak = 0.4889 * MEASURED_BF16_TFLOPS()
            peak_name, peak_src = "tf32_peak", ("0.4889 x measured cuBLAS bf16 burst (MEASURED_PEAKS.json), nominal "
                                                "tf32/bf16 ratio 1.1/2.25")
            what = "the emulation's own work: 4 TF32 split products per product"
        else:
            kname = "k_theta_b3 (BF16 split contractions, mma.sync m16n8k16)"
            flops = sliced_mma_per_block(prob.nk) * 7 / SLICE_PAIRS * 4096.0 * prob.nx * prob.nx
            peak = MEASURED_BF16_TFLOPS()
            peak_name, peak_src = "bf16_peak", "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"
            what = "the emulation's own work: 7 BF16 split products per product"
        forms[key] = {
            "workload": f"double-well physics on a 128^2 x 128^2 grid (268M points), FP32 state, dt={prob.dt:g}",
            "value": prob.points * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
            "kernel_ms": dict(zip(w2.STEP_KERNELS, [float(x) for x in kp])),
            "roofline_theta": {"bound": "hbm", "kernel": kname,
                               "achieved": theta_gbs, "peak": MEASURED_HBM_GBS(), "unit": "GB/s",
                               "frac": theta_gbs / MEASURED_HBM_GBS(),
                               "bytes_rule": "predictor 8 B/point (f in, Theta f out), corrector 16 B/point "
                                             "(f~, f and the increment in, f out)",
                               "method_flops_per_launch": method,
                               "method_tflops": method / (theta_ms * 1e-3) / 1e12,
                               "method_frac_of_" + peak_name: method / (theta_ms * 1e-3) / 1e12 / peak,
                               peak_name: peak, peak_name + "_source": peak_src,
                               "executed": {"what": what,
                                            "mma_tflops": flops / (theta_ms * 1e-3) / 1e12,
                                            "mma_frac_of_" + peak_name: flops / (theta_ms * 1e-3) / 1e12 / peak}},
            "step_hbm_frac": 36.0 * prob.points / (ms / k * 1e-3) / 1e9 / MEASURED_HBM_GBS(),
        }
        ctx.close()
        torch.cuda.empty_cache()
        # the same form on the 64^4 workload of the FP64 headline (same grid, same physics)
        p64, f64 = inputs.workload_dwell()
        c64 = w2.Context.from_problem(p64, precision=prec)
        c64.set_state(torch.from_numpy(f64.astype(np.float32)).cuda())
        c64.step(args.warmup)
        k64 = max(k, 20)
        ms64 = timed(c64.step, k64)
        forms[key]["on_64^4"] = {"value": p64.points * k64 / (ms64 / 1e3), "unit": UNIT, "steps": k64,
                                 "ms_per_step": ms64 / k64}
        c64.close()
        # its error against the FP64 path on the 64^4 workload after 500 steps (the
        # batching workload's length), observables every 50 steps
        if not args.no_form_error:
            p64, f64 = inputs.workload_dwell()
            a = w2.Context.from_problem(p64, precision=w2.W2_F64_SLICED)
            b = w2.Context.from_problem(p64, precision=prec)
            a.set_state(f64)
            b.set_state(f64.astype(np.float32))
            worst = {"mass": 0.0, "energy": 0.0, "entropy_lin_abs": 0.0, "n1_max_rel": 0.0, "n12_max_rel": 0.0}
            for _ in range(10):
                a.step(50)
                b.step(50)
                oa, ob = a.observables(), b.observables()
                cur = {"mass": abs(ob.mass - oa.mass) / abs(oa.mass), "energy": abs(ob.energy - oa.energy) / abs(oa.energy),
                       "entropy_lin_abs": abs(ob.entropy_lin - oa.entropy_lin),
                       "n1_max_rel": float(np.abs(ob.n1 - oa.n1).max() / np.abs(oa.n1).max()),
                       "n12_max_rel": float(np.abs(ob.n12 - oa.n12).max() / np.abs(oa.n12).max())}
                worst = {k: max(worst[k], cur[k]) for k in worst}
            fa, fb = a.get_state(), b.get_state().astype(np.float64)
            forms[key]["error_vs_fp64_path_64^4_500_steps"] = dict(
                rel_l2=float(np.linalg.norm(fb - fa) / np.linalg.norm(fa)),
                observables_worst_over_10_checkpoints=worst,
                reference="W2_F64_SLICED (held to the FP64 oracle at 1e-10)")
            a.close()
            b.close()
    # precision form on the paper's full plasma mesh (nonlinear Landau damping)
    if not args.no_plasma:
        forms["plasma_landau_256x128"] = bench_plasma(args, timed)
    # batching form: 64 uneven instances, one graph-captured persistent step
    if not args.no_batching:
        probs, states = inputs.workload_batch(64, seed=3)
        bt = w2.Batch(probs)
        for i, f in enumerate(states):
            bt.set_state(i, f.astype(np.float32))
        del states
        tuning = bt.autotune()
        bt.step(args.warmup)
        ms = timed(bt.step, k)
        pts = sum(p.points for p in probs)
        forms["batching"] = {
            "workload": "64 instances, nx in {24,32,48,64}, nk in {32,48,64}, gamma in U[0.2,2] (seed 3), "
                        f"{pts / 1e6:.1f}M points in total, FP32 state, TF32 split contractions",
            "value": pts * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
            "autotuned": tuning, "launches_per_step": 1}
        bt.close()
    if not args.no_learned:
        forms["learned"] = bench_learned(args, timed)
    if not args.no_sem:
        forms[f"nonperiodic_correlated_{args.sem_nx}x128"] = bench_sem(args, timed)
    return forms


def sem_flops(nx, np_):
    """Algorithmic FP64 flops of one non-periodic operator (2 per multiply-add):
    the one-body tables G = U-Toeplitz x psi, the products G1 F and F G2^T per
    point X, and the two-body chain per X (F Phi^T, Ph T, Eh B, S [Ei|Er]^T on
    the half y1 plane)."""
    Ny, Nyh = 2 * ((nx - 1) // 2) + 1, (nx - 1) // 2 + 1
    one = 2.0 * (2 * nx) * (2 * nx - 1) * np_ * np_ + 2.0 * nx * nx * 2 * np_ ** 3
    two = 2.0 * nx * nx * (2 * np_ * np_ * Ny + 2 * Nyh * 2 * np_ * Ny + 2 * np_ * 2 * Nyh * Ny + np_ * np_ * 2 * Ny)
    return one, two


def bench_sem(args, timed):
    """The strongly correlated example on the paper's mesh: 201^2 x (8 x 16)^2
    points (6.6e8) on [-15, 15]^2 x [-10 pi/3, 10 pi/3]^2, Hamiltonian IV
    (Hartree + Hedin-Lundqvist XC + smoothed Coulomb pair + external well,
    soft 1), dt = 0.01, FP64 state and results; the operator's products from
    exact slices on the BF16 tensor cores (W2_F64_SLICED), and the same
    operator on the FP64 pipe (W2_F64) timed beside it."""
    import torch

    from paper_2511_11354_gb300 import inputs, w2
    prob, f = inputs.workload_correlated("IV", soft=1.0, nx=args.sem_nx)
    d = torch.from_numpy(f).cuda()
    del f
    out = torch.empty_like(d)
    one, two = sem_flops(prob.nx, prob.np_)
    ctx = w2.SemContext.from_problem(prob, precision=w2.W2_F64_SLICED)
    ctx.set_state(d)
    ob0 = ctx.observables()
    ctx.step(1)
    k = max(1, args.sem_steps)
    ms = timed(ctx.step, k)
    ms_theta = timed(lambda n: ctx.theta(d, out), 1)
    ms_adv = timed(lambda n: ctx.advect(d, out), 1)
    ob = ctx.observables()
    t0 = time.perf_counter()
    occ, s_corr = ctx.occupations()
    ms_occ = 1e3 * (time.perf_counter() - t0)
    ctx.close()
    pipe = w2.SemContext.from_problem(prob, precision=w2.W2_F64)
    pipe.theta(d, out)
    ms_theta_pipe = timed(lambda n: pipe.theta(d, out), 1)
    pipe.close()
    pk = _pipe_peaks()
    peak64, mma_ceiling = pk["fp64_dfma_tflops"], pk["mma_sync_bf16_tflops"]
    bf16 = MEASURED_BF16_TFLOPS(sustained=True)
    sliced_flops = 21.0 * (one + two)
    ach = sliced_flops / (ms_theta * 1e-3) / 1e12
    ach64 = (one + two) / (ms_theta_pipe * 1e-3) / 1e12
    ach64s = (one + two) / (ms_theta * 1e-3) / 1e12
    res = {"workload": f"strongly correlated example, Hamiltonian IV, {prob.nx}^2 x 128^2 mesh "
                       f"({prob.points / 1e6:.0f}M points), box [-15, 15]^2, 8 Chebyshev cells x 16 points per "
                       "momentum axis, FP64 state, operator products from exact slices on the BF16 tensor cores, "
                       "dt = 0.01",
           "value": prob.points * k / (ms / 1e3), "unit": UNIT, "steps": k, "warmup": 1, "ms_per_step": ms / k,
           "theta_ms": ms_theta, "advect_ms": ms_adv,
           "roofline": {"bound": "tensor", "kernel": "k_gemms (sliced FP64 products, BF16 mma.sync m16n8k16)",
                        "achieved": ach64s, "peak": bf16, "unit": "TFLOP/s", "frac": ach64s / bf16,
                        "flops_per_operator": one + two,
                        "flops_rule": "the method's FP64 flops of the operator's products (2 per multiply-add) "
                                      "over the whole operator call (slicing, tables and densities included)",
                        "peak_source": "bf16_tflops_sustained of measured (MEASURED_PEAKS.json, cuBLAS)",
                        "executed": {"what": "the emulation's own work: 21 exact BF16 slice products per FP64 "
                                             "product", "slice_flops_per_operator": sliced_flops,
                                     "slice_tflops": ach, "slice_frac_of_bf16_peak": ach / bf16,
                                     "mma_sync_bf16_ceiling_tflops": mma_ceiling,
                                     "slice_frac_of_mma_sync_ceiling": ach / mma_ceiling,
                                     "ceiling_source": "register-only mma.sync m16n8k16 BF16 loop, measured live by "
                                                       "bench_pipe_peaks.cu"}},
           "fp64_pipe_path": {"theta_ms": ms_theta_pipe, "bound": "alu", "achieved": ach64, "peak": peak64,
                              "unit": "TFLOP/s", "frac": ach64 / peak64, "flops_per_operator": one + two,
                              "two_body_share_of_flops": two / (one + two),
                              "peak_source": "fp64_dfma_tflops measured live by "
                                             "bench_pipe_peaks.cu"},
           "mass_drift": (ob.mass - ob0.mass) / ob0.mass, "energy": ob.energy,
           "correlation_entropy": s_corr, "occupations_top3": [float(v) for v in occ[:3]], "occupations_ms": ms_occ}
    del d, out
    torch.cuda.empty_cache()
    return res


def bench_plasma(args, timed):
    """Nonlinear quantum Landau damping (eps = 0.1, k = 0.4) on the paper's
    mesh: 256^2 x 128^2 points (1.07e9), box [-5 pi, 5 pi)^2, momentum spacing
    0.1, neutralised Poisson Hartree, Hedin-Lundqvist XC, smoothed Coulomb
    pair (soft 1), dt = 0.01; the precision form (the FP64 paths stop at
    nk = 64).  The separable initial state is built on the device."""
    import torch

    from paper_2511_11354_gb300 import inputs, w2
    prob = inputs.plasma_problem("landau", nx=256, nk=128)
    a, b = inputs.plasma_factors(prob, "landau")
    at = torch.from_numpy(a.astype(np.float32)).cuda()
    bt = torch.from_numpy(b.astype(np.float32)).cuda()
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F32_TF32X3)
    f0 = (at[:, None, None, None] * at[None, :, None, None]) * (bt[None, None, :, None] * bt[None, None, None, :])
    ctx.set_state(f0.contiguous())
    del f0
    torch.cuda.empty_cache()
    ob0 = ctx.observables()
    ctx.step(args.warmup)
    k = max(3, min(args.form_steps, 10))
    ms = timed(ctx.step, k)
    kp = ctx.step_profile(3)
    ob = ctx.observables()
    out = {"workload": "nonlinear quantum Landau damping, 256^2 x 128^2 mesh (1.07e9 points), FP32 state, "
                       "TF32 split contractions, Poisson Hartree + H-L XC + smoothed Coulomb pair, dt = 0.01",
           "value": prob.points * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
           "kernel_ms": dict(zip(w2.STEP_KERNELS, [float(x) for x in kp])),
           "mass_drift": (ob.mass - ob0.mass) / ob0.mass, "status": ob.status}
    ctx.close()
    torch.cuda.empty_cache()
    return out


def bench_learned(args, timed):
    """Learned form on the 64^4 double-well workload: a kernel network (the
    two-body term's structure: linear in f with a shift kernel that depends
    on the pair distance; 4 layers, width 256, BF16 products, FP32
    accumulation) trained on snapshots of an exact trajectory (random spatial
    points of each) stands in for the two-body term.  Runs of args.learned_steps
    steps on the sliced FP64 path with the exact term judging the network every
    50 steps; speed on both FP64 paths."""
    import torch

    from paper_2511_11354_gb300 import inputs, learned, w2
    prob, f0 = inputs.workload_dwell()
    k = args.learned_steps
    snaps, per = args.learned_snapshots, 32
    t0 = time.perf_counter()
    F, P, D = learned.make_kernel_dataset(prob, f0, snapshots=snaps, stride=1, points_per_snapshot=per, seed=4)
    t_data = time.perf_counter() - t0
    mlp = w2.MLP(prob.nk, hidden=256, max_rows=prob.nx, kind="kernel")
    mlp.set_scales(1.0, 1.0, 3.0 * float(F.square().mean().sqrt()) / float(P.square().mean().sqrt()))
    t0 = time.perf_counter()
    losses = learned.train_kernel(mlp, prob, F, P, D, steps=args.learned_train_steps, batch=1024, lr=3e-3,
                                  lr_final=1e-5, seed=4)
    t_train = time.perf_counter() - t0
    del F, P, D
    torch.cuda.empty_cache()
    f0d = torch.from_numpy(f0).cuda()
    tol = 1e-2

    def make(prec, net=None, judge=0):
        c = w2.Context.from_problem(prob, precision=prec)
        c.set_state(f0d)
        if net is not None:
            c.attach_learned(net, judge, tol)
        return c

    zero = learned.zero_network(prob.nk, 32, prob.nx * prob.nx)
    out = {
        "workload": f"double-well physics on the 64^2 x 64^2 grid, FP64 step with the two-body term from a kernel "
                    f"network (the pair term's shift kernel per pair distance; 4 layers, width 256, BF16 products, "
                    f"FP32 accumulation) trained on {snaps} snapshots x {per} spatial points of an exact trajectory "
                    f"({args.learned_train_steps} Adam steps, batch 1024); judge every 50 steps, tolerance {tol}",
        "unit": UNIT, "steps": k, "dataset_s": t_data, "train_s": t_train,
        "train_rel_loss_first_last": [losses[0], float(np.mean(losses[-50:]))],
    }
    # accuracy over the long run on the sliced path (the exact term judges every 50 steps)
    exact = make(w2.W2_F64_SLICED)
    ms_exact = timed(exact.step, k)
    net = make(w2.W2_F64_SLICED, mlp, 50)
    ms_net = timed(net.step, k)
    rep = net.learned_report()
    nopair = make(w2.W2_F64_SLICED, zero)
    nopair.step(k)
    fe, fn, f0p = exact.get_state(), net.get_state(), nopair.get_state()
    out["sliced"] = {
        "value": prob.points * k / (ms_net / 1e3), "ms_per_step": ms_net / k, "exact_ms_per_step": ms_exact / k,
        "speedup_vs_exact": ms_exact / ms_net, "judge": rep,
        "rel_l2_vs_exact": float(np.linalg.norm(fn - fe) / np.linalg.norm(fe)),
        "rel_l2_without_two_body_term": float(np.linalg.norm(f0p - fe) / np.linalg.norm(fe)),
    }
    for c in (exact, net, nopair):
        c.close()
    # speed on the FP64-pipe path (a shorter run: it is 8x slower)
    kp = min(k, 50)
    exact = make(w2.W2_F64)
    ms_exact = timed(exact.step, kp)
    net = make(w2.W2_F64, mlp, 0)
    ms_net = timed(net.step, kp)
    out["fp64_pipe"] = {"value": prob.points * kp / (ms_net / 1e3), "steps": kp, "ms_per_step": ms_net / kp,
                        "exact_ms_per_step": ms_exact / kp, "speedup_vs_exact": ms_exact / ms_net}
    exact.close()
    net.close()
    out["value"] = out["sliced"]["value"]
    out["accuracy_note"] = ("the network's table replaces the exact pair table in the same sweep, so the step costs "
                            "what the exact step costs; its error is that of the learned kernel (BF16 network), "
                            "above the 1e-6 bar of the precision forms")
    mlp.close()
    zero.close()
    return out


SLICE_PAIRS = 21  # digit pairs (s, t), s + t <= 5, of the sliced FP64 sweep


def sliced_mma_per_block(nk):
    """mma.m16n8k16 instructions one k_theta_s block executes (all 21 digit
    pairs): the two dense one-body contractions plus the sheared pair tiles
    over the k-steps each tile group touches."""
    rt = nk // 16
    one_body = 2 * rt * (nk // 16) * SLICE_PAIRS * 2 * (nk // 16)
    pair = 0
    for r in range(rt):
        r0 = 16 * r
        cfirst, clast = r0 // 8, min((r0 + 15 + nk - 1) // 8, (2 * nk - 2) // 8)
        ntile = clast - cfirst + 1
        half = (ntile + 1) // 2
        for lo, hi in ((cfirst, cfirst + half), (cfirst + half, clast + 1)):
            c = lo
            while c < hi:
                nt = min(3, hi - c)
                klo = max(0, 8 * c - nk + 1) & ~15
                khi = min(nk - 1, 8 * (c + nt - 1) + 7)
                pair += len(range(klo, khi + 1, 16)) * SLICE_PAIRS * nt
                c += nt
    return one_body + pair


def theta_mma_per_block(nk):
    """mma.m16n8k8 tiles of one Theta block (per product): two dense nk x nk x nk
    contractions plus the sheared pair term over the k-steps it can touch."""
    dense = 2 * (nk // 16) * (nk // 8) * (nk // 8)
    pair = 0
    for w in range(nk // 16):
        r0 = 16 * w
        for c in range(r0 // 8, min((r0 + 15 + nk - 1) // 8, (2 * nk - 2) // 8) + 1):
            nlo, nhi = max(0, 8 * c - nk + 1), min(nk - 1, 8 * c + 7)
            pair += (nhi - (nlo & ~7)) // 8 + 1
    return dense + pair


def MEASURED_BF16_TFLOPS(sustained=False):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["bf16_tflops_sustained" if sustained else "bf16_tflops"])
    except Exception:
        return 1700.0 if sustained else 1900.0  # fallback figures of the profiling recipe


def MEASURED_HBM_GBS():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except Exception:
        return 6800.0  # fallback figure of the profiling recipe


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, whole Lawson
    steps of the same 64^4 workload (one warm-up step: the oracle has no state
    to warm).  At most --ref-max-steps steps are timed so that the arm ends
    within a few minutes; the line says how many."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2511_11354_gb300 import inputs
    oracle.build()
    prob, f0 = inputs.workload_dwell()
    o = oracle.Oracle(prob)
    f = o.step(f0, 1)
    n = max(1, min(args.steps, args.ref_max_steps))
    t0 = time.perf_counter()
    f = o.step(f, n)
    el = time.perf_counter() - t0
    value = prob.points * n / el
    sample = (f"{n} oracle Lawson step(s) of the full {prob.nx}^2 x {prob.nk}^2 workload after one untimed step "
              f"({el:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "steps_timed": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_desc(prob),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.Oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=250)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="w2", choices=["w2", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-max-steps", type=int, default=60,
                    help="reference arm: at most this many full oracle steps are timed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-form-error", action="store_true")
    ap.add_argument("--form-steps", type=int, default=20)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision form (for profiling commands)")
    ap.add_argument("--no-plasma", action="store_true", help="skip the plasma form (for profiling commands)")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching form (for profiling commands)")
    ap.add_argument("--no-sem", action="store_true", help="skip the non-periodic (spectral-element) form")
    ap.add_argument("--sem-steps", type=int, default=2)
    ap.add_argument("--sem-nx", type=int, default=201, help="spatial points per axis of the non-periodic form")
    ap.add_argument("--only-sem", action="store_true", help="run only the non-periodic form (for profiling commands)")
    ap.add_argument("--only-forms", action="store_true", help="run only the forms (for profiling commands)")
    ap.add_argument("--min-reps", type=int, default=5, help="repetitions of the K-step timed loop (at least)")
    ap.add_argument("--min-timed-seconds", type=float, default=2.0,
                    help="keep repeating the K-step timed loop until this much timed work")
    ap.add_argument("--learned-steps", type=int, default=1000)
    ap.add_argument("--learned-snapshots", type=int, default=2000)
    ap.add_argument("--learned-train-steps", type=int, default=12000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2511_11354_gb300 import build as w2build
    from paper_2511_11354_gb300 import inputs, w2

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w2build.build()
    if args.only_sem:
        def timed_only(step, k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            step(k)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        if rank == 0:
            print(json.dumps({"impl": "w2", "only_sem": True, "sem": bench_sem(args, timed_only)}), flush=True)
        return
    if args.only_forms:
        forms = bench_forms(args, torch.cuda.synchronize)
        if rank == 0:
            print(json.dumps({"impl": "w2", "only_forms": True, "forms": forms}), flush=True)
        return

    prob, f0 = inputs.workload_dwell()
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    f_dev = torch.from_numpy(f0).cuda()
    ctx.set_state(f_dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x):
        return x if ws == 1 else reduce_max(x, dist, "cuda")

    # ---- device-resident timed region: exactly K steps, repeated ----------
    # Each repetition times K graph-replayed steps between a barrier and a
    # synchronize; the line reports the median repetition (value, ms_per_step)
    # and the spread over all of them.  Repetitions continue until at least
    # --min-timed-seconds of timed work so that the clock sampler sees the
    # GPU under load.
    ctx.step(args.warmup)
    barrier()
    clocks = ClockSampler(local)
    rep_ms = []
    t_start = time.perf_counter()
    while True:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        ctx.step(args.steps)
        e1.record(stream)
        barrier()
        rep_ms.append(max_over_ranks(e0.elapsed_time(e1)))
        done = len(rep_ms) >= args.min_reps and time.perf_counter() - t_start >= args.min_timed_seconds
        if ws > 1:  # every rank takes the same decision
            done = reduce_max(1.0 if done else 0.0, dist, "cuda") > 0.5
        if done or len(rep_ms) >= 1000:
            break
    clk = clocks.stop()
    ms = statistics.median(rep_ms)
    ob = ctx.observables()
    value = whole_job_rate(prob.points, args.steps, ws, ms)
    reps = {"repetitions": len(rep_ms), "ms_per_step_median": ms / args.steps,
            "ms_per_step_min": min(rep_ms) / args.steps, "ms_per_step_max": max(rep_ms) / args.steps,
            "value_min": whole_job_rate(prob.points, args.steps, ws, max(rep_ms)),
            "value_max": whole_job_rate(prob.points, args.steps, ws, min(rep_ms)),
            "rule": "each repetition times exactly K steps between barriers; value and ms_per_step are the median"}
    # occupation numbers and correlation entropy of the evolved state (device, synchronous)
    ctx.occupations()
    t_occ = time.perf_counter()
    occ, s_corr = ctx.occupations()
    ms_occ = (time.perf_counter() - t_occ) * 1e3

    # ---- per-kernel times (events around every launch, same stream) -------
    kprof = ctx.step_profile(min(args.steps, 50))
    k_theta = 0.5 * (kprof[2] + kprof[7])
    fp64_flops = theta_flops_per_point(prob.nk) * prob.points   # the FP64 contraction of one sweep
    alg_flops = SLICE_PAIRS * fp64_flops                          # its 21 slice products
    exec_flops = sliced_mma_per_block(prob.nk) * 4096.0 * prob.nx * prob.nx
    bf16_peak = MEASURED_BF16_TFLOPS(sustained=True)
    theta_gbs = 40.0 * prob.points / ((kprof[2] + kprof[7]) * 1e-3) / 1e9
    shift_bytes = 32.0 * prob.points  # two arrays read and two written, 8 B each
    k_shift = kprof[4]
    step_bytes = 72.0 * prob.points   # algorithmic bytes of a whole step

    # ---- the same workload with exchange symmetry declared (the state is an
    # exchange-symmetrised product, so the sliced sweeps take the blocks with
    # i1 <= i2 and write the mirrors transposed); a secondary measurement:
    # the headline above runs every block
    sy = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    sy.set_exchange_symmetry(True)
    sy.set_state(f_dev)
    sy.step(args.warmup)
    sym_ms = []
    for _ in range(max(1, min(len(rep_ms), 5))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        sy.step(args.steps)
        e1.record(stream)
        barrier()
        sym_ms.append(max_over_ranks(e0.elapsed_time(e1)))
    ms_sym = statistics.median(sym_ms)
    kprof_sym = sy.step_profile(min(args.steps, 50))
    # agreement with the full sweep: the same number of steps from the same state
    chk_a = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    chk_a.set_state(f_dev)
    sy.set_state(f_dev)
    chk_a.step(20)
    sy.step(20)
    ga, gs = chk_a.get_state(), sy.get_state()
    sym_rel = float(np.linalg.norm(gs - ga) / np.linalg.norm(ga))
    del ga, gs
    chk_a.close()
    sy.close()
    sym_theta_gbs = 40.0 * prob.points / ((kprof_sym[2] + kprof_sym[7]) * 1e-3) / 1e9
    exchange_symmetric = {
        "what": "W2_F64_SLICED with w2_set_exchange_symmetry: the sweeps compute the blocks with i1 <= i2 and "
                "write each mirror block transposed (the workload's state is exchange symmetric); the headline "
                "value runs every block",
        "value": whole_job_rate(prob.points, args.steps, ws, ms_sym), "ms_per_step": ms_sym / args.steps,
        "kernel_ms": dict(zip(w2.STEP_KERNELS, [float(x) for x in kprof_sym])),
        "theta_roofline": {"bound": "hbm", "achieved": sym_theta_gbs, "peak": MEASURED_HBM_GBS(), "unit": "GB/s",
                           "frac": sym_theta_gbs / MEASURED_HBM_GBS(),
                           "bytes_rule": "the method's bytes of every block (16 B/point predictor, 24 corrector)"},
        "rel_l2_vs_full_sweep_after_20_steps": sym_rel,
    }

    # ---- the same workload with the sweeps' slice products on tcgen05 (MMA
    # into tensor memory) instead of mma.sync; a secondary measurement
    tc = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    tc.set_tensor_path(True)
    tc.set_state(f_dev)
    tc.step(args.warmup)
    tc_ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        tc.step(args.steps)
        e1.record(stream)
        barrier()
        tc_ms.append(max_over_ranks(e0.elapsed_time(e1)))
    ms_tc = statistics.median(tc_ms)
    kprof_tc = tc.step_profile(min(args.steps, 50))
    chk_a = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    chk_a.set_state(f_dev)
    tc.set_state(f_dev)
    chk_a.step(20)
    tc.step(20)
    ga, gt = chk_a.get_state(), tc.get_state()
    tc_rel = float(np.linalg.norm(gt - ga) / np.linalg.norm(ga))
    del ga, gt
    chk_a.close()
    tc.close()
    tcgen05_sweep = {
        "what": "W2_F64_SLICED with w2_set_tensor_path(1): the same 21 slice products on tcgen05 (BF16 operands "
                "in shared memory, FP32 accumulators in tensor memory, one CTA of 215 KB per SM); the headline "
                "runs them on mma.sync, the faster path for this operator",
        "value": whole_job_rate(prob.points, args.steps, ws, ms_tc), "ms_per_step": ms_tc / args.steps,
        "kernel_ms": dict(zip(w2.STEP_KERNELS, [float(x) for x in kprof_tc])),
        "rel_l2_vs_mma_sync_after_20_steps": tc_rel,
    }

    # ---- the FP64-pipe path (DMMA sweep, FP64 shift) on the same workload ---
    pipe = w2.Context.from_problem(prob)
    pipe.set_state(f_dev)
    pipe.step(args.warmup)
    kp = min(args.steps, 50)
    barrier()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    pipe.step(kp)
    p1.record(stream)
    barrier()
    ms_pipe = max_over_ranks(p0.elapsed_time(p1))
    kprof_pipe = pipe.step_profile(min(kp, 20))
    pipe.close()
    peaks = _pipe_peaks()
    k_theta_pipe = 0.5 * (kprof_pipe[2] + kprof_pipe[7])

    # ---- end to end through the C ABI: pinned host state in, observables out.
    # Each step's input is copied from the host (w2_stage_state: the copy of
    # step k+1's input runs on the context's copy stream during step k) and
    # its observables are copied back to the host (w2_observables_enqueue into
    # one of two pinned slots) and read by the host while step k+1 runs
    # (w2_observables_collect); the last step's are read before the clock stops.
    ctx.set_state(f_dev)
    ctx.step(1)
    host = torch.from_numpy(f0).pin_memory()
    h2d = host.numel() * host.element_size()
    d2h = 8 * (8 + prob.nx + prob.nx * prob.nx)
    for _ in range(2):  # warm-up: the step graph of each of the two state buffers is captured here
        ctx.stage_state(host)
        ctx.use_staged_state()
        ctx.step(1)
        ctx.observables()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    torch.cuda.synchronize()  # the first copy starts after t0
    ctx.stage_state(host)
    e2e_obs = []
    for k in range(args.steps):
        ctx.use_staged_state()
        if k + 1 < args.steps:
            ctx.stage_state(host)
        ctx.step(1)
        ctx.observables_enqueue(k % 2)
        if k > 0:
            e2e_obs.append(ctx.observables_collect((k - 1) % 2))
    e2e_obs.append(ctx.observables_collect((args.steps - 1) % 2))
    t1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(t0.elapsed_time(t1))
    e2e = whole_job_rate(prob.points, args.steps, ws, ms_e2e)

    ctx.close()
    forms = None if args.no_forms else bench_forms(args, barrier)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = _oracle_sample(prob, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _workload_desc(prob),
            "clocks": clk, "timing": reps,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "pipeline": "w2_stage_state copies step k+1's input from pinned host memory during step k; "
                                "w2_use_staged_state takes it in (the staging and state buffers trade places, "
                                "then the new state's per-X sums); every step's observables are copied to "
                                "pinned host memory (w2_observables_enqueue) and read by the host while the "
                                "next step runs (w2_observables_collect)"},
            "gpu_launches": (len(w2.STEP_KERNELS) - 1) * args.steps,
            "gpu_launches_rule": "launches of this library's kernels in one timed repetition of K steps (7 per "
                                 "step: slot 0 of the step profile, the per-X sums of f^n, comes from the "
                                 "previous corrector and launches nothing)",
            "roofline": {"bound": "hbm", "kernel": "k_theta_s (sliced FP64 sweep, BF16 mma.sync m16n8k16)",
                         "achieved": theta_gbs, "peak": MEASURED_HBM_GBS(), "unit": "GB/s",
                         "frac": theta_gbs / MEASURED_HBM_GBS(), "traffic": _theta_traffic(),
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "peak_source": "hbm_gbs of measured (MEASURED_PEAKS.json, copy)",
                         "bytes_rule": "algorithmic: predictor reads f and writes Theta f (16 B/point), corrector "
                                       "reads f~ and h and writes f (24 B/point); achieved = both launches' bytes "
                                       "over both launches' time",
                         "bytes_per_launch": {"predictor": 16.0 * prob.points, "corrector": 24.0 * prob.points},
                         "ms_per_launch": {"predictor": float(kprof[2]), "corrector": float(kprof[7])},
                         "why_hbm": "the method's own work, 2 (2 nk + mean anti-diagonal) FP64 flop per point "
                                    "(341 at nk = 64) over 16-24 B per point, is under the ridge point of the BF16 "
                                    "tensor peak, so HBM is the binding roofline of the contraction",
                         "method_fp64_flops_per_launch": fp64_flops,
                         "method_fp64_tflops": fp64_flops / (k_theta * 1e-3) / 1e12,
                         "method_fp64_frac_of_bf16_peak": fp64_flops / (k_theta * 1e-3) / 1e12 / bf16_peak,
                         "bf16_peak": bf16_peak,
                         "bf16_peak_source": "bf16_tflops_sustained of measured (MEASURED_PEAKS.json, cuBLAS)",
                         "executed": {"what": "the emulation's own work, not the method's: 21 exact BF16 slice "
                                              "products per FP64 product",
                                      "slice_flops_per_launch": alg_flops, "mma_flops_per_launch": exec_flops,
                                      "slice_tflops": alg_flops / (k_theta * 1e-3) / 1e12,
                                      "mma_sync_bf16_ceiling_tflops": peaks["mma_sync_bf16_tflops"],
                                      "mma_frac_of_mma_sync_ceiling":
                                          exec_flops / (k_theta * 1e-3) / 1e12 / peaks["mma_sync_bf16_tflops"],
                                      "ceiling_source": "register-only mma.sync m16n8k16 BF16 loop, measured live "
                                                        "by bench_pipe_peaks.cu"}},
            "roofline_shift": {"bound": "hbm", "kernel": "k_adv_df<64,1,1> (x1 lines, double-float)",
                               "achieved": shift_bytes / (k_shift * 1e-3) / 1e9,
                               "peak": MEASURED_HBM_GBS(), "unit": "GB/s",
                               "frac": shift_bytes / (k_shift * 1e-3) / 1e9 / MEASURED_HBM_GBS(),
                               "bytes_per_launch": shift_bytes, "ms_per_launch": k_shift,
                               "peak_source": "hbm_gbs of measured (MEASURED_PEAKS.json)"},
            "step_hbm_frac": step_bytes / (ms / args.steps * 1e-3) / 1e9 / MEASURED_HBM_GBS(),
            "kernel_ms": dict(zip(w2.STEP_KERNELS, [float(x) for x in kprof])),
            "exchange_symmetric": exchange_symmetric,
            "tcgen05_sweep": tcgen05_sweep,
            "fp64_pipe_path": {
                "what": "W2_F64: DMMA m8n8k4 sweep and FP64 spline shift on the FP64 pipe, same workload",
                "value": whole_job_rate(prob.points, kp, ws, ms_pipe), "unit": UNIT, "steps": kp,
                "ms_per_step": ms_pipe / kp,
                "kernel_ms": dict(zip(w2.STEP_KERNELS, [float(x) for x in kprof_pipe])),
                "theta_fp64_tflops": fp64_flops / (k_theta_pipe * 1e-3) / 1e12,
                "fp64_dmma_peak_tflops": peaks["fp64_dmma_tflops"], "fp64_dfma_peak_tflops": peaks["fp64_dfma_tflops"],
                "peak_source": "measured live by bench_pipe_peaks.cu"},
            "observables": {"mass": ob.mass, "energy": ob.energy, "entropy_lin": ob.entropy_lin,
                            "status": ob.status, "correlation_entropy": s_corr,
                            "occupations_top3": [float(v) for v in occ[:3]],
                            "occupations_ms": ms_occ},
            "cpu_baseline": cpu,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
