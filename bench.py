"""Benchmark of the FBC Green's-function pad update on GB300.

One step = one pad update u <- G f (forward line transform with the neutral
projection, per-mode contraction, inverse transform) of the paper-scale
single instance: N_I = 4000 interface and N_P = 6000 pad columns on
concentric rings, L = 256 repeats, cubic medium C11 = 1.5, C12 = 1.0,
C44 = 0.9, one right-hand side of N(0, 1) forces (seed 1).  Metric: pad
updates as Gpair-modes/s, one pair-mode being one (pad column, interface
column, wavenumber k = 0..L/2, right-hand side) 3x3 block product.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  ``--impl reference`` times the CPU oracle
(the plain FP64 real-space sum) on the host cores instead; see the design
notes for how its sample is extrapolated.
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

from paper_2105_08798_gb300 import inputs  # noqa: E402

WORKLOAD = "ring4000x6000_L256_cubic"
METRIC = "FBC pad updates/sec (Gpair-modes/s) at stated error vs FP64 oracle; roofline fraction"
UNIT = "Gpair-modes/s"
FLOPS_PER_PAIR_MODE = 36  # two real 3x3 matrix-vector products (x and y' halves)
X2_INSTR_PER_MAC = 12     # double-float MAC: 1 FMUL + 3 FFMA + 8 FADD (each one FP32-pipe lane slot)
L2_BYTES = 129 * 1024 * 1024


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    if os.path.exists(path):
        with open(path) as fh:
            m = json.load(fh)
        out.update({k: m[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "sm_max_mhz") if k in m})
        out["source"] = "measured"
    # plain-ALU peaks from unit counts and the maximum SM clock: 152 SMs,
    # 128 FP32 FMA lanes per SM per clock; FP64 at the GB300 nominal 1.25 TFLOP/s
    clk = out["sm_max_mhz"] * 1e6
    out["fp32_tflops"] = 152 * 128 * 2 * clk / 1e12
    out["fp32_tinstr"] = 152 * 128 * clk / 1e12
    out["fp64_tflops"] = 1.25 * clk / 2.07e9
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"fbc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_forces(w, rank: int):
    """Replicas: rank r updates its own instance of the workload, with forces seeded seed + r."""
    return w.forces(seed=w.seed + rank)


def job_step_ms(step_ms: float, world: int, dist=None, device="cuda") -> float:
    """The whole job's step time: the maximum over ranks of each rank's own CUDA-event time."""
    if world > 1:
        import torch

        t = torch.tensor([step_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    return step_ms


def job_value(pair_modes: float, world: int, step_ms: float) -> float:
    """Whole-job throughput in Gpair-modes/s: the pair-modes of all ranks over the slowest rank's step."""
    return world * pair_modes / (step_ms * 1e-3) / 1e9


def oracle_sample(w, xy_i, xy_p, f, n_cols: int = 1):
    """The oracle's bounded sample: every repeat of the first n_cols pad columns
    (all of their differences are tabulated first, as setup)."""
    import oracle

    oracle.build()
    cols = np.arange(n_cols)
    samples = np.array([[a, p] for a in cols for p in range(w.L)], dtype=np.int64)
    fp = oracle.project_neutral(f)
    d_list, d_index = oracle.difference_index(xy_i, xy_p[cols])
    t0 = time.perf_counter()
    table = oracle.kernel_table(w.material, w.L, w.c, d_list, nquad=64)
    t_table = time.perf_counter() - t0
    samp_col = np.repeat(np.arange(n_cols), w.L).astype(np.int32)
    samp_p = np.tile(np.arange(w.L), n_cols).astype(np.int32)
    return samples, fp, d_index, table, samp_col, samp_p, t_table


def run_reference(args, w):
    """CPU oracle arm: time the plain real-space sum on a bounded sample."""
    import oracle

    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    xy_i, xy_p = w.geometry()
    f = w.forces()[:1]  # one right-hand side per sampled step; extrapolated over all of them below
    samples, fp, d_index, table, samp_col, samp_p, t_table = oracle_sample(w, xy_i, xy_p, f)
    for _ in range(args.warmup):
        oracle.real_space_sum(d_index, table, fp, samp_col, samp_p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.real_space_sum(d_index, table, fp, samp_col, samp_p)
    dt = (time.perf_counter() - t0) / args.steps
    # extrapolate one sampled step (len(samples) pad atoms, one right-hand side) to the whole update
    # (N_P L pad atoms for each of the n_rhs right-hand sides)
    t_full = dt * (w.n_p * w.L * w.n_rhs) / len(samples)
    value = w.pair_modes / t_full / 1e9
    info = oracle.sys_info()
    sample = (f"{len(samples)} pad atoms (all {w.L} repeats of 1 pad column, 1 right-hand side) per step, full "
              f"real-space sum over {w.n_i} x {w.L} interface atoms; extrapolated "
              f"x{w.n_p * w.L * w.n_rhs // len(samples)} to the whole update; "
              f"kernel tabulation for the sample ({t_table:.1f} s) is setup and untimed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_full * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_i": w.n_i, "n_p": w.n_p, "L": w.L, "n_rhs": w.n_rhs,
                   "material": w.material.get("kind"), "sampled": True},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle", "sample": sample,
                         "cpu": info["cpu"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_device_steps(torch, plan, fd, ud, steps, warmup, flush_buf, project=True):
    """Per-step CUDA events around the apply on the launching stream; L2 flushed between steps."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush_buf.zero_()
        plan.apply(fd, ud, project=project, stream=stream)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stage = np.zeros(3)
    plan.set_timing(True)
    for i in range(steps):
        flush_buf.zero_()
        starts[i].record(stream)
        plan.apply(fd, ud, project=project, stream=stream)
        ends[i].record(stream)
        stage += np.asarray(plan.stage_times())  # waits for this step's events
    plan.set_timing(False)
    torch.cuda.synchronize()
    plan.sync_status()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return ms, stage / steps


def time_harmonic_step(torch, fbc, plan, w, xy_i, xy_p, ud, steps, flush_buf):
    """One iteration of the harmonic half of Algorithm 1 on the device: the incompatibility force of the
    synthetic spring model (Eq. 21) from the core, interface and pad displacements, then the relaxed pad
    update (Algorithm 2 with the du_max cap) and the zero mean (Eq. 23).  Inputs resident, L2 flushed."""
    R, L = w.n_rhs, w.L
    xy_c = inputs.core_sites(w.n_i)
    K = fbc.fbc_spring_constants(1.0, 0.4, 1.0)
    gen = torch.Generator(device="cuda").manual_seed(7)
    u_c = 0.05 * torch.randn((R, len(xy_c), L, 3), dtype=torch.float64, device="cuda", generator=gen)
    u_i = 0.05 * torch.randn((R, w.n_i, L, 3), dtype=torch.float64, device="cuda", generator=gen)
    fs = [torch.empty((R, w.n_i, L, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
    alpha = torch.ones(R, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    with fbc.Stencil(xy_i, [xy_c, xy_i, xy_p], L, K) as st:
        def one(it):
            st.incompat_force([u_c, u_i, ud], f=fs[it % 2], stream=stream)
            plan.apply_relaxed(fs[it % 2], fs[(it + 1) % 2] if it else None, ud, alpha, du_max=0.02,
                               zero_mean=True, stream=stream)

        for it in range(3):
            flush_buf.zero_()
            one(it)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        ev_f = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush_buf.zero_()
            ev[i][0].record(stream)
            ev_f[i][0].record(stream)
            st.incompat_force([u_c, u_i, ud], f=fs[i % 2], stream=stream)
            ev_f[i][1].record(stream)
            plan.apply_relaxed(fs[i % 2], fs[(i + 1) % 2], ud, alpha, du_max=0.02, zero_mean=True, stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        plan.sync_status()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ms_f = float(np.mean([a.elapsed_time(b) for a, b in ev_f]))
    prec = {v: k for k, v in fbc.PRECISIONS.items()}[plan.info()["precision"]]
    return {"precision": prec, "ms_per_step": ms, "incompat_force_ms": ms_f,
            "value": w.pair_modes / (ms * 1e-3) / 1e9, "core_sites": len(xy_c),
            "model": "spring k1 = 1, k2 = 0.4, c = 1; du_max = 0.02; zero mean"}


TENSOR = {"tf32": 1, "bf16x2": 3, "bf16x3": 6}  # tensor-core products per block product (split terms)
DTYPE = {"fp64": "f64", "f32x2": "f32x2 (double-float, FP64-accurate)", "fp32": "f32",
         "tf32": "tf32 x f32-accumulate (k = 0 in double-float)",
         "bf16x2": "bf16 2-term split x f32-accumulate (k = 0 in double-float)",
         "bf16x3": "bf16 3-term split x f32-accumulate (k = 0 in double-float)",
         "fft64": "f64 (in-plane FFT form)",
         "fft32": "f32 (in-plane FFT form; k = 0 in f64)"}


def mode_bands(L):
    """k = 0, low 1..L/8, high L/8+1..L/2 (reading of the mode bands)."""
    return {"k0": (0, 0), "low": (1, L // 8), "high": (L // 8 + 1, L // 2)}


def band_errors(got, ref, L):
    """Relative L2 error per mode band of one pad column's line (got, ref: [L][3])."""
    E = np.fft.rfft(got - ref, axis=0)
    R = np.fft.rfft(ref, axis=0)
    out = {}
    for name, (lo, hi) in mode_bands(L).items():
        out[name] = float(np.linalg.norm(E[lo:hi + 1]) / max(np.linalg.norm(R[lo:hi + 1]), 1e-300))
    return out


def launches_per_apply(precision, info):
    """Kernels one apply launches: forward, projection, contraction (k = 0 separately for the FP32 and
    tensor forms; per streamed chunk: network, near copy, contraction), inverse."""
    K = info["K"]
    if precision in ("fft64", "fft32"):
        R, Q = info["max_rhs"], max(1, info["fft_chunk_items"])
        if precision == "fft64":
            return 2 + 3 * -(-(R * K) // Q) + 1
        return 2 + 3 * (-(-R // Q) - (-(R * (K - 1)) // min(2 * Q, 65535))) + 1
    if info.get("surrogate_attached"):
        chunks = -(-(K - 1) // max(1, info["surrogate_chunk"]))
        contract = 1 + 3 * chunks
    elif precision in ("fp64", "f32x2"):
        contract = 1
    else:
        contract = 2
    return 2 + contract + 1


def run_ours(args, w):
    import torch

    from paper_2105_08798_gb300 import build as fbc_build
    from paper_2105_08798_gb300 import fbc

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    fbc_build.build()
    fbc.load()
    pk = peaks()
    R = w.n_rhs
    xy_i, xy_p = w.geometry()
    f = rank_forces(w, rank)
    t0 = time.perf_counter()
    plan = fbc.Plan(xy_i, xy_p, w.L, w.material, precision=args.precision, max_rhs=R)
    plan.tabulate()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros((R, w.n_p, w.L, 3), dtype=torch.float64, device="cuda")
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    pm = w.pair_modes
    keep = 2  # pad columns whose outputs are kept for the error check (all rhs 0 and R-1 repeats)
    rows = sorted({0, R - 1})

    def snap():
        return ud[rows, :keep].cpu().numpy()

    variants, outputs = {}, {}

    def variant(prec, steps):
        plan.set_precision(prec)
        vms, vstage = time_device_steps(torch, plan, fd, ud, steps, 2, flush_buf)
        outputs[prec] = snap()
        variants[prec] = {"ms_per_step": float(np.mean(vms)), "value": pm / (np.mean(vms) * 1e-3) / 1e9,
                          "contract_ms": float(vstage[1])}

    surrogate = None
    if args.surrogate:
        # ablation: the same plan with its exact tables first, then with the learned far field
        variant(args.precision, max(2, args.steps // 2))
        variants["exact_table"] = variants.pop(args.precision)
        outputs["exact_table"] = outputs.pop(args.precision)
        t1 = time.perf_counter()
        S = fbc.Surrogate(width=128, seed=1)
        loss = S.train(plan, n_samples=1 << 20, r_min=8.0, epochs=50, batch=4096, lr=2e-3, seed=2)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t1
        before = plan.info()
        plan.attach_surrogate(S, r_min=8.0, release_tables=True)
        after = plan.info()
        surrogate = {"width": 128, "r_min": 8.0, "train_samples": 1 << 20, "epochs": 50, "train_s": train_s,
                     "final_loss": loss, "far_differences": after["n_far_d"], "used_differences": after["n_used_d"],
                     "chunk_modes": after["surrogate_chunk"],
                     "table_bytes_released": before["table_bytes"] + before["workspace_bytes"]
                     - after["workspace_bytes"],
                     "surrogate_bytes": after["surrogate_bytes"]}

    # headline (a plan with released tables keeps its precision)
    if not args.surrogate:
        plan.set_precision(args.precision)
    info = plan.info()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, stage = time_device_steps(torch, plan, fd, ud, args.steps, args.warmup, flush_buf)
    torch.cuda.synchronize()
    step_ms = job_step_ms(float(np.sum(ms)) / args.steps, world, dist if world > 1 else None)
    value = job_value(pm, world, step_ms)
    outputs["headline"] = snap()

    # the other precisions on the same plan and inputs (not after the tables were released); at the
    # multi-rhs sizes the FP64 and double-float forms (tens of seconds per step) are left out
    if not args.surrogate:
        others = (("fp64", "f32x2", "fp32", "fft64", "fft32") if R == 1
                  else ("fp32", "tf32", "bf16x2", "bf16x3", "fft64", "fft32"))
        for prec in others:
            if prec != args.precision:
                variant(prec, max(2, args.steps // 2))
        plan.set_precision(args.precision)
        if R == 1:
            variants["harmonic_step"] = time_harmonic_step(torch, fbc, plan, w, xy_i, xy_p, ud,
                                                           max(3, args.steps // 2), flush_buf)
        if args.precision in TENSOR and w.n_i > 1024:
            # the same precision with the whole interface sum in one tensor-memory accumulation group
            with fbc.Plan(xy_i, xy_p, w.L, w.material, precision=args.precision, max_rhs=R,
                          tc_fast_accumulate=True) as p1:
                p1.tabulate()
                vms, vstage = time_device_steps(torch, p1, fd, ud, max(2, args.steps // 2), 2, flush_buf)
                outputs["fast_accumulate"] = snap()
                variants["fast_accumulate"] = {"precision": args.precision, "ms_per_step": float(np.mean(vms)),
                                               "value": pm / (np.mean(vms) * 1e-3) / 1e9,
                                               "contract_ms": float(vstage[1])}

    # end-to-end through the host entry point: pinned host f in, host u out
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.zeros((R, w.n_p, w.L, 3), dtype=torch.float64).pin_memory()
    for _ in range(2):
        plan.apply_host(fh, uh)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        flush_buf.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        plan.apply_host(fh, uh)
        e2e_t.append(time.perf_counter() - t1)
    e2e_s = job_step_ms(float(np.mean(e2e_t)) * 1e3, world, dist if world > 1 else None) * 1e-3
    h2d = f.nbytes
    d2h = uh.numel() * 8
    del fh, uh

    # error against the FP64 oracle at the sampled pad atoms (all repeats of the first pad column, right-hand
    # sides 0 and R-1), per mode band, and the CPU baseline
    errors, bands, cpu = {}, {}, None
    if rank == 0 and not args.skip_oracle:
        import oracle

        samples, fp, d_index, table, samp_col, samp_p, t_table = oracle_sample(w, xy_i, xy_p, f[rows])
        ref = oracle.real_space_sum(d_index, table, fp, samp_col, samp_p)  # [len(rows)][L][3]
        for name, u in outputs.items():
            got = u[:, samples[:, 0], samples[:, 1]]
            errors[name] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            bands[name] = band_errors(got[0], ref[0], w.L)
        # timed oracle sum on the same sample (one right-hand side), repeated to ~10 s of CPU work
        fp1 = np.ascontiguousarray(fp[:1])
        reps, t_cpu = 0, 0.0
        while t_cpu < 10.0 and reps < 200:
            t1 = time.perf_counter()
            oracle.real_space_sum(d_index, table, fp1, samp_col, samp_p)
            t_cpu += time.perf_counter() - t1
            reps += 1
        t_full = (t_cpu / reps) * (w.n_p * w.L * R) / len(samples)
        sinfo = oracle.sys_info()
        cpu = {"value": pm / t_full / 1e9, "unit": UNIT, "cores": sinfo["cores"], "kind": "oracle",
               "sample": (f"real-space sum at {len(samples)} pad atoms (1 pad column, all repeats, 1 right-hand "
                          f"side) x {reps} repetitions ({t_cpu:.1f} s), extrapolated to N_P L n_rhs = "
                          f"{w.n_p * w.L * R} pad-atom updates; kernel tabulation for the sample ({t_table:.1f} s) "
                          f"untimed"),
               "cpu": sinfo["cpu"]}
        for name in variants:
            variants[name]["rel_l2_vs_oracle"] = errors.get(name)
            variants[name]["rel_l2_by_band"] = bands.get(name)

    # roofline of the dominant kernel (the per-mode contraction stage, timed by the plan's events on the
    # launching stream over the timed steps)
    contract_ms = float(stage[1])
    p = args.precision
    if p in TENSOR:
        # issued split products (TENSOR[p] bf16/tf32 products per block product), 36 flops each
        achieved = TENSOR[p] * FLOPS_PER_PAIR_MODE * pm / (contract_ms * 1e-3) / 1e12
        base = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        peak = base * (1.1 / 2.25 if p == "tf32" else 1.0)
        peak_name = ("measured sustained bf16 dense" + (" x nominal tf32/bf16 ratio 1.1/2.25" if p == "tf32" else "")
                     + f" ({pk['source']})")
        bound = "tensor"
    elif p == "fp64":
        achieved = FLOPS_PER_PAIR_MODE * pm / (contract_ms * 1e-3) / 1e12
        peak, peak_name, bound = pk["fp64_tflops"], "fp64 nominal 1.25 TFLOP/s scaled to max SM clock", "alu"
    else:
        # CUDA-core FP32-pipe work: FFMA, FMUL and FADD each take one lane-slot of the FMA pipes, so the
        # ceiling is an instruction rate: 152 SMs x 128 lanes x max SM clock
        per_pm = (FLOPS_PER_PAIR_MODE // 2) * (X2_INSTR_PER_MAC if p == "f32x2" else 1)
        achieved = per_pm * pm / (contract_ms * 1e-3) / 1e12
        peak, bound = pk["fp32_tinstr"], "alu"
        peak_name = ("FP32-pipe lane instructions: 152 SM x 128 lanes x max SM clock; "
                     f"{per_pm} per pair-mode ({'12 per double-float MAC' if p == 'f32x2' else '1 FFMA per MAC'})")
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "contract_traffic.json")
    if os.path.exists(tpath) and not args.surrogate:
        with open(tpath) as fh_:
            tr = json.load(fh_)
        ent = tr.get(f"{w.name}/{p}")
        if ent and ent.get("source_sha256") == source_digest(ent.get("sources", [])):
            traffic = ent.get("dram_bytes_per_apply_contraction")
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[p] + (" with learned far field" if args.surrogate else ""),
        "data": "synthetic",
        "config": {"workload": w.name, "n_i": w.n_i, "n_p": w.n_p, "L": w.L, "n_rhs": R,
                   "material": w.material.get("kind"), "precision": p, "surrogate": bool(args.surrogate),
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "rel_l2_vs_oracle": errors.get("headline"),
        "rel_l2_by_band": bands.get("headline"),
        "setup_s": setup_s,
        "stage_ms": {"forward": float(stage[0]), "contract": contract_ms, "inverse": float(stage[2])},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s" if p in TENSOR or p == "fp64" else "T FP32-pipe instr/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_name,
                     "useful_tflops": FLOPS_PER_PAIR_MODE * pm / (contract_ms * 1e-3) / 1e12},
        "variants": variants,
        "e2e": {"value": job_value(pm, world, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3},
        "gpu_launches": launches_per_apply(p, info) * args.steps,
        "clocks": clocks,
        "plan": {k: info[k] for k in ("n_tiles_a", "n_tiles_b", "sub_w", "sub_h", "n_used_d", "table_bytes",
                                      "workspace_bytes")},
    }
    if surrogate is not None:
        line["surrogate"] = surrogate
    if cpu is not None:
        line["cpu_baseline"] = cpu
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def source_digest(files):
    """SHA-256 over the named source files (relative to the repository root); '' if any is missing."""
    import hashlib

    h = hashlib.sha256()
    for rel in files:
        path = os.path.join(ROOT, rel)
        if not os.path.exists(path):
            return ""
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "f32x2", "fp32", "tf32", "bf16x2", "bf16x3", "fft64", "fft32"],
                    default=None,
                    help="contraction precision (default: f32x2 for one right-hand side, bf16x2 for several)")
    ap.add_argument("--workload", choices=sorted(inputs.WORKLOADS), default=WORKLOAD)
    ap.add_argument("--surrogate", action="store_true",
                    help="train the learned far field (width 128, 2^20 samples, 50 epochs), attach it with "
                         "r_min = 8 and release the K-slice tables; the exact-table path is timed first")
    ap.add_argument("--skip-oracle", action="store_true", help="no oracle error check / CPU baseline")
    args = ap.parse_args(argv)
    w = inputs.WORKLOADS[args.workload]
    if args.precision is None:
        args.precision = "f32x2" if w.n_rhs == 1 else "bf16x2"
    if args.surrogate and args.precision not in ("fp32", "tf32", "bf16x2", "bf16x3"):
        ap.error("--surrogate serves the FP32 and tensor-core precisions")
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
