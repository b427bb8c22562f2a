"""Benchmark of the FBC Green's-function pad update on GB300.

One step = one pad update u <- G f (forward line transform with the neutral
projection, per-mode contraction, inverse transform) of the largest
single-GPU workload: N_I = 8000 interface and N_P = 12000 pad columns on
concentric rings, L = 1024 repeats, 64 right-hand sides of N(0, 1) forces
(seed 4), isotropic medium (mu = 1, nu = 0.3).  Metric: pad updates as
Gpair-modes/s, one pair-mode being one (pad column, interface column,
wavenumber k = 0..L/2, right-hand side) 3x3 block product.  The timed form
is the dense per-mode contraction at FP64 accuracy: with several right-hand
sides on the tensor cores (six fixed-point bf16 slices per operand, exact
FP32 accumulation per slice diagonal), with one in double-float on the FP32
pipes.  The double-float form, the reduced-precision tensor-core forms and
the in-plane FFT forms are measured beside it, each with its error against
the FP64 oracle per mode band.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision P] [--surrogate]

Prints ONE JSON line on rank 0.  ``--impl reference`` times the CPU oracle
(the plain FP64 real-space sum) on the host cores instead, on a bounded
sample of the same workload (some repeats of one pad column per step).
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

WORKLOAD = "ring8000x12000_L1024_rhs64_iso"
METRIC = "FBC pad updates/sec (Gpair-modes/s) at stated error vs FP64 oracle; roofline fraction"
UNIT = "Gpair-modes/s"
FLOPS_PER_PAIR_MODE = 36  # useful: two real 3x3 matrix-vector products (x and y' halves) = 18 MACs
X2_INSTR_PER_MAC = 10     # double-float MAC: 1 FMUL + 3 FFMA + 6 FADD (each one FP32-pipe lane slot)
L2_BYTES = 129 * 1024 * 1024
VARIANT_SECONDS = 8.0     # time budget of each beside-measured form (after one untimed step)


def peaks(n_sm: int = 152):
    """Roofline denominators: the measured copy bandwidth and bf16 rates, and the CUDA-core peaks derived
    from unit counts (n_sm SMs read from the device, 128 FP32 FMA lanes per SM per clock) and the maximum
    SM clock; FP64 at the GB300 nominal 1.25 TFLOP/s scaled to that clock."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    if os.path.exists(path):
        with open(path) as fh:
            m = json.load(fh)
        out.update({k: m[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "sm_max_mhz") if k in m})
        out["source"] = "measured"
    clk = out["sm_max_mhz"] * 1e6
    out["n_sm"] = n_sm
    out["fp32_tflops"] = n_sm * 128 * 2 * clk / 1e12
    out["fp32_tinstr"] = n_sm * 128 * clk / 1e12
    out["fp64_tflops"] = 1.25 * clk / 2.07e9 * n_sm / 152
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


def sample_columns(n_p: int, n: int = 8) -> np.ndarray:
    """Pad columns at whose every repeat the oracle checks the result: the n/2 innermost and the n/2
    outermost of the ring order (the innermost carry the largest high-mode terms)."""
    h = n // 2
    return np.array(sorted(set(range(min(h, n_p))) | set(range(max(0, n_p - (n - h)), n_p))), dtype=np.int64)


def oracle_table(w, xy_i, xy_p_cols, rich=(4, 6)):
    """The oracle's real-space kernel for the differences of the given pad columns (setup, untimed)."""
    import oracle

    oracle.build()
    d_list, d_index = oracle.difference_index(xy_i, xy_p_cols)
    t0 = time.perf_counter()
    table = oracle.kernel_table(w.material, w.L, w.c, d_list, n=rich[0], N=rich[1], nquad=64)
    return d_index, table, time.perf_counter() - t0


def oracle_check(w, xy_i, xy_p, f, cols, rows, out):
    """The oracle's side of the error check (into ``out``): the real-space sum at every repeat of the
    sampled pad columns for the sampled right-hand sides, and the Richardson truncation of the kernel
    itself -- Eq. 36 at the plan's (n, N) = (4, 6) against (8, 8), the most accurate order (pinned against
    the brute-force image sum of Eq. 32 in the oracle tests) -- at the innermost sampled column."""
    try:
        import oracle

        nt = max(1, oracle.n_threads() - 2)
        fp = oracle.project_neutral(f[rows])
        oracle.build()
        d_list, d_index = oracle.difference_index(xy_i, xy_p[cols])
        t0 = time.perf_counter()
        table = oracle.kernel_table(w.material, w.L, w.c, d_list, nquad=64, nthreads=nt)
        out["t_table"] = time.perf_counter() - t0
        samp_col = np.repeat(np.arange(len(cols)), w.L).astype(np.int32)
        samp_p = np.tile(np.arange(w.L), len(cols)).astype(np.int32)
        t0 = time.perf_counter()
        out["ref"] = oracle.real_space_sum(d_index, table, fp, samp_col, samp_p, nthreads=nt).reshape(
            len(rows), len(cols), w.L, 3)
        out["t_check"] = time.perf_counter() - t0
        out["threads"] = nt
        del table
        d1, di1 = oracle.difference_index(xy_i, xy_p[cols[:1]])
        sc, sp = np.zeros(w.L, np.int32), np.arange(w.L, dtype=np.int32)
        u = {}
        for nN in ((4, 6), (8, 8)):
            t = oracle.kernel_table(w.material, w.L, w.c, d1, n=nN[0], N=nN[1], nquad=64, nthreads=nt)
            u[nN] = oracle.real_space_sum(di1, t, fp[:1], sc, sp, nthreads=nt)
        out["trunc"] = {"rich": [4, 6], "vs_rich": [8, 8],
                        "rel_l2": float(np.linalg.norm(u[(4, 6)] - u[(8, 8)]) / np.linalg.norm(u[(8, 8)])),
                        "sample": f"every repeat of pad column {int(cols[0])}, right-hand side {rows[0]}",
                        "note": "the error of the tabulated kernel itself against the periodic Green function "
                                "of Eq. 32 (rel_l2_vs_oracle compares with the oracle's own (4, 6) kernel)"}
    except Exception as e:  # reported by the main thread
        out["error"] = repr(e)


def cpu_sample(w):
    """The bounded sample both CPU measurements time: repeats 0..n-1 (n = min(L, 128)) of pad column 0,
    right-hand side 0, as a share of the whole update's N_P L n_rhs pad atoms."""
    n_rep = min(w.L, 128)
    return n_rep, n_rep / float(w.n_p * w.L * w.n_rhs)


def run_reference(args, w):
    """CPU oracle arm: time the plain real-space sum on a bounded sample of the workload."""
    import oracle

    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    xy_i, xy_p = w.geometry()
    # right-hand side 0 alone: the generator fills [n_rhs][n_i][L][3] in order, so this is forces()[:1]
    fp = oracle.project_neutral(inputs.forces(1, w.n_i, w.L, w.seed))
    n_rep, share = cpu_sample(w)
    d_index, table, t_table = oracle_table(w, xy_i, xy_p[:1])
    samp_col = np.zeros(n_rep, dtype=np.int32)
    samp_p = np.arange(n_rep, dtype=np.int32)
    for _ in range(args.warmup):
        oracle.real_space_sum(d_index, table, fp, samp_col, samp_p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.real_space_sum(d_index, table, fp, samp_col, samp_p)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = w.pair_modes * share / dt / 1e9
    # the same sum on one core, over a quarter of the sample's pad atoms (after the timed steps)
    m1 = max(1, n_rep // 4)
    t1 = time.perf_counter()
    oracle.real_space_sum(d_index, table, fp, samp_col[:m1], samp_p[:m1], nthreads=1)
    t_one = time.perf_counter() - t1
    info = oracle.sys_info()
    sample = (f"{n_rep} pad atoms (repeats 0..{n_rep - 1} of pad column 0, right-hand side 0) per step: the full "
              f"real-space sum over {w.n_i} x {w.L} interface atoms each, {share:.3g} of the update; kernel "
              f"tabulation for the sample ({t_table:.1f} s) is setup and untimed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_i": w.n_i, "n_p": w.n_p, "L": w.L, "n_rhs": w.n_rhs,
                   "material": w.material.get("kind"), "sampled": True},
        "extrapolated_full_update_ms": dt / share * 1e3,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle", "sample": sample,
                         "cpu": info["cpu"],
                         "one_core": {"value": w.pair_modes * share * (m1 / n_rep) / t_one / 1e9, "unit": UNIT,
                                      "cores": 1, "sample": f"repeats 0..{m1 - 1} of pad column 0, once ({t_one:.1f} s)"}},
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


# tensor-core products per block product (split terms; bf16x6: the 26 fixed-point slice products)
TENSOR = {"tf32": 1, "bf16x2": 3, "bf16x3": 6, "bf16x6": 26}
DTYPE = {"fp64": "f64", "f32x2": "f32x2 (double-float, FP64-accurate)", "fp32": "f32",
         "tf32": "tf32 x f32-accumulate (k = 0 in double-float)",
         "bf16x2": "bf16 2-term split x f32-accumulate (k = 0 in double-float)",
         "bf16x3": "bf16 3-term split x f32-accumulate (k = 0 in double-float)",
         "fft64": "f64 (in-plane FFT form)",
         "fft32": "f32 (in-plane FFT form; k = 0 in f64)",
         "bf16x6": "bf16 6-slice fixed-point split x exact f32 accumulation (FP64-accurate; k = 0 in double-float)"}
FFT = ("fft64", "fft32")


def mode_bands(L):
    """k = 0, low 1..L/8, high L/8+1..L/2 (reading of the mode bands)."""
    return {"k0": (0, 0), "low": (1, L // 8), "high": (L // 8 + 1, L // 2)}


def band_errors(got, ref, L):
    """Relative L2 error per mode band of pad-column lines (got, ref: [..., L, 3], the line on axis -2)."""
    E = np.fft.rfft(got - ref, axis=-2)
    R = np.fft.rfft(ref, axis=-2)
    out = {}
    for name, (lo, hi) in mode_bands(L).items():
        out[name] = float(np.linalg.norm(E[..., lo:hi + 1, :]) / max(np.linalg.norm(R[..., lo:hi + 1, :]), 1e-300))
    return out


def launches_per_apply(precision, info):
    """Kernels one apply launches: forward, projection, contraction (k = 0 separately for the FP32 and
    tensor forms, plus the tensor forms' split of the force operand; per streamed chunk: network, near
    copy, contraction), inverse."""
    K = info["K"]
    if precision in FFT:
        R, Q = info["max_rhs"], max(1, info["fft_chunk_items"])
        if precision == "fft64":
            return 2 + 3 * -(-(R * K) // Q) + 1
        return 2 + 3 * (-(-R // Q) - (-(R * (K - 1)) // min(2 * Q, 65535))) + 1
    if info.get("surrogate_attached"):
        chunks = -(-(K - 1) // max(1, info["surrogate_chunk"]))
        contract = 1 + 3 * chunks
    elif precision in ("fp64", "f32x2"):
        contract = 1
    elif precision == "bf16x6":
        contract = 4  # k = 0, force scales, force slices, contraction
    elif precision in TENSOR:
        contract = 3
    else:
        contract = 2
    return 2 + contract + 1


def contraction_roofline(p, pm, contract_ms, pk):
    """Roofline of the per-mode contraction stage: ALGORITHMIC work = 36 useful flops per pair-mode (two
    real 3x3 matrix-vector products) over the stage's time, against the peak of the arithmetic the form
    runs on; what the form actually issues (split products, double-float instructions) is reported beside."""
    t = contract_ms * 1e-3
    useful = FLOPS_PER_PAIR_MODE * pm / t / 1e12
    if p in TENSOR:
        base = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        peak = base * (1.1 / 2.25 if p == "tf32" else 1.0)
        src = ("measured sustained bf16 dense" + (" x nominal tf32/bf16 ratio 1.1/2.25" if p == "tf32" else "")
               + f" ({pk['source']})")
        issued = {"what": f"{TENSOR[p]} {'tf32' if p == 'tf32' else 'bf16'} products per useful product",
                  "tflops": TENSOR[p] * useful, "frac": TENSOR[p] * useful / peak}
        return {"bound": "tensor", "achieved": useful, "peak": peak, "unit": "TFLOP/s", "frac": useful / peak,
                "peak_source": src, "issued": issued}
    if p == "fp64":
        return {"bound": "alu", "achieved": useful, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
                "frac": useful / pk["fp64_tflops"],
                "peak_source": "FP64 nominal 1.25 TFLOP/s scaled to the maximum SM clock (not measured)"}
    peak = pk["fp32_tflops"]
    src = (f"FP32 FMA: {pk['n_sm']} SMs x 128 lanes x 2 flops x maximum SM clock (derived from unit counts, "
           "not measured)")
    out = {"bound": "alu", "achieved": useful, "peak": peak, "unit": "TFLOP/s", "frac": useful / peak,
           "peak_source": src}
    if p == "f32x2":
        per_pm = (FLOPS_PER_PAIR_MODE // 2) * X2_INSTR_PER_MAC
        ti = per_pm * pm / t / 1e12
        out["issued"] = {"what": f"FP32-pipe lane instructions, {X2_INSTR_PER_MAC} per double-float MAC "
                                 f"({per_pm} per pair-mode)", "t_instr_per_s": ti, "peak_t_instr_per_s":
                         pk["fp32_tinstr"], "frac": ti / pk["fp32_tinstr"]}
    elif p in FFT:
        out["effective"] = ("the in-plane FFT form does O(M log M) work per mode, not 36 flops per pair-mode: "
                            "achieved counts the dense form's useful flops (an effective rate)")
    return out


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
    pk = peaks(torch.cuda.get_device_properties(local).multi_processor_count)
    pk["probe_fp32_tflops"] = fbc.fbc_measure_fma_peak(False)
    pk["probe_fp64_tflops"] = fbc.fbc_measure_fma_peak(True)
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
    cols = sample_columns(w.n_p, 8)
    rows = sorted({0, R - 1})
    cols_d = torch.as_tensor(cols, device="cuda")
    # the oracle's side of the error check needs only f and the geometry: it runs on the host cores (all
    # but two, left to the launching thread) while the device is timed, and is joined before the end-to-end
    # measurement, whose copies share the host's memory bandwidth
    check_thread, check_out = None, {}
    if rank == 0 and not args.skip_oracle:
        import threading

        check_thread = threading.Thread(target=oracle_check, args=(w, xy_i, xy_p, f, cols, rows, check_out),
                                        daemon=True)
        check_thread.start()

    def snap():
        return ud.index_select(0, torch.as_tensor(rows, device="cuda")).index_select(1, cols_d).cpu().numpy()

    variants, outputs = {}, {}

    def time_capped(p1, budget_s, cap):
        """One untimed step, then as many timed steps as fit the budget (at least 1, at most cap)."""
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        flush_buf.zero_()
        p1.apply(fd, ud)
        torch.cuda.synchronize()
        one = time.perf_counter() - t1
        n = int(max(1, min(cap, budget_s // max(one, 1e-3))))
        return time_device_steps(torch, p1, fd, ud, n, 0, flush_buf) + (n,)

    def variant(prec):
        plan.set_precision(prec)
        vms, vstage, n = time_capped(plan, VARIANT_SECONDS, max(2, args.steps // 2))
        outputs[prec] = snap()
        variants[prec] = {"ms_per_step": float(np.mean(vms)), "value": pm / (np.mean(vms) * 1e-3) / 1e9,
                          "contract_ms": float(vstage[1]), "steps": n, "dtype": DTYPE[prec]}
        if prec in FFT:
            variants[prec]["note"] = "effective rate: pair-modes of the dense form per second"

    surrogate = None
    if args.surrogate:
        # ablation: the same plan with its exact tables first, then with the learned far field
        variant(args.precision)
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

    # the other forms on the same plan and inputs (not after the tables were released); the dense FP64
    # form, several times slower than double-float at the same accuracy, only at one right-hand side
    if not args.surrogate and not args.no_variants:
        others = (("fp64", "f32x2", "fp32", "fft64", "fft32") if R == 1
                  else ("f32x2", "bf16x6", "fp32", "tf32", "bf16x2", "bf16x3", "fft64", "fft32"))
        for prec in others:
            if prec != args.precision:
                variant(prec)
        plan.set_precision(args.precision)
        if R == 1:
            variants["harmonic_step"] = time_harmonic_step(torch, fbc, plan, w, xy_i, xy_p, ud,
                                                           max(3, args.steps // 2), flush_buf)
        if R > 1 and w.n_i > 1024:
            # BF16x2 with the whole interface sum in one tensor-memory accumulation group
            with fbc.Plan(xy_i, xy_p, w.L, w.material, precision="bf16x2", max_rhs=R,
                          tc_fast_accumulate=True) as p1:
                p1.tabulate()
                vms, vstage, n = time_capped(p1, VARIANT_SECONDS, max(2, args.steps // 2))
                outputs["fast_accumulate"] = snap()
                variants["fast_accumulate"] = {"precision": "bf16x2", "ms_per_step": float(np.mean(vms)),
                                               "value": pm / (np.mean(vms) * 1e-3) / 1e9,
                                               "contract_ms": float(vstage[1]), "steps": n}

    if args.hmatrix:
        # the paper's comparison form (Sec. 3.2, App.): the H-matrix of the same Green matrix at the paper's
        # settings, built once (setup), applied like the plan
        t1 = time.perf_counter()
        try:
            H = fbc.HMatrix(plan, eps=1e-5, gamma=2.0, b_min=20)
        except fbc.FBCError as exc:  # e.g. the factors do not fit on the device at this size
            H = None
            variants["hmatrix"] = {"unavailable": str(exc), "eps": 1e-5, "gamma": 2.0, "b_min": 20,
                                   "build_s": time.perf_counter() - t1}
            torch.cuda.empty_cache()
    if args.hmatrix and H is not None:
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t1
        hi = H.info()

        class _HApply:  # the interface time_device_steps uses; the H-matrix has no stage events
            def apply(self, f_, u_, **kw):
                return H.apply(f_, u_, **kw)

            def set_timing(self, on):
                pass

            def stage_times(self):
                return [0.0, 0.0, 0.0]

            def sync_status(self):
                pass

        vms, _, n = time_capped(_HApply(), VARIANT_SECONDS, max(2, args.steps // 2))
        outputs["hmatrix"] = snap()
        dense_bytes = 9.0 * w.n_p * w.n_i * w.L * w.L * 4
        variants["hmatrix"] = {"ms_per_step": float(np.mean(vms)), "value": pm / (np.mean(vms) * 1e-3) / 1e9,
                               "steps": n, "dtype": "f32 factors, double-float sums",
                               "note": "effective rate: pair-modes of the dense form per second",
                               "eps": 1e-5, "gamma": 2.0, "b_min": 20, "build_s": build_s,
                               "factor_bytes": hi["factor_bytes"] + hi["dense_bytes"],
                               "dense_matrix_fp32_bytes": dense_bytes,
                               "factor_gbs": (hi["factor_bytes"] + hi["dense_bytes"]) / (np.mean(vms) * 1e-3) / 1e9,
                               "n_lowrank": hi["n_lowrank"], "n_dense": hi["n_dense"], "rank_sum": hi["rank_sum"],
                               "rank_max": hi["rank_max"], "n_capped": hi["n_capped"], "n_waves": hi["n_waves"]}
        H.close()
        torch.cuda.empty_cache()

    # end-to-end through the host entry point: pinned host f in, host u out, in the headline form
    if check_thread is not None:
        check_thread.join()
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.zeros((R, w.n_p, w.L, 3), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    plan.apply_host(fh, uh)
    one = time.perf_counter() - t1
    e2e_t = []
    for _ in range(int(max(2, min(max(3, args.steps // 2), 2 * VARIANT_SECONDS // max(one, 1e-3))))):
        flush_buf.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        plan.apply_host(fh, uh)
        e2e_t.append(time.perf_counter() - t1)
    e2e_s = job_step_ms(float(np.mean(e2e_t)) * 1e3, world, dist if world > 1 else None) * 1e-3
    h2d = f.nbytes
    d2h = uh.numel() * 8
    del fh, uh

    # error against the FP64 oracle at every repeat of the sampled pad columns for right-hand sides 0 and
    # R - 1, per mode band; the Richardson truncation of the kernel; the CPU baseline
    errors, bands, cpu, trunc = {}, {}, None, None
    if rank == 0 and not args.skip_oracle:
        import oracle

        if "error" in check_out:
            raise RuntimeError(f"oracle check failed: {check_out['error']}")
        ref = check_out["ref"]
        for name, u in outputs.items():
            errors[name] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
            bands[name] = band_errors(u, ref, w.L)
        trunc = check_out["trunc"]
        fp = oracle.project_neutral(f[:1])
        # timed oracle on the bounded sample of the reference arm, repeated to ~10 s of CPU work
        n_rep, share = cpu_sample(w)
        d0, t0_, _ = oracle_table(w, xy_i, xy_p[:1])
        sc0, sp0 = np.zeros(n_rep, np.int32), np.arange(n_rep, dtype=np.int32)
        reps, t_cpu = 0, 0.0
        while t_cpu < 10.0 and reps < 200:
            t1 = time.perf_counter()
            oracle.real_space_sum(d0, t0_, fp[:1], sc0, sp0)
            t_cpu += time.perf_counter() - t1
            reps += 1
        # the same sum on one core, over a quarter of the sample's pad atoms
        m1 = max(1, n_rep // 4)
        t1 = time.perf_counter()
        oracle.real_space_sum(d0, t0_, fp[:1], sc0[:m1], sp0[:m1], nthreads=1)
        t_one = time.perf_counter() - t1
        sinfo = oracle.sys_info()
        cpu = {"value": pm * share / (t_cpu / reps) / 1e9, "unit": UNIT, "cores": sinfo["cores"], "kind": "oracle",
               "one_core": {"value": pm * share * (m1 / n_rep) / t_one / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"repeats 0..{m1 - 1} of pad column 0, right-hand side 0, once ({t_one:.1f} s)"},
               "sample": (f"real-space sum at {n_rep} pad atoms (repeats 0..{n_rep - 1} of pad column 0, right-hand "
                          f"side 0) x {reps} repetitions ({t_cpu:.1f} s): {share:.3g} of the update per repetition; "
                          "kernel tabulation for the sample untimed"),
               "cpu": sinfo["cpu"]}
        for name in variants:
            if name in errors:
                variants[name]["rel_l2_vs_oracle"] = errors[name]
                variants[name]["rel_l2_by_band"] = bands[name]
        check = {"pad_columns": [int(c) for c in cols], "rhs": rows, "repeats": "all",
                 "oracle_s": check_out["t_check"], "oracle_table_s": check_out["t_table"],
                 "oracle_threads": check_out["threads"]}
    else:
        check = None

    p = args.precision
    contract_ms = float(stage[1])
    roof = contraction_roofline(p, pm, contract_ms, pk)
    if roof["bound"] == "alu":
        # the unit-count peak above is the denominator; the probe's measured rate stands beside it
        probe = pk.get("probe_fp64_tflops" if p == "fp64" else "probe_fp32_tflops")
        if probe:
            roof["measured_peak"] = {"tflops": probe, "frac": roof["achieved"] / probe,
                                     "how": "fbc_measure_fma_peak: 8 independent FMA chains per thread, "
                                            "8 x 256 threads per SM, CUDA events"}
            if "t_instr_per_s" in roof.get("issued", {}):
                roof["issued"]["frac_of_measured"] = roof["issued"]["t_instr_per_s"] / (probe / 2.0)
    roof["kernel"] = {"f32x2": "k_contract_x2_rb" if R > 1 else "k_contract_x2", "fp64": "k_contract_fp64",
                      "bf16x6": "k_contract_oz",
                      "fp32": "k_contract_fp32_rb" if R > 1 else "k_contract_fp32"}.get(
        p, "k_contract_tc" if p in TENSOR else "k_fft_* (in-plane FFT contraction)")
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "contract_traffic.json")
    if os.path.exists(tpath) and not args.surrogate:
        with open(tpath) as fh_:
            tr = json.load(fh_)
        ent = tr.get(f"{w.name}/{p}")
        if ent and ent.get("source_sha256") == source_digest(ent.get("sources", [])):
            traffic = ent.get("dram_bytes_per_apply_contraction")
    roof["traffic"] = traffic
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
        "error_check": check,
        "kernel_truncation": trunc,
        "setup_s": setup_s,
        "stage_ms": {"forward": float(stage[0]), "contract": contract_ms, "inverse": float(stage[2])},
        "roofline": roof,
        "variants": variants,
        "e2e": {"value": job_value(pm, world, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3, "steps": len(e2e_t)},
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


def run_batch(args):
    """The batched workload: 64 uneven instances (N_I ~ U[500, 8000], N_P = 1.5 N_I, L in {32, ..., 512}),
    16 right-hand sides each, rhs j scaled by 0.5^j.  One step = one update of every instance by the batch:
    batched line transforms and one persistent contraction launch over all instances' work items, replayed
    from a CUDA graph (the autotuned configuration).  Beside it: the same update as a loop of per-plan
    applies, and other precisions.  Error: every repeat of pad column 0 of every instance, right-hand side
    0, against the oracle."""
    import torch

    from paper_2105_08798_gb300 import build as fbc_build
    from paper_2105_08798_gb300 import fbc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fbc_build.build()
    fbc.load()
    pk = peaks(torch.cuda.get_device_properties(local).multi_processor_count)
    specs = inputs.batch_instances()
    prec = args.precision
    t0 = time.perf_counter()
    plans, fs, us, geo, pm = [], [], [], [], 0.0
    for sp in specs:
        xy_i, xy_p = inputs.ring_geometry(sp["n_i"], sp["n_p"])
        f = inputs.forces(sp["n_rhs"], sp["n_i"], sp["L"], sp["seed"], decay=0.5)
        p = fbc.Plan(xy_i, xy_p, sp["L"], sp["material"], precision=prec, max_rhs=sp["n_rhs"])
        p.tabulate()
        plans.append(p)
        fs.append(torch.from_numpy(f).cuda())
        us.append(torch.zeros((sp["n_rhs"], sp["n_p"], sp["L"], 3), dtype=torch.float64, device="cuda"))
        geo.append((xy_i, xy_p, f[:1]))
        pm += sp["n_p"] * sp["n_i"] * (sp["L"] // 2 + 1) * sp["n_rhs"]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    check_out = {}
    if not args.skip_oracle:
        import threading

        def check():
            try:
                import oracle

                nt = max(1, oracle.n_threads() - 2)
                out = []
                for sp, (xy_i, xy_p, f0) in zip(specs, geo):
                    L = sp["L"]
                    d_list, d_index = oracle.difference_index(xy_i, xy_p[:1])
                    table = oracle.kernel_table(sp["material"], L, 1.0, d_list, nthreads=nt)
                    out.append(oracle.real_space_sum(d_index, table, oracle.project_neutral(f0),
                                                     np.zeros(L, np.int32), np.arange(L, dtype=np.int32),
                                                     nthreads=nt)[0])
                check_out["ref"] = out
            except Exception as e:  # reported by the main thread
                check_out["error"] = repr(e)

        th = threading.Thread(target=check, daemon=True)
        th.start()
    else:
        th = None
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def time_it(fn, steps, warmup):
        for _ in range(warmup):
            flush_buf.zero_()
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush_buf.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    batch = fbc.Batch(plans, fs, us)
    batch.apply()
    tune_ms = batch.autotune()
    info = batch.info()
    with ClockSampler(local) as clk:
        ms = time_it(lambda: batch.apply(stream=stream), args.steps, args.warmup)
    plans[0].sync_status()
    outs = [u[0, 0].cpu().numpy() for u in us]
    step_ms = float(np.mean(ms))
    variants = {}

    def loop():
        for p, f, u in zip(plans, fs, us):
            p.apply(f, u, stream=stream)

    lms = time_it(loop, max(2, args.steps // 2), 1)
    variants["per_plan_loop"] = {"precision": prec, "ms_per_step": float(np.mean(lms)),
                                 "value": pm / (np.mean(lms) * 1e-3) / 1e9,
                                 "note": "the same update as one fbc_apply per instance (each with its own launches)"}
    batch.close()
    for other in ("fp32", "bf16x2", "tf32"):
        if other == prec:
            continue
        for p in plans:
            p.set_precision(other)
        with fbc.Batch(plans, fs, us) as b2:
            b2.apply()
            b2.autotune()
            vms = time_it(lambda: b2.apply(stream=stream), max(2, args.steps // 2), 1)
        variants[f"batch_{other}"] = {"ms_per_step": float(np.mean(vms)), "value": pm / (np.mean(vms) * 1e-3) / 1e9}
    errors = None
    if th is not None:
        th.join()
        if "error" in check_out:
            raise RuntimeError(f"oracle check failed: {check_out['error']}")
        per = [float(np.linalg.norm(o - r) / np.linalg.norm(r)) for o, r in zip(outs, check_out["ref"])]
        errors = {"max": max(per), "median": float(np.median(per)), "per_instance": per,
                  "sample": "every repeat of pad column 0 of each instance, right-hand side 0"}
    for p in plans:
        p.close()
    line = {
        "metric": METRIC, "value": pm / (step_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": "batch64_rhs16_iso", "instances": len(specs), "n_rhs": 16,
                   "pair_modes": pm, "precision": prec, "l2": "flushed between steps (256 MB write)",
                   "graph": True, "parallelism": "single"},
        "batch": {"autotuned_contract_ms": tune_ms, "rhs_per_cta": info.get("rhs_per_cta"),
                  "launch_form": ["one persistent launch over all items", "per-instance launches in the graph"][
                      info.get("launch_form", 0)],
                  "grid": info["grid"], "lpt_order": info["lpt_order"], "work_items": info["n_contract_items"],
                  "kernel_launches": info["kernel_launches"]},
        "rel_l2_vs_oracle": errors, "setup_s": setup_s, "variants": variants,
        "gpu_launches": info["kernel_launches"] * args.steps, "clocks": clk.summary(),
        "peaks": {"bf16_tflops_sustained": pk.get("bf16_tflops_sustained")},
    }
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--precision", choices=["fp64", "f32x2", "fp32", "tf32", "bf16x2", "bf16x3", "fft64", "fft32",
                                                "bf16x6"],
                    default=None,
                    help="contraction form of the timed steps (default: the dense FP64-accurate form, bf16x6 "
                         "with several right-hand sides, f32x2 with one)")
    ap.add_argument("--workload", choices=sorted(inputs.WORKLOADS) + ["batch"], default=WORKLOAD,
                    help="a named single instance, or 'batch': 64 uneven instances with 16 right-hand sides each")
    ap.add_argument("--surrogate", action="store_true",
                    help="train the learned far field (width 128, 2^20 samples, 50 epochs), attach it with "
                         "r_min = 8 and release the K-slice tables; the exact-table path is timed first")
    ap.add_argument("--skip-oracle", action="store_true", help="no oracle error check / CPU baseline")
    ap.add_argument("--no-variants", action="store_true",
                    help="time the headline form only (no other forms beside it), e.g. for a launch list")
    ap.add_argument("--hmatrix", action="store_true",
                    help="also build the H-matrix of the same Green matrix (eps 1e-5, gamma 2, b_min 20) and time "
                         "its apply as a variant")
    args = ap.parse_args(argv)
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no reference arm; "
                              "run the single-instance workloads"}), flush=True)
            return 0
        if args.precision is None:
            args.precision = "bf16x2"
        return run_batch(args)
    w = inputs.WORKLOADS[args.workload]
    if args.precision is None:
        args.precision = "bf16x6" if w.n_rhs > 1 and not args.surrogate else "f32x2"
    if args.surrogate and args.precision not in ("fp32", "tf32", "bf16x2", "bf16x3"):
        ap.error("--surrogate serves the FP32 and tensor-core precisions")
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
