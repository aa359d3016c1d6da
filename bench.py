"""Benchmark: energy+gradient evaluations per second of split-CTMRG on GB300.

One step = one call of the engine's ``energy_grad``: initial environment,
`sweeps` full directional steps (left, top, right, bottom), 2x2-patch energy,
and the reverse pass through all of it.  Workload (default): 2x2 cell, d=2,
D=8, chi=128, J1-J2 Heisenberg with J2/J1=0.5, seeded N(0,1) tensors with a
Neel-biased component (synthetic; ipeps_inputs.config("d8_chi128_2x2_j1j2")).

Prints one JSON line (rank 0).  Run ``--impl reference`` to time the FP64 CPU
oracle on the same workload (bounded sample, host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ipeps_inputs as I  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64, nominal (about 152 SMs x 2.07 GHz x 4 flop/clk/SM)
TC_CORNER_DRAM_BYTES = 6.576915e9 + 0.52181376e9   # ncu, tc_gemm_kernel on one 8192^3 product
SLICE_CORNER_DRAM_BYTES = 6.583486e9 + 0.520848e9  # ncu, slice_gemm_kernel on one 8192^3 product


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(name, sweeps):
    A, c = I.config(name)
    if c["rotated"]:
        h_nn, h_diag = I.heisenberg_bond_rotated(), None
    else:
        h_nn = I.heisenberg_bond()
        h_diag = c["J2"] * I.heisenberg_bond() if c["J2"] else None
    if sweeps is None:
        sweeps = c["sweeps"]
    desc = (f"{name}: {c['Lx']}x{c['Ly']} cell, d={c['p']}, D={c['D']}, chi={c['chi']}, "
            f"{'rotated ' if c['rotated'] else ''}Heisenberg J1=1" + (f", J2={c['J2']}" if c["J2"] else "")
            + f", {sweeps} directional sweeps per evaluation")
    return A, c, h_nn, h_diag, sweeps, desc


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


CPU_WORKLOAD, CPU_SWEEPS = "d4_chi32_2x2", 2


def oracle_evaluation(name=CPU_WORKLOAD, sweeps=CPU_SWEEPS):
    """One whole energy+gradient evaluation of the FP64 oracle (initial
    environment, `sweeps` full steps, 2x2 energy, reverse-mode autograd) on the
    host cores, timed; returns (seconds, energy, threads)."""
    import torch
    from oracle import ctmrg as C
    from oracle import energy as En
    torch.set_num_threads(os.cpu_count() or 1)
    A, c, h_nn, h_diag, _, _ = workload(name, sweeps)
    t0 = time.perf_counter()
    Ao = torch.tensor(A).requires_grad_(True)
    Ac = [[Ao[x, y] for y in range(c["Ly"])] for x in range(c["Lx"])]
    e = En.energy_per_site(Ac, C.split_ctmrg(Ac, c["chi"], sweeps), h_nn, h_diag)
    e.backward()
    return time.perf_counter() - t0, float(e.detach()), torch.get_num_threads()


def cpu_baseline(name, c, A, h_nn, h_diag, sweeps, budget_s=20.0):
    """The FP64 oracle timed on the host cores: one whole energy+gradient
    evaluation of the 2x2, D=4, chi=32 workload (2 sweeps), which it finishes
    in seconds.  The D=8 workload takes the oracle hours per evaluation; its
    figure is reported beside as an estimate scaled from a bounded sample
    (``estimate_of``, see d8_estimate), not as a timing."""
    t, e, threads = oracle_evaluation()
    est = d8_estimate(name, c, A, h_nn, h_diag, sweeps, budget_s=budget_s)
    return {"value": 1.0 / t, "unit": "evals/s", "cores": threads, "kind": "oracle",
            "sample": f"one whole oracle energy+gradient evaluation of {CPU_WORKLOAD} (2x2 cell, d=2, D=4, chi=32, "
                      f"Heisenberg J=1, {CPU_SWEEPS} sweeps, autograd reverse pass) timed on the host: {t:.2f} s, "
                      f"E={e:.12f}",
            "workload": CPU_WORKLOAD, "sweeps": CPU_SWEEPS,
            "estimate_of": {"workload": name, "value": est["value"], "unit": "evals/s", "kind": "estimate",
                            "how": est["sample"]}}


def d8_estimate(name, c, A, h_nn, h_diag, sweeps, budget_s=20.0):
    """An ESTIMATE, not a timing: the FP64 oracle timed on a bounded sample of
    the workload and scaled to one energy+gradient evaluation.

    Sample: (1) the oracle's initial environment; (2) single-column projector
    stages of a left move (every colour's rho networks, decompositions and the
    absorption), as many as fit in about half the budget; (3) one product of
    two closed enlarged corners, the (chi D^2)^3 contraction the oracle's 2x2
    energy is made of, on matrices of that exact shape.  Scaling: forward =
    init + 4 * sweeps moves x Ly columns + the energy (per patch the oracle
    performs 50 such corner products: two closed-closed, two with both physical
    pairs open (p^4 = 16 each) and four with one open pair (p^2 = 4 each));
    one evaluation = forward + reverse, the reverse counted as twice the
    forward (reverse-mode autograd)."""
    import torch
    from oracle import ctmrg as C
    torch.set_num_threads(os.cpu_count() or 1)
    Ac = C.as_cell(A)
    t0 = time.perf_counter()
    env = C.initial_env(Ac, c["chi"])
    t_init = time.perf_counter() - t0
    n, t_col = 0, 0.0
    while n == 0 or (t_col < budget_s / 2 and n < 8):   # at least one column stage
        t1 = time.perf_counter()
        with torch.no_grad():
            C.split_column_projectors(Ac, env, n % c["Ly"], c["chi"])
        t_col += time.perf_counter() - t1
        n += 1
    per_col = t_col / n
    N = c["chi"] * c["D"] ** 2
    g = torch.Generator().manual_seed(0)
    X = torch.randn((N, N), dtype=torch.float64, generator=g)
    Y = torch.randn((N, N), dtype=torch.float64, generator=g)
    t1 = time.perf_counter()
    torch.einsum("ra,rb->ab", X, Y)
    t_prod = time.perf_counter() - t1
    del X, Y
    moves = 4 * sweeps
    cols_per_move = c["Ly"]  # left/right moves; top/bottom use Lx rows (square cells here)
    n_patch = c["Lx"] * c["Ly"]
    fwd = t_init + moves * cols_per_move * per_col + 50 * n_patch * t_prod
    t_eval = 3.0 * fwd
    return {"value": 1.0 / t_eval, "unit": "evals/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"oracle initial environment ({t_init:.2f} s), {n} single-column projector stages of a "
                      f"left move ({per_col:.2f} s each) and one {N}^3 closed-corner product "
                      f"({t_prod:.2f} s) at {name} on the host; scaled to one energy+gradient evaluation "
                      f"as 3x the forward ({moves} moves x {cols_per_move} columns + {50 * n_patch} corner "
                      f"products of the 2x2 energy)"}


FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz


def roofline_of(fam, p, peaks, src, prec):
    """Roofline of the dominant kernel family `fam` of a step, from the engine's
    profiler record p = {ms, launches, flops, bytes} over the timed steps.

    tensor: the 3xTF32 tcgen05 contraction against the TF32 peak (the measured
    bf16 figure, sustained, times the nominal TF32/BF16 ratio 1.1/2.25); achieved
    counts the algorithmic 2MNK only, while the pipe executes three TF32 products
    per multiply-add.  svd, and contract at precisions 0 and 3: FP64 ALU.
    contract at precisions 1 and 2: FP32 ALU (its FP64 Gram products are the
    smaller part).  other (packing, copies, scaling): HBM bytes against the
    measured copy bandwidth."""
    ms = p["ms"]
    if fam == "other":
        achieved = p["bytes"] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        peak = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "other (packing, copies, scaling)",
                "peak_source": f"{src} copy bandwidth"}
    achieved = p["flops"] / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    if fam == "tensor" and prec == 4:
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # DRAM bytes (read + write) of one 8192^3 enlarged-corner product from one
                # ncu capture of the current kernel
                "traffic": SLICE_CORNER_DRAM_BYTES,
                "traffic_launch": "8192^3 corner product (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "kernel": "slice_gemm_kernel (BF16 digit-slice tcgen05 contraction)",
                "peak_source": f"{src} bf16 sustained",
                "tensor_pipe_frac": 10.0 * achieved / peak,
                "note": "achieved counts 2MNK; the pipe executes ten BF16 products per multiply-add"}
    if fam == "tensor":
        bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        peak = bf16 * 1.1 / 2.25
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # DRAM bytes (read + write) of one 8192^3 enlarged-corner product, the kernel's
                # dominant launch shape, from one ncu capture of the current kernel
                "traffic": TC_CORNER_DRAM_BYTES,
                "traffic_launch": "8192^3 corner product (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "kernel": "tc_gemm_kernel (3xTF32 tcgen05 contraction)",
                "peak_source": f"TF32 = {src} bf16 sustained x 1.1/2.25 (nominal ratio)",
                "tensor_pipe_frac": 3.0 * achieved / peak}
    if fam == "contract" and prec in (1, 2):
        return {"bound": "alu", "achieved": achieved, "peak": FP32_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_NOMINAL_TFLOPS, "traffic": None, "kernel": "contract_kernel (FP32 ALU)",
                "peak_source": "FP32 nominal (152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz); none measured"}
    return {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None, "kernel": fam + " (FP64 ALU)",
            "peak_source": "FP64 nominal (152 SMs x 2.07 GHz x 4 flop/clk/SM); no FP64 figure measured"}


def arm_config(desc, prec, world):
    """The `config` of a bench line; the reference arm reports the same one."""
    return {"workload": desc, "precision": prec, "l2": "flushed (256 MiB write) before every step",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def aggregate_over_ranks(total_ms, steps, world, dist, device):
    """Timed milliseconds of the slowest rank (all-reduce MAX) and the whole-job
    throughput: the units all ranks processed divided by that time."""
    import torch
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / steps
    return ms_per_step, world * 1000.0 / ms_per_step


def run_reference(args):
    """The FP64 oracle on the host cores, on this arm's workload and metric.
    One evaluation at D=8, chi=128 takes the oracle hours, so each of the W + K
    steps times a bounded sample of it (the initial environment, one column
    stage of a left move, one closed-corner product of the energy) and scales
    it to one evaluation: ``value`` is that estimate, labelled as such, and
    ``ms_per_step`` the measured wall time of a sample step.  One whole oracle
    evaluation of the small 2x2, D=4, chi=32 workload is timed beside it."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    A, c, h_nn, h_diag, sweeps, desc = workload(args.config, args.sweeps)
    prec = args.precision if args.precision is not None else c.get("bench_precision", 0)
    steps = max(1, args.steps)
    budget = args.cpu_budget if args.warmup + steps == 1 else 0.0
    timed, wall = [], 0.0
    for i in range(args.warmup + steps):
        t0 = time.perf_counter()
        est = d8_estimate(args.config, c, A, h_nn, h_diag, sweeps, budget_s=budget)
        if i >= args.warmup:
            timed.append(est)
            wall += time.perf_counter() - t0
    t_eval = sum(1.0 / e["value"] for e in timed) / len(timed)
    t_small, e_small, threads = oracle_evaluation()
    cb = {"value": 1.0 / t_eval, "unit": "evals/s", "cores": threads, "kind": "oracle",
          "value_kind": "estimate scaled from a bounded sample per step",
          "sample": f"mean of {len(timed)} timed steps after {args.warmup} untimed ones; each step: "
                    + timed[-1]["sample"],
          "measured_small": {"workload": CPU_WORKLOAD, "sweeps": CPU_SWEEPS, "value": 1.0 / t_small,
                             "unit": "evals/s", "kind": "one whole oracle evaluation, timed"}}
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "evals/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": arm_config(desc, prec, world),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


DTYPES = {0: "f64", 1: "tf32x3 (f32 accumulate) + f32 + f64", 2: "f32 + f64", 3: "f64",
          4: "bf16 x4 digit slices (exact f32 level sums) + f32 + f64"}

METRIC = "energy+gradient evals/s (split-CTMRG, D=8 chi=128) & TFLOP/s vs peak, vs FP64"


def _cpu_args(args):
    A, c, h_nn, h_diag, sweeps, _ = workload(args.config, args.sweeps)
    return c, A, h_nn, h_diag, sweeps, args.cpu_budget


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1,
                    help="timed evaluations (one evaluation of the default workload takes about 48 s)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="d8_chi128_2x2_j1j2", choices=sorted(I.WORKLOADS))
    ap.add_argument("--sweeps", type=int, default=None)
    ap.add_argument("--precision", type=int, default=None,
                    help="0 FP64, 1 mixed (3xTF32 tensor cores), 2 mixed on CUDA cores, 3 FP64 with randomized "
                         "projectors, 4 mixed with BF16 digit slices on the tensor cores; default per workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the kernels' split-K rules (no tuning)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--algorithm", default="split", choices=["split", "conventional"],
                    help="split CTMRG (the method) or the conventional double-layer CTMRG it is compared with")
    ap.add_argument("--move-scaling", action="store_true",
                    help="time one directional move of the split and the conventional CTMRG against D at "
                         "fixed chi (the paper's Fig. 5a comparison) instead of the evaluation")
    ap.add_argument("--forward", action="store_true",
                    help="time the forward pieces of the workload (initial environment, one move, 2x2 energy) "
                         "and report the peak device workspace, for workloads whose gradient does not fit")
    ap.add_argument("--chi", type=int, default=128, help="environment dimension of --move-scaling")
    ap.add_argument("--Ds", default="4,5,6,7,8", help="comma-separated bulk dimensions of --move-scaling")
    ap.add_argument("--p", type=int, default=2,
                    help="physical dimension of --move-scaling (4: the paper's coarse-grained honeycomb sites)")
    ap.add_argument("--kernel", default=None, choices=["corner-product"],
                    help="time one kernel alone instead of the evaluation (profiling aid)")
    ap.add_argument("--workspace-gb", type=float, default=None)
    ap.add_argument("--precisions", default=None,
                    help="comma-separated precisions: one evaluation each at equal sweeps and cutoff (the FP64 "
                         "form beside the mixed ones), precision 0 first for the gradient reference")
    ap.add_argument("--cutoff", type=float, default=1e-5, help="projector cutoff of --precisions")
    ap.add_argument("--oracle-energy", action="store_true", help="--precisions: also the oracle's forward energy")
    ap.add_argument("--implicit", action="store_true",
                    help="the implicit fixed-point gradient of the converged environment beside the checkpointed "
                         "one (same precision): time, sweeps, solver iterations and peak workspace of each")
    ap.add_argument("--max-sweeps", type=int, default=60, help="--implicit: sweep limit of the run to convergence")
    ap.add_argument("--max-iter", type=int, default=60, help="--implicit: iteration limit of the adjoint solve")
    ap.add_argument("--near-product", type=float, default=None,
                    help="--implicit: replace the workload's tensors by a near-product state of the same shape "
                         "(0.8|0> + 0.6|1> on the zero bond index plus this much N(0,1) noise, seed 5)")
    ap.add_argument("--lbfgs", type=int, default=0,
                    help="run the L-BFGS optimisation of the workload for this many energy+gradient evaluations")
    args = ap.parse_args()
    if args.implicit:
        return run_implicit(args)
    if args.lbfgs:
        return run_lbfgs(args)
    if args.precisions:
        return run_precisions(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return run_kernel(args)
    if args.forward:
        return run_forward(args)
    if args.move_scaling:
        return run_move_scaling(args, chi=args.chi, Ds=tuple(int(d) for d in args.Ds.split(",")), p=args.p)

    import torch
    import paper_2502_10298_gb300 as S
    if not args.no_cpu and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        # the oracle's thread pool is started before the first GPU call
        cpu_first = cpu_baseline(args.config, *_cpu_args(args))
    else:
        cpu_first = None

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    S.load_library()
    A, c, h_nn, h_diag, sweeps, desc = workload(args.config, args.sweeps)
    At = torch.tensor(A, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    stream = torch.cuda.current_stream()
    prec = args.precision if args.precision is not None else c.get("bench_precision", 0)
    algo = 1 if args.algorithm == "conventional" else 0
    s = S.SplitCTMRG(c["Lx"], c["Ly"], c["p"], c["D"], c["chi"], precision=prec,
                     workspace_bytes=args_ws(c, args.workspace_gb), algorithm=algo)
    if algo:
        desc = desc + ", conventional double-layer CTMRG"

    def step():
        return s.energy_grad(At, sweeps, h_nn, h_diag)

    # the warm-up steps also run the split-K autotuner (each shape's candidates
    # are complete contractions); the timed steps use its choices
    if not args.no_autotune:
        S.sctm_autotune(s.h, True)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    S.sctm_autotune(s.h, False)
    torch.cuda.synchronize()
    tuned = S.sctm_autotune_table(s.h)
    if dist:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    total_ms = 0.0
    e_val = None
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e_val, g = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
    clocks = clk.stop()
    torch.cuda.synchronize()
    ms_per_step, value = aggregate_over_ranks(total_ms, args.steps, world, dist, "cuda")
    # how converged the environment of the evaluation is: one more full step from
    # it, and the change of the normalised corner spectra (split_ctmrg_run's measure)
    _, conv_delta = S.split_ctmrg_run(s.h, 1)
    # per-family breakdown from one extra, untimed step with the engine's event profiler
    flush.zero_()
    torch.cuda.synchronize()
    S.sctm_profile(s.h, True)
    step()
    prof = S.sctm_profile(s.h, False)
    prof_steps = 1

    # end-to-end through the host-buffer C-ABI call (H2D of A, D2H of grad + energy inside the timing)
    e2e = None
    if not args.no_e2e:
        A_host = torch.tensor(A).pin_memory().numpy()
        g_host = torch.empty(A.shape, dtype=torch.float64).pin_memory().numpy()
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e = max(1, args.steps)
        for _ in range(n_e2e):
            S.energy_grad_host(s.h, A_host, sweeps, h_nn, h_diag, grad_out=g_host)
        t_e2e = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": world / t_e2e, "unit": "evals/s", "h2d_bytes_per_step": int(A.nbytes),
               "d2h_bytes_per_step": int(A.nbytes) + 8}

    peaks, src = load_peaks()
    tot_ms = sum(v["ms"] for v in prof.values())
    fams = {k: {"ms_per_step": v["ms"] / prof_steps, "launches_per_step": v["launches"] / prof_steps,
                "share_of_device_time": v["ms"] / tot_ms if tot_ms else None,
                "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] else 0.0}
            for k, v in prof.items()}
    fam = max(prof, key=lambda k: prof[k]["ms"])
    p = prof[fam]
    roof = roofline_of(fam, p, peaks, src, prec)
    roof["share_of_device_time"] = p["ms"] / tot_ms if tot_ms else None
    roof["families"] = fams
    cpu = None
    if cpu_first is not None and rank == 0:
        cpu = cpu_first
        # the GPU on the same small evaluation the oracle was timed on
        Ac_, cc_, hn_, hd_, sw_, _ = workload(CPU_WORKLOAD, CPU_SWEEPS)
        At_ = torch.tensor(Ac_, device="cuda")
        with S.SplitCTMRG(cc_["Lx"], cc_["Ly"], cc_["p"], cc_["D"], cc_["chi"], precision=prec) as s2:
            s2.energy_grad(At_, sw_, hn_, hd_)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                s2.energy_grad(At_, sw_, hn_, hd_)
            torch.cuda.synchronize()
            cpu["gpu_same_workload"] = {"value": 3.0 / (time.perf_counter() - t0), "unit": "evals/s",
                                        "precision": prec}
    launches = int(sum(v["launches"] for v in prof.values()) / prof_steps)
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[prec],
            "data": "synthetic",
            "config": arm_config(desc, prec, world),
            "energy_per_site": e_val, "convergence_delta": conv_delta, "clocks": clocks, "e2e": e2e,
            "autotune": {"shapes": len(tuned), "changed": sum(1 for r in tuned if r["chosen_splits"] != r["rule_splits"]),
                         "ms_saved_per_call_sum": sum(r["rule_ms"] - r["chosen_ms"] for r in tuned)},
            "gpu_launches": launches,
            "roofline": roof, "cpu_baseline": cpu,
            "workspace_high_water_bytes": S.sctm_workspace_high_water(s.h)}
    s.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_kernel(args):
    """One enlarged-corner product of the 2x2 energy, (chi D^2)^3 = 8192^3 at the
    D=8, chi=128 workload, through sctm_einsum on the tensor cores (precision 1:
    3xTF32; precision 4: BF16 digit slices): the dominant kernel of an
    evaluation, timed alone (burst) with CUDA events."""
    import torch
    import paper_2502_10298_gb300 as S
    A, c = I.config(args.config)
    n = c["chi"] * c["D"] ** 2
    prec = args.precision if args.precision is not None else 1
    h = S.sctm_create(1, 1, 2, 2, 4, precision=prec, workspace_bytes=int(2 * 16 * n * n + (1 << 30)))
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    Y = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    Z = torch.empty((n, n), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        S.sctm_einsum(h, "ra,rb->ab", X, Y, Z)
    torch.cuda.synchronize()
    S.sctm_profile(h, True)
    for _ in range(args.steps):
        S.sctm_einsum(h, "ra,rb->ab", X, Y, Z)
    prof = S.sctm_profile(h, False)
    S.sctm_destroy(h)
    t = prof["tensor"]
    peaks, src = load_peaks()
    ach = t["flops"] / (t["ms"] * 1e-3) / 1e12
    bf16 = peaks.get("bf16_tflops", 1900.0)
    if prec == 4:
        kern, peak, products, psrc = "slice_gemm_kernel", bf16, 10, f"{src} bf16 burst"
    else:
        kern, peak, products, psrc = "tc_gemm_kernel", bf16 * 1.1 / 2.25, 3, f"{src} bf16 burst x 1.1/2.25"
    print(json.dumps({"kernel": kern, "precision": prec, "shape": [n, n, n], "launches": t["launches"],
                      "ms_per_launch": t["ms"] / max(1, t["launches"]), "achieved_tflops": ach,
                      "peak_tflops": peak, "frac": ach / peak, "tensor_pipe_frac": products * ach / peak,
                      "pack_ms_per_step": prof["other"]["ms"] / max(1, args.steps),
                      "peak_source": psrc}))
    return 0


def run_forward(args):
    """Device time (CUDA events) of the initial environment, of one directional
    move (mean over the second of two sweeps) and of the 2x2 energy for the
    workload, in the handle's precision, and the peak device workspace."""
    import torch
    import paper_2502_10298_gb300 as S
    A, c, h_nn, h_diag, _, desc = workload(args.config, args.sweeps)
    prec = args.precision if args.precision is not None else c.get("bench_precision", 0)
    algo = 1 if args.algorithm == "conventional" else 0
    At = torch.tensor(A, device="cuda")

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        out = fn()
        ev1.record()
        torch.cuda.synchronize()
        return out, ev0.elapsed_time(ev1)

    ws = int(args.workspace_gb * 2**30) if args.workspace_gb else 200 * 2**30
    with S.SplitCTMRG(c["Lx"], c["Ly"], c["p"], c["D"], c["chi"], precision=prec, workspace_bytes=ws,
                      algorithm=algo) as s:
        _, t_init = timed(lambda: s.init(At))
        timed(lambda: s.sweeps(1))
        _, t_sweep = timed(lambda: s.sweeps(1))
        e, t_energy = timed(lambda: s.energy(h_nn, h_diag))
        print(json.dumps({"workload": desc, "algorithm": args.algorithm, "precision": prec,
                          "init_ms": t_init, "ms_per_move": t_sweep / 4, "energy_ms": t_energy,
                          "energy_per_site": e, "workspace_high_water_bytes": S.sctm_workspace_high_water(s.h)}))
    return 0



def run_implicit(args):
    """Energy gradient of the converged environment two ways, in the handle's
    precision: implicitly (energy_grad_implicit: run to the fixed point, one
    step's reverse pass per adjoint iteration) and by the checkpointed reverse
    pass through as many sweeps as the run took.  Reports seconds (CUDA events),
    sweeps, solver iterations, the fixed-point check and the peak workspace of
    each, and the relative difference of the two gradients.  A state whose
    projector gauge is not fixed between steps is reported as refused."""
    import torch
    import paper_2502_10298_gb300 as S
    A, c, h_nn, h_diag, _, desc = workload(args.config, args.sweeps)
    if args.near_product is not None:
        rng = np.random.default_rng(5)
        A = np.zeros_like(A)
        A[:, :, 0, 0, 0, 0, 0] = 0.8
        A[:, :, 1, 0, 0, 0, 0] = 0.6
        A = A + args.near_product * rng.standard_normal(A.shape)
        desc += f" (near-product state, noise {args.near_product})"
    prec = args.precision if args.precision is not None else c.get("bench_precision", 0)
    At = torch.tensor(A, device="cuda")
    ws = args_ws(c, args.workspace_gb)
    out = {"workload": desc, "precision": prec, "dtype": DTYPES[prec]}

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        r = fn()
        ev1.record()
        torch.cuda.synchronize()
        return r, ev0.elapsed_time(ev1) / 1e3

    g_imp = None
    with S.SplitCTMRG(c["Lx"], c["Ly"], c["p"], c["D"], c["chi"], precision=prec, workspace_bytes=ws) as s:
        try:
            (e, g_imp, info), sec = timed(lambda: s.energy_grad_implicit(At, h_nn, h_diag, max_sweeps=args.max_sweeps,
                                                                         max_iter=args.max_iter))
            out["implicit"] = {"seconds": sec, "energy_per_site": e, **info,
                               "workspace_high_water_bytes": S.sctm_workspace_high_water(s.h)}
        except S.SctmError as ex:
            out["implicit"] = {"refused": str(ex)}
    sweeps = out["implicit"].get("sweeps") or c["sweeps"]
    with S.SplitCTMRG(c["Lx"], c["Ly"], c["p"], c["D"], c["chi"], precision=prec, workspace_bytes=ws) as s:
        (e, g), sec = timed(lambda: s.energy_grad(At, sweeps, h_nn, h_diag))
        out["checkpointed"] = {"seconds": sec, "sweeps": sweeps, "energy_per_site": e,
                               "workspace_high_water_bytes": S.sctm_workspace_high_water(s.h)}
    if g_imp is not None:
        out["grad_rel_diff"] = float((g_imp - g).norm() / g.norm())
    print(json.dumps(out))
    return 0

def run_move_scaling(args, chi=128, Ds=(4, 5, 6, 7, 8), p=2):
    """Device time of one directional move (mean over a sweep of four, after one
    warm-up sweep) for the split CTMRG in both yellow/red orders (App. B) and
    the conventional CTMRG at fixed chi, 1x1 cell, seeded N(0,1) tensor, mixed
    precision (--precision, default 1): the shape of the paper's Fig. 5a (time
    of one absorption step against the bulk bond dimension)."""
    import torch
    import paper_2502_10298_gb300 as S
    prec = args.precision if args.precision is not None else 1
    rows = []
    for D in Ds:
        A = I.random_cell(1, 1, p, D, seed=0)
        At = torch.tensor(A, device="cuda")
        row = {"D": D, "chi": chi, "p": p, "precision": prec}
        for name, algo, order in (("split", 0, 0), ("split_alt_order", 0, 1), ("conventional", 1, 0)):
            n = chi * D * D
            ws = int(min(200 * 2**30, max(8 * 2**30, 40 * n * n * 8)))
            with S.SplitCTMRG(1, 1, p, D, chi, precision=prec, workspace_bytes=ws, algorithm=algo,
                              projector_order=order) as s:
                s.init(At)
                s.sweeps(1)
                torch.cuda.synchronize()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record()
                s.sweeps(1)
                ev1.record()
                torch.cuda.synchronize()
                row[name + "_ms_per_move"] = ev0.elapsed_time(ev1) / 4
        rows.append(row)
        print(json.dumps(row), flush=True)
    return 0


def run_precisions(args):
    """The plain FP64 form beside the mixed forms at equal sweeps and cutoff:
    one timed energy+gradient evaluation per precision (after a warm-up of the
    kernels on a small cell), its energy against the FP64 oracle's forward pass
    (same sweeps and cutoff) and its gradient against the FP64 GPU form's
    (precision 0, which matches the oracle's autograd to 1e-10 where that runs).
    One JSON line per precision."""
    import torch
    import paper_2502_10298_gb300 as S
    from oracle import ctmrg as C
    from oracle import energy as En
    S.load_library()
    A, c, h_nn, h_diag, sweeps, desc = workload(args.config, args.sweeps)
    cut = args.cutoff
    precs = [int(x) for x in args.precisions.split(",")]
    e_or = None
    if args.oracle_energy:
        import torch as T
        T.set_num_threads(os.cpu_count() or 1)
        old = C.CUTOFF
        C.CUTOFF = cut
        t0 = time.perf_counter()
        with T.no_grad():
            Ac = C.as_cell(A)
            e_or = float(En.energy_per_site(Ac, C.split_ctmrg(Ac, c["chi"], sweeps), h_nn, h_diag))
        C.CUTOFF = old
        print(json.dumps({"oracle_energy": e_or, "seconds": time.perf_counter() - t0, "cutoff": cut}), flush=True)
    At = torch.tensor(A, device="cuda")
    with S.SplitCTMRG(1, 1, 2, 2, 8, precision=4) as w:   # load and warm every kernel once
        w.energy_grad(torch.tensor(I.random_cell(1, 1, 2, 2, seed=1), device="cuda"), 1, I.heisenberg_bond())
    g_ref = None
    for prec in precs:
        with S.SplitCTMRG(c["Lx"], c["Ly"], c["p"], c["D"], c["chi"], precision=prec, svd_cutoff=cut,
                          workspace_bytes=args_ws(c, args.workspace_gb)) as s:
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            e, g = s.energy_grad(At, sweeps, h_nn, h_diag)
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
        if prec == 0:
            g_ref = g.clone()
        line = {"workload": desc, "precision": prec, "dtype": DTYPES[prec], "cutoff": cut, "sweeps": sweeps,
                "evals_per_s": 1000.0 / ms, "ms": ms, "energy_per_site": e,
                "energy_err_vs_oracle": (e - e_or) if e_or is not None else None,
                "grad_rel_err_vs_fp64_gpu": (float((g - g_ref).norm() / g_ref.norm()) if g_ref is not None else None)}
        print(json.dumps(line), flush=True)
    return 0


def run_lbfgs(args):
    """The variational loop of the workload: L-BFGS over energy_grad for a
    fixed number of energy+gradient evaluations (10 for the D=8 workload),
    from its seeded tensors.  Prints the energy trace and evals/s."""
    import torch
    import paper_2502_10298_gb300 as S
    S.load_library()
    A, c, h_nn, h_diag, sweeps, desc = workload(args.config, args.sweeps)
    prec = args.precision if args.precision is not None else c.get("bench_precision", 0)
    At = torch.tensor(A, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, trace = S.lbfgs(At, c["chi"], sweeps, h_nn, h_diag, evaluations=args.lbfgs, precision=prec,
                       workspace_bytes=args_ws(c, args.workspace_gb))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    print(json.dumps({"workload": desc, "precision": prec, "dtype": DTYPES[prec], "optimizer": "L-BFGS (strong Wolfe)",
                      "evaluations": len(trace), "seconds": wall, "evals_per_s": len(trace) / wall,
                      "energy_first": trace[0]["energy"], "energy_last": trace[-1]["energy"],
                      "energy_best": min(t["energy"] for t in trace), "trace": trace}))
    return 0


def args_ws(c, gb=None):
    """Device workspace: one taped 2x2 patch of the energy (about 220 enlarged-corner
    sized buffers of (chi D^2)^2 doubles, gradients included) plus a taped sweep."""
    import torch
    if gb:
        return int(gb * 2**30)
    n = c["chi"] * c["D"] ** 2
    need = 220 * n * n * 8 + 16 * 2**30
    # at most the free device memory less 12 GiB (CUDA context, library state
    # and the caller's tensors)
    cap = torch.cuda.mem_get_info()[0] - 12 * 2**30 if torch.cuda.is_available() else 240 * 2**30
    return int(min(cap, max(8 * 2**30, need)))


if __name__ == "__main__":
    sys.exit(main())
