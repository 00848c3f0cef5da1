"""Benchmark: time-to-1e-8 residual and GDoF/s per sweep of the decoupled Stokes multigrid.

Workload (one "step"): one full solve, from a zero initial guess to ||b - K x|| <= 1e-8 ||b||,
of the 128^3-cell unit cube (8.6M DoF) with three seeded mesh-aligned boxes of viscosity
ratio 1e4, no-slip walls and manufactured forcing, decoupled form, FP64, flexible GMRES
preconditioned by the V_var(3,3) Uzawa multigrid.  Beside it the same run reports the strain
form and the FP32-refined variant on the same workload, per-sweep throughput of the operator
apply and the smoother passes, the roofline of the dominant kernel, an end-to-end number
through the host-buffer C entry point, and the CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sdx|reference]
Multi-GPU (torchrun): every rank solves its own replica (no data exchange; weak scaling).
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

FP64_PEAK_FLOP_PER_CLK_PER_SM = 4  # 2 DFMA per clock per SM (GB300: 1.25 TFLOP/s FP64 nominal)
# DRAM bytes (read + write) of one launch of the red FP64 velocity pass on the 128^3 workload,
# from the ncu capture summarised in profiles/k_vel_uniform_three_boxes_128.md
VEL_PASS_DRAM_BYTES_128 = 124941568 + 14626816
# the same for the red FP64 pressure pass (profiles/k_pre_uniform_three_boxes_128.md)
PRE_PASS_DRAM_BYTES_128 = 98697984 + 4342016
# Both captures predate the current build of these kernels, whose thread index is now split
# with 32-bit instead of 64-bit divisions (same loads and stores); the line therefore reports
# `traffic` as null and the earlier counters under their own key.
TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the build before the thread index was "
                "split with 32-bit divisions; the current kernel reads and writes the same addresses")
# the kernel of the benchmark's `roofline` object: the largest share of the step in the launch
# list summarised in profiles/ (the pressure pass runs on every level)
DOMINANT_KERNEL = "pressure_pass"
N_SM = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sdx", choices=["sdx", "reference"])
    ap.add_argument("--n", type=int, default=128, help="cells per side (workload size)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--mode", default="solve", choices=["solve", "sweep", "levels", "guess", "batch", "paper", "conv",
                                                        "p1p0"],
                    help="sweep: only time the operator apply and smoother passes (profiling); "
                         "guess: only the learned-initial-guess experiment; batch: only the batched workload")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"], help="arithmetic of --mode sweep")
    ap.add_argument("--form", default="tr", choices=["tr", "sym", "grad"])
    ap.add_argument("--coarse-form", default="sym", choices=["tr", "sym", "grad"],
                    help="form of the coarser levels in --mode levels")
    ap.add_argument("--beta", type=float, default=1.0 / 24.0,
                    help="pressure-stabilisation constant of the three-box workload (tau = beta h^2 / mu)")
    ap.add_argument("--maxit", type=int, default=500,
                    help="iteration cap per solve (profiling runs use a small cap)")
    ap.add_argument("--no-details", action="store_true", help="skip sweeps, e2e, variants, CPU leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 48-instance batched workload")
    ap.add_argument("--no-layer", action="store_true", help="skip the 256^3 mixed-precision workload")
    ap.add_argument("--no-guess", action="store_true", help="skip the learned-initial-guess experiment")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's columns problem (time per cycle, rate)")
    ap.add_argument("--guess-samples", type=int, default=192, help="training solves at 64^3")
    ap.add_argument("--guess-epochs", type=int, default=12)
    ap.add_argument("--guess-eval", type=int, default=4, help="unseen 128^3 instances to evaluate")
    ap.add_argument("--guess-smooth", default="4", help="comma-separated Uzawa smoothing steps applied to the guess")
    ap.add_argument("--batch-count", type=int, default=48, help="instances of the batched workload")
    ap.add_argument("--conv-n", type=int, default=64, help="cells per side of --mode conv")
    return ap.parse_args()


def job_time_ms(ms_local, device):
    """The job's time per step: the maximum over ranks (replicas run independent solves; the
    job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(free_per_rank, world_size, ms):
    """Whole-job throughput in GDoF/s: every rank solves its own problem of free_per_rank DoF."""
    return world_size * free_per_rank / (ms * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


RESTART = 30  # FGMRES restart length of the benchmark solve


def workload_config(n, beta, ws):
    """The `config` object of both arms' lines: the workload and the solver, nothing measured.
    The three-box workload has no-slip walls, so the velocities of the boundary nodes are fixed
    and (n+1)^3 pressures + 3 (n-1)^3 interior velocities are free."""
    free = (n + 1) ** 3 + 3 * (n - 1) ** 3
    levels = (n // 8).bit_length()  # cells per side halve down to the 8^3 coarsest grid
    return {"workload": f"three_boxes_{n}: {n}^3 cells ({free} free DoF), 3 seeded boxes on the 1/8 lattice, mu ratio 1e4, no-slip walls, manufactured forcing",
            "form": "decoupled (a_tr with interface strain rows) on the finest level, a_sym on the coarser levels",
            "solver": f"FGMRES({RESTART}) + V_var(3,3) Uzawa multigrid, {levels} levels, coarsest 8^3 dense FP64 inverse",
            "rtol": 1e-8, "pspg_beta": beta,
            "l2": "inputs larger than L2 (each 4-component FP64 vector is 69 MB at 128^3; solver working set > 4 GB)",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if s[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(beta=1.0 / 24.0):
    """The oracle as it stands: FGMRES + V-cycle solve of the same workload family at 32^3
    (same boxes, contrast, walls and forcing, and the same solver: a_tr on the finest level,
    a_sym on the coarser ones, the same beta; a bounded sample of the 128^3 job)."""
    from oracle.solvers import Hierarchy as OH, fgmres, vcycle_preconditioner
    from paper_1604_07994_gb300 import workloads as W
    p = W.three_boxes(32, 8, contrast=1e4)
    H = OH(32, 8, p.cell_mu().ravel(), p.face, "tr", beta=beta, coarse_form="sym")
    L = H.levels[0]
    b = L.disc.rhs(p.nodal_forcing())
    t0 = time.perf_counter()
    c0 = time.process_time()
    x, hist = fgmres(L.K, vcycle_preconditioner(H), b, L.free, rtol=1e-8, restart=30, maxit=400)
    dt = time.perf_counter() - t0
    cpu = time.process_time() - c0
    free = int(L.free.sum())
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    # threads actually used: CPU seconds of the process (all threads) over the wall time
    used = round(cpu / dt, 1) if dt > 0 else None
    return {"value": free / dt / 1e9, "unit": "GDoF/s (solved to 1e-8)", "cores": used,
            "cpu_seconds": cpu, "host_cores_available": cores, "kind": "oracle",
            "sample": f"oracle FGMRES(30)+V_var solve to 1e-8 of the same workload at 32^3 cells "
                      f"({free} free DoF; a_tr finest, a_sym coarser levels, beta {beta:.6g}), "
                      f"{dt:.1f} s wall, {cpu:.1f} s CPU; scipy CSR products are "
                      f"single-threaded, the BLAS calls (dense coarsest solve, vector kernels) use the "
                      f"BLAS thread pool; cores = CPU / wall"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1604_07994_gb300 import workloads as W  # noqa: F401
    times = []
    res = None
    for _ in range(args.warmup + args.steps):
        res = oracle_sample(args.beta)
        times.append(res)
    vals = [r["value"] for r in times[args.warmup:]]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": "time-to-1e-8 residual & GDoF/s per sweep: decoupled vs strain, FP32-refined vs FP64",
            "value": v, "unit": "GDoF/s (solved to 1e-8)", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n, args.beta, ws),
            "cpu_baseline": {**times[-1], "value": v},
            "e2e": {"value": v, "unit": "GDoF/s (solved to 1e-8)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "sweep":
        run_sweeps(args)
        return
    if args.mode == "levels":
        run_levels(args)
        return
    if args.mode in ("guess", "batch", "paper", "conv", "p1p0"):
        import torch
        torch.cuda.set_device(0)
        from paper_1604_07994_gb300 import sdx
        out = {"guess": run_guess, "batch": run_batch, "paper": run_paper, "conv": run_conv,
               "p1p0": run_p1p0}[args.mode](args, sdx, torch)
        print(json.dumps({"mode": args.mode, **out}), flush=True)
        return
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1604_07994_gb300 import sdx
    from paper_1604_07994_gb300 import workloads as W

    n = args.n
    prob = W.three_boxes(n, 8, contrast=1e4)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    # decoupled operator a_tr on the finest level; the coarser levels use a_sym (the coarse-grid
    # swap of Sec. 5 extended to every coarse level), FP64 throughout
    H = sdx.Hierarchy.from_problem(prob, form="tr", coarse_form="sym", prec=sdx.PREC_FP64, beta=args.beta)
    setup_s = time.perf_counter() - t0
    _, nodes, free = H.sdx_level_size(0)
    f = torch.from_numpy(prob.nodal_forcing().ravel()).to(dev)
    b = torch.zeros(4 * nodes, dtype=torch.float64, device=dev)
    H.sdx_rhs(f, b)
    x = torch.zeros_like(b)

    def step(h, xv):
        xv.zero_()
        return h.sdx_solve(b, xv, rtol=1e-8, maxit=args.maxit, outer=sdx.OUTER_FGMRES, restart=RESTART,
                           allow_noconv=args.maxit < 500)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        st = step(H, x)
    barrier()
    print(json.dumps({"launches_before_timed_region": sdx.sdx_kernel_launches()}), file=sys.stderr, flush=True)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sdx.sdx_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        st = step(H, x)
        iters.append(st["iterations"])
    e1.record(stream)
    barrier()
    launches = sdx.sdx_kernel_launches() - l0
    clk = clocks.stop()
    ms = job_time_ms(e0.elapsed_time(e1) / args.steps, dev)
    value = job_value(free, ws, ms)
    final_res = st["res"] / st["bnorm"]

    extra = {}
    if rank == 0 and not args.no_details:
        extra = measure_details(args, H, prob, b, x, nodes, free, stream, torch, sdx, W)
    if ws > 1:
        torch.distributed.barrier()
    if rank != 0:
        return
    pk = peaks()
    # roofline objects of the finest level's red velocity and pressure passes (FP64-pipe bound);
    # the pressure pass has the largest share of the step's launch list and is the `roofline`
    rl = extra.get("roofline_kernel", {})
    peak_fp64 = N_SM * FP64_PEAK_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    roofs = {}
    for key, kernel, traffic in (
            ("pressure_pass", "k_pre_uniform<double> (red pressure Gauss-Seidel pass, finest level)",
             PRE_PASS_DRAM_BYTES_128),
            ("velocity_pass", "k_vel_uniform<double, a_tr> (red velocity Gauss-Seidel pass, finest level)",
             VEL_PASS_DRAM_BYTES_128)):
        r = rl.get(key)
        if not r:
            continue
        achieved = r["flops"] / (r["ms"] * 1e-3) / 1e12
        roofs[key] = {"bound": "alu", "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
                      "frac": achieved / peak_fp64, "traffic": None,
                      "traffic_last_capture": traffic if n == 128 else None, "traffic_note": TRAFFIC_NOTE,
                      "kernel": kernel,
                      "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (nominal 1.25 TFLOP/s)",
                      "algorithmic_bytes_per_launch": r["bytes"],
                      "hbm_gbs_at_that_time": r["bytes"] / (r["ms"] * 1e-3) / 1e9,
                      "hbm_peak_gbs_measured": pk.get("hbm_gbs")}
    # the kernel with the largest share of the step in the launch list (profiles/)
    roof = roofs.get(DOMINANT_KERNEL)
    line = {
        "metric": "time-to-1e-8 residual & GDoF/s per sweep: decoupled vs strain, FP32-refined vs FP64",
        "value": value, "unit": "GDoF/s (solved to 1e-8)", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n, args.beta, ws),
        "solve": {"time_to_1e8_s": ms * 1e-3, "iterations": iters, "final_rel_res": final_res,
                  "free_dofs": int(free), "setup_s": setup_s},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        "roofline_other_kernels": {k: v for k, v in roofs.items() if k != DOMINANT_KERNEL},
    }
    line.update({k: v for k, v in extra.items() if k != "roofline_kernel"})
    print(json.dumps(line), flush=True)


def _time(fn, reps, stream, torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _guarded(block):
    """Run one supplementary measurement block; a failure is reported in its place (with the
    exception) instead of taking the benchmark line, measured before it, down with it."""
    try:
        return block()
    except Exception as e:  # noqa: BLE001 - reported in the output line
        return {"error": repr(e)}


def measure_details(args, H, prob, b, x, nodes, free, stream, torch, sdx, W):
    out = {}
    n = prob.n
    nn = nodes
    con = torch.from_numpy(H.sdx_constraint_mask(0)).to(b.device)
    xr = torch.from_numpy(W.random_vector(n, 5).ravel()).to(b.device)
    xr[con] = 0.0
    y = torch.empty_like(xr)
    reps = 20
    t_apply = _time(lambda: H.sdx_apply(0, xr, y), reps, stream, torch)
    xs = xr.clone()
    t_vel = _time(lambda: H.sdx_smooth_pass(0, 0, 0, b, xs), reps, stream, torch)
    t_pre = _time(lambda: H.sdx_smooth_pass(0, 1, 0, b, xs), reps, stream, torch)
    t_uz = _time(lambda: H.sdx_uzawa(0, b, xs), 5, stream, torch)
    xv = torch.zeros_like(b)
    t_vc = _time(lambda: H.sdx_vcycle(b, xv), 3, stream, torch)
    half = nn / 2.0
    sweeps = {
        "apply_K1_K2": {"ms": t_apply, "gdofs": free / (t_apply * 1e-3) / 1e9, "bytes_per_node": 64},
        "velocity_pass": {"ms": t_vel, "gdofs": (3 * half) / (t_vel * 1e-3) / 1e9, "bytes_per_node": 58},
        "pressure_pass": {"ms": t_pre, "gdofs": half / (t_pre * 1e-3) / 1e9, "bytes_per_node": 44},
        "uzawa_step": {"ms": t_uz, "gdofs": free / (t_uz * 1e-3) / 1e9},
        "vcycle_ms": t_vc,
    }
    for k in ("apply_K1_K2", "velocity_pass", "pressure_pass"):
        s = sweeps[k]
        s["gbs"] = s["bytes_per_node"] * nn / (s["ms"] * 1e-3) / 1e9
    out["sweeps_fp64_decoupled"] = sweeps
    # algorithmic flops of one velocity colour pass (decoupled, per updated node):
    # 3 x (7-point Laplacian 8 + B^T p row 16 + update 4) + 7 shared p differences = 91
    out["roofline_kernel"] = {"velocity_pass": {"ms": t_vel, "flops": 91.0 * half, "bytes": 58.0 * nn},
                              # pressure pass, per updated node: B u row 21 differences + 3 x 13
                              # for their weighted sums, C p 8, update 4 = 72
                              "pressure_pass": {"ms": t_pre, "flops": 72.0 * half, "bytes": 44.0 * nn}}
    out["vcycle_levels_fp64"] = _guarded(lambda: level_gbs(level_times(H, sdx, torch, stream, "fp64")))
    out["sweeps_fp32_decoupled"] = _guarded(lambda: fp32_sweeps(prob, xr, b, con, nn, stream, torch, sdx))
    out["cube_inclusion_16"] = _guarded(lambda: run_cube16(sdx, torch, W, stream))
    # e2e: through the host-buffer entry point
    bh = b.cpu().numpy().copy()
    xh = np.zeros_like(bh)
    H.sdx_solve_host(bh, xh, rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)
    t0 = time.perf_counter()
    k_e2e = max(1, min(args.steps, 3))
    for _ in range(k_e2e):
        xh[:] = 0.0
        H.sdx_solve_host(bh, xh, rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)
    te = (time.perf_counter() - t0) / k_e2e
    out["e2e"] = {"value": free / te / 1e9, "unit": "GDoF/s (solved to 1e-8)",
                  "h2d_bytes_per_step": int(2 * bh.nbytes), "d2h_bytes_per_step": int(xh.nbytes),
                  "entry_point": "sdx_solve_host (host b and x0 in, host x out)"}
    if not args.no_variants:
        var = {}
        for name, form, prec, cform in (("strain_fp64", "sym", sdx.PREC_FP64, None),
                                        ("decoupled_tr_coarse_fp64", "tr", sdx.PREC_FP64, None),
                                        ("decoupled_fp32_refined", "tr", sdx.PREC_FP32_REFINED, "sym"),
                                        ("strain_fp32_refined", "sym", sdx.PREC_FP32_REFINED, None),
                                        ("decoupled_tr_coarse_fp32_refined", "tr", sdx.PREC_FP32_REFINED, None)):
            H2 = sdx.Hierarchy.from_problem(prob, form=form, prec=prec, coarse_form=cform, beta=args.beta)
            x2 = torch.zeros_like(b)
            st = H2.sdx_solve(b, x2, rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)
            reps2 = 2
            tt = _time(lambda: (x2.zero_(), H2.sdx_solve(b, x2, rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)), reps2, stream, torch)
            st = H2.sdx_solve(b, x2.zero_(), rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)
            dx = solution_diff(x2, x, nn) if form == "tr" else None
            var[name] = {"time_to_1e8_s": tt * 1e-3, "gdofs": free / (tt * 1e-3) / 1e9,
                         "iterations": st["iterations"], "final_rel_res": st["res"] / st["bnorm"],
                         "coarse_levels": cform or form,
                         "rel_l2_diff_vs_headline_solution": dx}
            if form == "sym":
                ta = _time(lambda: H2.sdx_apply(0, xr, y), reps, stream, torch)
                tv = _time(lambda: H2.sdx_smooth_pass(0, 0, 0, b, xs), reps, stream, torch)
                var[name]["apply_ms"] = ta
                var[name]["velocity_pass_ms"] = tv
            H2.close()
        out["variants"] = var
    if not args.no_layer:
        out["top_layer_256"] = _guarded(lambda: run_layer(args, sdx, torch, W, stream))
    if not args.no_batch:
        out["batched_48"] = _guarded(lambda: run_batch(args, sdx, torch))
    if not args.no_guess:
        out["learned_guess"] = _guarded(lambda: run_guess(args, sdx, torch))
    if not args.no_paper:
        out["paper_columns"] = _guarded(lambda: run_paper(args, sdx, torch))
        out["p1p0"] = _guarded(lambda: run_p1p0(args, sdx, torch))
    if not args.no_cpu and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        out["cpu_baseline"] = _guarded(lambda: oracle_sample(args.beta))
    return out


def solution_diff(xa, xb, nn):
    """Relative L2 difference of two solutions after removing the difference's pressure mean
    (without a traction face the pressure is determined up to a constant)."""
    d = xa - xb
    d[3 * nn:] -= d[3 * nn:].mean()
    return float(d.norm() / xb.norm())


def run_layer(args, sdx, torch, W, stream):
    """256^3 cells, top layer z >= 7/8 of viscosity 1e3, traction-free top, free-slip sides,
    no-slip bottom, Gaussian-blob buoyancy: FP64 cycles vs FP32 cycles in FP64 refinement,
    decoupled form (a_sym on the coarse levels), FGMRES to 1e-8."""
    prob = W.top_layer(256, 8)
    f = torch.from_numpy(prob.nodal_forcing().ravel()).cuda()
    res = {"workload": "top_layer_256: 256^3 cells, layer z >= 7/8 mu 1e3 over mu 1, traction top, free-slip sides, no-slip bottom, Gaussian-blob forcing"}
    sols = {}
    for name, prec in (("fp64", sdx.PREC_FP64), ("fp32_refined", sdx.PREC_FP32_REFINED)):
        t0 = time.perf_counter()
        H = sdx.Hierarchy.from_problem(prob, form="tr", coarse_form="sym", prec=prec)
        setup = time.perf_counter() - t0
        _, nn, free = H.sdx_level_size(0)
        b = torch.zeros(4 * nn, dtype=torch.float64, device="cuda")
        H.sdx_rhs(f, b)
        x = torch.zeros_like(b)
        st = H.sdx_solve(b, x, rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)
        tt = _time(lambda: (x.zero_(), H.sdx_solve(b, x, rtol=1e-8, maxit=500, outer=sdx.OUTER_FGMRES, restart=30)), 2, stream, torch)
        res[name] = {"time_to_1e8_s": tt * 1e-3, "gdofs": free / (tt * 1e-3) / 1e9, "iterations": st["iterations"],
                     "final_rel_res": st["res"] / st["bnorm"], "free_dofs": free, "setup_s": setup}
        sols[name] = x
        H.close()
    d = sols["fp32_refined"] - sols["fp64"]
    res["fp32_refined"]["rel_l2_diff_vs_fp64_solution"] = float(d.norm() / sols["fp64"].norm())
    res["speedup_fp32_refined_vs_fp64"] = res["fp64"]["time_to_1e8_s"] / res["fp32_refined"]["time_to_1e8_s"]
    return res


def run_batch(args, sdx, torch, count=None):
    """48 independent instances, sizes uniform in {32,48,64,96}^3, 1-4 boxes, contrast
    log-uniform in [1, 1e6], Gaussian-blob forcing; FP32 cycles in FP64 refinement, decoupled
    form (a_sym on the coarse levels); one batch (the persistent work-queue solver, and the
    lock-step solver with one launch per phase) vs the same instances solved one after another."""
    from paper_1604_07994_gb300 import workloads as W
    count = count or args.batch_count
    probs = W.batched_instances(count)
    t0 = time.perf_counter()
    B = sdx.Batch(probs, prec=sdx.PREC_FP32_REFINED, coarse_form="sym", autotune=True)
    setup = time.perf_counter() - t0
    bs, xs, free, sizes = [], [], 0, []
    for i, p in enumerate(probs):
        H = B.instance(i)
        free += H.sdx_level_size(0)[2]
        sizes.append([H.sdx_level_size(l)[1:] for l in range(H.sdx_levels())])  # (nodes, free) per level
        f = torch.from_numpy(p.nodal_forcing().ravel()).cuda()
        b = torch.zeros(4 * p.nodes, dtype=torch.float64, device="cuda")
        H.sdx_rhs(f, b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    def timed(lockstep):
        if lockstep:
            os.environ["SDX_BATCH_LOCKSTEP"] = "1"
        else:
            os.environ.pop("SDX_BATCH_LOCKSTEP", None)
        st = B.sdx_batch_solve(bs, xs, rtol=1e-8, maxit=400, restart=30)
        torch.cuda.synchronize()
        l0 = sdx.sdx_kernel_launches()
        ts = []
        for _ in range(3):
            for x in xs:
                x.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            st = B.sdx_batch_solve(bs, xs, rtol=1e-8, maxit=400, restart=30)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t1)
        os.environ.pop("SDX_BATCH_LOCKSTEP", None)
        return min(ts), (sdx.sdx_kernel_launches() - l0) / 3, st
    t_lock, launches_lock, st_lock = timed(True)
    tb, launches, st = timed(False)
    its = [s["iterations"] for s in st]
    shapes = [B.sdx_batch_shape(lv) for lv in range(4)]
    # the same instances, one hierarchy after another (same solver settings)
    tseq, its_seq = 0.0, []
    for p, b in zip(probs, bs):
        H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form="sym", prec=sdx.PREC_FP32_REFINED)
        x = torch.zeros_like(b)
        H.sdx_solve(b, x, rtol=1e-8, maxit=400, outer=sdx.OUTER_FGMRES, restart=30)
        x.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s1 = H.sdx_solve(b, x, rtol=1e-8, maxit=400, outer=sdx.OUTER_FGMRES, restart=30)
        torch.cuda.synchronize()
        tseq += time.perf_counter() - t1
        its_seq.append(s1["iterations"])
        H.close()
    B.close()
    # algorithmic bytes of the solves (a lower bound of their traffic): per FGMRES iteration one
    # FP32 V_var(3,3) cycle (per level l with N_l nodes: 2 nu_l Uzawa steps of 3 velocity passes
    # x 30 B and 2 pressure passes x 24 B per node, the residual 34 B, restriction 16 + 16 and
    # prolongation 16 + 32 B per fine / coarse node; the coarsest dense FP64 mat-vec) and one FP64
    # operator apply (64 B per node); Krylov vectors and the FP64/FP32 conversions not counted
    pk = peaks().get("hbm_gbs")
    total = 0.0
    for lv, it in zip(sizes, its):
        ns = [nodes for nodes, _ in lv]
        cyc = 0.0
        for l, N in enumerate(ns[:-1]):
            nu = 3 + 2 * l
            cyc += N * (2 * nu * (3 * 30 + 2 * 24) + 34 + 16 + 32) + ns[l + 1] * (16 + 16)
        cyc += 8.0 * float(lv[-1][1]) ** 2  # the coarsest inverse over its free unknowns
        total += it * (cyc + 64.0 * ns[0])
    hbm = {"algorithmic_gbs_lower_bound": total / tb / 1e9,
           "frac_of_measured_hbm": total / tb / 1e9 / pk if pk else None,
           "lockstep_frac_of_measured_hbm": total / t_lock / 1e9 / pk if pk else None,
           "counted": "per FGMRES iteration: the FP32 V-cycle's passes, residuals and transfers on every level, the coarsest mat-vec, one FP64 apply; Krylov vectors and conversions not counted"}
    return {"workload": f"{count} instances, sizes {sorted(set(p.n for p in probs))}^3 cells, 1-4 boxes, contrast log-uniform in [1, 1e6], Gaussian-blob forcing",
            "hbm_roofline": hbm,
            "total_free_dofs": int(free), "time_to_1e8_s": tb, "gdofs": free / tb / 1e9, "all_converged": all(s["status"] == 0 for s in st),
            "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)), "setup_s": setup,
            "gpu_launches_per_solve": int(launches), "block_shapes_per_level": shapes,
            "solver": "one persistent launch over a device work queue: per-instance FGMRES(30) + V_var(3,3), no host synchronisation until the batch is done",
            "lockstep_per_phase_launches": {"time_to_1e8_s": t_lock, "gdofs": free / t_lock / 1e9,
                                            "gpu_launches_per_solve": int(launches_lock),
                                            "iterations_max": int(max(s["iterations"] for s in st_lock))},
            "sequential_single_solves_s": tseq, "sequential_iterations_mean": float(np.mean(its_seq)),
            "sequential_gdofs": free / tseq / 1e9,
            "speedup_batched_vs_sequential": tseq / tb, "speedup_queue_vs_lockstep": t_lock / tb}


def vcycle_rate(torch, vcycle, residual, x, nn, w=None, cycles=40, last=10):
    """Asymptotic residual reduction rate of the plain V-cycle iteration x <- x + M(0 - K x)
    (Sec. 5, Table timeANDconv) from the start vector x [4 nn], updated in place: vcycle(x)
    runs one cycle on x with a zero right-hand side, residual(x) returns K x up to sign.  The
    iterate is renormalised to a unit residual after every cycle, and, when the pressure has a
    constant mode (no traction face; weights w of sum_b w_b p_b = 0 given), that mode is
    projected out first: it lies in the kernel of K, so without the projection the
    renormalisation amplifies it until rounding in K x dominates the residual.  Returns the
    geometric mean of the last `last` reductions and all of them."""
    def project():
        if w is not None:
            x[3 * nn:] -= torch.dot(w, x[3 * nn:]) / w.sum()
    project()
    prev = float(torch.linalg.norm(residual(x)))
    rates = []
    for _ in range(cycles):
        vcycle(x)
        project()
        cur = float(torch.linalg.norm(residual(x)))
        rates.append(cur / prev)
        x /= cur
        prev = 1.0
    return float(np.exp(np.mean(np.log(rates[-last:])))), rates


def run_paper(args, sdx, torch, cycles=40):
    """The paper's own measurement (Sec. 5, Table timeANDconv): the viscosity-columns problem
    with free-slip faces at levels 5 (128^3 cells) and 6 (256^3), time of one V_var(3,3) cycle
    and the asymptotic residual reduction rate rho for the strain, decoupled ("modified
    stencil") and gradient forms.  rho: plain V-cycles from a seeded random x, renormalised and
    with the pressure constant projected out every cycle (vcycle_rate), geometric mean of the
    last 10 reductions."""
    from paper_1604_07994_gb300 import workloads as W
    out = {"problem": "viscosity columns (Sec. 4.2.4), free-slip faces, coarsest grid 8^3, FP64",
           "paper_xeon_32_cores": {"L5": {"strain": [1.18, 0.296], "decoupled": [1.12, 0.244], "gradient": [1.34, 0.240]},
                                   "L6": {"strain": [3.02, 0.280], "decoupled": [2.45, 0.242], "gradient": [2.64, 0.240]},
                                   "columns": "[seconds per V_var(3,3) cycle, rho]"}}
    for lvl, n in (("L5", 128), ("L6", 256)):
        prob = W.viscosity_columns(n, 8)
        cell_mu = torch.from_numpy(np.ascontiguousarray(prob.cell_mu(), dtype=np.float64)).cuda()
        w = pressure_weights_t(torch, n, cell_mu)
        res = {}
        for name, form in (("strain", "sym"), ("decoupled", "tr"), ("gradient", "grad")):
            H = sdx.Hierarchy.from_problem(prob, form=form, prec=sdx.PREC_FP64)
            _, nn, _ = H.sdx_level_size(0)
            con = torch.from_numpy(H.sdx_constraint_mask(0)).cuda()
            x = torch.from_numpy(W.random_vector(n, 77).ravel()).cuda()
            x[con] = 0
            zero = torch.zeros_like(x)
            r = torch.empty_like(x)

            def residual(v):
                H.sdx_residual(0, zero, v, r)
                return r

            rho, rates = vcycle_rate(torch, lambda v: H.sdx_vcycle(zero, v), residual, x, nn, w, cycles)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                H.sdx_vcycle(zero, x)
            e1.record()
            torch.cuda.synchronize()
            res[name] = {"seconds_per_cycle": e0.elapsed_time(e1) / 5e3, "rho": rho,
                         "reductions_first_last": [rates[:3], rates[-3:]]}
            H.close()
        out[lvl] = res
    out["relative_differences"] = run_paper_tables(args, sdx, torch)
    out["relative_differences_layers"] = run_paper_tables(args, sdx, torch, problem="layers")
    return out


def _kuhn_vertex_offsets():
    """The six Kuhn tetrahedra of a cube: for each axis permutation s the vertices c, c + e_s1,
    c + e_s1 + e_s2, c + (1,1,1), as (di, dj, dk) offsets from the cube's lowest corner c."""
    from itertools import permutations
    out = []
    for s in permutations(range(3)):
        off = [0, 0, 0]
        verts = [(0, 0, 0)]
        for ax in s:
            off[ax] += 1
            verts.append(tuple(off))
        out.append(verts)
    return out


def _corner(g, n, d):
    """View of a nodal grid g [(n+1)^3, index (k, j, i)] at corner d = (di, dj, dk) of every cell."""
    return g[d[2]:d[2] + n, d[1]:d[1] + n, d[0]:d[0] + n]


def _mass_quadratic(torch, v, n, weight):
    """v^T M_w v for one nodal P1 field v [(n+1)^3] (x fastest): the consistent mass matrix
    with a per-cell weight w, per tetrahedron |T| w ((sum_a v_a)^2 + sum_a v_a^2) / 20."""
    g = v.reshape(n + 1, n + 1, n + 1)
    tot = torch.zeros((), dtype=v.dtype, device=v.device)
    for verts in _kuhn_vertex_offsets():
        c = [_corner(g, n, d) for d in verts]
        s = c[0] + c[1] + c[2] + c[3]
        q = c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]
        tot = tot + (weight * (s * s + q)).sum()
    return tot * (1.0 / (6.0 * n ** 3)) / 20.0


def pressure_weights_t(torch, n, cell_mu):
    """w_b = int lambda_b / mu = sum over the tetrahedra T at node b of |T| / (4 mu_T), the
    weights of the discrete constraint int p / mu = 0 (cell_mu: [n, n, n] as (k, j, i))."""
    w = torch.zeros((n + 1,) * 3, dtype=torch.float64, device=cell_mu.device)
    share = (1.0 / (6.0 * n ** 3) / 4.0) / cell_mu
    for verts in _kuhn_vertex_offsets():
        for d in verts:
            _corner(w, n, d).add_(share)
    return w.reshape(-1)


def table_norms(torch, x, n, cell_mu, apply_sym):
    """The norms of the paper's error tables (Sec. 3 definitions) of an SoA pair x = (u, p)
    [4 (n+1)^3]: ||u||_0 (consistent mass), ||u||_V = a_sym(u, u)^(1/2) from apply_sym (the
    strain-form operator applied to (u, 0)), ||p||_Q = (p / (2 mu), p)_0^(1/2)."""
    nn = (n + 1) ** 3
    l2 = sum(float(_mass_quadratic(torch, x[c * nn:(c + 1) * nn], n, 1.0)) for c in range(3)) ** 0.5
    v = x.clone()
    v[3 * nn:] = 0.0
    y = apply_sym(v)
    en = float(torch.dot(v[:3 * nn], y[:3 * nn])) ** 0.5
    q = float(_mass_quadratic(torch, x[3 * nn:], n, 0.5 / cell_mu)) ** 0.5
    return np.array([l2, en, q])


def relative_differences(torch, sols, n, cell_mu, apply_sym, ref="strain"):
    """||X - U|| / ||U|| in the three table norms for every solution X in sols against U =
    sols[ref], pressures first normalised to int p / mu = 0 (no traction face)."""
    nn = (n + 1) ** 3
    w = pressure_weights_t(torch, n, cell_mu)
    sols = {k: v.clone() for k, v in sols.items()}
    for v in sols.values():
        v[3 * nn:] -= torch.dot(w, v[3 * nn:]) / w.sum()
    U = sols[ref]
    base = table_norms(torch, U, n, cell_mu, apply_sym)
    return {k: (table_norms(torch, v - U, n, cell_mu, apply_sym) / base).tolist()
            for k, v in sols.items() if k != ref}


# The paper's P1-P1 relative differences to the strain form on the columns problem (Sec. 4.2.4,
# tables "columns-laplace-p1p1" and "columns-stencil-p1p1"): [||.||_0, ||.||_V, ||.||_Q].
PAPER_COLUMNS_P1P1 = {
    2: {"gradient": [7.4550e-02, 9.2581e-02, 2.7609e-01], "decoupled": [1.3890e-02, 2.4189e-02, 7.7949e-02]},
    3: {"gradient": [3.0104e-02, 6.0398e-02, 1.8003e-01], "decoupled": [4.2414e-03, 1.2312e-02, 4.8195e-02]},
    4: {"gradient": [2.1227e-02, 4.7364e-02, 1.1179e-01], "decoupled": [1.1370e-03, 6.2303e-03, 2.5287e-02]},
    5: {"gradient": [2.0227e-02, 4.3246e-02, 8.0546e-02], "decoupled": [2.9449e-04, 3.1918e-03, 1.3274e-02]},
    6: {"gradient": [2.0098e-02, 4.2121e-02, 6.9997e-02], "decoupled": [7.5985e-05, 1.6675e-03, 6.8175e-03]},
}


# The paper's P1-P0 relative differences on the layers problem (Sec. 4.2.3, tables
# "layers-laplace" and "layers-stencil"; no P1-P1 table is printed for it).
PAPER_LAYERS_P1P0 = {
    2: {"gradient": [3.1359e-01, 4.8968e-01, 2.5337e-01], "decoupled": [3.6872e-02, 5.2343e-02, 5.9058e-02]},
    3: {"gradient": [3.1095e-01, 5.1625e-01, 2.6207e-01], "decoupled": [1.0722e-02, 2.2601e-02, 2.1634e-02]},
    4: {"gradient": [3.0922e-01, 5.2354e-01, 2.6458e-01], "decoupled": [2.8306e-03, 1.0224e-02, 8.3074e-03]},
}


def run_paper_tables(args, sdx, torch, levels=(2, 3, 4, 5, 6), problem="columns"):
    """The paper's error tables of the columns problem (Sec. 4.2.4) or the layers problem
    (Sec. 4.2.3) on the GPU path: at level L (4 * 2^L cells per side, coarsest grid 8^3 below
    level 2's 16^3) solve the strain, decoupled and gradient forms to 1e-10 with FGMRES +
    V_var(3,3), then report the relative differences of the decoupled and gradient solutions
    to the strain solution in ||.||_0, ||.||_V and ||.||_Q beside the paper's values."""
    from paper_1604_07994_gb300 import workloads as W
    if problem == "columns":
        make, paper = W.viscosity_columns, {"paper_p1p1": PAPER_COLUMNS_P1P1}
        title = "viscosity columns (Sec. 4.2.4), FP64, solves to 1e-10"
    else:
        make, paper = W.viscosity_layers, {"paper_p1p0": PAPER_LAYERS_P1P0}
        title = "viscosity layers (Sec. 4.2.3), FP64, solves to 1e-10"
    out = {"problem": title,
           "norms": "[||u||_0, ||u||_V = a_sym(u,u)^1/2, ||p||_Q = (p/(2mu), p)^1/2], relative to the strain solution"}
    for key, tab in paper.items():
        out[key] = {f"L{k}": v for k, v in tab.items() if k in levels}
    for lvl in levels:
        n = 4 * 2 ** lvl
        prob = make(n, 8)
        f = torch.from_numpy(prob.nodal_forcing().ravel()).cuda()
        cell_mu = torch.from_numpy(np.ascontiguousarray(prob.cell_mu(), dtype=np.float64)).cuda()
        sols, solves, H_sym = {}, {}, None
        try:
            for name, form in (("strain", "sym"), ("decoupled", "tr"), ("gradient", "grad")):
                H = sdx.Hierarchy.from_problem(prob, form=form, prec=sdx.PREC_FP64)
                _, nn, _ = H.sdx_level_size(0)
                b = torch.zeros(4 * nn, dtype=torch.float64, device="cuda")
                H.sdx_rhs(f, b)
                x = torch.zeros_like(b)
                t0 = time.perf_counter()
                st = H.sdx_solve(b, x, rtol=1e-10, maxit=300, outer=sdx.OUTER_FGMRES, restart=30, allow_noconv=True)
                torch.cuda.synchronize()
                solves[name] = {"iterations": st["iterations"], "final_rel_res": st["res"] / st["bnorm"],
                                "seconds": time.perf_counter() - t0}
                sols[name] = x
                if form == "sym":
                    H_sym = H
                else:
                    H.close()

            def apply_sym(v):
                y = torch.empty_like(v)
                H_sym.sdx_apply(0, v, y)
                return y

            out[f"L{lvl}"] = {"cells": n, "solves": solves,
                              "relative_differences": relative_differences(torch, sols, n, cell_mu, apply_sym)}
        except Exception as e:  # a measurement block: report, keep the benchmark line
            out[f"L{lvl}"] = {"cells": n, "solves": solves, "error": repr(e)}
        finally:
            if H_sym is not None:
                H_sym.close()
    return out


def run_conv(args, sdx, torch):
    """The network alone on an n^3 cell grid: time of one forward pass and of one forward +
    backward pass (loss and all gradients) from seeded random inputs; algorithmic tensor
    flops = sum over layers of 2 * cells * 27 * C_in * C_out (forward), three times that with
    the backward pass (input and weight gradients)."""
    n = args.conv_n
    rng = np.random.Generator(np.random.PCG64(12))
    V = n ** 3
    x = torch.from_numpy(rng.standard_normal((V, 16)).astype(np.float32)).cuda().to(torch.bfloat16)
    t = torch.from_numpy(rng.standard_normal((V, 16)).astype(np.float32)).cuda()
    y = torch.empty((V, 16), dtype=torch.float32, device="cuda")
    net = sdx.Net(seed=5)
    layers = [(16, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 32, 1), (32, 32, 1),
              (32, 16, 0), (16, 16, 0), (16, 16, 0)]
    fwd_flops = sum(2.0 * (V / 8 ** lv) * 27 * ci * co for ci, co, lv in layers)
    stream = torch.cuda.current_stream()
    t_f = _time(lambda: net.forward(n, x, y), 5, stream, torch)
    t_fb = _time(lambda: net.loss_grad(n, x, t), 5, stream, torch)
    pk = peaks().get("bf16_tflops")
    # single convolutions of every shape at its level's size: brick kernel vs per-tap gather
    single = {}
    for ci, co, lv in sorted(set(layers)):
        m = n >> lv
        xs = torch.from_numpy(rng.standard_normal((m ** 3, ci)).astype(np.float32)).cuda().to(torch.bfloat16)
        ws = torch.from_numpy((rng.standard_normal((27, co, ci)) / np.sqrt(27 * ci)).astype(np.float32)).cuda().to(torch.bfloat16)
        ys = torch.empty((m ** 3, co), dtype=torch.float32, device="cuda")
        fl = 2.0 * m ** 3 * 27 * ci * co
        row = {}
        for tag, env in (("brick", None), ("gather", "1")):
            if env:
                os.environ["SDX_CONV_GATHER"] = env
            else:
                os.environ.pop("SDX_CONV_GATHER", None)
            tt = _time(lambda: sdx.sdx_conv3(m, ci, co, xs, ws, None, 0, ys), 10, stream, torch)
            row[tag] = {"ms": tt, "tflops": fl / (tt * 1e-3) / 1e12}
        os.environ.pop("SDX_CONV_GATHER", None)
        dz = torch.from_numpy(rng.standard_normal((m ** 3, co)).astype(np.float32)).cuda().to(torch.bfloat16)
        dw = torch.zeros((27, co, ci), dtype=torch.float32, device="cuda")
        tw = _time(lambda: sdx.sdx_conv3_wgrad(m, ci, co, xs, dz, dw), 10, stream, torch)
        row["wgrad"] = {"ms": tw, "tflops": fl / (tw * 1e-3) / 1e12}
        single[f"{ci}->{co} at {m}^3"] = row
    # inference on the 128^3 evaluation grid (the learned guess's use)
    t_inf = None
    if n != 128:
        V2 = 128 ** 3
        x2 = torch.from_numpy(rng.standard_normal((V2, 16)).astype(np.float32)).cuda().to(torch.bfloat16)
        y2 = torch.empty((V2, 16), dtype=torch.float32, device="cuda")
        t_inf = _time(lambda: net.forward(128, x2, y2), 5, stream, torch)
    return {"n": n, "cells": V, "forward_ms": t_f, "forward_backward_ms": t_fb,
            "forward_tflops": fwd_flops / (t_f * 1e-3) / 1e12, "train_step_tflops": 3 * fwd_flops / (t_fb * 1e-3) / 1e12,
            "forward_128_ms": t_inf, "single_convolutions": single, "bf16_peak_tflops_measured": pk}


def run_guess(args, sdx, torch):
    """Learned initial guess: train the network on solves at 64^3 (random boxes, contrast
    1-1e4, Gaussian blobs), then solve unseen 128^3 layouts from zero and from the guess to the
    same residual; times of the guess include the prediction."""
    from paper_1604_07994_gb300 import guess, workloads as W
    X, T, gen = guess.training_set(args.guess_samples, n=64)
    net = sdx.Net(seed=11)
    hist, t_train = guess.train(net, X, T, epochs=args.guess_epochs, batch=8, lr=2e-3)
    evalp = [W.random_instance(128, 8, 90000 + k, 8, log10_contrast=(0.0, 4.0), forcing="blobs")
             for k in range(args.guess_eval)]
    steps = tuple(int(k) for k in args.guess_smooth.split(","))
    ev = guess.evaluate(net, evalp, smooth_steps=steps)
    out = {"training_set": gen, "epochs": args.guess_epochs, "train_s": t_train, "loss_first_last": [hist[0], hist[-1]],
           "eval": ev, "iterations_zero_mean": float(np.mean([e["zero"]["iterations"] for e in ev]))}
    z = sum(e["zero"]["seconds"] for e in ev)
    for k in steps:
        key = f"guess_s{k}"
        out[f"iterations_{key}_mean"] = float(np.mean([e[key]["iterations"] for e in ev]))
        out[f"wall_time_saved_frac_{key}"] = (z - sum(e[key]["seconds"] for e in ev)) / z
    return out


def level_gbs(rows):
    """Algorithmic GB/s of the transfers per level (FP64): restriction reads the fine residual
    (32 B per fine node) and writes the coarse right-hand side (32 B per coarse node);
    prolongation reads the coarse correction (32 B per coarse node) and reads and writes the
    fine iterate (64 B per fine node)."""
    for l, row in enumerate(rows[:-1]):
        nf, nc = row["nodes"], rows[l + 1]["nodes"]
        if "restrict_ms" in row:
            row["restrict_gbs"] = (32 * nf + 32 * nc) / (row["restrict_ms"] * 1e-3) / 1e9
            row["prolong_gbs"] = (32 * nc + 64 * nf) / (row["prolong_ms"] * 1e-3) / 1e9
    return rows


def fp32_sweeps(prob, xr, b, con, nn, stream, torch, sdx, reps=20):
    """The FP32 kernels of the refined solve's cycle on the finest level of the benchmark
    workload: apply, red velocity pass, red pressure pass, with algorithmic GB/s (FP32 bytes
    per node: apply 32 + 2, velocity pass 7 x 4 + 2, pressure pass 5.5 x 4 + 2) and the
    velocity pass as an HBM roofline against the measured copy bandwidth."""
    H = sdx.Hierarchy.from_problem(prob, form="tr", coarse_form="sym", prec=sdx.PREC_FP32_REFINED)
    try:
        x32 = xr.float()
        b32 = b.float()
        b32[con] = 0.0
        y = torch.empty_like(x32)
        xs = x32.clone()
        t = {"apply": _time(lambda: H.sdx_apply_f32(0, x32, y), reps, stream, torch),
             "velocity_pass": _time(lambda: H.sdx_smooth_pass_f32(0, 0, 0, b32, xs), reps, stream, torch),
             "pressure_pass": _time(lambda: H.sdx_smooth_pass_f32(0, 1, 0, b32, xs), reps, stream, torch)}
        xv = torch.zeros_like(x32)
        bpn = {"apply": 34, "velocity_pass": 30, "pressure_pass": 24}
        out = {k: {"ms": v, "bytes_per_node": bpn[k], "gbs": bpn[k] * nn / (v * 1e-3) / 1e9} for k, v in t.items()}
        out["uzawa_step_ms"] = _time(lambda: H.sdx_uzawa_f32(0, b32, xs, 1), 5, stream, torch)
        pk = peaks().get("hbm_gbs")
        g = out["velocity_pass"]["gbs"]
        out["roofline_fp32"] = {"bound": "hbm", "achieved": g, "peak": pk, "unit": "GB/s",
                                "frac": g / pk if pk else None, "traffic": None,
                                "kernel": "red FP32 velocity pass (special rows staged + k_vel_uniform<float, a_tr>)",
                                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)"}
        del xv
        return out
    finally:
        H.close()


def run_cube16(sdx, torch, W, stream):
    """The 16^3 cube inclusion ([0.25, 0.75]^3, mu 10 inside, 1 outside, no-slip, manufactured
    forcing), FP64 decoupled form: one operator apply and a solve to 1e-8 from zero."""
    p = W.cube_inclusion(16, 4)
    H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form="sym", prec=sdx.PREC_FP64)
    try:
        _, nodes, free = H.sdx_level_size(0)
        b = torch.zeros(4 * nodes, dtype=torch.float64, device="cuda")
        H.sdx_rhs(torch.from_numpy(p.nodal_forcing().ravel()).cuda(), b)
        y = torch.empty_like(b)
        t_ap = _time(lambda: H.sdx_apply(0, b, y), 20, stream, torch)
        x = torch.zeros_like(b)
        st = {}

        def solve():
            x.zero_()
            st.update(H.sdx_solve(b, x, rtol=1e-8, maxit=200, outer=sdx.OUTER_FGMRES, restart=30))
        t_s = _time(solve, 5, stream, torch)
        return {"cells": 16, "free_dofs": free, "apply_ms": t_ap, "time_to_1e8_ms": t_s,
                "iterations": st["iterations"], "final_rel_res": st["res"] / st["bnorm"]}
    finally:
        H.close()


def level_times(H, sdx, torch, stream, prec="fp64", reps=20):
    """CUDA-event times of the pieces of one V_var cycle on every level of a hierarchy: one
    Uzawa step (nu = 3 + 2l of them pre and post), the residual, restriction, prolongation, and
    the cycle time they add up to on that level (launched one call at a time, so each piece
    also carries its launch latency; inside the captured cycle the same kernels run back to
    back)."""
    nl = H.sdx_levels()
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = []
    vecs = []
    for l in range(nl):
        _, nodes, free = H.sdx_level_size(l)
        x = torch.zeros(4 * nodes, dtype=dt, device="cuda")
        b = torch.zeros(4 * nodes, dtype=dt, device="cuda")
        vecs.append((x, b, nodes, free))
    for l in range(nl):
        x, b, nodes, free = vecs[l]
        row = {"level": l, "nodes": nodes, "free_dofs": free}
        if l == nl - 1:
            out.append(row)
            continue
        nu = 3 + 2 * l
        if prec == "fp64":
            t_uz = _time(lambda: H.sdx_uzawa(l, b, x), reps, stream, torch)
            r = torch.empty_like(x)
            t_res = _time(lambda: H.sdx_residual(l, b, x, r), reps, stream, torch)
            bc = vecs[l + 1][1]
            t_rs = _time(lambda: H.sdx_restrict(l, r, bc), reps, stream, torch)
            t_pr = _time(lambda: H.sdx_prolong_add(l, vecs[l + 1][0], x), reps, stream, torch)
            row.update({"uzawa_step_ms": t_uz, "residual_ms": t_res, "restrict_ms": t_rs, "prolong_ms": t_pr,
                        "nu": nu, "level_cycle_ms": 2 * nu * t_uz + t_res + t_rs + t_pr})
        else:
            t_st = _time(lambda: H.sdx_uzawa_f32(l, b, x, nu), reps, stream, torch)
            y = torch.empty_like(x)
            t_ap = _time(lambda: H.sdx_apply_f32(l, x, y), reps, stream, torch)
            row.update({"nu_steps_ms": t_st, "apply_ms": t_ap, "nu": nu,
                        "level_cycle_ms": 2 * t_st + t_ap})
        out.append(row)
    return out


def run_p1p0(args, sdx, torch, levels=(0, 1, 2, 3, 4, 5)):
    """The P1-P0 scheme of Sec. 3 on the GPU: the Couette flow of Sec. 4.2.2 (mu1/mu2 = 1e3,
    exact Dirichlet data lifted through the residual, gamma = 1) at levels 0-5 (4^3 to 128^3
    cells): solve time, FGMRES iterations and the largest nodal velocity error against the
    exact solution (second order: the ratio between levels tends to 4); and the columns
    problem of Sec. 4.2.4 at 128^3: time to 1e-8, iterations and the largest element-wise mass
    imbalance of the post-processed fluxes relative to the largest flux."""
    from paper_1604_07994_gb300 import workloads as W
    out = {"couette": {}}
    prev = None
    for lvl in levels:
        n = 4 << lvl
        c = (np.arange(n) + 0.5) / n
        _, Y, _ = np.meshgrid(c, c, c, indexing="ij")  # [k, j, i]: y = j
        ids = (Y >= 0.5).astype(np.uint8)
        p = W.Problem(n=n, n_coarse=2 if n == 4 else 4, cell_id=ids, mu=np.array([1.0, 1e-3]),
                      face=(0,) * 6, forcing=None, name=f"couette_{n}")
        H = sdx.P1P0(p)
        _, nodes, tets, free = H.size(0)
        nn3 = 3 * nodes
        g = np.arange(n + 1) / n
        _, yy, xx = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
        u_ex = np.stack([0.5 * (1 - xx ** 2), xx * (yy - 0.5), 0 * xx]).ravel()
        bnd = np.zeros((n + 1,) * 3, dtype=bool)
        bnd[[0, -1]] = bnd[:, [0, -1]] = bnd[:, :, [0, -1]] = True
        con = np.tile(bnd.ravel(), 3)  # every face Dirichlet: the boundary nodes' components
        xD = np.concatenate([np.where(con, u_ex, 0.0), np.zeros(tets)])
        # load f = (3 mu, 0, 0): nodal values are the mean over the cells around each node
        mu_c = np.where(ids > 0, 1e-3, 1.0)
        fn = np.zeros((n + 1,) * 3)
        m = np.zeros((n + 1,) * 3)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    fn[dk:dk + n, dj:dj + n, di:di + n] += mu_c
                    m[dk:dk + n, dj:dj + n, di:di + n] += 1.0
        f = np.zeros((3, nodes))
        f[0] = (3.0 * fn / m).ravel()
        b = torch.zeros(nn3 + tets, dtype=torch.float64, device="cuda")
        H.rhs(torch.from_numpy(f.ravel()).cuda(), b)
        r = torch.empty_like(b)
        H.residual(0, b, torch.from_numpy(xD).cuda(), r)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = H.solve(r, x, rtol=1e-10, maxit=400, restart=30)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        uh = np.where(con, u_ex, x[:nn3].cpu().numpy())
        err = float(np.abs(uh - u_ex).max())
        row = {"cells": n, "free_dofs": free, "solve_s": ts, "iterations": st["iterations"],
               "max_nodal_velocity_error": err}
        if prev is not None:
            row["error_ratio_to_coarser"] = prev / err
        prev = err
        out["couette"][f"L{lvl}"] = row
    nc = 128 if args.n >= 128 else args.n
    p = W.viscosity_columns(nc, 4)
    H = sdx.P1P0(p, form="tr")
    _, nodes, tets, free = H.size(0)
    b = torch.zeros(3 * nodes + tets, dtype=torch.float64, device="cuda")
    H.rhs(torch.from_numpy(p.nodal_forcing().ravel()).cuda(), b)
    x = torch.zeros_like(b)
    H.solve(b, x, rtol=1e-8, maxit=400, restart=30)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = H.solve(b, x, rtol=1e-8, maxit=400, restart=30)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    flux = torch.empty(4 * tets, dtype=torch.float64, device="cuda")
    bal = torch.empty(tets, dtype=torch.float64, device="cuda")
    H.fluxes(x, flux, bal)
    # the operator apply against both roofs: algorithmic bytes = x read and y written once
    # (8 B per unknown each) plus the node info and cell ids (3 B per node); algorithmic flops =
    # 75 per node (7-point Laplacians 3 x 8, the P0 gradient over the 24 tetrahedra around the
    # node 48, scaling 3) + 14 per tetrahedron (divergence 6, four penalised facets 8)
    y = torch.empty_like(x)
    t_ap = _time(lambda: H.apply(0, x, y), 20, torch.cuda.current_stream(), torch)
    by = 16.0 * (3 * nodes + tets) + 3.0 * nodes
    fl = 75.0 * nodes + 14.0 * tets
    pk = peaks().get("hbm_gbs")
    fp64_peak = N_SM * FP64_PEAK_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    gbs, tfl = by / (t_ap * 1e-3) / 1e9, fl / (t_ap * 1e-3) / 1e12
    out["apply_128"] = {"ms": t_ap, "algorithmic_gbs": gbs, "frac_of_measured_hbm": gbs / pk if pk else None,
                        "algorithmic_tflops": tfl, "frac_of_fp64_peak": tfl / fp64_peak}
    out["columns"] = {"cells": nc, "free_dofs": free, "time_to_1e8_s": ts, "gdofs": free / ts / 1e9,
                      "iterations": st["iterations"],
                      "max_element_imbalance_over_max_flux": float(bal.abs().max() / flux.abs().max())}
    return out


def run_levels(args):
    """Per-level times of the V-cycle on the benchmark workload (decoupled form on the finest
    level, strain form below, as the headline solve), FP64 and FP32, and the whole captured
    cycle for comparison."""
    import torch
    from paper_1604_07994_gb300 import sdx
    from paper_1604_07994_gb300 import workloads as W
    torch.cuda.set_device(0)
    prob = W.three_boxes(args.n, 8, contrast=1e4)
    stream = torch.cuda.current_stream()
    res = {"mode": "levels", "n": args.n}
    for prec, p in (("fp64", sdx.PREC_FP64), ("fp32", sdx.PREC_FP32_REFINED)):
        H = sdx.Hierarchy.from_problem(prob, form="tr", coarse_form=args.coarse_form, prec=p, beta=args.beta)
        _, nodes, _ = H.sdx_level_size(0)
        b = torch.zeros(4 * nodes, dtype=torch.float64, device="cuda")
        f = torch.from_numpy(prob.nodal_forcing().ravel()).cuda()
        H.sdx_rhs(f, b)
        xv = torch.zeros_like(b)
        t_vc = _time(lambda: H.sdx_vcycle(b, xv), 10, stream, torch)
        lv = level_times(H, sdx, torch, stream, prec)
        res[prec] = {"vcycle_ms": t_vc, "levels": lv,
                     "finest_share": lv[0]["level_cycle_ms"] / max(sum(r.get("level_cycle_ms", 0) for r in lv), 1e-12)}
        H.close()
    print(json.dumps(res), flush=True)


def run_sweeps(args):
    """Per-sweep timing on the benchmark workload: operator apply, velocity and pressure
    colour passes of the finest level, FP64 or FP32, one form."""
    import torch
    from paper_1604_07994_gb300 import sdx
    from paper_1604_07994_gb300 import workloads as W
    torch.cuda.set_device(0)
    prob = W.three_boxes(args.n, 8, contrast=1e4)
    prec = sdx.PREC_FP64 if args.prec == "fp64" else sdx.PREC_FP32_REFINED
    H = sdx.Hierarchy.from_problem(prob, form=args.form, prec=prec, beta=args.beta)
    _, nn, free = H.sdx_level_size(0)
    dt = torch.float64 if args.prec == "fp64" else torch.float32
    con = torch.from_numpy(H.sdx_constraint_mask(0)).cuda()
    x = torch.from_numpy(W.random_vector(args.n, 5).ravel()).cuda().to(dt)
    bv = torch.from_numpy(W.random_vector(args.n, 6).ravel()).cuda().to(dt)
    x[con] = 0
    bv[con] = 0
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    if args.prec == "fp64":
        ops = {"apply": lambda: H.sdx_apply(0, x, y),
               "velocity_pass": lambda: H.sdx_smooth_pass(0, 0, 0, bv, x),
               "pressure_pass": lambda: H.sdx_smooth_pass(0, 1, 0, bv, x)}
    else:
        ops = {"apply": lambda: H.sdx_apply_f32(0, x, y),
               "velocity_pass": lambda: H.sdx_smooth_pass_f32(0, 0, 0, bv, x),
               "pressure_pass": lambda: H.sdx_smooth_pass_f32(0, 1, 0, bv, x)}
    w = 4 if args.prec == "fp32" else 8
    bytes_per_node = {"apply": 8 * w, "velocity_pass": 7 * w + 2, "pressure_pass": 5.5 * w + 2}
    res = {}
    for _ in range(args.warmup):
        for f in ops.values():
            f()
    torch.cuda.synchronize()
    for name, f in ops.items():
        ms = _time(f, args.steps, stream, torch)
        rows = free if name == "apply" else (3 * nn / 2 if name == "velocity_pass" else nn / 2)
        res[name] = {"ms": ms, "gdofs": rows / (ms * 1e-3) / 1e9,
                     "algorithmic_gbs": bytes_per_node[name] * nn / (ms * 1e-3) / 1e9}
    print(json.dumps({"mode": "sweep", "n": args.n, "prec": args.prec, "form": args.form, "nodes": nn,
                      "free_dofs": free, "sweeps": res}), flush=True)


if __name__ == "__main__":
    main()
