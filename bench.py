"""Benchmark: walker-moves per second of the SAIL annealing path on one GB300 (or N, one
independent inversion per GPU).

Workload (paper scale): 200 tau points uniform on [0, 8], 1000 bins on [0, 20], the
truncated double Lorentzian (centres 2 / 5, HWHM 0.3 / 0.5, weights 0.6 / 0.4), relative
noise 1e-4, 4096 walkers, FP32 moves with FP64 residual recomputation every 50 sweeps,
imprinted branching every 100 sweeps, a 20000-sweep geometric schedule T 10 -> 1e-9 (units
of the start residue).  One step is one block: 100 sweeps x 1000 moves x 4096 walkers =
4.096e8 walker-moves, plus two residual recomputations, the branching solve and imprint,
and the block statistics read back to the host.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import paper_scale_double_lorentz  # noqa: E402

N_TAU, N_OMEGA, N_WALKERS = 200, 1000, 4096
SWEEPS_PER_BLOCK, RESYNC_EVERY, N_SWEEPS = 100, 50, 20000
NOISE = 1e-4
WORKLOAD = (f"paper_scale_double_lorentz: N_tau={N_TAU} on [0,8], N_omega={N_OMEGA} on [0,20], "
            f"{N_WALKERS} walkers, sigma={NOISE:g}*F, FP32 moves, tensor-core (BF16 x6) resync every {RESYNC_EVERY} sweeps, "
            f"branching every {SWEEPS_PER_BLOCK} sweeps (f=1/4, t=0.1), {N_SWEEPS}-sweep schedule T 10->1e-9")
WORKLOAD_TO_TARGET = WORKLOAD.replace("schedule T 10->1e-9", "schedule T 1e6->0.03 absolute, move scale 0.1/N_omega")
METRIC = "walker-moves/s"
MOVES_PER_STEP = SWEEPS_PER_BLOCK * N_OMEGA * N_WALKERS


RESYNC_KIND = 2    # residual recomputation on the tensor cores (tcgen05, BF16, three pieces, six products)

# Time to target: each inversion runs until chi2 of its averaged spectrum is <= 1.2 N_tau
# (checked at every block end) or 20000 sweeps, on the schedule measured to reach that target
# (geometric from an absolute 1e6 to 0.03, move scale d = 0.1 / N_omega).
TTT_SWEEPS, TTT_T_START, TTT_T_END, TTT_D_FACTOR, TTT_TARGET = 20000, 1e6, 0.03, 0.1, 1.2
TTT_INVERSIONS = 4


def params_for(seed: int, timing: bool = True, resync_every: int = RESYNC_EVERY, resync_kind: int = RESYNC_KIND,
               sweep_lanes: int = 0, index_walk: int = 0, shared_bins: int = 0, sweep_loop: int = 0,
               noise: float = NOISE, schedule: str = "paper", fp64_accept: int = 0):
    import paper_1609_07936_gb300 as sail
    P = paper_scale_double_lorentz(noise, n_walkers=N_WALKERS)
    if schedule == "to_target":
        temps = dict(T_start_abs=TTT_T_START, T_end_abs=TTT_T_END, move_scale=TTT_D_FACTOR / N_OMEGA)
    else:
        temps = dict(T_start=10.0, T_end=1e-9)
    prm = sail.Params(n_walkers=N_WALKERS, precision=sail.PREC_FP32, n_sweeps=N_SWEEPS,
                      sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=resync_every, branching=True,
                      A=P.A, B=P.B, seed=seed, timing=timing,
                      resync_kind=resync_kind, sweep_lanes=sweep_lanes, index_walk_len=index_walk,
                      shared_bins=shared_bins, sweep_loop=sweep_loop, fp64_accept=fp64_accept, **temps)
    return P, prm


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, gpu_index: int):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != gpu_index:
                    continue
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- ranks
def aggregate(ms: float, moves: float, dist=None, device="cpu"):
    """Whole-job figures over the ranks: the slowest rank's time, the sum of every rank's
    walker-moves, and their ratio (walker-moves per second)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    m = torch.tensor([moves], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
    ms_max, total = float(t.item()), float(m.item())
    return ms_max, total, total / (ms_max * 1e-3)


# ---------------------------------------------------------------- GPU arm
def measure_read_bandwidth(torch, sail, nbytes: int, reps: int) -> float:
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    buf.fill_(1)
    st = torch.cuda.current_stream()
    sail._capi.read_bandwidth_probe(buf, 1, st)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(3):
        e0.record(st)
        sail._capi.read_bandwidth_probe(buf, reps, st)
        e1.record(st)
        st.synchronize()
        best = max(best, nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del buf
    return best


def measure_smem_bandwidth(torch, sail, reps: int) -> float:
    st = torch.cuda.current_stream()
    sail._capi.smem_bandwidth_probe(64, st)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(3):
        e0.record(st)
        nbytes = sail._capi.smem_bandwidth_probe(reps, st)
        e1.record(st)
        st.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def kernel_traffic():
    """DRAM traffic per sweep launch from the committed ncu summary, if the kernel source
    is unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "sweep_fp32_paper_scale.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        csrc = os.path.join(ROOT, "paper_1609_07936_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("sweep_group.cuh", "sweep_fp32.cu"))
        if hashlib.sha256(src).hexdigest() != rec.get("source_sha256"):
            return None
        return rec.get("dram_bytes_per_launch")
    except Exception:
        return None


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_1609_07936_gb300 as sail
    torch.cuda.set_device(local_rank)
    sail.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier(device_ids=[local_rank])
        torch.cuda.synchronize()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # roofline denominators: shared-memory read bandwidth (the sweep's kernel tables live
    # there) and, for reference, the read bandwidth of an L2-resident buffer (32 MiB, x400)
    smem_gbs = measure_smem_bandwidth(torch, sail, 20000)
    l2_gbs = measure_read_bandwidth(torch, sail, 32 << 20, 400)

    # warm-up: W blocks on a separate handle (same configuration, other seed)
    P, prm = params_for(seed=1000 + rank, resync_every=args.resync_every, resync_kind=args.resync_kind,
                        sweep_lanes=args.sweep_lanes, index_walk=args.index_walk,
                        shared_bins=args.shared_bins, sweep_loop=args.sweep_loop, schedule=args.schedule,
                        fp64_accept=args.fp64_accept)
    warm = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    warm.anneal(args.warmup)
    warm.close()
    del warm

    P, prm = params_for(seed=rank, resync_every=args.resync_every, resync_kind=args.resync_kind,
                        sweep_lanes=args.sweep_lanes, index_walk=args.index_walk,
                        shared_bins=args.shared_bins, sweep_loop=args.sweep_loop, schedule=args.schedule,
                        fp64_accept=args.fp64_accept)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    st = g.stream
    info0 = g.info()
    clocks = Clocks(os.path.join(args.clocks_dir, f"clocks_rank{rank}.csv") if args.clocks_dir
                    else f"/tmp/sail_clocks_{os.getpid()}_{rank}.csv")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clocks:
        time.sleep(0.3)
        barrier()
        e0.record(st)
        stats = []
        for k in range(args.steps):
            stats += g.anneal(1)
            flush.zero_()       # L2 flushed between steps (256 MiB write on the same stream)
        e1.record(st)
        barrier()
    ms = e0.elapsed_time(e1)
    info1 = g.info()
    ms_max, moves, value = aggregate(ms, info1["moves"] - info0["moves"], dist, "cuda")
    sweep_ms = info1["sweep_ms"] - info0["sweep_ms"]
    sweep_n = info1["sweep_launches"] - info0["sweep_launches"]
    launches = info1["kernel_launches"] - info0["kernel_launches"] + args.steps  # + one flush per step
    own_launches = info1["kernel_launches"] - info0["kernel_launches"]
    moves_per_launch = (info1["moves"] - info0["moves"]) / max(sweep_n, 1)
    # algorithmic bytes of a walker-move (Sec. 2.2: the update needs the two kernel columns of
    # the proposed bins and nothing else of size N_tau): b_p and b_s read and, on acceptance,
    # written (16 B); then, unless the move fails the positivity test (checked before delta
    # chi2), the columns Khat_p and Khat_s in FP32 (2 N_tau 4 B)
    col_bytes = 2 * N_TAU * 4
    pos_frac = sum(b["positivity_rejected"] for b in stats) / max(len(stats), 1)
    bytes_per_move = 16 + (1.0 - pos_frac) * col_bytes
    bytes_rule = f"16 + (1 - positivity-rejected fraction {pos_frac:.4f}) x 2 x {N_TAU} x 4"
    if args.shared_bins:
        # shared bins: a group of W walkers reads one move's columns once
        bytes_per_move = 16 + col_bytes / args.shared_bins
        bytes_rule = f"16 + 2 x {N_TAU} x 4 / {args.shared_bins} (columns read once per group of {args.shared_bins} walkers)"

    launch_s = sweep_ms / max(sweep_n, 1) * 1e-3
    achieved = moves_per_launch * bytes_per_move / launch_s / 1e9
    clk = clocks.summary(local_rank)
    # the sweep is bound by FP32 arithmetic issue and its latency (not HBM, no contraction):
    # algorithmic FP32 work of a walker-move (Sec. 2.2), per tau point: for a move that passes
    # the positivity test d_i = eps M_i - delta_p Khat_ip - delta_s Khat_is (1 multiply + 2 FMA =
    # 5 flops) and d_i (2 R_i + d_i) accumulated (2 FMA = 4 flops); for an accepted move
    # R_i += d_i, M_i -= d_i (2 flops).  Peak: SMs x 128 FP32 lanes x 2 flops (FMA) x the
    # maximum SM clock.
    acc_frac = sum(b["acceptance"] for b in stats) / max(len(stats), 1)
    flops_per_move = N_TAU * (9.0 * (1.0 - pos_frac) + 2.0 * acc_frac)
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    sm_max_mhz = clk.get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12
    fp32_achieved = moves_per_launch * flops_per_move / launch_s / 1e12

    # end to end through the public API from host buffers: create (H2D of inputs and tables),
    # K blocks (per-block statistics D2H), average (D2H of the spectrum and errors)
    e2e = None
    if not args.no_e2e:
        P2, prm2 = params_for(seed=rank + 77, timing=False, resync_kind=args.resync_kind,
                              sweep_lanes=args.sweep_lanes, index_walk=args.index_walk,
                              shared_bins=args.shared_bins, sweep_loop=args.sweep_loop, schedule=args.schedule,
                        fp64_accept=args.fp64_accept)
        barrier()
        t0 = time.perf_counter()
        h = sail.Sail(P2.tau, P2.F, P2.sigma, P2.omega, prm2)
        for k in range(args.steps):
            h.anneal(1)
        mean, err, used, c2 = h.average()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_t = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(t_t, op=dist.ReduceOp.MAX)
        pad = (N_TAU + 31) // 32 * 32
        # what sail_create copies: both kernel tables, Fhat (FP64 + FP32), centres, beta,
        # the temperature table, the start spectrum and residual
        h2d = N_OMEGA * pad * 12 + pad * 12 + N_OMEGA * 12 + N_SWEEPS * 8 + N_OMEGA * 8 + pad * 8
        # per block: counters (32 B), Delta (8 B), imprint count (4 B); at the end the mean
        # and error spectra, the count used and chi2 of the mean
        d2h = args.steps * (32 + 8 + 4) + 2 * N_OMEGA * 8 + 4 + 8
        e2e = {"value": args.steps * MOVES_PER_STEP * world / float(t_t.item()), "unit": METRIC,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "wall_s": float(t_t.item()), "chi2_of_mean": c2, "walkers_averaged": used}
        h.close()

    # the other two noise levels of the workload (sigma = 1e-3 F and 1e-5 F): the same timed
    # steps on their own handles, walker-moves/s from CUDA events on the handle's stream
    noise_levels = []
    if not args.no_noise_levels:
        for lvl in (1e-3, 1e-5):
            P3, prm3 = params_for(seed=rank + 500, resync_kind=args.resync_kind, sweep_lanes=args.sweep_lanes,
                                  index_walk=args.index_walk, shared_bins=args.shared_bins,
                                  sweep_loop=args.sweep_loop, noise=lvl, schedule=args.schedule,
                                  fp64_accept=args.fp64_accept)
            h3 = sail.Sail(P3.tau, P3.F, P3.sigma, P3.omega, prm3)
            h3.anneal(args.warmup)
            m0 = h3.info()["moves"]
            barrier()
            e0.record(h3.stream)
            for k in range(args.steps):
                h3.anneal(1)
                flush.zero_()
            e1.record(h3.stream)
            barrier()
            ms3, moves3, value3 = aggregate(e0.elapsed_time(e1), h3.info()["moves"] - m0, dist, "cuda")
            noise_levels.append({"sigma": f"{lvl:g} F", "value": value3, "unit": "walker-moves/s",
                                 "ms_per_step": ms3 / args.steps})
            h3.close()

    # inversions/s to target chi2 (p50 / p99), mixed precision against the plain FP64
    # recomputation of the residual (the same served FP32 sweep; only the recomputation differs)
    ttt = None
    if not args.no_to_target:
        ttt = to_target(sail, torch, args.ttt_inversions, args.resync_kind, seed0=100 * rank,
                        fp64_accept=args.fp64_accept)
        ttt64 = to_target(sail, torch, args.ttt_inversions, 3, seed0=100 * rank)
        ttt["vs_plain_fp64_resync"] = {
            "fp64_resync": ttt64,
            "inversions_per_s_ratio": (ttt["inversions_per_s"] / ttt64["inversions_per_s"]
                                       if ttt64["inversions_per_s"] > 0 else None),
            "equal_final_chi2": "both legs stop at the same target chi2 (or the same sweep budget)"}

    # the uneven batch (256 inversions sharing launches) as an extra field of the same line
    batch = None
    if not args.no_batch:
        batch = batch_leg(sail, torch, args.batch_size, 1, 2, args.resync_kind)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_walkers)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "walker-moves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (WORKLOAD_TO_TARGET if args.schedule == "to_target" else WORKLOAD)
                       + (f", index walk of {args.index_walk} steps" if args.index_walk else "")
                       + (f", bins shared by groups of {args.shared_bins} walkers" if args.shared_bins else ""), "step": f"one block: {SWEEPS_PER_BLOCK} sweeps x {N_OMEGA} moves x "
                       f"{N_WALKERS} walkers + 2 resyncs + branching", "walkers_per_gpu": N_WALKERS,
                       "l2": "flushed between steps (256 MiB write)", "parallelism": f"{world} independent inversions"},
            "roofline": {"kernel": "sweep_shared" if args.shared_bins else "sweep_fp32", "bound": "smem",
                         "achieved": achieved, "peak": smem_gbs, "unit": "GB/s", "frac": achieved / smem_gbs,
                         "traffic": None if (args.shared_bins or args.index_walk) else kernel_traffic(),
                         "traffic_note": "DRAM bytes per sweep launch (ncu); the sweep's operands live in shared memory",
                         "peak_source": "measured live in this run (not in MEASURED_PEAKS.json, which has HBM and bf16 only): "
                                        "conflict-free 16-byte shared-memory loads, 2 blocks x 1024 threads per SM",
                         "algorithmic_bytes_per_move": bytes_per_move, "bytes_per_move_rule": bytes_rule,
                         "moves_per_launch": moves_per_launch, "launch_ms": sweep_ms / max(sweep_n, 1),
                         "achieved_rule": "moves_per_launch x algorithmic_bytes_per_move / launch_ms (CUDA events "
                                          "around every sweep launch on the handle's stream)",
                         "alu": {"bound": "alu", "achieved": fp32_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                                 "frac": fp32_achieved / fp32_peak,
                                 "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x {sm_max_mhz:.0f} MHz",
                                 "algorithmic_flops_per_move": flops_per_move,
                                 "flops_per_move_rule": f"{N_TAU} x (9 x (1 - positivity-rejected {pos_frac:.4f}) "
                                                        f"+ 2 x accepted {acc_frac:.4f})"},
                         "l2_read_gbs_measured": l2_gbs,
                         "sweep_lanes_per_walker": g.info().get("sweep_lanes"),
                         "sweep_share_of_step": sweep_ms / ms},
            "kernel_ms": {"sweep": sweep_ms, "resync": info1["resync_ms"] - info0["resync_ms"],
                          "branch": info1["branch_ms"] - info0["branch_ms"], "total": ms},
            "e2e": e2e, "gpu_launches": own_launches, "clocks": clk, "cpu_baseline": cpu,
            "other_noise_levels": noise_levels, "to_target": ttt, "uneven_batch": batch,
            "last_block": stats[-1] if stats else None,
        }
        if args.fp64_accept:
            out["fp64_accept"] = {"mode": args.fp64_accept,
                                  "rechecks": info1["fp64_rechecks"] - info0["fp64_rechecks"],
                                  "flips": info1["fp64_flips"] - info0["fp64_flips"],
                                  "rechecks_per_move": (info1["fp64_rechecks"] - info0["fp64_rechecks"]) /
                                                       max(info1["moves"] - info0["moves"], 1)}
        print(json.dumps(out), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()


def to_target(sail, torch, n_inv: int, resync_kind: int, noise: float = NOISE, seed0: int = 0, fp64_accept: int = 0):
    """n_inv inversions of the workload (4096 walkers each, seeds seed0..), one after another
    through the public API, each from its host arrays to its averaged spectrum on the host and
    stopped at chi2 of the averaged spectrum <= 1.2 N_tau (checked at every block end) or at
    20000 sweeps.  Time to target is each inversion's own wall time; inversions/s counts the
    converged ones over the total wall time."""
    P = paper_scale_double_lorentz(noise, n_walkers=N_WALKERS)
    res = []
    torch.cuda.synchronize()
    t_all = time.perf_counter()
    for k in range(n_inv):
        prm = sail.Params(n_walkers=N_WALKERS, precision=sail.PREC_FP32, n_sweeps=TTT_SWEEPS,
                          sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY, branching=True,
                          T_start_abs=TTT_T_START, T_end_abs=TTT_T_END, move_scale=TTT_D_FACTOR / N_OMEGA,
                          A=P.A, B=P.B, seed=seed0 + k, target_chi2=TTT_TARGET * N_TAU, resync_kind=resync_kind,
                          fp64_accept=fp64_accept)
        t0 = time.perf_counter()
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        g.anneal()
        mean, err, used, c2 = g.average()
        dt = time.perf_counter() - t0
        inf = g.info()
        res.append({"converged": bool(c2 <= TTT_TARGET * N_TAU), "sweeps": inf["sweeps_done"], "chi2_of_mean": c2,
                    "time_s": dt, "fp64_rechecks": inf["fp64_rechecks"], "fp64_flips": inf["fp64_flips"]})
        g.close()
    wall = time.perf_counter() - t_all
    t = np.array([x["time_s"] for x in res])
    conv = np.array([x["converged"] for x in res])
    moves = sum(x["sweeps"] for x in res) * N_OMEGA * N_WALKERS
    pct = lambda q: float(np.percentile(t[conv], q)) if conv.any() else None
    return {"inversions": n_inv, "target": f"chi2 of the averaged spectrum <= {TTT_TARGET} N_tau = {TTT_TARGET * N_TAU:g}",
            "converged_fraction": float(conv.mean()), "time_to_target_p50_s": pct(50), "time_to_target_p99_s": pct(99),
            "inversions_per_s": float(conv.sum()) / wall, "wall_s": wall, "walker_moves_per_s": moves / wall,
            "sweeps_to_target": [x["sweeps"] for x in res], "final_chi2": [x["chi2_of_mean"] for x in res],
            "times_s": t.tolist(),
            "schedule": f"geometric T {TTT_T_START:g} -> {TTT_T_END:g} (absolute) over {TTT_SWEEPS} sweeps, "
                        f"move scale {TTT_D_FACTOR:g} / N_omega, branching every {SWEEPS_PER_BLOCK} sweeps",
            "resync": {0: "fp32-fma", 1: "tensor-tf32x3", 2: "tensor-bf16x6", 3: "fp64-fma"}[resync_kind],
            **({"fp64_accept": {"mode": fp64_accept, "rechecks": sum(x["fp64_rechecks"] for x in res),
                                "flips": sum(x["fp64_flips"] for x in res),
                                "rechecks_per_move": sum(x["fp64_rechecks"] for x in res) / max(moves, 1)}}
               if fp64_accept else {})}


# ---------------------------------------------------------------- CPU oracle
def cpu_baseline(n_walkers: int):
    """The FP64 oracle on a bounded sample of the same workload: n_walkers walkers for one
    block (100 sweeps, two residual recomputations, one branching), all host cores."""
    import oracle as O
    P = paper_scale_double_lorentz(NOISE, n_walkers=n_walkers)
    sched = O.Schedule(n_sweeps=N_SWEEPS, sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY,
                       branching=True, T_start=10.0, T_end=1e-9, seed=0)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers, sched)
    t0 = time.perf_counter()
    an.run(SWEEPS_PER_BLOCK)
    dt = time.perf_counter() - t0
    moves = SWEEPS_PER_BLOCK * N_OMEGA * n_walkers
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": moves / dt, "unit": "walker-moves/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_walkers} walkers x {SWEEPS_PER_BLOCK} sweeps (one block with 2 resyncs and a "
                      f"branching) of the paper-scale workload, {moves:.3g} moves in {dt:.1f} s"}


# ---------------------------------------------------------------- uneven batch and serving
def batch_leg(sail, torch, batch_size: int, steps: int, warmup: int, resync_kind: int) -> dict:
    """256 independent inversions (n_tau U{50..500}, n_omega U{200..2000}, walkers U{256..4096},
    noise log-uniform [1e-5, 1e-3], 1-4 random peaks) annealed together: one persistent sweep
    launch per class of problems and segment, tensor-core resync, branching every 100 sweeps,
    autotuned mapping.  walker-moves/s over `steps` blocks of every inversion (CUDA events on the
    batch's stream) after `warmup` blocks (which include the autotuner's trials)."""
    from workloads import random_batch_problem
    probs = [random_batch_problem(i, seed=0) for i in range(batch_size)]
    items = []
    for i, P in enumerate(probs):
        prm = sail.Params(n_walkers=P.n_walkers, precision=sail.PREC_FP32, n_sweeps=N_SWEEPS,
                          sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY, branching=True,
                          T_start=10.0, T_end=1e-9, A=P.A, B=P.B, seed=i, resync_kind=resync_kind)
        items.append((P.tau, P.F, P.sigma, P.omega, prm))
    t0 = time.perf_counter()
    batch = sail.Batch(items, autotune=True)
    t_create = time.perf_counter() - t0
    batch.anneal(warmup)
    moves0 = sum(h.info()["moves"] for h in batch.handles)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = batch.stream
    e0.record(st)
    batch.anneal(steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    moves = sum(h.info()["moves"] for h in batch.handles) - moves0
    per_inv = float(np.mean([N_SWEEPS * P.n_walkers * P.n_omega for P in probs]))
    value = moves / (ms * 1e-3)
    out = {"value": value, "unit": "walker-moves/s", "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
           "workload": f"uneven batch: {len(probs)} inversions, n_tau U{{50..500}}, n_omega U{{200..2000}}, "
                       f"walkers U{{256..4096}} (total {sum(P.n_walkers for P in probs)}), noise log-U[1e-5,1e-3], "
                       f"one persistent sweep launch per class and {RESYNC_EVERY}-sweep segment",
           "step": f"one block ({SWEEPS_PER_BLOCK} sweeps) of every inversion",
           "inversions_per_s": value / per_inv, "moves_per_inversion": per_inv,
           "tuning": batch.tuning(), "create_s": t_create}
    batch.close()
    return out


def run_batch(args):
    """The uneven batch as its own benchmark line (see batch_leg)."""
    import torch
    import paper_1609_07936_gb300 as sail
    sail.load()
    b = batch_leg(sail, torch, args.batch_size, args.steps, args.warmup, args.resync_kind)
    out = {"metric": METRIC, "value": b["value"], "unit": "walker-moves/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": b["workload"], "step": b["step"]},
           "inversions_per_s": b["inversions_per_s"], "moves_per_inversion": b["moves_per_inversion"],
           "tuning": b["tuning"], "create_s": b["create_s"]}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Poisson arrivals of inversion requests (sizes as the uneven batch), each run until the
    averaged spectrum reaches chi2 <= 1.2 n_tau or its sweep budget ends, on the to-target
    schedule; continuous batching on one device buffer (admission cap) driven by the server's
    worker thread while this thread submits requests at their arrival times and polls for
    completions.  Latency and time to target come from the server's own clock (submission of
    the host arrays to the averaged spectrum on the host)."""
    import torch
    import paper_1609_07936_gb300 as sail
    from workloads import random_batch_problem
    sail.load()
    rng = np.random.default_rng(12345)
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / args.rate)
        if t > args.duration:
            break
        arrivals.append(t)
    free, _ = torch.cuda.mem_get_info()
    cap = int(min(150e9, free - (4 << 30)))
    server = sail.Server(workspace_bytes=cap, max_resident=args.max_resident, max_walkers=1 << 22,
                         sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY)
    probs, rids = {}, []
    server.start()
    t_start = time.perf_counter()
    queue_trace = []
    done = set()
    nxt = 0
    while nxt < len(arrivals) or len(done) < len(arrivals):
        now = time.perf_counter() - t_start
        if args.drain is not None and nxt >= len(arrivals) and now > args.duration + args.drain:
            break                       # bounded run: stop serving the drain budget after the arrivals
        while nxt < len(arrivals) and arrivals[nxt] <= now:
            P = random_batch_problem(nxt, seed=99, max_tau=args.max_tau, max_omega=args.max_omega,
                                     max_walkers=args.max_walkers)
            prm = sail.Params(n_walkers=P.n_walkers, precision=sail.PREC_FP32, n_sweeps=args.serve_sweeps,
                              sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY, branching=True,
                              T_start_abs=TTT_T_START, T_end_abs=TTT_T_END, move_scale=TTT_D_FACTOR / P.n_omega,
                              A=P.A, B=P.B, seed=nxt, target_chi2=TTT_TARGET * P.n_tau, resync_kind=args.resync_kind)
            rid = server.submit(P.tau, P.F, P.sigma, P.omega, prm)
            probs[rid] = P
            rids.append(rid)
            nxt += 1
        completed, active, queued = server.poll()
        done.update(completed)
        if not queue_trace or now - queue_trace[-1][0] >= 1.0:
            queue_trace.append((round(now, 1), active, queued, len(done)))
        time.sleep(0.005)
    server.stop()                       # the worker finishes the step it is in
    wall = time.perf_counter() - t_start
    all_infos = [server.request_info(r) for r in rids]
    # walker-moves of every request, finished or not (the device's throughput under the load)
    moves = sum(i["sweeps"] * probs[r].n_walkers * probs[r].n_omega for r, i in zip(rids, all_infos))
    n_admitted = sum(1 for i in all_infos if i["t_admit"] >= 0)
    n_unfinished = sum(1 for i in all_infos if i["state"] in (0, 1))
    infos = [i for i in all_infos if i["state"] == 2]            # latency statistics: completed requests
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos], dtype=float)
    wait = np.array([i["t_admit"] - i["t_submit"] for i in infos], dtype=float)
    conv = np.array([bool(i["converged"]) for i in infos], dtype=bool)
    sweeps = np.array([i["sweeps"] for i in infos], dtype=float)
    ttt = lat[conv]
    pct = lambda x, q: float(np.percentile(x, q)) if x.size else None   # null when none converged
    out = {"metric": "inversions/s (served)", "value": len(done) / wall, "unit": "inversions/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"served: Poisson arrivals {args.rate}/s for {args.duration} s ({len(arrivals)} requests), "
                                  f"sizes as the uneven batch (n_tau U{{50..{args.max_tau}}}, n_omega U{{200..{args.max_omega}}}, "
                                  f"walkers U{{256..{args.max_walkers}}}), target chi2 <= {TTT_TARGET} n_tau, budget "
                                  f"{args.serve_sweeps} sweeps, T {TTT_T_START:g} -> {TTT_T_END:g} absolute, move scale "
                                  f"{TTT_D_FACTOR:g} / n_omega, admission cap {cap / 1e9:.0f} GB, at most "
                                  f"{args.max_resident} resident",
                      "resync": {0: "fp32-fma", 1: "tensor-tf32x3", 2: "tensor-bf16x6", 3: "fp64-fma"}[args.resync_kind]},
           "wall_s": wall, "walker_moves_per_s": moves / wall,
           "submitted": len(rids), "admitted": n_admitted, "completed": len(infos),
           "unfinished_at_stop": n_unfinished,
           "stop": ("all requests completed" if args.drain is None or not n_unfinished else
                    f"{args.drain:g} s after the last arrival; latency statistics over the completed requests"),
           "latency_p50_s": pct(lat, 50), "latency_p99_s": pct(lat, 99),
           "admission_wait_p50_s": pct(wait, 50), "admission_wait_p99_s": pct(wait, 99),
           "converged_fraction": float(conv.mean()) if conv.size else None,
           "converged_per_s": float(conv.sum()) / wall,
           "time_to_target_p50_s": pct(ttt, 50), "time_to_target_p99_s": pct(ttt, 99),
           "sweeps_to_target_p50": pct(sweeps[conv], 50),
           "queue_trace": {"columns": ["t_s", "resident", "queued", "completed"], "rows": queue_trace[::max(1, len(queue_trace) // 40)]}}
    print(json.dumps(out), flush=True)
    server.close()


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, --warmup untimed and --steps timed
    steps, each step one block (100 sweeps, two residual recomputations, one branching) of the
    paper-scale workload on a walker sample sized from a one-block calibration run so that the
    whole run takes about --ref-seconds.  Under a multi-rank launch rank 0 alone runs it."""
    if rank != 0:
        return
    import oracle as O
    sched = O.Schedule(n_sweeps=N_SWEEPS, sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY,
                       branching=True, T_start=10.0, T_end=1e-9, seed=0)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cal_w = max(8, cores)
    P = paper_scale_double_lorentz(NOISE, n_walkers=cal_w)
    cal = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, cal_w, sched)
    t0 = time.perf_counter()
    cal.run(SWEEPS_PER_BLOCK)
    t_block = time.perf_counter() - t0               # one block of cal_w walkers
    blocks = args.steps + args.warmup
    fit = int(args.ref_seconds / max(blocks * t_block, 1e-9) * cal_w)
    n_w = max(cal_w, min(args.cpu_sample_walkers, fit // cal_w * cal_w))
    P = paper_scale_double_lorentz(NOISE, n_walkers=n_w)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_w, sched)
    for _ in range(args.warmup):
        an.run(SWEEPS_PER_BLOCK)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        an.run(SWEEPS_PER_BLOCK)
    dt = time.perf_counter() - t0
    moves = args.steps * SWEEPS_PER_BLOCK * N_OMEGA * n_w
    value = moves / dt
    cpu = {"value": value, "unit": "walker-moves/s", "cores": cores, "kind": "oracle",
           "sample": f"{n_w} of the {N_WALKERS} walkers, {args.warmup} untimed + {args.steps} timed blocks of "
                     f"{SWEEPS_PER_BLOCK} sweeps (2 resyncs and a branching each), {moves:.3g} moves in {dt:.1f} s"}
    out = {"metric": METRIC, "value": value, "unit": "walker-moves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "ms_per_step_scaled": {"value": MOVES_PER_STEP / value * 1e3,
                                  "rule": f"one block of all {N_WALKERS} walkers at the sample's walker-moves/s "
                                          "(extrapolated, not run)"},
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "parallelism": "CPU oracle, OpenMP over walkers",
                      "step": f"one block (100 sweeps, 2 resyncs, a branching) of a {n_w}-walker sample "
                              f"of the {N_WALKERS} walkers"},
           "cpu_baseline": cpu,
           "e2e": {"value": value, "unit": "walker-moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_precision(args):
    """The precision configuration: 512 tau x 2048 bins, 16384 walkers, a 1-4 peak random
    spectrum, FP32 moves.  For each residual recomputation (FP32-FMA GEMM, tcgen05 TF32 x3,
    tcgen05 BF16 x6 fed by tensor copies, FP64-FMA): two blocks of 50 sweeps with a
    recomputation every 10, its time per call from CUDA events, and the error of the residual
    it leaves against the FP64 validation path's sequential recomputation from the same spectra
    on 256 sampled walkers (relative to the model value sum_j K_ij a_j).  Then the error of a
    result: 256 walkers of the same problem annealed with the same seed by the FP64 validation
    path (the oracle's arithmetic) and by the mixed-precision path (FP32 moves, BF16 x6
    recomputation), their averaged spectra and chi2 of the averages compared, beside the same
    comparison between two seeds of the mixed path (the method's own spread)."""
    import torch
    import paper_1609_07936_gb300 as sail
    from workloads import precision_random_peaks
    sail.load()
    P = precision_random_peaks(0)
    Fh = P.F / P.sigma
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(P.n_walkers, 256, replace=False))
    ref = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                    sail.Params(n_walkers=sample.size, precision=sail.PREC_FP64, n_sweeps=10, A=P.A, B=P.B))
    kinds, moves, sweep_ms = [], 0.0, 0.0
    names = {0: "fp32-fma", 1: "tcgen05-tf32x3", 2: "tcgen05-bf16x6", 3: "fp64-fma"}
    for kind in [int(k) for k in args.resync_kinds.split(",")]:
        name = names[kind]
        prm = sail.Params(n_walkers=P.n_walkers, precision=sail.PREC_FP32, n_sweeps=100, sweeps_per_block=50,
                          resync_every=10, branching=False, T_start=10.0, T_end=1e-3, A=P.A, B=P.B, seed=3,
                          resync_kind=kind, timing=True, shared_bins=args.shared_bins)
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        g.anneal()
        torch.cuda.synchronize()
        inf = g.info()
        a, R, chi2, _, _ = g.state()
        ref.set_state(a[sample])
        R64 = ref.state()[1]
        model = Fh[None, :] - R64
        err = np.abs(R[sample] - R64)
        rel = err / np.maximum(model, 1e-300)
        kinds.append({"resync": name, "ms_per_call": inf["resync_ms"] / max(inf["resync_launches"], 1),
                      "max_err_rel_model": float(rel.max()), "rms_err_rel_model": float(np.sqrt(np.mean(rel ** 2))),
                      "max_err_over_sigma": float(err.max())})
        moves += inf["moves"]
        sweep_ms += inf["sweep_ms"]
        g.close()
    ref.close()
    flop = 2.0 * P.n_walkers * P.n_omega * P.n_tau
    for k in kinds:
        k["useful_tflops"] = flop / (k["ms_per_call"] * 1e-3) / 1e12

    result_error = None
    if not args.no_result_error:
        W = 256
        sched = dict(n_walkers=W, n_sweeps=args.result_sweeps, sweeps_per_block=SWEEPS_PER_BLOCK,
                     resync_every=RESYNC_EVERY, branching=True, T_start_abs=TTT_T_START, T_end_abs=TTT_T_END,
                     move_scale=TTT_D_FACTOR / P.n_omega, A=P.A, B=P.B)
        runs = {}
        for tag, precision, seed in (("fp64", sail.PREC_FP64, 5), ("mixed", sail.PREC_FP32, 5),
                                     ("mixed_other_seed", sail.PREC_FP32, 6)):
            h = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                          sail.Params(precision=precision, seed=seed, resync_kind=RESYNC_KIND, **sched))
            h.anneal()
            mean, err_, used, c2 = h.average()
            runs[tag] = (mean, c2)
            h.close()
        l2 = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
        result_error = {
            "walkers": W, "sweeps": args.result_sweeps,
            "schedule": f"geometric T {TTT_T_START:g} -> {TTT_T_END:g} absolute, branching every {SWEEPS_PER_BLOCK}",
            "spectrum_rel_l2_mixed_vs_fp64": l2(runs["mixed"][0], runs["fp64"][0]),
            "spectrum_rel_l2_mixed_seed_vs_seed": l2(runs["mixed_other_seed"][0], runs["mixed"][0]),
            "chi2_of_mean": {k: v[1] for k, v in runs.items()},
            "reading": "same seed: the FP64 path takes the oracle's decisions; the mixed path parts from it as "
                       "FP32 rounding flips decisions, so its distance to the FP64 result is compared with the "
                       "distance between two seeds of the mixed path"}
    out = {"metric": METRIC, "value": moves / (sweep_ms * 1e-3), "unit": "walker-moves/s", "n_gpus": 1,
           "steps": 3, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "precision: 512 tau x 2048 bins, 16384 walkers, random 1-4 peaks, FP32 moves, "
                                  "residual recomputation every 10 sweeps by each method"
                                  + (f", bins shared by groups of {args.shared_bins} walkers" if args.shared_bins else ""),
                      "step": "two blocks of 50 sweeps per recomputation method"},
           "resync": kinds, "result_error": result_error}
    print(json.dumps(out), flush=True)


def run_versus_fp64(args):
    """Served mixed precision against the plain FP64 path at equal final chi2.  A closed set of
    requests, sizes as the uneven batch with the ranges' upper ends lowered (n_tau U{50..200},
    n_omega U{200..800}, walkers U{256..1024}) so that the FP64 path finishes in seconds, all
    with the served schedule (T 1e-2 chi2_0 -> 0.3 absolute over --cmp-sweeps sweeps, branching
    every 100, recomputation every 50), is inverted three ways:
      fp64:        the plain FP64 path, one handle after another: FP64 spectra and moves, sums
                   in the oracle's order, FP64 residual recomputation;
      mixed:       FP32 moves with the tcgen05 BF16 x6 recomputation and FP64 residuals, one
                   handle after another, each stopping at the first block end where chi2 of
                   its averaged spectrum is at or below what the FP64 path ended with (else at
                   the end of the same schedule);
      mixed_served: the same as mixed, all requests submitted to one server at once
                   (continuous batching: they share persistent sweep launches);
      mixed_reseeded: mixed with other seeds and no target, the yardstick for "equal": how far
                   two runs of the same precision land apart.
    Each leg's wall time covers create (host arrays in), the anneal and the averaged spectrum
    back on the host.  Reports inversions/s of each leg and, per request, the final chi2 of the
    averaged spectrum of each leg."""
    import torch
    import paper_1609_07936_gb300 as sail
    from workloads import random_batch_problem
    sail.load()
    probs = [random_batch_problem(i, seed=77, max_tau=200, max_omega=800, max_walkers=1024)
             for i in range(args.cmp_requests)]

    def prm(P, i, precision, target=0.0):
        return sail.Params(n_walkers=P.n_walkers, precision=precision, n_sweeps=args.cmp_sweeps,
                           sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY, branching=True,
                           T_start=1e-2, T_end_abs=0.3, A=P.A, B=P.B, seed=i, target_chi2=target,
                           resync_kind=RESYNC_KIND)

    # warm-up: module loading and first launches of both paths, outside the timed legs
    for precision in (sail.PREC_FP64, sail.PREC_FP32):
        P = probs[0]
        w = prm(P, 0, precision)
        w.n_sweeps = 2 * SWEEPS_PER_BLOCK
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega, w)
        g.anneal()
        g.average()
        g.close()
    torch.cuda.synchronize()

    def one_by_one(precision, targets, seed0=0):
        out = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, P in enumerate(probs):
            g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm(P, seed0 + i, precision, targets[i]))
            g.anneal()
            _, _, _, c2 = g.average()
            out.append((c2, g.info()["sweeps_done"]))
            g.close()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    wall64, res64 = one_by_one(sail.PREC_FP64, [0.0] * len(probs))
    targets = [c2 for c2, _ in res64]
    wall32, res32 = one_by_one(sail.PREC_FP32, targets)
    _, resr = one_by_one(sail.PREC_FP32, [0.0] * len(probs), seed0=1000)

    need = sum(sail.workspace_size(P.n_tau, P.n_omega, prm(P, i, sail.PREC_FP32)) for i, P in enumerate(probs))
    server = sail.Server(workspace_bytes=2 * need + (64 << 20), max_resident=len(probs), max_walkers=1 << 20,
                         sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rids = [server.submit(P.tau, P.F, P.sigma, P.omega, prm(P, i, sail.PREC_FP32, targets[i]))
            for i, P in enumerate(probs)]
    resv = {}
    while len(resv) < len(rids):
        completed, _, _ = server.step()
        for rid in completed:
            r = server.result(rid)
            resv[rid] = (r["chi2_of_mean"], r["sweeps"])
    torch.cuda.synchronize()
    walls = time.perf_counter() - t0
    server.close()
    ress = [resv[r] for r in rids]

    per = []
    for i, P in enumerate(probs):
        per.append({"n_tau": P.n_tau, "n_omega": P.n_omega, "walkers": P.n_walkers,
                    "chi2_fp64": res64[i][0], "chi2_mixed": res32[i][0], "chi2_mixed_served": ress[i][0],
                    "chi2_mixed_reseeded": resr[i][0],
                    "sweeps_fp64": res64[i][1], "sweeps_mixed": res32[i][1], "sweeps_mixed_served": ress[i][1]})
    r32 = np.array([p["chi2_mixed"] / p["chi2_fp64"] for p in per])
    rsv = np.array([p["chi2_mixed_served"] / p["chi2_fp64"] for p in per])
    rsd = np.array([p["chi2_mixed_reseeded"] / p["chi2_mixed"] for p in per])
    gm = lambda r: float(np.exp(np.mean(np.log(r))))
    n = len(probs)
    out = {"metric": "inversions/sec at equal final chi2", "value": n / walls, "unit": "inversions/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{n} requests, n_tau U{{50..200}} x n_omega U{{200..800}} x walkers U{{256..1024}}, "
                                  f"random 1-4 peaks, noise log-uniform [1e-5, 1e-3], {args.cmp_sweeps}-sweep schedule "
                                  "T 1e-2 chi2_0 -> 0.3 absolute, branching every 100 sweeps, recomputation every 50",
                      "target": "chi2 of the averaged spectrum <= the FP64 path's final value, or the schedule's end"},
           "inversions_per_s": {"fp64": n / wall64, "mixed": n / wall32, "mixed_served": n / walls},
           "wall_s": {"fp64": wall64, "mixed": wall32, "mixed_served": walls},
           "speedup_served_vs_fp64": wall64 / walls,
           "reached_fp64_chi2": {"mixed": float(np.mean(r32 <= 1.0)), "mixed_served": float(np.mean(rsv <= 1.0))},
           "chi2_ratio_to_fp64": {"mixed_geomean": gm(r32), "mixed_median": float(np.median(r32)),
                                  "mixed_min": float(r32.min()), "mixed_max": float(r32.max()),
                                  "served_geomean": gm(rsv), "served_max": float(rsv.max())},
           "chi2_ratio_reseeded_to_mixed": {"geomean": gm(rsd), "median": float(np.median(rsd)),
                                            "min": float(rsd.min()), "max": float(rsd.max())},
           "requests": per}
    print(json.dumps(out), flush=True)


def run_band(args):
    """The paper's example (Sec. lorentzian-model): the two-peak Lorentzian band on 1000 bins of
    [0, 3.5], 1500 walkers, exact data and correlated undersampling noise at relative levels
    1e-5, 1e-4 and 1e-2 (Sec. resampling), annealed with the paper's protocol (self-cooling,
    adaptive branching, smoothing 1e-2).  Reports, per level, the skew of the averaged spectrum
    about w = 1.5 (the paper: 0.004, 0.017, 0.05 for exact, 1e-5, 1e-4), chi2 of the average per
    tau point, the relative L2 error against the true bin masses and the maxima of the smoothed
    average."""
    import torch
    import paper_1609_07936_gb300 as sail
    from workloads import bin_masses, lorentzian_band, lorentzian_band_peaks, skew
    sail.load()
    results, moves, dev_ms = [], 0.0, 0.0
    for level in (0.0, 1e-5, 1e-4, 1e-2):
        P = lorentzian_band(level, seed=7)
        if args.band_schedule == "to_target":
            sched = dict(T_start_abs=TTT_T_START, T_end_abs=TTT_T_END, move_scale=TTT_D_FACTOR / P.n_omega,
                         smooth_s=args.band_smooth)
        else:
            sched = dict(schedule_kind=sail.SCHEDULE_SELF_COOLING, adaptive_branching=True, smooth_s=1e-2,
                         T_end_abs=0.3)
        prm = sail.Params(n_walkers=P.n_walkers, precision=sail.PREC_FP32, n_sweeps=args.band_sweeps,
                          sweeps_per_block=SWEEPS_PER_BLOCK, resync_every=RESYNC_EVERY, branching=True,
                          A=P.A, B=P.B, seed=11, resync_kind=args.resync_kind,
                          target_chi2=1.2 * P.n_tau, timing=True, sweep_loop=args.sweep_loop, **sched)
        t0 = time.perf_counter()
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        g.anneal()
        mean, err, used, c2 = g.average()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        inf = g.info()
        truth = bin_masses(lorentzian_band_peaks(), P.W, P.n_omega, P.extra["band"]) / P.d_omega
        # maxima of the average after a 0.0875-wide box filter (25 bins), above 20% of its peak
        sm = np.convolve(mean, np.ones(25) / 25.0, mode="same")
        maxima = [float(P.omega[j]) for j in range(1, P.n_omega - 1)
                  if sm[j] > sm[j - 1] and sm[j] >= sm[j + 1] and sm[j] > 0.2 * sm.max()]
        results.append({"noise": level, "skew": skew(mean, P.omega), "chi2_per_tau": c2 / P.n_tau,
                        "rel_l2_error": float(np.linalg.norm(mean - truth) / np.linalg.norm(truth)),
                        "maxima": maxima[:6], "sweeps": inf["sweeps_done"], "walkers_averaged": used,
                        "wall_s": wall, "sequences_equivalent": P.extra["sequences_equivalent"]})
        moves += inf["moves"]
        dev_ms += inf["sweep_ms"] + inf["resync_ms"] + inf["branch_ms"]
        g.close()
    out = {"metric": METRIC, "value": moves / (dev_ms * 1e-3), "unit": "walker-moves/s", "n_gpus": 1,
           "steps": len(results), "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Lorentzian band (HWHM 1 at 1 and 2, band [0.5, 2.5]), 1000 bins on [0, 3.5], "
                                  "160 tau points at 0.05, 1500 walkers, "
                                  + ("self-cooling + adaptive branching + smoothing 1e-2"
                                     if args.band_schedule == "protocol" else
                                     f"geometric T 1e6 -> 0.03, move scale 0.1/N_omega, smoothing {args.band_smooth:g}")
                                  + f", {args.band_sweeps} sweeps or chi2 <= 1.2 n_tau",
                      "step": "one inversion per noise level"},
           "band": results}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-walkers", type=int, default=1024,
                    help="CPU oracle: walkers of the sample (the reference arm: at most this many)")
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="reference arm: the walker sample is sized so the run takes about this long")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default="",
                    help="directory for the raw nvidia-smi clock samples of the timed region (default: /tmp)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-to-target", action="store_true", help="skip the time-to-target legs")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-batch leg")
    ap.add_argument("--schedule", default="paper", choices=["paper", "to_target"],
                    help="temperature schedule of the timed blocks: the paper's (T 10 -> 1e-9 chi2_0, move "
                         "scale 1/N_omega) or the to-target one (T 1e6 -> 0.03 absolute, 0.1/N_omega)")
    ap.add_argument("--ttt-inversions", type=int, default=TTT_INVERSIONS,
                    help="time to target: inversions of the workload submitted together")
    ap.add_argument("--no-noise-levels", action="store_true",
                    help="skip the timed steps at the workload's other noise levels (1e-3, 1e-5)")
    ap.add_argument("--workload", default="paper_scale", choices=["paper_scale", "batch", "serve", "band", "precision", "versus_fp64"])
    ap.add_argument("--band-sweeps", type=int, default=20000, help="band example: sweep budget per inversion")
    ap.add_argument("--band-schedule", default="protocol", choices=["protocol", "to_target"],
                    help="band example: the paper's protocol (self-cooling, adaptive branching, smoothing 1e-2, "
                         "to 0.3) or the geometric to-target schedule")
    ap.add_argument("--band-smooth", type=float, default=0.0,
                    help="band example with the to-target schedule: smoothing strength")
    ap.add_argument("--batch-size", type=int, default=256)
    ap.add_argument("--rate", type=float, default=2.0, help="serving: request arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--fp64-accept", type=int, default=0, choices=[0, 1, 2],
                    help="decisions near the acceptance threshold taken again in FP64 (1), or all (2)")
    ap.add_argument("--max-resident", type=int, default=1024,
                    help="serving: at most this many requests resident at once (the rest queue)")
    ap.add_argument("--drain", type=float, default=None,
                    help="serving: stop this many seconds after the last arrival (default: when all are done)")
    ap.add_argument("--serve-sweeps", type=int, default=20000, help="serving: sweep budget per request")
    ap.add_argument("--max-tau", type=int, default=500, help="serving: upper end of the n_tau range")
    ap.add_argument("--max-omega", type=int, default=2000, help="serving: upper end of the n_omega range")
    ap.add_argument("--max-walkers", type=int, default=4096, help="serving: upper end of the walker range")
    ap.add_argument("--cmp-requests", type=int, default=12, help="versus_fp64: requests in the closed set")
    ap.add_argument("--cmp-sweeps", type=int, default=400, help="versus_fp64: sweeps of the schedule")
    ap.add_argument("--resync-kind", type=int, default=RESYNC_KIND, choices=[0, 1, 2],
                    help="residual recomputation: 0 = FP32-FMA GEMM, 1 = tensor cores (tcgen05 TF32 x3), "
                         "2 = tensor cores (tcgen05 BF16 x6)")
    ap.add_argument("--index-walk", type=int, default=0, choices=range(8),
                    help="steps of the index walk choosing a move's bins (0: uniform bins, the paper's runs)")
    ap.add_argument("--sweep-loop", type=int, default=0, choices=[0, 1, 2],
                    help="FP32 move loop: 0 choose by walkers per SM, 1 one move at a time, 2 look-ahead")
    ap.add_argument("--shared-bins", type=int, default=0, choices=[0, 2, 4, 8],
                    help="walkers per group proposing the same bins (0: every walker its own, the paper's move)")
    ap.add_argument("--sweep-lanes", type=int, default=0, choices=[0, 8, 16],
                    help="GPU lanes per walker in the FP32 sweep (0: the library's choice)")
    ap.add_argument("--no-result-error", action="store_true",
                    help="precision workload: skip the mixed-vs-FP64 comparison of a result")
    ap.add_argument("--result-sweeps", type=int, default=1000,
                    help="precision workload: sweeps of the mixed-vs-FP64 result comparison")
    ap.add_argument("--resync-kinds", default="0,1,2",
                    help="precision workload: residual recomputations to run (0 FP32-FMA, 1 TF32 x3, 2 BF16 x6, 3 FP64)")
    ap.add_argument("--resync-every", type=int, default=RESYNC_EVERY,
                    help="sweeps per sweep-kernel launch; smaller values give short launches for profiling")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "band":
        run_band(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "versus_fp64":
        run_versus_fp64(args)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
