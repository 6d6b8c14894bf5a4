"""Throughput of batched PDBO GDA on GB300: restart-iterations/s on dense QUBO n=20,000.

Workload (the headline configuration): dense QUBO, n = 20,000, integer entries uniform in
[-100, 100] (diagonal = linear term), seed 0; B = 1,024 restarts; BF16 tcgen05 contraction with
FP32 accumulation and FP32 master iterates; evaluation (rounding + exact int64 objective +
argmin) every K = 50 iterations.  One step = K GDA iterations + one evaluation.

Reported (one JSON line on rank 0):
  value       restart-iterations/s with the instance resident in HBM (device events)
  e2e         the same metric through the public C ABI with host buffers: every step creates
              the problem from pinned host Q, c (H2D), runs K iterations and reads the best
              (x*, F*) back (D2H)
  roofline    the tcgen05 update kernel: 2 n^2 B flop per launch / its average launch time
              (CUDA events around each launch inside the timed region), against the measured
              burst BF16 peak (the kernel is timed in a region of well under a second); the
              fraction of the sustained peak beside it
  cpu_baseline the FP64 oracle on the host cores, on a bounded sample (restart subset)
  time_to_target  device seconds until the best objective reaches the FP64 oracle's best
  plain_fp32_form the plain FP32 CUDA-core form on the same instance: its throughput, and the best
              objectives of both forms after the same T iterations
  other_configs   the other benchmark configurations (N = 1 only): Max-Cut on an Erdos-Renyi
              graph (n = 2,000, B = 256), dense QUBO n = 5,000 (B = 256, BF16), Max-Cut on the
              100 x 100 torus and on a random 4-regular graph (n = 20,000; B = 512; E4M3 weights
              and the plain FP32 form), and 64 dense instances of uneven n in one grouped launch
              (B = 128): restart-iterations/s and a roofline each, with the bytes or flops it counts
``--impl reference`` times the oracle alone (the reference arm of this comparison).
Multi-GPU: ``--gpus N`` starts N ranks under torch.distributed.run (or runs as one of them when
launched so); every rank runs its own B restarts (different seeds) of the same instance, and
after every step (K iterations + one evaluation) the ranks exchange their best candidates (the
lexicographic minimum of (F, t, rank, restart) and the winner's bits); value = all ranks'
restart-iterations / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_VARS = 20000
RESTARTS = 1024
RESTARTS_DEFAULT = RESTARTS
K_EVAL = 50
METRIC = "GDA restart-iterations/s at n=20k dense QUBO"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes (read + write) per launch of the update kernel: dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of that launch on this workload; keyed by (tile
# width, n, restarts), with the capture it came from
MEASURED_TRAFFIC = {(512, 20000, 1024): (1.169179e9 + 0.180734e9,
                                         "ncu capture of one k_tc_pair<EPI_UPDATE> launch, n=20000, B=1024")}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return dict(FALLBACK_PEAKS), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------------
def oracle_sample(Q, c, p, seconds: float, restarts: int = 16, A=None, cp=None):
    """Time the FP64 oracle on `restarts` restarts of the workload for about `seconds`."""
    import oracle as O
    if A is None:
        A, cp = O.canonicalize(Q, c)
    X, _ = O.init_state(Q.shape[0], restarts, p.seed, p.ybar)
    Y = np.full_like(X, p.ybar)
    it = 0
    t0 = time.perf_counter()
    while True:
        X, Y, _ = O.gda_step(A, cp, X, Y, p.alpha, p.beta, p.delta, p.grad_tol)
        it += 1
        el = time.perf_counter() - t0
        if el >= seconds and it >= 2:
            break
    return restarts * it / el, it, el, A, cp


def oracle_threads():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


def load_target(key):
    path = os.path.join(ROOT, "tests", "golden", "oracle_targets.json")
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except OSError:
        return None


def time_to_target(S, torch, Q, c, seed, stream, dev, target, iters=2000, world=1):
    """One full solve (T iterations, K-blocks replayed from CUDA graphs): the time until the best
    objective first reaches the target.  One rank: device time, an event after every block.
    Several ranks (each its own restarts, seeded by rank): after every block the ranks exchange
    their best candidates (step_loop), and the time is the slowest rank's host clock at the first
    block whose global best reaches the target."""
    import torch.distributed as dist
    p = W.dense_params(Q, restarts=RESTARTS_DEFAULT, iters=iters, eval_every=K_EVAL, seed=seed)
    P = S.Problem.dense(Q, c, precision=S.SBO_BF16, stream=stream)
    P.start(S.params(**p.asdict()))
    blocks = iters // K_EVAL
    if world > 1:
        dist.barrier()
        t0 = time.perf_counter()
        stamps = []

        def block():
            P.run(K_EVAL)

        def best():
            out = P.best()                       # synchronises this rank's stream
            stamps.append(time.perf_counter() - t0)
            return out
        gtrace = step_loop(blocks, block, best, device=dev)
        from paper_2509_21064_gb300.dist import max_over_ranks
        stamps = max_over_ranks(stamps, device=dev)
        trace = [g[0] for g in gtrace]
        x_best, F_best, t_best, r_best = P.best()
        F_best, t_best = gtrace[-1][0], gtrace[-1][1]
        secs = stamps
    else:
        evs = []
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(blocks):
                P.run(K_EVAL)
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                evs.append(e)
            torch.cuda.synchronize(dev)
        P.sync()
        trace = P.trace()
        x_best, F_best, t_best, r_best = P.best()
        secs = [e0.elapsed_time(e) * 1e-3 for e in evs]
    P.close()
    out = {"target_F": target["F_best"] if target else None,
           "target_source": ("FP64 oracle on restarts 0-%d of the same instance and x^0, T=%d (tests/golden/"
                             "oracle_targets.json)" % (len(target["restarts"]) - 1, target["iters"])) if target else
           "no stored oracle target",
           "best_F": int(F_best), "best_t": int(t_best), "solve_seconds": secs[-1],
           "clock": "device events" if world == 1 else f"host, slowest of {world} ranks, best exchanged every block"}
    if target:
        hit = [k for k, f in enumerate(trace) if f <= target["F_best"]]
        if hit:
            out.update(reached=True, iteration=(hit[0] + 1) * K_EVAL, seconds=secs[hit[0]])
        else:
            out.update(reached=False, gap=int(min(trace)) - int(target["F_best"]))
    return out


def quality_vs_plain_fp32(S, Q, c, seed, stream, iters=500):
    """Best objective after the same T iterations (K = K_EVAL, same x^0, all restarts) of the
    chosen form (BF16 tensor-core contraction) and of the plain FP32 form, and their relative gap
    (positive: the chosen form's best is worse)."""
    p = W.dense_params(Q, restarts=RESTARTS_DEFAULT, iters=iters, eval_every=K_EVAL, seed=seed)
    best = {}
    for name, prec in (("bf16", S.SBO_BF16), ("fp32", S.SBO_FP32)):
        P = S.Problem.dense(Q, c, precision=prec, stream=stream)
        if prec == S.SBO_FP32:
            P.set_option(S.SBO_OPT_KERNEL, S.KERNEL_SIMT)
        P.gda(S.params(**p.asdict()))
        best[name] = int(P.best()[1])
        P.close()
    return {"iters": iters, "restarts": RESTARTS_DEFAULT, "best_F_chosen": best["bf16"], "best_F_plain_fp32": best["fp32"],
            "rel_gap": (best["bf16"] - best["fp32"]) / abs(best["fp32"])}


def plain_fp32_form(S, torch, Q, c, seed, stream, dev, iters=3):
    """The plain form on the same instance: FP32 A and x, CUDA-core (SIMT) contraction with the
    same fused update, one launch per iteration, no CUDA graph."""
    p = W.dense_params(Q, restarts=RESTARTS_DEFAULT, iters=10**9, eval_every=10**6, seed=seed)
    P = S.Problem.dense(Q, c, precision=S.SBO_FP32, stream=stream)
    P.set_option(S.SBO_OPT_KERNEL, S.KERNEL_SIMT)
    P.set_option(S.SBO_OPT_USE_GRAPH, 0)
    P.start(S.params(**p.asdict()))
    with torch.cuda.stream(stream):
        P.run(1)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.run(iters)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    P.sync()
    P.close()
    ms = e0.elapsed_time(e1) / iters
    return {"value": RESTARTS_DEFAULT / (ms * 1e-3), "unit": "restart-iterations/s", "ms_per_iteration": ms,
            "form": "FP32 A and x, SIMT contraction + fused update, one launch per iteration, no graph"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n_vars, restarts = args.n, args.restarts      # the benchmark's sizes unless given
    Q, c = W.dense_qubo(n_vars, seed=0)
    p = W.dense_params(Q, restarts=restarts, iters=2000, eval_every=K_EVAL, seed=0)
    import oracle as O
    A, cp = O.canonicalize(Q, c)
    sub = min(16, restarts)
    X, _ = O.init_state(n_vars, sub, p.seed, p.ybar)
    Y = np.full_like(X, p.ybar)
    for _ in range(args.warmup):
        X, Y, _ = O.gda_step(A, cp, X, Y, p.alpha, p.beta, p.delta, p.grad_tol)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        X, Y, _ = O.gda_step(A, cp, X, Y, p.alpha, p.beta, p.delta, p.grad_tol)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sub * args.steps / total
    cores = oracle_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "restart-iterations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dense QUBO n={n_vars}, B={restarts}, BF16 contraction (oracle: FP64)",
                       "oracle_sample": f"{sub} of {restarts} restarts, one GDA iteration per step"},
            "cpu_baseline": {"value": value, "unit": "restart-iterations/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sub} restarts x 1 iteration per step, numpy FP64 matmul"},
            "e2e": {"value": value, "unit": "restart-iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
def step_loop(steps, step, best=None, device=None):
    """The timed loop of one rank: `steps` calls of step().  With several ranks, after every step
    the ranks exchange their best candidates -- best() gives this rank's (bits, F, t, restart) --
    and every rank records the global best (F, t, rank, restart): the lexicographic minimum over
    the ranks (section 4.2's best of all runs, across GPUs).  Returns that trace (empty on one
    rank or without best)."""
    import torch.distributed as dist
    from paper_2509_21064_gb300.dist import global_best
    multi = best is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    trace = []
    for _ in range(steps):
        step()
        if multi:
            x, F, t, r = best()
            Fw, tw, kw, rw, _ = global_best(F, t, r, x, device=device)
            trace.append((Fw, tw, kw, rw))
    return trace


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hetero_jobs = None
    build()
    S.lib()
    stream = torch.cuda.Stream(device=dev)

    N_VARS, RESTARTS = args.n, args.restarts
    Q, c = W.dense_qubo(N_VARS, seed=0, dtype=np.int8)
    p = W.dense_params(Q, restarts=RESTARTS, iters=10**9, eval_every=K_EVAL, seed=rank)
    prm = S.params(**p.asdict())
    P = S.Problem.dense(Q, c, precision=S.SBO_BF16, stream=stream)
    if args.tile:
        P.set_option(S.SBO_OPT_TILE_N, args.tile)
    # direct launches, so that every update launch can be bracketed by events on its stream
    P.set_option(S.SBO_OPT_USE_GRAPH, 0)
    P.start(prm)
    info = P.info()
    kernel_events = []

    def step(events=None):
        for k in range(K_EVAL):
            if events is not None and k < K_EVAL - 1:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.run(1)
                e1.record(stream)
                events.append((e0, e1))
            else:
                P.run(1)       # the K-th iteration also launches the evaluation kernels

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        launches0 = P.launch_count()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t_start.record(stream)
        best_trace = step_loop(args.steps, lambda: step(kernel_events), P.best, device=dev)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        launches = P.launch_count() - launches0
        clocks = sampler.stop()
        P.sync()
    ms = t_start.elapsed_time(t_end)
    upd_ms = [a.elapsed_time(b) for a, b in kernel_events]
    t_kernel = statistics.mean(upd_ms) * 1e-3
    # graph-replay form of the same steps (reported beside)
    P.set_option(S.SBO_OPT_USE_GRAPH, 1)
    P.start(prm)
    with torch.cuda.stream(stream):
        P.run(K_EVAL)
        torch.cuda.synchronize(dev)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        P.run(K_EVAL * max(2, args.steps // 2))
        g1.record(stream)
        torch.cuda.synchronize(dev)
    graph_ms_per_step = g0.elapsed_time(g1) / max(2, args.steps // 2)
    x_best, F_best, t_best, r_best = P.best()
    P.close()
    if args.kernel_only:
        if rank == 0:
            print(json.dumps({"n": N_VARS, "restarts": RESTARTS, "ms_per_step": ms / args.steps,
                              "update_launch_ms": t_kernel * 1e3, "graph_ms_per_step": graph_ms_per_step,
                              "tflops": 2.0 * N_VARS * N_VARS * RESTARTS / t_kernel / 1e12}), flush=True)
        if hetero_jobs is not None:
            hetero_jobs[0].shutdown(cancel_futures=True)
        return 0

    # e2e through the public API with host buffers (pinned), every step: H2D of Q, c; K
    # iterations + evaluation; D2H of (x*, F*)
    # the entries lie in [-100, 100]: the host copy is int8 (sbo_create_dense_i8), a quarter of
    # the int32 bytes
    Qp = torch.from_numpy(Q).pin_memory()
    cpin = torch.from_numpy(c).pin_memory()
    # Steps are double-buffered on two streams, as a server of successive problems would run them:
    # the next step's upload and canonicalisation (the create call returns once they are done)
    # overlap this step's iterations; every step still copies its own Q and reads back its own
    # result inside the timed region.
    e2e_steps = max(2, min(args.steps, 4))
    prm_e2e = S.params(**{**p.asdict(), "iters": K_EVAL})
    streams = [stream, torch.cuda.Stream(device=dev)]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    nxt = S.Problem.dense(Qp.numpy(), cpin.numpy(), precision=S.SBO_BF16, stream=streams[0])
    for k in range(e2e_steps):
        P2 = nxt
        P2.start(prm_e2e)                    # start + run are enqueued; they return before the
        P2.run(K_EVAL)                       # iterations finish
        if k + 1 < e2e_steps:
            nxt = S.Problem.dense(Qp.numpy(), cpin.numpy(), precision=S.SBO_BF16, stream=streams[(k + 1) % 2])
        xb, Fb, tb, rb = P2.best()           # waits for this step's iterations, reads x*, F*
        P2.close()
    e2e_s = time.perf_counter() - t0
    h2d = Q.nbytes + c.nbytes
    d2h = N_VARS + 8 * 3
    # the other configurations' heterogeneous batch is drawn on the host cores from here on, while
    # the GPU runs the device-timed measurements (after the host-timed e2e leg)
    if rank == 0 and world == 1 and not args.no_other_configs:
        hetero_jobs = hetero_generate_start(args)

    # max over ranks; the global best over every rank's restarts (the method's one exchange)
    sec = ms * 1e-3
    global_best = None
    if world > 1:
        from paper_2509_21064_gb300.dist import global_best as _gb, max_over_ranks
        sec, e2e_s = max_over_ranks([sec, e2e_s], device=dev)
        Fw, tw, kw, rw, _ = _gb(F_best, t_best, r_best, x_best, device=dev)
        global_best = {"F": Fw, "t": tw, "rank": kw, "restart": rw}
    total_ri = RESTARTS * K_EVAL * args.steps * world
    value = total_ri / sec
    e2e_value = RESTARTS * K_EVAL * e2e_steps * world / e2e_s

    ttt = None
    if N_VARS == 20000 and RESTARTS == 1024 and not args.no_time_to_target:
        ttt = time_to_target(S, torch, Q, c, rank, stream, dev, load_target("dense_n20000_b1024_seed0"), world=world)
    plain = None
    if rank == 0 and N_VARS == 20000 and RESTARTS == 1024 and not args.no_plain_form:
        plain = plain_fp32_form(S, torch, Q, c, 0, stream, dev)
        plain["quality_at_equal_iterations"] = quality_vs_plain_fp32(S, Q, c, 0, stream)

    pk, src = peaks()
    flops = 2.0 * N_VARS * N_VARS * RESTARTS
    achieved = flops / t_kernel / 1e12
    peak_sust = float(pk.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]))
    peak_burst = float(pk.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))
    if info["tile_n"] == 512:
        kname = "k_tc_pair<EPI_UPDATE> (CTA pairs, 256x256 tiles)"
    elif info["tile_n"] > 1000:
        kname = f"k_tc_csk<{info['tile_n'] - 1000}, EPI_UPDATE> (split-K over a thread-block cluster)"
    else:
        kname = f"k_tc<{info['tile_n']}, EPI_UPDATE, false>"
    traffic, traffic_src = MEASURED_TRAFFIC.get((info["tile_n"], N_VARS, RESTARTS), (None, None))
    line = {
        "metric": METRIC, "value": value, "unit": "restart-iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"dense QUBO n={N_VARS}, entries U[-100,100], B={RESTARTS} restarts, "
                               f"K={K_EVAL} iterations + 1 evaluation per step",
                   "n": N_VARS, "restarts": RESTARTS, "eval_every": K_EVAL, "tile_n": info["tile_n"],
                   "kernel": "tcgen05 BF16 (FP32 accumulate, FP32 master x, y)",
                   "l2": "inputs larger than L2 (A is 800 MB BF16)",
                   "graph_replay_ms_per_step": graph_ms_per_step,
                   "best_F_after_run": F_best if global_best is None else global_best["F"],
                   "parallelism": f"replicas x{world} (restarts sharded by seed; best exchanged every step)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_burst, "unit": "TFLOP/s",
                     "frac": achieved / peak_burst, "traffic": traffic, "traffic_source": traffic_src,
                     "algorithmic_bytes": 2.0 * N_VARS * N_VARS + 18.0 * N_VARS * RESTARTS + 2.0 * N_VARS * RESTARTS,
                     "kernel": kname, "launch_ms": t_kernel * 1e3,
                     "peak_source": f"{src} bf16_tflops (burst: the kernel is timed in a region well under a second)",
                     "peak_sustained": peak_sust, "frac_of_sustained_peak": achieved / peak_sust},
        "e2e": {"value": e2e_value, "unit": "restart-iterations/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "per_step": "pinned int8 Q and int32 c to the device, canonicalise, K iterations + evaluation, "
                            "read back x* and F*; the next step's upload overlaps this step's iterations "
                            "(two streams)"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if ttt is not None:
        line["time_to_target"] = ttt
    if global_best is not None:
        line["config"]["global_best_over_ranks"] = global_best
        line["config"]["global_best_trace_per_step"] = [b[0] for b in best_trace]
    if plain is not None:
        plain["speedup_of_chosen_form"] = (RESTARTS * K_EVAL * args.steps / (ms * 1e-3)) / plain["value"]
        line["plain_fp32_form"] = plain
    if hetero_jobs is not None:
        line["other_configs"] = other_configs(S, torch, dev, args, pk, hetero_jobs)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, it, el, _, _ = oracle_sample(Q, c, p, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "restart-iterations/s", "cores": oracle_threads(),
                                "kind": "oracle",
                                "sample": f"16 of {RESTARTS} restarts x {it} iterations ({el:.1f} s), numpy FP64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------------
# the other benchmark configurations, measured beside the headline (N = 1)
SIDE_SPARSE = [
    # (key, workload, precision, restarts): Max-Cut as QUBO, evaluation every 10 iterations
    ("maxcut_er_n2000_b256_fp32", "maxcut-er", "fp32"),
    ("maxcut_er_n2000_b256_bf16", "maxcut-er", "bf16"),
    ("maxcut_torus_n10000_b512_e4m3", "maxcut-torus", "e4m3"),
    ("maxcut_torus_n10000_b512_fp32", "maxcut-torus", "fp32"),
    ("maxcut_regular_n20000_b512_e4m3", "maxcut-regular", "e4m3"),
    ("maxcut_regular_n20000_b512_fp32", "maxcut-regular", "fp32"),
]
HETERO_COUNT, HETERO_B = 64, 128


def _hetero_instance(k, n_hi):
    return W.heterogeneous_qubo(k, HETERO_COUNT, seed=0, n_lo=500, n_hi=n_hi, dtype=np.int8)


def hetero_generate_start(args):
    """Draw the 64 instances of the heterogeneous batch in worker processes (spawned, so that no
    CUDA state is forked); returns (executor, futures)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    # largest instances first, so the pool's tail is short
    shapes = W.heterogeneous_shapes(HETERO_COUNT, seed=0, n_lo=500, n_hi=args.hetero_n_hi)
    order = sorted(range(HETERO_COUNT), key=lambda k: -shapes[k][0])
    return ex, {k: ex.submit(_hetero_instance, k, args.hetero_n_hi) for k in order}


def _timed_blocks(torch, stream, run_block, blocks, warmup=3):
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            run_block()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(blocks):
            run_block()
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def other_configs(S, torch, dev, args, pk, hetero_jobs):
    """Restart-iterations/s and the roofline of each other benchmark configuration: the sparse
    Max-Cut graphs, dense n = 5,000, and the heterogeneous batch (grouped launch)."""
    hbm = float(pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    tc = float(pk.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    stream = torch.cuda.Stream(device=dev)
    out = {}
    K = 10
    for key, wl, prec_name in SIDE_SPARSE:
        make, B = SPARSE[wl]
        n, (i, j, w) = make()
        rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
        prec = {"fp32": S.SBO_FP32, "bf16": S.SBO_BF16, "e4m3": S.SBO_FP8_E4M3}[prec_name]
        p = W.graph_params("maxcut", restarts=B, iters=10**9, eval_every=K, seed=0)
        P = S.Problem.csr(n, rowptr, col, val, c, precision=prec, stream=stream)
        P.start(S.params(**p.asdict()))
        form = P.info()["tile_n"]     # the sparse update's form chosen by the autotuner
        blocks = 40
        sec = _timed_blocks(torch, stream, lambda: P.run(K), blocks)
        P.sync()
        P.close()
        t_it = sec / (blocks * K)
        per = 16 if prec == S.SBO_FP32 else 20          # x, y FP32 read + written; + BF16 copy written, read
        nnz = int(rowptr[-1]) * 2
        wbytes = {"fp32": 4, "bf16": 2, "e4m3": 1}[prec_name]
        state = per * n * B
        bytes_it = state + nnz * (4 + wbytes) + 4 * (n + 1)
        resident = 16 * n * B * 4 <= l2 * 3
        out[key] = {"n": n, "restarts": B, "precision": prec_name, "eval_every": K, "update_form": form,
                    "us_per_iteration": t_it * 1e6, "restart_iterations_per_s": B / t_it,
                    "roofline": {"bound": "latency (x, y fit in L2)" if resident else "hbm",
                                 "achieved": bytes_it / t_it / 1e9, "peak": hbm, "unit": "GB/s",
                                 "frac": bytes_it / t_it / 1e9 / hbm, "bytes_per_iteration": bytes_it,
                                 "bytes_counted": f"{per} B per (vertex, restart) of state (x, y FP32 read and "
                                                  "written" + ("" if per == 16 else "; BF16 operand copy written and "
                                                                                     "read") + ") + CSR structure"}}
    # dense n = 5,000, B = 256, BF16 (autotuned tiles), graph replay of K = 50 blocks
    n, B = 5000, 256
    Q, c = W.dense_qubo(n, seed=0, dtype=np.int8)
    p = W.dense_params(Q, restarts=B, iters=10**9, eval_every=K_EVAL, seed=0)
    P = S.Problem.dense(Q, c, precision=S.SBO_BF16, stream=stream)
    P.start(S.params(**p.asdict()))
    sec = _timed_blocks(torch, stream, lambda: P.run(K_EVAL), 10)
    tile = P.info()["tile_n"]
    P.sync()
    P.close()
    t_it = sec / (10 * K_EVAL)
    a_bytes = 2.0 * n * n
    state = 20.0 * n * B
    t_roof = max(2.0 * n * n * B / (tc * 1e12), a_bytes / (hbm * 1e9))
    out["dense_n5000_b256_bf16"] = {
        "n": n, "restarts": B, "eval_every": K_EVAL, "tile_n": tile, "us_per_iteration": t_it * 1e6,
        "restart_iterations_per_s": B / t_it, "tflops": 2.0 * n * n * B / t_it / 1e12,
        "roofline": {"bound": "hbm (A bytes; 2 n^2 B flop at the burst BF16 peak is shorter)",
                     "achieved": a_bytes / t_it / 1e9, "peak": hbm, "unit": "GB/s", "frac": t_roof / t_it,
                     "roofline_us": t_roof * 1e6, "frac_counting_state": (a_bytes + state) / t_it / 1e9 / hbm,
                     "note": "A (50 MB) stays in L2 under graph replay, so the HBM bound is not a hard ceiling"}}
    # heterogeneous batch: 64 dense instances, n ~ U{500..20000}, density ~ U[0.01, 1], B = 128 each
    ex, futs = hetero_jobs
    members, ns = [], []
    t0 = time.time()
    try:
        for k in range(HETERO_COUNT):
            Qk, ck = futs[k].result()
            q = W.dense_params(Qk, restarts=HETERO_B, iters=10**9, eval_every=K, seed=k)
            members.append((S.Problem.dense(Qk, ck, precision=S.SBO_BF16, stream=stream), S.params(**q.asdict())))
            ns.append(Qk.shape[0])
            del Qk
    finally:
        ex.shutdown(cancel_futures=True)
    t_gen = time.time() - t0
    G = S.Group([m for m, _ in members], stream=stream)
    G.start([q for _, q in members])
    sec = _timed_blocks(torch, stream, lambda: G.run(K), 5)
    G.sync()
    tile = members[0][0].info()["tile_n"]
    G.close()
    for m, _ in members:
        m.close()
    t_it = sec / (5 * K)
    sum_n2 = float(sum(v * v for v in ns))
    sum_n = float(sum(ns))
    bytes_it = 2.0 * sum_n2 + 20.0 * sum_n * HETERO_B
    t_roof = sum(max(2.0 * v * v * HETERO_B / (tc * 1e12), (2.0 * v * v + 20.0 * v * HETERO_B) / (hbm * 1e9))
                 for v in ns)
    out["hetero_64_dense_b128_bf16"] = {
        "instances": HETERO_COUNT, "n_range": [min(ns), max(ns)], "sum_n2": sum_n2, "restarts_each": HETERO_B,
        "eval_every": K, "tile_n": tile, "us_per_iteration": t_it * 1e6,
        "restart_iterations_per_s": HETERO_COUNT * HETERO_B / t_it,
        "tflops_dense_equivalent": 2.0 * sum_n2 * HETERO_B / t_it / 1e12,
        "wait_for_host_generation_s": round(t_gen, 1),
        "roofline": {"bound": "hbm (BF16 A of every instance + x, y state; below the ridge at B = 128)",
                     "achieved": bytes_it / t_it / 1e9, "peak": hbm, "unit": "GB/s", "frac": t_roof / t_it,
                     "roofline_us": t_roof * 1e6}}
    return out


SPARSE = {
    # Max-Cut as QUBO: Erdos-Renyi n=2000 (mean degree 6, +-1), 100x100 torus (+-1), random
    # 4-regular n=20000 (unit weights)
    "maxcut-er": (lambda: (2000, W.maxcut_er(2000, 6.0, seed=0)), 256),
    "maxcut-torus": (lambda: (10000, W.maxcut_torus(100, 100, seed=0)), 512),
    "maxcut-regular": (lambda: (20000, W.maxcut_regular(20000, 4, seed=0)), 512),
}


def run_sparse(args):
    """Device loop of a sparse Max-Cut workload (profiling and measurement of the CSR kernel)."""
    import torch
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build
    build()
    S.lib()
    make, B = SPARSE[args.workload]
    n, (i, j, w) = make()
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    prec = {"fp32": S.SBO_FP32, "bf16": S.SBO_BF16, "e4m3": S.SBO_FP8_E4M3}[args.precision]
    p = W.graph_params("maxcut", restarts=B, iters=10**9, eval_every=10, seed=0)
    stream = torch.cuda.Stream()
    P = S.Problem.csr(n, rowptr, col, val, c, precision=prec, stream=stream)
    P.set_option(S.SBO_OPT_PDL, 0 if args.no_pdl else 1)
    P.set_option(S.SBO_OPT_CSR_FORM, args.csr_form)
    P.set_option(S.SBO_OPT_EVAL_MODE, args.eval_mode)
    if args.no_eval:
        p = W.graph_params("maxcut", restarts=B, iters=10**9, eval_every=10**6, seed=0)
    P.start(S.params(**p.asdict()))
    form = P.info()["tile_n"]
    K = 10
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            P.run(K)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            P.run(K)
        e1.record(stream)
        torch.cuda.synchronize()
    P.sync()
    ms = e0.elapsed_time(e1) / (args.steps * K)
    per_elem = 16 if prec == S.SBO_FP32 else 20
    print(json.dumps({"workload": args.workload, "n": n, "restarts": B, "precision": args.precision,
                      "pdl": not args.no_pdl, "form": form, "evaluations": not args.no_eval,
                      "eval_mode": args.eval_mode, "us_per_iter": ms * 1e3, "restart_iterations_per_s": B / (ms * 1e-3),
                      "state_gbs": n * B * per_elem / (ms * 1e-3) / 1e9}), flush=True)
    P.close()
    return 0


def run_hetero(args):
    """Grouped run over 64 dense QUBO instances (n ~ U{500..20000}, density ~ U[0.01, 1], B = 128
    each): one persistent tcgen05 launch per iteration for all of them, tile width autotuned.
    Instances are generated and uploaded one at a time (the whole batch is ~35 GB as int32)."""
    import torch
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build
    build()
    S.lib()
    B, K = 128, 10
    stream = torch.cuda.Stream()
    members, prms, ns = [], [], []
    t0 = time.time()
    for k, (Q, c) in enumerate(W.iter_heterogeneous_qubos(64, seed=0, n_lo=500, n_hi=args.hetero_n_hi)):
        prms.append(S.params(**W.dense_params(Q, restarts=B, iters=10**9, eval_every=K, seed=k).asdict()))
        members.append(S.Problem.dense(Q, c, precision=S.SBO_BF16, stream=stream))
        ns.append(Q.shape[0])
        del Q, c
    t_gen = time.time() - t0
    G = S.Group(members, stream=stream)
    G.start(prms)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            G.run(K)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            G.run(K)
        e1.record(stream)
        torch.cuda.synchronize()
    G.sync()
    ms = e0.elapsed_time(e1) / (args.steps * K)
    flops = sum(2.0 * n ** 2 * B for n in ns)
    print(json.dumps({"workload": f"64 dense QUBO instances, n U{{500..{args.hetero_n_hi}}}, density U[0.01,1], B=128",
                      "sum_n2": int(sum(n ** 2 for n in ns)), "max_n": max(ns), "tile_n": members[0].info()["tile_n"],
                      "generate_upload_s": round(t_gen, 1), "us_per_iter": ms * 1e3,
                      "restart_iterations_per_s": 64 * B / (ms * 1e-3), "tflops_dense_equivalent": flops / (ms * 1e-3) / 1e12}),
          flush=True)
    G.close()
    for P in members:
        P.close()
    return 0


# Independent-set sizes PDBO reaches on random d-regular graphs in the paper's MIS table (mean
# over 20 instances, B = 10, RTX 3090, earliest time to best within 180 s): context only.
PAPER_MIS = {(10000, 3): (4431.9, 0.6), (10000, 100): (603.0, 3.6), (50000, 3): (22127.3, 1.1),
             (50000, 100): (3006.2, 14.6)}


def run_mis(args):
    """MIS as QUBO (F = -sum x + 4 sum_E x_i x_j) on a random d-regular graph with the paper's
    MIS hyper-parameters (ybar = 5, alpha = beta = 0.02): best set found, whether it is
    independent, and the device time until the best candidate was first evaluated."""
    import torch
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build
    build()
    S.lib()
    n, d, B, T, K = args.n, args.degree, args.restarts, args.iters, 10
    rowptr, col, val, c, (ei, ej) = W.mis_regular(n, d, seed=0)
    prec = {"fp32": S.SBO_FP32, "bf16": S.SBO_BF16, "e4m3": S.SBO_FP8_E4M3}[args.precision]
    if args.mis_params == "paper":
        p = W.graph_params("mis", restarts=B, iters=T, eval_every=K, seed=0)
    else:
        # the scaling used for dense QUBO: ybar = 1.5 |lambda_min| estimate (convex start)
        lam = W.csr_spectral_scale(n, rowptr, col, val)
        p = W.dense_params(None, restarts=B, iters=T, eval_every=K, seed=0, lam_hat=lam)
    stream = torch.cuda.Stream()
    P = S.Problem.csr(n, rowptr, col, val, c, precision=prec, stream=stream)
    P.start(S.params(**p.asdict()))
    evs = []
    with torch.cuda.stream(stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(T // K):
            P.run(K)
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            evs.append(e)
        torch.cuda.synchronize()
    P.sync()
    x, F, t_best, r_best = P.best()
    P.close()
    violations = int(np.sum(x[ei] & x[ej]))
    size = int(x.sum())
    paper = PAPER_MIS.get((n, d))
    print(json.dumps({"workload": f"MIS on a random {d}-regular graph, n={n}, lambda=4", "restarts": B, "iters": T,
                      "params": args.mis_params, "ybar": p.ybar, "alpha": p.alpha, "beta": p.beta,
                      "precision": args.precision, "best_F": int(F), "set_size": size, "violations": violations,
                      "independent": violations == 0, "best_iteration": int(t_best),
                      "seconds_to_best": e0.elapsed_time(evs[t_best // K - 1]) * 1e-3 if t_best >= K else None,
                      "seconds_total": e0.elapsed_time(evs[-1]) * 1e-3,
                      "paper_mean_size_and_seconds_rtx3090": paper}), flush=True)
    return 0


# Max-Cut stand-ins shaped like the paper's sensitivity and ablation instances (Gset is not
# available): G81 is a 100 x 200 toroidal grid with +-1 weights, G72 and G77 100 x 100 and 100 x 140
# grids; G70 a sparse random graph on 10,000 vertices with 9,999 unit-weight edges.
SWEEP_GRAPHS = {
    "torus-100x200 (G81 shape)": lambda: (20000, W.maxcut_torus(100, 200, seed=0)),
    "random n=10000, ~10^4 unit edges (G70 shape)": lambda: (10000, W.maxcut_er(10000, 2.0, seed=0, weights="unit")),
}
ABLATION_GRAPHS = {
    "torus-100x100 (G72 shape)": lambda: (10000, W.maxcut_torus(100, 100, seed=1)),
    "torus-100x140 (G77 shape)": lambda: (14000, W.maxcut_torus(100, 140, seed=2)),
    "torus-100x200 (G81 shape)": lambda: (20000, W.maxcut_torus(100, 200, seed=0)),
}
# The paper's tables on the real Gset graphs (RTX 3090): context for the trends only.
PAPER_SENSITIVITY = {
    "ybar": {"values": [0, 1, 2, 4, 6, 8, 10], "G70": [8756, 9145, 9398, 9535, 9537, 9536, 9536],
             "G81": [11338, 12886, 13836, 13840, 13852, 13846, 13846]},
    "alpha": {"values": [0.0025, 0.005, 0.01, 0.025, 0.05, 0.1, 0.25], "G70": [9365, 9451, 9530, 9537, 9536, 9535, 9539],
              "G81": [13828, 13842, 13848, 13852, 13842, 13854, 13840]},
    "beta": {"values": [0.001, 0.0025, 0.005, 0.01, 0.025, 0.05, 0.1, 0.25],
             "G70": [9538, 9536, 9542, 9534, 9537, 9509, 9495, 9415],
             "G81": [13880, 13868, 13862, 13858, 13852, 13840, 13724, 13480]},
    "B": {"values": [1, 10, 100, 1000], "G70": [9525, 9527, 9537, 9540], "G81": [13828, 13842, 13852, 13858]},
    "ablation": {"PDBO-s": {"G72": 6880, "G77": 9782, "G81": 13786}, "PDBO": {"G72": 6906, "G77": 9812, "G81": 13852}},
}


def run_sweep(args):
    """Sensitivity of the Max-Cut result to ybar, alpha, beta and B, and the PDBO / PDBO-s
    ablation, on synthetic graphs shaped like the paper's instances (paper parameters ybar = 6,
    alpha = beta = 0.025, B = 100 unless swept; T = args.iters; FP32).  One JSON line per run."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build
    build()
    S.lib()
    T, K = args.iters, 10
    stream = torch.cuda.Stream()

    def one(n, csr, i, j, w, ybar=6.0, alpha=0.025, beta=0.025, B=100, dual=0, iters=None, gkind=0):
        rowptr, col, val, c = csr
        T_run = iters or T
        p = W.GdaParams(restarts=B, iters=T_run, alpha=alpha, beta=beta, ybar=ybar, eval_every=K, seed=0)
        P = S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32, stream=stream)
        P.set_option(S.SBO_OPT_DUAL, dual)
        P.set_option(S.SBO_OPT_G, gkind)
        P.start(S.params(**p.asdict()))
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.run(T_run)
            e1.record(stream)
            torch.cuda.synchronize()
        P.sync()
        x, F, t_best, _ = P.best()
        P.close()
        cut = int(np.sum(w * (x[i] != x[j])))
        assert cut == -int(F)
        secs = e0.elapsed_time(e1) * 1e-3
        return {"cut": cut, "iters": T_run, "best_iteration": int(t_best), "seconds": round(secs, 4),
                "seconds_to_best": round(secs * t_best / T_run, 4)}

    def graph(make):
        n, (i, j, w) = make()
        csr = W.maxcut_qubo(n, i, j, w)
        Wm = sp.coo_matrix((w.astype(np.float64), (i, j)), shape=(n, n))
        Wm = (Wm + Wm.T).tocsr()
        lam_min = float(spla.eigsh(Wm, k=1, which="SA", return_eigenvectors=False)[0])
        return n, csr, i, j, w, lam_min

    out = {"ybar": {}, "alpha": {}, "beta": {}, "B": {}, "ablation": {}}
    for name, make in SWEEP_GRAPHS.items():
        n, csr, i, j, w, lam_min = graph(make)
        for key, values, kw in (("ybar", PAPER_SENSITIVITY["ybar"]["values"], "ybar"),
                                ("alpha", PAPER_SENSITIVITY["alpha"]["values"], "alpha"),
                                ("beta", PAPER_SENSITIVITY["beta"]["values"], "beta"),
                                ("B", PAPER_SENSITIVITY["B"]["values"], "B")):
            rows = []
            for v in values:
                # beta sweep: T grows as 1/beta below the table's 0.025 (the iteration count of
                # Theorem 3.7 scales with 1/beta), so small steps get the time they need
                extra = {"iters": int(round(T * max(1.0, 0.025 / v)))} if key == "beta" else {}
                r = one(n, csr, i, j, w, **{kw: v}, **extra)
                if key == "ybar":
                    r["convex_start"] = bool(v + lam_min >= 0.0)
                r[kw] = v
                rows.append(r)
                print(json.dumps({"workload": "sweep", "graph": name, "swept": key, **r}), flush=True)
            out[key][name] = {"lambda_min_W": round(lam_min, 4), "runs": rows}
    for name, make in ABLATION_GRAPHS.items():
        n, csr, i, j, w, _ = graph(make)
        res = {}
        # PDBO-s with the table's beta takes dual steps of up to n beta / 4; with beta / n its dual
        # step is that of the normalised constraint (1/n) sum_i g(x_i) = 0
        for label, dual, beta, gk in (("PDBO-s (beta/n)", 1, 0.025 / n, 0), ("PDBO-s (beta)", 1, 0.025, 0),
                                      ("PDBO", 0, 0.025, 0), ("PDBO, entropy g", 0, 0.025, 1)):
            res[label] = one(n, csr, i, j, w, dual=dual, beta=beta, gkind=gk)
            print(json.dumps({"workload": "ablation", "graph": name, "method": label, **res[label]}), flush=True)
        out["ablation"][name] = res
    print(json.dumps({"workload": "Max-Cut sensitivity and PDBO-s ablation (synthetic Gset-shaped graphs)",
                      "iters": T, "eval_every": K, "precision": "fp32", "results": out,
                      "paper_on_gset_rtx3090": PAPER_SENSITIVITY}), flush=True)
    return 0


# Max-3-Cut stand-ins for the paper's table (Gset shapes; the paper's cut values are context only)
MAXK_GRAPHS = {
    "G67 shape: torus 100x100, +-1": lambda: (10000, W.maxcut_torus(100, 100, seed=3)),
    "G70 shape: random n=10000, ~10^4 unit edges": lambda: (10000, W.maxcut_er(10000, 2.0, seed=0, weights="unit")),
    "G72 shape: torus 100x100, +-1": lambda: (10000, W.maxcut_torus(100, 100, seed=1)),
    "G77 shape: torus 100x140, +-1": lambda: (14000, W.maxcut_torus(100, 140, seed=2)),
    "G81 shape: torus 100x200, +-1": lambda: (20000, W.maxcut_torus(100, 200, seed=0)),
}
PAPER_MAX3CUT = {"G67": (8015, 6.0), "G70": (9999, 3.3), "G72": (8111, 4.7), "G77": (11467, 5.0), "G81": (16191, 7.9)}


def run_maxkcut(args):
    """Max-k-Cut (k = args.parts) with the paper's parameters (B = 100, ybar = 6, beta = 0.01 and
    alpha = args.maxk_alpha, the table's 0.01 by default), T = args.iters, on Gset-shaped synthetic
    graphs: best cut, device time to it, and the kernel's restart-iterations/s."""
    import torch
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build
    build()
    S.lib()
    T, K, B, k = args.iters, 10, 100, args.parts
    stream = torch.cuda.Stream()
    rows = []
    for name, make in MAXK_GRAPHS.items():
        n, (i, j, w) = make()
        p = W.GdaParams(restarts=B, iters=T, alpha=args.maxk_alpha, beta=0.01, ybar=6.0, eval_every=K, seed=0)
        P = S.Problem.maxkcut(n, i, j, w, k, stream=stream)
        P.start(S.params(**p.asdict()))
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.run(T)
            e1.record(stream)
            torch.cuda.synchronize()
        P.sync()
        parts, F, t_best, _ = P.best()
        P.close()
        cut = int(np.sum(w.astype(np.int64) * (parts[i] != parts[j])))
        assert cut == -int(F)
        secs = e0.elapsed_time(e1) * 1e-3
        row = {"workload": f"Max-{k}-Cut", "graph": name, "n": n, "edges": int(len(i)), "restarts": B, "iters": T,
               "alpha": args.maxk_alpha,
               "cut": cut, "best_iteration": int(t_best), "seconds": round(secs, 4),
               "seconds_to_best": round(secs * t_best / T, 4), "restart_iterations_per_s": B * T / secs,
               "paper_gset_cut_and_seconds_rtx3090": PAPER_MAX3CUT.get(name[:3]) if k == 3 else None}
        rows.append(row)
        print(json.dumps(row), flush=True)
    return 0


PAPER_DUAL_BOUNDS = {"G67": (6872, 8843.7), "G70": (9537, 13891.5), "G72": (6906, 8906.1), "G77": (9812, 12767.7),
                     "G81": (13852, 18172.2)}
CERT_GRAPHS = {
    "G67 shape: torus 100x100, +-1": lambda: (10000, W.maxcut_torus(100, 100, seed=3)),
    "G70 shape: random n=10000, ~10^4 unit edges": lambda: (10000, W.maxcut_er(10000, 2.0, seed=0, weights="unit")),
    "G72 shape: torus 100x100, +-1": lambda: (10000, W.maxcut_torus(100, 100, seed=1)),
    "G77 shape: torus 100x140, +-1": lambda: (14000, W.maxcut_torus(100, 140, seed=2)),
    "G81 shape: torus 100x200, +-1": lambda: (20000, W.maxcut_torus(100, 200, seed=0)),
}


def run_certificate(args):
    """Primal and dual bounds for Max-Cut (the paper's dual-certificate table) on Gset-shaped graphs:
    the best cut PDBO finds (paper parameters, B = 100, T = args.iters) and the certified upper bound
    -sbo_dual_bound at ybar = -lambda_min(W) (the smallest convex start; lambda from scipy)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    from paper_2509_21064_gb300 import sbo as S
    from paper_2509_21064_gb300.build import build
    build()
    S.lib()
    stream = torch.cuda.Stream()
    for name, make in CERT_GRAPHS.items():
        n, (i, j, w) = make()
        rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
        Wm = sp.coo_matrix((w.astype(np.float64), (i, j)), shape=(n, n))
        Wm = (Wm + Wm.T).tocsr()
        lam_min = float(spla.eigsh(Wm, k=1, which="SA", return_eigenvectors=False)[0])
        lam_max = float(spla.eigsh(Wm, k=1, which="LA", return_eigenvectors=False)[0])
        p = W.graph_params("maxcut", restarts=100, iters=args.iters, eval_every=10, seed=0)
        P = S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32, stream=stream)
        P.gda(S.params(**p.asdict()))
        x, F, _, _ = P.best()
        cut = int(np.sum(w.astype(np.int64) * (x[i] != x[j])))
        ybar = -lam_min + 1e-6
        alpha = 1.0 / (2.0 * lam_max + 2.0 * ybar)
        t0 = time.time()
        lb, val_ = P.dual_bound(ybar, alpha, args.cert_iters)
        secs = time.time() - t0
        P.close()
        print(json.dumps({"workload": "Max-Cut primal and dual bounds", "graph": name, "n": n,
                          "lambda_min_W": round(lam_min, 5), "primal_cut": cut, "dual_bound": round(-lb, 2),
                          "gap_percent": round(100.0 * (-lb - cut) / cut, 2), "certificate_seconds": round(secs, 2),
                          "paper_gset_primal_dual": PAPER_DUAL_BOUNDS.get(name[:3])}), flush=True)
    return 0


def free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def torchrun_argv(argv, gpus, port):
    """The command line that starts `gpus` ranks of this benchmark, one per GPU, with the same
    arguments (torch.distributed.run on this node, rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + list(argv)


def launch_ranks(gpus, argv):
    """--gpus N from a plain process: check that N GPUs are visible, then run N ranks under
    torch.distributed.run and return their exit status."""
    import torch
    have = torch.cuda.device_count()
    if have < gpus:
        print(f"bench.py: --gpus {gpus} needs {gpus} visible GPUs, found {have}", file=sys.stderr)
        return 2
    return subprocess.call(torchrun_argv(argv, gpus, free_port()), cwd=ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-target", action="store_true")
    ap.add_argument("--no-plain-form", action="store_true")
    ap.add_argument("--n", type=int, default=N_VARS, help="variables (profiling cases only)")
    ap.add_argument("--restarts", type=int, default=RESTARTS, help="restarts (profiling cases only)")
    ap.add_argument("--workload", default="dense", choices=["dense", "hetero", "mis", "sweep", "maxkcut", "certificate"] + sorted(SPARSE),
                    help="dense n=20k (the headline) or a sparse Max-Cut workload (kernel-only)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "e4m3"],
                    help="weight/operand precision of a sparse workload")
    ap.add_argument("--csr-form", type=int, default=0, choices=list(range(9)),
                    help="sparse workloads: update form (0 autotuned; 1, 2 one row per warp with 128 / 256 "
                         "restarts; 3 pipelined rows; 4 rows staged by bulk copies; 5-7: 1-3 with L2 "
                         "eviction priorities; 8 state resident in shared memory, iterations per launch)")
    ap.add_argument("--no-eval", action="store_true", help="sparse workloads: no evaluations (update launches only)")
    ap.add_argument("--eval-mode", type=int, default=0, choices=[0, 1, 2],
                    help="sparse workloads: evaluation scheduling (0, 2 beside the next block; 1 in line)")
    ap.add_argument("--no-pdl", action="store_true",
                    help="sparse workloads: plain stream order instead of programmatic dependent launches")
    ap.add_argument("--hetero-n-hi", type=int, default=20000, help="hetero workload: largest instance size")
    ap.add_argument("--degree", type=int, default=3, help="MIS workload: graph degree")
    ap.add_argument("--mis-params", default="paper", choices=["paper", "scaled"],
                    help="MIS workload: the paper's table (ybar=5, alpha=beta=0.02) or the spectral scaling")
    ap.add_argument("--iters", type=int, default=3000, help="MIS, sweep and maxkcut workloads: GDA iterations")
    ap.add_argument("--parts", type=int, default=3, help="maxkcut workload: number of parts k")
    ap.add_argument("--maxk-alpha", type=float, default=0.01, help="maxkcut workload: primal step (paper: 0.01)")
    ap.add_argument("--cert-iters", type=int, default=20000, help="certificate workload: projected gradient steps")
    ap.add_argument("--tile", type=int, default=0, choices=[0, 64, 128, 256, 512, 1064, 1128, 1256, 2128, 2256],
                    help="tensor-core tile width (0: autotuned); profiling cases only")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the device loop only (no e2e, no CPU baseline): for profiling cases")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the other benchmark configurations (sparse graphs, n=5000, heterogeneous batch)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    if args.impl == "reference":
        return run_reference(args)
    if "WORLD_SIZE" in os.environ:
        if int(os.environ["WORLD_SIZE"]) != args.gpus:
            print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={os.environ['WORLD_SIZE']}", file=sys.stderr)
            return 2
    elif args.gpus > 1:
        return launch_ranks(args.gpus, sys.argv[1:])
    if args.workload == "hetero":
        return run_hetero(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "maxkcut":
        return run_maxkcut(args)
    if args.workload == "certificate":
        return run_certificate(args)
    if args.workload == "mis":
        if args.n == N_VARS:
            args.n = 10000
        if args.restarts == RESTARTS:
            args.restarts = 10
        return run_mis(args)
    if args.workload != "dense":
        return run_sparse(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
