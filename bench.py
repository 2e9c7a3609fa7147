"""Benchmark of parallel GOM (weighted Max-Cut) on GB300.

A step is one generation of parallel GOMEA (Alg. 3): generation start, group
order, one mixing launch per colour group, generation end.  The metric is GOM
trials per second (a trial is one (individual, FOS element) pair, donor-less
trials included); time-to-target and the mixing kernel's HBM roofline
fraction are reported beside it.

Default workload: 2D torus 1000x1000 (n = 1,000,000, 2,000,000 edges), int32
weights uniform in [1,100] from seed 1, neighbourhood FOS, Welsh-Powell
colouring, population 256, Philox seed 1.  The default line also carries, as
`extras`, plain GOM on the 100x100 torus (trials/s, time to target with the
IMS and the bounded linkage tree), batched against sequential plain GOM on
the 256-instance mix, and the learned trial filter against plain GOM.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gom|reference]
                [--workload NAME] [--pop P]
Under torchrun (N > 1) each rank runs an independent replica (seed + rank):
replicas only, weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2203_08680_gb300 import instances as I  # noqa: E402

WORKLOADS = {
    # name: (graph builder, population, description)
    "torus100": (lambda: I.torus2d(100), 64,
                 "2D torus 100x100 (n=10,000, 20,000 edges), int32 weights U[1,100] seed 1, pop 64"),
    "torus10": (lambda: I.torus2d(10), 16,
                "2D torus 10x10 (n=100, 200 edges), int32 weights U[1,100] seed 1, pop 16"),
    "torus3d50": (lambda: I.torus3d(50), 512,
                  "3D torus 50^3 (n=125,000, 375,000 edges), int32 weights U[1,100], pop 512"),
    "rreg1m_d3": (lambda: I.random_regular(1_000_000, 3), 512,
                  "random 3-regular n=1,000,000, int32 weights U[1,100], pop 512"),
    "rreg1m_d6": (lambda: I.random_regular(1_000_000, 6), 512,
                  "random 6-regular n=1,000,000, int32 weights U[1,100], pop 512"),
    "rreg1m_d12": (lambda: I.random_regular(1_000_000, 12), 512,
                   "random 12-regular n=1,000,000, int32 weights U[1,100], pop 512"),
    "torus1000": (lambda: I.torus2d(1000), 256,
                  "2D torus 1000x1000 (n=1,000,000), int32 weights U[1,100], pop 256"),
    "torus100_lt128": (lambda: I.torus2d(100), 1024,
                       "2D torus 100x100 (n=10,000, 20,000 edges), int32 weights U[1,100] seed 1, pop 1024, "
                       "bounded linkage tree FOS (UPGMA on the weights, sets of up to 128 variables)"),
}
# workloads whose FOS is the bounded linkage tree (Sec. 4.1), by bound; the rest use the neighbourhood FOS
WORKLOAD_BFLT = {"torus100_lt128": 128}
BFLT_ORACLE_NOTE = ("the oracle states UPGMA plainly (every cluster pair rescanned per merge), which takes "
                    "hours at n = 10,000; no CPU figure for linkage-tree workloads")
BATCH_WORKLOADS = {
    "batch256": "256 independent Max-Cut instances in one persistent launch: random d-regular graphs, n "
                "log-uniform in [1000, 65536] (even), d uniform in 3..8, int32 weights U[1,100], pop uniform "
                "over {32, 64, 128, 256}, graph and Philox seeds 1..256",
}
# autotuner candidates: (warps per block, register budget in resident blocks, grid cap, item cost)
LEARNED_WORKLOADS = {
    "learned1000": "learned trial filter on the 2D torus 1000x1000 (n=1,000,000), int32 weights U[1,100], pop 256: "
                   "MLP (16 features, 64 hidden, bf16 weights, fp32 accumulation) trained on the log of 50 plain "
                   "generations (label: the element had an improving trial), then run to the fitness plain GOM "
                   "reaches at generation 200",
}
BATCH_CONFIGS = [(4, 3, 0, 300), (4, 3, 0, 100), (4, 3, 0, 1000), (2, 3, 0, 300), (4, 2, 0, 300), (8, 3, 0, 300),
                 (8, 2, 0, 300)]
SEED = 1
# the largest single-GPU plain configuration: the 1000x1000 torus (the learned filter's graph), plain GOM
DEFAULT_WORKLOAD = "torus1000"
L2_BYTES = 129 * 1024 * 1024
METRIC = "GOM trials/sec (plain parallel GOM, weighted Max-Cut)"


def mixing_bytes_per_generation(g, eptr, evars, p: int) -> int:
    """Algorithmic bytes of all mixing launches of one generation: per element
    j, p (|C_j| + 2|F_j|) / 8 bytes of bit-sliced population (parent closure
    C_j = F_j u adj(F_j), donor bits and the write on F_j) plus the element's
    adjacency, 8 bytes per CSR entry of its variables and 4 bytes per
    variable, read once for all p individuals."""
    import scipy.sparse as sp
    n = g.n
    m = len(eptr) - 1
    sizes = np.diff(eptr)
    A = sp.csr_matrix((np.ones(len(g.col), dtype=np.int8), g.col, g.row_ptr), shape=(n, n))
    AI = (A + sp.identity(n, dtype=np.int8, format="csr")).tocsr()
    closure = np.zeros(m, dtype=np.int64)
    chunk = 65536
    for a in range(0, m, chunk):
        b = min(m, a + chunk)
        rows = np.repeat(np.arange(b - a), sizes[a:b])
        M = sp.csr_matrix((np.ones(len(rows), dtype=np.int8), (rows, evars[eptr[a]:eptr[b]])),
                          shape=(b - a, n))
        closure[a:b] = np.diff((M @ AI).tocsr().indptr)
    deg = np.diff(g.row_ptr)
    csr_bytes = 8 * np.add.reduceat(deg[evars], eptr[:-1]) + 4 * sizes
    pop_bytes = p * (closure + 2 * sizes) / 8.0
    return int(round(float(pop_bytes.sum() + csr_bytes.sum())))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """sha256 prefix of every device-code source of the library (kernels,
    shared device headers, the parameter structures)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2203_08680_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")) or fn == "gom_internal.h":
            with open(os.path.join(csrc, fn), "rb") as fh:
                h.update(fn.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on this workload with the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(f"{kernel.split()[0]}:{workload}")
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            # samples go to a file of their own; the line reports their summary
            fd, self.path = tempfile.mkstemp(prefix="gom_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def dist_max(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_threads() -> int:
    from oracle import oracle as O
    return max(1, O.max_threads())


class OracleSample:
    """The CPU oracle as it stands on one workload, timed on bounded samples:
    a step is one generation (its multi-threaded form for threads > 1) of the
    whole population, or, when that would take longer than step_s, of an
    evenly spread subset of the individuals sized from a probe generation
    (trials of one group are independent, so a subset's trials are the
    workload's own)."""

    def __init__(self, g, p: int, seed: int, threads: int = 1, step_s: float = 0.5):
        from oracle import oracle as O
        ep, ev = O.build_fos(g)
        k, co = O.color(g, ep, ev)
        self.run = O.Run(g, ep, ev, co, k, p, seed)
        self.p, self.m, self.threads = p, len(ep) - 1, threads
        self.only = None
        probe = self._subset(min(p, max(threads, 4)))
        t0 = time.perf_counter()
        self.step(probe)
        rate = len(probe) * self.m / (time.perf_counter() - t0)
        want = max(threads, int(rate * step_s / max(self.m, 1)))  # at least one individual per thread
        if want < p:
            self.only = self._subset(max(1, want))

    def _subset(self, q: int):
        return None if q >= self.p else [int(i) for i in np.linspace(0, self.p - 1, q).round()]

    def step(self, only="default"):
        only = self.only if isinstance(only, str) else only
        self.run.generation(threads=self.threads, only=only)
        return (self.p if only is None else len(only)) * self.m

    def describe(self) -> str:
        who = "the whole population" if self.only is None else f"{len(self.only)} of {self.p} individuals"
        return f"generations of {who}, {self.threads} thread(s)"


def oracle_trials_per_sec(g, p: int, seed: int, budget_s: float, warmup: int = 0, steps: int = None,
                          threads: int = 1):
    """The CPU oracle timed on bounded samples (OracleSample): steps until
    budget_s, or `steps` steps after `warmup`.  Returns (trials/s, steps,
    seconds, sample description)."""
    S = OracleSample(g, p, seed, threads)
    for _ in range(warmup):
        S.step()
    gens, trials, t0 = 0, 0, time.perf_counter()
    while True:
        trials += S.step()
        gens += 1
        el = time.perf_counter() - t0
        if (steps is not None and gens >= steps) or (steps is None and el >= budget_s):
            break
    return trials / el, gens, el, S.describe()


def run_reference(args, wl, rank, world):
    """Reference arm: the CPU oracle on this workload, rank 0 only."""
    if rank != 0:
        return
    if wl in BATCH_WORKLOADS:
        # steps: one oracle generation each of the first warmup + steps instances of the mix
        mix = I.batch_mix(seed=SEED)[: args.warmup + args.steps]
        graphs = [I.random_regular(n, d, s) for n, d, p, s in mix]
        nth = oracle_threads()
        oracle_batch_sample(graphs[: args.warmup], mix[: args.warmup], float("inf"), nth)
        val, ninst, done, el = oracle_batch_sample(graphs[args.warmup:], mix[args.warmup:], float("inf"), nth)
        line = {"impl": "reference", "metric": "GOM trials/sec (batched parallel GOM, weighted Max-Cut)",
                "value": val, "unit": "trials/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * el / max(ninst, 1), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": wl, "description": BATCH_WORKLOADS[wl]},
                "cpu_baseline": {"value": val, "unit": "trials/s", "cores": nth, "kind": "oracle",
                                 "sample": f"one generation of each of instances {args.warmup}.."
                                           f"{args.warmup + ninst - 1} of the mix, {nth} threads"},
                "e2e": {"value": val, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if wl in WORKLOAD_BFLT:
        print(json.dumps({"impl": "reference", "unavailable": BFLT_ORACLE_NOTE}), flush=True)
        return
    # the learned workload's reference is the oracle on its graph (plain GOM, no filter)
    build, p, desc = WORKLOADS["torus1000" if wl in LEARNED_WORKLOADS else wl]
    g = build()
    nth = oracle_threads()
    val, gens, el, what = oracle_trials_per_sec(g, p, SEED, 0.0, warmup=args.warmup, steps=args.steps,
                                                threads=nth)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "trials/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / gens,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": wl, "description": desc},
            "cpu_baseline": {"value": val, "unit": "trials/s", "cores": nth, "kind": "oracle",
                             "sample": f"{gens} steps after {args.warmup} warm-up; a step is one of the "
                                       f"{what}"},
            "e2e": {"value": val, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, wl, rank, world, local):
    import torch

    from paper_2203_08680_gb300 import gom

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build, p, desc = WORKLOADS[wl]
    if args.pop:
        p = args.pop
    g = build()
    seed = SEED + rank
    stream = torch.cuda.current_stream()
    bflt = WORKLOAD_BFLT.get(wl, 0)
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bflt) if bflt else None
    bits = None if args.bitsliced == "auto" else args.bitsliced == "on"
    P = gom.Population(g, p, seed, fos=fos, stream=stream,
                       persistent=None if args.path == "auto" else args.path == "persistent", bitsliced=bits)
    m, k = P.m, P.k
    persistent = bool(gom.gom_get_option(P.ctx, gom.GOM_OPT_PERSISTENT))
    bitsliced = bool(gom.gom_get_option(P.ctx, gom.GOM_OPT_BITSLICED))
    trials_per_step = p * m
    ex = gom.gom_fos_export(P.fos)
    mix_bytes = mixing_bytes_per_generation(g, ex["elem_ptr"], ex["elem_vars"], p)
    gen_bytes = mix_bytes + g.n * p // 4 + 16 * p  # + clone of the population, fitness and flags
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    # warm-up generations (untimed)
    P.generation(args.warmup, want_stats=False)
    torch.cuda.synchronize()
    if not persistent:
        gom.gom_set_timing(P.ctx, True)
        gom.gom_read_timing(P.ctx)  # reset
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    dist_barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xFF)  # L2 flush between timed generations (outside the events)
            ev0[s].record(stream)
            gom.gom_generation(P.ctx, 1, gom.INT64_MAX, want_stats=False)
            ev1[s].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    launches_per_step = gom.gom_launches_per_generation(P.ctx) + (0 if persistent else 1)
    if persistent:
        dom = {"kernel": "k_run_bs (persistent generation kernel, bit-sliced mixing)" if bitsliced else
               "k_run (persistent generation kernel)", "bytes_per_launch": gen_bytes,
               "avg_ms": sum(step_ms) / len(step_ms), "launches": args.steps}
    else:
        mix_ms, mix_launches = gom.gom_read_timing(P.ctx)
        gom.gom_set_timing(P.ctx, False)
        dom = {"kernel": "k_mix_bs" if bitsliced else "k_mix", "bytes_per_launch": mix_bytes / k,
               "avg_ms": mix_ms / max(mix_launches, 1), "launches": mix_launches}
    dist_barrier(world)
    total_ms = dist_max(sum(step_ms), world)
    value = world * trials_per_step * args.steps / (total_ms / 1e3)

    # the mixing kernel alone: per-launch events on the graph path
    mix = None
    if args.mix_steps > 0:
        Q = gom.Population(g, p, seed, stream=stream, persistent=False, fos=P.fos, bitsliced=bitsliced)
        Q.generation(args.warmup, want_stats=False)
        gom.gom_set_timing(Q.ctx, True)
        gom.gom_read_timing(Q.ctx)
        for s in range(args.mix_steps):
            flush.fill_(s & 0xFF)
            gom.gom_generation(Q.ctx, 1, gom.INT64_MAX, want_stats=False)
        mix_ms, mix_launches = gom.gom_read_timing(Q.ctx)
        peak, peak_kind = peaks()
        avg = mix_ms / max(mix_launches, 1)
        ach = (mix_bytes / k) / (avg / 1e3) / 1e9
        mix = {"kernel": "k_mix_bs" if bitsliced else "k_mix", "avg_launch_ms": avg, "launches": mix_launches,
               "algorithmic_bytes_per_launch": mix_bytes / k, "achieved_gbs": ach, "frac": ach / peak}
        del Q

    # time to target: fresh population, within 0.1% of the closed-form optimum
    # (every edge cut on an even torus) or a generation cap
    ttt = None
    if not args.no_ttt:
        ttt = time_to_target(args, g, p, seed, stream, wl, fos)
        if wl == "torus100":
            ttt.update(torus100_ttt_extras(args, g, seed, stream))

    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, g, p, seed, stream, dev, world, ex, m, trials_per_step, bflt)

    # CPU baseline: the oracle, bounded sample, rank 0
    cpu = None
    if rank == 0 and not args.no_cpu and bflt:
        cpu = {"value": None, "kind": "oracle", "unavailable": BFLT_ORACLE_NOTE}
    elif rank == 0 and not args.no_cpu:
        nth = oracle_threads()
        cval, cgens, cel, cwhat = oracle_trials_per_sec(g, p, seed, args.cpu_seconds / 2, threads=nth)
        sval, sgens, sel, swhat = oracle_trials_per_sec(g, p, seed, args.cpu_seconds / 2)
        cpu = {"value": cval, "unit": "trials/s", "cores": nth, "kind": "oracle",
               "sample": f"{cgens} {cwhat} from initialisation ({cel:.1f} s)",
               "single_thread": {"value": sval, "cores": 1,
                                 "sample": f"{sgens} {swhat} from initialisation ({sel:.1f} s)"}}
    line = finish(args, wl, rank, world, desc, p, m, k, value, total_ms, dom, mix, ttt, e2e,
                  launches_per_step, clk, cpu, persistent)
    line["config"]["mixing"] = "bit-sliced" if bitsliced else "per-lane"
    return line


def torus100_ttt_extras(args, g, seed, stream):
    """Time-to-target runs beside plain GOM on the 100x100 torus: the IMS over
    the neighbourhood FOS, and the paper's bounded linkage tree (bounds 100
    and 128, p = --lt-pop) alone and under the IMS."""
    out = {"ims": ims_time_to_target(args, g, seed, stream)}
    out["linkage_tree"] = [linkage_tree_time_to_target(args, g, seed, stream, b) for b in (100, 128)]
    out["linkage_tree"].append(ims_time_to_target(args, g, seed, stream, bflt=128, base=128, c=2, chunk=16))
    # Forced Improvement (Sec. 4), which the paper's parallel GOMEA leaves out: the neighbourhood FOS at p = 64
    # and the paper's linkage tree at its bound of 100
    out["forced_improvement"] = {"plain_p64": time_to_target(args, g, 64, seed, stream, "torus100", fi=True),
                                 "linkage_tree_100": linkage_tree_time_to_target(args, g, seed, stream, 100, fi=True)}
    return out


def extras(args, rank, world, local):
    """The rest of the metric, measured in the same run as the headline line:
    plain GOM on the 100x100 torus (trials/s and time to target, with the IMS
    and linkage-tree runs), batched against sequential plain GOM on the
    256-instance mix, and the learned trial filter against plain GOM on the
    1000x1000 torus."""
    import copy

    import torch
    stream = torch.cuda.current_stream()
    out = {}
    t0 = time.perf_counter()
    a = copy.copy(args)
    a.no_cpu, a.no_e2e, a.mix_steps = True, True, 0
    a.steps = min(args.steps, 200)
    a.ims_seconds = min(args.ims_seconds, 5.0)
    build, p, desc = WORKLOADS["torus100"]
    g = build()
    line = run_gpu(a, "torus100", rank, world, local)
    out["torus100"] = {"description": desc, "trials_per_sec": line["value"], "ms_per_generation": line["ms_per_step"],
                       "roofline_frac": line["roofline"]["frac"], "time_to_target": line["time_to_target"],
                       "seconds": time.perf_counter() - t0}
    t0 = time.perf_counter()
    b = copy.copy(args)
    b.no_cpu, b.no_e2e = True, True
    b.steps = min(args.steps, 20)
    bl = run_batch(b, "batch256", rank, world, local)
    out["batch256"] = {"description": BATCH_WORKLOADS["batch256"], "trials_per_sec": bl["value"],
                       "ms_per_generation": bl["ms_per_step"], "plain_gpu": bl["plain_gpu"],
                       "speedup_of_batch_over_plain": bl["plain_gpu"]["speedup_of_batch"],
                       "roofline_frac": bl["roofline"]["frac"], "batch_config": bl["config"]["batch_config"],
                       "seconds": time.perf_counter() - t0}
    t0 = time.perf_counter()
    ll = run_learned(args, "learned1000", rank, world, local)
    out["learned1000"] = {"description": LEARNED_WORKLOADS["learned1000"], "plain_ms": ll["plain"]["ms"],
                          "learned_ms": ll["value"], "reached": ll["learned"]["reached"],
                          "speedup_vs_plain": ll["speedup_vs_plain"], "target": ll["config"]["target"],
                          "generations_filtered": ll["learned"]["generations_filtered"],
                          "seconds": time.perf_counter() - t0}
    return out


def oracle_batch_sample(graphs, mix, budget_s: float, threads: int, max_instances: int = None):
    """The oracle on the instances of a batch taken in order, one generation
    each, until budget_s seconds of generations (set-up not timed) or
    max_instances; returns (trials/s, instances, trials, seconds)."""
    from oracle import oracle as O
    done, el, ninst = 0, 0.0, 0
    for g, (n, d, p, sd) in zip(graphs, mix):
        ep, ev = O.build_fos(g)
        kk, co = O.color(g, ep, ev)
        run = O.Run(g, ep, ev, co, kk, p, sd)
        t0 = time.perf_counter()
        run.generation(threads=threads)
        el += time.perf_counter() - t0
        done += p * (len(ep) - 1)
        ninst += 1
        if el > budget_s or (max_instances is not None and ninst >= max_instances):
            break
    return done / el, ninst, done, el


def run_batch(args, wl, rank, world, local):
    """Batched GOM: every instance of the mix, one persistent launch per
    generation (gom_batch_generation); beside it the same instances run one
    after another with their own gom_generation calls (plain GPU GOM).  Both
    give every instance the same generations bit for bit, so the ratio of
    their generation times is also their ratio of time to any target."""
    import torch

    from paper_2203_08680_gb300 import gom
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    mix = I.batch_mix(seed=SEED + rank)[: args.batch_count]
    graphs = [I.random_regular(n, d, s) for n, d, p, s in mix]
    pops = [gom.Population(g, p, s, stream=stream) for g, (n, d, p, s) in zip(graphs, mix)]
    ctxs = [P.ctx for P in pops]
    trials_per_step = sum(P.p * P.m for P in pops)
    mix_bytes = 0
    for g, P in zip(graphs, pops):
        ex = gom.gom_fos_export(P.fos)
        mix_bytes += mixing_bytes_per_generation(g, ex["elem_ptr"], ex["elem_vars"], P.p) + g.n * P.p // 4 + 16 * P.p
    # autotuner: the configuration with the fastest generations (state restored after every trial)
    scratch = torch.empty(gom.gom_batch_scratch_bytes(ctxs) + 256, dtype=torch.uint8, device=dev)
    scratch = scratch[(-scratch.data_ptr()) % 256:]
    best, tune_ms = gom.gom_batch_autotune(ctxs, BATCH_CONFIGS, 2, scratch, stream)
    del scratch
    ws = torch.empty(gom.gom_batch_workspace_bytes(len(ctxs)) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    batch = gom.gom_batch_create(ctxs, BATCH_CONFIGS[best], ws, stream)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        gom.gom_batch_generation(batch, 1, want_counts=False)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    dist_barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xFF)
            ev0[s].record(stream)
            gom.gom_batch_generation(batch, 1, want_counts=False)
            ev1[s].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    dist_barrier(world)
    total_ms = dist_max(sum(step_ms), world)
    value = world * trials_per_step * args.steps / (total_ms / 1e3)
    # plain GPU GOM: the instances one after another, each its own persistent launch
    plain_steps = max(1, min(args.steps, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_ms = 0.0
    for s in range(plain_steps):
        flush.fill_(s & 0xFF)
        e0.record(stream)
        for P in pops:
            gom.gom_generation(P.ctx, 1, gom.INT64_MAX, want_stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms += e0.elapsed_time(e1)
    plain_ms /= plain_steps
    batch_ms = total_ms / args.steps
    # end to end through the C ABI from host buffers: FOS, colouring, uploads, the
    # batch, args.steps batched generations, populations and fitness back to host
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hctx, keep, h2d, d2h = [], [], 0, 0
        for g, (n, d, p, sd) in zip(graphs, mix):
            G = gom.Graph(g)
            fos = gom.gom_build_fos(G)
            gom.gom_color_fos(G, fos)
            nb = gom.gom_workspace_bytes(G, fos, p)
            w = torch.empty(nb, dtype=torch.uint8, device=dev)
            hctx.append(gom.gom_init_population(G, fos, p, sd, w, nb, stream))
            keep.append((G, fos))
            h2d += G.row_ptr.nbytes + G.col.nbytes + G.weight.nbytes
        w2 = torch.empty(gom.gom_batch_workspace_bytes(len(hctx)) + 256, dtype=torch.uint8, device=dev)
        w2 = w2[(-w2.data_ptr()) % 256:]
        b2 = gom.gom_batch_create(hctx, BATCH_CONFIGS[best], w2, stream)
        gom.gom_batch_generation(b2, args.steps)
        outs = []
        for c, (n, d, p, sd) in zip(hctx, mix):
            dpop = torch.empty((p, n), dtype=torch.uint8, device=dev)
            dfit = torch.empty(p, dtype=torch.int64, device=dev)
            gom.gom_get_population(c, dpop, dfit, False)
            outs.append((dpop.to("cpu"), dfit.to("cpu")))
            d2h += p * n + 8 * p
        torch.cuda.synchronize()
        e2e_s = dist_max(time.perf_counter() - t0, world)
        e2e = {"value": trials_per_step * args.steps * world / e2e_s, "unit": "trials/s",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps)}
        del b2, hctx, outs
    cpu = None
    if rank == 0 and not args.no_cpu:
        # the oracle on instances of the mix taken in order, one generation each, within the budget
        nth = oracle_threads()
        val, ninst, done, el = oracle_batch_sample(graphs, mix, args.cpu_seconds, nth)
        cpu = {"value": val, "unit": "trials/s", "cores": nth, "kind": "oracle",
               "sample": f"one generation of each of the first {ninst} instances of the mix ({done} trials in "
                         f"{el:.1f} s of generations, {nth} threads)"}
    peak, peak_kind = peaks()
    achieved = mix_bytes / (batch_ms / 1e3) / 1e9
    line = {
        "metric": "GOM trials/sec (batched parallel GOM, weighted Max-Cut)", "value": value, "unit": "trials/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": wl if len(pops) == 256 else f"{wl}[:{len(pops)}]", "description": BATCH_WORKLOADS[wl],
                   "instances": len(pops),
                   "trials_per_generation": trials_per_step, "batch_config": list(BATCH_CONFIGS[best]),
                   "autotune_ms_per_generation": dict(zip(["x".join(map(str, c)) for c in BATCH_CONFIGS], tune_ms)),
                   "grid": gom.gom_batch_layout(batch, 0)[2],
                   "l2": "flushed between timed generations (2x L2 buffer write)",
                   "parallelism": f"replicas{world}"},
        "plain_gpu": {"ms_per_generation": plain_ms, "trials_per_sec": trials_per_step / (plain_ms / 1e3),
                      "launches_per_generation": len(pops), "generations_timed": plain_steps,
                      "speedup_of_batch": plain_ms / batch_ms},
        "roofline": {"bound": "hbm", "kernel": "k_batch (batched persistent generation kernel)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(wl, "k_batch"), "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": mix_bytes, "avg_launch_ms": batch_ms,
                     "launches_timed": args.steps},
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    return line


def run_learned(args, wl, rank, world, local):
    """Learned trial filter against plain GOM on the same GPU: both start from
    the same population; plain runs 200 generations, whose final best fitness
    is the target; the learned run logs 50 plain generations, trains its MLP,
    then runs with the filter until the target (at most 400 generations in
    all).  Times are wall clock with the device synchronised, training
    included."""
    import torch

    from paper_2203_08680_gb300 import gom
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    g = I.torus2d(1000)
    p, seed, warm, total = 256, SEED + rank, 50, 200

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    A = gom.Population(g, p, seed, stream=stream)
    (stA, nA), tA = timed(lambda: A.generation(total))
    target = stA[-1]["best_fitness"]
    trials_plain = p * A.m * nA

    B = gom.Population(g, p, seed, stream=stream, fos=A.fos)
    cap = 1 << 20
    ws = torch.empty(gom.gom_filter_workspace_bytes(B.ctx, cap) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    gom.gom_filter_attach(B.ctx, ws, cap)
    gom.gom_set_option(B.ctx, gom.GOM_OPT_FILTER_LABEL, args.learn_label)
    gom.gom_filter_set_mode(B.ctx, 1)
    (stB1, n1), t1 = timed(lambda: B.generation(warm, target))
    tr, t2 = timed(lambda: gom.gom_filter_train(B.ctx, epochs=args.learn_epochs, learning_rate=0.02, pos_weight=1.0,
                                                target_recall=args.learn_recall))
    gom.gom_filter_configure(B.ctx, tr["threshold"], args.learn_recall, args.learn_min_recall)
    gom.gom_filter_set_mode(B.ctx, 2)
    reached, n2, t3, best = bool(stB1 and stB1[-1]["reached_target"]), 0, 0.0, stB1[-1]["best_fitness"]
    while not reached and n1 + n2 < 2 * total:
        (st, n), dt = timed(lambda: B.generation(25, target))
        n2 += n
        t3 += dt
        best = st[-1]["best_fitness"]
        reached = bool(st[-1]["reached_target"])
    fs = gom.gom_filter_stats(B.ctx)
    learned_s = t1 + t2 + t3
    line = {
        "metric": "time to target cut (learned trial filter vs plain GOM, same GPU)", "value": learned_s * 1e3,
        "unit": "ms", "n_gpus": world, "steps": n1 + n2, "warmup": 0, "ms_per_step": learned_s * 1e3 / max(n1 + n2, 1),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": wl, "description": LEARNED_WORKLOADS[wl], "population": p, "elements": A.m,
                   "target": target, "target_source": f"plain GOM best fitness at generation {total}",
                   "parallelism": f"replicas{world}"},
        "plain": {"ms": tA * 1e3, "generations": nA, "trials_per_sec": trials_plain / tA},
        "learned": {"reached": reached, "best": best, "generations_logged": n1, "generations_filtered": n2,
                    "log_ms": t1 * 1e3, "train_ms": t2 * 1e3, "filtered_ms": t3 * 1e3,
                    "ms_per_filtered_generation": t3 * 1e3 / max(n2, 1), "train": tr, "filter": fs},
        "speedup_vs_plain": tA / learned_s if reached else None,
        "gpu_launches": None,
    }
    return line


def time_to_target(args, g, p, seed, stream, wl, fos=None, fi=False):
    import torch

    from paper_2203_08680_gb300 import gom
    tw = g.total_weight()
    target = int(math.ceil(0.999 * tw))
    P2 = gom.Population(g, p, seed, fos=fos, stream=stream, forced_improvement=fi or None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats, nrun = P2.generation(args.ttt_gens, target)
    e1.record(stream)
    torch.cuda.synchronize()
    ttt = {"target": target, "forced_improvement": fi, "closed_form_optimum": tw if wl.startswith("torus") else None,
           "reached": bool(stats and stats[-1]["reached_target"]), "generations": nrun,
           "best": stats[-1]["best_fitness"] if stats else None, "ms": e0.elapsed_time(e1),
           "max_generations": args.ttt_gens}
    del P2
    return ttt


def linkage_tree_time_to_target(args, g, seed, stream, bound, fi=False):
    """Time to target with the paper's linkage model: the bounded fixed
    linkage tree (UPGMA on the weights, Sec. 4.1) at `bound` variables, one
    population of --lt-pop individuals, up to --lt-gens generations.  The
    set-up (tree, colouring, initial population) is timed apart."""
    import torch

    from paper_2203_08680_gb300 import gom
    tw = g.total_weight()
    target = int(math.ceil(0.999 * tw))
    t0 = time.perf_counter()
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bound)
    P = gom.Population(g, args.lt_pop, seed, fos=fos, stream=stream, forced_improvement=fi or None)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats, nrun = P.generation(args.lt_gens, target)
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"fos": f"bounded linkage tree, bound {bound}", "forced_improvement": fi, "population": args.lt_pop,
           "colours": P.k,
           "target": target, "reached": bool(stats and stats[-1]["reached_target"]), "generations": nrun,
           "best": stats[-1]["best_fitness"] if stats else None, "ms": e0.elapsed_time(e1),
           "setup_ms": setup_s * 1e3, "max_generations": args.lt_gens}
    del P
    return out


def ims_time_to_target(args, g, seed, stream, bflt=0, base=None, c=None, chunk=1024):
    """Time to target of the Interleaved Multi-start Scheme (Sec. 6.3):
    populations of base_pop * 2^i individuals (up to 1024), P_i one generation
    per c of P_{i-1}, advanced in batched calls of `chunk` P_0 generations
    until a population reaches the target or the time budget runs out; the
    neighbourhood FOS, or the bounded linkage tree with bound `bflt`."""
    import torch

    from paper_2203_08680_gb300 import gom
    base = args.ims_base if base is None else base
    c = args.ims_c if c is None else c
    tw = g.total_weight()
    target = int(math.ceil(0.999 * tw))
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bflt) if bflt else gom.gom_build_fos(g)
    gom.gom_color_fos(g, fos)
    nb = gom.gom_ims_workspace_bytes(g, fos, base, 1024)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    ims = gom.gom_ims_create(g, fos, base, c, 1024, seed, ws, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    best, res = None, None
    while True:
        res = gom.gom_ims_run(ims, chunk, target)
        best = res["best_fitness"] if best is None else max(best, res["best_fitness"])
        if res["reached"] or time.perf_counter() - t0 > args.ims_seconds:
            break
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"fos": f"bounded linkage tree, bound {bflt}" if bflt else "neighbourhood", "target": target,
           "closed_form_optimum": tw, "reached": bool(res["reached"]), "ms": e0.elapsed_time(e1),
           "p0_generations": res["steps"], "p0_generations_per_call": chunk, "best": best, "base_pop": base,
           "c": c, "max_pop": 1024, "populations": gom.gom_ims_num_populations(ims)}
    if res["reached"]:
        out.update(reached_step=res["reached_step"], reached_population=res["reached_population"],
                   reached_generation=res["reached_generation"])
    del ims
    return out


def end_to_end(args, g, p, seed, stream, dev, world, ex, m, trials_per_step, bflt=0):
    """End to end through the C ABI from host buffers: FOS, colouring, upload,
    generations with host statistics, population and fitness back to host."""
    import torch

    from paper_2203_08680_gb300 import gom
    torch.cuda.synchronize()
    marks = [("start", time.perf_counter())]
    G = gom.Graph(g)
    fos = gom.gom_build_fos(G, gom.GOM_FOS_BFLT, bflt) if bflt else gom.gom_build_fos(G)
    marks.append(("fos_ms", time.perf_counter()))
    gom.gom_color_fos(G, fos)
    marks.append(("colouring_ms", time.perf_counter()))
    nbytes = gom.gom_workspace_bytes(G, fos, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    marks.append(("workspace_ms", time.perf_counter()))
    # element tables built on the host, uploads, initial population, fitness, elitist (synchronous)
    ctx = gom.gom_init_population(G, fos, p, seed, ws, nbytes, stream)
    marks.append(("tables_upload_init_ms", time.perf_counter()))
    est, _ = gom.gom_generation(ctx, args.steps, gom.INT64_MAX, True)
    torch.cuda.synchronize()
    marks.append(("generations_ms", time.perf_counter()))
    dpop = torch.empty((p, g.n), dtype=torch.uint8, device=dev)
    dfit = torch.empty(p, dtype=torch.int64, device=dev)
    gom.gom_get_population(ctx, dpop, dfit, True)
    hpop = torch.empty((p, g.n), dtype=torch.uint8, pin_memory=True)
    hfit = torch.empty(p, dtype=torch.int64, pin_memory=True)
    hpop.copy_(dpop, non_blocking=True)
    hfit.copy_(dfit, non_blocking=True)
    torch.cuda.synchronize()
    marks.append(("export_download_ms", time.perf_counter()))
    e2e_s = marks[-1][1] - marks[0][1]
    breakdown = {name: 1e3 * (t - marks[i][1]) for i, (name, t) in enumerate(marks[1:])}
    e2e_s = dist_max(e2e_s, world)
    h2d = (G.row_ptr.nbytes + G.col.nbytes + G.weight.nbytes + ex["elem_ptr"].nbytes // 2 +
           ex["elem_vars"].nbytes + 8 * (m + 1) + 8 * int(np.diff(G.row_ptr).sum()) + 2 * (len(ex["elem_vars"]) + m))
    d2h = 64 * args.steps + p * g.n + 8 * p
    del ctx, ws
    return {"value": trials_per_step * args.steps * world / e2e_s, "unit": "trials/s",
            "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
            "generations": args.steps, "total_ms": 1e3 * e2e_s, "breakdown": breakdown}


def finish(args, wl, rank, world, desc, p, m, k, value, total_ms, dom, mix, ttt, e2e, launches_per_step, clk,
           cpu, persistent):
    peak, peak_kind = peaks()
    achieved = dom["bytes_per_launch"] / (dom["avg_ms"] / 1e3) / 1e9 if dom["launches"] else None
    line = {
        "metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": wl, "description": desc, "population": p, "elements": m, "colours": k,
                   "path": "persistent" if persistent else "graph",
                   "l2": "flushed between timed generations (2x L2 buffer write)",
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "kernel": dom["kernel"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": profiled_traffic(wl, dom["kernel"]),
                     "peak_source": peak_kind, "algorithmic_bytes_per_launch": dom["bytes_per_launch"],
                     "avg_launch_ms": dom["avg_ms"], "launches_timed": dom["launches"]},
        "mix_kernel": mix,
        "time_to_target": ttt,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gom", choices=["gom", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the torus100, batch256 and learned1000 keys")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(LEARNED_WORKLOADS))
    ap.add_argument("--learn-recall", type=float, default=0.7, help="learned filter: recall target")
    ap.add_argument("--learn-min-recall", type=float, default=0.35, help="learned filter: self-disable recall")
    ap.add_argument("--learn-label", type=int, default=1, choices=[0, 1],
                    help="learned filter: useful = 0 an accepted trial, 1 an improving trial")
    ap.add_argument("--learn-epochs", type=int, default=25, help="learned filter: training epochs (full batch)")
    ap.add_argument("--pop", type=int, default=0)
    ap.add_argument("--ttt-gens", type=int, default=500)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-count", type=int, default=256,
                    help="batch workloads: the first N instances of the mix (a smaller case for profiling)")
    ap.add_argument("--lt-pop", type=int, default=1024, help="linkage-tree time-to-target runs: population")
    ap.add_argument("--lt-gens", type=int, default=400, help="linkage-tree time-to-target runs: generation cap")
    ap.add_argument("--ims-base", type=int, default=16, help="IMS base population (time-to-target run)")
    ap.add_argument("--ims-c", type=int, default=4, help="IMS generation ratio c")
    ap.add_argument("--ims-seconds", type=float, default=20.0, help="IMS time-to-target budget")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-target run")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run")
    ap.add_argument("--path", default="auto", choices=["auto", "persistent", "graph"])
    ap.add_argument("--bitsliced", default="auto", choices=["auto", "on", "off"],
                    help="mixing on bit-planes (GOM_OPT_BITSLICED) or per lane; auto = the library's default")
    ap.add_argument("--mix-steps", type=int, default=50,
                    help="generations timed per mixing launch on the graph path (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, args.workload, rank, world)
    elif args.workload in BATCH_WORKLOADS:
        line = run_batch(args, args.workload, rank, world, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
    elif args.workload in LEARNED_WORKLOADS:
        line = run_learned(args, args.workload, rank, world, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
    else:
        line = run_gpu(args, args.workload, rank, world, local)
        if args.workload == DEFAULT_WORKLOAD and not args.no_extras:
            line["extras"] = extras(args, rank, world, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
