#!/usr/bin/env python
"""Throughput of the tropical contraction hot path on GB300.

Workload (one step): B instances of the 24x24 open square-lattice Ising spin
glass, J ~ N(0, 1) and h ~ N(0, 0.1^2) as float32, contracted along one greedy
order (seeded randomized greedy, 16384 restarts, host-side and untimed); for each
instance the step computes E_min (forward contraction keeping checkpoints) and
the ground state sigma* (argmax traceback).  Couplings are resident in HBM
before the timed region.  Metric: instances/s over all ranks.

The default line also carries sub-records measured in the same run: the
max-plus GEMM on the two step shapes that carry the 3-regular N = 200
contraction, and the 2048-instance mixed-size +-J batch (E_min + exact count)
against its one-by-one paths.  cpu_baseline is the CPU oracle on all host
cores (one process per core, each on a bounded prefix of its own instance).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
  python bench.py --impl reference ...   # the CPU oracle, a bounded sample per step
  python bench.py --workload mixed|cubic|max2sat|sample|chimera   # other workloads (one JSON line each)

Multi-GPU (torchrun): every rank contracts its own instances (weak scaling, no
data exchange); the slowest rank's time is reported.
"""
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

METRIC = "tropical Gop/s & % of FP32/INT32 peak; instances/s for (E, σ*, count)"
L = 24
FIELD_SIGMA = 0.1
ORDER_SEED, ORDER_RESTARTS = 1, 16384
WORKLOAD = (f"square{L}x{L} open Ising glass, J~N(0,1) fp32, h~N(0,0.1^2) fp32, "
            f"greedy order (seed {ORDER_SEED}, {ORDER_RESTARTS} restarts); per instance E_min "
            f"+ sigma* (checkpointed forward + argmax traceback), batched over the step's "
            f"instances")
KIND_BOUND = {"gate": "hbm", "transpose": "hbm", "leaves": "hbm", "trace": "latency",
              "gemm": "alu", "other": "hbm", "chain": "hbm"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=48)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--L", type=int, default=24, help="lattice side (profiling runs only)")
    ap.add_argument("--mode", default="config", choices=["config", "energy"],
                    help="config: E_min + sigma* (the workload); energy: E_min only (profiling)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the GEMM and mixed-batch sub-records of the default run")
    ap.add_argument("--restarts", type=int, default=ORDER_RESTARTS,
                    help="greedy restarts of the (untimed) order search")
    ap.add_argument("--quiet", action="store_true", help="print only value and kernel shares")
    ap.add_argument("--workload", default="square24",
                    choices=["square24", "mixed", "cubic", "max2sat", "sample", "chimera"],
                    help="mixed: batch of +-J lattices with L uniform in 8..20, E_min + count")
    ap.add_argument("--mixed-n", type=int, default=2048, help="instances of the mixed batch")
    ap.add_argument("--chimera-L", type=int, default=8,
                    help="chimera workload: L x L unit cells (8: 512 spins)")
    ap.add_argument("--one-by-one-only", action="store_true",
                    help="mixed workload: time only the one-by-one sample (run by bench.py "
                         "itself with TN_NO_GRAPH=1 for the plain unbatched path)")
    ap.add_argument("--gemm", action="store_true",
                    help="max-plus GEMM microbenchmark (FP32 and INT32) instead of the workload")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tops(sm_mhz, sms=None):
    # SMs x 128 FP32 lanes x clock: one lane-instruction per lane per clock
    # (the device's SM count unless given)
    if sms is None:
        sms = sm_count()
    return sms * 128 * sm_mhz * 1e6 * 1e-12


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


CHAIN_SOURCES = ("kernels.cu", "chain_dev.cuh", "jit.cpp")   # define every chain kernel


def sources_hash():
    h = hashlib.sha256()
    for f in CHAIN_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2008_06888_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kind):
    """DRAM bytes per launch from the committed ncu summary, if the kernel sources still match."""
    path = os.path.join(ROOT, "profiles", f"{kind}_kernel_square24.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].rsplit(": ", 1)
            vals[k.strip()] = v.strip()
    if vals.get("chain sources sha256[:16]") != sources_hash():
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def make_instances(rank, batch, side=L):
    import instances as I
    return [I.square_lattice(side, coupling="gauss", field_sigma=FIELD_SIGMA, seed=1000 * rank + k)
            for k in range(batch)]


# ---- CPU oracle baseline: the oracle as it stands (numpy float64 variable
# elimination, row-by-row order, sigma* by its argmax backtracking), one
# single-threaded process per host core, each on its own instance.

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def elimination_work(inst, order):
    """Cumulative table entries of the oracle's eliminations along ``order`` (the
    union scope of each bucket, q^|scope| entries): its work is proportional to
    them, which converts a timed prefix of eliminations into a fraction of an
    instance."""
    q = inst["q"]
    scopes = [set(e) for e in inst["edges"].tolist()] + [{i} for i in range(inst["n"])]
    out, tot = [], 0.0
    for v in order:
        bucket = [s for s in scopes if v in s]
        scopes = [s for s in scopes if v not in s]
        u = set().union(*bucket)
        tot += float(q) ** len(u)
        out.append(tot)
        scopes.append(u - {v})
    return out


def _oracle_prefix(job):
    """Worker: the oracle on the first k eliminations of instance `seed` (seconds)."""
    seed, k = job
    import instances as I
    import oracle as O
    inst = I.square_lattice(L, coupling="gauss", field_sigma=FIELD_SIGMA, seed=seed)
    t0 = time.perf_counter()
    O.solve(inst, order=I.square_sweep_order(L), count=False, config=True, max_eliminations=k)
    return time.perf_counter() - t0


class OracleBaseline:
    """Each step: every host core runs the oracle on the first k eliminations of
    its own 24x24 instance; the instances-worth of work done is the sum of the
    prefixes' shares of a whole instance's table entries (elimination_work),
    and the step's time is the wall time until the last core finishes."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        import instances as I
        self.cores = cores or host_cores()
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        # spawn: no fork of a process that may hold a CUDA context
        self.pool = mp.get_context("spawn").Pool(self.cores)
        inst = I.square_lattice(L, coupling="gauss", field_sigma=FIELD_SIGMA, seed=0)
        self.work = elimination_work(inst, I.square_sweep_order(L))
        self.k = L + 1

    def calibrate(self, budget_s):
        """Choose the prefix length so that a step (every core busy, sharing the
        host's memory bandwidth) takes about budget_s of wall time."""
        k0 = L + 5
        jobs = [(1 + c, k0) for c in range(self.cores)]
        t0 = max(self.pool.map(_oracle_prefix, jobs, chunksize=1))
        per = t0 / self.work[k0 - 1]
        k = k0
        while k < len(self.work) and self.work[k] * per < budget_s:
            k += 1
        self.k = k
        return k

    def step(self, base_seed=0):
        jobs = [(base_seed + c, self.k) for c in range(self.cores)]
        t0 = time.perf_counter()
        times = self.pool.map(_oracle_prefix, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        frac = self.work[self.k - 1] / self.work[-1]
        return self.cores * frac, wall, max(times)

    def close(self):
        self.pool.close()
        self.pool.join()

    def describe(self):
        frac = self.work[self.k - 1] / self.work[-1]
        return (f"CPU oracle (numpy float64 variable elimination, row-by-row order, sigma* by "
                f"argmax backtracking) on {self.cores} host cores, one single-threaded process "
                f"per core, each on its own instance: the first {self.k} of {L * L} "
                f"eliminations, {100 * frac:.2f}% of an instance's table entries (work is "
                f"proportional to them); value = instances-worth of entries / wall time")


def cpu_baseline(budget_s=10.0):
    ob = OracleBaseline()
    try:
        ob.calibrate(budget_s)
        inst_done, wall, _ = ob.step(base_seed=100)
        return {"value": inst_done / wall, "unit": "instances/s", "cores": ob.cores,
                "kind": "oracle", "sample": ob.describe() + f" ({wall:.1f} s wall)"}
    finally:
        ob.close()


def workload_config(batch, world):
    return {"workload": WORKLOAD, "global_batch": batch * world,
            "instances_per_step_per_gpu": batch,
            "l2": "flushed between timed steps (256 MB write)"}


def run_reference(args):
    """The oracle on the host cores, same metric, unit and config as the native arm;
    each step a bounded sample (see OracleBaseline) sized to a few seconds."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    ob = OracleBaseline()
    try:
        ob.calibrate(5.0)
        done, walls = 0.0, []
        for i in range(args.warmup + args.steps):
            d, wall, _ = ob.step(base_seed=1000 + i * ob.cores)
            if i >= args.warmup:
                done += d
                walls.append(wall)
        desc = ob.describe()
    finally:
        ob.close()
    val = done / sum(walls)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "instances/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(walls)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.batch, world),
            "cpu_baseline": {"value": val, "unit": "instances/s", "cores": ob.cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": "instances/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


GEMM_SHAPES = [(1, 4096, 4096, 4096), (64, 512, 512, 512), (16, 1024, 1024, 256),
               (8, 131072, 1024, 512), (32, 2048, 256, 16384)]
# the two steps that carry 99% of the multiply-adds of the 3-regular N = 200
# contraction (greedy order): (batch, M, N, K)
GEMM_3REG = [(8, 131072, 1024, 512), (32, 2048, 256, 16384)]


def sm_count():
    """SMs of the current device (152 on a GB300; that figure without a device)."""
    import torch
    if not torch.cuda.is_available():
        return 152
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def measure_gemm(shapes, reps=5):
    """Max-plus GEMM through tn_maxplus_gemm, FP32 and INT32, CUDA events."""
    import torch
    from paper_2008_06888_gb300 import binding as B
    pk, how = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    sms = sm_count()
    # non-tensor FP32 peak, an FMA counted as 2 ops: SMs x 128 lanes x 2 x clock
    peak_ops = sms * 128 * 2 * sm_max * 1e6
    issue_peak = sms * 128 * sm_max * 1e6
    out = {}
    for dt in (torch.float32, torch.int32):
        for (bt, M, N, K) in shapes:
            if dt == torch.float32:
                A = torch.randn(bt, M, K, device="cuda")
                Bm = torch.randn(bt, K, N, device="cuda")
            else:
                A = torch.randint(-100, 100, (bt, M, K), device="cuda", dtype=torch.int32)
                Bm = torch.randint(-100, 100, (bt, K, N), device="cuda", dtype=torch.int32)
            C = torch.empty(bt, M, N, device="cuda", dtype=dt)
            for _ in range(3):
                B.tn_maxplus_gemm(A, Bm, C)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                B.tn_maxplus_gemm(A, Bm, C)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            macs = bt * M * N * K
            ops = 2 * macs / (ms * 1e-3)
            # ALU instructions one multiply-add needs: an add and half a three-input
            # max (FP32), or one fused add-max (INT32)
            ipm = 1.5 if dt == torch.float32 else 1.0
            out[f"{str(dt).split('.')[-1]}_{bt}x{M}x{N}x{K}"] = {
                "ms": ms, "tropical_Top_s": ops / 1e12, "T_MAC_s": macs / (ms * 1e-3) / 1e12,
                "frac_of_fp32_nontensor_peak": ops / peak_ops,
                "alu_issue_frac": ipm * macs / (ms * 1e-3) / issue_peak}
            del A, Bm, C
    torch.cuda.empty_cache()
    return out, {"peak_ops_per_s": peak_ops,
                 "peak": f"{sms} SMs x 128 FP32 lanes x 2 (FMA = 2 ops) x max SM clock",
                 "issue_peak_lane_instr_per_s": issue_peak,
                 "issue_peak": f"{sms} SMs x 128 lanes x max SM clock (one ALU instruction per "
                               f"lane per clock); alu_issue_frac counts the ALU instructions "
                               f"the multiply-adds need"}


def run_gemm(args):
    """Max-plus GEMM: square 4096^3, batched shapes and the dominant step shapes of
    the 3-regular N = 200 contraction."""
    import torch
    torch.cuda.set_device(0)
    clocks = Clocks(0)
    clocks.start()
    out, meta = measure_gemm(GEMM_SHAPES)
    clk = clocks.stop()
    print(json.dumps(dict({"gemm": out, "clocks": clk}, **meta)), flush=True)


def measure_mixed(n_inst, steps, warmup, plain=True):
    """Mixed batch of +-J square lattices (L uniform in 8..20, base seed 2026), E_min and
    exact count each, through tn_batch_run (grouped batches), against the same
    instances one by one (graph-replayed, and the plain path in a child process)."""
    import torch
    import instances as I
    import paper_2008_06888_gb300 as P
    from paper_2008_06888_gb300 import binding as B
    insts = I.mixed_square_batch(n_inst, Lmin=8, Lmax=20, seed=2026)
    sgs = [P.SpinGlass(x, order="sweep",
                       seq=I.square_sweep_order(int(round(np.sqrt(x["n"]))))) for x in insts]
    ctxs = [s.ctx for s in sgs]
    sub = list(range(0, len(insts), max(1, len(insts) // 128)))

    def one_by_one():
        for k in sub[:4]:
            sgs[k].count(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in sub:
            sgs[k].count(3)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / len(sub)

    try:
        for _ in range(warmup):
            st, E, counts, status = B.tn_batch_run(ctxs, limbs_per=4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            st, E, counts, status = B.tn_batch_run(ctxs, limbs_per=4)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        # kernel shares of one batched pass (events around every launch)
        for c in ctxs:
            B.tn_profile_reset(c)
            B.tn_set_profiling(c, True)
        B.tn_batch_run(ctxs, limbs_per=4)
        torch.cuda.synchronize()
        prof = {k: {"launches": 0, "ms": 0.0, "bytes": 0.0, "macs": 0.0} for k in B.KIND_NAMES}
        for c in ctxs:
            for i, k in enumerate(B.KIND_NAMES):
                v = B.tn_profile_get(c, i)
                for f in prof[k]:
                    prof[k][f] += v[f]
            B.tn_set_profiling(c, False)
        dt1 = one_by_one()
        ok = int(np.sum(status == 0))
    finally:
        for s_ in sgs:
            s_.close()
        torch.cuda.empty_cache()
    total_ms = sum(v["ms"] for v in prof.values())
    plain_s = None
    if plain:
        # the plain path (every kernel launched directly, no graphs): a fresh
        # process, since graph use is fixed per process
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", "mixed",
                                "--mixed-n", str(n_inst), "--one-by-one-only"],
                               env=dict(os.environ, TN_NO_GRAPH="1"), capture_output=True,
                               text=True, timeout=600)
            lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
            if r.returncode == 0 and lines:
                plain_s = json.loads(lines[-1])["one_by_one_s"]
        except Exception:
            plain_s = None
    return {
        "value": len(insts) / dt, "unit": "instances/s",
        "workload": f"{len(insts)} +-J square lattices, L uniform in 8..20 (base seed 2026), "
                    f"row-by-row order, E_min + exact count (3 primes + witness), grouped "
                    f"batches through tn_batch_run",
        "ms_per_batch": dt * 1e3, "steps": steps, "instances_ok": ok,
        "unbatched_instances_per_s": 1.0 / dt1, "unbatched_sample": len(sub),
        "batched_over_unbatched": (len(insts) / dt) * dt1,
        "unbatched_plain_instances_per_s": None if plain_s is None else 1.0 / plain_s,
        "batched_over_unbatched_plain": None if plain_s is None else (len(insts) / dt) * plain_s,
        "roofline": roofline_of(prof, None),
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"],
                        "share": v["ms"] / max(total_ms, 1e-9)} for k, v in prof.items()}}


def run_mixed(args):
    import torch
    torch.cuda.set_device(0)
    if args.one_by_one_only:
        import instances as I
        import paper_2008_06888_gb300 as P
        insts = I.mixed_square_batch(args.mixed_n, Lmin=8, Lmax=20, seed=2026)
        sub = list(range(0, len(insts), max(1, len(insts) // 128)))
        sgs = {k: P.SpinGlass(insts[k], order="sweep",
                              seq=I.square_sweep_order(int(round(np.sqrt(insts[k]["n"])))))
               for k in sub}
        for k in sub[:4]:
            sgs[k].count(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in sub:
            sgs[k].count(3)
        torch.cuda.synchronize()
        print(json.dumps({"one_by_one_s": (time.perf_counter() - t0) / len(sub),
                          "sample": len(sub)}), flush=True)
        return
    clocks = Clocks(0)
    clocks.start()
    rec = measure_mixed(args.mixed_n, args.steps, args.warmup)
    clk = clocks.stop()
    rec = dict({"metric": METRIC}, **rec)
    rec["clocks"] = clk
    print(json.dumps(rec), flush=True)


def roofline_of(prof, clk):
    """Roofline entry of the kernel kind with the most device time in ``prof``."""
    pk, how = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    launches = max(d["launches"], 1)
    avg_ms = d["ms"] / launches
    if KIND_BOUND[dom] == "alu":
        achieved = 2 * d["macs"] / launches / (avg_ms / 1e3) / 1e12
        peak = alu_peak_tops(pk.get("sm_max_mhz", 2070.0))
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": "SMs x 128 lanes x max clock (one lane-op per clock)"}
    achieved = d["bytes"] / launches / (avg_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": dom,
            "peak_source": how, "bytes_per_launch": d["bytes"] / launches,
            "avg_launch_ms": avg_ms}


def run_ensemble(args):
    """Ensembles on one plan per graph, batched over coupling sets.

    cubic:   6x6x6 open cubic lattice (216 spins, 540 bonds, one greedy order);
             value = Gaussian J, E_min + sigma* per instance (tn_config_batch);
             also +-J E_min + exact count (tn_count_batch) on the same plan.
    max2sat: Max-2-SAT on random 3-regular graphs, N = 160 variables, 240
             clauses with random literal signs; 8 graphs (one greedy order each)
             x B sign patterns per graph; value = min violated clauses + exact
             number of optimal assignments per instance (tn_count_batch); also
             +-J Ising spin glasses on the same graphs and orders, same mode.
    Graphs run one after another (their batch arenas are freed in between);
    the reported time is the sum of the graphs' timed steps.
    """
    import torch
    import instances as I
    import paper_2008_06888_gb300 as P
    from paper_2008_06888_gb300 import binding as B
    torch.cuda.set_device(0)
    rng = np.random.default_rng(2008)

    if args.workload == "cubic":
        # arenas per instance at peak 2^30: ~40 GB with checkpoints, ~77 GB counting
        Bsz = args.batch if args.batch != 48 else 4
        Bc = max(1, Bsz // 2)
        n_units = 1

        def make_unit(g):
            base = I.cubic_lattice(6, coupling="gauss", seed=1)
            sg = P.SpinGlass(base, order="greedy", seed=ORDER_SEED, restarts=4096)
            Jg = np.stack([I.cubic_lattice(6, coupling="gauss", seed=100 + k)["J"]
                           for k in range(Bsz)])
            Jp = np.stack([I.cubic_lattice(6, coupling="pm1", seed=100 + k)["J"]
                           for k in range(Bc)])
            return [sg], (sg, Jg, None, "config"), (sg, Jp, None, "count")

        desc = (f"cubic 6x6x6 open Ising glass (216 spins, 540 bonds), greedy order (seed "
                f"{ORDER_SEED}, 4096 restarts); value: J~N(0,1) fp32, h=0, E_min + sigma* per "
                f"instance, batch {Bsz}; other: +-J, E_min + exact count (3 primes + witness), "
                f"batch {Bc}")
        other_key = "pm_count"
    else:
        Bsz = args.batch if args.batch != 48 else 16
        n_units = 8

        def make_unit(g):
            sat0 = I.max2sat_regular3(160, seed=500 + g)
            sats = [dict(sat0, clauses=np.where(rng.integers(0, 2, sat0["clauses"].shape) == 1,
                                                -np.abs(sat0["clauses"]),
                                                np.abs(sat0["clauses"])).astype(np.int32))
                    for _ in range(Bsz)]
            ms_ = P.Max2SAT(sats[0], order="greedy", seed=ORDER_SEED, restarts=1024)
            cp = [P.Max2SAT.couplings(x) for x in sats]
            edges = cp[0][0]
            ising = dict(n=160, q=2, edges=edges, J=np.ones(len(edges), np.float32), h=None)
            sg = P.SpinGlass(ising, order="greedy", seed=ORDER_SEED, restarts=1024)
            Jp = np.where(rng.integers(0, 2, (Bsz, len(edges))) == 1, -1.0, 1.0).astype(np.float32)
            return ([ms_, sg], (ms_, np.stack([c[1] for c in cp]), np.stack([c[2] for c in cp]),
                                "count"), (sg, Jp, None, "count"))

        desc = ("Max-2-SAT on random 3-regular graphs (pairing model), N = 160 variables, 240 "
                "clauses, literal signs uniform; 8 graphs x " + str(Bsz) + " sign patterns, one "
                "greedy order per graph (seed 1, 1024 restarts); per instance the minimum "
                "number of violated clauses and the exact number of optimal assignments; "
                "other: +-J spin glasses on the same graphs, same mode")
        other_key = "pm_ising"

    def run(w):
        obj, J, h, mode = w
        if mode == "config":
            B.tn_config_batch(obj.ctx, J, h, obj.n, want_sigma=True)
        else:
            obj.count_batch(J, h, 3, limbs_per=4)

    def timed(w, profile=False):
        obj = w[0]
        B.tn_profile_reset(obj.ctx)
        B.tn_set_profiling(obj.ctx, profile)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run(w)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        prof = {k: B.tn_profile_get(obj.ctx, i) for i, k in enumerate(B.KIND_NAMES)}
        B.tn_set_profiling(obj.ctx, False)
        return dt, prof

    prof = {k: {"launches": 0, "ms": 0.0, "bytes": 0.0, "macs": 0.0} for k in B.KIND_NAMES}
    t_main = t_other = 0.0
    n_main = n_other = 0
    peaks_l2 = []
    unb = None
    clocks = Clocks(0)
    clocks.start()
    for g in range(n_units):
        objs, wm, wo = make_unit(g)
        peaks_l2.append(round(wm[0].log2_peak, 2))
        for _ in range(args.warmup):
            run(wm)
            run(wo)
        dt, _ = timed(wm)
        t_main += dt
        n_main += wm[1].shape[0] * args.steps
        dt, _ = timed(wo)
        t_other += dt
        n_other += wo[1].shape[0] * args.steps
        _, pr = timed(wm, profile=True)
        for k, v in pr.items():
            for f in prof[k]:
                prof[k][f] += v[f]
        if g == 0:
            # one by one: instances of the first graph through the unbatched call
            obj, J, h, mode = wm
            K1 = min(4, J.shape[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(K1):
                B.tn_set_couplings(obj.ctx, J[k], None if h is None else h[k])
                if mode == "config":
                    B.tn_config(obj.ctx, obj.n)
                else:
                    obj.count(3)
            torch.cuda.synchronize()
            unb = K1 / (time.perf_counter() - t0)
        for o in objs:
            o.close()
    clk = clocks.stop()
    total_ms = sum(v["ms"] for v in prof.values())
    print(json.dumps({
        "metric": METRIC, "value": n_main / t_main, "unit": "instances/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_main * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.workload == "cubic" else "int32",
        "data": "synthetic",
        "config": {"workload": desc, "instances_per_step": n_main // args.steps,
                   "log2_peak_elements": peaks_l2},
        other_key: {"value": n_other / t_other, "unit": "instances/s",
                    "instances_per_step": n_other // args.steps},
        "unbatched_instances_per_s": unb,
        "roofline": roofline_of(prof, clk),
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"] / args.steps,
                        "share": v["ms"] / max(total_ms, 1e-9)} for k, v in prof.items()},
        "gpu_launches": int(sum(v["launches"] for v in prof.values())),
        "cpu_baseline": None, "clocks": clk}), flush=True)


def run_chimera(args):
    """Chimera L x L K_{4,4} cells (L = 8: 512 spins, 1472 couplers), +-J, h = 0, cell-row
    order: E_min and the exact ground-state count with 3 primes' range (at L = 8 the 61-bit
    planes would need ~1.1 TB, so the count runs in 31-bit passes: 6 + a witness), and the
    residual entropy ln(count) / N.  Instances one after another (seeds 1..steps)."""
    import torch
    import instances as I
    import paper_2008_06888_gb300 as P
    from paper_2008_06888_gb300 import binding as B
    torch.cuda.set_device(0)
    L8 = args.chimera_L
    seq = I.chimera_sweep_order(L8)
    rows = []
    clocks = Clocks(0)
    clocks.start()
    t_all = 0.0
    for k in range(args.warmup + args.steps):
        inst = I.chimera(L8, coupling="pm1", seed=1 + k)
        sg = P.SpinGlass(inst, order="sweep", seq=seq)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E = sg.energy()
        t1 = time.perf_counter()
        c, ln, E2 = sg.count(3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        sg.close()
        if k >= args.warmup:
            t_all += t2 - t0
            rows.append({"seed": 1 + k, "E_min": E, "count": str(c), "entropy_per_spin": ln / inst["n"],
                         "energy_s": t1 - t0, "count_s": t2 - t1, "E_count_pass": E2})
    clk = clocks.stop()
    n = len(rows)
    print(json.dumps({
        "metric": METRIC, "value": n / t_all, "unit": "instances/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(n, 1),
        "higher_is_better": True, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"chimera {L8}x{L8} K44 cells ({8 * L8 * L8} spins), +-J, h=0, "
                               f"cell-row order; E_min + exact count (range of 3 61-bit "
                               f"primes; in 31-bit passes when their planes do not fit) per "
                               f"instance"},
        "instances": rows, "clocks": clk}), flush=True)


def run_sample(args):
    """Uniform ground-state samples (tn_sample) of a degenerate 16x16 +-J lattice:
    256 steps, each one batched count of 2 x 16 pinned instances."""
    import torch
    import instances as I
    import paper_2008_06888_gb300 as P
    torch.cuda.set_device(0)
    inst = I.square_lattice(16, coupling="pm1", seed=3)
    sg = P.SpinGlass(inst, order="greedy", seed=ORDER_SEED, restarts=1024)
    count, ln, E = sg.count(3)
    sg.sample(2, seed=0)            # builds the pinned program and its graphs
    S = 16
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(max(1, args.steps)):
        sig = sg.sample(S, seed=100 + k)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    distinct = len({row.tobytes() for row in sig})
    print(json.dumps({
        "metric": "uniform ground-state samples/s", "value": S / dt, "unit": "samples/s",
        "n_gpus": 1, "steps": args.steps, "higher_is_better": True, "data": "synthetic",
        "dtype": "int32",
        "config": {"workload": "square16x16 open +-J Ising glass (seed 3), greedy order; "
                               "16 samples per call, each spin fixed by its conditional "
                               "probability from exact counts (3 primes + witness)",
                   "log2_peak_elements": sg.log2_peak},
        "ground_states": str(count), "E_min": E, "distinct_in_last_call": distinct,
        "count_calls_per_call": inst["n"] + 1, "instances_per_count_call": 2 * S,
        "ms_per_call": dt * 1e3}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.gemm:
        return run_gemm(args)
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload in ("cubic", "max2sat"):
        return run_ensemble(args)
    if args.workload == "sample":
        return run_sample(args)
    if args.workload == "chimera":
        return run_chimera(args)
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2008_06888_gb300 as P
    from paper_2008_06888_gb300 import binding as B

    insts = make_instances(rank, args.batch, args.L)
    sg = P.SpinGlass(insts[0], order="greedy", seed=ORDER_SEED, restarts=args.restarts)
    stream = torch.cuda.current_stream(dev)
    sg.set_stream(stream.cuda_stream)
    # couplings of the whole batch, resident in HBM: (B, n_edges) and (B, n_spins)
    Jd = torch.tensor(np.stack([x["J"] for x in insts]), device=dev)
    hd = torch.tensor(np.stack([x["h"] for x in insts]), device=dev)
    Jh = np.stack([x["J"] for x in insts])
    hh = np.stack([x["h"] for x in insts])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)    # > 129 MB L2

    def step():
        # one batched execution of the plan over all B instances
        if args.mode == "energy":
            B.tn_energy_batch(sg.ctx, Jd, hd)
        else:
            B.tn_config_batch(sg.ctx, Jd, hd, sg.n, want_sigma=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def timed(K, profile=False):
        B.tn_profile_reset(sg.ctx)
        B.tn_set_profiling(sg.ctx, profile)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(K):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        prof = {B.KIND_NAMES[k]: B.tn_profile_get(sg.ctx, k) for k in range(len(B.KIND_NAMES))}
        total = B.tn_profile_get(sg.ctx, -1)
        B.tn_set_profiling(sg.ctx, False)
        return ms, prof, total

    clocks = Clocks(local)
    clocks.start()
    ms, _, total = timed(args.steps)
    clk = clocks.stop()
    from paper_2008_06888_gb300 import shard
    ms = shard.max_over_ranks(ms, world, dev)
    inst_total = args.batch * args.steps * world
    value = inst_total / (ms / 1e3)

    # per-kernel durations: the same K steps again with CUDA events around every launch
    ms_p, prof, _ = timed(args.steps, profile=True)

    # end to end through the C ABI with host buffers: couplings in, E and sigma* out
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        E, sigma = B.tn_config_batch(sg.ctx, Jh, hh, sg.n, want_sigma=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = shard.max_over_ranks(e2e_s, world, dev)
    e2e = {"value": inst_total / e2e_s, "unit": "instances/s",
           "h2d_bytes_per_step": args.batch * 4 * (sg.m + sg.n),
           "d2h_bytes_per_step": args.batch * (sg.n + 4)}
    # the one-by-one path on the same instances (unbatched, each through tn_config)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.batch):
        B.tn_set_couplings(sg.ctx, insts[k]["J"], insts[k]["h"])
        B.tn_config(sg.ctx, sg.n)
    torch.cuda.synchronize()
    unbatched = args.batch / (time.perf_counter() - t0)

    pk, how = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    launches = max(d["launches"], 1)
    avg_ms = d["ms"] / launches
    bound = KIND_BOUND[dom]
    sms = sm_count()
    tropical_ops = 2 * total["macs"] / (ms / 1e3)
    if bound == "hbm":
        achieved = d["bytes"] / launches / (avg_ms / 1e3) / 1e9
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(dom),
                "kernel": dom, "peak_source": how,
                "bytes_per_launch": d["bytes"] / launches, "avg_launch_ms": avg_ms}
    else:
        achieved = 2 * d["macs"] / launches / (avg_ms / 1e3) / 1e12
        peak = alu_peak_tops(pk.get("sm_max_mhz", 2070.0))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(dom), "kernel": dom,
                "peak_source": f"{sms} SMs x 128 lanes x max clock (one lane-op per clock)"}
    # the metric's own "% of the FP32 non-tensor peak" for the whole step: tropical
    # ops (a multiply-add = 2) over SMs x 128 lanes x 2 x clock
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = sms * 128 * 2 * sm_max * 1e6
    tropical = {"gop_s": tropical_ops / 1e9, "macs_per_step": total["macs"] / args.steps,
                "frac_of_fp32_nontensor_peak": tropical_ops / fp32_peak,
                "peak_gop_s": fp32_peak / 1e9,
                "peak": f"{sms} SMs x 128 FP32 lanes x 2 (FMA = 2 ops) x {sm_max:.0f} MHz"}
    sg.close()
    del Jd, hd, flush
    torch.cuda.empty_cache()

    # sub-records measured in the same run (rank 0, one GPU): the max-plus GEMM on
    # the 3-regular N = 200 step shapes and the mixed-size batch of +-J lattices
    sub = {}
    if rank == 0 and world == 1 and not args.no_sub and args.L == L:
        g, meta = measure_gemm(GEMM_3REG, reps=3)
        sub["gemm_3regular_steps"] = dict({"shapes": g}, **meta)
        sub["mixed_batch"] = measure_mixed(2048, steps=3, warmup=2)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.L == L:
        cpu = cpu_baseline(10.0)

    if rank == 0:
        cfg = workload_config(args.batch, world)
        if not (args.L == L and args.mode == "config"):
            cfg["workload"] = f"square{args.L}x{args.L} Gaussian, mode {args.mode} (profiling run)"
        line = {"metric": METRIC, "value": value, "unit": "instances/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg,
                "plan": {"log2_peak_elements": sg.log2_peak, "log2_macs": sg.log2_ops},
                "tropical": tropical,
                "unbatched_instances_per_s": unbatched,
                "roofline": roof,
                "kernels": {k: {"launches": v["launches"], "ms": v["ms"],
                                "share": v["ms"] / max(ms_p, 1e-9)} for k, v in prof.items()},
                "gpu_launches": total["launches"],
                "e2e": e2e, "cpu_baseline": cpu, "clocks": clk}
        line.update(sub)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
