"""Benchmark of the GB300 algebraic-signature equi-join.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large] [--impl reference]

One step = one whole signature hash join T = Join(R, S) on device-resident
inputs: signatures of R, build of the signature hash table, probe with every
S key (S signature, table walk, byte-exact verification, output compaction).
The workload is synthetic (workloads.CONFIGS).  Rank 0 prints one JSON line.

Multi-GPU: the join does not shard here (replicas only): every rank runs its
own copy of the workload and the value is the sum of S tuples over ranks
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "probe tuples/s"
UNIT = "tuples/s"
L2_BYTES = 126 * 2 ** 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload_desc(name: str, spec) -> str:
    return (f"{name}: |R|={spec.m:,} x |S|={spec.n:,}, key length {spec.r_len[0]}-{spec.r_len[1]} B "
            f"{spec.alphabet}, {int(spec.frac_copy * 100)}% S copies"
            + (f" (Zipf {spec.zipf_s})" if spec.zipf_s else "")
            + (f", {int(spec.frac_near * 100)}% near-duplicates" if spec.frac_near else "")
            + (f", {spec.dup_frac:.0%} of R keys duplicated {spec.dup[0]}-{spec.dup[1]}x" if spec.dup_frac else ""))


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


# --------------------------------------------------------------------------- reference arm (the CPU oracle)

def cpu_oracle_slice(wl, frac0: float, frac1: float, cores: int) -> tuple[float, int]:
    """The oracle on the host on the rows [frac0, frac1) of both relations (the
    same fraction of R and of S, consecutive rows): signatures of every key of
    both slices, then the exact Grace hash join of the two slices.  Returns
    (seconds, S keys of the slice).  The whole relations are frac 0..1."""
    import oracle
    from workloads import Relation

    def part(rel):
        a, b = int(rel.n * frac0), int(rel.n * frac1)
        return Relation(rel.arena, rel.off[a:b + 1].copy(), rel.ids[a:b].copy())
    Rs, Ss = part(wl.R), part(wl.S)
    t0 = time.perf_counter()
    oracle.sig_batch(Rs.arena, Rs.off, nthreads=cores)
    oracle.sig_batch(Ss.arena, Ss.off, nthreads=cores)
    oracle.join_grace(Rs, Ss, log2_parts=10, nthreads=cores)
    return time.perf_counter() - t0, Ss.n


def cpu_baseline_full(wl, cores: int) -> dict:
    """The oracle timed once on all of R and all of S (signatures of every key,
    then the Grace hash join): S tuples per second of the whole join."""
    t, n_s = cpu_oracle_slice(wl, 0.0, 1.0, cores)
    return {"value": n_s / t, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": t,
            "sample": f"all of R ({wl.R.n:,} keys) and all of S ({wl.S.n:,} keys): signatures of every key and "
                      f"the Grace hash join, one timed run"}


def run_reference(args):
    """The reference arm: the CPU oracle, each step on a consecutive 1/k of R and
    of S (k sized so that the whole run takes about a minute); value = the S
    keys of a step / its time, median over the steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    spec = workloads.CONFIGS[args.workload]
    wl = workloads.generate(spec)
    cores = os.cpu_count() or 1
    t_cal, _ = cpu_oracle_slice(wl, 0.0, 1.0 / 200, cores)        # calibration on 1/200 of the join
    budget = 45.0 / max(1, args.steps + args.warmup)
    k = int(min(200, max(1, math.ceil(t_cal * 200 / budget))))
    secs, vals = [], []
    for i in range(args.warmup + args.steps):
        j = i % k
        t, n_s = cpu_oracle_slice(wl, j / k, (j + 1) / k, cores)
        if i >= args.warmup:
            secs.append(t)
            vals.append(n_s / t)
    value = statistics.median(vals)
    ms = statistics.median(secs) * 1e3
    sample = (f"each step: a consecutive 1/{k} of R and of S ({wl.R.n // k:,} R and {wl.S.n // k:,} S keys), "
              f"signatures of every key and the Grace hash join of the two slices")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": workload_desc(args.workload, spec)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- batch and serving legs

SERVE_SECONDS = 2.0
LOAD_FACTORS = (0.5, 0.35, 0.25)   # candidates of the single join's load-factor tuning


BATCH_WAVE_BYTES = 110 * 10 ** 9      # key bytes per wave of the full batch (with offsets and workspace < 120 GB)
BATCH_SAMPLE_BYTES = 300 * 10 ** 6    # largest join (R + S key bytes) of a wave checked against the oracle


def batch_leg(ag, steps: int):
    """The 512-join batch at full size (|R| log-normal median 20,000 in
    [1,000, 1,000,000], |S| = 10 |R|, three key-length bands; about 430 GB of
    keys) in waves of consecutive joins of at most BATCH_WAVE_BYTES key bytes.
    Each wave is generated on the device (untimed), its load factor and
    signature kernel shape autotuned, its per-join pair counts checked against
    the generator's and two of its joins (the smallest and a seeded random one
    under BATCH_SAMPLE_BYTES) checked byte for byte against the host generator
    and pair for pair against the oracle; then its graph-captured batch run is
    timed (inputs far larger than L2).  S tuples/s over the timed runs."""
    import random
    import time
    import torch
    import oracle
    from paper_2411_18183_gb300 import tune
    from workloads import device as gdev
    spec = workloads.BatchSpec()
    specs = spec.joins()
    t0 = time.time()
    plan = gdev.plan_batch(specs)
    groups = gdev.waves(plan, BATCH_WAVE_BYTES)
    rng = random.Random(spec.seed)
    shapes = ag.sig_shapes()
    cores = os.cpu_count() or 1
    out_waves, total_ms, total_s, total_bytes, sampled = [], 0.0, 0, 0, 0
    for j0, j1 in groups:
        tg = time.time()
        w = gdev.fill_wave(plan, j0, j1)
        gen_s = time.time() - tg
        R = ag.DeviceRelation(w.arenaR, w.offR, None)
        S = ag.DeviceRelation(w.arenaS, w.offS, None)
        caps = [max(64, int(e * 1.25) + 64) for e in w.expected]
        gb, tried, shape_tried = tune.autotune(R, S, w.ranges, caps)
        gb.counts.zero_()
        gb.replay()
        torch.cuda.synchronize()
        if gb.counts.cpu().tolist() != list(w.expected):
            raise SystemExit(f"batch leg: wave {j0}-{j1}: per-join pair counts differ from the generator's")
        # two joins of the wave against the host generator and the oracle
        sizes = {j: plan.key_bytes(j, j + 1) for j in range(j0, j1)}
        small = [j for j in range(j0, j1) if sizes[j] <= BATCH_SAMPLE_BYTES]
        picks = sorted({min(sizes, key=sizes.get)} | ({rng.choice(small)} if small else set()))
        checked = []
        for j in picks:
            wl = workloads.generate(specs[j])
            rb, re_, sb, se = w.ranges[j - j0]
            for dev_arena, dev_off, rel, a, b in ((w.arenaR, w.offR, wl.R, rb, re_), (w.arenaS, w.offS, wl.S, sb, se)):
                lo, hi = int(dev_off[a]), int(dev_off[b])
                if not np.array_equal(dev_arena[lo:hi].cpu().numpy(), rel.arena[: rel.nbytes]):
                    raise SystemExit(f"batch leg: join {j}: device-generated bytes differ from the host generator's")
            want = oracle.join_grace(wl.R, wl.S, nthreads=cores)
            got = oracle.sort_pairs(gb.result(j - j0).cpu().numpy().view(np.uint32))
            if not np.array_equal(got, want):
                raise SystemExit(f"batch leg: join {j}: pairs differ from the oracle's")
            checked.append({"join": j, "R": specs[j].m, "S": specs[j].n, "key_bytes": sizes[j], "pairs": len(want)})
        sampled += len(checked)
        ms = gb.time_ms(reps=max(3, steps))
        total_ms += ms
        total_s += w.nS
        total_bytes += w.key_bytes
        out_waves.append({"joins": [j0, j1], "rows": {"R": w.mR, "S": w.nS}, "key_bytes": w.key_bytes,
                          "generate_s": round(gen_s, 2), "load_factor": gb.lf, "sig_shape": shapes[gb.shape],
                          "tuning_ms": tried, "shape_tuning_ms": {str(shapes[k]): v for k, v in shape_tried.items()},
                          "ms": ms, "tuples_per_s": w.nS / (ms * 1e-3), "oracle_checked": checked})
        del gb, R, S, w
        torch.cuda.empty_cache()
    del plan
    torch.cuda.empty_cache()
    return {"workload": f"{spec.n_joins} joins, |R| log-normal median {spec.r_median:g} (sigma {spec.sigma:g}) in "
                        f"[{spec.r_range[0]}, {spec.r_range[1]}], |S| = {spec.s_factor} |R|, key bands "
                        f"{list(spec.bands)} B, {int(spec.frac_copy * 100)}% S copies; full size, in waves of "
                        f"<= {BATCH_WAVE_BYTES / 1e9:g} GB of keys generated on the device",
            "joins": spec.n_joins, "rows": {"R": plan_rows(specs, "m"), "S": plan_rows(specs, "n")},
            "key_bytes": total_bytes, "waves": out_waves, "ms_total": total_ms,
            "tuples_per_s": total_s / (total_ms * 1e-3), "key_GBps": total_bytes / (total_ms * 1e-3) / 1e9,
            "joins_per_s": spec.n_joins / (total_ms * 1e-3), "oracle_checked_joins": sampled,
            "pair_counts": "every join equals the generator's count", "wall_s": round(time.time() - t0, 1),
            "l2": "inputs of each wave far larger than L2", "gpu_launches_per_batch": 5, "cuda_graph": True}


def plan_rows(specs, field):
    return sum(getattr(sp, field) for sp in specs)


SERVE_OVERLOAD = 4.0     # arrival-rate multiple of the serving leg's second run, in which the budget binds


def serve_leg(ag):
    """Poisson arrivals (2,000 joins/s) of join requests over a resident pool
    of 64 joins at the stated request size (about 64 GB of XML-like keys,
    generated on the device), admitted under the 120 GB device-memory bound
    and continuously batched on 4 streams.  A second run offers
    SERVE_OVERLOAD times the rate, so that admission waits on the budget.
    Every request's pair count equals the generator's."""
    import torch
    from paper_2411_18183_gb300 import serve
    from workloads import device as gdev
    spec = workloads.SERVE_SPEC
    plan = gdev.plan_batch(spec.joins())
    w = gdev.fill_wave(plan, 0, spec.n_joins)
    del plan
    torch.cuda.empty_cache()
    pool = serve.DevicePool.from_device(ag.DeviceRelation(w.arenaR, w.offR, None),
                                        ag.DeviceRelation(w.arenaS, w.offS, None), w.ranges, w.expected)
    ex = serve.GpuExecutor(pool, n_slots=4, max_batch=64)

    def one(rate, seconds, seed):
        srv = serve.Server(ex, budget_bytes=workloads.SERVE_BUDGET_BYTES, max_batch=64)
        reqs = srv.run(serve.poisson_arrivals(rate, seconds, pool.n, seed=seed), timeout=300.0)
        bad = [r.rid for r in reqs if r.count != pool.expected[r.pool_index]]
        if bad:
            raise SystemExit(f"serving leg: {len(bad)} requests got a wrong pair count")
        s = serve.summarize(reqs)
        tuples = sum(pool.ranges[r.pool_index][3] - pool.ranges[r.pool_index][2] for r in reqs)
        s.update({"rate_per_s": rate, "seconds": seconds, "peak_admitted_bytes": srv.ledger.peak,
                  "budget_bytes": workloads.SERVE_BUDGET_BYTES, "batches": srv.batches,
                  "tuples_per_s": tuples / s["span_s"] if s["span_s"] else None})
        return s

    serve.Server(ex, budget_bytes=workloads.SERVE_BUDGET_BYTES, max_batch=64).run(
        serve.poisson_arrivals(workloads.SERVE_RATE, 0.2, pool.n, seed=1))             # warm-up
    s = one(workloads.SERVE_RATE, SERVE_SECONDS, spec.seed)
    s["overload"] = one(workloads.SERVE_RATE * SERVE_OVERLOAD, SERVE_SECONDS / 2, spec.seed + 1)
    s.update({"workload": f"Poisson {workloads.SERVE_RATE:g} joins/s for {SERVE_SECONDS:g} s over a pool of "
                          f"{pool.n} joins at full request size: |R| log-normal median {spec.r_median:g} in "
                          f"[{spec.r_range[0]}, {spec.r_range[1]}], |S| = {spec.s_factor_range[0]}-"
                          f"{spec.s_factor_range[1]} |R|, XML-like keys {spec.bands[0][0]}-{spec.bands[0][1]} B, "
                          f"{int(spec.frac_copy * 100)}% S copies; pool generated on the device",
              "pool_key_bytes": w.key_bytes, "pool_rows": {"R": w.mR, "S": w.nS}, "streams": 4})
    del ex, pool, w
    torch.cuda.empty_cache()
    return s


SWEEP_LENGTHS = (16, 64, 256, 1024, 4096, 8192)


def length_sweep_leg(ag, reps: int = 5):
    """Whole-join S tuples/s of the signature join and of the full-string GPU join
    (plain and tagged slots) for fixed key lengths, |R| = 10,000, |S| = 100,000,
    30% of S copies an R key (the plain workload's shape at one length)."""
    import torch
    out = []
    for i, L in enumerate(SWEEP_LENGTHS):
        spec = workloads.JoinSpec(m=10_000, n=100_000, r_len=(L, L), s_len=(L, L), alphabet="printable",
                                  frac_copy=0.30, seed=20181 + i)
        wl = workloads.generate(spec)
        R = ag.DeviceRelation.from_host(wl.R.arena, wl.R.off, wl.R.ids)
        S = ag.DeviceRelation.from_host(wl.S.arena, wl.S.off, wl.S.ids)
        pairs = torch.empty(2 * (wl.expected_pairs() + 1024), dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        ws = ag.alloc_ws(ag.join_ws_bytes(R.n, S.n, 0.5))
        bws = ag.alloc_ws(ag.baseline_ws_bytes(R.n, S.n, 0.5))
        stream = torch.cuda.current_stream()
        runs = {"signature": lambda: ag.join_into(R, S, ws, pairs, count, 0.5, sync=False, stream=stream),
                "fullstring_plain": lambda: ag.baseline_join_into(R, S, bws, pairs, count, 0.5, tagged=False,
                                                                  sync=False, stream=stream),
                "fullstring_tagged": lambda: ag.baseline_join_into(R, S, bws, pairs, count, 0.5, tagged=True,
                                                                   sync=False, stream=stream)}
        row = {"key_bytes": L}
        for name, f in runs.items():
            f()
            torch.cuda.synchronize()
            if int(count.item()) != wl.expected_pairs():
                raise SystemExit(f"length sweep: {name} found {int(count.item())} pairs at {L} B")
            for _ in range(2):
                f()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                f()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[name] = {"ms": ms, "tuples_per_s": S.n / (ms * 1e-3)}
        row["speedup_vs_plain"] = row["fullstring_plain"]["ms"] / row["signature"]["ms"]
        row["speedup_vs_tagged"] = row["fullstring_tagged"]["ms"] / row["signature"]["ms"]
        out.append(row)
        del R, S, ws, bws, pairs
    return {"workload": "|R| = 10,000 x |S| = 100,000 printable keys of one fixed length, 30% S copies; "
                        "whole join (both relations' signatures or hashes, build, probe, verify, compaction)",
            "rows": out}


# --------------------------------------------------------------------------- replicas on N GPUs

def max_over_ranks(dist, x: float, device) -> float:
    """The largest x over the ranks (the slowest replica's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput of `world` replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (max_ms * 1e-3)


# --------------------------------------------------------------------------- GPU arm

TUNE_ROUNDS = 3
FLUSH_BYTES = 512 << 20          # written between timed steps: four times the 129 MB L2
_flush_buf = None


def flush_l2(stream):
    """Evict L2 by writing a buffer four times its size on the stream."""
    import torch
    global _flush_buf
    if _flush_buf is None:
        _flush_buf = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        _flush_buf.fill_(0x5A)


def tune_load_factor(make_run, stream):
    """The fastest of LOAD_FACTORS for a join: each candidate's run() is timed
    over two joins per round, in TUNE_ROUNDS rounds that interleave the
    candidates (so a drift of the clock or the memory system hits them all);
    a candidate's time is its median round.  Returns (best, {lf: ms})."""
    import torch
    runs = {}
    for cand in LOAD_FACTORS:
        runs[cand] = make_run(cand)
        runs[cand]()
    torch.cuda.synchronize()
    times = {cand: [] for cand in LOAD_FACTORS}
    for _ in range(TUNE_ROUNDS):
        for cand in LOAD_FACTORS:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                runs[cand]()
            e1.record(stream)
            torch.cuda.synchronize()
            times[cand].append(e0.elapsed_time(e1) / 2)
    med = {str(c): statistics.median(v) for c, v in times.items()}
    best = min(LOAD_FACTORS, key=lambda c: med[str(c)])
    runs.clear()
    torch.cuda.empty_cache()
    return best, med


def run_gpu(args):
    import torch
    import paper_2411_18183_gb300 as ag

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def ranks_max(x: float) -> float:
        return max_over_ranks(dist, x, "cuda")

    spec = workloads.CONFIGS[args.workload]
    t_gen = time.perf_counter()
    # inputs live in pinned host memory (for the end-to-end leg) and are copied once
    # to device memory (for the device-resident leg)
    pinned = []

    def alloc(nbytes):
        t = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        pinned.append(t)
        return t.numpy()

    wl = workloads.generate(spec, alloc=alloc)
    t_gen = time.perf_counter() - t_gen
    m, n = wl.R.n, wl.S.n
    key_bytes = wl.R.nbytes + wl.S.nbytes

    def host_rel(rel):
        return (torch.from_numpy(rel.arena), torch.from_numpy(rel.off.view(np.int64)).pin_memory(),
                torch.from_numpy(rel.ids.view(np.int32)).pin_memory())

    hR, hS = host_rel(wl.R), host_rel(wl.S)
    dR = ag.DeviceRelation(hR[0].cuda(), hR[1].cuda(), hR[2].cuda())
    dS = ag.DeviceRelation(hS[0].cuda(), hS[1].cuda(), hS[2].cuda())
    cap = int(max(1024, wl.expected_pairs() * 1.25 + 1024))
    pairs = torch.empty(2 * cap, dtype=torch.int32, device="cuda")
    sigR = torch.empty(m, dtype=torch.int64, device="cuda")
    sigS = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    # one step = the whole signature join, as four library calls (one kernel each
    # but the build): sig(R), build, sig(S), probe with the S signatures
    PH = ("sig_R", "build", "sig_S", "verify")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(PH) + 1)] for _ in range(args.steps)]

    def make_step(lf):
        ws = ag.alloc_ws(ag.join_ws_bytes(m, n, lf))
        tb = ag.join_table_bytes(m, lf)
        count = ws[tb:tb + 8].view(torch.int64)

        def step(evs=None):
            if evs:
                evs[0].record(stream)
            ag.sig_compute(dR, sigR, stream=stream)
            if evs:
                evs[1].record(stream)
            t = ag.join_build(dR, ws[:tb], lf, sigR=sigR, stream=stream)
            if evs:
                evs[2].record(stream)
            ag.sig_compute(dS, sigS, stream=stream)
            if evs:
                evs[3].record(stream)
            ag.join_probe_sigs(t, dS, sigS, pairs, count, sync=False, stream=stream)
            if evs:
                evs[4].record(stream)
            return t
        return step, ws, tb, count

    # the table's load factor: given, or the fastest of a few, each timed over two
    # joins before the timed region (the batch leg tunes its own the same way)
    lf_tuning = {}
    if args.load_factor is None:
        lf, lf_tuning = tune_load_factor(lambda cand: make_step(cand)[0], stream)
    else:
        lf = args.load_factor
    step, ws, tb, count = make_step(lf)

    # correctness of the timed configuration: total pairs = the generator's ground truth
    step()
    torch.cuda.synchronize()
    total_pairs = int(count.item())
    expected = wl.expected_pairs()
    if total_pairs != expected:
        raise SystemExit(f"pair count {total_pairs} != expected {expected}")

    # the whole join as one library call (as_join: S's signatures on a side stream overlap R's
    # signatures and the build), the timed step of the headline value
    jws = ag.alloc_ws(ag.join_ws_bytes(m, n, lf))
    jcount = torch.zeros(1, dtype=torch.int64, device="cuda")

    def whole_join():
        ag.join_into(dR, dS, jws, pairs, jcount, lf, sync=False, stream=stream)
    whole_join()
    torch.cuda.synchronize()
    if int(jcount.item()) != expected:
        raise SystemExit(f"whole join: pair count {int(jcount.item())} != expected {expected}")

    for _ in range(args.warmup):
        step()
        whole_join()
    barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    barrier()
    # K whole joins (the headline), each bracketed by CUDA events, L2 flushed between them ...
    wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        wev[k][0].record(stream)
        whole_join()
        wev[k][1].record(stream)
        flush_l2(stream)                                # between steps, outside the steps' events
    # ... then K joins as the four calls, with events between the kernels (the per-kernel split),
    # each followed (after an L2 flush) by the probe of the same table as one call, whose kernel
    # computes S's signatures and probes in one pass (the whole join's pass over S), and by the
    # build without given signatures, whose kernel computes R's signatures and inserts them (the
    # whole join's pass over R, the table clear included)
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fcount = torch.zeros(1, dtype=torch.int64, device="cuda")
    table_cap = 0
    for k in range(args.steps):
        t_k = step(ev[k])
        flush_l2(stream)
        fev[k][0].record(stream)
        ag.join_probe(t_k, dS, pairs, fcount, sigS_out=sigS, sync=False, stream=stream)
        fev[k][1].record(stream)
        flush_l2(stream)
        bev[k][0].record(stream)
        table_cap = int(ag.join_build(dR, ws[:tb], lf, stream=stream).cap)
        bev[k][1].record(stream)
        flush_l2(stream)
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    phase_ms = {ph: [e[i].elapsed_time(e[i + 1]) for e in ev] for i, ph in enumerate(PH)}
    split_ms = [e[0].elapsed_time(e[len(PH)]) for e in ev]
    step_ms = [a.elapsed_time(b) for a, b in wev]
    ms_per_step = ranks_max(sum(step_ms)) / args.steps   # the K steps' own event time, flushes excluded
    value = replica_value(n, world, ms_per_step)

    # the same-GPU comparison join on full strings (plain and tagged variants), each
    # with its own load factor tuned the same way, timed like the signature join's steps
    # (L2 flushed between joins, each join's own CUDA-event time)
    def timed_reps(run, reps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in evs:
            a.record(stream)
            run()
            b.record(stream)
            flush_l2(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in evs)

    baseline = {}
    for tagged in (False, True):
        def make_brun(cand, tagged=tagged):
            bws_c = ag.alloc_ws(ag.baseline_ws_bytes(m, n, cand))
            bcount_c = torch.zeros(1, dtype=torch.int64, device="cuda")

            def run():
                ag.baseline_join_into(dR, dS, bws_c, pairs, bcount_c, cand, tagged=tagged, sync=False, stream=stream)
            return run
        if args.load_factor is None:
            blf, btune = tune_load_factor(make_brun, stream)
        else:
            blf, btune = args.load_factor, None
        bws = ag.alloc_ws(ag.baseline_ws_bytes(m, n, blf))
        bcount = torch.zeros(1, dtype=torch.int64, device="cuda")
        st, bcnt = ag.baseline_join_into(dR, dS, bws, pairs, bcount, blf, tagged=tagged, sync=True)
        if bcnt != total_pairs:
            raise SystemExit(f"comparison join found {bcnt} pairs, signature join {total_pairs}")
        for _ in range(2):
            ag.baseline_join_into(dR, dS, bws, pairs, bcount, blf, tagged=tagged, sync=False, stream=stream)
        bms = timed_reps(lambda: ag.baseline_join_into(dR, dS, bws, pairs, bcount, blf, tagged=tagged, sync=False,
                                                       stream=stream), max(3, min(10, args.steps)))
        baseline["tagged" if tagged else "plain"] = {"ms_per_join": bms, "tuples_per_s": n / (bms * 1e-3),
                                                     "load_factor": blf, "load_factor_tuning_ms": btune}
        del bws

    # the radix-partitioned signature join (R and S split by the bucket hash's top
    # bits, one table per partition) on the same inputs, against the step above
    pws = ag.alloc_ws(ag.join_part_ws_bytes(m, n, lf))
    st, pcnt = ag.join_partitioned_into(dR, dS, pws, pairs, bcount, lf, sync=True)
    if pcnt != total_pairs:
        raise SystemExit(f"partitioned join found {pcnt} pairs, signature join {total_pairs}")
    for _ in range(2):
        ag.join_partitioned_into(dR, dS, pws, pairs, bcount, lf, sync=False, stream=stream)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    breps = max(3, min(10, args.steps))
    b0.record(stream)
    for _ in range(breps):
        ag.join_partitioned_into(dR, dS, pws, pairs, bcount, lf, sync=False, stream=stream)
    b1.record(stream)
    torch.cuda.synchronize()
    pms = b0.elapsed_time(b1) / breps
    part_bits = 0
    while part_bits < 12 and (m >> (part_bits + 10)) > 0:
        part_bits += 1
    partitioned = {"ms_per_join": pms, "tuples_per_s": n / (pms * 1e-3), "partition_bits": part_bits,
                   "speedup_vs_unpartitioned": ms_per_step / pms}
    del pws

    # the prefix join (keys equal on their first 256 bytes) on the same inputs
    PREFIX_LEN = 256
    xws = ag.alloc_ws(ag.join_prefix_ws_bytes(m, n, lf))
    xpairs = torch.empty(2 * (2 * total_pairs + 1024), dtype=torch.int32, device="cuda")
    st, xcnt = ag.join_prefix_into(dR, dS, PREFIX_LEN, xws, xpairs, bcount, lf, sync=True)
    if xcnt < total_pairs:
        raise SystemExit(f"prefix join found {xcnt} pairs, fewer than the exact join's {total_pairs}")
    for _ in range(2):
        ag.join_prefix_into(dR, dS, PREFIX_LEN, xws, xpairs, bcount, lf, sync=False, stream=stream)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(breps):
        ag.join_prefix_into(dR, dS, PREFIX_LEN, xws, xpairs, bcount, lf, sync=False, stream=stream)
    b1.record(stream)
    torch.cuda.synchronize()
    xms = b0.elapsed_time(b1) / breps
    prefix_join = {"prefix_len": PREFIX_LEN, "ms_per_join": xms, "tuples_per_s": n / (xms * 1e-3), "pairs": xcnt}
    del xws, xpairs

    # the paper's own variants on the same resident inputs: the probe of Figure 2 on
    # signatures only (no byte verification; its extra pairs are signature collisions),
    # with four components and with the paper's two (sig_{alpha,2}), and the exact
    # join on two-component signatures
    def variant(ncomp, mode, field=16):
        def sig(rel, out):
            if field == 8:
                ag.sig_compute_gf8(rel, out, stream=stream)
            else:
                ag.sig_compute(rel, out, stream=stream, n_components=ncomp)

        def run():
            sig(dR, sigR)
            t = ag.join_build(dR, ws[:tb], lf, sigR=sigR, stream=stream)
            sig(dS, sigS)
            ag.join_probe_mode(t, dS, sigS, pairs, count, mode=mode, sync=False, stream=stream)
        run()
        torch.cuda.synchronize()
        cnt = int(count.item())
        if cnt < total_pairs or (mode == "inner" and cnt != total_pairs):
            raise SystemExit(f"variant n={ncomp} {mode}: {cnt} pairs, exact join {total_pairs}")
        for _ in range(2):
            run()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vreps = max(3, min(10, args.steps))
        v0.record(stream)
        for _ in range(vreps):
            run()
        v1.record(stream)
        torch.cuda.synchronize()
        vms = v0.elapsed_time(v1) / vreps
        return {"ms_per_join": vms, "tuples_per_s": n / (vms * 1e-3), "pairs": cnt,
                "collision_pairs": cnt - total_pairs,
                "speedup_vs_fullstring": {k: (n / (vms * 1e-3)) / v["tuples_per_s"] for k, v in baseline.items()}}

    paper_variants = {
        "note": "Figure 2's probe outputs on a signature match; these runs time it on the same inputs "
                "(signatures of R, build, signatures of S, probe) and count the pairs it adds to the "
                "exact join (signature collisions); gf8 = byte symbols over GF(2^8), 4 components",
        "sig_only_n4": variant(4, "sig_only"),
        "sig_only_n2": variant(2, "sig_only"),
        "exact_n2": variant(2, "inner"),
        "sig_only_gf8": variant(4, "sig_only", field=8),
        "exact_gf8": variant(4, "inner", field=8),
    }
    # the byte-symbol signature kernel alone on S (keys / CUDA-event time)
    for _ in range(2):
        ag.sig_compute_gf8(dS, sigS, stream=stream)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(5):
        ag.sig_compute_gf8(dS, sigS, stream=stream)
    g1.record(stream)
    torch.cuda.synchronize()
    gms = g0.elapsed_time(g1) / 5
    paper_variants["gf8_signature_kernel_S"] = {"ms": gms, "key_gbps": wl.S.nbytes / (gms * 1e-3) / 1e9}

    # cumulative (prefix) signatures of S at 256-byte blocks: the layout pass and the
    # signatures pass, timed apart (keys / CUDA-event time)
    def cumulative(block_bytes=256, reps=5):
        lib = ag.load()
        pref = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        pws = ag.alloc_ws(int(lib.as_sig_prefix_ws_bytes(n)))
        offs = lambda: lib.as_sig_prefix_offsets(dS.off.data_ptr(), n, block_bytes, pref.data_ptr(), pws.data_ptr(),
                                                 pws.numel(), stream.cuda_stream)
        if offs() != 0:
            raise SystemExit("prefix offsets failed")
        torch.cuda.synchronize()
        total = int(pref[n].item())
        pout = torch.empty(max(1, total), dtype=torch.int64, device="cuda")
        sigs = lambda: lib.as_sig_prefixes(dS.arena.data_ptr(), dS.off.data_ptr(), n, block_bytes, pref.data_ptr(),
                                           pout.data_ptr(), stream.cuda_stream)
        res = {"block_bytes": block_bytes, "entries": total}
        for name, f in (("offsets", offs), ("prefixes", sigs)):
            for _ in range(2):
                f()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(reps):
                f()
            c1.record(stream)
            torch.cuda.synchronize()
            res[name + "_ms"] = c0.elapsed_time(c1) / reps
        last = pout[(pref[1:] - 1)]                     # each key's last entry is its signature
        res["last_equals_signature"] = bool(torch.equal(last, sigS_exact))
        res["key_gbps"] = wl.S.nbytes / (res["prefixes_ms"] * 1e-3) / 1e9
        return res

    ag.sig_compute(dS, sigS, stream=stream)
    sigS_exact = sigS.clone()
    cumulative_sigs = cumulative()
    del sigS_exact

    hbm, peak_kind = peaks()

    # end to end from pinned host buffers through the package's host-relation join
    # (stream.HostStreamJoin: copies of S chunks overlapped with the kernels of the
    # previous chunk; the pairs come back to pinned host memory)
    from paper_2411_18183_gb300.stream import HostStreamJoin
    target = 512 << 20                                  # about 512 MB of S keys per chunk
    chunk_rows = max(1, min(n, int(n * target / max(1, wl.S.nbytes))))
    chunk_bytes = int(1.1 * wl.S.nbytes * chunk_rows / max(1, n)) + (1 << 20)
    sj = HostStreamJoin(max_m=m, max_r_bytes=hR[0].numel(), max_chunk_rows=chunk_rows, max_chunk_bytes=chunk_bytes,
                        cap_pairs=int(2 * expected + (1 << 16)), max_chunks=4096, load_factor=lf)
    cuts = sj.chunks(wl.S.off)
    out_host = torch.empty(2 * sj.cap, dtype=torch.int32).pin_memory()
    h2d = (sum(int(t.numel() * t.element_size()) for t in hR)
           + sum((((int(wl.S.off[b]) + 15) & ~15) + 16 - (int(wl.S.off[a]) & ~15)) + 8 * (b - a + 1) + 4 * (b - a)
                 for a, b in zip(cuts, cuts[1:])))
    # the host link's pinned copy rate alone (1 GiB host -> device), for the record next to e2e
    hprobe = hS[0][: min(hS[0].numel(), 1 << 30)]
    dprobe = torch.empty(hprobe.numel(), dtype=torch.uint8, device="cuda")
    dprobe.copy_(hprobe, non_blocking=True)
    torch.cuda.synchronize()
    rates = []
    for _ in range(5):                                  # the best of five single copies
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        with torch.cuda.stream(stream):
            dprobe.copy_(hprobe, non_blocking=True)
        h1.record(stream)
        torch.cuda.synchronize()
        rates.append(hprobe.numel() / (h0.elapsed_time(h1) * 1e-3) / 1e9)
    h2d_gbs = max(rates)
    del dprobe
    e2e_steps = max(3, min(args.steps, 9))
    for _ in range(max(2, args.warmup)):                # warm-up runs (the first timed run after a single
        if sj.run(hR, hS, cuts, out_host) != expected:  # warm-up was seen to take several times the rest)
            raise SystemExit("end-to-end join: wrong pair count")
    barrier()
    te = time.perf_counter()
    e2e_runs = []
    for _ in range(e2e_steps):
        t_run = time.perf_counter()
        cnt = sj.run(hR, hS, cuts, out_host)
        e2e_runs.append((time.perf_counter() - t_run) * 1e3)
    barrier()
    e2e_mean_s = ranks_max((time.perf_counter() - te) / e2e_steps)
    # the median run: single runs were seen to take 2-4x the others at times (the host's memory and link
    # are shared with other jobs), so the mean of a few runs moves by that much from run to run; both kept
    e2e_s = ranks_max(statistics.median(e2e_runs) / 1e3)
    e2e_value = replica_value(n, world, e2e_s * 1e3)
    d2h = 8 * cnt + 8 * (len(cuts) - 1)
    del sj

    # rooflines of the step's kernels from their live CUDA-event times (algorithmic bytes / launch)
    lensS = np.diff(wl.S.off).astype(np.int64)
    lensR = np.diff(wl.R.off).astype(np.int64)
    src = wl.s_src[wl.s_kind == 1]
    verified_bytes = int((wl.r_mult[src].astype(np.int64) * lensS[wl.s_kind == 1]).sum())
    alg = {
        "sig_R": wl.R.nbytes + 8 * (m + 1) + 8 * m,                    # keys, offsets, signatures out
        "sig_S": wl.S.nbytes + 8 * (n + 1) + 8 * n,
        "build": 8 * m + 8 * (m + 1) + 16 * m,                          # sigR, offsets, one slot per row
        "verify": (8 * n + 8 * (n + 1) + 4 * n + 16 * n                # sig, offsets, id, first slot per S key
                   + total_pairs * (16 + 4 + 8)                        # offR pair, idR, output pair
                   + 2 * verified_bytes),                              # R and S key bytes compared
    }
    fused = n >= FUSED_PROBE_FROM                       # the whole join's S pass is one kernel
    # the whole join's R pass: signatures and inserts in one kernel, after the table clear
    phase_ms["sig_build_R"] = [a.elapsed_time(b) for a, b in bev]
    alg["sig_build_R"] = wl.R.nbytes + 8 * (m + 1) + 8 * m + 16 * m + 16 * table_cap
    phases = PH + ("sig_build_R",)
    if fused:                                          # its time from the probe calls after the split steps
        phase_ms["sig_probe_S"] = [a.elapsed_time(b) for a, b in fev]
        alg["sig_probe_S"] = alg["sig_S"] + alg["verify"]
        phases = phases + ("sig_probe_S",)
    kernels = {}
    for ph in phases:
        avg = statistics.mean(phase_ms[ph])
        kernels[ph] = {"ms": avg, "algorithmic_bytes": alg[ph], "gbps": alg[ph] / (avg * 1e-3) / 1e9,
                       "frac_hbm": alg[ph] / (avg * 1e-3) / 1e9 / hbm}
    # the dominant kernel of the timed step: the fused S pass, or the larger of the S signatures and the probe
    dom = "sig_probe_S" if fused else max(("sig_S", "verify"), key=lambda ph: kernels[ph]["ms"])
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            d = json.load(f)
        ent = d.get(KERNEL_NAMES[dom], {})
        if ent.get("kernel_rev") == KERNEL_REVS[KERNEL_NAMES[dom]] and ent.get("per_byte_of_keys"):
            keyb = wl.S.nbytes if dom in ("sig_S", "sig_probe_S") else 2 * verified_bytes
            traffic = ent["per_byte_of_keys"] * keyb

    extra = {}
    if not args.no_extra:
        extra["batch"] = batch_leg(ag, args.steps)
        extra["serving"] = serve_leg(ag)
        extra["length_sweep"] = length_sweep_leg(ag)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_full(wl, os.cpu_count() or 1)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, spec), "load_factor": lf,
                   "load_factor_tuning_ms": lf_tuning or None,
                   "l2": f"L2 flushed between timed steps ({FLUSH_BYTES >> 20} MB written); ms_per_step is the "
                         f"steps' own CUDA-event time, flushes excluded; inputs {key_bytes / 1e9:.2f} GB of keys",
                   "parallelism": f"replicas{world}"},
        "p50_ms": pct(step_ms, 50), "p99_ms": pct(step_ms, 99),
        "split_step_ms": statistics.mean(split_ms),
        "probe_tuples_per_s_probe_phase": n / ((kernels["sig_S"]["ms"] + kernels["verify"]["ms"]) * 1e-3),
        "key_gbps": key_bytes / (ms_per_step * 1e-3) / 1e9,
        "kernels": kernels,
        "fullstring_gpu_join": baseline,
        "partitioned_join": partitioned,
        "prefix_join": prefix_join,
        "speedup_vs_fullstring": {k: value / v["tuples_per_s"] for k, v in baseline.items()},
        "paper_variants": paper_variants,
        "cumulative_signatures": cumulative_sigs,
        "pairs": total_pairs,
        "device_bytes": {"table": ag.join_table_bytes(m, lf), "signatures": 8 * (m + n),
                         "join_workspace": ag.join_ws_bytes(m, n, lf), "pairs_buffer": 8 * cap,
                         "inputs": key_bytes + 12 * (m + n + 2),
                         "note": "per join: the hash table (slots, R signatures, flags, matched-R bitmap), R's and "
                                 "S's signatures, the pair buffer and the resident relations (keys, offsets, ids)"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3, "stat": f"median of {e2e_steps} timed runs (mean in mean_ms)",
                "mean_ms": e2e_mean_s * 1e3, "runs_ms": [round(x, 2) for x in e2e_runs], "chunks": len(cuts) - 1,
                "h2d_pinned_gbs": h2d_gbs,
                "copy_bound_ms": (h2d + d2h) / (h2d_gbs * 1e9) * 1e3,
                "path": "stream.HostStreamJoin: pinned host R and S, S copied in chunks under the kernels"},
        "gpu_launches": (2 if fused else 3) * args.steps,
        "roofline": {"bound": "hbm", "kernel": KERNEL_NAMES[dom], "achieved": kernels[dom]["gbps"], "peak": hbm,
                     "peak_kind": f"{peak_kind} (copy bandwidth, burst)", "unit": "GB/s",
                     "frac": kernels[dom]["frac_hbm"], "traffic": traffic,
                     "algorithmic_bytes": alg[dom],
                     "kernels": {ph: {"kernel": KERNEL_NAMES[ph], "ms": round(kernels[ph]["ms"], 4),
                                      "achieved": round(kernels[ph]["gbps"], 1),
                                      "frac": round(kernels[ph]["frac_hbm"], 4)} for ph in phases}},
        "cpu_baseline": cpu,
        "gen_s": t_gen,
        **extra,
    }
    # a compact summary at the end of the line (where a truncated tail still shows it)
    summ = {"step_ms": round(ms_per_step, 4),
            "kernel_frac_hbm": {ph: round(kernels[ph]["frac_hbm"], 3) for ph in phases},
            "speedup_vs_fullstring": {k: round(v, 3) for k, v in line["speedup_vs_fullstring"].items()},
            "e2e_ms": round(e2e_s * 1e3, 2), "h2d_pinned_gbs": round(h2d_gbs, 1)}
    if "length_sweep" in extra:
        summ["length_sweep_speedup_vs_tagged"] = {str(r["key_bytes"]): round(r["speedup_vs_tagged"], 3)
                                                  for r in extra["length_sweep"]["rows"]}
    line["summary"] = summ
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# revision of each kernel's code; profiles/traffic.json holds counters per revision
KERNEL_REVS = {"sig_key_kernel": "v4", "build_kernel": "v8", "verify_kernel": "v17", "sig_key_kernel+probe": "v2",
               "sig_key_kernel+build": "v1"}
KERNEL_NAMES = {"sig_R": "sig_key_kernel", "sig_S": "sig_key_kernel", "build": "build_kernel",
                "verify": "verify_kernel", "sig_probe_S": "sig_key_kernel+probe", "sig_build_R": "sig_key_kernel+build"}
FUSED_PROBE_FROM = 1 << 19    # S keys from which the library's probe computes signatures and probes in one kernel


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="large", choices=sorted(workloads.CONFIGS))
    ap.add_argument("--load-factor", type=float, default=None,
                    help="table load factor; default: the fastest of %s, tuned before the timed steps" %
                         (LOAD_FACTORS,))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch and serving legs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
