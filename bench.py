"""Benchmark: exact-r instances/s of the batched GPU search on one GB300.

Workload (default): a batch of 4096 random binary automata, n uniform in
[64, 192], delta iid uniform (seeds 0..4095, SplitMix64 recipe of gen.py),
bitsets of three 64-bit words.  One step solves the whole batch: r and the
least shortest reset word of every instance.

  value         instances/s of sw_batch_device, automata already in HBM,
                CUDA events on the search stream; L2 flushed between steps.
  e2e           the same through sw_batch with host buffers (automata copied
                in and results copied out inside the timed region).
  roofline      the meet kernel (the dominant kernel), integer-ALU bound:
                the 32-bit ANDs of its walk (one per bitmap word per state)
                plus 25 operations per 32-bit word of each transposed
                backward row, against 2 ANDs per three-input LOP3 x the
                measured LOP3 rate per SM clock x SMs x maximum SM clock.
  roofline_hbm  the expansion and compaction kernels against the measured
                HBM copy bandwidth: algorithmic bytes per candidate and per
                stored set over their event time.
  serving       sw_server under Poisson arrivals (n~U[32,128], k in 2..4)
                at 0.5, 0.8 and 1.0 x the batched capacity: p50/p99 latency,
                instances/s, admissions while other searches ran.
  one_at_a_time sw_reset_threshold in a loop over a sample, and the batched
                call on the same sample.
  cpu_baseline  the CPU oracle (bidirectional) on a fixed sample of the
                workload's stratum n <= 100 (--cpu-full: of the whole
                workload), every instance run to completion: all cores and
                single-threaded.

--workload hard300 / hard400 (/ hard500 / hard570): one hard random
automaton (seed 0) searched alone, with r, time, peak sets, pairs/s, and the
agreement of two direction schedules.

--impl reference times the CPU oracle instead (the reference arm).
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

from paper_2207_05495_gb300 import gen  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Shared memory: 32 banks x 4 B per clock per SM.  (The integer peak is
# measured at run time by sw_probe_int_peak: LOP3 per SM clock.)
SMEM_BYTES_PER_CLK_SM = 128
SM_MAX_MHZ_FALLBACK = 2070.0
N_SMS_NOMINAL = 152
# DRAM bytes (read + write) of the meet kernel per backward row it
# transposes, from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the meet launches of one step of the first 512
# automata of this workload; the full workload is too large for a
# multi-pass capture, so its traffic per launch is this figure times the
# rows one launch transposes (profiles/meet_traffic_batch512_c3.md;
# recaptured whenever the kernel changes).
MEET_DRAM_BYTES_PER_ROW = 13.47


def rank_seeds(rank: int, count: int) -> range:
    """Weak scaling: rank r solves its own `count` automata, seeds
    r*count .. (r+1)*count - 1 (no data exchange between ranks)."""
    return range(rank * count, (rank + 1) * count)


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time is the slowest rank's."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name: str, rank: int = 0):
    if name == "c3":
        count = 4096
        seeds = rank_seeds(rank, count)
        return [gen.random_automaton_ranged(64, 192, 2, s) for s in seeds], {
            "workload": "batch of 4096 random binary automata, n~U[64,192], k=2, seeds 0..4095, 3x64-bit bitsets",
            "instances": count, "n_range": [64, 192], "k": 2}
    if name == "c1":
        return [gen.random_automaton(40, 2, 0)], {"workload": "single random binary automaton n=40 k=2 seed 0",
                                                  "instances": 1}
    if name == "cerny":
        return [gen.cerny(n) for n in range(16, 29)], {"workload": "Cerny automata n=16..28", "instances": 13}
    if name in ("beam1000", "beam2000", "beam5000"):
        n = int(name[4:])
        return [gen.random_automaton(n, 2, 0)], {
            "workload": f"beam upper bound: random binary automaton n={n} k=2 seed 0, beam n*ceil(log2 n) = "
                        f"{n * int(np.ceil(np.log2(n)))}, {(n + 63) // 64}x64-bit bitsets", "instances": 1}
    if name in ("hard300", "hard400", "hard500", "hard570"):
        n = int(name[4:])
        return [gen.random_automaton(n, 2, 0)], {
            "workload": f"hard single instance: random binary automaton n={n} k=2 seed 0, "
                        f"{(n + 63) // 64}x64-bit bitsets", "instances": 1}
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1)  # touches 256 MiB, larger than the 129 MB L2


def _oracle_init():
    sys.path.insert(0, ROOT)


def _oracle_one(d):
    """One oracle search (bidirectional BFS) in a worker; its own CPU time."""
    import oracle
    t0 = time.process_time()
    r = oracle.bidir(d)[0]
    return r, time.process_time() - t0


def cpu_fixed_sample(pool, sample):
    """Runs every automaton of `sample` through the oracle on the pool (one
    process per core), each to completion; returns (wall seconds, summed
    per-instance CPU seconds, r values)."""
    t0 = time.perf_counter()
    res = pool.map(_oracle_one, sample, chunksize=1)
    wall = time.perf_counter() - t0
    return wall, sum(t for _, t in res), [r for r, _ in res]


def stratified_seeds(count: int, m: int):
    """m seeds spread evenly over 0..count-1 (0, count/m, 2 count/m, ...)."""
    return [i * count // m for i in range(m)]


def oracle_pool(cores: int):
    import multiprocessing as mp
    import oracle
    oracle.build()
    return mp.get_context("spawn").Pool(cores, initializer=_oracle_init)


def run_reference(args, ds, cfg, rank, world):
    """The reference arm: the CPU oracle as it stands, on the machine's host
    cores.  The oracle's cost per instance has a heavy tail (from 0.01 s to
    over a minute on one core for this workload), so a step cannot hold an
    unbiased sample and stay short; each step takes the next `cores`
    instances (in seed order) of the workload's stratum n <= 100 and runs
    every one to completion.  The stratum is declared in the line."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    stratum = [d for d in ds if d.shape[1] <= args.ref_n_max]
    per = cores
    need = per * (args.warmup + args.steps)
    sample = [stratum[i % len(stratum)] for i in range(need)]
    with oracle_pool(cores) as pool:
        for s in range(args.warmup):
            cpu_fixed_sample(pool, sample[s * per:(s + 1) * per])
        tot_wall, tot_cpu, done = 0.0, 0.0, 0
        for s in range(args.warmup, args.warmup + args.steps):
            wall, cpu_s, rs = cpu_fixed_sample(pool, sample[s * per:(s + 1) * per])
            tot_wall += wall
            tot_cpu += cpu_s
            done += len(rs)
    v = done / tot_wall if tot_wall else 0.0
    smp = (f"each step: the next {per} instances in seed order of the workload's stratum n <= {args.ref_n_max} "
           f"({len(stratum)} of {len(ds)} instances), every one run to completion; {done} instances timed")
    line = {"impl": "reference", "metric": "exact-r instances/sec", "value": v, "unit": "instances/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "instances/s", "cores": cores, "kind": "oracle", "sample": smp,
                             "single_thread": done / tot_cpu if tot_cpu else 0.0},
            "e2e": {"value": v, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_line(ds, m: int, cores: int, n_max: int = 0):
    """The oracle on a fixed sample of the workload, every instance run to
    completion: all cores (one process per core) and single-threaded (the
    summed per-instance CPU times).  n_max = 0: m instances at evenly spread
    seeds of the whole workload (unbiased, but its hardest instances take
    minutes each on one core); n_max > 0: m instances evenly spread over the
    stratum n <= n_max (bounded, and stated as such)."""
    pool_idx = [i for i in range(len(ds)) if n_max <= 0 or ds[i].shape[1] <= n_max]
    m = min(m, len(pool_idx))
    idx = [pool_idx[j] for j in stratified_seeds(len(pool_idx), m)]
    with oracle_pool(min(cores, m)) as pool:
        wall, cpu_s, rs = cpu_fixed_sample(pool, [ds[i] for i in idx])
    where = (f"the stratum n <= {n_max} ({len(pool_idx)} of {len(ds)} instances)" if n_max > 0
             else "the whole workload")
    return {"value": m / wall, "unit": "instances/s", "cores": min(cores, m), "kind": "oracle",
            "single_thread": m / cpu_s if cpu_s else 0.0,
            "sample": f"{m} instances evenly spread over {where}, indices {idx[0]}, {idx[1] if m > 1 else ''}, ... "
                      f"{idx[-1]}, each run to completion by the bidirectional oracle; wall {wall:.1f} s on "
                      f"{min(cores, m)} processes, {cpu_s:.1f} s of summed CPU time"}


def serve_bench(sw, torch, stream, args):
    """Poisson arrivals into sw_server at lambda = 0.5, 0.8 and 1.0 x the
    batched capacity on the same requests; latency = submit to poll."""
    m = args.serve_requests
    ds = []
    for i in range(m):
        st = gen._Stream(100000 + i)
        n = 32 + int(gen.below(st.draw(1), 97)[0])
        k = 2 + int(gen.below(st.draw(1), 3)[0])
        ds.append(gen.random_automaton(n, k, 200000 + i))
    hs = [sw.load(d) for d in ds]
    ws = sw.workspace(16 << 30)
    # capacity: the same requests as one batch
    sw.sw_batch(hs[:64], ws=ws, word_cap=4096)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r_batch, _ = sw.sw_batch(hs, ws=ws, word_cap=4096)
    torch.cuda.synchronize()
    cap = m / (time.perf_counter() - t0)
    del ws
    arr = gen.splitmix64_block(0xC5, 0, m)
    u = (arr >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    runs = []
    for frac in (0.5, 0.8, 1.0):
        lam = frac * cap
        gaps = -np.log(1.0 - u) / lam
        srv = sw.Server(sw.workspace(16 << 30), n_max=128, k_max=4, max_requests=m, word_cap=4096)
        sub_t = np.zeros(m)
        lat = np.zeros(m)
        got = 0
        t_start = time.perf_counter()
        next_t = t_start
        i = 0
        while got < m:
            now = time.perf_counter()
            while i < m and now >= next_t:
                if srv.submit(hs[i], i) != 0:
                    break
                sub_t[i] = time.perf_counter()
                next_t += gaps[i]
                i += 1
            res = srv.poll()
            while res is not None:
                lat[res[0]] = time.perf_counter() - sub_t[res[0]]
                if res[3] != 0 or res[1] != r_batch[res[0]]:
                    raise RuntimeError(f"served request {res[0]}: code {res[3]}, r {res[1]} != {r_batch[res[0]]}")
                got += 1
                res = srv.poll()
            if time.perf_counter() - t_start > 120:
                raise RuntimeError("serving run exceeded 120 s")
            time.sleep(0.0002)
        total = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        runs.append({"lambda_frac": frac, "lambda_per_s": lam, "instances_per_s": m / total,
                     "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                     "admitted_while_running": st["admitted_while_1"], "max_active": st["max_active"]})
    return {"requests": m, "arrivals": "Poisson, SplitMix64 seed 0xC5", "batched_capacity_per_s": cap,
            "workload": "random automata n~U[32,128], k~U{2,3,4}", "runs": runs}


def meet_roofline(stats, nsm):
    """The meet kernel against the integer pipe: int32 operations it
    performs (64 per 64-bit lane word of a warp-wide AND step, 25 per 32-bit
    word of every transposed backward row) over its summed event time."""
    meet_ms = sum(s["meet_ms"] for s in stats) / len(stats)
    pairs = sum(s["pairs"] for s in stats) / len(stats)
    iters = sum(s["and_iters"] for s in stats) / len(stats)
    rows_t = sum(s["rows_transposed"] for s in stats) / len(stats)
    launches = sum(s["meet_launches"] for s in stats) / len(stats)
    lw = max(1, stats[-1]["meet_lane_words"])
    return meet_ms, pairs, iters, rows_t, launches, lw


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3",
                    choices=["c3", "c1", "cerny", "hard300", "hard400", "hard500", "hard570", "beam1000", "beam2000",
                             "beam5000"])
    ap.add_argument("--ws-gb", type=float, default=160.0)
    ap.add_argument("--cpu-sample", type=int, default=160,
                    help="instances of the fixed sample the CPU oracle runs to completion")
    ap.add_argument("--cpu-full", action="store_true",
                    help="CPU sample spread over the whole workload instead of the stratum n <= --ref-n-max "
                         "(unbiased; several minutes on the heavy-tailed instances)")
    ap.add_argument("--ref-n-max", type=int, default=100,
                    help="reference arm: the stratum (n <= this) its steps draw instances from")
    ap.add_argument("--one-sample", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--count", type=int, default=0, help="use only the first COUNT instances (small cases)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--opt", action="append", default=[],
                    help="override a search option after tuning, e.g. --opt meet_lane_words=4")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--one-schedule", action="store_true",
                    help="hard workloads: skip the second (balanced) schedule")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    ds, cfg = workload(args.workload, rank)
    cfg = dict(cfg)
    if args.count and args.count < len(ds):
        ds = ds[: args.count]
        cfg["workload"] += f" (first {args.count} only)"
        cfg["instances"] = args.count
    cfg["l2"] = "flushed between steps (256 MiB write)"
    cfg["parallelism"] = f"replicas x{world} (independent instances per GPU)"

    hard = args.workload.startswith("hard") or args.workload.startswith("beam")
    if args.impl == "reference":
        if args.workload.startswith("beam"):
            if rank == 0:
                run_reference_beam(args, ds[0], cfg)
            return
        if hard:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle does not finish a random "
                                  "automaton of this size (about 1e14 candidate pairs at the meet)"}), flush=True)
            return
        run_reference(args, ds, cfg, rank, world)
        return

    # CPU baseline first: its process pool is spawned before any CUDA work
    cpu = None
    if rank == 0 and not args.no_cpu and not hard:
        cpu = cpu_baseline_line(ds, min(args.cpu_sample, len(ds)), os.cpu_count() or 1,
                                0 if args.cpu_full else args.ref_n_max)

    import torch
    import torch.distributed as dist
    from paper_2207_05495_gb300 import build, sw
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    count = len(ds)
    from paper_2207_05495_gb300 import autotune
    tuned = autotune.apply(max((d.shape[1] + 63) // 64 for d in ds), int(ds[0].shape[0]))
    cfg["options"] = dict(tuned) if tuned else {}
    if args.opt:
        o = sw.sw_get_options()
        for kv in args.opt:
            k, v = kv.split("=")
            setattr(o, k, type(getattr(o, k))(float(v)) if isinstance(getattr(o, k), float) else int(v))
            cfg["options"][k] = v
        sw.sw_set_options(o)
    if not cfg["options"]:
        cfg["options"] = "library defaults"
    props = torch.cuda.get_device_properties(local)
    nsm = props.multi_processor_count
    # the integer peak of the meet and marking kernels: the measured LOP3
    # issue rate per SM clock, times the two bitmap-word ANDs one
    # three-input LOP3 retires, times SMs and the maximum SM clock
    lop3_probe = sw.sw_probe_int_peak()
    peak = 2 * lop3_probe * nsm * SM_MAX_MHZ_FALLBACK * 1e6 / 1e12
    smem_peak = SMEM_BYTES_PER_CLK_SM * nsm * SM_MAX_MHZ_FALLBACK * 1e6 / 1e12
    hbm_peak = hbm_peak_gbs()
    if args.workload.startswith("beam"):
        line = run_beam(args, ds[0], cfg, sw, torch, local, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    if hard:
        line = run_hard(args, ds[0], cfg, sw, torch, local, world, peak, nsm)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    ns = np.array([d.shape[1] for d in ds], np.int32)
    ks = np.array([d.shape[0] for d in ds], np.int32)
    W = int(max((int(n) + 63) // 64 for n in ns))
    flat = np.concatenate([d.ravel() for d in ds]).astype(np.int32)
    offs = np.concatenate([[0], np.cumsum([d.size for d in ds])[:-1]]).astype(np.int64)
    word_cap = 1024
    word_off = np.arange(count + 1, dtype=np.int64) * word_cap
    stream = torch.cuda.Stream()
    ws = sw.workspace(int(args.ws_gb * (1 << 30)))
    d_delta = torch.from_numpy(flat).cuda()
    d_r = torch.zeros(count, dtype=torch.int32, device="cuda")
    d_words = torch.zeros(int(word_off[-1]), dtype=torch.uint8, device="cuda")
    l2 = torch.zeros(64 << 20, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step():
        rc = sw.sw_batch_device(ns, ks, d_delta, offs, stream=stream, ws=ws, d_r=d_r, d_words=d_words,
                                word_off=word_off)
        if rc != 0:
            bad = (d_r.cpu().numpy() < 0).nonzero()[0]
            raise RuntimeError(f"sw_batch_device failed: {rc}; failed instances {bad[:20].tolist()} "
                               f"n={ns[bad[:20]].tolist()} stats={sw.sw_last_stats()}")

    for _ in range(args.warmup):
        step()
    sw.sw_set_timing(True)
    times, stats = [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush_l2(l2)
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1))
            stats.append(sw.sw_last_stats())
    sw.sw_set_timing(False)
    ms = float(np.mean(times))
    if world > 1:
        ms = max_over_ranks(ms, dist, "cuda")
    value = count * world / (ms * 1e-3)

    # results of the last timed step, checked: every word resets Q
    r = d_r.cpu().numpy()
    words = d_words.cpu().numpy()
    for i in range(count):
        st = np.arange(ns[i])
        for a in words[word_off[i]: word_off[i] + r[i]]:
            st = ds[i][a][st]
        assert r[i] >= 0 and len(np.unique(st)) == 1, f"instance {i}: word does not reset"

    # end to end: host automata in, host results out, through sw_batch
    hs = [sw.load(d) for d in ds]
    e2e_t = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        rh, wh = sw.sw_batch(hs, stream=stream, ws=ws, word_cap=word_cap)
        torch.cuda.synchronize()
        barrier()
        if it >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    assert (rh == r).all()
    e2e_s = float(np.mean(e2e_t))
    h2d = int(sum(d.size for d in ds) * 2)  # uint16 transition tables
    d2h = int(4 * count + int(r.sum()))
    # sets the compaction stored per step (every computed level but the roots)
    survivors = 0
    for h in hs:
        fs, bs = sw.sw_level_sizes(h)
        survivors += sum(fs[1:]) + sum(bs[1:])

    # one at a time vs batched, on the same sample
    m = min(args.one_sample, count)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(m):
        sw.sw_reset_threshold(hs[i], stream=stream, ws=ws, word_cap=word_cap)
    torch.cuda.synchronize()
    one_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    sw.sw_batch(hs[:m], stream=stream, ws=ws, word_cap=word_cap)
    torch.cuda.synchronize()
    batch_m_s = time.perf_counter() - t0

    st = stats[-1]
    meet_ms, pairs, iters, rows_t, launches, lw = meet_roofline(stats, nsm)
    ops = iters * 64 * lw + rows_t * 2 * W * 25
    smem_bytes = iters * 256 * lw + rows_t * 8 * W
    sec = meet_ms * 1e-3
    achieved = ops / sec / 1e12 if sec > 0 else 0.0
    clocks = clk.summary()
    cand = sum(s["candidates"] for s in stats) / len(stats)
    expand_ms = sum(s["expand_ms"] for s in stats) / len(stats)
    compact_ms = sum(s["compact_ms"] for s in stats) / len(stats)
    k0 = float(np.mean(ks))
    hbm = {
        "k_expand": hbm_line(expand_ms, cand * (8 * W / k0 + 8 * W + 8 + 8), hbm_peak,
                             "per candidate: 8W/k B of parent read, 8W B written, an 8 B table slot read "
                             "(CAS), 8 B slot index written"),
        "compaction": hbm_line(compact_ms, cand * 18 + survivors * (24 * W + 36), hbm_peak,
                               "per candidate: 8 B slot index and 8 B table slot read, 1 B flag written and "
                               "read; per stored set: 8W B read twice and written once, 8 B parent link, 16 B "
                               "record, 4 B permutation entry and 8 B table slot written"),
    }
    serving = serve_bench(sw, torch, stream, args) if rank == 0 and not args.no_serve else None
    line = {
        "metric": "exact-r instances/sec", "value": value, "unit": "instances/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
        "e2e": {"value": count * world / e2e_s, "unit": "instances/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "kernel": "k_meet_bm", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": (MEET_DRAM_BYTES_PER_ROW * rows_t / max(launches, 1)
                                 if args.workload == "c3" and MEET_DRAM_BYTES_PER_ROW else None),
                     "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum per transposed backward row, "
                                      "measured on the first 512 automata of this workload, times rows per launch",
                     "work": "int32 ops executed: 64 per 64-bit lane word per warp AND step + 25 per transposed "
                             "32-bit row word",
                     "lane_words": lw, "and_steps_per_step": iters, "rows_transposed_per_step": rows_t,
                     "smem_tbs": smem_bytes / sec / 1e12 if sec > 0 else 0.0, "smem_peak_tbs": smem_peak,
                     "pairs_per_step": pairs, "pairs_per_sec_in_kernel": pairs / sec if sec > 0 else 0.0,
                     "launches_per_step": launches, "avg_launch_ms": meet_ms / max(launches, 1),
                     "peak_basis": f"2 ANDs per three-input LOP3 x {lop3_probe:.1f} LOP3/SM/clock measured "
                                   f"(sw_probe_int_peak) x {nsm} SMs x {SM_MAX_MHZ_FALLBACK:.0f} MHz (max SM clock)",
                     "lop3_probe_per_clk_per_sm": lop3_probe},
        "roofline_hbm": hbm,
        "roofline_mark": mark_roofline(stats, lw, W, peak),
        "subset_checks_per_sec": pairs / (ms * 1e-3),
        "kernel_ms_per_step": {"meet": meet_ms, "expand": expand_ms, "compact": compact_ms,
                               "mark": sum(s["mark_ms"] for s in stats) / len(stats),
                               "words": sum(s["words_ms"] for s in stats) / len(stats),
                               "host_wall": sum(s["run_ms"] for s in stats) / len(stats),
                               "host_wait": sum(s["sync_ms"] for s in stats) / len(stats),
                               "host_select": sum(s["select_ms"] for s in stats) / len(stats),
                               "host_update": sum(s["update_ms"] for s in stats) / len(stats),
                               **{k: sum(s[m] for s in stats) / len(stats)
                                  for k, m in (("host_stage", "stage_ms"), ("host_plan", "plan_ms"),
                                               ("host_post", "post_ms"), ("upload_fill_rehash", "table_ms"),
                                               ("between_iterations", "gap_ms"))}},
        "iterations_per_step": st["iterations"], "waves": st["waves"], "evictions": st["evictions"],
        "arena_peak_sets": st["arena_peak"], "candidates_per_step": cand, "stored_sets_per_step": survivors,
        "one_at_a_time": {"value": m / one_s, "unit": "instances/s", "sample": f"first {m} instances",
                          "batched_same_sample": m / batch_m_s},
        "serving": serving,
        "clocks": clocks,
        "gpu_launches": int(st.get("launches", 0)),
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        barrier()  # rank 0 may still have been serving
        dist.destroy_process_group()


def mark_roofline(stats, lw, W, peak):
    """The inclusion-marking kernel (only with sw_options.reduce = 1), on the
    same integer-pipe terms as the meet kernel; None when it did not run."""
    ms = sum(s["mark_ms"] for s in stats) / len(stats)
    if ms <= 0:
        return None
    steps = sum(s["mark_steps"] for s in stats) / len(stats)
    rows = sum(s["mark_rows"] for s in stats) / len(stats)
    ops = steps * 64 * lw + rows * 2 * W * 25
    achieved = ops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "k_mark_bm", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak if peak else None, "ms_per_step": ms, "and_steps_per_step": steps,
            "rows_transposed_per_step": rows, "pairs_per_step": sum(s["mark_pairs"] for s in stats) / len(stats)}


def hbm_peak_gbs():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def hbm_line(ms, nbytes, peak, basis):
    """An HBM-bound kernel's algorithmic bytes per step over its event time."""
    p, src = peak
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return {"bound": "hbm", "achieved": gbs, "peak": p, "unit": "GB/s", "frac": gbs / p if p else None,
            "peak_basis": f"{src} copy bandwidth", "bytes_per_step": nbytes, "ms_per_step": ms, "traffic": None,
            "bytes_basis": basis}


def run_beam(args, d, cfg, sw, torch, local, world):
    """The beam upper bound of Section 2.1.3 on one large automaton: W
    warm-up and K timed calls of sw_beam with beam n * ceil(log2 n)."""
    n = d.shape[1]
    B = n * int(np.ceil(np.log2(n)))
    ws = sw.workspace(int(min(args.ws_gb, 64) * (1 << 30)))
    stream = torch.cuda.Stream()

    def once():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R, w = sw.sw_beam(d, B, stream=stream, ws=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        return R, w, e0.elapsed_time(e1) * 1e-3

    for _ in range(args.warmup):
        once()
    with Clocks(local) as clk:
        runs = [once() for _ in range(args.steps)]
    R, w, _ = runs[-1]
    sec = float(np.mean([x[2] for x in runs]))
    states = np.arange(n)
    for a in w:
        states = d[a][states]
    return {
        "metric": "beam upper bounds/sec", "value": 1.0 / sec, "unit": "instances/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
        "e2e": {"value": 1.0 / sec, "unit": "instances/s", "h2d_bytes_per_step": int(d.size * 2),
                "d2h_bytes_per_step": 4 + R},
        "beam": {"n": n, "beam": B, "R": R, "word_resets": bool(len(np.unique(states)) == 1 and len(w) == R),
                 "seconds": sec, "mean_r_fit_2.284n^0.515": 2.284 * n ** 0.515},
        "clocks": clk.summary(), "cpu_baseline": None,
    }


def run_reference_beam(args, d, cfg):
    """The reference arm of a beam workload: the oracle's beam (oracle.beam)
    with the same beam size, once, on one host core."""
    import oracle
    oracle.build()
    n = d.shape[1]
    B = n * int(np.ceil(np.log2(n)))
    if n > 1000:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle's beam sorts with a bit-by-bit set "
                          f"comparison: about 1e10 operations per level at n={n}, hours for one automaton"}),
              flush=True)
        return
    t0 = time.process_time()
    R, _, _ = oracle.beam(d, B)
    sec = time.process_time() - t0
    print(json.dumps({"impl": "reference", "metric": "beam upper bounds/sec", "value": 1.0 / sec,
                      "unit": "instances/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": sec * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                      "data": "synthetic", "config": cfg, "R": R,
                      "cpu_baseline": {"value": 1.0 / sec, "unit": "instances/s", "cores": 1, "kind": "oracle",
                                       "sample": "the one automaton of the workload, oracle.beam, one core"},
                      "e2e": {"value": 1.0 / sec, "unit": "instances/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def tensor_core_pairs_per_s(torch, K: int, M: int = 16384, N: int = 16384):
    """The ceiling of a tensor-core meet, measured: X subset of Y as a dense
    0/1 contraction (|X intersect Y| = |X|), here a library fp8 GEMM
    (torch._scaled_mm, e4m3 x e4m3 with fp32 accumulation, exact for
    counts <= 576) of M forward rows by N backward sets over K = 64W state
    columns, without the epilogue a meet would add.  Returns pairs/s and
    TFLOP/s, best of 20 after warm-up; None where fp8 GEMMs are missing."""
    try:
        a = (torch.rand(M, K, device="cuda") < 0.3).to(torch.float8_e4m3fn)
        b = (torch.rand(N, K, device="cuda") < 0.5).to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda")

        def f():
            return torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.float32)

        c = f()
        want = a[:64].float() @ b[:64].float().t()
        exact = bool(torch.equal(c[:64, :64], want))
        for _ in range(3):
            f()
        best = None
        for _ in range(20):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            best = t if best is None else min(best, t)
        return {"gemm": "torch._scaled_mm e4m3 x e4m3 -> fp32", "shape_mkn": [M, K, N], "exact": exact,
                "seconds": best, "pairs_per_s": M * N / best, "tflops": 2.0 * M * N * K / best / 1e12}
    except (RuntimeError, TypeError, AttributeError) as e:
        return {"gemm": "torch._scaled_mm e4m3", "unavailable": str(e)[:200]}


def schedules_agree(a, b, words_unique: bool) -> bool:
    """Whether two searches of one automaton under different direction
    schedules agree: a and b are (r, word, forward sizes, backward sizes).
    r and the sizes of every level both computed must be equal; the words
    must be equal only when the search returns a unique word (the plain
    search's least word), not with a reduced side or the inverse phase,
    whose word depends on where the searches met."""
    r, w, fs, bs = a
    r2, w2, fs2, bs2 = b
    m_, mb = min(len(fs), len(fs2)), min(len(bs), len(bs2))
    return r == r2 and fs[:m_] == fs2[:m_] and bs[:mb] == bs2[:mb] and (w == w2 or not words_unique)


def run_hard(args, d, cfg, sw, torch, local, world, peak, nsm):
    """A hard single instance: W warm-up and K timed searches with the
    library's direction rule, then one with "expand the smaller side"
    (a huge SetCost); both must return the same r and word."""
    n = d.shape[1]
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    ws = sw.workspace(min(int(args.ws_gb * (1 << 30)), int(free * 0.8)))
    stream = torch.cuda.Stream()
    h = sw.load(d)

    def once():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r, w = sw.sw_reset_threshold(h, stream=stream, ws=ws, word_cap=4096)
        e1.record(stream)
        torch.cuda.synchronize()
        return r, w, e0.elapsed_time(e1) * 1e-3, sw.sw_last_stats(), sw.sw_level_sizes(h)

    for _ in range(args.warmup):
        once()
    sw.sw_set_timing(True)
    runs = []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            runs.append(once())
    r, w, _, st, (fs, bs) = runs[-1]
    sec = float(np.mean([x[2] for x in runs]))
    if args.one_schedule:
        r2, w2, sec2, st2, (fs2, bs2) = r, w, sec, st, (fs, bs)
    else:
        old = sw.sw_get_options()
        o = sw.sw_get_options()
        o.set_cost = 1e9
        sw.sw_set_options(o)
        r2, w2, sec2, st2, (fs2, bs2) = once()
        sw.sw_set_options(old)
    sw.sw_set_timing(False)
    states = np.arange(n)
    for a in w:
        states = d[a][states]
    opts = sw.sw_get_options()
    agree = schedules_agree((r, w, fs, bs), (r2, w2, fs2, bs2),
                            words_unique=opts.reduce == 0 and opts.dfs_sets == 0)
    meet_ms, pairs, iters, rows_t, launches, lw = meet_roofline([x[3] for x in runs], nsm)
    W = (n + 63) // 64
    ops = iters * 64 * lw + rows_t * 2 * W * 25
    achieved = ops / (meet_ms * 1e-3) / 1e12 if meet_ms > 0 else 0.0
    return {
        "metric": "exact-r instances/sec", "value": 1.0 / sec, "unit": "instances/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
        "e2e": {"value": 1.0 / sec, "unit": "instances/s", "h2d_bytes_per_step": int(d.size * 2),
                "d2h_bytes_per_step": 4 + r},
        "hard": {"n": n, "r": r, "word_resets": bool(len(np.unique(states)) == 1 and len(w) == r),
                 "seconds": sec, "fwd_levels": len(fs) - 1, "bwd_levels": len(bs) - 1,
                 "peak_sets": st["arena_peak"], "pairs": st["pairs"], "pairs_per_s": st["pairs"] / sec,
                 "pairs_per_s_in_meet_kernel": pairs / (meet_ms * 1e-3) if meet_ms > 0 else None,
                 "meet_ms": meet_ms, "expand_ms": st["expand_ms"], "compact_ms": st["compact_ms"],
                 "mark_ms": st["mark_ms"], "mark_pairs": st["mark_pairs"],
                 "inverse_phase": {"ran": bool(st["dfs_instances"]), "chunks": st["dfs_chunks"],
                                   "sets": st["dfs_sets"], "depth": r - (len(fs) - 1) - (len(bs) - 1)},
                 "balanced_schedule": {"r": r2, "seconds": sec2, "peak_sets": st2["arena_peak"],
                                       "pairs": st2["pairs"], "fwd_levels": len(fs2) - 1,
                                       "bwd_levels": len(bs2) - 1},
                 "schedules_agree": None if args.one_schedule else bool(agree),
                 "tensor_core_meet_ceiling": tensor_core_pairs_per_s(torch, 64 * W)},
        "roofline": {"bound": "alu", "kernel": "k_meet_bm", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak if peak else None, "traffic": None, "lane_words": lw},
        "clocks": clk.summary(), "gpu_launches": int(st["launches"]), "cpu_baseline": None,
    }


if __name__ == "__main__":
    main()
