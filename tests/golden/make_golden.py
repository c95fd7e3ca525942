"""Writes tests/golden/c3_sample.json: r and the least reset word, computed by
the CPU oracle alone (oracle.bidir), for a sample of the instances of the
4096-automaton workload (n uniform in [64, 192], k = 2, seeds 0..4095).

Sample: every 64th seed; an instance whose oracle run exceeds the per-instance
time cap is left out (the file lists which).  Run from the repository root:
    python tests/golden/make_golden.py [cap_seconds]
"""

import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(ROOT, "tests", "golden", "c3_sample.json")


def one(seed):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2207_05495_gb300 import gen
    d = gen.random_automaton_ranged(64, 192, 2, seed)
    t = time.time()
    r, w, fs, bs = oracle.bidir(d)
    return {"seed": seed, "n": int(d.shape[1]), "r": r, "word": w, "oracle_s": round(time.time() - t, 2)}


def main():
    cap = float(sys.argv[1]) if len(sys.argv) > 1 else 300.0
    seeds = list(range(0, 4096, 64))
    ctx = mp.get_context("spawn")
    out, skipped = [], []
    with ctx.Pool(os.cpu_count()) as pool:
        jobs = {s: pool.apply_async(one, (s,)) for s in seeds}
        t0 = time.time()
        for s in seeds:
            try:
                out.append(jobs[s].get(timeout=max(1.0, cap - (time.time() - t0))))
            except mp.TimeoutError:
                skipped.append(s)
        pool.terminate()
    doc = {"_about": "CPU oracle (oracle.bidir) results for every 64th seed of the workload "
                     "'4096 random binary automata, n~U[64,192], k=2'; written by tests/golden/make_golden.py",
           "cap_seconds": cap, "skipped_seeds": skipped, "instances": sorted(out, key=lambda e: e["seed"])}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=1)
    print(f"wrote {len(out)} instances, skipped {len(skipped)}")


if __name__ == "__main__":
    main()
