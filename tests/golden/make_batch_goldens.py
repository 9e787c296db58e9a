"""Write the CPU oracle's per-graph layout quality for the batch workloads:

- tests/golden/oracle_batch_small.json: every graph of the small batch
  workload (12 graphs, 1 k - 12 k nodes, 4 - 12 paths), layout seeds 1-128,
  one thread (the sequential reading of the method); single layouts of
  1 k-node graphs vary by tens of percent from seed to seed, so the
  comparison needs this many seeds to resolve a few percent;
- tests/golden/oracle_batch_highpath.json: four small graphs of the
  256-subgraph workload with many paths per node (1.1 k - 3.9 k nodes,
  65 - 88 paths), layout seeds 1-16, one thread: the graphs where many
  updates meet few nodes;
- tests/golden/oracle_batch256_subset.json: a fixed subset of 16 graphs of
  the 256-subgraph workload spanning its size range (the graphs at 16 evenly
  spaced ranks 0..240 of 256 by size), each under the layout
  seed the batch gives it (graph index + 1); one thread below 1 M steps,
  Hogwild! threads above.

For each graph and layout seed this runs Algorithm 1 in the oracle (FP64)
from the generator's initial layout and records the sampled path stress
(Eq. 2) of the result under a fixed stress seed. Only the oracle and the
input generator are called; graphs run in parallel worker processes.

    python tests/golden/make_batch_goldens.py [--workload batch_small|highpath|batch256] [--workers 4]
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))
T = 30
THETA = 0.99
PER_STEP = 100
STRESS_SEED = 7
SMALL_SEEDS = list(range(1, 129))
SEED_CHUNK = 16              # seeds per worker job (the small record)
HIGHPATH_INDICES = [73, 52, 21, 80]  # batch256 graphs of 1,097, 1,336, 2,951 and 3,928 nodes, 65-88 paths
HIGHPATH_SEEDS = list(range(1, 17))
SUBSET_SIZE = 16
SUBSET_TOP_RANK = 240       # ranks 0..240 of 256 by step count: the largest graphs stay out (CPU time)
THREADED_ABOVE = 1_000_000  # steps; larger subset graphs use Hogwild! threads


def subset_indices():
    """Graph indices of the batch256 subset: 16 evenly spaced ranks (0 to 240)
    of the graphs ordered by node count x path count (the size of their path
    data), from the batch's shape table alone."""
    from synth import BATCH_CONFIGS, batch_shapes
    cfg = BATCH_CONFIGS["batch256"]
    shapes = batch_shapes(cfg["n_graphs"], cfg["nodes"], cfg["paths"], cfg["seed"])
    size = np.array([v * p for v, p, _ in shapes], dtype=np.float64)
    order = np.argsort(size, kind="stable")
    return [int(order[int(round(q))]) for q in np.linspace(0, SUBSET_TOP_RANK, SUBSET_SIZE)]


def _one(job):
    import oracle as O
    from synth import make_batch
    workload, k, seeds, threads = job
    g = make_batch(workload, indices=[k])[0]
    if threads is None:
        threads = 1 if g.n_steps <= THREADED_ABOVE else max(1, (os.cpu_count() or 2) // 2)
    t0 = time.time()
    init = O.sampled_stress(g, g.init_xy, per_step=PER_STEP, seed=STRESS_SEED)["mean"]
    runs = []
    for s in seeds:
        xy, _ = O.layout(g, g.init_xy, T=T, theta=THETA, seed=s, n_threads=threads)
        runs.append(O.sampled_stress(g, xy, per_step=PER_STEP, seed=STRESS_SEED)["mean"])
    return k, dict(index=k, n_nodes=g.n_nodes, n_paths=g.n_paths, n_steps=g.n_steps, init_stress=init,
                   seeds=seeds, stress=runs, oracle_threads=threads, seconds=round(time.time() - t0, 1))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="batch_small", choices=["batch_small", "batch256", "highpath"])
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    from synth import BATCH_CONFIGS
    from bench import strip_comments  # the oracle source's hash ignores comments and white-space layout
    sha = hashlib.sha1(strip_comments(open(os.path.join(ROOT, "oracle", "pgsgd_oracle.c")).read()).encode()).hexdigest()[:12]
    if args.workload == "batch_small":
        idx = list(range(BATCH_CONFIGS["batch_small"]["n_graphs"]))
        jobs = [("batch_small", k, SMALL_SEEDS[c:c + SEED_CHUNK], 1) for k in idx
                for c in range(0, len(SMALL_SEEDS), SEED_CHUNK)]
        out = os.path.join(HERE, "oracle_batch_small.json")
    elif args.workload == "highpath":
        idx = HIGHPATH_INDICES
        jobs = [("batch256", k, HIGHPATH_SEEDS[c:c + SEED_CHUNK // 4], 1) for k in idx
                for c in range(0, len(HIGHPATH_SEEDS), SEED_CHUNK // 4)]
        out = os.path.join(HERE, "oracle_batch_highpath.json")
    else:
        idx = subset_indices()
        jobs = [("batch256", k, [k + 1], None) for k in idx]
        out = os.path.join(HERE, "oracle_batch256_subset.json")
    recs = {}
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for k, rec in pool.imap_unordered(_one, jobs):
            if k in recs:  # another chunk of this graph's seeds
                have = recs[k]
                pairs = sorted(zip(have["seeds"] + rec["seeds"], have["stress"] + rec["stress"]))
                have["seeds"], have["stress"] = [a for a, _ in pairs], [b for _, b in pairs]
                have["seconds"] = round(have["seconds"] + rec["seconds"], 1)
            else:
                recs[k] = rec
            print(k, rec["seeds"][0], len(rec["seeds"]), rec["seconds"], flush=True)
    graphs = [recs[k] for k in idx]
    data = dict(workload=args.workload, oracle_sha=sha, iterations=T, theta=THETA, updates_per_step=10,
                stress_samples_per_step=PER_STEP, stress_seed=STRESS_SEED, graphs=graphs)
    if args.workload == "highpath":
        data["source_workload"] = "batch256"
        data["seeds"] = HIGHPATH_SEEDS
        for g in graphs:
            g.pop("oracle_threads")
    if args.workload == "batch_small":
        data["seeds"] = SMALL_SEEDS
        for g in graphs:  # the small record keeps its original per-graph fields
            for f in ("index", "seeds", "oracle_threads"):
                g.pop(f)
    with open(out, "w") as f:
        json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
