"""Write tests/golden/oracle_batch_small.json: the CPU oracle's layout quality
on every graph of the small batch workload (12 graphs, 1 k - 12 k nodes,
4 - 12 paths).

For each graph and layout seed this runs Algorithm 1 in the oracle (FP64,
one thread: the sequential reading of the method) from the generator's
initial layout and records the sampled path stress (Eq. 2) of the result
under a fixed stress seed. Only the oracle and the input generator are
called; graphs run in parallel worker processes.

    python tests/golden/make_batch_goldens.py [--workers 4]
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_batch_small.json")
SEEDS = [1, 2, 3]
T = 30
THETA = 0.99
PER_STEP = 100
STRESS_SEED = 7


def _one(k):
    import oracle as O
    from synth import make_batch
    g = make_batch("batch_small")[k]
    t0 = time.time()
    init = O.sampled_stress(g, g.init_xy, per_step=PER_STEP, seed=STRESS_SEED)["mean"]
    runs = []
    for s in SEEDS:
        xy, _ = O.layout(g, g.init_xy, T=T, theta=THETA, seed=s, n_threads=1)
        runs.append(O.sampled_stress(g, xy, per_step=PER_STEP, seed=STRESS_SEED)["mean"])
    return k, dict(n_nodes=g.n_nodes, n_paths=g.n_paths, n_steps=g.n_steps, init_stress=init, stress=runs,
                   seconds=round(time.time() - t0, 1))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    from synth import BATCH_CONFIGS
    n = BATCH_CONFIGS["batch_small"]["n_graphs"]
    from bench import strip_comments  # the oracle source's hash ignores comments and white-space layout
    sha = hashlib.sha1(strip_comments(open(os.path.join(ROOT, "oracle", "pgsgd_oracle.c")).read()).encode()).hexdigest()[:12]
    graphs = [None] * n
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for k, rec in pool.imap_unordered(_one, range(n)):
            graphs[k] = rec
            print(k, rec, flush=True)
    data = dict(workload="batch_small", oracle_sha=sha, iterations=T, theta=THETA, updates_per_step=10,
                seeds=SEEDS, stress_samples_per_step=PER_STEP, stress_seed=STRESS_SEED, graphs=graphs)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
