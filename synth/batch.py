"""Seeded batches of many small pangenome graphs, and their concatenation.

A batch is n_graphs independent graphs from the single-graph generator
(``make_graph`` with the "mid" variation parameters), each with its own
generator seed: node counts log-uniform in [nodes_lo, nodes_hi] (the backbone
is sized so that backbone plus bubble nodes come to about that count) and
path counts uniform in [paths_lo, paths_hi]. Only inputs are built here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .pangenome import CONFIGS, Graph, make_graph

#: The batch workload: 256 subgraphs, 1 k - 200 k nodes, 4 - 90 paths.
BATCH_CONFIGS = {
    "batch256": dict(n_graphs=256, nodes=(1_000, 200_000), paths=(4, 90), seed=11, base="mid"),
    "batch_small": dict(n_graphs=12, nodes=(1_000, 12_000), paths=(4, 12), seed=5, base="mid"),
    # the same distributions, a quarter of the graphs: a profiling case of ~1.5 GB
    "batch_prof": dict(n_graphs=64, nodes=(1_000, 200_000), paths=(4, 90), seed=13, base="mid"),
}


def batch_shapes(n_graphs, nodes, paths, seed):
    """(node count, path count, generator seed) of every graph."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(nodes[0]), np.log(nodes[1])
    v = np.rint(np.exp(rng.uniform(lo, hi, size=n_graphs))).astype(np.int64)
    p = rng.integers(paths[0], paths[1] + 1, size=n_graphs)
    gs = rng.integers(1, 2**31 - 1, size=n_graphs)
    return [(int(a), int(b), int(c)) for a, b, c in zip(v, p, gs)]


def make_batch(name_or_cfg="batch256", indices=None, **overrides) -> list[Graph]:
    """The batch's graphs (only those at `indices`, if given)."""
    cfg = dict(BATCH_CONFIGS[name_or_cfg]) if isinstance(name_or_cfg, str) else dict(name_or_cfg)
    cfg.update(overrides)
    base = dict(CONFIGS[cfg["base"]])
    shapes = batch_shapes(cfg["n_graphs"], cfg["nodes"], cfg["paths"], cfg["seed"])
    graphs = []
    for k in (range(len(shapes)) if indices is None else indices):
        v, p, gs = shapes[k]
        backbone = max(2, int(round(v / (1.0 + base["p_site"]))))
        graphs.append(make_graph(base, gen_seed=gs, backbone=backbone, paths=p))
    return graphs


@dataclass
class BatchArrays:
    """The graphs concatenated as pgsgd_batch_create takes them (local node ids)."""
    graph_node_off: np.ndarray  # uint64 [G + 1]
    graph_path_off: np.ndarray  # uint64 [G + 1]
    node_len: np.ndarray        # uint32 [V]
    path_off: np.ndarray        # uint64 [P + 1]
    step_node: np.ndarray       # uint32 [S], local to the step's graph
    step_rev: np.ndarray        # uint8 [S]
    step_pos: np.ndarray        # int64 [S]
    init_xy: np.ndarray         # float64 [V, 4]

    @property
    def n_graphs(self) -> int:
        return int(self.graph_node_off.shape[0] - 1)

    def graph_xy(self, xy, g):
        """Rows of graph g in a [V, 4] batch layout."""
        return xy[int(self.graph_node_off[g]):int(self.graph_node_off[g + 1])]


def concat(graphs) -> BatchArrays:
    G = len(graphs)
    gno = np.zeros(G + 1, np.uint64)
    gpo = np.zeros(G + 1, np.uint64)
    gno[1:] = np.cumsum([g.n_nodes for g in graphs])
    gpo[1:] = np.cumsum([g.n_paths for g in graphs])
    steps = np.cumsum([0] + [g.n_steps for g in graphs])
    path_off = np.concatenate([np.zeros(1, np.uint64)] +
                              [g.path_off[1:] + np.uint64(steps[k]) for k, g in enumerate(graphs)])
    return BatchArrays(graph_node_off=gno, graph_path_off=gpo,
                       node_len=np.concatenate([g.node_len for g in graphs]),
                       path_off=path_off.astype(np.uint64),
                       step_node=np.concatenate([g.step_node for g in graphs]),
                       step_rev=np.concatenate([g.step_rev for g in graphs]),
                       step_pos=np.concatenate([g.step_pos for g in graphs]),
                       init_xy=np.concatenate([g.init_xy for g in graphs]))
