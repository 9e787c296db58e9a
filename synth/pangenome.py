"""Seeded synthetic pangenome graphs shaped like the paper's workloads.

The paper lays out HPRC chromosome graphs and the HLA-DRB1 / MHC graphs
(Section III, Table I; Section VII-A, Table VI). None of those datasets is
available here, so these generators stand in for them. A graph is a linear
backbone of nodes that every path follows, with the variation the paper's
Section II-A describes:

* substitution bubbles: a backbone node that is a variant site owns one
  alternative node of the same length; a path takes the alternative with a
  fixed probability (0.5 per path at a site, so 0.05 per node when 10 % of the
  nodes are sites);
* deletions: a path skips a node;
* inversions: a path traverses a run of nodes in reverse order and reverse
  orientation;
* tandem duplications: a path re-traverses the run of nodes just behind it.

Node ids: backbone nodes are 0..B-1 in backbone order; alternative nodes follow
as B..B+sites-1. Every path step stores its node id, its orientation
(1 = reverse) and the int64 nucleotide position at which the path enters it.

The initial layout (a caller input: the paper does not say how it is made)
puts each node on the x axis at its backbone nucleotide position, from
x = pos to x = pos + len, y = 0 (an alternative node takes its site's
position), then adds N(0, 1) jitter to all four coordinates and rounds them to
FP32. It is returned as float64 holding FP32-representable values.

All randomness comes from numpy's PCG64, seeded by ``gen_seed``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

#: The three single-graph workloads: tiny (oracle runs in seconds), mid, and a
#: chromosome-scale graph of 5 M backbone nodes and 90 paths.
CONFIGS = {
    "tiny": dict(backbone=2_000, paths=8, len_mean=8.0, len_cap=1024,
                 tail_prob=0.0, tail_range=(1_000, 100_000),
                 p_site=0.1, p_alt=0.5, p_del=0.01,
                 p_inv=0.002, inv_len=(5, 50), p_dup=0.0, dup_len=(10, 200),
                 gen_seed=1),
    "mid": dict(backbone=200_000, paths=32, len_mean=8.0, len_cap=1024,
                tail_prob=0.0, tail_range=(1_000, 100_000),
                p_site=0.1, p_alt=0.5, p_del=0.01,
                p_inv=0.002, inv_len=(5, 50), p_dup=0.001, dup_len=(10, 200),
                gen_seed=2),
    "chrom": dict(backbone=5_000_000, paths=90, len_mean=30.0, len_cap=100_000,
                  tail_prob=1e-4, tail_range=(1_000, 100_000),
                  p_site=0.1, p_alt=0.5, p_del=0.01,
                  p_inv=0.0005, inv_len=(5, 50), p_dup=0.0005, dup_len=(10, 200),
                  gen_seed=3),
}


@dataclass
class Graph:
    node_len: np.ndarray   # uint32 [V]
    path_off: np.ndarray   # uint64 [P + 1]; path p owns steps [off[p], off[p+1])
    step_node: np.ndarray  # uint32 [S]
    step_rev: np.ndarray   # uint8  [S]
    step_pos: np.ndarray   # int64  [S]; nucleotide position where the step starts
    init_xy: np.ndarray    # float64 [V, 4] = (sx, sy, ex, ey), FP32-representable
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.node_len.shape[0])

    @property
    def n_paths(self) -> int:
        return int(self.path_off.shape[0] - 1)

    @property
    def n_steps(self) -> int:
        return int(self.path_off[-1])

    def path_lengths(self) -> np.ndarray:
        return np.diff(self.path_off.astype(np.int64))

    def path_nt_lengths(self) -> np.ndarray:
        """Nucleotide length of every path (0 for an empty path)."""
        off = self.path_off.astype(np.int64)
        out = np.zeros(self.n_paths, dtype=np.int64)
        nz = off[1:] > off[:-1]
        last = off[1:][nz] - 1
        out[nz] = self.step_pos[last] + self.node_len[self.step_node[last]].astype(np.int64)
        return out


def _node_lengths(rng, n, len_mean, len_cap, tail_prob, tail_range):
    lens = rng.geometric(1.0 / len_mean, size=n).astype(np.int64)
    np.minimum(lens, len_cap, out=lens)
    if tail_prob > 0:
        n_tail = rng.binomial(n, tail_prob)
        if n_tail:
            where = rng.choice(n, size=n_tail, replace=False)
            lo, hi = np.log(tail_range[0]), np.log(tail_range[1])
            lens[where] = np.rint(np.exp(rng.uniform(lo, hi, size=n_tail))).astype(np.int64)
    return lens.astype(np.uint32)


def _event_positions(rng, n, prob):
    """Sorted positions in [0, n) of independent Bernoulli(prob) events."""
    if prob <= 0:
        return np.zeros(0, dtype=np.int64)
    k = rng.binomial(n, prob)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def _one_path(rng, cfg, n_back, site_alt, node_len):
    """Return (node ids, orientations) of one path over the backbone."""
    inv = _event_positions(rng, n_back, cfg["p_inv"])
    dup = _event_positions(rng, n_back, cfg["p_dup"])
    ev_pos = np.concatenate([inv, dup])
    ev_kind = np.concatenate([np.zeros(len(inv), np.int8), np.ones(len(dup), np.int8)])
    order = np.argsort(ev_pos, kind="stable")
    ev_pos, ev_kind = ev_pos[order], ev_kind[order]
    ilo, ihi = cfg["inv_len"]
    dlo, dhi = cfg["dup_len"]
    ev_len = np.where(ev_kind == 0,
                      rng.integers(ilo, ihi + 1, size=len(ev_pos)),
                      rng.integers(dlo, dhi + 1, size=len(ev_pos)))
    pieces_idx, pieces_rev = [], []
    cursor = 0
    for pos, kind, ln in zip(ev_pos.tolist(), ev_kind.tolist(), ev_len.tolist()):
        if pos < cursor:
            continue  # inside an inversion already emitted
        if kind == 0:  # inversion of [pos, pos + ln)
            end = min(pos + ln, n_back)
            pieces_idx.append(np.arange(cursor, pos, dtype=np.int64))
            pieces_rev.append(np.zeros(pos - cursor, np.uint8))
            pieces_idx.append(np.arange(end - 1, pos - 1, -1, dtype=np.int64))
            pieces_rev.append(np.ones(end - pos, np.uint8))
            cursor = end
        else:  # after node pos, revisit the ln nodes ending at pos
            pieces_idx.append(np.arange(cursor, pos + 1, dtype=np.int64))
            pieces_rev.append(np.zeros(pos + 1 - cursor, np.uint8))
            start = max(0, pos + 1 - ln)
            pieces_idx.append(np.arange(start, pos + 1, dtype=np.int64))
            pieces_rev.append(np.zeros(pos + 1 - start, np.uint8))
            cursor = pos + 1
    pieces_idx.append(np.arange(cursor, n_back, dtype=np.int64))
    pieces_rev.append(np.zeros(n_back - cursor, np.uint8))
    bb = np.concatenate(pieces_idx)
    rev = np.concatenate(pieces_rev)
    # deletions: drop each visit with probability p_del
    dels = _event_positions(rng, len(bb), cfg["p_del"])
    if len(dels):
        keep = np.ones(len(bb), bool)
        keep[dels] = False
        bb, rev = bb[keep], rev[keep]
    # bubbles: at a site, take the alternative node with probability p_alt
    node = bb.copy()
    at_site = np.nonzero(site_alt[bb] >= 0)[0]
    take = at_site[rng.random(len(at_site)) < cfg["p_alt"]]
    node[take] = site_alt[bb[take]]
    return node.astype(np.uint32), rev


def _assemble(node_len, paths, init_xy, meta):
    lens = np.array([len(n) for n, _ in paths], dtype=np.uint64)
    path_off = np.zeros(len(paths) + 1, dtype=np.uint64)
    np.cumsum(lens, out=path_off[1:])
    S = int(path_off[-1])
    step_node = np.empty(S, np.uint32)
    step_rev = np.empty(S, np.uint8)
    step_pos = np.empty(S, np.int64)
    for p, (n, r) in enumerate(paths):
        a, b = int(path_off[p]), int(path_off[p + 1])
        step_node[a:b] = n
        step_rev[a:b] = r
        if b > a:
            nl = node_len[n].astype(np.int64)
            step_pos[a] = 0
            np.cumsum(nl[:-1], out=step_pos[a + 1:b])
    return Graph(node_len=node_len, path_off=path_off, step_node=step_node,
                 step_rev=step_rev, step_pos=step_pos, init_xy=init_xy, meta=meta)


def _init_layout(rng, x_start, node_len):
    V = len(node_len)
    xy = np.empty((V, 4), dtype=np.float64)
    xy[:, 0] = x_start
    xy[:, 1] = 0.0
    xy[:, 2] = x_start + node_len.astype(np.float64)
    xy[:, 3] = 0.0
    xy += rng.standard_normal((V, 4))
    return xy.astype(np.float32).astype(np.float64)


def make_graph(name_or_cfg, gen_seed=None, **overrides) -> Graph:
    """Build one of CONFIGS (by name) or a config dict, seeded by gen_seed."""
    if isinstance(name_or_cfg, str):
        cfg = dict(CONFIGS[name_or_cfg])
        name = name_or_cfg
    else:
        cfg = dict(name_or_cfg)
        name = cfg.get("name", "custom")
    cfg.update(overrides)
    if gen_seed is not None:
        cfg["gen_seed"] = gen_seed
    rng = np.random.Generator(np.random.PCG64(cfg["gen_seed"]))
    B = int(cfg["backbone"])
    back_len = _node_lengths(rng, B, cfg["len_mean"], cfg["len_cap"],
                             cfg["tail_prob"], cfg["tail_range"])
    sites = np.nonzero(rng.random(B) < cfg["p_site"])[0]
    site_alt = np.full(B, -1, dtype=np.int64)
    site_alt[sites] = B + np.arange(len(sites))
    node_len = np.concatenate([back_len, back_len[sites]]).astype(np.uint32)
    paths = [_one_path(rng, cfg, B, site_alt, node_len) for _ in range(int(cfg["paths"]))]
    back_pos = np.zeros(B, np.int64)
    np.cumsum(back_len[:-1].astype(np.int64), out=back_pos[1:])
    x_start = np.concatenate([back_pos, back_pos[sites]]).astype(np.float64)
    init_xy = _init_layout(rng, x_start, node_len)
    meta = dict(name=name, **{k: v for k, v in cfg.items()},
                sites=int(len(sites)))
    return _assemble(node_len, paths, init_xy, meta)


def make_custom(node_len, paths, init_xy=None, seed=0) -> Graph:
    """Graph from explicit node lengths and paths given as lists of
    (node id, orientation) pairs. The default layout is a jittered line."""
    node_len = np.asarray(node_len, dtype=np.uint32)
    ps = []
    for path in paths:
        if len(path):
            arr = np.asarray(path, dtype=np.int64).reshape(-1, 2)
            ps.append((arr[:, 0].astype(np.uint32), arr[:, 1].astype(np.uint8)))
        else:
            ps.append((np.zeros(0, np.uint32), np.zeros(0, np.uint8)))
    if init_xy is None:
        rng = np.random.Generator(np.random.PCG64(seed))
        x = np.zeros(len(node_len), np.float64)
        np.cumsum(node_len[:-1].astype(np.float64), out=x[1:])
        init_xy = _init_layout(rng, x, node_len)
    return _assemble(node_len, ps, np.asarray(init_xy, np.float64), dict(name="custom"))


def make_linear_path(n_nodes, len_mean=8.0, seed=0, jitter=1.0) -> Graph:
    """One path visiting n_nodes forward nodes in order. Its exact zero-stress
    layout is every node on a line at its nucleotide position."""
    rng = np.random.Generator(np.random.PCG64(seed))
    node_len = rng.geometric(1.0 / len_mean, size=n_nodes).astype(np.uint32)
    path = [(v, 0) for v in range(n_nodes)]
    x = np.zeros(n_nodes, np.float64)
    np.cumsum(node_len[:-1].astype(np.float64), out=x[1:])
    xy = np.stack([x, np.zeros_like(x), x + node_len, np.zeros_like(x)], axis=1)
    xy = (xy + jitter * rng.standard_normal(xy.shape)).astype(np.float32).astype(np.float64)
    return make_custom(node_len, [path], init_xy=xy)
