"""Path stress (Eq. 1) on the GPU: equal to the oracle's brute force on the
same layout, and tracked by the sampled path stress (Eq. 2) across layouts of
different quality (Section VI-B, Fig. 11: correlation 0.995)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from synth import make_custom, make_graph

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pg():
    import paper_2409_00876_gb300 as pg
    pg.load_library()
    return pg


def test_hand_worked_three_node_layout(pg):
    gold = json.load(open(os.path.join(GOLDEN, "path_stress_3node.json")))
    g = make_custom([2, 3, 1], [[(0, 0), (1, 0), (2, 0)]], init_xy=np.array(gold["layout"], np.float64))
    G = pg.Graph.from_synth(g)
    G.set_coords(g.init_xy)
    val, pairs = G.full_stress()
    assert pairs == 3
    assert abs(val - float(Fraction(*gold["path_stress"]))) <= 1e-6


@pytest.mark.parametrize("iters", [0, 3, 30])
def test_full_stress_matches_oracle(pg, iters):
    g = make_graph("tiny")
    G = pg.Graph.from_synth(g)
    G.set_coords(g.init_xy)
    if iters:
        G.layout(30, theta=0.99, seed=2, iter_end=iters)
    xy = G.get_coords()
    val, pairs = G.full_stress()
    want, want_pairs = O.full_stress(g, xy)
    assert pairs == want_pairs
    assert abs(val - want) <= 1e-5 * want


def test_sampled_stress_tracks_full_stress_on_gpu(pg):
    g = make_graph("tiny", backbone=400, paths=6)
    rng = np.random.default_rng(4)
    full, samp = [], []
    for k in range(40):
        G = pg.Graph.from_synth(g)
        G.set_coords(g.init_xy + rng.normal(0, 1 + 10 * (k % 5), g.init_xy.shape))
        its = int(rng.integers(0, 31))
        if its:
            G.layout(30, theta=0.99, seed=k, iter_end=its)
        full.append(G.full_stress()[0])
        samp.append(G.stress(100, seed=k)["mean"])
    r = np.corrcoef(np.log(full), np.log(samp))[0, 1]
    assert r > 0.97, r
