"""The in-repo L2 and HBM random-read probes that set the rooflines of the update kernel."""
import pytest

pytestmark = pytest.mark.gpu


def test_l2_bandwidth_is_plausible():
    import paper_2409_00876_gb300 as pg
    stream = pg.l2_bandwidth(64 << 20, 10, 0)
    rand = pg.l2_bandwidth(64 << 20, 2, 1)
    # above any HBM3e figure and below an absurd bound; random sectors cost more than streaming
    assert 5_000 < stream < 200_000, stream
    assert 500 < rand < stream * 1.5, (rand, stream)


def test_hbm_random_read_rate_is_plausible():
    import paper_2409_00876_gb300 as pg
    steps = pg.hbm_gather_rate(4 << 30, 2, 0)
    with_nodes = pg.hbm_gather_rate(4 << 30, 2, 1)
    # every read costs at least one 32-byte sector of DRAM traffic, which cannot exceed
    # ~1.5x the copy peak; and a random read rate below 1e9/s would mean a broken probe
    for r in (steps, with_nodes):
        assert 1e9 < r < 1.5 * 8e12 / 32, (steps, with_nodes)
