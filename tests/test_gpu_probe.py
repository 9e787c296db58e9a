"""The in-repo L2 bandwidth probe that sets the roofline of L2-resident graphs."""
import pytest

pytestmark = pytest.mark.gpu


def test_l2_bandwidth_is_plausible():
    import paper_2409_00876_gb300 as pg
    stream = pg.l2_bandwidth(64 << 20, 10, 0)
    rand = pg.l2_bandwidth(64 << 20, 2, 1)
    # above any HBM3e figure and below an absurd bound; random sectors cost more than streaming
    assert 5_000 < stream < 200_000, stream
    assert 500 < rand < stream * 1.5, (rand, stream)
