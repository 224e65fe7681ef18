"""The library's measurement probes on the GPU: the L2 read rate and the
random-row fetch rate that bound the gather phase."""
import pytest

pytestmark = pytest.mark.gpu


def test_l2_read_probe_gives_a_plausible_rate():
    import paper_2006_06743_gb300 as sng
    gbs = sng.measure_l2_read(48 << 20, 20)
    assert 500.0 < gbs < 200_000.0


@pytest.mark.parametrize("row_bytes", [64, 128, 256])
def test_random_row_probe_gives_a_plausible_rate(row_bytes):
    import paper_2006_06743_gb300 as sng
    r = sng.measure_random_rows(1 << 20, row_bytes, 1 << 24)
    # more than 10^8 rows/s, and no more bytes per second than a generous
    # bound on what the SMs can read from L2
    assert 1e8 < r and r * row_bytes < 100e12


def test_random_row_probe_rate_grows_with_warps_in_flight():
    import paper_2006_06743_gb300 as sng
    lo = sng.measure_random_rows(1 << 20, 128, 1 << 25, blocks_per_sm=1)
    hi = sng.measure_random_rows(1 << 20, 128, 1 << 25, blocks_per_sm=4)
    assert hi > 1.5 * lo
