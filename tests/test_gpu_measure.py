"""num_measure_gather_rate: the random-read ceiling that bench.py reports the kernels against."""
import pytest

pytestmark = pytest.mark.gpu


def test_gather_rate_is_plausible_and_cache_sensitive():
    from paper_2509_10722_b300 import capi
    big4 = capi.num_measure_gather_rate(20_000_000, 10_000_000, 4, 2)  # 40 MB vector
    big8 = capi.num_measure_gather_rate(20_000_000, 1_000_000, 8, 2)   # 8 MB vector
    small = capi.num_measure_gather_rate(20_000_000, 4096, 4, 2)       # 16 KB: stays in L1
    for r in (big4, big8, small):
        assert 1e9 < r < 1e13, r
    # reads served by L1 come back faster than reads that go to L2
    assert small > 1.3 * big4, (small, big4)


@pytest.mark.parametrize("count,vec_len,vec_bytes,repeats", [
    (0, 100, 4, 1), (100, 0, 4, 1), (100, 100, 3, 1), (100, 100, 4, 0),
    (100, 2**31, 4, 1), (100, 100, 4, 1001)])
def test_gather_rate_rejects_bad_arguments(count, vec_len, vec_bytes, repeats):
    from paper_2509_10722_b300 import capi
    with pytest.raises(capi.NumError) as e:
        capi.num_measure_gather_rate(count, vec_len, vec_bytes, repeats)
    assert e.value.code == capi.NUM_ERR_INVALID


def test_scatter_rate_is_plausible_and_below_the_gather_rate():
    """Random plain stores: measured at about 184 G/s into an L2-resident 40 MB vector
    against about 270 G/s for reads, and at about 34 G/s into a 220 MB one (partial-sector
    writes beyond the L2), which is why no kernel here pushes values to a permuted copy."""
    from paper_2509_10722_b300 import capi
    st = capi.num_measure_scatter_rate(20_000_000, 10_000_000, 4, 2)
    ld = capi.num_measure_gather_rate(20_000_000, 10_000_000, 4, 2)
    assert 1e9 < st < 1e13, st
    assert st < 1.2 * ld, (st, ld)


def test_scatter_rate_rejects_bad_arguments():
    from paper_2509_10722_b300 import capi
    with pytest.raises(capi.NumError) as e:
        capi.num_measure_scatter_rate(100, 100, 2, 1)
    assert e.value.code == capi.NUM_ERR_INVALID
