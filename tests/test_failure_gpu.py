"""Failure detection without a GPU fault: a bounded device wait that runs out
reports SCAN_ETIMEOUT, and the context keeps working afterwards."""
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


def test_bounded_wait_times_out_and_context_survives():
    for limit_ns in (1_000_000, 20_000_000):
        st = gbscan.load().scan_selftest_wait_timeout(limit_ns, None)
        assert st == gbscan.SCAN_ETIMEOUT, gbscan.load().scan_last_error()
    v = synth.uniform_values(3, 50_000, 11)
    col = gbscan.Column.from_host(v, 11)
    assert col.run(10, 900).pair() == oracle.scan_values(v, 10, 900)
    col.close()


def test_bad_arguments_are_refused_before_any_launch():
    assert gbscan.load().scan_selftest_wait_timeout(0, None) == gbscan.SCAN_EINVAL
    with pytest.raises(gbscan.ScanError) as e:
        gbscan.Column.from_host(synth.uniform_values(1, 10, 4), 40)
    assert e.value.status == gbscan.SCAN_EINVAL
