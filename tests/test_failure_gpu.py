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


def test_select_waits_on_a_silent_cta_give_up_and_the_next_select_is_exact():
    """The select's CTAs wait on each other's tagged totals; with one CTA that
    never publishes, every bounded wait must run out (SCAN_ETIMEOUT), and a
    normal select on the same column afterwards must still be exact."""
    n, b = 3 * (1 << 20) + 77, 12
    v = synth.uniform_values(5, n, b)
    col = gbscan.Column.from_host(v, b)
    lib = gbscan.load()
    for limit_ns in (2_000_000, 20_000_000):
        st = lib.scan_selftest_select_timeout(col.handle, limit_ns, None)
        assert st == gbscan.SCAN_ETIMEOUT, lib.scan_last_error()
    assert lib.scan_selftest_select_timeout(col.handle, 0, None) == gbscan.SCAN_EINVAL
    want, k = oracle.select_values(v, 100, 900)
    pos = torch.empty(k, dtype=torch.int32, device="cuda")
    assert col.select(100, 900, pos) == k
    assert (pos.cpu().numpy().view("uint32") == want).all()
    col.close()


def test_bad_arguments_are_refused_before_any_launch():
    assert gbscan.load().scan_selftest_wait_timeout(0, None) == gbscan.SCAN_EINVAL
    with pytest.raises(gbscan.ScanError) as e:
        gbscan.Column.from_host(synth.uniform_values(1, 10, 4), 40)
    assert e.value.status == gbscan.SCAN_EINVAL
