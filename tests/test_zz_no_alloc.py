"""The allocation-free scan entry point (scan_run_packed_noalloc).

It serves callers that cannot allocate device memory while they scan
(allocator-free serving loops, fixed-budget engines, plug-ins whose host owns
the device memory).  Its result
must equal the regular entry point's, exactly, on consecutive calls that
reuse the shared static scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("b,n,strategy", [(8, 1 << 22, "branchfree"), (13, 300 * 1024 + 77, "branchy"),
                                          (32, 5 * 1024 + 3, "branchfree"), (1, 1000, "auto")])
def test_noalloc_matches_the_regular_entry_point_on_consecutive_calls(b, n, strategy):
    base = 0 if b == 32 else 11
    v = synth.uniform_values(synth.seed_for(99, b, n), n, b, base)
    col = gbscan.Column.from_host(v, b, base)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    preds = [synth.pick_range(synth.seed_for(99, b, i), b, s, base) for i, s in enumerate([0.1, 0.7])]
    for lo, hi in preds + [preds[0]]:                # two different calls, then a repeat
        want = col.run(lo, hi, "branchfree" if strategy == "auto" else strategy)
        gbscan.scan_run_packed_noalloc(col.dev_packed, n, b, base, lo, hi, out, status, strategy)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert int(status.cpu()[0]) == 0
        assert (int(got[0]), int(got[1]), int(got[2])) == (want.count, want.sum, want.blocks_scanned)
    col.close()


def test_noalloc_empty_range_and_limits():
    v = synth.uniform_values(5, 4096, 9)
    col = gbscan.Column.from_host(v, 9)
    out = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gbscan.scan_run_packed_noalloc(col.dev_packed, 4096, 9, 0, 50, 50, out, status)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0)
    with pytest.raises(gbscan.ScanError) as e:    # beyond the maximum column length
        gbscan.scan_run_packed_noalloc(col.dev_packed, (1 << 31) + 1, 9, 0, 0, 10, out, status)
    assert e.value.status == gbscan.SCAN_EINVAL and "2^31" in str(e.value)
    with pytest.raises(gbscan.ScanError):          # zone skipping needs allocated state
        gbscan.scan_run_packed_noalloc(col.dev_packed, 4096, 9, 0, 0, 10, out, status, "zone_bf")
    col.close()
