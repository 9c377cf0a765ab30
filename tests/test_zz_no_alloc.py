"""The allocation-free scan entry point (scan_run_packed_noalloc).

It serves callers that cannot allocate device memory while they scan
(allocator-free serving loops, fixed-budget engines, plug-ins whose host owns
the device memory).  Its COUNT and SUM must equal the oracle's brute force over
the generator's raw values, and the regular entry point's result, exactly, on
consecutive calls that reuse the shared static scratch.  One case runs in a
fresh process where the allocation-free call is the first scan launch of the
process (so it also does the module load, the kernel attribute set-up and the
scratch address lookup).  This file is collected last on purpose.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from paper_2606_22423_gb300 import gbscan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


@pytest.mark.parametrize("b,n,strategy", [(8, 1 << 22, "branchfree"), (13, 300 * 1024 + 77, "branchy"),
                                          (32, 5 * 1024 + 3, "branchfree"), (1, 1000, "auto")])
def test_noalloc_matches_the_oracle_on_consecutive_calls(b, n, strategy):
    base = 0 if b == 32 else 11
    v = synth.uniform_values(synth.seed_for(99, b, n), n, b, base)
    col = gbscan.Column.from_host(v, b, base)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    preds = [synth.pick_range(synth.seed_for(99, b, i), b, s, base) for i, s in enumerate([0.1, 0.7])]
    for lo, hi in preds + [preds[0]]:                # two different calls, then a repeat
        want = oracle.scan_values(v, lo, hi)
        gbscan.scan_run_packed_noalloc(col.dev_packed, n, b, base, lo, hi, out, status, strategy)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert int(status.cpu()[0]) == 0
        assert (int(got[0]), int(got[1])) == want
        assert int(got[2]) == (n + 1023) // 1024    # a full scan reads every block
        regular = col.run(lo, hi, "branchfree" if strategy == "auto" else strategy)
        assert (regular.count, regular.sum, regular.blocks_scanned) == (int(got[0]), int(got[1]), int(got[2]))
    col.close()


def test_noalloc_with_a_tuned_sixteen_warp_shape():
    """The allocation-free scan launches with the installed (tuned) shape: 16
    warps and 2-block tiles of the 2-lane geometry at b = 15 still give the
    oracle's result from the static scratch."""
    b, n = 15, 120 * 1024 + 5
    v = synth.uniform_values(synth.seed_for(97, b), n, b, 3)
    col = gbscan.Column.from_host(v, b, 3)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    lo, hi = synth.pick_range(synth.seed_for(97, b, 1), b, 0.3, 3)
    try:
        gbscan.shape_set(b, "branchfree", dict(warps=16, stages=2, tile_blocks=2, vote_rows=0, vec_lanes=2))
        for _ in range(2):
            gbscan.scan_run_packed_noalloc(col.dev_packed, n, b, 3, lo, hi, out, status)
            torch.cuda.synchronize()
            assert int(status.cpu()[0]) == 0
            assert tuple(int(x) for x in out.cpu()[:2]) == oracle.scan_values(v, lo, hi)
    finally:
        gbscan.shape_set(b, "branchfree", None)
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


FIRST_CALL = r"""
import sys
sys.path.insert(0, %(root)r)
import numpy as np
import torch
import oracle, synth
from paper_2606_22423_gb300 import gbscan

gbscan.load()
n, b, base = 200 * 1024 + 321, 27, 5
v = synth.uniform_values(synth.seed_for(98, b), n, b, base)
words = oracle.pack(v, b, base)                       # packed on the host by the oracle
packed = torch.from_numpy(words.view(np.int32)).cuda()  # a plain copy: no library kernel has run yet
out = torch.zeros(4, dtype=torch.int64, device="cuda")
status = torch.zeros(1, dtype=torch.int32, device="cuda")
lo, hi = synth.pick_range(synth.seed_for(98, b, 1), b, 0.3, base)
want = oracle.scan_values(v, lo, hi)
for _ in range(2):                                    # the first scan launch of the process, then again
    gbscan.scan_run_packed_noalloc(packed.data_ptr(), n, b, base, lo, hi, out, status, "branchy")
    torch.cuda.synchronize()
    got = out.cpu().tolist()
    assert int(status.item()) == 0, status
    assert (got[0], got[1]) == want, (got, want)
col = gbscan.Column.from_packed(packed.data_ptr(), n, b, base)   # a regular scan afterwards
r = col.run(lo, hi, "branchy")
assert (r.count, r.sum) == want
col.close()
print("first-call ok", want)
"""


def test_noalloc_as_the_first_scan_of_a_fresh_process(tmp_path):
    import oracle as _o

    _o.build()
    script = tmp_path / "first_call.py"
    script.write_text(FIRST_CALL % {"root": ROOT})
    r = subprocess.run([sys.executable, str(script)], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "first-call ok" in r.stdout
