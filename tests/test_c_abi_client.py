"""The boundary from plain C.  tests/c_abi_client.c includes only
include/gbscan.h and links only libgbscan.so: on CPU it must compile and link
cleanly (every call it makes is declared and exported); on the GPU every
strategy's COUNT, SUM and blocks read must equal the oracle's, and so must a
scan after the client tunes its launch shape and round-trips the cache."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_client.c")
CUDA_LIB = "/usr/local/cuda/lib64"


def _build_client(tmp_path):
    import __graft_entry__

    __graft_entry__.build()
    from paper_2606_22423_gb300 import gbscan

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    libdir = os.path.dirname(gbscan.LIB_PATH)
    exe = str(tmp_path / "c_abi_client")
    cmd = [gcc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
           "-o", exe, "-L", libdir, "-lgbscan", f"-Wl,-rpath,{libdir}"]
    if os.path.isdir(CUDA_LIB):
        cmd.append(f"-Wl,-rpath-link,{CUDA_LIB}")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def test_c_client_compiles_and_links_against_the_library(tmp_path):
    exe = _build_client(tmp_path)
    assert os.access(exe, os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("n,b,base,sigma,order", [(300 * 1024 + 555, 11, 7, 0.1, None),
                                                  (70_000, 3, 0, 0.5, 0.0),
                                                  (5 * 1024, 32, 0, 0.01, None),
                                                  (1 << 20, 16, 1000, 1e-3, 0.0)])
def test_c_client_matches_the_oracle_for_every_strategy(tmp_path, n, b, base, sigma, order):
    exe = _build_client(tmp_path)
    seed = synth.seed_for(77, b, n)
    v = (synth.uniform_values(seed, n, b, base) if order is None
         else synth.clustered_values(seed, n, b, order, base))
    lo, hi = synth.pick_range(seed + 1, b, sigma, base)
    path = tmp_path / "values.bin"
    np.ascontiguousarray(v, dtype=np.uint32).tofile(path)
    cache = tmp_path / "shapes.txt"
    r = subprocess.run([exe, str(path), str(n), str(b), str(base), str(lo), str(hi), str(cache)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln.split() for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 9
    shape, tuned = lines[7], lines[8]
    assert shape[0] == "shape" and tuned[0] == "tuned"
    assert open(cache).read().startswith("gbscan-shapes 3\ndevice ")
    assert (int(tuned[1]), int(tuned[2])) == oracle.scan_values(v, lo, hi)
    assert int(tuned[3]) == (n + 1023) // 1024
    lines = lines[:7]
    want = oracle.scan_values(v, lo, hi)
    words = oracle.pack(v, b, base)
    zmin, zmax = oracle.zonemap(words, n, b, base)
    _, _, zone_blocks = oracle.scan_zoneskip(words, zmin, zmax, n, b, base, lo, hi)
    sums = oracle.blocksums(words, n, b, base)
    _, _, agg_blocks = oracle.scan_zoneagg(words, zmin, zmax, sums, n, b, base, lo, hi)
    full_blocks = (n + 1023) // 1024
    expect_blocks = {1: full_blocks, 2: full_blocks, 3: zone_blocks, 4: zone_blocks, 5: agg_blocks, 6: agg_blocks}
    for strat, count, total, blocks in lines:
        assert (int(count), int(total)) == want, (strat, count, total, want)
        if int(strat) in expect_blocks:
            assert int(blocks) == expect_blocks[int(strat)], (strat, blocks)
