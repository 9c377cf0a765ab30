"""Launch shapes and the autotuner's cache, on CPU (no kernel runs): the
candidate shapes obey the documented rules, illegal shapes are refused with the
rule they break, and the versioned cache file round-trips and is validated
line by line, all or nothing."""
import os

import pytest

from paper_2606_22423_gb300 import gbscan

KINDS = ["branchfree", "branchy", "zone_bf", "zone_br"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    gbscan.load()
    gbscan.autotune_reset()
    yield
    gbscan.autotune_reset()


def legal(kind, b, s):
    """The header's rules, restated."""
    full = kind in ("branchfree", "branchy")
    default = 4 if b <= 16 else 2
    lanes = s.get("vec_lanes", 0)
    if lanes not in (0, default) and not (lanes == 2 and full and 9 <= b <= 16):
        return False
    step = lanes or default
    smem = s["warps"] * s["stages"] * (s["tile_blocks"] * 128 * b + 12)
    return (1 <= s["warps"] <= (16 if full else 8) and 1 <= s["stages"] <= 6
            and s["tile_blocks"] >= step and s["tile_blocks"] % step == 0
            and s["tile_blocks"] <= (64 if full else 32)
            and (s["vote_rows"] == 0 or (kind == "branchy" and b <= 21 and s["vote_rows"] in (1, 2, 3)))
            and smem <= 226 * 1024)


@pytest.mark.parametrize("kind", KINDS)
def test_candidates_are_legal_and_include_more_warps_and_vote_forms(kind):
    for b in range(1, 33):
        cands = gbscan.shape_candidates(b, kind)
        assert cands, (kind, b)
        assert len({tuple(c.values()) for c in cands}) == len(cands)       # no duplicates
        for c in cands:
            assert legal(kind, b, c), (kind, b, c)
        rule = gbscan.shape_get(b, kind)
        assert legal(kind, b, rule) and rule["warps"] == 8 and rule["vote_rows"] == 0
        if kind in ("branchfree", "branchy"):
            assert max(c["warps"] for c in cands) > 8
        if kind == "branchy" and b <= 21:
            assert {c["vote_rows"] for c in cands} == {0, 1, 2, 3}
        if kind in ("branchfree", "branchy") and 9 <= b <= 16:       # the 2-lane geometry with 16 warps
            assert any(c["vec_lanes"] == 2 and c["warps"] == 16 for c in cands)
        else:
            assert all(c["vec_lanes"] == 0 for c in cands)


def test_illegal_shapes_are_refused_with_the_rule():
    cases = [(8, "branchfree", dict(warps=17, stages=3, tile_blocks=8), "warps"),
             (8, "zone_bf", dict(warps=12, stages=3, tile_blocks=8), "warps"),
             (8, "branchfree", dict(warps=8, stages=0, tile_blocks=8), "stages"),
             (8, "branchfree", dict(warps=8, stages=3, tile_blocks=6), "multiple of the warp step"),
             (20, "branchfree", dict(warps=8, stages=3, tile_blocks=3), "multiple of the warp step"),
             (1, "zone_bf", dict(warps=8, stages=3, tile_blocks=36), "at most 32"),
             (8, "branchfree", dict(warps=8, stages=3, tile_blocks=8, vote_rows=1), "row vote"),
             (24, "branchy", dict(warps=8, stages=3, tile_blocks=2, vote_rows=1), "row vote"),
             (22, "branchy", dict(warps=16, stages=2, tile_blocks=2, vote_rows=2), "row vote"),
             (8, "branchfree", dict(warps=16, stages=2, tile_blocks=4, vote_rows=2), "row vote"),
             (8, "branchy", dict(warps=16, stages=2, tile_blocks=4, vote_rows=4), "0, 1, 2 or 3"),
             (32, "branchfree", dict(warps=16, stages=4, tile_blocks=2), "226 KB"),
             (8, "branchfree", dict(warps=16, stages=2, tile_blocks=4, vec_lanes=2), "vec_lanes"),
             (12, "zone_bf", dict(warps=8, stages=2, tile_blocks=4, vec_lanes=2), "vec_lanes"),
             (12, "branchfree", dict(warps=16, stages=2, tile_blocks=3, vec_lanes=2), "multiple of the warp step")]
    for b, kind, shape, why in cases:
        with pytest.raises(gbscan.ScanError) as e:
            gbscan.shape_set(b, kind, shape)
        assert e.value.status == gbscan.SCAN_EINVAL and why in str(e.value), (shape, str(e.value))
    with pytest.raises(gbscan.ScanError):
        gbscan.shape_set(0, "branchfree", dict(warps=8, stages=3, tile_blocks=8))
    for b in (1, 8, 32):
        assert gbscan.shape_get(b, "branchfree") == gbscan.shape_get(b, "branchy")    # nothing installed


def test_set_get_and_back_to_the_rule():
    rule = gbscan.shape_get(12, "branchy")
    s = dict(warps=16, stages=2, tile_blocks=4, vote_rows=1, vec_lanes=0)
    gbscan.shape_set(12, "branchy", s)
    assert gbscan.shape_get(12, "branchy") == s
    assert gbscan.shape_get(12, "branchfree") != s                 # per kernel
    gbscan.shape_set(12, "branchy", None)
    assert gbscan.shape_get(12, "branchy") == rule


def test_cache_round_trip(tmp_path):
    installed = {(3, "branchfree"): dict(warps=16, stages=3, tile_blocks=8, vote_rows=0, vec_lanes=0),
                 (9, "branchy"): dict(warps=12, stages=2, tile_blocks=4, vote_rows=1, vec_lanes=0),
                 (15, "branchy"): dict(warps=16, stages=2, tile_blocks=2, vote_rows=1, vec_lanes=2),
                 (16, "zone_bf"): dict(warps=8, stages=2, tile_blocks=4, vote_rows=0, vec_lanes=0),
                 (30, "zone_br"): dict(warps=8, stages=2, tile_blocks=2, vote_rows=0, vec_lanes=0)}
    gbscan.autotune_reset()
    for (b, kind), s in installed.items():
        gbscan.shape_set(b, kind, s)
    path = str(tmp_path / "shapes.txt")
    gbscan.autotune_save(path)
    lines = open(path).read().splitlines()
    assert lines[0] == "gbscan-shapes 3" and lines[1].startswith("device ")
    assert len([ln for ln in lines[2:] if ln and not ln.startswith("#")]) == len(installed)
    gbscan.autotune_reset()
    assert gbscan.shape_get(3, "branchfree")["warps"] == 8
    gbscan.autotune_load(path)
    for (b, kind), s in installed.items():
        assert gbscan.shape_get(b, kind) == s
    # zone_agg strategies share the zone-skip kernels' shapes
    assert gbscan.shape_get(16, "zone_agg_bf") == installed[(16, "zone_bf")]
    gbscan.autotune_reset()


def _write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_cache_validation_is_all_or_nothing(tmp_path):
    gbscan.autotune_reset()
    keep = dict(warps=12, stages=2, tile_blocks=4, vote_rows=0, vec_lanes=0)
    gbscan.shape_set(5, "branchfree", keep)
    good = str(tmp_path / "good.txt")
    gbscan.autotune_save(good)
    head, device = open(good).read().splitlines()[:2]
    row = "full_bf 7 16 2 8 0 0 10.0 12.0"
    cases = [("gbscan-shapes 3\n", "device line"),
             ("gbscan-shape 3\n" + device + "\n", "not a gbscan shape cache"),
             ("gbscan-shapes 1\n" + device + "\n", "version 1"),
             ("gbscan-shapes 2\n" + device + "\n", "version 2"),
             (head + "\ndevice Other_GPU 7\n" + row + "\n", "tuned on 'Other_GPU 7'"),
             (head + "\n" + device + "\nfull_xx 7 16 3 8 0 0 1 1\n", "unknown kernel kind"),
             (head + "\n" + device + "\nfull_bf 7 16 3 6 0 0 1 1\n", "multiple of the warp step"),
             (head + "\n" + device + "\nqueue_bf 7 12 3 8 0 0 1 1\n", "warps"),
             (head + "\n" + device + "\nfull_bf 7 16 2 8 0 2 1 1\n", "vec_lanes"),
             (head + "\n" + device + "\n" + row + "\n" + row + "\n", "duplicate"),
             (head + "\n" + device + "\nfull_bf 7 16 3\n", "expected"),
             (head + "\n" + device + "\n" + row + " extra\n", "expected")]
    for i, (text, why) in enumerate(cases):
        with pytest.raises(gbscan.ScanError) as e:
            gbscan.autotune_load(_write(tmp_path, f"bad{i}.txt", text))
        assert e.value.status == gbscan.SCAN_EINVAL and why in str(e.value), (i, str(e.value))
        assert gbscan.shape_get(5, "branchfree") == keep                  # unchanged
    with pytest.raises(gbscan.ScanError):
        gbscan.autotune_load(str(tmp_path / "missing.txt"))
    # comments and blank lines are allowed; a valid file replaces the table
    gbscan.autotune_load(_write(tmp_path, "ok.txt", head + "\n" + device + "\n# note\n\n" + row + "\n"))
    assert gbscan.shape_get(7, "branchfree") == dict(warps=16, stages=2, tile_blocks=8, vote_rows=0, vec_lanes=0)
    assert gbscan.shape_get(5, "branchfree")["warps"] == 8                # replaced, not merged
    gbscan.autotune_reset()
    assert os.path.exists(good)


def test_batch_shapes_candidates_rules_and_cache(tmp_path):
    gbscan.autotune_reset()
    for br in (False, True):
        for b in range(1, 33):
            rule = gbscan.batch_shape_get(b, br)
            step = 4 if b <= 16 else 2
            # the rule: 2 stages of about 6 KB (one warp step where a step is larger), 8 warps
            # unless two such CTAs would not share an SM (112 KB of slots each at most)
            assert rule["stages"] == 2 and rule["vote_rows"] == 0 and rule["vec_lanes"] == 0
            assert rule["tile_blocks"] % step == 0
            assert rule["tile_blocks"] * 128 * b <= 6 * 1024 or rule["tile_blocks"] == step
            slots = rule["warps"] * rule["stages"] * (rule["tile_blocks"] * 128 * b + 24)
            assert slots <= 112 * 1024
            assert rule["warps"] == 8 or (rule["warps"] + 1) * 2 * (rule["tile_blocks"] * 128 * b + 24) > 112 * 1024
            cands = gbscan.batch_shape_candidates(b, br)
            assert cands and max(c["warps"] for c in cands) <= 8 and min(c["warps"] for c in cands) == 4
            for c in cands:
                assert c["vote_rows"] == 0 and c["tile_blocks"] % step == 0 and c["tile_blocks"] <= 64
                assert c["warps"] * c["stages"] * (c["tile_blocks"] * 128 * b + 24) <= 112 * 1024
    assert [gbscan.batch_shape_get(b)["warps"] for b in (1, 13, 14, 16, 27, 28, 32)] == [8, 8, 7, 6, 8, 7, 6]
    with pytest.raises(gbscan.ScanError) as e:
        gbscan.batch_shape_set(9, False, dict(warps=8, stages=2, tile_blocks=4, vote_rows=1))
    assert "row vote" in str(e.value)
    with pytest.raises(gbscan.ScanError) as e:
        gbscan.batch_shape_set(32, True, dict(warps=16, stages=3, tile_blocks=4))
    assert "226 KB" in str(e.value)
    s = dict(warps=16, stages=2, tile_blocks=4, vote_rows=0, vec_lanes=0)
    gbscan.batch_shape_set(9, True, s)
    assert gbscan.batch_shape_get(9, True) == s and gbscan.batch_shape_get(9, False)["warps"] == 8
    path = str(tmp_path / "b.txt")
    gbscan.autotune_save(path)
    assert "batch_br 9 16 2 4 0 0" in open(path).read()
    gbscan.autotune_reset()
    assert gbscan.batch_shape_get(9, True)["warps"] == 8
    gbscan.autotune_load(path)
    assert gbscan.batch_shape_get(9, True) == s
    gbscan.autotune_reset()
