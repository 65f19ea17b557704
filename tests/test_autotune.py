"""Autotuner host logic (CPU): candidate space, selection, JSON cache."""

import json

import synth
from paper_2410_04974_gb300 import autotune


def test_candidate_space_and_selection(tmp_path):
    cams = synth.ring_cameras(2, 64, 48)
    space = autotune.candidate_space(tiles=((16, 16), (16, 8)), batches=(256, 512), persistent=(True, False))
    assert len(space) == 8
    cost = {(16, 16, 256, True): 3.0, (16, 16, 512, True): 2.0, (16, 8, 512, False): 1.5}
    seen = []

    def fake(c):
        seen.append(c)
        return cost.get((c["tile"][0], c["tile"][1], c["batch"], c["persistent"]), 5.0)

    cache = str(tmp_path / "tune.json")
    r = autotune.tune(None, 1000, 3, cams, space=space, cache=cache, measure=fake, device_name="fake")
    assert (r["tile"], r["batch"], r["persistent"]) == ([16, 8], 512, False)
    assert r["ms"] == 1.5 and not r["cached"] and len(seen) == 8
    data = json.load(open(cache))
    assert len(data) == 1
    # second call: served from the cache, nothing measured
    r2 = autotune.tune(None, 1000, 3, cams, space=space, cache=cache, measure=fake, device_name="fake")
    assert r2["cached"] and r2["tile"] == [16, 8] and len(seen) == 8
    # a different frame shape is a different entry
    r3 = autotune.tune(None, 1001, 3, cams, space=space, cache=cache, measure=fake, device_name="fake")
    assert not r3["cached"] and len(json.load(open(cache))) == 2


def test_signature_depends_on_camera_sizes():
    a = autotune.signature("g", 10, 3, synth.ring_cameras(2, 64, 48), autotune.candidate_space())
    b = autotune.signature("g", 10, 3, synth.ring_cameras(2, 64, 64), autotune.candidate_space())
    c = autotune.signature("g", 10, 3, synth.ring_cameras(2, 64, 48), autotune.candidate_space())
    assert a != b and a == c
