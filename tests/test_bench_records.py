"""The stored measurement records that bench.py reads, checked against the current sources (CPU).

bench.py scales the DRAM traffic of its roofline kernels from ncu captures stored in
profiles/roofline_traffic.json, and uses each capture only while the hash of the kernel's source
(bench.kernel_source_sha) is unchanged.  A kernel edited after its capture would silently drop the
line's `traffic` to null; this test fails instead, so the capture is retaken with the change.
"""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def records():
    with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("key", ["fine:precision0", "fine:precision3", "level1:precision0", "level1:precision3"])
def test_traffic_capture_matches_current_kernel_source(key):
    ent = records()[key]
    kind, prec = key.split(":")
    assert ent["kernel_source_sha"] == bench.kernel_source_sha(kind, int(prec[len("precision"):]))
    # the capture covers the kernel's whole traffic: DRAM bytes within 10% of the algorithmic bytes
    ratio = ent["dram_bytes_per_launch"] / ent["algorithmic_bytes_per_launch"]
    assert abs(ratio - ent["ratio"]) < 1e-3 and 0.9 < ratio < 1.1
    assert os.path.exists(os.path.join(ROOT, ent["source"]))


def test_load_traffic_scales_to_the_launch():
    t, src = bench.load_traffic("fine", 0, 1.0e9)
    ent = records()["fine:precision0"]
    assert t == pytest.approx(1.0e9 * ent["dram_bytes_per_launch"] / ent["algorithmic_bytes_per_launch"])
    assert "scaled to this launch" in src
