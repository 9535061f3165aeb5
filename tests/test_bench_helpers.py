"""Host-side pieces of bench.py that need no GPU: the traffic record lookup keyed
by the kernel-source hash, the roofline helpers and the JSON shapes."""
import json
import os

import pytest

import bench


def test_traffic_record_matches_current_sources():
    """When profiles/traffic.md holds a record for the current kernel sources, its
    DRAM bytes per launch are close to the algorithmic bytes."""
    t = bench.ncu_traffic("tet_generic_mixed_aos_6M")
    if t is None:
        pytest.skip("kernel sources changed since profiles/traffic.md was captured (traffic reads null)")
    # the DRAM bytes of a launch are within a few percent of the algorithmic bytes
    assert 0.95 * 1.536e9 <= t <= 1.02 * 1.536e9
    p = bench.ncu_traffic("prism_generic_mixed_aos_2M")
    assert p is not None and 0.95 * 1.584e9 <= p <= 1.02 * 1.584e9


def test_traffic_lookup_needs_the_hash(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("tet_generic_mixed_aos_6M") is None


def test_rooflines_of_the_alu_bound_forms():
    f = bench.fp64_pipe(7000.0, "tet_poisson_tet1")
    assert f["peak"] == pytest.approx(2 * 152 * 2.07e9 / 1e12)
    assert f["achieved"] == pytest.approx(7000e6 * 77 / 1e12)
    assert 0 < f["frac"] < 1
    i = bench.issue_roofline(19000.0, "tet_poisson_tet1")
    assert i["peak"] == pytest.approx(4 * 32 * 152 * 2.07e9 / 1e12)
    assert i["frac"] == pytest.approx(19000e6 * 1436 / 1e12 / i["peak"])


def test_shape_and_context_records_are_json():
    assert bench.shape_dict((64, 0)) == {"elements_per_block": 64, "persistent": 0, "threads_per_element": 1}
    assert bench.shape_dict((32, 1, 2))["threads_per_element"] == 2
    ctx = bench.paper_context()
    json.dumps(ctx)
    assert ctx["melem_s"]["Tesla K20m"]["laplace_tet"] == pytest.approx(1000 / 2.02, abs=0.1)
