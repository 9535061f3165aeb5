"""Host-side pieces of bench.py that need no GPU: the ncu record lookup keyed by
the kernel-source hash, the roofline helpers and the JSON shapes."""
import json

import pytest

import bench


def _records():
    with open(bench.NCU_RECORDS) as f:
        return json.load(f)["records"]


def test_ncu_records_are_well_formed():
    recs = _records()
    assert recs
    for tag, r in recs.items():
        assert len(r["source_hash"]) == 16 and r["elements"] > 0 and r["kernel"]
        assert any(k in r for k in ("dram_bytes", "fp64_pipe_inst_per_elem", "inst_per_elem")), tag


def test_ncu_record_needs_the_current_hash(monkeypatch):
    recs = _records()
    tag, r = next(iter(recs.items()))
    field = next(k for k in ("dram_bytes", "fp64_pipe_inst_per_elem", "inst_per_elem") if k in r)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: r["source_hash"])
    assert bench.ncu_record(tag, field) == pytest.approx(float(r[field]))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.ncu_record(tag, field) is None
    assert bench.ncu_record("no such kernel", field) is None


def test_traffic_records_close_to_the_algorithmic_bytes():
    """Every DRAM-bytes record of a full-size capture is within a few percent of
    the algorithmic bytes of its launch (no re-reads)."""
    alg = {"tet_generic_mixed_aos": 256, "prism_generic_mixed_aos": 792, "tet_generic_fp64_aos": 416}
    for tag, r in _records().items():
        if "dram_bytes" in r and tag in alg and r.get("full_size", True):
            assert 0.9 * alg[tag] * r["elements"] <= r["dram_bytes"] <= 1.02 * alg[tag] * r["elements"], tag


def test_rooflines_of_the_alu_bound_forms():
    f = bench.pipe_roofline(7000.0, 77.0, 152, 2070.0, bench.FP64_PIPE_PER_CLK_SM, "FP64-pipe", "t")
    assert f["peak"] == pytest.approx(2 * 152 * 2.07e9 / 1e12)
    assert f["achieved"] == pytest.approx(7000e6 * 77 / 1e12)
    assert 0 < f["frac"] < 1 and f["bound"] == "alu"
    i = bench.pipe_roofline(19000.0, 1436.0, 152, 2070.0, bench.ISSUE_PER_CLK_SM, "thread", "t")
    assert i["peak"] == pytest.approx(4 * 32 * 152 * 2.07e9 / 1e12)
    assert i["frac"] == pytest.approx(19000e6 * 1436 / 1e12 / i["peak"])
    n = bench.pipe_roofline(19000.0, None, 152, 1900.0, bench.ISSUE_PER_CLK_SM, "thread", "t")
    assert n["frac"] is None and n["achieved"] is None and n["peak"] == pytest.approx(4 * 32 * 152 * 1.9e9 / 1e12)
    h = bench.hbm_roofline(6_000_000, 416, 1.0, 6781.1, "measured")
    assert h["achieved"] == pytest.approx(6e6 * 416 / 1e-3 / 1e9) and h["bound"] == "hbm"


def test_shape_and_context_records_are_json():
    assert bench.shape_dict((64, 0)) == {"elements_per_block": 64, "persistent": 0, "threads_per_element": 1}
    assert bench.shape_dict((32, 1, 2))["threads_per_element"] == 2
    ctx = bench.paper_context()
    json.dumps(ctx)
    assert ctx["melem_s"]["Tesla K20m"]["laplace_tet"] == pytest.approx(1000 / 2.02, abs=0.1)


def test_source_hash_ignores_comments_only():
    src = "template <int K> // bound\n__global__ void k(float *p) {\n    /* body */ p[0] = K; }\n"
    edited = src.replace("// bound", "// another note").replace("/* body */", "/* the\nbody */")
    assert bench.code_only(src) == bench.code_only(edited)
    assert bench.code_only(src) != bench.code_only(src.replace("p[0] = K", "p[0] = 2 * K"))
