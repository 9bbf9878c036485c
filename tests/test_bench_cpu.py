"""Host-side helpers of the benchmark (CPU only)."""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_traffic_key_ignores_comments_and_layout():
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* note */\n}\n"
    b = "int f(int x) {\n    return 2 * x;\n}\n// trailing remark\n"
    c = "int f(int x) { return 3 * x; }\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_traffic_records_resolve_only_for_their_sources():
    # a committed record is used only while the code it was captured from is
    # unchanged (the bench then reports traffic: null until it is re-taken)
    import json
    recs = json.load(open(bench.TRAFFIC_JSON))
    assert recs
    for kernel, rec in recs.items():
        assert kernel in bench.KERNEL_SOURCES, kernel
        assert rec["dram_bytes_per_unit"] > 0 and rec["captured_units"] > 0
        cur = bench._source_hash(bench.KERNEL_SOURCES[kernel])
        got = bench._traffic_record(kernel)
        assert (got is not None) == (rec["source_hash"] == cur), kernel


def test_ablation_inputs_switch_variation_off_per_map():
    g = torch.Generator().manual_seed(3)
    pl = torch.rand(3, 8, 8, generator=g) + 0.5
    s = 1.0 - 0.05 * torch.rand(3, 8, 8, generator=g)
    pl_x, s_x = bench.ablation_inputs(pl, s, s_var=False, l_var=False)
    assert s_x is None
    for b in range(3):
        assert torch.allclose(pl_x[b], torch.full((8, 8), float(pl[b].mean())))
    pl_y, s_y = bench.ablation_inputs(pl, s, s_var=True, l_var=True)
    assert pl_y is pl and s_y is s
    assert [r[0] for r in bench.ABLATION_SCENARIOS][0] == "no effects"


def test_flop_count_grows_with_iterations_and_size():
    f = bench.fp32_flops_per_map
    per_iter = f(256, 2.0) - f(256, 1.0)
    assert per_iter > 0 and f(256, 0.0) > 0
    assert f(512, 1.0) > 4 * f(256, 1.0)           # n^2 log n
