"""The allocation-free steady entry point (vs_solve_steady_noalloc), called
through the C ABI, gives the same temperatures as vs_solve_steady.

This file is collected last on purpose: the entry point shares one fixed
device array across calls, and a run that stops at the first failure has then
already run every other test. It must also pass alone in a fresh process."""
import ctypes

import pytest
import torch

import synth

from _util import ENG_TOL_K, inputs, vs_params, vs_stack

pytestmark = pytest.mark.gpu


def _call_noalloc(vs, k, pd, pl, s, params, out):
    info = vs._SolveInfo()
    stream = torch.cuda.current_stream().cuda_stream
    rc = vs.lib().vs_solve_steady_noalloc(
        k.handle, pd.data_ptr(), pl.data_ptr(), s.data_ptr() if s is not None else None,
        ctypes.byref(params._c()), out.data_ptr(), ctypes.byref(info), stream)
    return rc, info


@pytest.mark.parametrize("name", ["c1_64", "c3_256", "c3_512"])
def test_noalloc_matches_allocating_entry_point_twice(name):
    import paper_2307_12119_gb300 as vs
    w = synth.workload(name)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    params = vs_params(w)
    pd, pl, s = inputs(w, count=2)
    out = torch.empty_like(pd)
    ref = torch.empty_like(pd)
    for i in range(2):                      # two calls in a row reuse the array
        rc, info = _call_noalloc(vs, k, pd[i], pl[i], s[i], params, out[i])
        assert rc == vs.VS_OK and info.status == vs.VS_OK
        _, rinfo = vs.solve_steady(k, pd[i], pl[i], s[i], params, ref[i])
        # streamed engine against the automatic engine (the cluster engine for
        # n <= 256: same arithmetic, other rounding)
        assert abs(info.iterations - rinfo["iterations"]) <= 1
        assert float((out[i] - ref[i]).abs().max()) <= ENG_TOL_K


def test_noalloc_rejects_grids_beyond_its_array():
    import paper_2307_12119_gb300 as vs
    w = synth.workload("c4_1024")
    k = vs.Kernel(vs_stack(w), vs.Grid(1024, w.die_m))
    z = torch.zeros(1024, 1024, device="cuda")
    rc, _ = _call_noalloc(vs, k, z, z, None, vs_params(w), z.clone())
    assert rc == vs.VS_ERR_INVALID_ARG
    assert "n <= 512" in vs.lib().vs_last_error().decode()


def test_noalloc_rejects_other_engines_and_precisions():
    """It runs the FP32 streamed engine only; asking for the cluster engine or
    for split precision is an argument error, not a silent substitution."""
    import paper_2307_12119_gb300 as vs
    w = synth.workload("c1_64")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    pd, pl, s = inputs(w, count=1)
    out = torch.empty_like(pd[0])
    for kw in ({"engine": vs.VS_ENGINE_CLUSTER}, {"precision": vs.VS_PREC_BF16_SPLIT}):
        rc, _ = _call_noalloc(vs, k, pd[0], pl[0], s[0], vs_params(w, **kw), out)
        assert rc == vs.VS_ERR_INVALID_ARG, kw
        assert "streamed engine only" in vs.lib().vs_last_error().decode()
    rc, info = _call_noalloc(vs, k, pd[0], pl[0], s[0], vs_params(w, engine=vs.VS_ENGINE_STREAMED), out)
    assert rc == vs.VS_OK and info.status == vs.VS_OK


def test_noalloc_takes_the_stopping_rule():
    """The error-estimate rule reaches the streamed engine behind the entry
    point: it stops as a one-map streamed plan with that rule does."""
    import paper_2307_12119_gb300 as vs
    w = synth.workload("c3_256")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    pd, pl, s = inputs(w, count=1)
    prm = vs_params(w, tol=1e-2, engine=vs.VS_ENGINE_STREAMED, stop_rule=vs.VS_STOP_ESTIMATE)
    out, ref = torch.empty_like(pd[0]), torch.empty_like(pd[0])
    rc, info = _call_noalloc(vs, k, pd[0], pl[0], s[0], prm, out)
    assert rc == vs.VS_OK and info.status == vs.VS_OK
    _, rinfo = vs.solve_steady(k, pd[0], pl[0], s[0], prm, ref)
    assert abs(info.iterations - rinfo["iterations"]) <= 1
    assert float((out - ref).abs().max()) <= ENG_TOL_K
    upd = vs_params(w, tol=1e-2, engine=vs.VS_ENGINE_STREAMED)
    rc, uinfo = _call_noalloc(vs, k, pd[0], pl[0], s[0], upd, out)
    assert rc == vs.VS_OK and info.iterations <= uinfo.iterations
