"""The C-ABI library builds, loads and exports every symbol include/varsim.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "varsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2307_12119_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("vs_make_kernel", "vs_solve_steady", "vs_solve_transient", "vs_solve_batch"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export(libpath):
    import paper_2307_12119_gb300 as vs
    assert sorted(vs.EXPORTS) == _declared()
    L = vs.lib()
    assert L.vs_version().decode().startswith("varsim-gb300")
    assert L.vs_status_string(vs.VS_ERR_RUNAWAY).decode() == "thermal or conductivity runaway"


def test_argument_errors_need_no_gpu(libpath):
    import paper_2307_12119_gb300 as vs
    L = vs.lib()
    h = ctypes.c_void_p()
    st = vs.Stack()._c()
    bad_grid = vs.Grid(100, 0.01)._c()          # not a power of two
    rc = L.vs_make_kernel(ctypes.byref(st), ctypes.byref(bad_grid), None, ctypes.byref(h), None)
    assert rc == vs.VS_ERR_INVALID_ARG
    assert "power of two" in L.vs_last_error().decode()
    st.n_layers = 0
    rc = L.vs_make_kernel(ctypes.byref(st), ctypes.byref(vs.Grid(64, 0.01)._c()), None,
                          ctypes.byref(h), None)
    assert rc == vs.VS_ERR_INVALID_ARG and h.value is None
    # the warm-start plan rejects a missing kernel or model before touching the device
    prm = vs.SolveParams()._c()
    rc = L.vs_warm_plan_create(None, 4, None, None, None, None, None, None, None,
                               ctypes.byref(prm), ctypes.byref(h), None)
    assert rc == vs.VS_ERR_INVALID_ARG and h.value is None
    assert L.vs_warm_plan_run(None, vs.VS_WARM_ALL, None) == vs.VS_ERR_INVALID_ARG
    assert L.vs_warm_plan_launches(None) == 0
    L.vs_warm_plan_free(None)
    c, r = ctypes.c_int(), ctypes.c_int()
    assert L.vs_model_shape(None, ctypes.byref(c), ctypes.byref(r)) == vs.VS_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2307_12119_gb300 as vs
    monkeypatch.setattr(vs, "_lib", None)
    monkeypatch.setattr(vs, "lib_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="libvarsim.so not found"):
        vs.lib()


def test_solve_params_marshal_the_physics_variants():
    import paper_2307_12119_gb300 as vs
    p = vs.SolveParams(0.03, 1e-3, 1e-4, 40, vs.VS_PREC_FP32, vs.VS_ENGINE_STREAMED,
                       conductivity=vs.VS_COND_KIRCHHOFF, eta=1.3, t_amb_K=318.15,
                       leak_table=[(0.0, 1.0), (50.0, 2.5), (100.0, 5.0)])
    c = p._c()
    assert (c.beta_per_K, c.alpha_per_K, c.tol_K, c.max_iter) == (0.03, 1e-3, 1e-4, 40)
    assert (c.precision, c.engine, c.conductivity) == (0, 1, 1)
    assert (c.eta, c.t_amb_K, c.leak_points) == (1.3, 318.15, 3)
    assert list(c.leak_theta_K[:3]) == [0.0, 50.0, 100.0]
    assert list(c.leak_g[:3]) == [1.0, 2.5, 5.0]
    # the default struct selects the linear models
    d = vs.SolveParams()._c()
    assert d.conductivity == vs.VS_COND_LINEAR and d.leak_points == 0
    # ... and the update stopping rule; the last field of the C struct
    assert d.stop_rule == vs.VS_STOP_UPDATE
    assert vs.SolveParams(stop_rule=vs.VS_STOP_ESTIMATE)._c().stop_rule == 1
    assert ctypes.sizeof(vs._SolveParams) == vs._SolveParams.stop_rule.offset + 8


def test_invalid_physics_parameters_need_no_gpu(libpath):
    # parameter validation runs before any device work; vs_plan_create with no
    # items reports the parameter error first
    import paper_2307_12119_gb300 as vs
    L = vs.lib()
    h = ctypes.c_void_p()
    cases = (({"conductivity": 3}, "conductivity model"),
             ({"conductivity": vs.VS_COND_KIRCHHOFF, "eta": 1.0, "t_amb_K": 300.0}, "Kirchhoff"),
             ({"leak_table": [(0.0, 1.0)]}, "leak_points"),
             ({"leak_table": [(5.0, 1.0), (1.0, 2.0)]}, "must increase"),
             ({"stop_rule": 2}, "stopping rule"))
    for kw, msg in cases:
        prm = vs.SolveParams(**kw)._c()
        item = (vs._BatchItem * 1)()
        rc = L.vs_plan_create(item, 1, ctypes.byref(prm), ctypes.byref(h), None)
        assert rc == vs.VS_ERR_INVALID_ARG, kw
        assert msg in L.vs_last_error().decode(), (kw, L.vs_last_error())
