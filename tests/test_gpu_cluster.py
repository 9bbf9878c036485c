"""GPU parity of the cluster engine (one thread-block cluster per map, the map
held in shared memory for the whole solve) against the FP64 oracle and
against the streamed engine on the same inputs, plus its statuses, warm
starts, launch grouping and argument checks."""
import numpy as np
import pytest
import torch

import synth

from _util import (ENG_TOL_K, REQ_MAX_K, REQ_REL_L2, errors, inputs, oracle_spectrum,
                   oracle_steady, vs_params, vs_stack)

pytestmark = pytest.mark.gpu


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def _kernel(w):
    vs = _vs()
    return vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))


def _solve(k, pd, pl, s, prm, theta_init=None):
    vs = _vs()
    th = torch.empty_like(pd)
    items = [(k, pd[i], pl[i], s[i] if s is not None else None, th[i],
              None if theta_init is None else theta_init[i]) for i in range(pd.shape[0])]
    plan = vs.Plan(items, prm)
    plan.run()
    return th, plan.info(), plan.launches


@pytest.mark.parametrize("name", ["tiny_32", "c1_64", "c3_128", "c2_256"])
def test_cluster_matches_oracle_and_streamed(name):
    vs = _vs()
    w = synth.workload(name)
    k = _kernel(w)
    pd, pl, s = inputs(w, count=3)
    thc, ic, launches = _solve(k, pd, pl, s, vs_params(w, engine=vs.VS_ENGINE_CLUSTER))
    assert launches == 1
    ths, is_, _ = _solve(k, pd, pl, s, vs_params(w, engine=vs.VS_ENGINE_STREAMED))
    Kt = oracle_spectrum(w)
    for i in range(3):
        assert ic[i]["status"] == vs.VS_OK
        ref, it = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(thc[i], ref)
        assert emax <= REQ_MAX_K and rel <= REQ_REL_L2
        assert emax <= ENG_TOL_K, (i, emax)
        assert 1 <= ic[i]["iterations"] < it
        # same arithmetic as the streamed engine, only the data movement differs
        assert abs(ic[i]["iterations"] - is_[i]["iterations"]) <= 1
        assert float((thc[i] - ths[i]).abs().max()) <= 2e-4
        assert ic[i]["mu_W"] == pytest.approx(float(pl[i].double().mean()), rel=1e-12)
        assert ic[i]["residual_K"] <= 1e-4


def test_cluster_is_the_automatic_engine_and_groups_launches_by_size():
    vs = _vs()
    ws = [synth.workload("c3_128"), synth.workload("c3_256"), synth.workload("c1_64")]
    ks = [_kernel(w) for w in ws]
    items, outs = [], []
    for i in range(7):                              # ragged: 7 maps over 3 sizes
        w = ws[i % 3]
        pd, pl, s = inputs(w, first=i)
        th = torch.empty_like(pd[0])
        items.append((ks[i % 3], pd[0], pl[0], s[0], th))
    plan = vs.Plan(items, vs_params(ws[0]))
    assert plan.launches == 3                       # one cluster launch per grid size
    plan.run()
    infos = plan.info()
    assert all(i["status"] == vs.VS_OK for i in infos)
    spectra = {w.n: oracle_spectrum(w) for w in ws}
    for i, (k, pd, pl, s, th) in enumerate(items):
        w = ws[i % 3]
        ref, _ = oracle_steady(w, spectra[w.n], pd, pl, s)
        emax, rel = errors(th, ref)
        assert emax <= ENG_TOL_K and rel <= REQ_REL_L2, (i, emax, rel)
    # a plan with a map outside [32, 256] runs on the streamed engine
    w5 = synth.workload("c3_512")
    k5 = _kernel(w5)
    pd, pl, s = inputs(w5)
    th5 = torch.empty_like(pd[0])
    assert vs.Plan(items[:1] + [(k5, pd[0], pl[0], s[0], th5)], vs_params(w5)).launches == 1


def test_cluster_full_batch_is_deterministic_and_graph_capturable():
    vs = _vs()
    w = synth.workload("c3_256")
    k = _kernel(w)
    pd, pl, s = inputs(w, count=40)
    th = torch.empty_like(pd)
    plan = vs.Plan([(k, pd[i], pl[i], s[i], th[i]) for i in range(40)],
                   vs_params(w, engine=vs.VS_ENGINE_CLUSTER))
    plan.run()
    a = th.clone()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            plan.run(stream)
    torch.cuda.current_stream().wait_stream(stream)
    th.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, th)
    assert all(i["status"] == vs.VS_OK for i in plan.info())


def test_cluster_warm_start_mixed_with_cold_maps():
    vs = _vs()
    w = synth.workload("c3_256")
    k = _kernel(w)
    pd, pl, s = inputs(w, count=4)
    cold, ic, _ = _solve(k, pd, pl, s, vs_params(w, tol=1e-5, engine=vs.VS_ENGINE_CLUSTER))
    init = cold + 0.5                               # close, but not the fixed point
    th = torch.empty_like(pd)
    items = [(k, pd[i], pl[i], s[i], th[i], init[i] if i % 2 == 0 else None) for i in range(4)]
    plan = vs.Plan(items, vs_params(w, engine=vs.VS_ENGINE_CLUSTER))
    plan.run()
    iw = plan.info()
    Kt = oracle_spectrum(w)
    for i in range(4):
        assert iw[i]["status"] == vs.VS_OK
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, _ = errors(th[i], ref)
        assert emax <= ENG_TOL_K
    # a warm start from the answer itself stops after the confirming iterate
    th2 = torch.empty_like(pd)
    plan = vs.Plan([(k, pd[i], pl[i], s[i], th2[i], cold[i]) for i in range(4)],
                   vs_params(w, engine=vs.VS_ENGINE_CLUSTER))
    plan.run()
    assert all(i["iterations"] <= 2 for i in plan.info())
    # and it agrees with the streamed engine given the same warm start
    th3 = torch.empty_like(pd)
    ps = vs.Plan([(k, pd[i], pl[i], s[i], th3[i], init[i] if i % 2 == 0 else None)
                  for i in range(4)], vs_params(w, engine=vs.VS_ENGINE_STREAMED))
    ps.run()
    assert float((th3 - th).abs().max()) <= 2e-4


def test_cluster_statuses_and_isolation():
    vs = _vs()
    w = synth.workload("c1_64")
    k = _kernel(w)
    pd, pl, s = inputs(w)
    cl = dict(engine=vs.VS_ENGINE_CLUSTER)
    _, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, max_iter=1, **cl))
    assert info["status"] == vs.VS_ERR_NO_CONVERGENCE and info["iterations"] == 1
    _, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, beta_per_K=0.2, **cl))
    assert info["status"] == vs.VS_ERR_RUNAWAY and info["iterations"] == 0
    _, info = vs.solve_steady(k, pd[0] * 80, pl[0], s[0], vs_params(w, alpha_per_K=2e-3, **cl))
    assert info["status"] == vs.VS_ERR_RUNAWAY
    bad = pd[0].clone()
    bad[40, 7] = float("nan")                       # a row owned by the second CTA
    th = torch.empty(3, w.n, w.n, device="cuda")
    infos = vs.solve_batch([(k, pd[0], pl[0], s[0], th[0]), (k, bad, pl[0], s[0], th[1]),
                            (k, pd[0], pl[0], s[0], th[2])], vs_params(w, **cl))
    assert [i["status"] for i in infos] == [vs.VS_OK, vs.VS_ERR_NONFINITE, vs.VS_OK]
    assert torch.equal(th[0], th[2])
    # without a variation field (s = 1)
    th1, info = vs.solve_steady(k, pd[0], pl[0], None, vs_params(w, **cl))
    th2, _ = vs.solve_steady(k, pd[0], pl[0], None, vs_params(w, engine=vs.VS_ENGINE_STREAMED))
    assert info["status"] == vs.VS_OK
    assert float((th1 - th2).abs().max()) <= 2e-4


@pytest.mark.parametrize("max_iter", [2, 3])
def test_cluster_stops_at_max_iter_in_the_early_decision(max_iter):
    """From the second iterate the cluster engine decides before the forward
    transform along x; a map stopped there by max_iter reports
    VS_ERR_NO_CONVERGENCE after exactly max_iter iterates, and its map is the
    same iterate the streamed engine (which decides after the transform)
    stops at."""
    vs = _vs()
    w = synth.workload("c2_256")
    k = _kernel(w)
    pd, pl, s = inputs(w, count=3)
    prm = lambda eng: vs_params(w, tol=1e-9, max_iter=max_iter, engine=eng)
    th_c, inf_c, _ = _solve(k, pd, pl, s, prm(vs.VS_ENGINE_CLUSTER))
    th_s, inf_s, _ = _solve(k, pd, pl, s, prm(vs.VS_ENGINE_STREAMED))
    for a, b in zip(inf_c, inf_s):
        assert a["status"] == b["status"] == vs.VS_ERR_NO_CONVERGENCE
        assert a["iterations"] == b["iterations"] == max_iter
        assert abs(a["residual_K"] - b["residual_K"]) <= 1e-3 * max(1.0, b["residual_K"])
    assert float((th_c - th_s).abs().max()) <= ENG_TOL_K


def test_cluster_argument_checks():
    vs = _vs()
    for name in ("tiny_16", "c3_512"):               # outside [32, 256]
        w = synth.workload(name)
        k = _kernel(w)
        pd, pl, s = inputs(w)
        with pytest.raises(vs.VarsimError):
            vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, engine=vs.VS_ENGINE_CLUSTER))
    # split precision with the cluster engine means the on-chip pair engine:
    # n = 256 only
    w = synth.workload("c3_128")
    k = _kernel(w)
    pd, pl, s = inputs(w)
    with pytest.raises(vs.VarsimError):
        vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, precision=vs.VS_PREC_BF16_SPLIT,
                                                          engine=vs.VS_ENGINE_CLUSTER))
    w = synth.workload("c3_256")
    k = _kernel(w)
    pd, pl, s = inputs(w)
    _, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, tol_K=1e-2,
                                                               precision=vs.VS_PREC_BF16_SPLIT,
                                                               engine=vs.VS_ENGINE_CLUSTER))
    assert info["status"] == vs.VS_OK
    with pytest.raises(vs.VarsimError):
        vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, engine=7))
