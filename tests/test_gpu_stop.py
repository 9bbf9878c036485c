"""The error-estimate stopping rule (VS_STOP_ESTIMATE) on every steady engine:
maps within the tolerance of the FP64 oracle's fixed point, fewer iterations
than the update rule, and the argument checks."""
import numpy as np
import pytest
import torch

import synth

from _util import REQ_MAX_K, REQ_REL_L2, errors, oracle_spectrum, oracle_steady, vs_params, vs_stack

pytestmark = pytest.mark.gpu

SPLIT_TOL_K = 1e-2


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def _run(vs, k, pd, pl, s, prm):
    th = torch.empty_like(pd)
    plan = vs.Plan([(k, pd[i], pl[i], s[i], th[i]) for i in range(pd.shape[0])], prm)
    plan.run()
    return th, plan.info()


def _picks(infos, th, count):
    iters = np.array([i["iterations"] for i in infos])
    rise = th.amax(dim=(1, 2)).cpu().numpy()
    picks = list(np.argsort(iters, kind="stable")[:4]) + list(np.argsort(-rise)[:4])
    picks = set(int(i) for i in picks)
    spread = iter(range(0, count, max(1, count // 16)))
    while len(picks) < min(16, count):
        picks.add(next(spread))
    return sorted(picks)


def test_estimate_rule_headline_batch_on_the_cluster_engine():
    """4096 maps of 256 x 256 on the cluster engine at 1e-2 K: every status,
    fewer iterations than the update rule, and 16+ maps (the 4 stopped
    earliest, the 4 with the largest rise, 8 spread over the batch) within
    1e-2 K of the oracle's fixed point (and the metric's 0.05 K, rel-L2 1e-4)."""
    vs = _vs()
    w, pd, pl, s = synth.batch_inputs(256, 4096, seed=synth.SEED)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    tol = 1e-2
    upd = dict(tol=tol, engine=vs.VS_ENGINE_CLUSTER)
    th_u, inf_u = _run(vs, k, pd, pl, s, vs_params(w, **upd))
    th, infos = _run(vs, k, pd, pl, s, vs_params(w, stop_rule=vs.VS_STOP_ESTIMATE, **upd))
    assert all(i["status"] == vs.VS_OK for i in infos)
    it_u = np.mean([i["iterations"] for i in inf_u])
    it_e = np.mean([i["iterations"] for i in infos])
    print("cluster engine at 1e-2 K: update rule %.3f iterations, estimate rule %.3f" % (it_u, it_e))
    assert it_e < it_u
    assert float((th - th_u).abs().max()) <= tol
    picks = _picks(infos, th, 4096)
    assert len(picks) >= 16
    Kt = oracle_spectrum(w)
    worst = 0.0
    for i in picks:
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(th[i], ref)
        assert emax <= tol and emax <= REQ_MAX_K and rel <= REQ_REL_L2, (i, emax, rel)
        worst = max(worst, emax)
    print("estimate rule: %d maps checked, worst max|dT| %.2e K" % (len(picks), worst))


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_estimate_rule_on_the_streamed_engine(tol):
    vs = _vs()
    w, pd, pl, s = synth.batch_inputs(256, 64, seed=synth.SEED + 5)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    eng = dict(tol=tol, engine=vs.VS_ENGINE_STREAMED)
    _, inf_u = _run(vs, k, pd, pl, s, vs_params(w, **eng))
    th, infos = _run(vs, k, pd, pl, s, vs_params(w, stop_rule=vs.VS_STOP_ESTIMATE, **eng))
    assert all(i["status"] == vs.VS_OK for i in infos)
    assert np.mean([i["iterations"] for i in infos]) < np.mean([i["iterations"] for i in inf_u])
    Kt = oracle_spectrum(w)
    for i in _picks(infos, th, 64)[:6]:
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(th[i], ref)
        # FP32 rounding of the engine (~1e-4 K at 100 K rises) on top of the rule's error
        assert emax <= tol + 2e-4 and rel <= REQ_REL_L2, (i, emax, rel)


def test_estimate_rule_on_the_pair_engine():
    vs = _vs()
    w, pd, pl, s = synth.batch_inputs(256, 64, seed=synth.SEED + 6)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    split = dict(tol=SPLIT_TOL_K, precision=vs.VS_PREC_BF16_SPLIT)
    _, inf_u = _run(vs, k, pd, pl, s, vs_params(w, **split))
    th, infos = _run(vs, k, pd, pl, s, vs_params(w, stop_rule=vs.VS_STOP_ESTIMATE, **split))
    assert all(i["status"] == vs.VS_OK for i in infos)
    assert np.mean([i["iterations"] for i in infos]) < np.mean([i["iterations"] for i in inf_u])
    Kt = oracle_spectrum(w)
    for i in _picks(infos, th, 64)[:6]:
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(th[i], ref)
        assert emax <= SPLIT_TOL_K and rel <= REQ_REL_L2, (i, emax, rel)


def test_stopping_rule_arguments():
    vs = _vs()
    w = synth.workload("c1_64")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    z = torch.zeros(1, 64, 64, device="cuda")
    with pytest.raises(vs.VarsimError) as e:
        vs.Plan([(k, z[0], z[0], None, z[0].clone())], vs_params(w, stop_rule=7))
    assert e.value.status == vs.VS_ERR_INVALID_ARG
    kt = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=1e-3))
    trace = torch.zeros(3, 64, 64, device="cuda")
    # the transient takes either rule (it applies to the implicit per-step fixed point)
    for leakage in (vs.VS_LEAK_LAGGED, vs.VS_LEAK_IMPLICIT):
        th, info = vs.solve_transient(kt, trace, z[0], None,
                                      vs_params(w, stop_rule=vs.VS_STOP_ESTIMATE), leakage=leakage)
        assert info["status"] == vs.VS_OK and float(th.abs().max()) == 0.0
    with pytest.raises(vs.VarsimError) as e:
        vs.solve_transient(kt, trace, z[0], None, vs_params(w, stop_rule=7))
    assert e.value.status == vs.VS_ERR_INVALID_ARG
