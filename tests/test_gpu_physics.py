"""GPU parity of the physics variants (piecewise-linear leakage, Sec. II-E;
kappa(T) through the Kirchhoff transform, Eq. 10) against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import solve as so

from _util import errors, oracle_spectrum, vs_params, vs_stack

pytestmark = pytest.mark.gpu

T_AMB, ETA = 318.15, 1.3
# exp(0.0275 theta): a leakage that grows faster than linear (the 64^2 maps
# converge with it; the hotter 256^2 maps run away, also in the oracle)
EXP_TABLE = [(x, float(np.exp(0.0275 * x))) for x in (0.0, 25.0, 50.0, 75.0, 100.0, 150.0, 250.0)]
# 1 + beta theta (1 + theta / 400): convex, converges on the 256^2 maps
CONVEX_TABLE = [(x, 1.0 + 0.0275 * x * (1.0 + x / 400.0))
                for x in (0.0, 25.0, 50.0, 75.0, 100.0, 150.0, 200.0, 300.0)]


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def _case(config, count, n=None):
    vs = _vs()
    w = synth.workload(config)
    if n is not None:
        w = dataclasses.replace(w, name="%s_%d" % (config, n), n=n)
    pd, pl, s = synth.steady_inputs(w, count, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    return vs, w, k, pd, pl, s


def _params(vs, w, kirchhoff, table, **kw):
    p = vs_params(w, **kw)
    if kirchhoff:
        p.conductivity, p.eta, p.t_amb_K = vs.VS_COND_KIRCHHOFF, ETA, T_AMB
    if table:
        p.leak_table = table
    return p


def _oracle(w, pd, pl, s, kirchhoff, table):
    Kt = oracle_spectrum(w)
    beta, alpha = w.physics.beta_per_K, w.physics.alpha_per_K
    leak = (lambda th: so.leak_pwl(th, [x for x, _ in table], [g for _, g in table])) if table \
        else (lambda th: 1.0 + beta * th)
    field = (lambda v: so.kirchhoff_theta(v, ETA, T_AMB)) if kirchhoff \
        else (lambda v: v / (1.0 - alpha * v))
    f64 = lambda t: t.double().cpu().numpy()
    th, _, _ = so.picard_physics(lambda x: so.spectral_convolve(Kt, x), f64(pd), f64(pl), f64(s),
                                 leak, field, tol=1e-10)
    return th


@pytest.mark.parametrize("engine", [1, 2])          # streamed, cluster
@pytest.mark.parametrize("kirchhoff,table", [(True, None), (False, EXP_TABLE), (True, EXP_TABLE),
                                             (False, CONVEX_TABLE), (True, CONVEX_TABLE)])
@pytest.mark.parametrize("config,n", [("c1_64", None), ("c2_256", None), ("c1_64", 128)])
def test_physics_variants_match_oracle(config, n, kirchhoff, table, engine):
    if config == "c2_256" and table is EXP_TABLE:
        pytest.skip("thermal runaway of the exponential leakage on these maps (oracle too)")
    vs, w, k, pd, pl, s = _case(config, 2, n)
    th = torch.empty_like(pd)
    # the stronger couplings contract slowly (an update of 1e-3 K can leave
    # 1e-2 K of error): stop at 2e-4 K and allow more iterations
    infos = vs.solve_batch([(k, pd[b], pl[b], s[b], th[b]) for b in range(2)],
                           _params(vs, w, kirchhoff, table, tol=2e-4, max_iter=400, engine=engine))
    for b in range(2):
        assert infos[b]["status"] == vs.VS_OK, infos[b]
        emax, rel = errors(th[b], _oracle(w, pd[b], pl[b], s[b], kirchhoff, table))
        assert emax <= 5e-3 and rel <= 2e-4, (b, emax, rel)


def test_linear_table_equals_the_linear_model():
    vs, w, k, pd, pl, s = _case("c2_256", 2)
    beta = w.physics.beta_per_K
    table = [(0.0, 1.0), (300.0, 1.0 + 300.0 * beta)]
    a = torch.empty_like(pd)
    b = torch.empty_like(pd)
    ia = vs.solve_batch([(k, pd[i], pl[i], s[i], a[i]) for i in range(2)],
                        vs_params(w, tol=1e-4, engine=vs.VS_ENGINE_STREAMED))
    infos = vs.solve_batch([(k, pd[i], pl[i], s[i], b[i]) for i in range(2)],
                           _params(vs, w, False, table, tol=1e-4))
    assert all(i["status"] == vs.VS_OK for i in ia + infos)
    # the same arithmetic up to the table's interpolation in FP32
    assert float((a - b).abs().max()) <= 2e-3


def test_physics_variant_full_batch_and_warm_start():
    vs = _vs()
    w, pd, pl, s = synth.batch_inputs(256, 4096, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    prm = _params(vs, w, True, CONVEX_TABLE, tol=1e-3, max_iter=200)
    th = torch.empty_like(pd)
    infos = vs.solve_batch([(k, pd[b], pl[b], s[b], th[b]) for b in range(4096)], prm)
    assert all(i["status"] == vs.VS_OK for i in infos)
    for b in (0, 2049, 4095):
        emax, rel = errors(th[b], _oracle(w, pd[b], pl[b], s[b], True, CONVEX_TABLE))
        assert emax <= 5e-3 and rel <= 2e-4, (b, emax, rel)
    # a warm start from a perturbed solution reaches the same fixed point
    th2 = torch.empty_like(pd[:4])
    init = (th[:4] * 0.9).contiguous()
    infos = vs.solve_batch([(k, pd[b], pl[b], s[b], th2[b], init[b]) for b in range(4)],
                           _params(vs, w, True, CONVEX_TABLE, tol=1e-3, max_iter=200))
    assert all(i["status"] == vs.VS_OK for i in infos)
    assert float((th2 - th[:4]).abs().max()) <= 1e-2


def test_physics_variants_on_both_engines_agree():
    """The cluster engine (the automatic choice for n <= 256) and the streamed
    engine give the same maps for the physics variants, warm starts included;
    the cluster engine's physics instantiation has one launch shape."""
    vs, w, k, pd, pl, s = _case("c2_256", 3)
    out = {}
    for eng in (vs.VS_ENGINE_STREAMED, vs.VS_ENGINE_CLUSTER):
        th = torch.empty_like(pd)
        # as in the oracle parity test: these couplings contract slowly, so stop
        # at 2e-4 K with room for iterations
        prm = _params(vs, w, True, CONVEX_TABLE, tol=2e-4, max_iter=400, engine=eng)
        infos = vs.solve_batch([(k, pd[b], pl[b], s[b], th[b]) for b in range(3)], prm)
        assert all(i["status"] == vs.VS_OK for i in infos), [(i["status"], i["iterations"]) for i in infos]
        init = (th * 0.95).contiguous()
        th2 = torch.empty_like(pd)
        infos = vs.solve_batch([(k, pd[b], pl[b], s[b], th2[b], init[b]) for b in range(3)], prm)
        assert all(i["status"] == vs.VS_OK for i in infos), [(i["status"], i["iterations"]) for i in infos]
        out[eng] = (th, th2)
    a, b = out[vs.VS_ENGINE_STREAMED], out[vs.VS_ENGINE_CLUSTER]
    assert float((a[0] - b[0]).abs().max()) <= 5e-3
    assert float((a[1] - b[1]).abs().max()) <= 5e-3
    z = torch.empty_like(pd[0])
    with pytest.raises(vs.VarsimError) as e:
        vs.Plan([(k, pd[0], pl[0], s[0], z)], _params(vs, w, True, None, engine=vs.VS_ENGINE_CLUSTER),
                shape=4)
    assert e.value.status == vs.VS_ERR_INVALID_ARG


def test_physics_variants_are_rejected_where_not_supported():
    vs, w, k, pd, pl, s = _case("c1_64", 1)
    prm = _params(vs, w, True, None)
    with pytest.raises(vs.VarsimError):
        vs.solve_steady_noalloc(k, pd[0], pl[0], s[0], prm)
    with pytest.raises(vs.VarsimError):
        vs.solve_closed_form(k, pd, pl, s, prm)
    bad = _params(vs, w, False, [(10.0, 1.0), (5.0, 2.0)])       # temperatures not increasing
    with pytest.raises(vs.VarsimError):
        vs.solve_steady(k, pd[0], pl[0], s[0], bad)


def test_kirchhoff_runaway_is_reported():
    vs, w, k, pd, pl, s = _case("c1_64", 1)
    hot = (pd[0] * 40).contiguous()       # s u beyond T_amb / (eta - 1)
    th, info = vs.solve_steady(k, hot, pl[0], s[0], _params(vs, w, True, None, beta_per_K=0.0))
    assert info["status"] == vs.VS_ERR_RUNAWAY
