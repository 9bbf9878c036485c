"""GPU parity of the steady solve (single map and batched persistent plans)
against the FP64 oracle, plus status/edge cases."""
import numpy as np
import pytest
import torch

import synth
from oracle import physics as ph
from oracle import solve as so

from _util import (ENG_TOL_K, REQ_MAX_K, REQ_REL_L2, errors, inputs, oracle_spectrum,
                   oracle_steady, vs_params, vs_stack)

pytestmark = pytest.mark.gpu


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def _kernel(w):
    vs = _vs()
    return vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))


@pytest.mark.parametrize("name", ["c1_64", "tiny_8", "tiny_16", "tiny_32", "c1_64/spherical"])
def test_single_map_matches_oracle(name):
    vs = _vs()
    w = synth.workload(name.split("/")[0])
    if name.endswith("/spherical"):
        w.corr = "spherical"                    # spherical correlation of the variation
    pd, pl, s = inputs(w)
    k = _kernel(w)
    th, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK
    ref, it = oracle_steady(w, oracle_spectrum(w), pd[0], pl[0], s[0])
    emax, rel = errors(th, ref)
    assert emax <= REQ_MAX_K and rel <= REQ_REL_L2
    assert emax <= ENG_TOL_K
    # the split iteration converges in fewer steps than plain Picard
    assert 1 <= info["iterations"] < it
    assert info["mu_W"] == pytest.approx(float(pl[0].double().mean()), rel=1e-12)


def test_full_size_256_single_map():
    vs = _vs()
    w = synth.workload("c2_256")
    pd, pl, s = inputs(w)
    k = _kernel(w)
    th, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK
    ref, _ = oracle_steady(w, oracle_spectrum(w), pd[0], pl[0], s[0])
    emax, rel = errors(th, ref)
    assert emax <= ENG_TOL_K and rel <= REQ_REL_L2


def test_uniform_variation_reduces_to_shift_invariant_closed_form():
    vs = _vs()
    w = synth.workload("c1_64")
    w.sigma = (0.0, 0.0)
    pd, pl, s = inputs(w)
    assert float(pl[0].max() - pl[0].min()) == 0.0
    k = _kernel(w)
    th, info = vs.solve_steady(k, pd[0], pl[0], None, vs_params(w, alpha_per_K=0.0))
    assert info["status"] == vs.VS_OK
    closed = so.shift_invariant(oracle_spectrum(w), pd[0].double().cpu().numpy(),
                                pl[0].double().cpu().numpy(), w.physics.beta_per_K)
    emax, rel = errors(th, closed)
    assert emax <= ENG_TOL_K
    # with no variation the first iterate is already the answer
    assert info["iterations"] <= 2


def test_linear_case_equals_plain_convolution():
    # beta = alpha = 0, s = 1: theta = L[P_dyn + P_leak0] exactly (one iteration)
    vs = _vs()
    w = synth.workload("c1_64")
    pd, pl, s = inputs(w)
    k = _kernel(w)
    th, info = vs.solve_steady(k, pd[0], pl[0], None, vs_params(w, beta_per_K=0.0, alpha_per_K=0.0))
    Kt = oracle_spectrum(w)
    ref = so.spectral_convolve(Kt, (pd[0] + pl[0]).double().cpu().numpy())
    emax, rel = errors(th, ref)
    assert emax <= 5e-4 and rel <= 2e-6
    assert info["iterations"] == 2          # the second iterate confirms convergence


def test_energy_balance_and_symmetry():
    vs = _vs()
    w = synth.workload("c1_64")
    k = _kernel(w)
    n = w.n
    yy, xx = torch.meshgrid(torch.arange(n), torch.arange(n), indexing="ij")
    q = (((xx + yy) % 2).float() * 0.004).cuda().contiguous()      # TC5 checkerboard
    zero = torch.zeros_like(q)
    th, _ = vs.solve_steady(k, q, zero, None, vs_params(w, beta_per_K=0.0, alpha_per_K=0.0))
    Kt = k.spectrum()
    assert float(th.double().mean()) == pytest.approx(Kt[0, 0] * float(q.double().mean()), rel=2e-6)
    t = th.cpu().numpy()
    assert np.max(np.abs(t - t.T)) <= 2e-5 * t.max()
    assert np.max(np.abs(t - t[::-1, ::-1])) <= 2e-5 * t.max()


def test_batch_mixed_sizes_matches_single_and_oracle():
    vs = _vs()
    ws = [synth.workload("c3_128"), synth.workload("c3_256"), synth.workload("c3_512")]
    kernels = [_kernel(w) for w in ws]
    items, refs = [], []
    for i in range(5):                              # ragged: 5 maps over 3 sizes
        w = ws[i % 3]
        pd, pl, s = inputs(w, first=i)
        th = torch.empty_like(pd[0])
        items.append((kernels[i % 3], pd[0], pl[0], s[0], th))
    # n = 512 puts the plan on the streamed engine; the single solves use it too
    streamed = dict(engine=vs.VS_ENGINE_STREAMED)
    infos = vs.solve_batch(items, vs_params(ws[0]))
    assert all(i["status"] == vs.VS_OK for i in infos)
    spectra = {w.n: oracle_spectrum(w) for w in ws}
    for i, (k, pd, pl, s, th) in enumerate(items):
        w = ws[i % 3]
        single, info1 = vs.solve_steady(k, pd, pl, s, vs_params(w, **streamed))
        assert info1["iterations"] == infos[i]["iterations"]
        assert float((single - th).abs().max()) <= 1e-4
        if i < 3:
            ref, _ = oracle_steady(w, spectra[w.n], pd, pl, s)
            emax, rel = errors(th, ref)
            assert emax <= ENG_TOL_K and rel <= REQ_REL_L2


@pytest.mark.parametrize("engine", [1, 2])          # streamed, cluster
def test_batch_is_deterministic_and_graph_capturable(engine):
    vs = _vs()
    w = synth.workload("c3_256")
    k = _kernel(w)
    pd, pl, s = inputs(w, count=12)
    th = torch.empty_like(pd)
    plan = vs.Plan([(k, pd[i], pl[i], s[i], th[i]) for i in range(12)],
                   vs_params(w, engine=engine))
    plan.run()
    a = th.clone()
    th.zero_()
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


def test_status_no_convergence_runaway_nonfinite():
    vs = _vs()
    w = synth.workload("c1_64")
    pd, pl, s = inputs(w)
    k = _kernel(w)
    _, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, max_iter=1))
    assert info["status"] == vs.VS_ERR_NO_CONVERGENCE
    _, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, beta_per_K=0.2))
    assert info["status"] == vs.VS_ERR_RUNAWAY          # beta mu max(K) >= 1
    _, info = vs.solve_steady(k, pd[0] * 80, pl[0], s[0], vs_params(w, alpha_per_K=2e-3))
    assert info["status"] == vs.VS_ERR_RUNAWAY          # 1 - alpha s u <= 0.05
    bad = pd[0].clone()
    bad[3, 5] = float("nan")
    _, info = vs.solve_steady(k, bad, pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_ERR_NONFINITE
    # a bad map in a batch does not abort the others
    th = torch.empty(2, w.n, w.n, device="cuda")
    infos = vs.solve_batch([(k, bad, pl[0], s[0], th[0]), (k, pd[0], pl[0], s[0], th[1])],
                           vs_params(w))
    assert [i["status"] for i in infos] == [vs.VS_ERR_NONFINITE, vs.VS_OK]


def test_argument_checks():
    vs = _vs()
    w = synth.workload("c1_64")
    pd, pl, s = inputs(w)
    k = _kernel(w)
    with pytest.raises(vs.VarsimError):
        vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, tol_K=0.0))
    with pytest.raises(ValueError):
        vs.solve_steady(k, pd[0][:32], pl[0], s[0], vs_params(w))
    with pytest.raises(vs.VarsimError):                     # transient needs dt
        vs.solve_transient(k, pd, pl[0], s[0], vs_params(w))


def test_plans_with_different_footprints_coexist():
    # a small plan created after a large one must not break the large one
    vs = _vs()
    big, small = synth.workload("c3_512"), synth.workload("tiny_16")
    kb, ks = _kernel(big), _kernel(small)
    pd, pl, s = inputs(big, count=2)
    th = torch.empty_like(pd)
    plan = vs.Plan([(kb, pd[i], pl[i], s[i], th[i]) for i in range(2)], vs_params(big))
    plan.run()
    a = th.clone()
    qd, ql, qs = inputs(small)
    vs.solve_steady(ks, qd[0], ql[0], qs[0], vs_params(small))
    th.zero_()
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(a, th)


@pytest.mark.parametrize("engine", [1, 2])          # streamed, cluster
def test_uniform_maps_converge_from_the_uniform_start(engine):
    # Uniform P_dyn and P_leak0 (s = 1): the fixed point is the uniform mode
    # u = K00 (P_dyn + P_leak0 (1 + beta phi(u))), which the cold start solves
    # as a scalar before the first transform, so the first iterate is already
    # the answer and the solve stops after one iteration.
    vs = _vs()
    w = synth.workload("c2_256")
    k = _kernel(w)
    Kt = oracle_spectrum(w)
    beta, alpha = w.physics.beta_per_K, w.physics.alpha_per_K
    c, m = 2.0e-3, 1.0e-3                                   # W per cell
    u = 0.0
    for _ in range(200):                                    # FP64 scalar fixed point
        u = Kt[0, 0] * (c + m * (1.0 + beta * u / (1.0 - alpha * u)))
    theta_star = u / (1.0 - alpha * u)
    pd = torch.full((w.n, w.n), c, device="cuda")
    pl = torch.full((w.n, w.n), m, device="cuda")
    th, info = vs.solve_steady(k, pd, pl, None, vs_params(w, tol=1e-2, engine=engine))
    assert info["status"] == vs.VS_OK and info["iterations"] == 1
    assert float((th.double() - theta_star).abs().max()) <= 1e-3 * theta_star
