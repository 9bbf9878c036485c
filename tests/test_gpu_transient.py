"""GPU parity of the transient (per-mode recursion of the superposition of
power differences) against the oracle's untruncated Duhamel sum."""
import numpy as np
import pytest
import torch

import synth
from oracle import physics as ph
from oracle import solve as so

from _util import REQ_MAX_K, errors, vs_params, vs_stack

pytestmark = pytest.mark.gpu


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def test_markov_trace_matches_duhamel():
    vs = _vs()
    w = synth.workload("c1_64")
    dt, steps = 1e-3, 30
    trace = synth.markov_trace(w, steps, device="cuda")
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    st = w.stack
    spectra = [so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                                st.heat_cap_J_m2K, j * dt) for j in range(1, steps + 1)]
    f64 = lambda t: t.double().cpu().numpy()
    ref = so.duhamel(spectra, f64(trace), f64(pl[0]), f64(s[0]), w.physics.beta_per_K,
                     w.physics.alpha_per_K)
    emax, rel = errors(th, ref)
    assert emax <= REQ_MAX_K
    assert emax <= 5e-3 and rel <= 2e-4


def test_constant_power_reaches_steady_state():
    vs = _vs()
    w = synth.workload("c1_64")
    w.stack.heat_cap_J_m2K = 20.0            # tau ~ 1.4 ms: settled after 150 steps
    dt, steps = 1e-3, 150
    pd, pl, s = synth.steady_inputs(w, 1, device="cuda")
    trace = pd[0].expand(steps, w.n, w.n).contiguous()
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    ss, _ = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w, tol_K=1e-5))
    assert info["status"] == vs.VS_OK
    assert float((th[-1] - ss).abs().max()) <= 2e-3
    mid = th[:, 20, 20].cpu().numpy()
    assert np.all(np.diff(mid) >= -1e-4)       # monotone heating from ambient


def test_transient_first_step_is_single_pole_response():
    # uniform power, no leakage: theta_1 = P (K - A + A (1 - rho)) per mode
    vs = _vs()
    w = synth.workload("c1_64")
    dt = 2e-3
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    q = torch.full((3, w.n, w.n), 1e-3, device="cuda")
    zero = torch.zeros(w.n, w.n, device="cuda")
    th, _ = vs.solve_transient(k, q, zero, None, vs_params(w, beta_per_K=0.0, alpha_per_K=0.0))
    st = w.stack
    for j in range(3):
        S = so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                             st.heat_cap_J_m2K, (j + 1) * dt)
        assert float(th[j].double().mean()) == pytest.approx(1e-3 * S[0, 0], rel=1e-4)


# ---------------------------------------------------------------- variants

def _tr_case(steps, dt=1e-3, config="c1_64"):
    vs = _vs()
    w = synth.workload(config)
    trace = synth.markov_trace(w, steps, device="cuda")
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    return vs, w, k, trace, pl[0], s[0]


def _oracle_variant(w, trace, pl, s, dt, window, implicit):
    st = w.stack
    need = trace.shape[0] if window == 0 else min(window - 1, trace.shape[0])
    spectra = [so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                                st.heat_cap_J_m2K, j * dt) for j in range(1, need + 1)]
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    f64 = lambda t: t.double().cpu().numpy()
    return so.transient_variants(spectra, Kt, f64(trace), f64(pl), f64(s), w.physics.beta_per_K,
                                 w.physics.alpha_per_K, window=window, implicit=implicit,
                                 tol=1e-10)


@pytest.mark.parametrize("window", [1, 2, 5, 12])
def test_windowed_superposition_matches_oracle(window):
    dt, steps = 1e-3, 24
    vs, w, k, trace, pl, s = _tr_case(steps, dt)
    th, info = vs.solve_transient(k, trace, pl, s, vs_params(w), window=window)
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    ref, _ = _oracle_variant(w, trace, pl, s, dt, window, False)
    emax, rel = errors(th, ref)
    assert emax <= 5e-3 and rel <= 2e-4


@pytest.mark.parametrize("window", [0, 5])
def test_implicit_leakage_matches_oracle(window):
    dt, steps = 1e-3, 16
    vs, w, k, trace, pl, s = _tr_case(steps, dt)
    th, info = vs.solve_transient(k, trace, pl, s, vs_params(w, tol_K=1e-4), window=window,
                                  leakage=vs.VS_LEAK_IMPLICIT)
    assert info["status"] == vs.VS_OK
    assert info["residual_K"] <= 1e-4
    ref, its = _oracle_variant(w, trace, pl, s, dt, window, True)
    emax, rel = errors(th, ref)
    assert emax <= 5e-3 and rel <= 2e-4
    # the GPU stops at 1e-4 K, the oracle at 1e-10 K: it takes fewer iterations
    assert steps <= info["iterations"] <= int(its.sum())
    # the implicit solution differs from the lagged one by more than the tolerance
    lag, _ = vs.solve_transient(k, trace, pl, s, vs_params(w), window=window)
    assert float((th - lag).abs().max()) > 1e-3


@pytest.mark.parametrize("config", ["c1_64", "c2_256"])
def test_implicit_reports_unconverged_steps(config):
    # 64^2 runs on the general engine, 256^2 on the persistent one
    vs, w, k, trace, pl, s = _tr_case(6, config=config)
    th, info = vs.solve_transient(k, trace, pl, s, vs_params(w, tol_K=1e-9, max_iter=2),
                                  leakage=vs.VS_LEAK_IMPLICIT)
    assert info["status"] == vs.VS_ERR_NO_CONVERGENCE
    assert info["iterations"] == 12 and info["residual_K"] > 1e-9
    assert bool(torch.isfinite(th).all())


@pytest.mark.parametrize("config,steps", [("c2_256", 40), ("c4_1024", 200)])
def test_variants_reduce_to_the_untruncated_lagged_solve(config, steps):
    # properties that hold at any size, checked at the bench's 1024^2 x 200:
    # a window longer than the trace is the untruncated sum, and without
    # leakage feedback the implicit steps equal the lagged ones
    vs, w, k, trace, pl, s = _tr_case(steps, 1e-3, config)
    prm = vs_params(w)
    ref, _ = vs.solve_transient(k, trace, pl, s, prm)
    long_, info = vs.solve_transient(k, trace, pl, s, prm, window=min(steps + 1, vs.VS_MAX_WINDOW))
    assert info["status"] == vs.VS_OK
    scale = float(ref.abs().max())
    assert float((long_ - ref).abs().max()) <= 2e-5 * scale
    nofb = vs_params(w, beta_per_K=0.0)
    a, _ = vs.solve_transient(k, trace, pl, s, nofb)
    b, info = vs.solve_transient(k, trace, pl, s, nofb, leakage=vs.VS_LEAK_IMPLICIT)
    assert info["status"] == vs.VS_OK and info["iterations"] <= 2 * steps
    assert float((a - b).abs().max()) <= 2e-5 * scale


def test_transient_options_are_validated():
    vs, w, k, trace, pl, s = _tr_case(2)
    for kw in ({"window": -1}, {"window": vs.VS_MAX_WINDOW + 1}, {"leakage": 7}):
        with pytest.raises(vs.VarsimError) as e:
            vs.solve_transient(k, trace, pl, s, vs_params(w), **kw)
        assert e.value.status == vs.VS_ERR_INVALID_ARG


def test_persistent_engine_at_512_against_the_oracle():
    """The single-map persistent transient engine at 512^2 (the 256^2 and
    1024^2 cases run in test_gpu_configs): 12 steps of a Markov trace with
    leakage and conductivity, element by element against the oracle."""
    from _util import step_spectra
    vs = _vs()
    w = synth.workload("c3_512")
    dt, steps = 1e-3, 12
    trace = synth.markov_trace(w, steps, device="cuda")
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    spectra = step_spectra(w, dt, steps)
    f64 = lambda t: t.double().cpu().numpy()
    ref = so.duhamel_modes(spectra, f64(trace), f64(pl[0]), f64(s[0]), w.physics.beta_per_K,
                           w.physics.alpha_per_K)
    emax, rel = errors(th, ref)
    assert emax <= REQ_MAX_K
    assert emax <= 5e-3 and rel <= 2e-4


def test_persistent_engine_implicit_leakage_at_256_against_the_oracle():
    """Implicit leakage on the persistent engine (256^2, 10 steps): every step
    iterated to 1e-4 K against the oracle's implicit superposition (iterated
    to 1e-10 K), element by element; fewer iterations than the oracle, at
    least one per step, and a result that differs from the lagged solve."""
    from _util import step_spectra
    vs = _vs()
    w = synth.workload("c2_256")
    dt, steps = 1e-3, 10
    trace = synth.markov_trace(w, steps, device="cuda")
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w, tol_K=1e-4),
                                  leakage=vs.VS_LEAK_IMPLICIT)
    assert info["status"] == vs.VS_OK and info["residual_K"] <= 1e-4
    spectra = step_spectra(w, dt, steps)
    st = w.stack
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    f64 = lambda t: t.double().cpu().numpy()
    ref, its = so.transient_variants(spectra, Kt, f64(trace), f64(pl[0]), f64(s[0]),
                                     w.physics.beta_per_K, w.physics.alpha_per_K, implicit=True,
                                     tol=1e-10)
    emax, rel = errors(th, ref)
    print("implicit 256^2: %d iterations over %d steps (oracle %d), max |dT| %.2e K"
          % (info["iterations"], steps, int(its.sum()), emax))
    assert emax <= 5e-3 and rel <= 2e-4
    assert steps <= info["iterations"] <= int(its.sum())
    lag, _ = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    assert float((th - lag).abs().max()) > 1e-3


@pytest.mark.parametrize("window", [1, 2, 5])
def test_persistent_engine_window_at_256_against_the_oracle(window):
    """The windowed superposition (lagged leakage) on the persistent engine at
    256^2: 12 steps against the oracle's windowed sum, element by element."""
    vs = _vs()
    dt, steps = 1e-3, 12
    vs_, w, k, trace, pl, s = _tr_case(steps, dt, "c2_256")
    th, info = vs.solve_transient(k, trace, pl, s, vs_params(w), window=window)
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    ref, _ = _oracle_variant(w, trace, pl, s, dt, window, False)
    emax, rel = errors(th, ref)
    assert emax <= 5e-3 and rel <= 2e-4


@pytest.mark.parametrize("config,steps", [("c3_512", 10), ("c4_1024", 8)])
def test_persistent_engine_window_at_512_and_1024_against_the_oracle(config, steps):
    """The paper's 5-step window on the persistent engine at 512^2 and at the
    bench's 1024^2 (where the row phase runs pass 0 in registers): the ring of
    the last four differences wraps at least once, element by element against
    the oracle's windowed sum."""
    vs = _vs()
    dt = 1e-3
    vs_, w, k, trace, pl, s = _tr_case(steps, dt, config)
    th, info = vs.solve_transient(k, trace, pl, s, vs_params(w), window=5)
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    ref, _ = _oracle_variant(w, trace, pl, s, dt, 5, False)
    emax, rel = errors(th, ref)
    assert emax <= 5e-3 and rel <= 2e-4


@pytest.mark.parametrize("config,steps", [("c1_64", 12), ("c2_256", 10)])
def test_implicit_leakage_with_the_error_estimate_stop(config, steps):
    """The per-step fixed point of implicit leakage stopped by the error
    estimate (64^2 on the general engine, 256^2 on the persistent one): every
    step within the bar of the oracle's implicit superposition iterated to
    1e-10 K, element by element, in no more iterations than the update rule
    takes at the same tolerance."""
    vs = _vs()
    dt = 1e-3
    vs_, w, k, trace, pl, s = _tr_case(steps, dt, config)
    est = vs_params(w, tol_K=1e-4, stop_rule=vs.VS_STOP_ESTIMATE)
    th, info = vs.solve_transient(k, trace, pl, s, est, leakage=vs.VS_LEAK_IMPLICIT)
    assert info["status"] == vs.VS_OK
    upd, info_u = vs.solve_transient(k, trace, pl, s, vs_params(w, tol_K=1e-4),
                                     leakage=vs.VS_LEAK_IMPLICIT)
    assert info_u["status"] == vs.VS_OK
    assert steps <= info["iterations"] <= info_u["iterations"]
    ref, _ = _oracle_variant(w, trace, pl, s, dt, 0, True)
    emax, rel = errors(th, ref)
    print("%s implicit: %d iterations with the estimate, %d with the update rule, "
          "max |dT| %.2e K" % (config, info["iterations"], info_u["iterations"], emax))
    assert emax <= 5e-3 and rel <= 2e-4
    assert float((th - upd).abs().max()) <= 1e-3
