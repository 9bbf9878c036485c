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
