"""A heat spreader wider than the die (Sec. II-B) on the GPU: the kernel
build, the steady solve and the transient against the FP64 oracle with the
same reading (the spreader changes the constant part of the Green's
function, i.e. the uniform mode; see tests/test_oracle_spreader.py for the
reading's pins against the finite-volume solve of the geometry)."""
import numpy as np
import pytest
import torch

import synth
from oracle import physics as ph
from oracle import solve as so

from _util import ENG_TOL_K, REQ_MAX_K, REQ_REL_L2, errors, oracle_steady, vs_params

pytestmark = pytest.mark.gpu


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def _stack(w, side_m, layer=2):
    vs = _vs()
    st = w.stack
    return vs.Stack(st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K, st.heat_cap_J_m2K,
                    spreader_layer=layer, spreader_side_m=side_m)


@pytest.mark.parametrize("name,side_mm", [("c1_64", 15.0), ("c1_64", 30.0), ("c2_256", 30.0)])
def test_spectrum_with_wide_spreader_matches_oracle(name, side_mm):
    vs = _vs()
    w = synth.workload(name)
    st = w.stack
    k = vs.Kernel(_stack(w, side_mm * 1e-3), vs.Grid(w.n, w.die_m))
    got = k.spectrum()
    ref = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                      spreader=(2, side_mm * 1e-3))
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    # only the uniform mode moves, and the wider spreader lowers it
    plain = vs.Kernel(_stack(w, 0.0, layer=0), vs.Grid(w.n, w.die_m)).spectrum()
    assert got[0, 0] < plain[0, 0]
    d = got - plain
    d[0, 0] = 0.0
    assert np.max(np.abs(d)) == 0.0


def test_die_sized_spreader_gives_the_plain_kernel():
    vs = _vs()
    w = synth.workload("c1_64")
    a = vs.Kernel(_stack(w, w.die_m), vs.Grid(w.n, w.die_m)).spectrum()
    b = vs.Kernel(_stack(w, 0.0, layer=0), vs.Grid(w.n, w.die_m)).spectrum()
    assert np.array_equal(a, b)


def test_steady_solve_with_wide_spreader():
    vs = _vs()
    w = synth.workload("c1_64")
    st = w.stack
    side = 20e-3
    k = vs.Kernel(_stack(w, side), vs.Grid(w.n, w.die_m))
    pd, pl, s = synth.steady_inputs(w, 2, device="cuda")
    th = torch.empty_like(pd)
    infos = vs.solve_batch([(k, pd[i], pl[i], s[i], th[i]) for i in range(2)], vs_params(w))
    assert all(i["status"] == vs.VS_OK for i in infos)
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                     spreader=(2, side))
    Kp = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    for i in range(2):
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(th[i], ref)
        assert emax <= ENG_TOL_K and rel <= REQ_REL_L2, (i, emax, rel)
        plain, _ = oracle_steady(w, Kp, pd[i], pl[i], s[i])
        assert float(th[i].double().mean()) < float(plain.mean())


def test_transient_with_wide_spreader():
    """The uniform mode's pole moves with the spreader: tau = C g^0_wide."""
    vs = _vs()
    w = synth.workload("c1_64")
    st = w.stack
    side, dt, steps = 20e-3, 1e-3, 30
    k = vs.Kernel(_stack(w, side), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    trace = synth.markov_trace(w, steps, device="cuda")
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK
    spectra = [so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                                st.heat_cap_J_m2K, j * dt, spreader=(2, side))
               for j in range(1, steps + 1)]
    f64 = lambda t: t.double().cpu().numpy()
    ref = so.duhamel_modes(spectra, f64(trace), f64(pl[0]), f64(s[0]), w.physics.beta_per_K,
                           w.physics.alpha_per_K)
    emax, rel = errors(th, ref)
    assert emax <= REQ_MAX_K
    assert emax <= 5e-3 and rel <= 2e-4


def test_wide_spreader_arguments_are_validated():
    vs = _vs()
    w = synth.workload("c1_64")
    with pytest.raises(vs.VarsimError) as e:
        vs.Kernel(_stack(w, 5e-3), vs.Grid(w.n, w.die_m))           # narrower than the die
    assert e.value.status == vs.VS_ERR_INVALID_ARG
    with pytest.raises(vs.VarsimError) as e:
        vs.Kernel(_stack(w, 20e-3, layer=3), vs.Grid(w.n, w.die_m))  # no such layer
    assert e.value.status == vs.VS_ERR_INVALID_ARG
