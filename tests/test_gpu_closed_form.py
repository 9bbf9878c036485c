"""GPU parity of the one-shot closed form (Eqs. 21, 25, 26) against the FP64
oracle, its exact special case, and its error against the iterated fixed
point."""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import solve as so

from _util import errors, oracle_spectrum, vs_params, vs_stack

pytestmark = pytest.mark.gpu


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


def _oracle(w, pd, pl, s, mode):
    f64 = lambda t: t.double().cpu().numpy()
    return so.closed_form(oracle_spectrum(w), f64(pd), f64(pl), f64(s), w.physics.beta_per_K,
                          w.physics.alpha_per_K, "impulse" if mode else "conv")


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("config,n", [("c1_64", None), ("c2_256", None), ("c1_64", 8),
                                      ("c2_256", 512)])
def test_closed_form_matches_oracle(config, n, mode):
    vs, w, k, pd, pl, s = _case(config, 3, n)
    th, infos = vs.solve_closed_form(k, pd, pl, s, vs_params(w), mode)
    assert all(i["status"] == vs.VS_OK and i["iterations"] == 0 for i in infos)
    for b in range(3):
        ref = _oracle(w, pd[b], pl[b], s[b], mode)
        emax, rel = errors(th[b], ref)
        assert emax <= 2e-3 and rel <= 2e-5, (b, emax, rel)
        assert infos[b]["mu_W"] == pytest.approx(float(pl[b].double().mean()), rel=1e-12)


def test_closed_form_full_batch_sampled_maps():
    # the bench's workload: 4096 maps of 256^2 in one call; maps are independent,
    # so sampled maps are checked one by one against the oracle
    vs = _vs()
    w, pd, pl, s = synth.batch_inputs(256, 4096, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    th, infos = vs.solve_closed_form(k, pd, pl, s, vs_params(w))
    assert all(i["status"] == vs.VS_OK for i in infos)
    for b in (0, 1777, 4095):
        emax, rel = errors(th[b], _oracle(w, pd[b], pl[b], s[b], 0))
        assert emax <= 2e-3 and rel <= 2e-5, (b, emax, rel)


def test_closed_form_without_variation_is_the_fixed_point():
    # uniform leakage and alpha = 0: Eq. 21 is exact, so the one-shot result is
    # the converged solve of the same maps
    vs, w, k, pd, _, _ = _case("c2_256", 2)
    pl = torch.full_like(pd, 2e-4)
    prm = vs_params(w, tol=1e-6, alpha_per_K=0.0)
    th, infos = vs.solve_closed_form(k, pd, pl, None, prm)
    for b in range(2):
        ref, info = vs.solve_steady(k, pd[b], pl[b], None, prm)
        assert info["status"] == vs.VS_OK
        assert float((th[b] - ref).abs().max()) <= 2e-5 * float(ref.abs().max()) + 1e-5


def test_closed_form_error_against_the_fixed_point():
    # the approximation's error, stated as a fraction of the maximum rise
    vs, w, k, pd, pl, s = _case("c2_256", 8)
    prm = vs_params(w, tol=1e-6)
    out = {}
    exact = torch.empty_like(pd)
    vs.solve_batch([(k, pd[b], pl[b], s[b], exact[b]) for b in range(8)], prm)
    rise = exact.amax(dim=(1, 2))
    for mode in (0, 1):
        th, _ = vs.solve_closed_form(k, pd, pl, s, prm, mode)
        err = (th - exact).abs().amax(dim=(1, 2)) / rise
        out[mode] = float(err.max())
    print("closed form, max error / max rise over 8 maps of 256^2: conv %.2f %%, impulse %.2f %%"
          % (100 * out[0], 100 * out[1]))
    # a measurement, not a bound from the paper: the FP64 oracle gives 6-12 % on
    # these maps (2.5-3 % on the 64^2 configuration); only sanity is asserted
    assert 0.0 < out[0] < 0.3 and 0.0 < out[1] < 0.3


def test_closed_form_flags_runaway_and_bad_arguments():
    vs, w, k, pd, pl, s = _case("c1_64", 2)
    hot = pl.clone()
    hot[1] *= 1e4                                     # beta mu max(K) > 1
    th, infos = vs.solve_closed_form(k, pd, hot, s, vs_params(w))
    assert infos[0]["status"] == vs.VS_OK
    assert infos[1]["status"] == vs.VS_ERR_RUNAWAY
    with pytest.raises(vs.VarsimError) as e:
        vs.solve_closed_form(k, pd, pl, s, vs_params(w), mode=5)
    assert e.value.status == vs.VS_ERR_INVALID_ARG
