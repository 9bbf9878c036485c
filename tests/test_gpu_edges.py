"""Edge cases: the largest grid the ABI takes (2048 x 2048), empty batches and
power maps that are zero everywhere."""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle import physics as ph

from _util import inputs, vs_params, vs_stack

pytestmark = pytest.mark.gpu


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def test_largest_grid_2048():
    vs = _vs()
    w = dataclasses.replace(synth.workload("c2_256"), name="c2_2048", n=2048)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    st = w.stack
    # the uniform mode of the imaged kernel depends on the cell, not on n: the
    # oracle evaluates it on a 16 x 16 die with the same cell
    cell = w.die_m / w.n
    K00 = ph.spectrum(16, 16 * cell, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)[0, 0]
    Kt = k.spectrum()
    assert Kt.shape == (2048, 2048)
    assert Kt[0, 0] == pytest.approx(K00, rel=1e-9)
    # linear solve of a checkerboard: energy balance and the die's symmetries
    n = w.n
    yy, xx = torch.meshgrid(torch.arange(n), torch.arange(n), indexing="ij")
    q = (((xx + yy) % 2).float() * 1e-4).cuda().contiguous()
    zero = torch.zeros_like(q)
    th, info = vs.solve_steady(k, q, zero, None, vs_params(w, beta_per_K=0.0, alpha_per_K=0.0))
    assert info["status"] == vs.VS_OK
    assert float(th.double().mean()) == pytest.approx(K00 * float(q.double().mean()), rel=2e-6)
    t = th.cpu().numpy()
    assert np.max(np.abs(t - t.T)) <= 2e-5 * t.max()
    # the full nonlinear solve converges at this size
    pd, pl, s = synth.steady_inputs(w, 1, device="cuda")
    th, info = vs.solve_steady(k, pd[0], pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK and 2 <= info["iterations"] <= 20
    assert bool(torch.isfinite(th).all()) and float(th.min()) > 0
    assert info["mu_W"] == pytest.approx(float(pl[0].double().mean()), rel=1e-12)


def test_empty_batches_are_rejected():
    vs = _vs()
    w = synth.workload("c1_64")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    with pytest.raises(vs.VarsimError) as e:
        vs.solve_batch([], vs_params(w))
    assert e.value.status == vs.VS_ERR_INVALID_ARG
    with pytest.raises(vs.VarsimError):
        vs.Plan([], vs_params(w))
    empty = torch.empty(0, w.n, w.n)
    with pytest.raises(vs.VarsimError):
        vs.solve_batch_host(k, empty, empty, None, params=vs_params(w))


@pytest.mark.parametrize("engine,precision", [(1, 0), (2, 0), (0, 1)])
def test_zero_power_gives_zero_rise(engine, precision):
    vs = _vs()
    w = synth.workload("c3_256")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    _, _, s = inputs(w, count=2)
    zero = torch.zeros(2, w.n, w.n, device="cuda")
    th = torch.full_like(zero, 7.0)
    infos = vs.solve_batch([(k, zero[i], zero[i], s[i], th[i]) for i in range(2)],
                           vs_params(w, engine=engine, precision=precision))
    assert all(i["status"] == vs.VS_OK for i in infos)
    assert all(i["mu_W"] == 0.0 for i in infos)
    assert float(th.abs().max()) == 0.0
