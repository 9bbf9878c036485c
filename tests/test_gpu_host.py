"""The host-memory batch solve (vs_solve_batch_host): chunked, with the copies
overlapping the solve. Every map must get exactly what the device-resident
batch solve gives it, for any chunking, both FP32 engines and the split
precision path, pinned or pageable host arrays."""
import pytest
import torch

import synth

from _util import ENG_TOL_K, REQ_REL_L2, errors, inputs, oracle_spectrum, oracle_steady, vs_params, vs_stack

pytestmark = pytest.mark.gpu


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def _kernel(w):
    vs = _vs()
    return vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))


def _device_reference(k, pd, pl, s, prm):
    vs = _vs()
    th = torch.empty_like(pd)
    infos = vs.solve_batch([(k, pd[i], pl[i], None if s is None else s[i], th[i])
                            for i in range(pd.shape[0])], prm)
    return th, infos


@pytest.mark.parametrize("name,count,chunk,engine", [
    ("c3_128", 10, 3, 2),        # cluster engine, tail chunk of 1
    ("c3_256", 7, 7, 2),         # one chunk
    ("c3_256", 9, 4, 1),         # streamed engine, tail chunk of 1
    ("c3_512", 5, 2, 0),         # automatic engine (streamed at 512^2)
])
def test_host_batch_equals_device_batch(name, count, chunk, engine):
    vs = _vs()
    w = synth.workload(name)
    k = _kernel(w)
    pd, pl, s = inputs(w, count=count)
    prm = vs_params(w, engine=engine)
    ref, iref = _device_reference(k, pd, pl, s, prm)
    hpd, hpl, hs = pd.cpu().pin_memory(), pl.cpu().pin_memory(), s.cpu().pin_memory()
    th, infos = vs.solve_batch_host(k, hpd, hpl, hs, params=prm, chunk_maps=chunk)
    assert not th.is_cuda
    assert torch.equal(th, ref.cpu())
    assert [i["iterations"] for i in infos] == [i["iterations"] for i in iref]
    assert all(i["status"] == vs.VS_OK for i in infos)
    Kt = oracle_spectrum(w)
    r, _ = oracle_steady(w, Kt, pd[count - 1], pl[count - 1], s[count - 1])
    emax, rel = errors(th[count - 1], r)
    assert emax <= ENG_TOL_K and rel <= REQ_REL_L2


def test_host_batch_pageable_split_precision_and_no_variation():
    vs = _vs()
    w = synth.workload("c3_256")
    k = _kernel(w)
    pd, pl, s = inputs(w, count=6)
    # pageable host arrays, s = 1
    prm = vs_params(w)
    ref, _ = _device_reference(k, pd, pl, None, prm)
    th, infos = vs.solve_batch_host(k, pd.cpu(), pl.cpu(), None, params=prm, chunk_maps=4)
    assert torch.equal(th, ref.cpu())
    # BF16 hi/lo split on tensor cores, default chunking
    prm = vs_params(w, tol_K=1e-2, precision=vs.VS_PREC_BF16_SPLIT)
    ref, _ = _device_reference(k, pd, pl, s, prm)
    th, infos = vs.solve_batch_host(k, pd.cpu().pin_memory(), pl.cpu().pin_memory(),
                                    s.cpu().pin_memory(), params=prm)
    assert torch.equal(th, ref.cpu())
    assert all(i["status"] == vs.VS_OK for i in infos)


def test_host_batch_statuses_and_argument_checks():
    vs = _vs()
    w = synth.workload("c1_64")
    k = _kernel(w)
    pd, pl, s = inputs(w, count=3)
    bad = pd.cpu().clone()
    bad[1, 3, 5] = float("nan")
    th, infos = vs.solve_batch_host(k, bad, pl.cpu(), s.cpu(), params=vs_params(w), chunk_maps=1)
    assert [i["status"] for i in infos] == [vs.VS_OK, vs.VS_ERR_NONFINITE, vs.VS_OK]
    with pytest.raises(TypeError):                       # device tensors are not host arrays
        vs.solve_batch_host(k, pd, pl.cpu(), s.cpu(), params=vs_params(w))
    with pytest.raises(ValueError):
        vs.solve_batch_host(k, pd.cpu()[:, :32], pl.cpu(), s.cpu(), params=vs_params(w))
    with pytest.raises(vs.VarsimError):
        vs.solve_batch_host(k, pd.cpu(), pl.cpu(), s.cpu(), params=vs_params(w, tol_K=0.0))


def test_host_plan_runs_repeatedly_and_checks_its_arguments():
    """vs_host_plan_*: one host plan, two batches in a row, each map equal to
    the device-resident batch solve; the conductivity field must match the
    plan's with_s."""
    vs = _vs()
    w = synth.workload("c3_256")
    k = _kernel(w)
    prm = vs_params(w, engine=2, tol=1e-2, stop_rule=vs.VS_STOP_ESTIMATE)
    hp = vs.HostPlan(k, 9, True, prm, chunk_maps=4)
    for seed in (synth.SEED + 71, synth.SEED + 72):
        pd, pl, s = synth.steady_inputs(w, 9, seed=seed, device="cuda")
        ref, iref = _device_reference(k, pd, pl, s, prm)
        th, infos = hp.run(pd.cpu().pin_memory(), pl.cpu().pin_memory(), s.cpu().pin_memory())
        assert torch.equal(th, ref.cpu())
        assert [i["iterations"] for i in infos] == [i["iterations"] for i in iref]
        assert all(i["status"] == vs.VS_OK for i in infos)
    with pytest.raises(vs.VarsimError) as e:
        hp.run(pd.cpu(), pl.cpu(), None)
    assert e.value.status == vs.VS_ERR_INVALID_ARG
    hp.close()
    hp2 = vs.HostPlan(k, 3, False, prm)
    th, infos = hp2.run(pd[:3].cpu(), pl[:3].cpu())
    ref, _ = _device_reference(k, pd[:3], pl[:3], None, prm)
    assert torch.equal(th, ref.cpu())
    with pytest.raises(vs.VarsimError):
        hp2.run(pd[:3].cpu(), pl[:3].cpu(), s[:3].cpu())
    hp2.close()
