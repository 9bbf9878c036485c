"""The remaining workload configurations at full size, checked against the
FP64 oracle on sampled outputs and on properties that hold at any size:

* batched Monte Carlo: 4096 variation samples (sigma U[5,10] %, correlation
  length U[0.5,3] mm) over power maps of mixed grid sizes 128^2 / 256^2 / 512^2
  in one plan, captured in a CUDA graph;
* transient at 1024^2: 200 steps of 1 ms with a Markov power trace.
"""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import solve as so

from _util import (ENG_TOL_K, REQ_MAX_K, REQ_REL_L2, errors, oracle_spectrum, oracle_steady,
                   step_spectra, vs_params, vs_stack)

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


def test_mixed_size_monte_carlo_batch_4096():
    vs = _vs()
    sizes = (128, 256, 512)
    total = 4096
    ws = {n: synth.workload("c3_%d" % n) for n in sizes}
    ks = {n: vs.Kernel(vs_stack(ws[n]), vs.Grid(n, ws[n].die_m)) for n in sizes}
    counts = {n: len(range(i0, total, 3)) for i0, n in enumerate(sizes)}
    # about 64 power maps in all: 22 floorplans per grid size, every sample its
    # own variation field
    data = {n: synth.steady_inputs(ws[n], counts[n], n_floorplans=22, device="cuda")
            for n in sizes}
    th = {n: torch.empty_like(data[n][0]) for n in sizes}
    items = []
    for i in range(total):
        n, j = sizes[i % 3], i // 3
        pd, pl, s = data[n]
        items.append((ks[n], pd[j], pl[j], s[j], th[n][j]))
    prm = vs_params(ws[256])
    plan = vs.Plan(items, prm)
    assert plan.launches == 1                  # a 512^2 map keeps the plan on the streamed engine
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            plan.run(stream)
    torch.cuda.current_stream().wait_stream(stream)
    g.replay()
    torch.cuda.synchronize()
    infos = plan.info()
    assert all(i["status"] == vs.VS_OK for i in infos)
    iters = np.array([i["iterations"] for i in infos])
    assert iters.min() >= 2 and iters.max() <= 25
    for n in sizes:
        assert bool(torch.isfinite(th[n]).all()) and float(th[n].min()) > 0
    # sampled maps of every size against the oracle
    for n in sizes:
        Kt = oracle_spectrum(ws[n])
        pd, pl, s = data[n]
        for j in (0, counts[n] - 1):
            ref, _ = oracle_steady(ws[n], Kt, pd[j], pl[j], s[j])
            emax, rel = errors(th[n][j], ref)
            assert emax <= ENG_TOL_K and rel <= REQ_REL_L2, (n, j, emax, rel)
    # the same maps of n <= 256 on the cluster engine: one launch per size
    th2 = {n: torch.empty_like(data[n][0]) for n in (128, 256)}
    items2 = []
    for i in range(total):
        n, j = sizes[i % 3], i // 3
        if n > 256:
            continue
        pd, pl, s = data[n]
        items2.append((ks[n], pd[j], pl[j], s[j], th2[n][j]))
    plan2 = vs.Plan(items2, vs_params(ws[256], engine=vs.VS_ENGINE_CLUSTER))
    assert plan2.launches == 2
    plan2.run()
    assert all(i["status"] == vs.VS_OK for i in plan2.info())
    for n in (128, 256):
        assert float((th2[n] - th[n]).abs().max()) <= 2e-4


def test_transient_1024_two_hundred_steps():
    vs = _vs()
    w = synth.workload("c4_1024")
    dt, steps = 1e-3, 200
    fix = json.load(open(os.path.join(HERE, "golden", "transient_mode00_c4_1024.json")))
    assert fix["dt_s"] == dt and len(fix["S00"]) == steps
    trace = synth.markov_trace(w, steps, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))

    # Linear case (no leakage, alpha = 0, s = 1): the map mean is the uniform
    # mode, so at every step it is the superposition (Eq. 36) of the uniform
    # mode's step responses over the mean power differences.
    zero = torch.zeros(w.n, w.n, device="cuda")
    th, info = vs.solve_transient(k, trace, zero, None,
                                  vs_params(w, beta_per_K=0.0, alpha_per_K=0.0))
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    pbar = trace.double().mean(dim=(1, 2)).cpu().numpy()
    dp = np.diff(np.concatenate([[0.0], pbar]))          # dp[m] = Pbar_{m+1} - Pbar_m
    S = np.array(fix["S00"])
    ref = np.array([np.dot(S[:m + 1], dp[m::-1]) for m in range(steps)])
    got = th.double().mean(dim=(1, 2)).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    del th

    # With leakage and temperature-dependent conductivity: statuses over all
    # 200 steps, and the first 8 steps element by element against the
    # oracle's superposition (Eq. 36 with the exact step spectra).
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    assert bool(torch.isfinite(th).all()) and float(th[-1].min()) > 0
    first = 8
    spectra = step_spectra(w, dt, first)
    f64 = lambda t: t.double().cpu().numpy()
    ref = so.duhamel_modes(spectra, f64(trace[:first]), f64(pl[0]), f64(s[0]),
                           w.physics.beta_per_K, w.physics.alpha_per_K)
    got = f64(th[:first])
    for j in range(first):
        d = got[j] - ref[j]
        emax = float(np.max(np.abs(d)))
        rel = float(np.linalg.norm(d) / np.linalg.norm(ref[j]))
        print("1024^2 step %d: max|dT| %.2e K, rel-L2 %.2e" % (j + 1, emax, rel))
        assert emax <= REQ_MAX_K, (j, emax)
        assert emax <= 5e-3 and rel <= 2e-4, (j, emax, rel)


def test_transient_256_every_step_of_two_hundred():
    """The transient at 256^2 (20 x 20 mm die, Markov power trace, leakage and
    conductivity on), 200 steps of 1 ms, every step element by element
    against the oracle's untruncated superposition (Eq. 36, lagged leakage)."""
    vs = _vs()
    w = synth.workload("c2_256")
    dt, steps = 1e-3, 200
    trace = synth.markov_trace(w, steps, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m), vs.KernelOpts(dt_s=dt))
    _, pl, s = synth.steady_inputs(w, 1, device="cuda")
    th, info = vs.solve_transient(k, trace, pl[0], s[0], vs_params(w))
    assert info["status"] == vs.VS_OK and info["iterations"] == steps
    spectra = step_spectra(w, dt, steps)
    f64 = lambda t: t.double().cpu().numpy()
    ref = so.duhamel_modes(spectra, f64(trace), f64(pl[0]), f64(s[0]), w.physics.beta_per_K,
                           w.physics.alpha_per_K)
    got = f64(th)
    d = got - ref
    emax_step = np.max(np.abs(d), axis=(1, 2))
    rel_step = np.linalg.norm(d.reshape(steps, -1), axis=1) / np.linalg.norm(ref.reshape(steps, -1),
                                                                             axis=1)
    print("256^2 transient: worst max|dT| %.2e K (step %d), worst rel-L2 %.2e (step %d), "
          "max rise %.1f K" % (emax_step.max(), emax_step.argmax() + 1, rel_step.max(),
                               rel_step.argmax() + 1, float(np.max(ref))))
    assert emax_step.max() <= REQ_MAX_K
    assert emax_step.max() <= 5e-3 and rel_step.max() <= 2e-4
