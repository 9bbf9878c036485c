"""Split-precision (BF16 hi/lo, FP32 accumulate) tcgen05 tensor-core path:
the cosine-transform building block against a plain PyTorch FP64 reference of
the same contraction, and the batched solve against the FP64 oracle and the
FP32 path."""
import math

import numpy as np
import pytest
import torch

import synth

from _util import REQ_MAX_K, errors, inputs, oracle_spectrum, oracle_steady, vs_params, vs_stack

pytestmark = pytest.mark.gpu

# BF16 hi/lo keeps ~16 significant bits of every operand and drops the lo*lo
# product: one transform is accurate to ~2^-16 ~ 1.5e-5 of its inputs' scale.
TC_REL = 6e-5
# The split path is run to a 1e-2 K update tolerance (its transforms carry
# ~1e-3 K of rounding at 30-130 K rises); it must stay within the 0.05 K bar.
TC_TOL_K = 1e-2


def _dct(n, inverse):
    j = torch.arange(n, dtype=torch.float64)
    k = torch.arange(n, dtype=torch.float64)
    if not inverse:
        return torch.cos(math.pi * j[:, None] * (2 * k[None, :] + 1) / (2 * n))
    w = torch.full((n,), 2.0, dtype=torch.float64)
    w[0] = 1.0
    return w[None, :] * torch.cos(math.pi * k[None, :] * (2 * j[:, None] + 1) / (2 * n)) / n


@pytest.mark.parametrize("n,rows", [(256, 256), (128, 384), (256, 1024), (512, 256), (1024, 128)])
@pytest.mark.parametrize("inverse", [False, True])
def test_tc_transform_matches_fp64_matmul(n, rows, inverse):
    import paper_2307_12119_gb300 as vs
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.rand(rows, n, device="cuda", generator=g) - 0.25
    y = vs.tc_transform(x, inverse=inverse)
    torch.cuda.synchronize()
    ref = x.double().cpu() @ _dct(n, inverse).T
    err = (y.double().cpu() - ref).abs().max().item()
    scale = (x.double().abs().cpu() @ _dct(n, inverse).abs().T).max().item()
    assert err <= TC_REL * scale, (err, scale)


def test_tc_round_trip():
    import paper_2307_12119_gb300 as vs
    x = torch.rand(256, 256, device="cuda") + 1.0
    back = vs.tc_transform(vs.tc_transform(x), inverse=True)
    assert float((back - x).abs().max()) <= 2e-4


@pytest.mark.parametrize("name,count", [("c2_256", 3), ("c3_128", 3), ("c3_512", 2),
                                        ("c4_1024", 1)])
def test_tc_solve_matches_oracle(name, count):
    # the 1024^2 case is the split-precision steady solve of the 1024^2
    # workload (its transient runs on the FP32 engine, tests/test_gpu_configs.py)
    import paper_2307_12119_gb300 as vs
    w = synth.workload(name)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    pd, pl, s = inputs(w, count=count)
    th = torch.empty_like(pd)
    prm = vs_params(w, tol_K=TC_TOL_K, precision=vs.VS_PREC_BF16_SPLIT)
    infos = vs.solve_batch([(k, pd[i], pl[i], s[i], th[i]) for i in range(count)], prm)
    assert all(i["status"] == vs.VS_OK for i in infos), infos
    Kt = oracle_spectrum(w)
    for i in range(count):
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(th[i], ref)
        assert emax <= REQ_MAX_K, (i, emax)
        assert rel <= 2e-4, (i, rel)


def test_tc_batch_agrees_with_fp32_path():
    import paper_2307_12119_gb300 as vs
    w = synth.workload("c3_256")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    pd, pl, s = inputs(w, count=40)
    a = torch.empty_like(pd)
    b = torch.empty_like(pd)
    items = lambda out: [(k, pd[i], pl[i], s[i], out[i]) for i in range(pd.shape[0])]
    vs.solve_batch(items(a), vs_params(w, tol_K=1e-5))
    infos = vs.solve_batch(items(b), vs_params(w, tol_K=TC_TOL_K, precision=vs.VS_PREC_BF16_SPLIT))
    assert all(i["status"] == vs.VS_OK for i in infos)
    assert float((a - b).abs().max()) <= 0.02


def test_tc_rejects_unsupported_sizes():
    import paper_2307_12119_gb300 as vs
    w = synth.workload("c1_64")                   # below the 128-row tile
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    pd, pl, s = inputs(w)
    th = torch.empty_like(pd[0])
    with pytest.raises(vs.VarsimError) as e:
        vs.solve_batch([(k, pd[0], pl[0], s[0], th)],
                       vs_params(w, precision=vs.VS_PREC_BF16_SPLIT))
    assert e.value.status == vs.VS_ERR_INVALID_ARG
    with pytest.raises(vs.VarsimError):
        vs.tc_transform(torch.zeros(128, 64, device="cuda"))
