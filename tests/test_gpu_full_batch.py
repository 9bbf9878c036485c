"""The benchmark's launch configuration at full size: 4096 maps of 256 x 256
in one plan (cluster and streamed engines), checked on sampled maps against
the FP64 oracle and on properties that hold for every map."""
import numpy as np
import pytest
import torch

import synth

from _util import ENG_TOL_K, REQ_REL_L2, errors, oracle_spectrum, oracle_steady, vs_params, vs_stack

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("engine", [2, 1])          # cluster, streamed
def test_full_batch_4096_at_256(engine):
    import paper_2307_12119_gb300 as vs
    w, pd, pl, s = synth.batch_inputs(256, 4096)
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    th = torch.empty_like(pd)
    plan = vs.Plan([(k, pd[i], pl[i], s[i], th[i]) for i in range(pd.shape[0])],
                   vs_params(w, engine=engine))
    plan.run()
    infos = plan.info()
    assert all(i["status"] == vs.VS_OK for i in infos)
    assert all(i["residual_K"] <= 1e-4 for i in infos)
    iters = np.array([i["iterations"] for i in infos])
    assert iters.min() >= 2 and iters.max() <= 20
    # every map: finite, positive rise
    assert torch.isfinite(th).all() and float(th.min()) > 0
    Kt = oracle_spectrum(w)
    for i in (0, 1, 2047, 4095):
        ref, _ = oracle_steady(w, Kt, pd[i], pl[i], s[i])
        emax, rel = errors(th[i], ref)
        assert emax <= ENG_TOL_K and rel <= REQ_REL_L2, (i, emax, rel)
