"""The effect ablation of the bench (the layout of the paper's table of errors):
every scenario on the GPU against the same scenario in the FP64 oracle, map
by map, and the table's summaries against the oracle's."""
import os
import sys

import numpy as np
import pytest
import torch

import synth
from oracle import solve as so

from _util import oracle_spectrum, vs_params, vs_stack

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


def test_effect_ablation_matches_oracle():
    import paper_2307_12119_gb300 as vs
    w = synth.workload("c1_64")
    pd, pl, s = synth.steady_inputs(w, 2, device="cuda")
    k = vs.Kernel(vs_stack(w), vs.Grid(w.n, w.die_m))
    mk = lambda prec: vs_params(w, precision=prec)
    maps = {}
    table = bench.effect_ablation(vs, k, w, pd, pl, s, mk, maps=maps)
    assert table["all_effects_not_ok"] == 0
    phy = w.physics
    Kt = oracle_spectrum(w)
    f64 = lambda t: t.double().cpu().numpy()

    def oracle(pl_x, s_x, beta, alpha, b):
        sx = np.ones((w.n, w.n)) if s_x is None else f64(s_x[b])
        th, _, _ = so.picard_split(Kt, f64(pd[b]), f64(pl_x[b]), sx, beta, alpha, tol=1e-10)
        return th

    def same_maps(gpu, ref, name):
        # element by element: every scenario is an FP32 solve to 1e-4 K
        for b in range(2):
            g = f64(gpu[b])
            emax = np.max(np.abs(g - ref[b]))
            rel = np.linalg.norm(g - ref[b]) / np.linalg.norm(ref[b])
            assert emax <= 2e-3 and rel <= 1e-4, (name, b, emax, rel)

    full = [oracle(pl, s, phy.beta_per_K, phy.alpha_per_K, b) for b in range(2)]
    same_maps(maps["all effects"], full, "all effects")
    for (name, s_var, a_on, l_var, b_on), row in zip(bench.ABLATION_SCENARIOS, table["rows"]):
        assert row["effects"] == name and row["not_ok"] == 0
        pl_x, s_x = bench.ablation_inputs(pl, s, s_var, l_var)
        refs = [oracle(pl_x, s_x, phy.beta_per_K if b_on else 0.0,
                       phy.alpha_per_K if a_on else 0.0, b) for b in range(2)]
        same_maps(maps[name], refs, name)
        devs = [np.max(np.abs(refs[b] - full[b])) for b in range(2)]
        assert row["max_dev_K_max"] == pytest.approx(max(devs), abs=5e-3), name
        assert row["max_dev_K_max"] > 0.0
    # the closed form's row: against the oracle's closed form, map by map
    cf_ref = [so.closed_form(Kt, f64(pd[b]), f64(pl[b]), f64(s[b]), phy.beta_per_K,
                             phy.alpha_per_K) for b in range(2)]
    same_maps(maps[table["rows"][-1]["effects"]], cf_ref, "closed form")
    cf = [np.max(np.abs(cf_ref[b] - full[b])) for b in range(2)]
    assert table["rows"][-1]["max_dev_K_max"] == pytest.approx(max(cf), abs=5e-3)
    # with every effect on except one group the deviation is below that of no effects
    assert all(r["max_dev_K_max"] < table["rows"][0]["max_dev_K_max"] for r in table["rows"][4:7])
