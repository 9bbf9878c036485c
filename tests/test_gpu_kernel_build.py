"""GPU parity of the Green's-function build (Hankel quadrature, fold, cosine
transform, spectral part) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import physics as ph

from _util import vs_stack

pytestmark = pytest.mark.gpu

STACKS = {
    "c1": ((0.5e-3, 0.02e-3, 3.5e-3), (130.0, 4.0, 400.0), 2.0e4),
    "thin_die": ((0.15e-3, 0.02e-3, 3.5e-3), (130.0, 4.0, 400.0), 2.0e4),   # paper's die
    "one_layer": ((0.4e-3,), (150.0,), 1.0e5),
}


def _vs():
    import paper_2307_12119_gb300 as vs
    return vs


@pytest.mark.parametrize("n,die_mm,stack", [(8, 10, "c1"), (64, 10, "c1"), (64, 10, "thin_die"),
                                             (256, 20, "c1"), (32, 4, "one_layer"),
                                             (512, 20, "c1")])
def test_spectrum_matches_oracle(n, die_mm, stack):
    vs = _vs()
    t, kap, h = STACKS[stack]
    k = vs.Kernel(vs.Stack(t, kap, h), vs.Grid(n, die_mm * 1e-3))
    got = k.spectrum()
    ref = ph.spectrum(n, die_mm * 1e-3, t, kap, h)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert np.allclose(got, got.T, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n,die_mm", [(64, 10), (256, 20), (1024, 20)])
def test_radial_table_matches_eigen_series(n, die_mm):
    vs = _vs()
    t, kap, h = STACKS["c1"]
    k = vs.Kernel(vs.Stack(t, kap, h), vs.Grid(n, die_mm * 1e-3))
    tab = k.radial()
    m = np.nonzero(tab)[0]
    m = np.unique(np.concatenate([[0], m]))
    # sample at most 4000 radii (all of them on the small grids)
    if m.size > 4000:
        m = np.unique(np.concatenate([m[:2000], m[:: max(1, m.size // 2000)]]))
    cell = die_mm * 1e-3 / n
    a = ph.disc_radius(cell)
    ref = ph.g_top_radial(cell * np.sqrt(m.astype(float)), t[0], kap[0], a)
    err = np.max(np.abs(tab[m] - ref)) / ref[0]
    assert err <= 1e-11


def test_hankel_entry_point_arbitrary_radii():
    vs = _vs()
    t, kap, h = STACKS["c1"]
    grid = vs.Grid(256, 20e-3)
    cell = 20e-3 / 256
    a = ph.disc_radius(cell)
    r = np.array([0.0, 1.05 * a, 1.5 * a, 3.3 * a, 17.2 * a, 123.4 * a, 20 * t[0]])
    got = vs.hankel_radial(vs.Stack(t, kap, h), grid, torch.tensor(r, device="cuda")).cpu().numpy()
    ref = ph.g_top_radial(r, t[0], kap[0], a)
    assert np.max(np.abs(got - ref)) <= 1e-11 * ref[0]


def test_fewer_quadrature_nodes_degrade_gracefully():
    # the 256-node rule holds to ~1e-12 at every lattice radius; 64 nodes do not
    vs = _vs()
    t, kap, h = STACKS["c1"]
    grid = vs.Grid(256, 20e-3)
    cell = 20e-3 / 256
    a = ph.disc_radius(cell)
    r = cell * np.sqrt(np.arange(0, 16000, 97).astype(float))
    r = r[(r == 0) | (r > a)]
    ref = ph.g_top_radial(r, t[0], kap[0], a)
    rt = torch.tensor(r, device="cuda")
    e256 = np.max(np.abs(vs.hankel_radial(vs.Stack(t, kap, h), grid, rt, 256).cpu().numpy() - ref))
    e64 = np.max(np.abs(vs.hankel_radial(vs.Stack(t, kap, h), grid, rt, 64).cpu().numpy() - ref))
    assert e256 <= 1e-11 * ref[0] < e64


def test_invalid_arguments_are_rejected():
    vs = _vs()
    with pytest.raises(vs.VarsimError) as e:
        vs.Kernel(vs.Stack((0.5e-3,), (-1.0,)), vs.Grid(64, 0.01))
    assert e.value.status == vs.VS_ERR_INVALID_ARG
    with pytest.raises(vs.VarsimError):
        vs.Kernel(vs.Stack(), vs.Grid(48, 0.01))
    with pytest.raises(vs.VarsimError):
        vs.Kernel(vs.Stack(), vs.Grid(4096, 0.01))
