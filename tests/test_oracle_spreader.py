"""A heat spreader wider than the die (Sec. II-B): the oracle's reading
against the brute-force finite-volume solve of the same geometry.

Sec. II-B splits the Green's function into a fast-decaying part and a
constant carried by the spreader. The oracle reads a wider spreader as a
change of that constant only (physics.ghat0_wide): the uniform mode of the
imaged kernel takes the spreader's footprint-mean impedance, every other
mode keeps the die-sized stack spectrum. `oracle/fv.py` solves the actual
geometry (die layers with the die's side walls on a centred, wider spreader
with its own walls and the convective bottom).

Pins (tolerances, measured values in brackets):
* side = die: the die-sized spectrum exactly;
* the footprint-mean impedance of the spreader alone (a uniform flux on the
  centred footprint, the mean rise over the footprint) against the
  finite-volume area mean: 1e-3 (0.6e-4 .. 3e-4);
* the whole stack under uniform power: the die's mean rise against
  g^0_wide q: 5e-3 (the die layers see the spreader's non-uniform top
  temperature, which the footprint mean averages; measured 1e-3 .. 2e-3);
* a wider spreader lowers g^0_wide monotonically.
The accuracy of the reading itself (a constant cannot cool the die's edges)
is measured, not pinned, in `test_wide_spreader_reading_against_the_exact_geometry`.
"""
import numpy as np
import pytest

from oracle import fv
from oracle import physics as ph

C1 = ((0.5e-3, 0.02e-3, 3.5e-3), (130.0, 4.0, 400.0), 2.0e4)
SLABS = (2.0, 0.2, 2.0)


def _fv_die_mean(n, L, t, kap, h, overhang, sources, slabs=None):
    """Richardson-extrapolated finite-volume area mean of the source-plane
    rise over the die for unit power in each source (summed)."""
    m = {}
    for r in (3, 5):
        _, info = fv.solve(n, L, t, kap, h, r, sources, slabs, overhang)
        m[r] = sum(info["die_mean"])
    return (25 * m[5] - 9 * m[3]) / 16


def test_die_sized_spreader_is_the_plain_stack():
    t, kap, h = C1
    g0 = float(ph.ghat(np.array([0.0]), t, kap, h)[0])
    assert ph.ghat0_wide(t, kap, h, 2, 10e-3, 10e-3) == pytest.approx(g0, rel=1e-14)
    K = ph.spectrum(8, 10e-3, t, kap, h)
    Kw = ph.spectrum(8, 10e-3, t, kap, h, spreader=(2, 10e-3))
    assert np.max(np.abs(K - Kw)) <= 1e-14 * np.max(K)


@pytest.mark.parametrize("stack", [((3.5e-3,), (400.0,), 2e4), ((1e-3, 2e-3), (150.0, 400.0), 5e3)])
@pytest.mark.parametrize("overhang", [2, 4])
def test_spreader_mean_impedance_against_fv(stack, overhang):
    t, kap, h = stack
    n, L = 8, 10e-3
    side = L + 2 * overhang * L / n
    allsrc = [(y, x) for y in range(n) for x in range(n)]
    mean = _fv_die_mean(n, L, t, kap, h, (overhang,) * len(t), allsrc)
    q = 1.0 / (L / n) ** 2                         # 1 W per cell
    Z = ph.spreader_mean_impedance(t, kap, h, 0, L, side)
    assert mean == pytest.approx(Z * q, rel=1e-3)


@pytest.mark.parametrize("overhang", [2, 4])
def test_uniform_power_mean_rise_on_a_wide_spreader(overhang):
    t, kap, h = C1
    n, L = 8, 10e-3
    side = L + 2 * overhang * L / n
    allsrc = [(y, x) for y in range(n) for x in range(n)]
    mean = _fv_die_mean(n, L, t, kap, h, (0, 0, overhang), allsrc, SLABS)
    q = 1.0 / (L / n) ** 2
    assert mean == pytest.approx(ph.ghat0_wide(t, kap, h, 2, L, side) * q, rel=5e-3)


def test_wider_spreader_lowers_the_uniform_mode():
    t, kap, h = C1
    g = [ph.ghat0_wide(t, kap, h, 2, 10e-3, side) for side in (10e-3, 12e-3, 15e-3, 20e-3, 30e-3)]
    assert all(b < a for a, b in zip(g, g[1:]))


def test_wide_spreader_reading_against_the_exact_geometry():
    """What the constant of Sec. II-B captures: single-cell sources on a
    10 mm die over a spreader 2.5 mm wider on every side, against the
    finite-volume solve of that geometry. Interior source: within 1.5 % of
    the source cell's rise (0.84 % measured; the die-sized kernel is 8 %
    off); corner source: within 10 % (7.9 %; die-sized 13 %): near the
    die's edge the wider spreader draws heat sideways, which no constant can
    follow."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_fv import model_square
    t, kap, h = C1
    n, L, ov = 8, 10e-3, 2
    side = L + 2 * ov * L / n
    src = [(3, 4), (0, 0)]
    T, _ = fv.solve_extrapolated(n, L, t, kap, h, (3, 5), src, SLABS, (0, 0, ov))
    sq = model_square(n, L, t, kap, h, 9, src)
    g0 = float(ph.ghat(np.array([0.0]), t, kap, h)[0])
    c = (ph.ghat0_wide(t, kap, h, 2, L, side) - g0) / L ** 2
    errs_wide, errs_die = [], []
    for k, (sy, sx) in enumerate(src):
        errs_wide.append(np.max(np.abs(T[k] - (sq[k] + c))) / (sq[k, sy, sx] + c))
        errs_die.append(np.max(np.abs(T[k] - sq[k])) / sq[k, sy, sx])
    assert errs_wide[0] <= 1.5e-2 and errs_die[0] > 5 * errs_wide[0]
    assert errs_wide[1] <= 1e-1 and errs_wide[1] < errs_die[1]


def test_spreader_series_converges():
    """The cosine series of the footprint-mean impedance, with its 1/M^2
    tail removed by one Richardson step, is converged at M = 2048 modes per
    axis (against M = 4096) to 1e-9."""
    t, kap, h = C1
    for side in (12.5e-3, 20e-3):
        a = ph.spreader_mean_impedance(t, kap, h, 2, 10e-3, side, terms=2048)
        b = ph.spreader_mean_impedance(t, kap, h, 2, 10e-3, side, terms=4096)
        assert a == pytest.approx(b, rel=1e-9)
