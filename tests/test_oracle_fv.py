"""P9: the oracle's layered Green's function against a brute-force
finite-volume solve of the steady heat equation (Eq. 1) on tiny grids.

`oracle/fv.py` discretises the layered box directly (adiabatic top and side
walls, perfect contact, convective bottom, a uniform square source per cell)
and shares no code with `oracle/physics.py`. Its O(h^2) error is removed by
Richardson extrapolation over two refinements. The analytic model uses a
uniform DISC of cell area as the source; for a like-for-like comparison the
model's response to the square is built from m x m sub-cell discs of the
same model at the finer grid n m (their union tends to the square as m
grows, error ~1/m^2). Tolerances (measured values in brackets):

* against the square built from 9 x 9 sub-discs: 2e-3 of the source cell's
  value (1.1e-3; the sub-disc approximation dominates, the finite-volume
  extrapolation agrees with the next refinement to 3e-5 .. 4e-4);
* against the model's own disc source: 1.5e-2 relative at the source cell
  and its four nearest neighbours (square against disc: -0.6 % at the
  centre, -0.7 % / +0.4 % at the edge / corner neighbours), and for the
  layered stack 5e-3 relative two or more cells away (0.36 %; the shape
  matters less with distance). A single thin layer on a nearly isothermal
  base decays within a few thicknesses, so there the shape matters more
  (2.0 % at the nearest neighbours; checked at 3e-2) and still matters two
  cells away, where only the square comparison is checked.

The TIM (20 um) is one slab at every refinement: its lateral conduction is
negligible and a single slab is exact for its through-thickness drop.
"""
import numpy as np
import pytest

from oracle import fv
from oracle import physics as ph
from oracle import solve as so

C1_STACK = ((0.5e-3, 0.02e-3, 3.5e-3), (130.0, 4.0, 400.0), 2.0e4)


def model_disc(n, L, t, kap, h, sources):
    """Columns of the model's mirror-image operator for unit power in each
    source cell (oracle: kernel_periodic + mirror_operator)."""
    Lm = so.mirror_operator(ph.kernel_periodic(n, L, t, kap, h))
    return np.array([Lm[:, sy * n + sx].reshape(n, n) for sy, sx in sources])


def model_square(n, L, t, kap, h, m, sources):
    """The model's response at the n x n cell centres to a unit square source
    filling one cell, as the mean of m x m sub-cell disc sources of the same
    model on the grid n m (m odd, so the cell centres are sub-cell centres)."""
    nf = n * m
    kper = ph.kernel_periodic(nf, L, t, kap, h)
    n2 = 2 * nf
    c = (m - 1) // 2
    iy = np.arange(n) * m + c
    out = np.zeros((len(sources), n, n))
    for k, (sy, sx) in enumerate(sources):
        for a in range(m):
            for b in range(m):
                jy, jx = sy * m + a, sx * m + b
                for ey in ((iy - jy) % n2, (iy + jy + 1) % n2):
                    for ex in ((iy - jx) % n2, (iy + jx + 1) % n2):
                        out[k] += kper[np.ix_(ey, ex)]
        out[k] /= m * m
    return out


def _check(n, L, stack, sources, m=9, square_tol=2e-3, disc_near_tol=1.5e-2, disc_far_tol=5e-3,
           cells_per_layer=None):
    t, kap, h = stack
    T, _ = fv.solve_extrapolated(n, L, t, kap, h, (3, 5), sources, cells_per_layer)
    sq = model_square(n, L, t, kap, h, m, sources)
    dc = model_disc(n, L, t, kap, h, sources)
    for k, (sy, sx) in enumerate(sources):
        self_v = sq[k, sy, sx]
        err = np.max(np.abs(T[k] - sq[k])) / self_v
        assert err <= square_tol, (k, err)
        yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        dist = np.abs(yy - sy) + np.abs(xx - sx)
        rel = np.abs(T[k] - dc[k]) / np.abs(dc[k])
        near = dist <= 1
        assert np.max(rel[near]) <= disc_near_tol, (k, np.max(rel[near]))
        far = (dist >= 2) & (np.abs(dc[k]) > 1e-3 * self_v)
        if disc_far_tol and far.any():
            assert np.max(rel[far]) <= disc_far_tol, (k, np.max(rel[far]))
    return T, sq, dc


def test_fv_conserves_heat_and_reproduces_the_series_resistance():
    """The discretisation itself: all heat leaves through the bottom, and a
    uniform flux over the whole die gives the 1-D series resistance exactly
    (no lateral flow; the linear profile in each slab is exact)."""
    t, kap, h = C1_STACK
    n, L = 4, 4e-3
    T, info = fv.solve(n, L, t, kap, h, 3, [(y, x) for y in range(n) for x in range(n)])
    assert np.allclose(info["bottom_heat_W"], 1.0, rtol=1e-10)
    uniform = T.sum(axis=0)                          # 1 W in every cell
    q = 1.0 / (L / n) ** 2
    series = q * (sum(a / b for a, b in zip(t, kap)) + 1.0 / h)
    assert np.allclose(uniform, series, rtol=1e-10)


C1_SLABS = (2.0, 0.2, 2.0)           # slabs per layer and unit of refinement


def test_fv_pins_the_layered_kernel_at_8x8():
    """The C1 stack (Si / TIM / Cu spreader, h = 2e4) on a 10 mm die, 8 x 8
    cells: a corner and an interior source."""
    _check(8, 10e-3, C1_STACK, [(0, 0), (3, 4)], cells_per_layer=C1_SLABS)


def test_fv_pins_the_layered_kernel_at_16x16():
    """The same stack at 16 x 16 cells (0.625 mm, closer to the silicon
    thickness): edge and interior sources."""
    _check(16, 10e-3, C1_STACK, [(0, 5), (7, 8)], cells_per_layer=C1_SLABS)


@pytest.mark.parametrize("stack", [((2e-3,), (130.0,), 1e5), ((1e-3,), (130.0,), 1e7)])
def test_fv_pins_a_single_layer(stack):
    """One layer: a thick slab with a convective bottom, and a thinner one
    on a nearly isothermal base (h = 1e7), where the response is local."""
    _check(8, 10e-3, stack, [(0, 0), (4, 4)], disc_near_tol=3e-2, disc_far_tol=None)
