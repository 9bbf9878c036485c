"""Brute-force finite-volume solve of the layered heat-conduction problem.

Test infrastructure only (see the package docstring). FP64, plain sparse
linear algebra. This module shares nothing with `physics.py` or `solve.py`:
it discretises the steady Fourier equation (Eq. 1 without the time term,
div(kappa grad T) = 0 inside the layers) directly, with the boundary
conditions of the model the rest of the oracle encodes analytically:

* layers run from the source plane (z = 0) down, each with its own
  thickness and conductivity, in perfect thermal contact (the chip parameter
  table of Sec. V-A: silicon, TIM, spreader);
* the power of a grid cell enters through the top face of that cell as a
  uniform flux; the rest of the top face is adiabatic;
* the side walls of every layer are adiabatic;
* the bottom face of the last layer loses heat to ambient through a
  convective coefficient h (temperatures are rises above ambient).

A layer may be wider than the die by a whole number of grid cells on every
side (a spreader larger than the die, Sec. II-B); the die's layers then sit
centred on it, and the wider layer's top face outside the die is adiabatic.

Discretisation. Every grid cell of the die (side cell = die / n) is split
into r x r finite-volume columns (r odd, so one column sits at the cell's
centre), and layer i into round(c_i r) slabs. Unknowns are the temperatures
of the finite volumes; the conductance between two neighbours is the
series (harmonic) combination of their half-cells, and the bottom half-cell
is in series with 1/h. The temperature of the source plane at a cell centre
is the top volume's temperature plus the drop across its upper half-slab,
q dz / (2 kappa), where q is the flux entering it. The second-order error
in the finite-volume size is removed by Richardson extrapolation over two
refinements r1 < r2: T = (r2^2 T(r2) - r1^2 T(r1)) / (r2^2 - r1^2).

The source of this discretisation is a uniform SQUARE of one cell; the
analytic model uses a uniform DISC of the same area (a = cell / sqrt(pi)).
The two agree far from the source; at the source cell and its nearest
neighbours they differ by a few tenths of a percent.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def _slabs(t, kappa, r, cells_per_layer):
    """Thickness and conductivity of every slab from the top down."""
    dz, kz, layer = [], [], []
    for i, (ti, ki, ci) in enumerate(zip(t, kappa, cells_per_layer)):
        m = max(1, int(round(ci * r)))
        dz += [ti / m] * m
        kz += [ki] * m
        layer += [i] * m
    return np.array(dz), np.array(kz), np.array(layer)


def conductance_matrix(n, die_m, t, kappa, h, r, cells_per_layer, overhang_cells=None):
    """Sparse symmetric conductance matrix (W/K) of the finite volumes.

    Returns (A, index, geom): A[i, j] = -G_ij for neighbours, A[i, i] = sum of
    the conductances of volume i (to ambient included); index[z, y, x] is the
    unknown number of a volume or -1 where the layer is absent; geom holds
    the lateral grid (N, hx, offset of the die in volumes) and the slabs."""
    ov = [0] * len(t) if overhang_cells is None else list(overhang_cells)
    ovmax = max(ov)
    hx = die_m / (n * r)
    N = (n + 2 * ovmax) * r                       # volumes per side of the widest layer
    dz, kz, layer = _slabs(t, kappa, r, cells_per_layer)
    NZ = len(dz)
    active = np.zeros((NZ, N, N), dtype=bool)
    for z in range(NZ):
        lo = (ovmax - ov[layer[z]]) * r
        active[z, lo:N - lo, lo:N - lo] = True
    index = -np.ones((NZ, N, N), dtype=np.int64)
    index[active] = np.arange(int(active.sum()))
    nun = int(active.sum())
    rows, cols, vals = [], [], []
    diag = np.zeros(nun)

    def couple(a, b, g):
        rows.extend([a, b])
        cols.extend([b, a])
        vals.extend([-g, -g])
        np.add.at(diag, a, g)
        np.add.at(diag, b, g)

    # lateral neighbours within a slab: kappa (dz hx) / hx
    Z = np.arange(NZ)[:, None, None] * np.ones((1, N, N), dtype=np.int64)
    for axis in (1, 2):
        a_sl = [slice(None)] * 3
        b_sl = [slice(None)] * 3
        a_sl[axis] = slice(0, N - 1)
        b_sl[axis] = slice(1, N)
        ia, ib = index[tuple(a_sl)], index[tuple(b_sl)]
        both = (ia >= 0) & (ib >= 0)
        zz = Z[tuple(a_sl)][both]
        couple(ia[both], ib[both], kz[zz] * dz[zz])
    # vertical neighbours: hx^2 / (dz_a / 2 kappa_a + dz_b / 2 kappa_b)
    ia, ib = index[:-1], index[1:]
    both = (ia >= 0) & (ib >= 0)
    za = Z[:-1][both]
    zb = za + 1
    couple(ia[both], ib[both], hx * hx / (dz[za] / (2 * kz[za]) + dz[zb] / (2 * kz[zb])))
    # bottom face to ambient
    bot = index[-1][index[-1] >= 0]
    g_bot = hx * hx / (dz[-1] / (2 * kz[-1]) + 1.0 / h)
    diag[bot] += g_bot
    rows.append(np.arange(nun))
    cols.append(np.arange(nun))
    vals.append(diag)
    A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nun, nun))
    geom = {"N": N, "hx": hx, "die_offset": ovmax * r, "dz": dz, "kz": kz, "g_bottom": g_bot}
    return A, index, geom


def solve(n, die_m, t, kappa, h, r, sources, cells_per_layer=None, overhang_cells=None):
    """Source-plane temperature rise at the n x n cell centres for unit power
    in each cell of `sources` (list of (y, x)), at refinement r (odd).

    Returns (theta[len(sources), n, n] in K/W, info) where info holds the
    number of unknowns and, per source, the heat leaving through the bottom
    (W; 1 by conservation) and the mean source-plane rise over the whole die
    area (every finite volume, not only the cell centres)."""
    if r % 2 != 1:
        raise ValueError("r must be odd (a finite volume at every cell centre)")
    cpl = [2.0] * len(t) if cells_per_layer is None else cells_per_layer
    A, index, g = conductance_matrix(n, die_m, t, kappa, h, r, cpl, overhang_cells)
    lu = spl.splu(A, permc_spec="MMD_AT_PLUS_A")
    N, off, hx = g["N"], g["die_offset"], g["hx"]
    top = index[0]
    c = (r - 1) // 2
    out = np.zeros((len(sources), n, n))
    bottom_heat, die_mean = [], []
    for k, (sy, sx) in enumerate(sources):
        q = np.zeros((N, N))                      # flux (W/m^2) into the top volumes
        y0, x0 = off + sy * r, off + sx * r
        q[y0:y0 + r, x0:x0 + r] = 1.0 / (r * hx) ** 2
        b = np.zeros(A.shape[0])
        b[top[top >= 0]] = (q * hx * hx)[top >= 0]
        T = lu.solve(b)
        Ttop = np.where(top >= 0, T[np.maximum(top, 0)], 0.0)
        surf = Ttop + q * g["dz"][0] / (2 * g["kz"][0])
        die = surf[off:off + n * r, off:off + n * r]
        out[k] = die[c::r, c::r]
        die_mean.append(float(die.mean()))
        bi = index[-1]
        bottom_heat.append(float(np.sum(T[bi[bi >= 0]]) * g["g_bottom"]))
    return out, {"unknowns": A.shape[0], "bottom_heat_W": bottom_heat, "die_mean": die_mean}


def solve_extrapolated(n, die_m, t, kappa, h, refinements, sources, cells_per_layer=None,
                       overhang_cells=None):
    """Richardson extrapolation of `solve` over two refinements (r1, r2):
    removes the O(volume size^2) error. Returns (theta, per-level thetas)."""
    r1, r2 = refinements
    T1, _ = solve(n, die_m, t, kappa, h, r1, sources, cells_per_layer, overhang_cells)
    T2, _ = solve(n, die_m, t, kappa, h, r2, sources, cells_per_layer, overhang_cells)
    return (r2 * r2 * T2 - r1 * r1 * T1) / (r2 * r2 - r1 * r1), (T1, T2)
