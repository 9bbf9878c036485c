"""Seeded synthetic inputs for the thermal solve (power maps, variation fields,
power traces).

This module is shared by the FP64 oracle and the CUDA path, so it holds none of
the solver's arithmetic: it only draws the inputs the method consumes.

* Power maps: rectangular blocks with uniform power density on a floor, plus
  small high-density hotspots painted last (the stress-test floorplans of the
  paper's evaluation, Sec. V-C test cases 2/4/5; block sizes and overlap order
  are unstated there, so later blocks simply overwrite earlier ones).
* Variation field z: white Gaussian noise smoothed by a Gaussian filter of std
  l/2 with mirror boundaries, then standardised per sample, so that neighbouring
  points within about l are strongly correlated (systematic within-die
  variation modelled as a correlated multivariate Gaussian, Sec. II-C).
* Baseline leakage P_leak0 = p_l * A_cell * exp(sigma * z) (the exponential
  variation factor of Eq. 4) and conductivity multiplier s = 1 - gamma*sigma*z
  (Sec. II-E): both come from the same field z.
* Power traces for the transient: every block follows its own 3-state Markov
  chain {floor, half power, full power}.

Everything is drawn with torch generators seeded from (config id, seed,
stream), on CPU or CUDA. Units: metres, watts per cell, kelvin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

SEED = 20230722
STREAM_FLOORPLAN, STREAM_FIELD, STREAM_TRACE = 0, 1, 2

MM = 1e-3
W_PER_MM2 = 1e6  # W/m^2


@dataclass
class Stack:
    """Layer stack (top = source layer first) with a convective bottom.

    Defaults follow the paper's chip parameter table (Sec. V-A) except the
    silicon thickness of the configured workloads (0.5 mm) and the heat-sink
    coefficient h, which the paper does not give.
    """
    thickness_m: tuple = (0.5 * MM, 0.02 * MM, 3.5 * MM)
    kappa_W_mK: tuple = (130.0, 4.0, 400.0)
    h_conv_W_m2K: float = 2.0e4
    heat_cap_J_m2K: float = 1.63e6 * 0.5 * MM


@dataclass
class Physics:
    """Leakage / conductivity coefficients (Eqs. 4-5, 9-12)."""
    beta_per_K: float = 0.0275          # paper's chip parameter table
    gamma: float = 0.3                  # c' * k0' (unstated in the paper)
    eta: float = 1.3                    # exponent of kappa(T) for Si (unstated)
    t_amb_K: float = 318.15             # paper's chip parameter table
    p_leak_W_m2: float = 0.1 * W_PER_MM2

    @property
    def alpha_per_K(self) -> float:
        return self.gamma * self.eta / self.t_amb_K


@dataclass
class Workload:
    name: str
    n: int
    die_m: float
    n_blocks: int
    dens_lo_W_m2: float
    dens_hi_W_m2: float
    floor_W_m2: float = 0.01 * W_PER_MM2
    n_hot: int = 0
    hot_W_m2: float = 5.0 * W_PER_MM2
    hot_size_m: float = 0.5 * MM
    sigma: tuple = (0.05, 0.05)        # range of the variation std
    corr_len_m: tuple = (1 * MM, 1 * MM)
    corr: str = "gaussian"             # "gaussian" or "spherical" (range = corr_len)
    stack: Stack = field(default_factory=Stack)
    physics: Physics = field(default_factory=Physics)
    config_id: int = 0

    @property
    def cell_m(self) -> float:
        return self.die_m / self.n


def workload(name: str) -> Workload:
    """Named synthetic workloads shaped like the paper's test cases."""
    if name == "c1_64":
        return Workload("c1_64", 64, 10 * MM, 8, 0.2e6, 2.0e6, sigma=(0.05, 0.05),
                        corr_len_m=(1 * MM, 1 * MM), config_id=1)
    if name == "c2_256":
        return Workload("c2_256", 256, 20 * MM, 32, 0.1e6, 3.0e6, n_hot=4,
                        sigma=(0.08, 0.08), corr_len_m=(2 * MM, 2 * MM), config_id=2)
    if name.startswith("c3_"):
        n = int(name.split("_")[1])
        return Workload(name, n, 20 * MM, 32, 0.1e6, 3.0e6, n_hot=4,
                        sigma=(0.05, 0.10), corr_len_m=(0.5 * MM, 3 * MM), config_id=3)
    if name == "c4_1024":
        return Workload("c4_1024", 1024, 20 * MM, 32, 0.1e6, 3.0e6, n_hot=4,
                        sigma=(0.08, 0.08), corr_len_m=(2 * MM, 2 * MM), config_id=4)
    if name.startswith("tiny_"):
        n = int(name.split("_")[1])
        return Workload(name, n, 10 * MM, 4, 0.2e6, 2.0e6, n_hot=1, hot_size_m=1.0 * MM,
                        sigma=(0.05, 0.05), corr_len_m=(1.5 * MM, 1.5 * MM), config_id=9)
    raise KeyError(name)


def _gen(device, config_id: int, seed: int, stream: int, sample: int = 0) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(((config_id * 1_000_003 + seed) * 7 + stream) * 1_000_033 + sample)
    return g


def _blocks(w: Workload, g: torch.Generator, device):
    """Draw block rectangles (in cells) and densities for one floorplan."""
    n = w.n
    rects = []
    for _ in range(w.n_blocks):
        u = torch.rand(5, generator=g, device=device, dtype=torch.float64).cpu().tolist()
        bw = max(1, int(round((0.05 + 0.25 * u[0]) * n)))
        bh = max(1, int(round((0.05 + 0.25 * u[1]) * n)))
        x0 = min(n - bw, int(u[2] * (n - bw + 1)))
        y0 = min(n - bh, int(u[3] * (n - bh + 1)))
        dens = w.dens_lo_W_m2 + (w.dens_hi_W_m2 - w.dens_lo_W_m2) * u[4]
        rects.append((x0, y0, bw, bh, dens))
    hs = max(1, int(round(w.hot_size_m / w.cell_m)))
    for _ in range(w.n_hot):
        u = torch.rand(2, generator=g, device=device, dtype=torch.float64).cpu().tolist()
        x0 = min(n - hs, int(u[0] * (n - hs + 1)))
        y0 = min(n - hs, int(u[1] * (n - hs + 1)))
        rects.append((x0, y0, hs, hs, w.hot_W_m2))
    return rects


def power_maps(w: Workload, count: int, seed: int = SEED, first: int = 0,
               device="cpu", dtype=torch.float32) -> torch.Tensor:
    """[count, n, n] dynamic power in W per cell (floorplan index first..)."""
    a_cell = w.cell_m ** 2
    out = torch.empty(count, w.n, w.n, device=device, dtype=torch.float64)
    for i in range(count):
        g = _gen(device, w.config_id, seed, STREAM_FLOORPLAN, first + i)
        out[i].fill_(w.floor_W_m2 * a_cell)
        for (x0, y0, bw, bh, dens) in _blocks(w, g, device):
            out[i, y0:y0 + bh, x0:x0 + bw] = dens * a_cell
    return out.to(dtype)


def variation_fields(w: Workload, count: int, seed: int = SEED, first: int = 0,
                     device="cpu", dtype=torch.float32, chunk: int = 256):
    """Standardised correlated Gaussian fields z [count, n, n] plus the per-sample
    (sigma, corr_len) they were drawn with.

    Smoothing is done on the mirror-extended (2n x 2n) field in the Fourier
    domain with a Gaussian of std corr_len/2, i.e. a Gaussian filter with
    reflecting boundaries. With w.corr == "spherical" the filter is instead the
    square root of the spectrum of the spherical correlation
    rho(r) = 1 - 1.5 r/phi + 0.5 (r/phi)^3 for r < phi, 0 beyond (phi =
    corr_len), the correlation Sec. II-C gives the systematic variation, taken
    on the periodic 2n x 2n grid (circulant embedding; negative spectral
    values from the truncation are clipped to zero).
    """
    n = w.n
    zs = torch.empty(count, n, n, device=device, dtype=torch.float64)
    params = torch.empty(count, 2, dtype=torch.float64)
    kx = torch.fft.fftfreq(2 * n, d=w.cell_m, device=device, dtype=torch.float64) * 2 * math.pi
    k2 = kx[:, None] ** 2 + kx[None, :] ** 2
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        white = torch.empty(c1 - c0, n, n, device=device, dtype=torch.float64)
        for j in range(c0, c1):
            g = _gen(device, w.config_id, seed, STREAM_FIELD, first + j)
            white[j - c0] = torch.randn(n, n, generator=g, device=device, dtype=torch.float64)
            u = torch.rand(2, generator=g, device=device, dtype=torch.float64).cpu()
            params[j, 0] = w.sigma[0] + (w.sigma[1] - w.sigma[0]) * u[0]
            params[j, 1] = w.corr_len_m[0] + (w.corr_len_m[1] - w.corr_len_m[0]) * u[1]
        ext = torch.cat([white, white.flip(-1)], dim=-1)
        ext = torch.cat([ext, ext.flip(-2)], dim=-2)
        if w.corr == "spherical":
            filt = _spherical_filter(n, w.cell_m, params[c0:c1, 1].to(device))
        else:
            sf = (params[c0:c1, 1] / 2).to(device)[:, None, None]
            filt = torch.exp(-0.5 * sf ** 2 * k2[None])
        sm = torch.fft.ifft2(torch.fft.fft2(ext) * filt).real[:, :n, :n]
        sm = sm - sm.mean(dim=(-1, -2), keepdim=True)
        sm = sm / sm.std(dim=(-1, -2), keepdim=True).clamp_min(1e-300)
        zs[c0:c1] = sm
    return zs.to(dtype), params


def _spherical_filter(n: int, cell_m: float, phi: torch.Tensor) -> torch.Tensor:
    """sqrt of the 2n x 2n periodic spectrum of the spherical correlation of
    range phi (one filter per entry of phi)."""
    d = torch.arange(2 * n, device=phi.device, dtype=torch.float64)
    d = torch.minimum(d, 2 * n - d) * cell_m
    r = torch.sqrt(d[:, None] ** 2 + d[None, :] ** 2)[None]
    x = (r / phi[:, None, None]).clamp(max=1.0)
    rho = 1.0 - 1.5 * x + 0.5 * x ** 3
    return torch.fft.fft2(rho).real.clamp_min(0.0).sqrt()


def leakage_and_conductivity(w: Workload, z: torch.Tensor, sigma: torch.Tensor,
                             dtype=torch.float32):
    """P_leak0 [W/cell] and the conductivity multiplier s from the same field z."""
    zz = z.to(torch.float64)
    sg = sigma.to(zz.device, torch.float64).reshape(-1, 1, 1)
    ph = w.physics
    p_leak0 = ph.p_leak_W_m2 * w.cell_m ** 2 * torch.exp(sg * zz)
    s = 1.0 - ph.gamma * sg * zz
    return p_leak0.to(dtype), s.to(dtype)


def steady_inputs(w: Workload, count: int, seed: int = SEED, first: int = 0,
                  n_floorplans: int | None = None, device="cpu", dtype=torch.float32):
    """(P_dyn, P_leak0, s), each [count, n, n]. Sample i uses floorplan
    i mod n_floorplans (every sample has its own variation field)."""
    nf = count if n_floorplans is None else min(count, n_floorplans)
    plans = power_maps(w, nf, seed, first, device, dtype)
    idx = torch.arange(count, device=device) % nf
    p_dyn = plans[idx].contiguous()
    z, params = variation_fields(w, count, seed, first, device, dtype)
    p_leak0, s = leakage_and_conductivity(w, z, params[:, 0], dtype)
    return p_dyn, p_leak0.contiguous(), s.contiguous()


def markov_trace(w: Workload, n_steps: int, seed: int = SEED, device="cpu",
                 dtype=torch.float32, p_stay: float = 0.8) -> torch.Tensor:
    """[n_steps, n, n] dynamic power trace; each block (and hotspot) switches
    among {floor, half, full} density with P(stay)=p_stay and the rest split
    evenly; initial states uniform."""
    a_cell = w.cell_m ** 2
    g = _gen(device, w.config_id, seed, STREAM_FLOORPLAN, 0)
    rects = _blocks(w, g, device)
    gt = _gen(device, w.config_id, seed, STREAM_TRACE, 0)
    nb = len(rects)
    state = torch.randint(0, 3, (nb,), generator=gt, device=device).cpu().tolist()
    out = torch.empty(n_steps, w.n, w.n, device=device, dtype=torch.float64)
    for t in range(n_steps):
        if t > 0:
            u = torch.rand(nb, 2, generator=gt, device=device, dtype=torch.float64).cpu().tolist()
            for b in range(nb):
                if u[b][0] >= p_stay:
                    state[b] = (state[b] + (1 if u[b][1] < 0.5 else 2)) % 3
        out[t].fill_(w.floor_W_m2 * a_cell)
        for b, (x0, y0, bw, bh, dens) in enumerate(rects):
            level = (w.floor_W_m2, 0.5 * dens, dens)[state[b]]
            out[t, y0:y0 + bh, x0:x0 + bw] = level * a_cell
    return out.to(dtype)


def batch_workload(n: int = 256, count: int = 4096) -> Workload:
    """Batched steady workload: `count` solves at n x n on a 20 x 20 mm die,
    each with its own variation field (sigma 8 %, correlation length 2 mm)
    over 64 floorplans of 32 blocks U[0.1, 3] W/mm^2 plus 4 hotspots of
    5 W/mm^2 (0.5 mm)."""
    w = Workload("batch_%d_x%d" % (n, count), n, 20 * MM, 32, 0.1e6, 3.0e6, n_hot=4,
                 sigma=(0.08, 0.08), corr_len_m=(2 * MM, 2 * MM), config_id=5)
    return w


def batch_inputs(n: int = 256, count: int = 4096, device="cuda", seed: int = SEED):
    w = batch_workload(n, count)
    pd, pl, s = steady_inputs(w, count, seed=seed, n_floorplans=64, device=device)
    return w, pd, pl, s
