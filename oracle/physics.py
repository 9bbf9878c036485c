"""Oracle physics: stack spectrum, radial Green's functions, spectral kernel.

Test infrastructure only (see the package docstring). All arithmetic is FP64.

Model (the paper measures its baseline Green's function with a modified
HotSpot, Sec. V-C; the analytic layered model below is this project's reading
of the heat equation, Eq. 1, for the stack of the chip parameter table):

* layers i = 0..M-1 from the source plane down, thickness t_i, conductivity
  kappa_i, perfect contact, convective coefficient h below the last layer,
  adiabatic top surface except for the source, adiabatic die side walls;
* g^(k) [K m^2 / W] is the 2-D Fourier transform of the source-plane
  temperature of a unit point source (Eq. 2 with f_sp the Green's function);
* every grid cell is a uniform disc source of the cell's area (radius
  a = cell/sqrt(pi)), temperatures are read at cell centres;
* the die walls are handled by mirror images (Sec. IV-F), i.e. even
  reflection at both walls in x and y, which makes the imaged kernel
  2L-periodic.

The radial Green's function is split as Sec. II-B describes it, into a part that
decays fast with r and a part carried by the heat spreader:
  g^(k) = g1(k) + R(k),  g1(k) = tanh(k t0)/(kappa0 k)
g1 is the top layer on an isothermal base; its radial function decays like
K0(pi r / 2 t0) and is summed in real space. R(k) decays like exp(-2 k t0) and
its image lattice is summed in the spectral domain (Poisson summation).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


# --------------------------------------------------------------------------- #
# Stack spectrum g^(k)                                                          #
# --------------------------------------------------------------------------- #

def _tanhc(x):
    """tanh(x)/x with the x -> 0 limit 1."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = np.abs(x) > 1e-8
    out[nz] = np.tanh(x[nz]) / x[nz]
    small = ~nz
    out[small] = 1.0 - x[small] ** 2 / 3.0
    return out


def impedance_below(k, t, kappa, h, first: int):
    """Spectral impedance Z_first(k) looking down from the top of layer
    `first`: Z_M = 1/h and, for each layer from the bottom up,
    Z_i = (Z_{i+1} + tanh(k t_i)/(kappa_i k)) / (1 + kappa_i k tanh(k t_i) Z_{i+1}).

    This is the steady heat equation (Eq. 1, no time derivative) in one layer
    for one lateral wavenumber k: T(z) = A cosh(kz) + B sinh(kz), with flux and
    temperature continuous across interfaces and -kappa dT/dz = h T at the
    bottom.
    """
    k = np.asarray(k, dtype=np.float64)
    Z = np.full_like(k, 1.0 / h)
    for i in range(len(t) - 1, first - 1, -1):
        kk = kappa[i] * k
        tau = np.tanh(k * t[i])
        Z = (Z + (t[i] / kappa[i]) * _tanhc(k * t[i])) / (1.0 + kk * tau * Z)
    return Z


def ghat(k, t, kappa, h):
    """g^(k) of the full stack [K m^2/W] (impedance at the source plane)."""
    return impedance_below(k, t, kappa, h, 0)


def ghat_top(k, t, kappa):
    """g1(k) = tanh(k t0)/(kappa0 k): the source layer alone on an isothermal
    base (the fast-decaying part of the Green's function, Sec. II-B)."""
    return (t[0] / kappa[0]) * _tanhc(np.asarray(k, dtype=np.float64) * t[0])


def ghat_rest(k, t, kappa, h):
    """R(k) = g^(k) - g1(k), written without cancellation:
    R = Z_1 sech^2(k t0) / (1 + kappa0 k tanh(k t0) Z_1), Z_1 = impedance below
    the source layer. Decays like exp(-2 k t0)."""
    k = np.asarray(k, dtype=np.float64)
    if len(t) == 1:
        Z1 = np.full_like(k, 1.0 / h)
    else:
        Z1 = impedance_below(k, t, kappa, h, 1)
    x = k * t[0]
    sech2 = np.where(x < 350.0, 1.0 / np.cosh(np.minimum(x, 350.0)) ** 2, 0.0)
    return Z1 * sech2 / (1.0 + kappa[0] * k * np.tanh(x) * Z1)


def ghat_transfer_matrix(k: float, t, kappa, h) -> float:
    """Independent form of g^(k) for pinning: multiply the 2x2 layer matrices
    [[cosh, sinh/(kappa k)], [kappa k sinh, cosh]] that map (T, downward flux)
    from the bottom to the top of each layer, impose flux = h T at the bottom
    and unit flux at the top, and read T at the top. Only for moderate k
    (cosh/sinh overflow otherwise)."""
    M = np.eye(2)
    for ti, ki in zip(t, kappa):
        c, s = math.cosh(k * ti), math.sinh(k * ti)
        L = np.array([[c, s / (ki * k)], [ki * k * s, c]])
        M = M @ L
    # bottom state (T_b, q_b) with q_b = h T_b; top = M @ bottom
    top = M @ np.array([1.0, h])
    return top[0] / top[1]


# --------------------------------------------------------------------------- #
# Radial Green's functions (inverse Hankel transform, Eq. 8 / Theorem I)      #
# --------------------------------------------------------------------------- #

def disc_radius(cell_m: float) -> float:
    """Radius of the disc with the area of one square cell."""
    return cell_m / math.sqrt(math.pi)


def halfspace_disc(r, kappa: float, a: float):
    """Source-plane temperature of a unit-power uniform disc (radius a) on a
    half-space: G(r) = (1/2pi) int g(k) D(ka) J0(kr) k dk with g = 1/(kappa k),
    D(x) = 2 J1(x)/x, evaluated in closed form with complete elliptic
    integrals (pin only; the Hankel-transform normalisation is Theorem I).
    r <= a: (2/(pi^2 kappa a)) E(r/a); r >= a: (2 r/(pi^2 kappa a^2))
    [E(a/r) - (1 - a^2/r^2) K(a/r)] (modulus arguments)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.empty_like(r)
    inside = r <= a
    m_in = (r[inside] / a) ** 2
    out[inside] = 2.0 / (math.pi ** 2 * kappa * a) * special.ellipe(m_in)
    ro = r[~inside]
    m_out = (a / ro) ** 2
    out[~inside] = (2.0 * ro / (math.pi ** 2 * kappa * a ** 2)) * (
        special.ellipe(m_out) - (1.0 - m_out) * special.ellipk(m_out))
    return out


def g_top_radial(r, t0: float, kappa0: float, a: float):
    """Radial Green's function of the top layer on an isothermal base for a
    unit disc source: G1(r) = (1/2pi) int g1(k) D(ka) J0(kr) k dk.

    Evaluated by the eigenfunction (residue) series of g1, which is
    independent of any Hankel quadrature: tanh(kt)/k = sum_j (2/t)/(k^2+mu_j^2),
    mu_j = (j+1/2) pi/t, and the disc-averaged 2-D kernel of 1/(k^2+mu^2) is
    K0(mu r) 2 I1(mu a)/(mu a) / 2pi for r > a (Graf's addition theorem), and
    [1 - mu a K1(mu a) I0(mu r)] / (pi mu^2 a^2) for r < a. Hence
      r > a : G1 = 1/(pi kappa t) sum_j K0(mu_j r) 2 I1(mu_j a)/(mu_j a)
      r = 0 : G1 = 1/(pi kappa t) sum_j 2 (1 - mu_j a K1(mu_j a)) / (mu_j a)^2
    The r = 0 series converges like 1/j^2; its tail beyond J (where
    mu a K1(mu a) is below 1e-20) is summed exactly with the trigamma function.
    Radii with 0 < r <= a are not needed on the cell-centre lattice and raise.
    """
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    pref = 1.0 / (math.pi * kappa0 * t0)
    zero = r == 0.0
    if np.any((r > 0) & (r <= a)):
        raise ValueError("radius inside the source disc (0 < r <= a)")
    if np.any(zero):
        J = int(math.ceil(55.0 * t0 / (math.pi * a))) + 1
        mu_a = (np.arange(J) + 0.5) * math.pi * a / t0
        s = np.sum(2.0 * (1.0 - mu_a * special.k1(mu_a)) / mu_a ** 2)
        tail = 2.0 * t0 ** 2 / (math.pi ** 2 * a ** 2) * special.polygamma(1, J + 0.5)
        out[zero] = pref * (s + tail)
    ro = r[~zero]
    if ro.size:
        # terms decay like exp(-mu_j (r - a)); stop when below 1e-20 relative
        jmax = np.ceil(46.0 * t0 / (math.pi * (ro - a))).astype(np.int64) + 2
        acc = np.zeros_like(ro)
        for j in range(int(jmax.max())):
            act = jmax > j
            mu = (j + 0.5) * math.pi / t0
            rr = ro[act]
            acc[act] += special.kve(0, mu * rr) * special.ive(1, mu * a) \
                * np.exp(-mu * (rr - a)) * 2.0 / (mu * a)
        out[~zero] = pref * acc
    return out


# --------------------------------------------------------------------------- #
# Spreader wider than the die (Sec. II-B)                                       #
# --------------------------------------------------------------------------- #

def spreader_mean_impedance(t, kappa, h, first: int, die_m: float, side_m: float,
                            terms: int = 2048):
    """Footprint-mean impedance [K m^2/W] of layers first..M-1 when they are
    a square of side side_m (>= die_m, adiabatic side walls, convective
    bottom) heated by a uniform flux over the centred die footprint of side
    die_m: the mean temperature rise over the footprint per unit flux.

    Cosine series of the wide layers (Neumann walls at 0 and side_m): with
    d_m = (1/L) int_a^{a+L} cos(m pi x / L_s) dx (d_0 = 1, a = (L_s - L)/2)
    the flux is q sum_{m,n} c_m c_n cos cos with c_m = eps_m (L/L_s) d_m
    (eps_0 = 1, eps_m = 2), each mode answers with Z(k_mn), k_mn = pi
    sqrt(m^2 + n^2) / L_s (the impedance recursion of `impedance_below`),
    and its footprint mean is d_m d_n: so the mean is
    sum_{m,n} w_m w_n Z(k_mn), w_m = eps_m (L/L_s) d_m^2. The terms fall like
    1/(m^2 n^2 sqrt(m^2+n^2)), so the sum over m, n < M misses a tail that
    falls like 1/M^2; it is removed by one Richardson step,
    S = (4 S_M - S_{M/2}) / 3, with M = `terms`. For side_m = die_m only
    m = n = 0 survives and the result is Z(0), the die-sized stack."""
    M = int(terms)
    if M < 4 or M % 2:
        raise ValueError("terms must be even and >= 4")
    return (4.0 * _spreader_partial(t, kappa, h, first, die_m, side_m, M)
            - _spreader_partial(t, kappa, h, first, die_m, side_m, M // 2)) / 3.0


def _spreader_partial(t, kappa, h, first, die_m, side_m, terms):
    """sum_{m, n < terms} w_m w_n Z(k_mn) of `spreader_mean_impedance`."""
    L, Ls = float(die_m), float(side_m)
    a = 0.5 * (Ls - L)
    m = np.arange(terms, dtype=np.float64)
    d = np.ones(terms)
    mm = m[1:]
    d[1:] = Ls / (mm * math.pi * L) * (np.sin(mm * math.pi * (a + L) / Ls)
                                       - np.sin(mm * math.pi * a / Ls))
    w = (L / Ls) * np.where(m == 0, 1.0, 2.0) * d * d
    keep = np.abs(w) > 0.0
    w, mk = w[keep], m[keep]
    k = math.pi * np.sqrt(mk[:, None] ** 2 + mk[None, :] ** 2) / Ls
    Z = impedance_below(k, t, kappa, h, first)
    return float(np.sum(w[:, None] * w[None, :] * Z))


def ghat0_wide(t, kappa, h, first: int, die_m: float, side_m: float):
    """g^ of the uniform mode when layers first.. are a spreader of side
    side_m under a die of side die_m: the die layers in series (1-D, the die's
    own walls are adiabatic) over the spreader's footprint-mean impedance.

    This is the reading of Sec. II-B's decomposition of the Green's function
    into a fast-decaying part and a CONSTANT carried by the spreader: a wider
    spreader changes only that constant, i.e. only the uniform mode of the
    imaged kernel; every other mode keeps the stack spectrum of
    `impedance_below`. Equal to ghat(0) for side_m = die_m."""
    if not 1 <= first < len(t):
        raise ValueError("the spreader is layers first..M-1 with 1 <= first < M")
    top = sum(float(t[i]) / float(kappa[i]) for i in range(first))
    return top + spreader_mean_impedance(t, kappa, h, first, die_m, side_m)


def _uniform_mode_shift(n, die_m, t, kappa, h, spreader):
    """Change of K~[0, 0] for a spreader (first, side_m) wider than the die:
    (g^0_wide - g^(0)) / cell^2 (the primary uniform term is g^(0) D(0) /
    cell^2), i.e. a constant (g^0_wide - g^(0)) / L^2 added to the Green's
    function. 0 without a spreader."""
    if spreader is None:
        return 0.0
    first, side_m = spreader
    g0 = float(ghat(np.array([0.0]), t, kappa, h)[0])
    cell = die_m / n
    return (ghat0_wide(t, kappa, h, first, die_m, side_m) - g0) / cell ** 2


# --------------------------------------------------------------------------- #
# Spectral kernel of the imaged die                                            #
# --------------------------------------------------------------------------- #

def _disc_factor(x):
    """D(x) = 2 J1(x)/x, D(0) = 1: 2-D Fourier transform of a unit disc."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x > 1e-8
    out[nz] = 2.0 * special.j1(x[nz]) / x[nz]
    out[~nz] = 1.0 - x[~nz] ** 2 / 8.0
    return out


def real_space_cutoff(t0: float, rel: float = 1e-18) -> float:
    """Radius beyond which the top-layer Green's function (decay K0(pi r/2t0))
    is below `rel` of its scale."""
    return 2.0 * t0 / math.pi * math.log(1.0 / rel) + 2.0 * t0


def spectrum(n: int, die_m: float, t, kappa, h, n_modes: int | None = None,
             rel: float = 1e-18, spreader=None):
    """K~[p, q] for p, q in [0, n_modes) (n_modes defaults to n).

    Definition (Sec. IV-F images + Eq. 2): with all mirror images the imaged
    kernel is the lattice sum of the cell Green's function G(r) over every
    lattice vector, and its cosine series on the 2n-periodic grid is
      K~[p,q] = sum_{m in Z^2} G(cell |m|) cos(pi p m_x / n) cos(pi q m_y / n).
    G = G1 + G_R (split of the module docstring):
      * the G1 part is summed directly over lattice points within the
        real-space cutoff (G1 evaluated by its eigenfunction series);
      * the G_R part is summed by Poisson summation,
        sum_m G_R(cell|m|) e^{-i w.m cell} = cell^-2 sum_{s,t} R(|k|) D(|k|a),
        k = (pi (p + 2 n s) / L, pi (q + 2 n t) / L), truncated where
        exp(-2 k t0) is below `rel`.
    spreader = (first, side_m): layers first.. are a spreader wider than the
    die (`ghat0_wide`): the uniform mode K~[0, 0] takes its g^0_wide.
    Returns the FP64 array [n_modes, n_modes] (row index = y mode).
    """
    t = tuple(float(x) for x in t)
    kappa = tuple(float(x) for x in kappa)
    nm = n if n_modes is None else n_modes
    cell = die_m / n
    a = disc_radius(cell)
    # --- real-space part: G1 on the lattice square [-R, R]^2
    R = int(math.ceil(real_space_cutoff(t[0], rel) / cell))
    m = np.arange(-R, R + 1)
    rad2 = m[:, None] ** 2 + m[None, :] ** 2
    uniq, inv = np.unique(rad2, return_inverse=True)
    g1 = g_top_radial(cell * np.sqrt(uniq.astype(np.float64)), t[0], kappa[0], a)
    G = g1[inv].reshape(rad2.shape)
    p = np.arange(nm)
    C = np.cos(np.pi * np.outer(p, m) / n)          # [nm, 2R+1]
    K1 = C @ G @ C.T
    # --- spectral part: aliases of R(k) D(ka)
    S = int(math.ceil((cell * math.log(1.0 / rel) / (2 * math.pi * t[0]) + 1) / 2)) + 1
    KR = np.zeros((nm, nm))
    for s_ in range(-S, S + 1):
        ky = np.pi * (p + 2 * n * s_) / die_m
        for t_ in range(-S, S + 1):
            kx = np.pi * (p + 2 * n * t_) / die_m
            kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
            KR += ghat_rest(kk, t, kappa, h) * _disc_factor(kk * a)
    KR /= cell ** 2
    K = K1 + KR
    K[0, 0] += _uniform_mode_shift(n, die_m, t, kappa, h, spreader)
    return K


def kernel_periodic(n: int, die_m: float, t, kappa, h, spreader=None):
    """Imaged kernel K_per(dy, dx) on the 2n x 2n periodic grid: the inverse
    2n-point DFT of the full spectrum K~[p, q], p, q in [0, 2n)."""
    Kfull = spectrum(n, die_m, t, kappa, h, n_modes=2 * n, spreader=spreader)
    return np.real(np.fft.ifft2(Kfull))


def alias_only_primary(n: int, die_m: float, t, kappa, h):
    """cell^-2 g^(|k_pq|) D(|k_pq| a) for the primary wavenumbers
    k = pi (p, q)/L: the part of K~ carried by the box's own cosine modes."""
    cell = die_m / n
    a = disc_radius(cell)
    p = np.arange(n)
    kk = np.pi * np.sqrt(p[:, None] ** 2 + p[None, :] ** 2) / die_m
    return ghat(kk, t, kappa, h) * _disc_factor(kk * a) / cell ** 2
