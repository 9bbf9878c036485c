"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(not against the oracle itself). CPU only."""
import functools
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy import integrate, special

import synth
from oracle import physics as ph
from oracle import solve as so

HERE = os.path.dirname(os.path.abspath(__file__))
STACK3 = ((0.5e-3, 0.02e-3, 3.5e-3), (130.0, 4.0, 400.0), 2.0e4)


# ---------------------------------------------------------------- P1: g^(k)

def test_ghat_matches_transfer_matrix_form():
    t, kap, h = STACK3
    for k in [1e-3, 0.5, 10.0, 300.0, 2e3, 8e3]:
        a = ph.ghat(np.array([k]), t, kap, h)[0]
        b = ph.ghat_transfer_matrix(k, t, kap, h)
        assert abs(a - b) <= 1e-12 * abs(b)


def test_ghat_limits_series_resistance_and_halfspace():
    t, kap, h = STACK3
    g0 = ph.ghat(np.array([0.0]), t, kap, h)[0]
    assert g0 == pytest.approx(sum(a / b for a, b in zip(t, kap)) + 1 / h, rel=1e-14)
    k = np.array([2e5, 1e6])
    assert np.allclose(ph.ghat(k, t, kap, h) * kap[0] * k, 1.0, rtol=1e-12)


def test_ghat_single_layer_closed_form():
    t, kap, h = (0.3e-3,), (150.0,), 5e3
    k = np.logspace(-1, 4.5, 25)
    T = np.tanh(k * t[0])
    closed = (kap[0] * k + h * T) / (kap[0] * k * (h + kap[0] * k * T))
    assert np.allclose(ph.ghat(k, t, kap, h), closed, rtol=1e-13)


def test_split_of_ghat_is_exact_and_rest_decays():
    t, kap, h = STACK3
    k = np.logspace(-3, 4.6, 60)
    g = ph.ghat(k, t, kap, h)
    assert np.allclose(ph.ghat_top(k, t, kap) + ph.ghat_rest(k, t, kap, h), g, rtol=1e-13)
    kk = np.array([3e4, 6e4])
    r = ph.ghat_rest(kk, t, kap, h)
    assert np.all(r < 4 * g[0] * np.exp(-2 * kk * t[0]) * 1.01)


# --------------------------------------------- P2: Hankel transform (Thm I)

def test_halfspace_disc_centre_and_far_field():
    kap, a = 130.0, 40e-6
    assert ph.halfspace_disc(0.0, kap, a)[0] == pytest.approx(1 / (math.pi * kap * a), rel=1e-14)
    r = np.array([200 * a, 2000 * a])
    assert np.allclose(ph.halfspace_disc(r, kap, a), 1 / (2 * math.pi * kap * r), rtol=3e-5)


def test_halfspace_disc_equals_numeric_hankel_integral():
    # (1/2pi) int (1/(kappa k)) D(ka) J0(kr) k dk, Theorem I normalisation
    kap, a = 130.0, 40e-6
    for r in [0.0, 0.5 * a, 1.7 * a, 6 * a]:
        f = lambda x: 2 * special.j1(x) / x * special.j0(x * r / a) if x > 0 else 1.0
        v, _ = integrate.quad(f, 0, 4000, limit=4000)
        # tail beyond x = 4000 averages out (integrand ~ x^-2 oscillating)
        assert v / (2 * math.pi * kap * a) == pytest.approx(ph.halfspace_disc(r, kap, a)[0], rel=2e-4)


def _disc_average_image_series(r, t, kap, a, J=4000, nr=80, nth=160):
    """Temperature at distance r of a unit-power uniform disc on a slab with
    adiabatic top and isothermal base at depth t, by the method of images in z
    (point sources at depth 2jt with sign (-1)^j) averaged over the disc by a
    2-D Gauss quadrature. Independent of the eigenfunction series."""
    x, wx = np.polynomial.legendre.leggauss(nr)
    th, wt = np.polynomial.legendre.leggauss(nth)
    rho = 0.5 * a * (x + 1)
    wr = 0.5 * a * wx
    ang = math.pi * (th + 1)
    wa = math.pi * wt
    px = rho[:, None] * np.cos(ang)[None, :]
    py = rho[:, None] * np.sin(ang)[None, :]
    d = np.sqrt((px - r) ** 2 + py ** 2)
    w = wr[:, None] * wa[None, :] * rho[:, None] / (math.pi * a * a)
    j = np.arange(1, J + 1)
    img = np.zeros_like(d)
    partial = []
    for jj in j:
        img += 2 * (-1) ** jj / np.sqrt(d ** 2 + (2 * jj * t) ** 2)
        if jj >= J - 1:
            partial.append(img.copy())
    img = 0.5 * (partial[0] + partial[1])       # average of two partial sums
    if r == 0.0:
        direct = 2.0 / a                        # mean of 1/d over the disc
    else:
        direct = np.sum(w / d)
    return (direct + np.sum(w * img)) / (2 * math.pi * kap)


@pytest.mark.parametrize("rfac", [0.0, 1.7724538509055159, 3.5449077018110318, 12.0])
def test_top_layer_green_eigen_series_vs_images(rfac):
    t, kap, a = 0.5e-3, 130.0, 44e-6
    r = rfac * a
    ref = _disc_average_image_series(r, t, kap, a)
    got = ph.g_top_radial(r, t, kap, a)[0]
    assert got == pytest.approx(ref, rel=2e-6)


def test_top_layer_green_thick_limit_is_halfspace():
    kap, a = 130.0, 44e-6
    g = ph.g_top_radial(0.0, 1.0, kap, a)[0]       # t = 1 m >> a
    assert g == pytest.approx(1 / (math.pi * kap * a), rel=1e-4)


def test_top_layer_green_by_hankel_quadrature():
    # G1 = halfspace - (1/2pi kappa) int (1 - tanh(kt)) D(ka) J0(kr) dk
    t, kap, a = 0.5e-3, 130.0, 44e-6
    for r in [0.0, 1.77 * a, 9 * a, 40 * a]:
        f = lambda k: (1 - math.tanh(k * t)) * 2 * special.j1(k * a) / (k * a) * special.j0(k * r) if k > 0 else 1.0
        v, _ = integrate.quad(f, 0, 45 / t, limit=2000, epsabs=0, epsrel=1e-12)
        ref = ph.halfspace_disc(r, kap, a)[0] - v / (2 * math.pi * kap)
        assert ph.g_top_radial(r, t, kap, a)[0] == pytest.approx(ref, rel=1e-11, abs=1e-12)


# ---------------------------------- P3: real/spectral split vs image road

def _image_road_kper(n, L, t, kap, h, Rmax, nodes=3000):
    cell = L / n
    a = ph.disc_radius(cell)
    R = int(math.ceil(Rmax / cell))
    m = np.arange(-R, R + 1)
    r2 = m[:, None] ** 2 + m[None, :] ** 2
    u, inv = np.unique(r2, return_inverse=True)
    r = cell * np.sqrt(u.astype(float))
    g1 = ph.g_top_radial(r, t[0], kap[0], a)
    Kmax = 45 / t[0]
    x, w = np.polynomial.legendre.leggauss(nodes)
    k = 0.5 * Kmax * (x + 1)
    w = 0.5 * Kmax * w
    f = ph.ghat_rest(k, t, kap, h) * 2 * special.j1(k * a) / (k * a) * k * w / (2 * math.pi)
    gR = np.array([np.sum(f * special.j0(k * rr)) for rr in r])
    G = (g1 + gR)[inv].reshape(r2.shape)
    Kp = np.zeros((2 * n, 2 * n))
    np.add.at(Kp, (m[:, None] % (2 * n), m[None, :] % (2 * n)), G)
    return Kp


@pytest.mark.parametrize("n", [8, 32])
@pytest.mark.parametrize("stack", [((0.5e-3,), (130.0,), 1e5),
                                   ((0.3e-3, 0.5e-3), (130.0, 400.0), 2e5)])
def test_kernel_split_equals_image_sum(stack, n):
    """The real-space/spectral split of the kernel against the plain image
    sum at 8^2 (cells wider than the silicon) and 32^2 (cells thinner than
    it, many lattice radii inside the real-space cutoff)."""
    t, kap, h = stack
    L = 4e-3
    g0 = ph.ghat(np.array([0.0]), t, kap, h)[0]
    lam = math.sqrt(sum(a * b for a, b in zip(t, kap)) * g0)
    Ki = _image_road_kper(n, L, t, kap, h, 32 * lam)
    Ks = ph.kernel_periodic(n, L, t, kap, h)
    assert np.max(np.abs(Ki - Ks)) <= 1e-9 * np.max(np.abs(Ks))


# ------------------------------------------- convolution: direct vs cosine

def test_direct_mirror_convolution_equals_dct_form_and_is_symmetric():
    t, kap, h = STACK3
    n, L = 16, 10e-3
    Kt = ph.spectrum(n, L, t, kap, h)
    Lm = so.mirror_operator(ph.kernel_periodic(n, L, t, kap, h))
    rng = np.random.default_rng(3)
    q = rng.random((n, n))
    a = so.direct_convolve(Lm, q)
    assert np.max(np.abs(a - so.spectral_convolve(Kt, q))) <= 1e-13 * np.max(np.abs(a))
    # P6 symmetry: mirror images make the operator commute with flips/transpose
    assert np.allclose(so.direct_convolve(Lm, q.T), a.T, rtol=1e-13)
    assert np.allclose(so.direct_convolve(Lm, q[::-1]), a[::-1], rtol=1e-13)
    # P5 energy balance: mean(L q) = K~[0,0] mean(q)
    assert a.mean() == pytest.approx(Kt[0, 0] * q.mean(), rel=1e-13)
    # the operator is symmetric (reciprocity) and positive
    assert np.allclose(Lm, Lm.T, rtol=1e-13)
    assert np.all(Lm > 0)


def test_uniform_power_gives_uniform_rise_close_to_1d_resistance():
    # TC4-like uniform map (Sec. V-C): theta = q K~[0,0] everywhere, and
    # K~[0,0] cell^2 = g^(0) up to the sub-cell alias terms (<1e-3)
    t, kap, h = STACK3
    n, L = 32, 10e-3
    Kt = ph.spectrum(n, L, t, kap, h)
    q = np.full((n, n), 0.01)
    th = so.spectral_convolve(Kt, q)
    assert np.ptp(th) <= 1e-12 * th.max()
    assert th[0, 0] == pytest.approx(0.01 * Kt[0, 0], rel=1e-13)
    g0 = ph.ghat(np.array([0.0]), t, kap, h)[0]
    assert Kt[0, 0] * (L / n) ** 2 == pytest.approx(g0, rel=1e-3)


def test_checkerboard_symmetry_tc5():
    t, kap, h = STACK3
    n, L = 16, 10e-3
    Kt = ph.spectrum(n, L, t, kap, h)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    q = ((xx + yy) % 2).astype(float) * 0.02
    th = so.spectral_convolve(Kt, q)
    assert np.allclose(th, th.T, rtol=1e-12)
    assert np.allclose(th, th[::-1, ::-1], rtol=1e-12)


# ----------------------------------------------- P6-P8: the fixed point

def _c1_inputs(n=32, sigma=0.05, gamma=None):
    w = synth.workload("c1_64")
    w.n = n
    if gamma is not None:
        w.physics.gamma = gamma
    w.sigma = (sigma, sigma)
    pd, pl, s = synth.steady_inputs(w, 1, dtype=torch.float64)
    return w, pd[0].numpy(), pl[0].numpy(), s[0].numpy()


def test_linearity_without_feedback():
    t, kap, h = STACK3
    n, L = 16, 10e-3
    Kt = ph.spectrum(n, L, t, kap, h)
    rng = np.random.default_rng(5)
    q1, q2 = rng.random((n, n)), rng.random((n, n))
    ones = np.ones((n, n))
    z = np.zeros((n, n))
    th1, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), q1, z, ones, 0.0, 0.0)
    th2, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), q2, z, ones, 0.0, 0.0)
    th3, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), 2 * q1 + q2, z, ones, 0.0, 0.0)
    assert np.allclose(th3, 2 * th1 + th2, rtol=1e-12)


def test_uniform_variation_reduces_to_shift_invariant_solution():
    # P7: no variation, alpha = 0: the converged fixed point is Eq. 21's
    # shift-invariant modified Green's function applied to P_dyn + mu
    w, pd, pl, s = _c1_inputs(32, sigma=0.0, gamma=0.0)
    st = w.stack
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    assert np.ptp(pl) == 0.0 and np.all(s == 1.0)
    th, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), pd, pl, s,
                         w.physics.beta_per_K, 0.0, tol=1e-11)
    closed = so.shift_invariant(Kt, pd, pl, w.physics.beta_per_K)
    assert np.max(np.abs(th - closed)) <= 1e-9


def test_split_and_unsplit_fixed_points_coincide_and_det_only_differs():
    # P8, and the paper's TC3 observation that ignoring the shift-variant part
    # moves the answer well beyond the tolerance
    w, pd, pl, s = _c1_inputs(32, sigma=0.08)
    st, phy = w.stack, w.physics
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    Lm = so.mirror_operator(ph.kernel_periodic(w.n, w.die_m, st.thickness_m, st.kappa_W_mK,
                                               st.h_conv_W_m2K))
    th1, _, it1 = so.picard(lambda x: so.direct_convolve(Lm, x), pd, pl, s,
                            phy.beta_per_K, phy.alpha_per_K, tol=1e-11)
    th2, _, it2 = so.picard_split(Kt, pd, pl, s, phy.beta_per_K, phy.alpha_per_K, tol=1e-11)
    assert np.max(np.abs(th1 - th2)) <= 1e-9
    assert it2 < it1
    det = so.shift_invariant(Kt, pd, pl, phy.beta_per_K)
    assert np.max(np.abs(det - th1)) > 0.05


def test_fixed_point_residual_is_small():
    w, pd, pl, s = _c1_inputs(16, sigma=0.08)
    st, phy = w.stack, w.physics
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    th, u, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), pd, pl, s,
                         phy.beta_per_K, phy.alpha_per_K, tol=1e-12)
    u2 = so.spectral_convolve(Kt, pd + pl * (1 + phy.beta_per_K * th))
    assert np.max(np.abs(u2 - u)) <= 1e-10
    assert np.allclose(th, s * u * (1 + phy.alpha_per_K * th), rtol=1e-12)


def test_runaway_is_reported():
    w, pd, pl, s = _c1_inputs(16)
    st = w.stack
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    with pytest.raises(so.SolveError):
        so.picard(lambda x: so.spectral_convolve(Kt, x), pd * 60, pl, s, 0.0, 5e-3)


# --------------------------------------------------------- P10: transient

def test_step_spectrum_limits_and_single_pole_law():
    t, kap, h = STACK3
    C = 1.63e6 * 0.5e-3
    n, L = 16, 10e-3
    Kt = ph.spectrum(n, L, t, kap, h)
    assert np.allclose(so.step_spectrum(n, L, t, kap, h, C, 1e3), Kt, rtol=1e-12)
    s = [so.step_spectrum(n, L, t, kap, h, C, j * 1e-3)[0, 0] for j in (1, 2, 5, 20, 50)]
    assert all(b > a for a, b in zip(s, s[1:]))
    g0 = ph.ghat(np.array([0.0]), t, kap, h)[0]
    tau = C * g0
    # the uniform mode decays with the single pole tau = C g^(0) (Eq. 35); the
    # sub-cell alias modes have tau < 1 ms and are settled after a few ms
    for tt, val in zip((5e-3, 20e-3, 50e-3), s[2:]):
        assert (Kt[0, 0] - val) * (L / n) ** 2 == pytest.approx(g0 * math.exp(-tt / tau), rel=1e-5)


def test_duhamel_constant_power_approaches_steady_fixed_point():
    w, pd, pl, s = _c1_inputs(8, sigma=0.08)
    st, phy = w.stack, w.physics
    C = 20.0   # small areal heat capacity: tau ~ 1 ms, steady within 60 steps
    dt = 1e-3
    spectra = [so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                                C, j * dt) for j in range(1, 61)]
    trace = np.repeat(pd[None], 60, axis=0)
    th = so.duhamel(spectra, trace, pl, s, phy.beta_per_K, phy.alpha_per_K)
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    ss, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), pd, pl, s,
                         phy.beta_per_K, phy.alpha_per_K, tol=1e-12)
    assert np.max(np.abs(th[-1] - ss)) <= 1e-6
    assert np.all(np.diff(th[:, 3, 3]) >= -1e-12)   # monotone rise


def test_duhamel_superposition_without_feedback():
    t, kap, h = STACK3
    n, L, C, dt = 8, 10e-3, 1.63e6 * 0.5e-3, 1e-3
    spectra = [so.step_spectrum(n, L, t, kap, h, C, j * dt) for j in range(1, 7)]
    rng = np.random.default_rng(11)
    a, b = rng.random((6, n, n)) * 0.01, rng.random((6, n, n)) * 0.01
    z, one = np.zeros((n, n)), np.ones((n, n))
    ta = so.duhamel(spectra, a, z, one, 0.0, 0.0)
    tb = so.duhamel(spectra, b, z, one, 0.0, 0.0)
    tab = so.duhamel(spectra, a + b, z, one, 0.0, 0.0)
    assert np.allclose(tab, ta + tb, rtol=1e-12)
    # constant power: theta_n = S_n * P
    c = np.repeat(a[:1], 6, axis=0)
    tc = so.duhamel(spectra, c, z, one, 0.0, 0.0)
    assert np.allclose(tc[4], so.spectral_convolve(spectra[4], a[0]), rtol=1e-12)


def test_duhamel_in_the_cosine_basis_is_the_same_sum():
    """duhamel_modes takes the sum of Eq. 36 mode by mode (the transform is
    linear): it must reproduce the term-by-term `duhamel` with leakage
    feedback and the conductivity factor on, up to rounding."""
    w, pd, pl, s = _c1_inputs(16, sigma=0.08)
    st, phy = w.stack, w.physics
    dt = 1e-3
    spectra = [so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                                st.heat_cap_J_m2K, j * dt) for j in range(1, 13)]
    rng = np.random.default_rng(5)
    trace = pd[None] * (0.5 + rng.random((12, 1, 1)))
    a = so.duhamel(spectra, trace, pl, s, phy.beta_per_K, phy.alpha_per_K)
    b = so.duhamel_modes(spectra, trace, pl, s, phy.beta_per_K, phy.alpha_per_K)
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))


# -------------------------------- P9c: piecewise-linear leakage, kappa(T)

def test_pwl_leakage_through_a_line_is_the_linear_model():
    n, L, t, kap, h, pd, pl = _cf_case(sigma=0.2)
    Kt = ph.spectrum(n, L, t, kap, h)
    s = 1.0 - 0.05 * np.random.default_rng(3).random((n, n))
    beta, alpha = 0.0275, 1.2e-3
    apply_L = lambda x: so.spectral_convolve(Kt, x)
    ref, _, _ = so.picard(apply_L, pd, pl, s, beta, alpha, tol=1e-12)
    for pts in ((0.0, 50.0), (-10.0, 3.0, 20.0, 200.0)):       # extrapolation and interior knots
        g = [1.0 + beta * x for x in pts]
        th, _, _ = so.picard_physics(apply_L, pd, pl, s, lambda x: so.leak_pwl(x, pts, g),
                                     lambda v: v / (1.0 - alpha * v), tol=1e-12)
        assert np.allclose(th, ref, rtol=1e-10, atol=1e-12)
    # interpolation on a known polyline
    assert so.leak_pwl(np.array([0.0, 5.0, 10.0, 15.0, 30.0]), (0.0, 10.0, 20.0),
                       (1.0, 2.0, 4.0)).tolist() == [1.0, 1.5, 2.0, 3.0, 6.0]


@pytest.mark.parametrize("eta", [1.3, 0.7, 2.0])
def test_kirchhoff_map_inverts_the_conductivity_integral(eta):
    t_amb = 318.15
    for theta in (0.5, 12.0, 60.0):
        U, _ = integrate.quad(lambda T: (T / t_amb) ** (-eta), t_amb, t_amb + theta,
                              epsabs=1e-13, epsrel=1e-13)
        assert so.kirchhoff_theta(np.array([U]), eta, t_amb)[0] == pytest.approx(theta, rel=1e-11)
    # second order: theta = U + eta U^2 / (2 T_amb) + O(U^3)
    U = 1e-3
    th = so.kirchhoff_theta(np.array([U]), eta, t_amb)[0]
    assert (th - U) / U ** 2 == pytest.approx(eta / (2 * t_amb), rel=1e-4)


def test_kirchhoff_uniform_power_without_leakage_is_the_uniform_mode():
    t, kap, h = STACK3
    n, L = 8, 10e-3
    Kt = ph.spectrum(n, L, t, kap, h)
    q = np.full((n, n), 2e-3)
    z, one = np.zeros((n, n)), np.ones((n, n))
    th, _, _ = so.picard_physics(lambda x: so.spectral_convolve(Kt, x), q, z, one,
                                 lambda x: 1.0, lambda v: so.kirchhoff_theta(v, 1.3, 318.15),
                                 tol=1e-13)
    U = Kt[0, 0] * 2e-3                        # the uniform mode of the imaged kernel
    assert np.allclose(th, 318.15 * ((1 - 0.3 * U / 318.15) ** (-1 / 0.3) - 1), rtol=1e-12)


def test_kirchhoff_fixed_point_residual():
    n, L, t, kap, h, pd, pl = _cf_case(sigma=0.2)
    Kt = ph.spectrum(n, L, t, kap, h)
    s = 1.0 - 0.05 * np.random.default_rng(5).random((n, n))
    pts, g = (0.0, 20.0, 40.0, 80.0), (1.0, 1.5, 2.3, 4.5)
    leak = lambda x: so.leak_pwl(x, pts, g)
    field = lambda v: so.kirchhoff_theta(v, 1.3, 318.15)
    th, u, _ = so.picard_physics(lambda x: so.spectral_convolve(Kt, x), pd, pl, s, leak, field,
                                 tol=1e-13)
    u2 = so.spectral_convolve(Kt, pd + pl * leak(th))
    assert np.max(np.abs(field(s * u2) - th)) <= 1e-11


# ------------------------------------------ P9b: one-shot closed form

def _cf_case(n=8, sigma=0.3, seed=9):
    t, kap, h = STACK3
    L = 10e-3
    rng = np.random.default_rng(seed)
    pd = rng.random((n, n)) * 0.05
    pl = 0.02 * np.exp(sigma * rng.standard_normal((n, n)))
    return n, L, t, kap, h, pd, pl


def test_closed_form_is_exact_without_variation():
    # uniform leakage, alpha = 0: Eq. 21 is the exact fixed point
    n, L, t, kap, h, pd, _ = _cf_case()
    Kt = ph.spectrum(n, L, t, kap, h)
    pl = np.full((n, n), 0.03)
    one = np.ones((n, n))
    ex, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), pd, pl, one, 0.0275, 0.0, tol=1e-13)
    for mode in ("conv", "impulse"):
        assert np.allclose(so.closed_form(Kt, pd, pl, one, 0.0275, 0.0, mode), ex, rtol=1e-10)


def test_closed_form_without_feedback_is_the_image_convolution():
    n, L, t, kap, h, pd, pl = _cf_case()
    Kt = ph.spectrum(n, L, t, kap, h)
    Lm = so.mirror_operator(ph.kernel_periodic(n, L, t, kap, h))
    s = 1.0 - 0.05 * np.random.default_rng(2).random((n, n))
    alpha = 1.2e-3
    u = so.direct_convolve(Lm, pd + pl)
    assert np.allclose(so.closed_form(Kt, pd, pl, s, 0.0, alpha), s * u / (1 - alpha * s * u),
                       rtol=1e-10)


def test_closed_form_random_part_by_dense_image_operators():
    # u = L_det (P_dyn + P_leak0) + P_var * (beta L_det L_det (P_dyn + P_leak0)) with
    # L_det = (I - beta mu L)^-1 L built from the dense mirror-image matrix
    n, L, t, kap, h, pd, pl = _cf_case()
    Kt = ph.spectrum(n, L, t, kap, h)
    Lm = so.mirror_operator(ph.kernel_periodic(n, L, t, kap, h))
    beta, mu = 0.0275, float(np.mean(pl))
    Ld = np.linalg.solve(np.eye(n * n) - beta * mu * Lm, Lm)
    q = (pd + pl).ravel()
    u = Ld @ q + (pl - mu).ravel() * (beta * (Ld @ (Ld @ q)))
    one = np.ones((n, n))
    assert np.allclose(so.closed_form(Kt, pd, pl, one, beta, 0.0), u.reshape(n, n), rtol=1e-9)


def test_closed_form_impulse_mode_is_exact_for_a_centred_impulse():
    # the paper's scaling by the total power is exact when the source is one
    # impulse at the centre
    n, L, t, kap, h, _, pl = _cf_case()
    Kt = ph.spectrum(n, L, t, kap, h)
    src = np.zeros((n, n))
    src[n // 2, n // 2] = 0.7
    pd = src - pl
    one = np.ones((n, n))
    a = so.closed_form(Kt, pd, pl, one, 0.0275, 1e-3, "conv")
    b = so.closed_form(Kt, pd, pl, one, 0.0275, 1e-3, "impulse")
    assert np.allclose(a, b, rtol=1e-12)


def test_closed_form_error_is_first_order_in_the_variation():
    # the Hadamard step is exact at zero variation and its error grows
    # linearly with the variation's amplitude
    n, L, t, kap, h, pd, _ = _cf_case()
    Kt = ph.spectrum(n, L, t, kap, h)
    v = np.random.default_rng(4).standard_normal((n, n))
    v -= v.mean()
    one = np.ones((n, n))
    errs = []
    for eps in (4e-3, 2e-3, 1e-3):
        pl = 0.03 + eps * v
        ex, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), pd, pl, one, 0.0275, 0.0,
                             tol=1e-14)
        errs.append(np.max(np.abs(so.closed_form(Kt, pd, pl, one, 0.0275, 0.0) - ex)))
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


# ------------------------------------ P10b: windowed / implicit transient

@functools.lru_cache(maxsize=None)
def _tr_spectra(n, steps, C, dt):
    t, kap, h = STACK3
    L = 10e-3
    spectra = [so.step_spectrum(n, L, t, kap, h, C, j * dt) for j in range(1, steps + 1)]
    return spectra, ph.spectrum(n, L, t, kap, h)


def _tr_setup(n=8, steps=12, C=1.63e6 * 0.5e-3, dt=1e-3, seed=3):
    spectra, Kt = _tr_spectra(n, steps, C, dt)
    rng = np.random.default_rng(seed)
    trace = rng.random((steps, n, n)) * 0.01
    return n, 10e-3, spectra, Kt, trace


def test_window_zero_or_longer_than_trace_is_the_untruncated_sum():
    n, L, spectra, Kt, trace = _tr_setup()
    rng = np.random.default_rng(4)
    pl, s = rng.random((n, n)) * 2e-3, 1.0 - 0.05 * rng.random((n, n))
    ref = so.duhamel(spectra, trace, pl, s, 0.0275, 1e-3)
    for K in (0, trace.shape[0] + 1):
        th, it = so.transient_variants(spectra, Kt, trace, pl, s, 0.0275, 1e-3, window=K)
        assert np.allclose(th, ref, rtol=1e-13, atol=0.0)
        assert np.all(it == 1)


def test_window_one_is_the_quasi_static_image_convolution():
    # every response settled: theta_n = mirror-image convolution of P_n (no
    # feedback), checked against the dense image operator
    t, kap, h = STACK3
    n, L, spectra, Kt, trace = _tr_setup()
    z, one = np.zeros((n, n)), np.ones((n, n))
    th, _ = so.transient_variants(spectra, Kt, trace, z, one, 0.0, 0.0, window=1)
    Lm = so.mirror_operator(ph.kernel_periodic(n, L, t, kap, h))
    for k in range(trace.shape[0]):
        assert np.allclose(th[k], so.direct_convolve(Lm, trace[k]), rtol=1e-10)


@pytest.mark.parametrize("K", [2, 3, 5])
def test_window_constant_power_jumps_to_steady_at_age_K(K):
    n, L, spectra, Kt, trace = _tr_setup()
    c = np.repeat(trace[:1], trace.shape[0], axis=0)
    z, one = np.zeros((n, n)), np.ones((n, n))
    th, _ = so.transient_variants(spectra, Kt, c, z, one, 0.0, 0.0, window=K)
    for k in range(trace.shape[0]):
        S = spectra[k] if k + 1 < K else Kt          # step n = k + 1 sees S_n, or S_inf
        assert np.allclose(th[k], so.spectral_convolve(S, c[0]), rtol=1e-12)


@pytest.mark.parametrize("K", [2, 5])
def test_window_telescopes_to_the_last_K_differences_plus_settled_power(K):
    # Sec. IV-E: with S_j = S_inf for j >= K the old differences sum to one power,
    # u_n = sum_{j<K} S_j * (P_{n-j+1} - P_{n-j}) + S_inf * P_{n-K+1}
    n, L, spectra, Kt, trace = _tr_setup()
    z, one = np.zeros((n, n)), np.ones((n, n))
    th, _ = so.transient_variants(spectra, Kt, trace, z, one, 0.0, 0.0, window=K)
    P = lambda m: trace[m - 1] if m >= 1 else np.zeros((n, n))    # 1-based, P_0 = 0
    for nn_ in range(1, trace.shape[0] + 1):
        u = sum(so.spectral_convolve(spectra[j - 1], P(nn_ - j + 1) - P(nn_ - j))
                for j in range(1, min(K, nn_ + 1)))
        if nn_ - K + 1 >= 1:
            u = u + so.spectral_convolve(Kt, P(nn_ - K + 1))
        assert np.allclose(th[nn_ - 1], u, rtol=1e-11, atol=1e-15)


def test_window_error_shrinks_with_the_window():
    n, L, spectra, Kt, trace = _tr_setup(steps=16)
    z, one = np.zeros((n, n)), np.ones((n, n))
    ref, _ = so.transient_variants(spectra, Kt, trace, z, one, 0.0, 0.0)
    errs = [np.max(np.abs(so.transient_variants(spectra, Kt, trace, z, one, 0.0, 0.0,
                                                window=K)[0] - ref)) for K in (2, 4, 8, 16)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[0] > 0.0


def test_implicit_without_leakage_feedback_equals_lagged():
    n, L, spectra, Kt, trace = _tr_setup()
    rng = np.random.default_rng(6)
    pl, s = rng.random((n, n)) * 2e-3, 1.0 - 0.05 * rng.random((n, n))
    for K in (0, 3):
        a, _ = so.transient_variants(spectra, Kt, trace, pl, s, 0.0, 1e-3, window=K)
        b, it = so.transient_variants(spectra, Kt, trace, pl, s, 0.0, 1e-3, window=K,
                                      implicit=True, tol=1e-13)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-15)
        assert np.all(it <= 2)


def test_implicit_steps_are_leakage_fixed_points():
    # each step's theta_n reproduces itself through P_n(theta_n) and the
    # superposition of the stored powers, within the iteration tolerance
    n, L, spectra, Kt, trace = _tr_setup()
    rng = np.random.default_rng(7)
    pl, s = 0.02 + rng.random((n, n)) * 0.02, 1.0 - 0.05 * rng.random((n, n))
    beta, alpha, tol = 0.0275, 1.2e-3, 1e-11
    th, it = so.transient_variants(spectra, Kt, trace, pl, s, beta, alpha, implicit=True, tol=tol)
    assert np.all(it >= 3)
    Ps = [trace[k] + pl * (1.0 + beta * th[k]) for k in range(trace.shape[0])]
    for k in range(trace.shape[0]):
        u = sum(so.spectral_convolve(spectra[j - 1], Ps[k - j + 1] - (Ps[k - j] if k - j >= 0 else 0.0))
                for j in range(1, k + 2))
        assert np.max(np.abs(so.phi(u, s, alpha) - th[k])) <= 100 * tol
    # lagged leakage trails the implicit one while the temperature rises
    lag, _ = so.transient_variants(spectra, Kt, trace, pl, s, beta, alpha)
    assert np.all(th[1:] >= lag[1:] - 1e-12) and np.max(th - lag) > 0.0


@pytest.mark.parametrize("K", [0, 4])
def test_implicit_constant_power_reaches_steady_fixed_point(K):
    w, pd, pl, s = _c1_inputs(8, sigma=0.08)
    st, phy = w.stack, w.physics
    C, dt, steps = 20.0, 1e-3, 40          # tau ~ 1 ms: settled well within 40 steps
    spectra = [so.step_spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                                C, j * dt) for j in range(1, (K or steps + 1))]
    Kt = ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    trace = np.repeat(pd[None], steps, axis=0)
    th, _ = so.transient_variants(spectra, Kt, trace, pl, s, phy.beta_per_K, phy.alpha_per_K,
                                  window=K, implicit=True, tol=1e-13)
    ss, _, _ = so.picard(lambda x: so.spectral_convolve(Kt, x), pd, pl, s,
                         phy.beta_per_K, phy.alpha_per_K, tol=1e-12)
    assert np.max(np.abs(th[-1] - ss)) <= 1e-6


# -------------------------------------------------- golden chip parameters

def test_defaults_follow_paper_chip_parameter_table():
    g = json.load(open(os.path.join(HERE, "golden", "chip_params.json")))
    st, phy = synth.Stack(), synth.Physics()
    assert phy.beta_per_K == g["beta_per_K"]
    assert phy.t_amb_K == g["ambient_K"]
    assert st.kappa_W_mK == (g["si_conductivity_W_mK"], g["tim_conductivity_W_mK"],
                             g["spreader_conductivity_W_mK"])
    assert st.thickness_m[1:] == (g["tim_thickness_mm"] * 1e-3, g["spreader_thickness_mm"] * 1e-3)


# ------------------------------------------- warm-start network reference

def test_cnn_oracle_gradient_matches_finite_differences():
    from oracle import cnn
    rng = np.random.default_rng(4)
    C, R, B = 2, 8, 2
    p = rng.normal(0, 0.4, cnn.n_params(C))
    x = rng.normal(0, 1, (B, 3, R, R))
    t = rng.normal(0, 1, (B, 1, R, R))
    loss, g = cnn.loss_and_grad(p, C, x, t)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp = np.mean((cnn.forward(p + e, C, x) - t) ** 2)
        lm = np.mean((cnn.forward(p - e, C, x) - t) ** 2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert loss == pytest.approx(np.mean((cnn.forward(p, C, x) - t) ** 2), rel=1e-14)


# ------------------------------------------- transient uniform mode (1024^2 fixture)

def test_uniform_mode_depends_on_cell_size_not_on_die_size():
    # The (0,0) cosine mode of the mirror-imaged kernel is the sum of the kernel
    # over the whole image lattice, so for a fixed cell it is the same for any
    # number of cells; this lets the 1024^2 transient be checked at any step
    # from uniform-mode values computed on a small die with the same cell.
    st = synth.workload("c4_1024").stack
    cell = 20e-3 / 1024
    args = (st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)
    assert ph.spectrum(32, 32 * cell, *args)[0, 0] == pytest.approx(
        ph.spectrum(16, 16 * cell, *args)[0, 0], rel=1e-12)
    for t_s in (1e-3, 40e-3):
        a = so.step_spectrum(16, 16 * cell, *args, st.heat_cap_J_m2K, t_s)[0, 0]
        b = so.step_spectrum(32, 32 * cell, *args, st.heat_cap_J_m2K, t_s)[0, 0]
        assert a == pytest.approx(b, rel=1e-12)


def test_transient_uniform_mode_fixture_is_current():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_transient_mode00", os.path.join(HERE, "golden", "make_transient_mode00.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    d = json.load(open(os.path.join(HERE, "golden", "transient_mode00_c4_1024.json")))
    assert len(d["S00"]) == mk.STEPS and d["dt_s"] == mk.DT_S
    for j in (1, 137):
        assert d["S00"][j - 1] == pytest.approx(mk.mode00(j), rel=1e-12)
    # the step response rises monotonically towards the steady uniform mode
    s = np.array(d["S00"])
    assert np.all(np.diff(s) > 0)


# ------------------------------------- input recipe: spherical correlation

def test_spherical_variation_fields_follow_the_spherical_correlation():
    # Sec. II-C: systematic variation with a spherical correlation of range phi.
    # Empirical correlation along x over many fields against
    # 1 - 1.5 r/phi + 0.5 (r/phi)^3 (0 beyond phi); standardised fields.
    w = synth.workload("c1_64")
    w.corr = "spherical"
    phi = 2.5e-3
    w.corr_len_m = (phi, phi)
    z, _ = synth.variation_fields(w, 256, dtype=torch.float64)
    z = z.numpy()
    c = w.cell_m
    for lag in (2, 6, 12, 20):
        r = lag * c
        a, b = z[:, 8:56, 8:56 - lag], z[:, 8:56, 8 + lag:56]
        emp = float(np.mean(a * b) / np.sqrt(np.mean(a * a) * np.mean(b * b)))
        x = min(r / phi, 1.0)
        ref = 1 - 1.5 * x + 0.5 * x ** 3
        assert emp == pytest.approx(ref, abs=0.06), (lag, emp, ref)
