"""Oracle solvers: mirror-image convolution, leakage/conductivity fixed point,
transient superposition.

Test infrastructure only (see the package docstring). FP64 throughout.

Model of the self-consistent temperature (this project's reading of
Eqs. 4-5, 9-12 and 13-16, generalised from a unit impulse to a power map):

* power P = P_dyn + P_leak0 (1 + beta theta)       (Eq. 13, Eq. 5)
* u = L[P], L = convolution with the imaged kernel (Eq. 2, Sec. IV-F)
* the Green's function is scaled at the field point by s (1 + alpha theta)
  (Eqs. 11-12; s carries the conductivity variation), so theta = s u (1 + alpha
  theta), i.e. theta = phi(u) = s u / (1 - alpha s u)
* the fixed point u = L[P_dyn + P_leak0 (1 + beta phi(u))] is what the
  paper's validation loop reaches by iterating power -> temperature ->
  leakage/conductivity until convergence (Sec. V-C).
"""
from __future__ import annotations

import numpy as np

from . import physics


# --------------------------------------------------------------------------- #
# Mirror-image convolution                                                      #
# --------------------------------------------------------------------------- #

def mirror_operator(kper: np.ndarray) -> np.ndarray:
    """Dense matrix of the mirror-image convolution on an n x n grid (n <= 64).

    The power map is extended to twice its size with even mirror images at the
    die edges (Sec. IV-F) and convolved circularly with the 2n-periodic kernel
    K_per; restricted to the die this is, for target i and source j,
      L_ij = sum over (ex, ey) in {i-j, i+j+1} of K_per(ey mod 2n, ex mod 2n)
    (four terms per pair). Row/column index = y*n + x.
    """
    n2 = kper.shape[0]
    n = n2 // 2
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    iy = iy.ravel()
    ix = ix.ravel()
    dy_m = (iy[:, None] - iy[None, :]) % n2
    dy_p = (iy[:, None] + iy[None, :] + 1) % n2
    dx_m = (ix[:, None] - ix[None, :]) % n2
    dx_p = (ix[:, None] + ix[None, :] + 1) % n2
    return (kper[dy_m, dx_m] + kper[dy_m, dx_p] + kper[dy_p, dx_m] + kper[dy_p, dx_p])


def direct_convolve(L: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Apply the dense mirror operator to maps q[..., n, n]."""
    n = q.shape[-1]
    flat = q.reshape(-1, n * n)
    return (flat @ L.T).reshape(q.shape)


def dct_matrix(n: int) -> np.ndarray:
    """C[p, j] = cos(pi p (2j + 1) / (2n)) (unnormalised DCT-II)."""
    p = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return np.cos(np.pi * p * (2 * j + 1) / (2 * n))


def idct_matrix(n: int) -> np.ndarray:
    """Exact inverse of dct_matrix: x_j = (1/n)[X_0 + 2 sum_{p>0} X_p C[p, j]]."""
    w = np.full(n, 2.0)
    w[0] = 1.0
    return (dct_matrix(n) * w[:, None]).T / n


def spectral_convolve(Kt: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Same operator in the cosine basis: L[q] = IDCT2(DCT2(q) * K~). The even
    extension of the map is what a DCT-II encodes, so the circular convolution
    of the mirrored map with K_per is diagonal in it (symmetric convolution
    theorem); dense cosine matrices, no fast transform."""
    n = q.shape[-1]
    C = dct_matrix(n)
    Ci = idct_matrix(n)
    X = C @ q @ C.T
    return Ci @ (X * Kt) @ Ci.T


# --------------------------------------------------------------------------- #
# Fixed point                                                                   #
# --------------------------------------------------------------------------- #

class SolveError(RuntimeError):
    pass


def phi(u, s, alpha):
    """theta = s u / (1 - alpha s u) (field-point factor, Eq. 12)."""
    return s * u / (1.0 - alpha * s * u)


def picard(apply_L, p_dyn, p_leak0, s, beta, alpha, tol=1e-8, max_iter=400,
           guard=0.05):
    """Plain Picard iteration on the unsplit fixed point from u = 0:
    u_{n+1} = L[P_dyn + P_leak0 (1 + beta phi(u_n))], stop when
    max |phi(u_{n+1}) - phi(u_n)| <= tol (the update-norm reading of the
    validation loop of Sec. V-C, which iterates until the temperatures settle).
    Raises if 1 - alpha s u <= guard (conductivity runaway) or max_iter is hit.
    Returns (theta, u, iterations)."""
    u = np.zeros_like(p_dyn)
    theta = np.zeros_like(p_dyn)
    for it in range(1, max_iter + 1):
        u = apply_L(p_dyn + p_leak0 * (1.0 + beta * theta))
        den = 1.0 - alpha * s * u
        if np.min(den) <= guard:
            raise SolveError("conductivity runaway: 1 - alpha s u <= %g" % guard)
        new = s * u / den
        if not np.all(np.isfinite(new)):
            raise SolveError("non-finite temperature")
        d = np.max(np.abs(new - theta))
        theta = new
        if d <= tol:
            return theta, u, it
    raise SolveError("no convergence in %d iterations" % max_iter)


def picard_split(Kt, p_dyn, p_leak0, s, beta, alpha, tol=1e-8, max_iter=400):
    """The mean/variation split of Sec. IV-C used as a preconditioner.

    mu = mean(P_leak0), P_leak0 = mu + P_var. The shift-invariant part has the
    modified kernel K_det = K~ / (1 - beta mu K~) (Eq. 21 with alpha = 0); the
    remaining shift-variant source is iterated:
      u_det = L_det[P_dyn + mu],
      c_{n+1} = L_det[P_var + beta (P_leak0 phi(u_det + c_n) - mu (u_det + c_n))].
    Since L_det = (I - beta mu L)^-1 L this has the same fixed point as
    `picard`. Spectral (dense cosine) operators. Returns (theta, u, iters)."""
    mu = float(np.mean(p_leak0))
    Kd = Kt / (1.0 - beta * mu * Kt)
    udet = spectral_convolve(Kd, p_dyn + mu)
    c = np.zeros_like(udet)
    theta = np.zeros_like(udet)
    for it in range(1, max_iter + 1):
        u = udet + c
        new = phi(u, s, alpha)
        d = np.max(np.abs(new - theta))
        theta = new
        if d <= tol and it > 1:
            return theta, u, it
        c = spectral_convolve(Kd, (p_leak0 - mu) + beta * (p_leak0 * theta - mu * u))
    raise SolveError("no convergence")


def picard_uniform_start(Kt, p_dyn, p_leak0, s, beta, alpha, tol, stop="update",
                         max_iter=100, guard=0.05):
    """The preconditioned iteration of the GPU engines, in FP64, with both
    stopping rules (a reading of this project: the paper iterates until the
    temperatures settle, Sec. V-C, and states no rule).

    Start: the die's uniform mode, the scalar fixed point
      u_bar = K00 (mean P_dyn + mu (1 + beta theta_bar)), theta_bar = u_bar / (1 - alpha u_bar),
    K00 the kernel's response to a uniform unit source; every cell starts at
    theta_bar (u_0 = phi^-1(theta_bar) = theta_bar / (s (1 + alpha theta_bar))).
    Preconditioner b = beta mu (1 + 2 alpha u_bar) (about the mean of
    beta P_leak0 dtheta/du), the mean/variation split of Sec. IV-C with the
    multiplier K~ / (1 - b K~) of Eq. 21:
      u_{n+1} = L_b[P_dyn + P_leak0 (1 + beta theta_n) - b u_n],  theta = phi(u),
    which has the fixed point of `picard` for every b.
    Stopping, with r_n = max |theta_n - theta_{n-1}|:
      "update":   r_n <= tol;
      "estimate": from n = 2 on, the a-posteriori error estimate of a
                  contraction, r_n q / (1 - q) <= tol with q = min(0.9,
                  4 r_n / r_{n-1}) (the factor seen over the last two updates,
                  times a safety factor 4); n = 1 uses the update rule.
    Returns (theta, iterations, updates)."""
    n = p_dyn.shape[0]
    mu = float(np.mean(p_leak0))
    k00 = float(spectral_convolve(Kt, np.ones_like(p_dyn))[0, 0])
    ub = 0.0
    for _ in range(200):
        ub_new = k00 * (float(np.mean(p_dyn)) + mu * (1.0 + beta * ub / (1.0 - alpha * ub)))
        if abs(ub_new - ub) <= 1e-14 * max(1.0, abs(ub_new)):
            ub = ub_new
            break
        ub = ub_new
    b = beta * mu * (1.0 + 2.0 * alpha * ub)
    Kb = Kt / (1.0 - b * Kt)
    th0 = ub / (1.0 - alpha * ub)
    theta = np.full((n, n), th0)
    u = th0 / (s * (1.0 + alpha * th0))        # phi(u) = theta_bar at every cell
    rs = []
    for it in range(1, max_iter + 1):
        u = spectral_convolve(Kb, p_dyn + p_leak0 * (1.0 + beta * theta) - b * u)
        den = 1.0 - alpha * s * u
        if np.min(den) <= guard:
            raise SolveError("conductivity runaway: 1 - alpha s u <= %g" % guard)
        new = s * u / den
        r = float(np.max(np.abs(new - theta)))
        theta = new
        rs.append(r)
        if stop_test(rs, tol, stop):
            return theta, it, rs
    raise SolveError("no convergence in %d iterations" % max_iter)


def stop_test(updates, tol, stop="update"):
    """Stopping rule after the iterate whose update is updates[-1] (the
    updates r_1 .. r_n so far, r = max |theta_n - theta_{n-1}|).
    "update": r_n <= tol. "estimate": for n >= 2, the error of a contraction
    with factor q after iterate n is at most r_n q / (1 - q) (the tail of the
    geometric series of the following updates); q is estimated as
    min(0.9, 4 r_n / r_{n-1}); stop when that estimate is <= tol."""
    r = updates[-1]
    if stop == "estimate" and len(updates) > 1:
        q = min(0.9, 4.0 * r / updates[-2])
        return r * q <= tol * (1.0 - q)
    return r <= tol


def shift_invariant(Kt, p_dyn, p_leak0, beta):
    """Closed form for a uniform leakage map (no variation, alpha = 0):
    u = IDCT(DCT(P_dyn + mu) K~ / (1 - beta mu K~)) (Eq. 21 with alpha = 0)."""
    mu = float(np.mean(p_leak0))
    return spectral_convolve(Kt / (1.0 - beta * mu * Kt), p_dyn + mu)


# --------------------------------------------------------------------------- #
# Richer physics: piecewise-linear leakage (Sec. II-E), kappa(T) (Eq. 10)         #
# --------------------------------------------------------------------------- #

def leak_pwl(theta, pts_theta, pts_g):
    """Piecewise-linear leakage factor g(theta), P_leak = P_leak0 g(theta)
    (the piecewise-linear leakage model Sec. II-E names for accuracy): linear
    interpolation through (pts_theta[i], pts_g[i]), pts_theta increasing, and
    the first / last segment extended beyond the table."""
    x = np.asarray(pts_theta, dtype=np.float64)
    y = np.asarray(pts_g, dtype=np.float64)
    i = np.clip(np.searchsorted(x, theta, side="right") - 1, 0, len(x) - 2)
    return y[i] + (y[i + 1] - y[i]) / (x[i + 1] - x[i]) * (theta - x[i])


def kirchhoff_theta(U, eta, t_amb, guard=0.05):
    """Temperature rise from the Kirchhoff variable U when the conductivity
    follows Eq. 10 with the reference at ambient, kappa = kappa_amb (T/T_amb)^-eta:
      U = int_{T_amb}^{T} (T'/T_amb)^-eta dT' = T_amb ((T/T_amb)^(1-eta) - 1) / (1 - eta),
    inverted: theta = T - T_amb = T_amb ((1 + (1 - eta) U / T_amb)^(1/(1-eta)) - 1).
    Raises where the base 1 + (1 - eta) U / T_amb is <= guard (the
    conductivity model breaks down)."""
    base = 1.0 + (1.0 - eta) * U / t_amb
    if np.min(base) <= guard:
        raise SolveError("conductivity runaway: Kirchhoff base <= %g" % guard)
    return t_amb * (base ** (1.0 / (1.0 - eta)) - 1.0)


def picard_physics(apply_L, p_dyn, p_leak0, s, leak, field, tol=1e-8, max_iter=400):
    """Plain Picard on the fixed point with a general leakage factor and
    field-point map, from u = 0:
      u_{n+1} = L[P_dyn + P_leak0 leak(theta_n)],  theta = field(s u)
    (leak(theta) = 1 + beta theta and field(v) = v / (1 - alpha v) give
    `picard`). Stops when max |theta_{n+1} - theta_n| <= tol.
    Returns (theta, u, iterations)."""
    theta = np.zeros_like(p_dyn)
    for it in range(1, max_iter + 1):
        u = apply_L(p_dyn + p_leak0 * leak(theta))
        new = field(s * u)
        if not np.all(np.isfinite(new)):
            raise SolveError("non-finite temperature")
        d = np.max(np.abs(new - theta))
        theta = new
        if d <= tol:
            return theta, u, it
    raise SolveError("no convergence in %d iterations" % max_iter)


# --------------------------------------------------------------------------- #
# One-shot closed form (Sec. IV-C, Eqs. 21, 25, 26)                             #
# --------------------------------------------------------------------------- #

def closed_form(Kt, p_dyn, p_leak0, s, beta, alpha, mode="conv"):
    """The paper's one-shot modified Green's functions combined by convolution
    and Hadamard product, instead of the iterated fixed point.

    Readings (the paper's Lemma I and F(mu) terms are not computable as printed):
    * deterministic part, Eq. 21 without its alpha term (F(mu) of a constant is
      a delta; alpha acts through phi at the field point as in the fixed point):
      L_det = K~ / (1 - beta mu K~), applied to the whole source P_dyn + P_leak0
      (a convolution, exact for the mean and for the variation's own heat);
    * random part, Eq. 25 to first order in the variation (the Q term of its
      denominator dropped, as the paper drops term V): per unit of variation
      the response is beta L_det^2 applied to the source;
    * Eq. 26: that response times the local variation P_leak0 - mu (Hadamard
      product). mode "conv" applies it to the actual power map; mode "impulse"
      takes the paper's form literally: the response to a unit impulse at the
      die's centre cell (n/2, n/2), scaled by the total power of the map.
    theta = phi(u_det + (P_leak0 - mu) * r, s, alpha)."""
    n = p_dyn.shape[-1]
    mu = float(np.mean(p_leak0))
    Ld = Kt / (1.0 - beta * mu * Kt)
    q = p_dyn + p_leak0
    u_det = spectral_convolve(Ld, q)
    if mode == "conv":
        r = spectral_convolve(beta * Ld * Ld, q)
    elif mode == "impulse":
        e = np.zeros((n, n))
        e[n // 2, n // 2] = 1.0
        r = spectral_convolve(beta * Ld * Ld, e) * float(np.sum(q))
    else:
        raise ValueError(mode)
    return phi(u_det + (p_leak0 - mu) * r, s, alpha)


# --------------------------------------------------------------------------- #
# Transient (Eqs. 27-37)                                                        #
# --------------------------------------------------------------------------- #

def step_spectrum(n, die_m, t, kappa, h, heat_cap, t_s, rel=1e-18, spreader=None):
    """Spectrum of the step-response Green's function at time t_s:
    single pole per spatial frequency with tau(k) = C g^(k) (Eq. 35 with the
    alpha term of tau dropped; C = areal heat capacity), so the response to a
    unit power step is g^(k) (1 - exp(-t / (C g^(k)))) (Eq. 35).

    Same real/spectral split as physics.spectrum: the top-layer part is static
    (the exp factor of the aliases with large k vanishes), the spectral part
    is R(k) - g^(k) exp(-t/(C g^(k))), which decays exponentially in k for t > 0.

    spreader = (first, side_m): a spreader wider than the die changes the
    uniform mode only (physics.ghat0_wide): its step response is
    g^0_wide (1 - exp(-t / (C g^0_wide))).
    """
    import math
    t = tuple(float(x) for x in t)
    kappa = tuple(float(x) for x in kappa)
    cell = die_m / n
    a = physics.disc_radius(cell)
    R = int(math.ceil(physics.real_space_cutoff(t[0], rel) / cell))
    m = np.arange(-R, R + 1)
    rad2 = m[:, None] ** 2 + m[None, :] ** 2
    uniq, inv = np.unique(rad2, return_inverse=True)
    g1 = physics.g_top_radial(cell * np.sqrt(uniq.astype(np.float64)), t[0], kappa[0], a)
    G = g1[inv].reshape(rad2.shape)
    p = np.arange(n)
    C = np.cos(np.pi * np.outer(p, m) / n)
    K1 = C @ G @ C.T
    rate = t_s * kappa[0] / heat_cap                    # large-k decay length of exp term
    dec = min(2 * t[0], rate)
    S = int(math.ceil((cell * math.log(1.0 / rel) / (math.pi * dec) + 1) / 2)) + 1
    KR = np.zeros((n, n))
    for s_ in range(-S, S + 1):
        ky = np.pi * (p + 2 * n * s_) / die_m
        for t_ in range(-S, S + 1):
            kx = np.pi * (p + 2 * n * t_) / die_m
            kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
            g = physics.ghat(kk, t, kappa, h)
            KR += (physics.ghat_rest(kk, t, kappa, h)
                   - g * np.exp(-t_s / (heat_cap * g))) * physics._disc_factor(kk * a)
    S_ = K1 + KR / cell ** 2
    if spreader is not None:
        # primary uniform term g (1 - e^{-t/(C g)}) with g^0_wide for g^(0)
        g0 = float(physics.ghat(np.array([0.0]), t, kappa, h)[0])
        gw = physics.ghat0_wide(t, kappa, h, spreader[0], die_m, spreader[1])
        S_[0, 0] += (gw * (1.0 - math.exp(-t_s / (heat_cap * gw)))
                     - g0 * (1.0 - math.exp(-t_s / (heat_cap * g0)))) / cell ** 2
    return S_


def duhamel(step_spectra, p_dyn_trace, p_leak0, s, beta, alpha):
    """Untruncated superposition of power differences (Eq. 36):
      u_n = sum_{j=1..n} S_j * (P_{n-j+1} - P_{n-j}),  P_0 = 0,
    with leakage lagged one step, P_m = P_dyn,m + P_leak0 (1 + beta theta_{m-1}),
    theta_0 = 0, and theta_n = phi(u_n). step_spectra[j-1] is S_j in the
    cosine basis. Returns theta[n_steps, n, n]."""
    n_steps = p_dyn_trace.shape[0]
    theta = np.zeros_like(p_dyn_trace)
    P = []
    th_prev = np.zeros_like(p_leak0)
    for k in range(n_steps):
        P.append(p_dyn_trace[k] + p_leak0 * (1.0 + beta * th_prev))
        u = np.zeros_like(p_leak0)
        for j in range(1, k + 2):
            m = k + 1 - j                        # P index (0-based) of P_{n-j+1}
            dP = P[m] - (P[m - 1] if m >= 1 else 0.0)
            u = u + spectral_convolve(step_spectra[j - 1], dP)
        th_prev = phi(u, s, alpha)
        theta[k] = th_prev
    return theta


def duhamel_modes(step_spectra, p_dyn_trace, p_leak0, s, beta, alpha):
    """The same untruncated superposition as `duhamel` (Eq. 36, lagged
    leakage), with the sum over past power differences taken mode by mode in
    the cosine basis: since L_S[q] = IDCT2(DCT2(q) S) is linear in q,
      u_n = IDCT2( sum_{j=1..n} S_j * DCT2(P_{n-j+1} - P_{n-j}) ),
    so every power difference is transformed once and every step needs one
    inverse transform instead of n. Equal to `duhamel` up to rounding; used
    for long traces. Returns theta[n_steps, n, n]."""
    n_steps = p_dyn_trace.shape[0]
    n = p_leak0.shape[-1]
    C = dct_matrix(n)
    Ci = idct_matrix(n)
    theta = np.zeros_like(p_dyn_trace)
    dP_hat = []                                  # DCT2 of P_m - P_{m-1}, m = 1..
    P_prev = np.zeros_like(p_leak0)
    th_prev = np.zeros_like(p_leak0)
    for k in range(n_steps):
        P_k = p_dyn_trace[k] + p_leak0 * (1.0 + beta * th_prev)
        dP_hat.append(C @ (P_k - P_prev) @ C.T)
        P_prev = P_k
        U = np.zeros_like(p_leak0)
        for j in range(1, k + 2):
            U = U + step_spectra[j - 1] * dP_hat[k + 1 - j]
        th_prev = phi(Ci @ U @ Ci.T, s, alpha)
        theta[k] = th_prev
    return theta


def transient_variants(step_spectra, steady_spectrum, p_dyn_trace, p_leak0, s, beta, alpha,
                       window=0, implicit=False, tol=1e-10, max_iter=200):
    """The two variants of the superposition of Sec. IV-E, in the paper's terms.

    * window K >= 1: beyond K steps the step response is taken as saturated,
      S_j = S_inf for every j >= K (Sec. IV-E: five 1 ms steps), and the sum
      of Eq. 36 is taken with those responses; K = 0 keeps every S_j.
    * implicit: the leakage of step n is taken at the temperature of step n
      itself (the leakage-aware step responses the paper substitutes in
      Sec. IV-E make the leakage of a step follow that step's own
      temperature). Each step iterates
          P_n = P_dyn,n + P_leak0 (1 + beta theta),  u_n = Eq. 36 sum,
          theta <- phi(u_n),
      from theta = theta_{n-1} (0 for the first step) until the largest
      change is <= tol. The history keeps the P_n of the last iteration, so
      u_n is exactly the Eq. 36 sum of the stored powers and theta_n = phi(u_n).
      Otherwise the leakage is lagged: P_n = P_dyn,n + P_leak0 (1 + beta
      theta_{n-1}).

    step_spectra[j-1] = S_j in the cosine basis (needed for j < K, or for
    every j when K = 0); steady_spectrum = S_inf = K~. Returns
    (theta[n_steps, n, n], iterations per step)."""
    n_steps = p_dyn_trace.shape[0]
    theta = np.zeros_like(p_dyn_trace)
    iters = np.zeros(n_steps, dtype=np.int64)
    P = []

    def response(j):
        if window and j >= window:
            return steady_spectrum
        return step_spectra[j - 1]

    def u_of(k, Pk):
        # Eq. 36 at step k + 1 (0-based k) with P_{k+1} = Pk
        u = np.zeros_like(p_leak0)
        for j in range(1, k + 2):
            m = k + 1 - j                        # 0-based index of P_{n-j+1}
            cur = Pk if m == k else P[m]
            prev = P[m - 1] if m >= 1 else 0.0
            u = u + spectral_convolve(response(j), cur - prev)
        return u

    th_prev = np.zeros_like(p_leak0)
    for k in range(n_steps):
        if not implicit:
            Pk = p_dyn_trace[k] + p_leak0 * (1.0 + beta * th_prev)
            th = phi(u_of(k, Pk), s, alpha)
            iters[k] = 1
        else:
            th = th_prev
            for it in range(1, max_iter + 1):
                Pk = p_dyn_trace[k] + p_leak0 * (1.0 + beta * th)
                new = phi(u_of(k, Pk), s, alpha)
                d = float(np.max(np.abs(new - th)))
                th = new
                if d <= tol:
                    break
            else:
                raise SolveError("transient step %d did not converge" % k)
            iters[k] = it
        P.append(Pk)
        theta[k] = th
        th_prev = th
    return theta, iters
