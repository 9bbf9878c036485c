"""The error-estimate stopping rule (vs_solve_params.stop_rule =
VS_STOP_ESTIMATE) on the oracle: pinned on exactly geometric update sequences,
whose errors are known in closed form, then checked on the workloads' maps
against the converged fixed point."""
import numpy as np
import pytest

import synth
from oracle import solve as so

from _util import oracle_spectrum


def _stop_at(rule, r1, rho, tol):
    rs = []
    for n in range(1, 400):
        rs.append(r1 * rho ** (n - 1))
        if so.stop_test(rs, tol, rule):
            return n
    raise AssertionError("no stop")


@pytest.mark.parametrize("rho", [1e-3, 0.01, 0.1, 0.3, 0.45, 0.6, 0.9])
@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_estimate_rule_on_geometric_updates(rho, tol):
    """Updates r_n = r_1 rho^(n-1): the error of iterate n is the tail
    sum_{j > n} r_j = r_n rho / (1 - rho). The estimate rule stops with that
    error <= tol for every rate up to its cap (0.9); below rho = 1/8 its
    estimate is under the update itself, so it stops no later than the update
    rule, and above it later."""
    r1 = 40.0
    err = lambda n: r1 * rho ** (n - 1) * rho / (1.0 - rho)
    n_est, n_upd = _stop_at("estimate", r1, rho, tol), _stop_at("update", r1, rho, tol)
    assert err(n_est) <= tol
    if rho < 0.125:
        assert n_est <= n_upd
    else:
        assert n_est >= n_upd


def test_update_rule_misses_slow_contractions():
    """The reason for the estimate rule at large rates: at rho = 0.9 the update
    rule stops with an error 9x its tolerance."""
    r1, rho, tol = 40.0, 0.9, 1e-2
    n = _stop_at("update", r1, rho, tol)
    assert r1 * rho ** (n - 1) * rho / (1 - rho) > 5 * tol


def _maps(name, count):
    if name == "c1_64":
        w = synth.workload("c1_64")
        pd, pl, s = synth.steady_inputs(w, count, device="cpu")
    else:
        w, pd, pl, s = synth.batch_inputs(256, count, device="cpu")
    f64 = lambda t: t.double().numpy()
    return w, oracle_spectrum(w), [(f64(pd[i]), f64(pl[i]), f64(s[i])) for i in range(count)]


@pytest.mark.parametrize("name,count", [("c1_64", 8), ("c2_256", 4)])
def test_engine_iteration_with_both_rules(name, count):
    """The engines' iteration (uniform start, preconditioner) reaches the fixed
    point of the plain Picard iteration; stopped by the estimate rule it is
    within tol of that fixed point at 1e-2 K and 1e-4 K, in fewer iterations
    than the update rule on average."""
    w, Kt, maps = _maps(name, count)
    beta, alpha = w.physics.beta_per_K, w.physics.alpha_per_K
    L = lambda x: so.spectral_convolve(Kt, x)
    its = {"update": [], "estimate": []}
    for pd, pl, s in maps:
        ref, _, _ = so.picard(L, pd, pl, s, beta, alpha, tol=1e-11)
        tight, _, _ = so.picard_uniform_start(Kt, pd, pl, s, beta, alpha, 1e-11)
        assert np.max(np.abs(tight - ref)) <= 1e-9
        for tol in (1e-2, 1e-4):
            for rule in ("update", "estimate"):
                th, n, rs = so.picard_uniform_start(Kt, pd, pl, s, beta, alpha, tol, stop=rule)
                assert np.max(np.abs(th - ref)) <= tol, (rule, tol, n, rs)
                its[rule].append(n)
    print(name, "mean iterations: update %.2f, estimate %.2f"
          % (np.mean(its["update"]), np.mean(its["estimate"])))
    assert np.mean(its["estimate"]) < np.mean(its["update"])
