"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded FP32 inputs."""
import numpy as np
import torch

import synth
from oracle import physics as ph
from oracle import solve as so

# Tolerances. The requirement is max |dT| <= 0.05 K and rel-L2 <= 1e-4 against
# the FP64 oracle. The FP32 path is expected to do far better: the cosine
# transforms carry ~1e-6 relative rounding (a few 1e-5 K at 30-130 K rises),
# and the fixed point stops at max |dtheta| <= 1e-4 K with contraction
# factor < 0.3, i.e. within ~5e-5 K of the fixed point. ENG_TOL_K states that
# engineering bound with margin.
REQ_MAX_K = 0.05
REQ_REL_L2 = 1e-4
ENG_TOL_K = 2e-3


def vs_stack(w: synth.Workload):
    import paper_2307_12119_gb300 as vs
    st = w.stack
    return vs.Stack(st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K, st.heat_cap_J_m2K)


def vs_params(w: synth.Workload, tol=1e-4, max_iter=50, **kw):
    import paper_2307_12119_gb300 as vs
    p = vs.SolveParams(w.physics.beta_per_K, w.physics.alpha_per_K, tol, max_iter)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def oracle_spectrum(w: synth.Workload):
    st = w.stack
    return ph.spectrum(w.n, w.die_m, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K)


def oracle_steady(w, Kt, pd, pl, s, beta=None, alpha=None, tol=1e-10):
    """Plain Picard (unsplit) with the dense-cosine spectral operator, FP64,
    on the FP32 inputs promoted to FP64."""
    f64 = lambda t: t.detach().double().cpu().numpy()
    b = w.physics.beta_per_K if beta is None else beta
    a = w.physics.alpha_per_K if alpha is None else alpha
    th, _, it = so.picard(lambda x: so.spectral_convolve(Kt, x), f64(pd), f64(pl), f64(s), b, a,
                          tol=tol, max_iter=400)
    return th, it


def errors(gpu, ref):
    g = gpu.detach().double().cpu().numpy()
    d = g - ref
    return float(np.max(np.abs(d))), float(np.linalg.norm(d) / np.linalg.norm(ref))


def inputs(w, count=1, seed=synth.SEED, first=0, n_floorplans=None):
    pd, pl, s = synth.steady_inputs(w, count, seed=seed, first=first, n_floorplans=n_floorplans,
                                    device="cuda")
    return pd, pl, s


def step_spectra(w, dt, steps, workers=None):
    """The oracle's step-response spectra S_1 .. S_steps of workload w
    (Eq. 35 per mode, oracle.solve.step_spectrum), computed in parallel in
    spawned worker processes (a forked child of a process that has used CUDA
    can hang; a spawned one starts clean)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    st = w.stack
    args = [(w.n, w.die_m, tuple(st.thickness_m), tuple(st.kappa_W_mK), st.h_conv_W_m2K,
             st.heat_cap_J_m2K, j * dt) for j in range(1, steps + 1)]
    workers = workers or max(1, min(steps, len(os.sched_getaffinity(0))))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(so.step_spectrum, *a) for a in args]
        return [f.result() for f in futs]
