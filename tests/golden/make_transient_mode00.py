"""Writes transient_mode00_c4_1024.json: the uniform-mode (p = q = 0) entry of
the oracle's step-response spectra S(j dt)[0][0], j = 1..200, for the 1024 x
1024 transient workload (20 x 20 mm die, dt = 1 ms).

Calls only oracle/ (and synth/ for the geometry). The uniform mode of the
mirror-imaged kernel depends on the cell size and the stack, not on the number
of cells, so the spectra are evaluated on a 16 x 16 die with the same cell
(tests/test_oracle_pins.py pins that invariance). The single-pole step response
is Eq. 35 (alpha term of the time constant dropped); the superposition that
uses these values is Eq. 36.

    python tests/golden/make_transient_mode00.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import solve as so  # noqa: E402

WORKLOAD = "c4_1024"
DT_S = 1e-3
STEPS = 200
SMALL_N = 16


def mode00(j: int) -> float:
    w = synth.workload(WORKLOAD)
    st = w.stack
    cell = w.die_m / w.n
    S = so.step_spectrum(SMALL_N, cell * SMALL_N, st.thickness_m, st.kappa_W_mK, st.h_conv_W_m2K,
                         st.heat_cap_J_m2K, j * DT_S)
    return float(S[0, 0])


def main():
    vals = [mode00(j) for j in range(1, STEPS + 1)]
    out = {"workload": WORKLOAD, "dt_s": DT_S, "small_n": SMALL_N,
           "what": "S(j dt)[0][0] for j = 1..%d (K per W per cell), oracle step_spectrum "
                   "(Eq. 35) on a %d x %d die with the workload's cell" % (STEPS, SMALL_N, SMALL_N),
           "S00": vals}
    with open(os.path.join(HERE, "transient_mode00_c4_1024.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
