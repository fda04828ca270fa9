"""Write the oracle's reference states used by the GPU parity tests.

Calls only oracle/ (and the shared input generators).  Output:
tests/golden/tg32_<recon>_<flux>_20steps.npz with the FP64 conservative state
of the Taylor-Green vortex (Sec. 3.1: Ma 0.1, Re 1600, gamma 1.4, Pr 0.72) on
32^3 cells after 20 CFL-0.5 steps, and the time reached.

    python tests/golden/make_oracle_goldens.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2005_08736_gb300 import inputs  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))
CASES = [("linear", "smooth", oracle.RECON_LINEAR, oracle.FLUX_SMOOTH, 0.0),
         ("wenoz", "full", oracle.RECON_WENO_Z, oracle.FLUX_FULL, 1.0)]


def main():
    n, steps = 32, 20
    prim = inputs.taylor_green(n)
    for rname, fname, recon, flux, C in CASES:
        t0 = time.time()
        s = oracle.Solver(oracle.Config(n, n, n, recon=recon, flux=flux, tau_num_C=C,
                                        prandtl=0.72, mu_ref=1 / 1600, cfl=0.5))
        s.set_state(oracle.conservative(prim, 1.4))
        s.step(steps)
        path = os.path.join(OUT, f"tg32_{rname}_{fname}_20steps.npz")
        np.savez_compressed(path, state=s.state(), t=s.t, steps=steps)
        print(path, f"t={s.t:.6g}", f"{time.time() - t0:.1f}s")


if __name__ == "__main__":
    main()
