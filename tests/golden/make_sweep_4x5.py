"""Writes sweep_4x5_dt10.npz: the oracle's evolution of the 4x5 adiabatic sweep
(20 atoms on a square lattice at 5 um, Omega 0 -> 2 pi -> 0 over 1 + 2 + 1 us,
delta -6 pi -> +6 pi over the 4 us, dt = 10 ns, 400 steps, complex128) from
|0...0>: the final state and <n_i> after every step (row 0 = the initial state).

The propagator is the oracle's Chebyshev expansion over the Gershgorin interval
(Tal-Ezer and Kosloff), which computes the same product of step exponentials
(Eq. (6)) as its Lanczos path; the oracle pins tie the two together. It takes
about two hours of one host core:
    python tests/golden/make_sweep_4x5.py

Calls only the oracle and the seeded input generator.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rydberg as O  # noqa: E402
from paper_2510_09813_b300 import workloads as W  # noqa: E402


def main():
    prob = W.adiabatic_sweep_lattice(4, 5)
    t0 = time.time()
    psi, occ = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi,
                        method="cheb")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_4x5_dt10.npz")
    np.savez_compressed(out, psi=psi, occ=np.asarray(occ))
    print(out, psi.shape, np.asarray(occ).shape, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
