"""Writes sweep_3x4_dt10.npz: the oracle's evolution of the 3x4 adiabatic sweep
(12 atoms at 5 um, Omega 0 -> 2 pi -> 0 over 1 + 2 + 1 us, delta -6 pi -> +6 pi,
dt = 10 ns, 400 steps, complex128, Krylov with full re-orthogonalisation at
tol 1e-14) from |0...0>: the final state and <n_i> after every step.

Calls only the oracle and the seeded input generator:
    python tests/golden/make_sweep_3x4.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rydberg as O  # noqa: E402
from paper_2510_09813_b300 import workloads as W  # noqa: E402


def main():
    prob = W.adiabatic_sweep_lattice(3, 4)
    psi, occ = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi,
                        method="krylov", tol=1e-14)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_3x4_dt10.npz")
    np.savez_compressed(out, psi=psi, occ=np.asarray(occ))
    print(out, psi.shape, np.asarray(occ).shape)


if __name__ == "__main__":
    main()
