"""Seeded synthetic inputs: registers (atom positions) and 1-ns pulse samples.

This module only *generates inputs*. It holds none of the emulation arithmetic
(no pair energies, no midpoint rule, no Hamiltonian), so both the CPU oracle
tests and the CUDA path can use it without sharing method code.

A problem is described exactly as the paper states it (Sec. II.A, Eq. (3) and
Sec. III): atom positions in micrometres, the interaction constant C6 in
rad*um^6/us, and Rabi frequency / detuning (/ phase) samples taken every
nanosecond, t_n = n ns for n = 0 .. t_ns-1 (Sec. III). Arrays are float64
with shape [rows][t_ns]; rows == 1 means the same pulse drives every atom.

Every generator takes an explicit integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi
# C6 for the 70S_{1/2} Rydberg state used by the workloads, rad*um^6/us.
C6_DEFAULT = 5420158.53


@dataclasses.dataclass
class Problem:
    """One emulation problem in the paper's terms (Sec. II.A, Sec. III)."""

    positions: np.ndarray  # [n_atoms][2] float64, um
    c6: float  # rad*um^6/us
    t_ns: int  # number of 1-ns samples (the sequence duration in ns)
    omega: np.ndarray  # [1 or n_atoms][t_ns] rad/us
    delta: np.ndarray  # [1 or n_atoms][t_ns] rad/us
    phi: np.ndarray | None = None  # [1 or n_atoms][t_ns] rad, None = 0
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def _rows(a, t_ns):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[None, :]
    assert a.shape[1] == t_ns
    return np.ascontiguousarray(a)


def chain(n: int, spacing_um: float) -> np.ndarray:
    """Atoms on a line at x = spacing * i."""
    pos = np.zeros((n, 2))
    pos[:, 0] = spacing_um * np.arange(n)
    return pos


def square_lattice(rows: int, cols: int, spacing_um: float) -> np.ndarray:
    """Row-major rows x cols square lattice."""
    pos = np.zeros((rows * cols, 2))
    for r in range(rows):
        for c in range(cols):
            pos[r * cols + c] = (c * spacing_um, r * spacing_um)
    return pos


def random_register(rng: np.random.Generator, n: int, side_um: float,
                    min_spacing_um: float = 5.0, max_failures: int = 100_000) -> np.ndarray:
    """Sequential rejection sampling of n points in [0, side]^2 with a minimum spacing.

    The whole draw restarts after `max_failures` consecutive rejections, which
    only happens near the random-sequential-adsorption jamming density.
    """
    while True:
        pts: list[tuple[float, float]] = []
        failures = 0
        while len(pts) < n and failures < max_failures:
            p = rng.uniform(0.0, side_um, size=2)
            if all((p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2 >= min_spacing_um ** 2 for q in pts):
                pts.append((float(p[0]), float(p[1])))
                failures = 0
            else:
                failures += 1
        if len(pts) == n:
            return np.array(pts, dtype=np.float64)


def piecewise_linear(t_ns: int, knot_values: np.ndarray) -> np.ndarray:
    """Samples at t_n = n ns of a piecewise-linear pulse through equally spaced knots.

    Knot k sits at t = (t_ns - 1) * k / (K - 1) ns, K = len(knot_values).
    """
    knots_t = np.linspace(0.0, float(t_ns - 1), len(knot_values))
    return np.interp(np.arange(t_ns, dtype=np.float64), knots_t, knot_values)


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------

def rabi_chain(n: int = 8, spacing_um: float = 6.0, omega: float = TWO_PI,
               t_ns: int = 1000) -> Problem:
    """1D chain, constant global drive Omega, delta = phi = 0, from |0...0>.

    Default: 8 atoms at 6 um, Omega = 2*pi rad/us, T = 1 us.
    """
    om = np.full((1, t_ns), omega)
    de = np.zeros((1, t_ns))
    return Problem(chain(n, spacing_um), C6_DEFAULT, t_ns, om, de, None,
                   name=f"rabi_chain_n{n}")


def adiabatic_sweep_lattice(rows: int = 4, cols: int = 5, spacing_um: float = 5.0,
                            t_ramp_ns: int = 1000, t_hold_ns: int = 2000,
                            omega_max: float = TWO_PI, delta_span: float = 6.0 * math.pi) -> Problem:
    """Square lattice under an adiabatic sweep.

    Omega ramps linearly 0 -> omega_max over t_ramp, holds for t_hold, ramps back
    to 0 over t_ramp; delta goes linearly from -delta_span to +delta_span over the
    whole sequence. Default: 4x5 at 5 um, 1 + 2 + 1 us, +-6*pi rad/us.
    """
    t_ns = 2 * t_ramp_ns + t_hold_ns
    t = np.arange(t_ns, dtype=np.float64)
    om = np.where(t < t_ramp_ns, omega_max * t / t_ramp_ns,
                  np.where(t < t_ramp_ns + t_hold_ns, omega_max,
                           omega_max * (t_ns - t) / t_ramp_ns))
    de = -delta_span + 2.0 * delta_span * t / t_ns
    return Problem(square_lattice(rows, cols, spacing_um), C6_DEFAULT, t_ns,
                   om[None, :], de[None, :], None,
                   name=f"adiabatic_{rows}x{cols}")


def random_box(seed: int = 3, n: int = 28, side_um: float = 30.0, t_ns: int = 2000) -> Problem:
    """Random register in a side x side box, per-atom constant drives.

    Omega_i ~ U(0.8, 1.2) * 2*pi rad/us, delta_i ~ Normal(0, sd = pi) rad/us,
    phi = 0. Default: 28 atoms in 30 x 30 um, T = 2 us.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = random_register(rng, n, side_um, 5.0)
    om_i = rng.uniform(0.8, 1.2, size=n) * TWO_PI
    de_i = rng.normal(0.0, math.pi, size=n)
    om = np.repeat(om_i[:, None], t_ns, axis=1)
    de = np.repeat(de_i[:, None], t_ns, axis=1)
    return Problem(pos, C6_DEFAULT, t_ns, om, de, None, name=f"random_box_n{n}_s{seed}")


def random_knot_problem(rng: np.random.Generator, n: int, t_ns: int, knots: int = 8,
                        with_phi: bool = False) -> Problem:
    """Random register (square of side 5*ceil(sqrt(n)) + 5 um, spacing >= 5 um) and
    global piecewise-linear Omega ~ U(0, 2*pi), delta ~ U(-4*pi, 4*pi) knots."""
    side = 5.0 * math.ceil(math.sqrt(n)) + 5.0
    pos = random_register(rng, n, side, 5.0)
    om = piecewise_linear(t_ns, rng.uniform(0.0, TWO_PI, size=knots))
    de = piecewise_linear(t_ns, rng.uniform(-4 * math.pi, 4 * math.pi, size=knots))
    ph = None
    if with_phi:
        ph = piecewise_linear(t_ns, rng.uniform(-math.pi, math.pi, size=knots))[None, :]
    return Problem(pos, C6_DEFAULT, t_ns, om[None, :], de[None, :], ph, name=f"knots_n{n}")


def batch_registers(seed: int = 4, count: int = 512, n_lo: int = 10, n_hi: int = 18,
                    t_ns: int = 1000) -> list[Problem]:
    """Independent registers with N uniform in [n_lo, n_hi] and 8-knot pulses."""
    out = []
    for r in range(count):
        rng = np.random.Generator(np.random.PCG64([seed, r]))
        n = int(rng.integers(n_lo, n_hi + 1))
        out.append(random_knot_problem(rng, n, t_ns))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    problem: Problem
    precision: str  # "c64" or "c128"


def serving_stream(seed: int = 5, count: int = 1000, rate_per_s: float = 200.0,
                   n_lo: int = 12, n_hi: int = 26, dt_ns: int = 10) -> list[Request]:
    """Poisson arrivals of solves with N in [n_lo, n_hi], T ~ U[0.5, 3] us rounded
    to dt, complex64 or complex128 with probability 1/2 each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    out = []
    for k in range(count):
        sub = np.random.Generator(np.random.PCG64([seed, k]))
        n = int(sub.integers(n_lo, n_hi + 1))
        t_ns = int(round(sub.uniform(500.0, 3000.0) / dt_ns)) * dt_ns
        prob = random_knot_problem(sub, n, t_ns)
        prec = "c64" if sub.uniform() < 0.5 else "c128"
        out.append(Request(float(arrivals[k]), prob, prec))
    return out


def random_state(seed: int, n: int, dtype=np.complex128) -> np.ndarray:
    """Normalised random complex state of 2**n amplitudes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def random_product_state(seed: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Per-atom single-qubit states (a_i, b_i) with |a|^2 + |b|^2 = 1, shape [n][2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = rng.uniform(0.2, 1.3, size=n)
    ph = rng.uniform(-math.pi, math.pi, size=n)
    return np.stack([np.cos(th) + 0j, np.sin(th) * np.exp(1j * ph)], axis=1)
