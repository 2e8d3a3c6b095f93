"""CPU oracle for the state-vector Rydberg emulator hot path (complex128, numpy/scipy).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module;
only tests/, the smoke check and the benchmark's CPU-baseline leg use it. It is
deliberately plain and slow, and shares no code with the CUDA library.

What it computes (arXiv 2510.09813):
  * Hilbert space of N two-level atoms, dimension 2**N (Sec. II.A, Eq. (1); the
    printed C^{2N} is read as (C^2)^{(x)N} = C^{2**N}).
  * Hamiltonian, Eq. (3), extended with a laser phase phi_i:
        H = sum_i Omega_i/2 (cos phi_i X_i - sin phi_i Y_i) - sum_i delta_i n_i
            + sum_{i<j} C6/|r_i - r_j|^6 n_i n_j .
    With Y = -i|0><1| + i|1><0|, the single-atom drive has <1|h|0> = Omega/2 e^{-i phi}
    and <0|h|1> = Omega/2 e^{+i phi}.
  * Basis order: row-major N-index tensor of Eq. (4) (Sec. II.B): atom 0 is the
    most significant bit, b = sum_i b_i 2^(N-1-i).
  * Time discretisation, Sec. III and Eq. (6): pulses sampled at t_n = n ns, held
    constant over each step of dt ns at their midpoint value
    (s[floor(m)] + s[ceil(m)])/2 with m = (n + 1/2) dt; psi_{k+1} = exp(-i H_k dt) psi_k.
  * Lanczos (Krylov) evaluation of exp(-i H dt) psi (Sec. III.A), here with full
    re-orthogonalisation and a tight tolerance so that it reproduces the exact
    product of exponentials; a dense expm path (N <= 12) is the brute-force check.
  * Observables <n_i> and bitstring sampling (the emulator results of Sec. III),
    pair correlations, energy moments and overlaps with a target state.
  * An independent Chebyshev propagator (Tal-Ezer and Kosloff) for the same
    product of step exponentials.
  * Exact gradients of occupation observables with respect to the pulse
    samples (Sec. V: the emulator is differentiable), by Frechet derivatives
    of the step exponentials.
  * The Lindblad master equation on the dense superoperator (Sec. III.A,
    open-system dynamics) with Rydberg dephasing and spontaneous decay.

Readings of points the paper leaves open are listed where they are used.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------
# Register: pair energies (Eq. (3), third term)
# ---------------------------------------------------------------------------


def pair_interactions(positions, c6: float) -> np.ndarray:
    """V[i, j] = C6 / |r_i - r_j|^6 for i != j, V[i, i] = 0 (Eq. (3)).

    The paper sums over i > j once per pair; V is returned symmetric so that the
    pair sum is 0.5 * sum_{i != j}. Coincident atoms are an error.
    """
    r = np.asarray(positions, dtype=np.float64)
    n = r.shape[0]
    V = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            d2 = float(np.sum((r[i] - r[j]) ** 2))
            if d2 == 0.0:
                raise ValueError(f"atoms {i} and {j} coincide")
            V[i, j] = c6 / d2 ** 3
    return V


# ---------------------------------------------------------------------------
# Time discretisation (Sec. III, Eq. (6))
# ---------------------------------------------------------------------------


def step_schedule(t_ns: int, dt_ns: int):
    """Steps covering [0, t_ns] ns with step dt_ns.

    Returns a list of (start_ns, length_ns). Reading: when t_ns is not a
    multiple of dt_ns the last step is shorter (t_ns mod dt_ns) and uses its
    own midpoint.
    """
    if dt_ns < 1 or t_ns < 1:
        raise ValueError("dt_ns and t_ns must be >= 1")
    out = []
    start = 0
    while start < t_ns:
        length = min(dt_ns, t_ns - start)
        out.append((start, length))
        start += length
    return out


def midpoint_value(samples_row: np.ndarray, start_ns: int, length_ns: int) -> float:
    """Midpoint rule of Sec. III: m = start + length/2 (= (n + 1/2) dt for a full
    step); value = (s[floor m] + s[ceil m]) / 2. Indices past the last sample
    (t_ns - 1) are clamped to it (reading: samples exist for t = 0 .. t_ns-1 ns)."""
    last = len(samples_row) - 1
    # m is start + length/2; work in half-nanoseconds to stay in integers.
    twice_m = 2 * start_ns + length_ns
    lo = min(twice_m // 2, last)
    hi = min((twice_m + 1) // 2, last)
    return 0.5 * (float(samples_row[lo]) + float(samples_row[hi]))


def step_parameters(n_atoms: int, t_ns: int, dt_ns: int, omega, delta, phi=None):
    """Per-step (tau_us, Omega_bar[N], delta_bar[N], phi_bar[N]) by the midpoint rule.

    Pulse arrays are [rows][t_ns] with rows == 1 (global) or rows == n_atoms.
    """
    def rows_of(a):
        a = np.asarray(a, dtype=np.float64)
        if a.ndim == 1:
            a = a[None, :]
        if a.shape[1] != t_ns or a.shape[0] not in (1, n_atoms):
            raise ValueError("pulse array has the wrong shape")
        return a

    om = rows_of(omega)
    de = rows_of(delta)
    ph = rows_of(phi) if phi is not None else np.zeros((1, t_ns))
    steps = []
    for start, length in step_schedule(t_ns, dt_ns):
        o = np.array([midpoint_value(om[i % om.shape[0]], start, length) for i in range(n_atoms)])
        d = np.array([midpoint_value(de[i % de.shape[0]], start, length) for i in range(n_atoms)])
        p = np.array([midpoint_value(ph[i % ph.shape[0]], start, length) for i in range(n_atoms)])
        steps.append((length / 1000.0, o, d, p))
    return steps


# ---------------------------------------------------------------------------
# Hamiltonian (Eq. (3)) in the basis of Eq. (4)
# ---------------------------------------------------------------------------


def atom_bit(n_atoms: int, i: int) -> int:
    """Bit position of atom i: atom 0 is the most significant bit (Eq. (4) row-major)."""
    return n_atoms - 1 - i


def occupation_bits(n_atoms: int, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """B[b - lo, i] = b_i (occupation of atom i in basis state b), float64."""
    if hi is None:
        hi = 2 ** n_atoms
    b = np.arange(lo, hi, dtype=np.int64)
    B = np.empty((hi - lo, n_atoms))
    for i in range(n_atoms):
        B[:, i] = (b >> atom_bit(n_atoms, i)) & 1
    return B


def diagonal_energies(V: np.ndarray, delta_bar: np.ndarray) -> np.ndarray:
    """E(b) = sum_{i<j} V_ij b_i b_j - sum_i delta_i b_i (the diagonal of Eq. (3))."""
    n = V.shape[0]
    D = 2 ** n
    E = np.empty(D)
    chunk = 1 << 18
    for lo in range(0, D, chunk):
        hi = min(D, lo + chunk)
        B = occupation_bits(n, lo, hi)
        E[lo:hi] = 0.5 * np.einsum("bi,bi->b", B @ V, B) - B @ delta_bar
    return E


def dense_hamiltonian(V, omega_bar, delta_bar, phi_bar) -> np.ndarray:
    """Dense 2^N x 2^N matrix of Eq. (3), built entry by entry (brute force, N <= 12)."""
    n = V.shape[0]
    D = 2 ** n
    H = np.zeros((D, D), dtype=np.complex128)
    for b in range(D):
        occ = [(b >> atom_bit(n, i)) & 1 for i in range(n)]
        e = 0.0
        for i in range(n):
            if occ[i]:
                e -= delta_bar[i]
                for j in range(i + 1, n):
                    if occ[j]:
                        e += V[i, j]
        H[b, b] = e
        for i in range(n):
            bp = b ^ (1 << atom_bit(n, i))
            # column b (source), row bp (target)
            if occ[i] == 0:  # |0> -> |1>: <1|h|0> = Omega/2 e^{-i phi}
                H[bp, b] += 0.5 * omega_bar[i] * np.exp(-1j * phi_bar[i])
            else:  # |1> -> |0>: <0|h|1> = Omega/2 e^{+i phi}
                H[bp, b] += 0.5 * omega_bar[i] * np.exp(1j * phi_bar[i])
    return H


def apply_hamiltonian(psi: np.ndarray, V, omega_bar, delta_bar, phi_bar, E=None) -> np.ndarray:
    """y = H psi without forming H: the diagonal of Eq. (3) times psi plus, per atom,
    the drive term acting on the atom's tensor axis (Sec. III.A: 'apply the diagonal,
    then add the Omega-scaled permutations')."""
    n = V.shape[0]
    if E is None:
        E = diagonal_energies(V, delta_bar)
    x = np.asarray(psi, dtype=np.complex128)
    y = E * x
    yt = y.reshape((2,) * n)
    xt = x.reshape((2,) * n)
    for i in range(n):
        up = 0.5 * omega_bar[i] * np.exp(-1j * phi_bar[i])  # <1|h|0>
        dn = 0.5 * omega_bar[i] * np.exp(1j * phi_bar[i])  # <0|h|1>
        sel0 = [slice(None)] * n
        sel1 = [slice(None)] * n
        sel0[i] = 0
        sel1[i] = 1
        yt[tuple(sel1)] += up * xt[tuple(sel0)]
        yt[tuple(sel0)] += dn * xt[tuple(sel1)]
    return y


def hamiltonian_rows(indices, x, V, omega_bar, delta_bar, phi_bar) -> np.ndarray:
    """(H x)[b] for each listed b, one row of Eq. (3) at a time: the diagonal
    element of b plus, per atom, the drive element between b and b with that
    atom's bit flipped. `x` may be any indexable of complex amplitudes (only the
    N + 1 entries each row touches are read)."""
    n = V.shape[0]
    out = np.empty(len(indices), dtype=np.complex128)
    for k, b in enumerate(indices):
        b = int(b)
        occ = [(b >> atom_bit(n, i)) & 1 for i in range(n)]
        e = 0.0
        for i in range(n):
            if occ[i]:
                e -= delta_bar[i]
                for j in range(i + 1, n):
                    if occ[j]:
                        e += V[i, j]
        acc = e * complex(x[b])
        for i in range(n):
            bp = b ^ (1 << atom_bit(n, i))
            if occ[i] == 0:  # row has the atom in |0>: <0|h|1>
                coef = 0.5 * omega_bar[i] * np.exp(1j * phi_bar[i])
            else:
                coef = 0.5 * omega_bar[i] * np.exp(-1j * phi_bar[i])
            acc += coef * complex(x[bp])
        out[k] = acc
    return out


# ---------------------------------------------------------------------------
# exp(-i H tau) psi
# ---------------------------------------------------------------------------


def tridiagonal(alpha, beta) -> np.ndarray:
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    for k in range(m - 1):
        T[k, k + 1] = T[k + 1, k] = beta[k]
    return T


def lanczos_expm(matvec, psi: np.ndarray, tau: float, tol: float = 1e-13, m_max: int = 60):
    """exp(-i tau H) psi by Lanczos (Sec. III.A), complex128.

    Krylov basis v_0 = psi/|psi|, three-term recurrence for H, then the basis is
    re-orthogonalised in full (classical Gram-Schmidt, twice) so the oracle does
    not depend on the recurrence's loss of orthogonality. The small problem
    exp(-i tau T_m) e_1 is evaluated with scipy's expm. The step is accepted when
    the a-posteriori estimate beta_m |[exp(-i tau T_m) e_1]_{m-1}| <= tol
    (relative to |psi|) or on breakdown; otherwise the Krylov space is reused
    for the largest tau / 2^k that meets tol and the remainder restarts.

    Returns (new_psi, stats) where stats = list of (krylov_dim, tau_taken).
    """
    psi = np.array(psi, dtype=np.complex128)
    remaining = float(tau)
    stats = []
    while remaining > 0.0:
        beta0 = np.linalg.norm(psi)
        if beta0 == 0.0:
            return psi, stats
        V = [psi / beta0]
        alpha: list[float] = []
        beta: list[float] = []
        accepted = None
        for j in range(m_max):
            w = matvec(V[j])
            a = float(np.vdot(V[j], w).real)
            w = w - a * V[j]
            if j > 0:
                w = w - beta[j - 1] * V[j - 1]
            Vm = np.array(V)
            for _ in range(2):
                w = w - Vm.T @ (Vm.conj() @ w)
            b = float(np.linalg.norm(w))
            alpha.append(a)
            T = tridiagonal(alpha, beta)
            u = scipy.linalg.expm(-1j * remaining * T)[:, 0]
            scale = max(1.0, float(np.max(np.abs(alpha))) if alpha else 1.0)
            if b <= 1e-14 * scale or b * abs(u[-1]) <= tol:
                accepted = (remaining, u)
                break
            if j == m_max - 1:
                t = remaining
                while True:
                    t *= 0.5
                    u = scipy.linalg.expm(-1j * t * T)[:, 0]
                    if b * abs(u[-1]) <= tol:
                        break
                accepted = (t, u)
                break
            beta.append(b)
            V.append(w / b)
        t, u = accepted
        m = len(u)
        psi = beta0 * (np.array(V[:m]).T @ u)
        stats.append((m, t))
        remaining -= t
        if remaining < 1e-15 * tau:
            remaining = 0.0
    return psi, stats


def chebyshev_expm(matvec, psi: np.ndarray, tau: float, e_min: float, e_max: float, tol: float = 1e-16):
    """exp(-i tau H) psi by the Chebyshev expansion of Tal-Ezer and Kosloff
    (J. Chem. Phys. 81, 3967 (1984)), an algorithm independent of Lanczos.

    With the spectrum of H inside [e_min, e_max], H = a + b X with
    a = (e_max + e_min) / 2, b = (e_max - e_min) / 2 and X's spectrum in
    [-1, 1]; then exp(-i tau H) = e^{-i a tau} sum_k c_k (-i)^k J_k(b tau) T_k(X)
    with c_0 = 1, c_k = 2, J_k the Bessel functions of the first kind and
    T_k the Chebyshev polynomials (three-term recurrence on vectors). The sum
    stops once k > b tau and |J_k(b tau)| < tol.
    """
    from scipy.special import jv
    psi = np.asarray(psi, dtype=np.complex128)
    a = 0.5 * (e_max + e_min)
    b = 0.5 * (e_max - e_min)
    if b <= 0.0:
        return np.exp(-1j * a * tau) * psi
    z = b * tau

    def X(v):
        return (matvec(v) - a * v) / b

    t_prev, t_cur = psi, X(psi)
    out = jv(0, z) * t_prev + 2.0 * (-1j) * jv(1, z) * t_cur
    k = 1
    while True:
        k += 1
        t_next = 2.0 * X(t_cur) - t_prev
        jk = jv(k, z)
        out = out + 2.0 * (-1j) ** k * jk * t_next
        t_prev, t_cur = t_cur, t_next
        if k > z and abs(jk) < tol:
            break
    return np.exp(-1j * a * tau) * out


def spectral_bounds(V, omega_bar, delta_bar, E=None):
    """Gershgorin interval of the Hamiltonian of Eq. (3): the diagonal range
    widened by the largest off-diagonal row sum, sum_i Omega_i / 2."""
    if E is None:
        E = diagonal_energies(V, delta_bar)
    r = 0.5 * float(np.sum(np.abs(omega_bar)))
    return float(np.min(E)) - r, float(np.max(E)) + r


def zero_state(n_atoms: int) -> np.ndarray:
    """|0...0> (Sec. II.B.2: the initial state of the QPU)."""
    psi = np.zeros(2 ** n_atoms, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def occupations(psi: np.ndarray) -> np.ndarray:
    """<n_i> = sum_b |psi_b|^2 b_i for every atom i."""
    n = int(round(math.log2(psi.size)))
    p = psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2
    out = np.zeros(n)
    pt = p.reshape((2,) * n)
    for i in range(n):
        axes = tuple(k for k in range(n) if k != i)
        out[i] = pt.sum(axis=axes)[1] if n > 1 else pt[1]
    return out


def correlations(psi: np.ndarray) -> np.ndarray:
    """<n_i n_j> = sum_b |psi_b|^2 b_i b_j for every pair of atoms (diagonal:
    <n_i>), as the bit matrix product B^T diag(p) B over basis indices b."""
    n = int(round(math.log2(psi.size)))
    p = psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2
    b = np.arange(psi.size)
    B = np.stack([(b >> (n - 1 - i)) & 1 for i in range(n)], axis=1).astype(np.float64)
    return B.T @ (p[:, None] * B)


def energy_moments(psi: np.ndarray, V, omega_bar, delta_bar, phi_bar=None):
    """(<psi|H|psi>, <psi|H^2|psi>) for the Hamiltonian of Eq. (3) with the
    given (constant) parameters; <H^2> = |H psi|^2 since H is Hermitian."""
    psi = np.asarray(psi, dtype=np.complex128)
    phi = np.zeros(V.shape[0]) if phi_bar is None else phi_bar
    y = apply_hamiltonian(psi, V, omega_bar, delta_bar, phi)
    return complex(np.vdot(psi, y)), float(np.vdot(y, y).real)


def evolve(positions, c6, t_ns, dt_ns, omega, delta, phi=None, psi0=None,
           method: str = "krylov", tol: float = 1e-13, m_max: int = 60,
           record_occupations: bool = True):
    """psi_K = exp(-i H_{K-1} tau) ... exp(-i H_0 tau) psi_0 (Eq. (6)).

    method = "dense" (expm of the brute-force matrix, N <= 12), "krylov", or
    "cheb" (Chebyshev expansion over the Gershgorin interval).
    Returns (psi_K, occ) where occ[k] = <n_i> after k steps (row 0 = psi_0).
    """
    V = pair_interactions(positions, c6)
    n = V.shape[0]
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    occ = [occupations(psi)] if record_occupations else []
    for tau, om, de, ph in step_parameters(n, t_ns, dt_ns, omega, delta, phi):
        if method == "dense":
            H = dense_hamiltonian(V, om, de, ph)
            psi = scipy.linalg.expm(-1j * tau * H) @ psi
        elif method == "cheb":
            E = diagonal_energies(V, de)
            lo, hi = spectral_bounds(V, om, de, E)
            psi = chebyshev_expm(lambda x: apply_hamiltonian(x, V, om, de, ph, E), psi, tau, lo, hi)
        else:
            E = diagonal_energies(V, de)
            psi, _ = lanczos_expm(lambda x: apply_hamiltonian(x, V, om, de, ph, E), psi, tau,
                                  tol=tol, m_max=m_max)
        if record_occupations:
            occ.append(occupations(psi))
    return psi, np.array(occ)


# ---------------------------------------------------------------------------
# Error metrics
# ---------------------------------------------------------------------------


def infidelity(a, b) -> float:
    """1 - |<a|b>|^2 / (|a|^2 |b|^2), overlap accumulated in complex128."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    return float(1.0 - abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def norm_difference(a, b) -> float:
    """|a - b| (the metric of Sec. III.A.1, Figs. 3-4)."""
    return float(np.linalg.norm(np.asarray(a, np.complex128) - np.asarray(b, np.complex128)))


def phase_min_norm_difference(a, b) -> float:
    """min over theta of |a - e^{i theta} b|. Expanding the square,
    |a|^2 + |b|^2 - 2 Re(e^{i theta} <a|b>) is smallest when e^{i theta} <a|b>
    is real and positive, i.e. e^{i theta} = conj(<a|b>) / |<a|b>|; the norm is
    then taken of the difference itself (no cancellation for close vectors)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    phase = np.conj(ov) / abs(ov) if abs(ov) > 0.0 else 1.0
    return float(np.linalg.norm(a - phase * b))


# ---------------------------------------------------------------------------
# Sampling: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) + inverse CDF
# ---------------------------------------------------------------------------

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds, written from its published definition.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key is advanced by the Weyl constants (W0, W1) between rounds.
    """
    c = [int(x) & _MASK for x in counter]
    k0, k1 = int(key[0]) & _MASK, int(key[1]) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & _MASK, p1 & _MASK,
             ((p0 >> 32) ^ c[3] ^ k1) & _MASK, p0 & _MASK]
    return c


def shot_uniform(seed: int, shot: int) -> float:
    """Uniform in [0, 1) for shot index `shot`: Philox4x32-10 with counter
    (shot mod 2^32, shot >> 32, 0, 0) and key (seed mod 2^32, seed >> 32);
    u = ((x0 << 21) | (x1 >> 11)) * 2^-53."""
    x = philox4x32_10((shot & _MASK, (shot >> 32) & _MASK, 0, 0), (seed & _MASK, (seed >> 32) & _MASK))
    u53 = (x[0] << 21) | (x[1] >> 11)
    return u53 * 2.0 ** -53


def sample_bitstrings(psi: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Basis indices b = min{b : cdf(b) > u * cdf(D-1)} with cdf the running sum of
    |psi_b|^2 in float64 (|psi_b|^2 = re^2 + im^2)."""
    p = psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2
    cdf = np.cumsum(p)
    total = cdf[-1]
    out = np.empty(shots, dtype=np.uint64)
    for s in range(shots):
        u = shot_uniform(seed, s)
        idx = int(np.searchsorted(cdf, u * total, side="right"))
        out[s] = min(idx, psi.size - 1)
    return out


# ---------------------------------------------------------------------------
# Overlap with a target state (fidelity; Sec. III emulator results)
# ---------------------------------------------------------------------------


def overlap(a, b):
    """(<a|b>, |a|^2, |b|^2) in complex128 / float64; the fidelity of b with
    the target a is |<a|b>|^2 / (|a|^2 |b|^2)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return complex(np.vdot(a, b)), float(np.vdot(a, a).real), float(np.vdot(b, b).real)


# ---------------------------------------------------------------------------
# Gradients of an occupation observable with respect to the pulse samples.
# Sec. V: the emulator is differentiable, i.e. derivatives of expectation
# values with respect to the tensors that define the pulse sequence exist.
# ---------------------------------------------------------------------------


def drive_generators(n_atoms: int, i: int, omega_bar_i: float, phi_bar_i: float):
    """dH/dOmega_i, dH/ddelta_i and dH/dphi_i of Eq. (3) (with the phase) as
    dense matrices, entry by entry (brute force, small N).

    Drive of atom i: <1|h|0> = Omega/2 e^{-i phi}, <0|h|1> = Omega/2 e^{+i phi}.
    d/dOmega: 1/2 e^{-i phi} and 1/2 e^{+i phi}; d/dphi: -i Omega/2 e^{-i phi}
    and +i Omega/2 e^{+i phi}; d/ddelta: -n_i on the diagonal."""
    D = 2 ** n_atoms
    g_om = np.zeros((D, D), dtype=np.complex128)
    g_ph = np.zeros((D, D), dtype=np.complex128)
    g_de = np.zeros((D, D), dtype=np.complex128)
    bit = atom_bit(n_atoms, i)
    for b in range(D):
        bp = b ^ (1 << bit)
        if (b >> bit) & 1 == 0:  # column b with b_i = 0, target row bp has b_i = 1
            g_om[bp, b] = 0.5 * np.exp(-1j * phi_bar_i)
            g_ph[bp, b] = -0.5j * omega_bar_i * np.exp(-1j * phi_bar_i)
        else:
            g_om[bp, b] = 0.5 * np.exp(1j * phi_bar_i)
            g_ph[bp, b] = 0.5j * omega_bar_i * np.exp(1j * phi_bar_i)
            g_de[b, b] = -1.0
    return g_om, g_de, g_ph


def midpoint_samples(t_ns: int, start_ns: int, length_ns: int):
    """The two sample indices the midpoint rule averages (Sec. III), each with
    weight 1/2 (they coincide when the midpoint falls on a sample)."""
    twice_m = 2 * start_ns + length_ns
    return min(twice_m // 2, t_ns - 1), min((twice_m + 1) // 2, t_ns - 1)


def occupation_gradient(positions, c6, t_ns, dt_ns, omega, delta, phi=None, weights=None, psi0=None):
    """Value and exact gradient of <O>(T) = <psi_K| sum_i w_i n_i |psi_K> with
    respect to every pulse sample (brute force, N <= 8).

    psi_{k+1} = U_k psi_k with U_k = exp(-i tau_k H_k) (Eq. (6)). For a step
    parameter theta of H_k, d<O>/dtheta = 2 Re <lambda_{k+1}| dU_k/dtheta |psi_k>
    with the costate lambda_K = O psi_K, lambda_k = U_k^dagger lambda_{k+1}.
    dU_k/dtheta is the Frechet derivative of expm at -i tau_k H_k in the
    direction -i tau_k dH/dtheta (scipy.linalg.expm_frechet, Al-Mohy and
    Higham 2009), so no commutation of H_k with dH/dtheta is assumed. The
    midpoint rule gives each step parameter the weight 1/2 on its two samples;
    a pulse array with one row is shared by all atoms, so its gradient sums
    over them.

    Returns (value, d_omega, d_delta, d_phi) with the arrays shaped like the
    inputs ([rows][t_ns]); d_phi is None when phi is None.
    """
    V = pair_interactions(positions, c6)
    n = V.shape[0]
    w = np.ones(n) if weights is None else np.asarray(weights, dtype=np.float64)
    om = np.atleast_2d(np.asarray(omega, dtype=np.float64))
    de = np.atleast_2d(np.asarray(delta, dtype=np.float64))
    ph = None if phi is None else np.atleast_2d(np.asarray(phi, dtype=np.float64))
    steps = step_parameters(n, t_ns, dt_ns, om, de, ph)
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    Hs, Us, psis = [], [], [psi]
    for tau, o, d, p in steps:
        H = dense_hamiltonian(V, o, d, p)
        U = scipy.linalg.expm(-1j * tau * H)
        Hs.append(H)
        Us.append(U)
        psis.append(U @ psis[-1])
    o_diag = occupation_bits(n) @ w
    value = float(np.real(np.vdot(psis[-1], o_diag * psis[-1])))
    d_om, d_de = np.zeros_like(om), np.zeros_like(de)
    d_ph = None if ph is None else np.zeros_like(ph)
    lam = o_diag * psis[-1]
    schedule = step_schedule(t_ns, dt_ns)
    for k in range(len(steps) - 1, -1, -1):
        tau, o, d, p = steps[k]
        lo, hi = midpoint_samples(t_ns, *schedule[k])
        for i in range(n):
            g_om, g_de, g_ph = drive_generators(n, i, o[i], p[i])
            for G, target in ((g_om, d_om), (g_de, d_de), (g_ph, d_ph)):
                if target is None:
                    continue
                dU = scipy.linalg.expm_frechet(-1j * tau * Hs[k], -1j * tau * G, compute_expm=False)
                g = 2.0 * np.real(np.vdot(lam, dU @ psis[k]))
                row = 0 if target.shape[0] == 1 else i
                target[row, lo] += 0.5 * g
                target[row, hi] += 0.5 * g
        lam = Us[k].conj().T @ lam
    return value, d_om, d_de, d_ph


# ---------------------------------------------------------------------------
# Open-system dynamics: the Lindblad master equation (Sec. III.A), dense.
# ---------------------------------------------------------------------------
# Reading of the noise channels, which the paper names without operators:
# per atom i, Rydberg dephasing L = sqrt(g_deph_i) n_i and spontaneous decay
# L = sqrt(g_relax_i) |0><1|_i, rates in 1/us.
#     d rho/dt = -i [H, rho] + sum_L (L rho L^dag - {L^dag L, rho} / 2)
# rho is stored row-major, vec(rho)[r * 2^N + c] = rho[r, c], so that
# vec(A rho B) = (A kron B^T) vec(rho).


def jump_operators(n_atoms: int, g_deph, g_relax):
    """The list of dense jump operators of the two channels (zero rates omitted)."""
    D = 2 ** n_atoms
    ops = []
    for i in range(n_atoms):
        bit = atom_bit(n_atoms, i)
        if g_deph[i] > 0.0:
            L = np.zeros((D, D), dtype=np.complex128)
            for b in range(D):
                if (b >> bit) & 1:
                    L[b, b] = math.sqrt(g_deph[i])
            ops.append(L)
        if g_relax[i] > 0.0:
            L = np.zeros((D, D), dtype=np.complex128)
            for b in range(D):
                if (b >> bit) & 1:  # |1> -> |0> on atom i
                    L[b ^ (1 << bit), b] = math.sqrt(g_relax[i])
            ops.append(L)
    return ops


def liouvillian(H, jumps) -> np.ndarray:
    """Dense superoperator of the master equation on row-major vec(rho)."""
    D = H.shape[0]
    I = np.eye(D)
    Lv = -1j * (np.kron(H, I) - np.kron(I, H.T))
    for L in jumps:
        LdL = L.conj().T @ L
        Lv += np.kron(L, L.conj()) - 0.5 * (np.kron(LdL, I) + np.kron(I, LdL.T))
    return Lv


def lindblad_evolve(positions, c6, t_ns, dt_ns, omega, delta, phi=None, g_deph=None, g_relax=None, rho0=None,
                    record_occupations: bool = True):
    """rho_K = exp(tau L_{K-1}) ... exp(tau L_0) rho_0 with the midpoint pulses of
    Sec. III held over each step (brute force, N <= 5). rho_0 defaults to
    |0...0><0...0|. Returns (rho_K [D][D], occ) with occ[k][i] = tr(rho_k n_i)."""
    V = pair_interactions(positions, c6)
    n = V.shape[0]
    D = 2 ** n
    gd = np.zeros(n) if g_deph is None else np.asarray(g_deph, dtype=np.float64)
    gr = np.zeros(n) if g_relax is None else np.asarray(g_relax, dtype=np.float64)
    jumps = jump_operators(n, gd, gr)
    if rho0 is None:
        rho = np.zeros((D, D), dtype=np.complex128)
        rho[0, 0] = 1.0
    else:
        rho = np.array(rho0, dtype=np.complex128).reshape(D, D)
    B = occupation_bits(n)
    occ = [np.real(np.diag(rho)) @ B] if record_occupations else []
    for tau, om, de, ph in step_parameters(n, t_ns, dt_ns, omega, delta, phi):
        Lv = liouvillian(dense_hamiltonian(V, om, de, ph), jumps)
        rho = (scipy.linalg.expm(tau * Lv) @ rho.reshape(-1)).reshape(D, D)
        if record_occupations:
            occ.append(np.real(np.diag(rho)) @ B)
    return rho, np.array(occ)
