"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
coefficient tables, closed forms (plane waves, a single Fourier mode, the
Ewald sum with a different splitting), a dense matrix built independently
(Kronecker products, brute-force loops), discrete eigenpairs, invariants the
paper states (Sec. 4.2: energy eq. E_new and overlaps eq. escpro conserved;
Sec. 5.1: contractive Taylor-4, time reversibility; eq. transf: time
rescaling) and finite differences of the energy (eq. new_EoM_b).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import emd_oracle as O
from paper_0812_2801_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_fd():
    out = {}
    with open(os.path.join(GOLDEN, "fd_coefficients.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            out[int(parts[0])] = np.array([float(Fraction(p)) for p in parts[1:]])
    return out


def golden_pz():
    out = {}
    with open(os.path.join(GOLDEN, "pz81_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def fd_matrix_1d(n, coeffs):
    """Periodic 1-D second-difference matrix (without 1/h^2) from given weights."""
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] += coeffs[0]
        for k in range(1, len(coeffs)):
            D[i, (i + k) % n] += coeffs[k]
            D[i, (i - k) % n] += coeffs[k]
    return D


def dense_kinetic(n, h, coeffs):
    D = fd_matrix_1d(n, coeffs)
    E = np.eye(n)
    # index (z, y, x) -> (z N + y) N + x: x is the last Kronecker factor
    lap = (np.kron(np.kron(D, E), E) + np.kron(np.kron(E, D), E)
           + np.kron(np.kron(E, E), D)) / (h * h)
    return -0.5 * lap


def brute_projector(center, sp, n, h):
    """p_J on the grid by plain loops over every point and every image."""
    L = n * h
    c = O.wrap(np.asarray(center, dtype=np.float64), L)
    p = np.zeros(n ** 3)
    rp2 = sp.r_proj * sp.r_proj
    for z in range(n):
        for y in range(n):
            for x in range(n):
                tot = 0.0
                for nz in (-1, 0, 1):
                    for ny in (-1, 0, 1):
                        for nx in (-1, 0, 1):
                            dx = (x * h - c[0]) - nx * L
                            dy = (y * h - c[1]) - ny * L
                            dz = (z * h - c[2]) - nz * L
                            d2 = dx * dx + dy * dy + dz * dz
                            if d2 < rp2:
                                tot += math.exp(-d2 / (2 * sp.r_c ** 2))
                p[(z * n + y) * n + x] = tot * math.pi ** -0.75 * sp.r_c ** -1.5
    return p


SMALL_SP = I.Species(z=4.0, a_loc=0.45, r_loc=2.0, r_c=0.55, h_kb=1.0, r_proj=1.9)


# --------------------------------------------------------------------------
# Finite differences
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_fd_coefficients_match_published_table(order):
    assert np.allclose(O.fd_coefficients(order), golden_fd()[order], rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [4, 6, 8])
def test_fd_symbol_has_design_order(order):
    """sigma(theta) = -(c0 + 2 sum c_k cos k theta) = theta^2 + O(theta^(p+2))."""
    c = golden_fd()[order]
    for theta in (0.2, 0.1):
        sig = -(c[0] + 2 * sum(c[k] * math.cos(k * theta) for k in range(1, len(c))))
        err = abs(sig - theta ** 2)
        assert err < 2.0 * theta ** (order + 2)


@pytest.mark.parametrize("order", [4, 8])
def test_laplacian_plane_wave_eigenvector(order):
    """A periodic plane wave is an exact eigenvector of the FD Laplacian."""
    n, h = 12, 0.3
    c = golden_fd()[order]
    m = np.array([1, -3, 5])
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ph = 2 * math.pi * (m[0] * x + m[1] * y + m[2] * z) / n
    u = np.exp(1j * ph)
    lam = 0.0
    for ma in m:
        th = 2 * math.pi * ma / n
        lam += -(c[0] + 2 * sum(c[k] * math.cos(k * th) for k in range(1, len(c))))
    got = O.laplacian(u, h, order)
    assert np.max(np.abs(got + lam / h ** 2 * u)) < 1e-12


# --------------------------------------------------------------------------
# Propagator pins
# --------------------------------------------------------------------------

def empty_tables():
    return O.AtomTables(loc=[], proj=[], pmerged=[])


def test_free_propagation_matches_mode_closed_form():
    """v = 0, no atoms: every Fourier mode is multiplied by T4(-i tau lam)^2
    per AETRS step, lam = sigma-sum / (2 h^2) (Sec. 5.1, eq. aetrs)."""
    n, h, order = 16, 0.3, 8
    rng = np.random.default_rng(0)
    psi0 = np.zeros((n, n, n), dtype=np.complex128)
    modes = [(1, 0, 2), (-3, 2, 1), (0, 7, -4), (8, -8, 5)]
    amps = rng.normal(size=len(modes)) + 1j * rng.normal(size=len(modes))
    c = golden_fd()[order]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    tau = 0.5 * 0.05
    H = O.Hamiltonian(np.zeros((n, n, n)), empty_tables(), I.SI_LIKE, h, order)
    psi = psi0.copy()
    for a, m in zip(amps, modes):
        psi += a * np.exp(2j * math.pi * (m[0] * x + m[1] * y + m[2] * z) / n)
    expect = np.zeros_like(psi)
    nsteps = 5
    for a, m in zip(amps, modes):
        lam = 0.0
        for ma in m:
            th = 2 * math.pi * ma / n
            lam += -(c[0] + 2 * sum(c[k] * math.cos(k * th) for k in range(1, len(c))))
        lam = 0.5 * lam / h ** 2
        xx = -1j * tau * lam
        t4 = 1 + xx + xx ** 2 / 2 + xx ** 3 / 6 + xx ** 4 / 24
        expect += a * t4 ** (2 * nsteps) * np.exp(2j * math.pi * (m[0] * x + m[1] * y + m[2] * z) / n)
    got = psi[None]
    for _ in range(nsteps):
        got = O.taylor4(O.taylor4(got, tau, H), tau, H)
    assert np.max(np.abs(got[0] - expect)) < 1e-12


def test_free_gaussian_wavepacket_spreads_like_continuum():
    """A free Gaussian (periodically repeated) follows the continuum closed
    form sigma^2 -> sigma^2 + i t up to the FD and Taylor error (~1e-6 here)."""
    n, h, order = 32, 0.3, 8
    L = n * h
    sig = 1.2
    z, y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")

    def packet(t):
        s2 = sig ** 2 + 1j * t
        out = np.zeros((n, n, n), dtype=np.complex128)
        for nx in (-1, 0, 1):
            for ny in (-1, 0, 1):
                for nz in (-1, 0, 1):
                    r2 = ((x - L / 2 - nx * L) ** 2 + (y - L / 2 - ny * L) ** 2
                          + (z - L / 2 - nz * L) ** 2)
                    out += (sig ** 2 / s2) ** 1.5 * np.exp(-r2 / (2 * s2))
        return out

    H = O.Hamiltonian(np.zeros((n, n, n)), empty_tables(), I.SI_LIKE, h, order)
    dt, nsteps = 0.05, 10
    psi = packet(0.0)[None]
    for _ in range(nsteps):
        psi = O.taylor4(O.taylor4(psi, 0.5 * dt, H), 0.5 * dt, H)
    assert np.max(np.abs(psi[0] - packet(dt * nsteps))) < 1e-5


def test_harmonic_oscillator_eigenstate_stationary_phase():
    """An exact discrete eigenpair (psi_e, e) evolves as T4(-i tau e)^(2n) psi_e."""
    n, h, order = 10, 0.3, 4
    L = n * h
    c = golden_fd()[order]
    coord = np.arange(n) * h
    z, y, x = np.meshgrid(coord, coord, coord, indexing="ij")
    w = 2.0
    v = 0.5 * w * w * ((x - L / 2) ** 2 + (y - L / 2) ** 2 + (z - L / 2) ** 2)
    Hd = dense_kinetic(n, h, c) + np.diag(v.ravel())
    evals, evecs = np.linalg.eigh(Hd)
    e0 = evals[0]
    psi_e = evecs[:, 0].reshape(n, n, n).astype(np.complex128)[None]
    H = O.Hamiltonian(v, empty_tables(), I.SI_LIKE, h, order)
    tau = 0.5 * 0.05
    psi = psi_e.copy()
    nsteps = 6
    for _ in range(nsteps):
        psi = O.taylor4(O.taylor4(psi, tau, H), tau, H)
    xx = -1j * tau * e0
    t4 = 1 + xx + xx ** 2 / 2 + xx ** 3 / 6 + xx ** 4 / 24
    assert np.max(np.abs(psi - t4 ** (2 * nsteps) * psi_e)) < 1e-12
    assert abs(e0 - 1.5 * w) < 0.5       # continuum ground state 3w/2, FD + box error


def _small_nl_system(seed=3):
    n, h, order = 8, 0.5, 4
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, n * h, size=(2, 3))
    coord = np.arange(n) * h
    z, y, x = np.meshgrid(coord, coord, coord, indexing="ij")
    v = 0.3 * np.cos(2 * math.pi * x / (n * h)) - 0.2 * np.sin(2 * math.pi * (y + z) / (n * h))
    return n, h, order, R, v


def test_hamiltonian_matches_dense_bruteforce_matrix():
    """H applied by the oracle equals an independently built dense matrix:
    Kronecker FD kinetic + diag(v) + sum_J h_J h^3 p_J p_J^T."""
    n, h, order, R, v = _small_nl_system()
    sp = SMALL_SP
    c = golden_fd()[order]
    Hd = dense_kinetic(n, h, c) + np.diag(v.ravel())
    for j in range(R.shape[0]):
        p = brute_projector(R[j], sp, n, h)
        Hd += sp.h_kb * h ** 3 * np.outer(p, p)
    H = O.Hamiltonian(v, O.atom_tables(R, sp, n, h), sp, h, order)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(3, n, n, n)) + 1j * rng.normal(size=(3, n, n, n))
    got = H.apply(u).reshape(3, -1)
    expect = (Hd @ u.reshape(3, -1).T).T
    assert np.max(np.abs(got - expect)) < 1e-11 * np.max(np.abs(expect))
    # one AETRS step with the same H in both halves against a dense polynomial
    tau = 0.02
    A = -1j * tau * Hd
    T4 = np.eye(n ** 3) + A + A @ A / 2 + A @ A @ A / 6 + A @ A @ A @ A / 24
    got2 = O.taylor4(O.taylor4(u, tau, H), tau, H).reshape(3, -1)
    exp2 = (T4 @ T4 @ u.reshape(3, -1).T).T
    assert np.max(np.abs(got2 - exp2)) < 1e-11 * np.max(np.abs(exp2))
    # and the Taylor polynomial is within its truncation bound of the exact exp
    E = scipy.linalg.expm(A)
    lam_max = np.max(np.abs(np.linalg.eigvalsh(Hd)))
    x = tau * lam_max
    bound = x ** 5 / 120 * math.exp(x)
    assert np.max(np.abs(T4 - E)) <= bound * 1.01 + 1e-14


def test_pointwise_hamiltonian_matches_whole_grid_apply():
    n, h, order, R, v = _small_nl_system(7)
    sp = SMALL_SP
    tables = O.atom_tables(R, sp, n, h)
    H = O.Hamiltonian(v, tables, sp, h, order)
    rng = np.random.default_rng(9)
    u = rng.normal(size=(2, n, n, n)) + 1j * rng.normal(size=(2, n, n, n))
    full = H.apply(u)
    c = O.projections(u, tables, sp, h)
    pts = [(0, 0, 0), (3, 7, 1), (7, 7, 7), (4, 2, 6)]
    got = O.hamiltonian_at_points(u, v, c, R, sp, h, order, pts, [0, 1])
    for k, (z, y, x) in enumerate(pts):
        for a in range(2):
            assert abs(got[a, k] - full[a, z, y, x]) < 1e-11 * np.max(np.abs(full))


def test_taylor4_contractive_and_round_trip_bound():
    """Sec. 5.1: Taylor-4 is contractive (norm never grows) below the stability
    edge; T4(+i tau H) T4(-i tau H) = 1 - O(x^6), bounded mode by mode."""
    n, h, order, R, v = _small_nl_system(11)
    sp = SMALL_SP
    H = O.Hamiltonian(v, O.atom_tables(R, sp, n, h), sp, h, order)
    rng = np.random.default_rng(1)
    u = rng.normal(size=(1, n, n, n)) + 1j * rng.normal(size=(1, n, n, n))
    tau = 0.02
    norms = [np.linalg.norm(u)]
    w = u
    for _ in range(6):
        w = O.taylor4(w, tau, H)
        norms.append(np.linalg.norm(w))
    assert all(b <= a * (1 + 1e-15) for a, b in zip(norms, norms[1:]))
    back = O.taylor4(O.taylor4(u, tau, H), -tau, H)
    c = golden_fd()[order]
    Hd = dense_kinetic(n, h, c) + np.diag(v.ravel())
    for j in range(R.shape[0]):
        p = brute_projector(R[j], sp, n, h)
        Hd += sp.h_kb * h ** 3 * np.outer(p, p)
    lam = np.linalg.eigvalsh(Hd)
    x = tau * lam
    t4p = 1 + 1j * x - x ** 2 / 2 - 1j * x ** 3 / 6 + x ** 4 / 24
    t4m = np.conj(t4p)
    bound = np.max(np.abs(t4p * t4m - 1))
    assert np.linalg.norm(back - u) <= bound * np.linalg.norm(u) * (1 + 1e-6) + 1e-13


def test_mu_scaling_is_exact():
    """eq. transf: with ions held fixed, (dt, mu) and (dt/mu, 1) give the same
    orbitals bit for bit (the propagator only sees tau = dt / (2 mu))."""
    s = I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=21)
    dt, mu = 0.3, 7.0
    a = O.run(s, 3, dt=dt, mu=mu, frozen_ions=True)
    b = O.run(s, 3, dt=dt / mu, mu=1.0, frozen_ions=True)
    assert np.array_equal(a.psi, b.psi)


# --------------------------------------------------------------------------
# Electrostatics and xc
# --------------------------------------------------------------------------

def test_poisson_single_mode_closed_form():
    n, h = 12, 0.4
    L = n * h
    coord = np.arange(n) * h
    z, y, x = np.meshgrid(coord, coord, coord, indexing="ij")
    G = 2 * math.pi * np.array([2, -1, 3]) / L
    rho = 0.7 * np.cos(G[0] * x + G[1] * y + G[2] * z)
    v = O.poisson(rho, h)
    assert np.max(np.abs(v - 4 * math.pi * rho / (G @ G))) < 1e-12


def test_gaussian_ion_charge_integrates_to_z():
    n, h = 32, 0.3
    R = np.array([[1.234, 4.5, 8.9], [7.7, 0.1, 3.3]])
    t = O.atom_tables(R, I.SI_LIKE, n, h)
    g = O.ion_charge(t, I.SI_LIKE, n)
    assert abs(g.sum() * h ** 3 - 2 * I.SI_LIKE.z) < 1e-10


def ewald_point_charges(R, Z, L, eta, rcut=14.0, gmax=12):
    """Standard Ewald energy of point charges with a neutralising background."""
    from scipy.special import erfc
    V = L ** 3
    na = R.shape[0]
    e_real = 0.0
    nmax = int(math.ceil(rcut / L)) + 1
    for j in range(na):
        for k in range(na):
            for nx in range(-nmax, nmax + 1):
                for ny in range(-nmax, nmax + 1):
                    for nz in range(-nmax, nmax + 1):
                        if j == k and nx == ny == nz == 0:
                            continue
                        d = np.linalg.norm(R[j] - R[k] - L * np.array([nx, ny, nz]))
                        if d < rcut:
                            e_real += 0.5 * Z * Z * erfc(eta * d) / d
    e_rec = 0.0
    for mx in range(-gmax, gmax + 1):
        for my in range(-gmax, gmax + 1):
            for mz in range(-gmax, gmax + 1):
                if mx == my == mz == 0:
                    continue
                G = 2 * math.pi * np.array([mx, my, mz]) / L
                g2 = G @ G
                S = np.sum(Z * np.exp(1j * (R @ G)))
                e_rec += 2 * math.pi / V * math.exp(-g2 / (4 * eta * eta)) / g2 * abs(S) ** 2
    e_self = -eta / math.sqrt(math.pi) * na * Z * Z
    Q = na * Z
    e_bg = -math.pi * Q * Q / (2 * V * eta * eta)
    return e_real + e_rec + e_self + e_bg


def test_ion_electrostatics_equals_ewald_with_other_splitting():
    """Grid Gaussian charges + self term + erfc short range reproduce the Ewald
    energy of point ions (computed with a different splitting parameter), up to
    the dropped G = 0 constant pi Q^2 / (2 V eta^2), eta = 1/(sqrt2 a)."""
    n, h = 32, 0.3
    L = n * h
    sp = I.SI_LIKE
    R = np.array([[1.2, 2.3, 3.1], [6.0, 5.5, 7.9], [3.3, 8.8, 0.4]])
    t = O.atom_tables(R, sp, n, h)
    g = O.ion_charge(t, sp, n)
    v = O.poisson(-g, h)
    e_sr, _ = O.short_range_ion(R, sp, L)
    ours = 0.5 * h ** 3 * np.sum(-g * v) - O.ion_self_energy(3, sp) + e_sr
    eta = 1 / (math.sqrt(2) * sp.a_loc)
    Q = 3 * sp.z
    ref = ewald_point_charges(R, sp.z, L, eta=0.45) + math.pi * Q * Q / (2 * L ** 3 * eta * eta)
    assert abs(ours - ref) < 1e-7 * abs(ref)


def test_pz81_constants_exchange_and_continuity():
    P = golden_pz()
    for k in ("gamma", "beta1", "beta2", "A", "B", "C", "D"):
        assert O.PZ81[k] == P[k]
    # the continuous C, D round to the published four-decimal values
    Pc = O.PZ81_C1
    for k in ("gamma", "beta1", "beta2", "A", "B"):
        assert Pc[k] == P[k]
    assert abs(Pc["C"] - P["C"]) < 5e-5 and Pc["C"] != P["C"]
    assert abs(Pc["D"] - P["D"]) < 5e-5 and Pc["D"] != P["D"]
    for rs in (0.5, 1.0, 2.0, 5.0):
        rho = 3.0 / (4 * math.pi * rs ** 3)
        eps, _ = O.lda_pz81(np.array([rho]))
        if rs >= 1:
            ec = P["gamma"] / (1 + P["beta1"] * math.sqrt(rs) + P["beta2"] * rs)
        else:
            ec = Pc["A"] * math.log(rs) + Pc["B"] + Pc["C"] * rs * math.log(rs) + Pc["D"] * rs
        assert abs(eps[0] - ec - P["eps_x_times_rs"] / rs) < 1e-12
    # eps_c and v_xc are continuous at r_s = 1 (v continuous <=> d eps/d r_s
    # continuous, given eps continuous): across rho1 (1 +- 1e-9) both move by
    # O(1e-9) only.  The published rounding leaves jumps of 3.2e-5 and 2.7e-5.
    rho1 = 3.0 / (4 * math.pi)
    lo = O.lda_pz81(np.array([rho1 * (1 + 1e-9)]))
    hi = O.lda_pz81(np.array([rho1 * (1 - 1e-9)]))
    assert abs(lo[0][0] - hi[0][0]) < 1e-9
    assert abs(lo[1][0] - hi[1][0]) < 1e-9
    # and the slope of v across r_s = 1 differs by O(1) only (no kink blowing up)
    d = 1e-6
    slope = [(O.lda_pz81(np.array([rho1 * (1 + s * d + d)]))[1][0]
              - O.lda_pz81(np.array([rho1 * (1 + s * d - d)]))[1][0]) / (2 * d * rho1)
             for s in (-2.0, 2.0)]
    assert abs(slope[0] - slope[1]) < 0.05 * abs(slope[0])


def test_lda_energy_continuous_along_a_path_through_rs_one():
    """E_xc = h^3 sum rho eps_xc along rho(s) = rho1 (1 + s), s in [-1e-3, 1e-3]
    on a single point: with continuous C, D its derivative equals h^3 v_xc
    rho1 on both sides of r_s = 1, so the integral of v along the path equals
    the change of E (no hidden jump)."""
    rho1 = 3.0 / (4 * math.pi)
    s = np.linspace(-1e-3, 1e-3, 20001)
    rho = rho1 * (1 + s)
    eps, v = O.lda_pz81(rho)
    e = rho * eps
    work = np.trapezoid(v, rho)
    assert abs((e[-1] - e[0]) - work) < 1e-12


def test_lda_potential_is_derivative_of_energy_density():
    """v_xc = d(rho eps_xc)/d rho, checked by central differences."""
    rho = np.array([1e-4, 3e-3, 0.05, 0.2, 0.9, 3.0])
    d = 1e-6 * rho
    ep, _ = O.lda_pz81(rho + d)
    em, _ = O.lda_pz81(rho - d)
    num = ((rho + d) * ep - (rho - d) * em) / (2 * d)
    _, v = O.lda_pz81(rho)
    assert np.max(np.abs(num - v) / np.abs(v)) < 1e-7


# --------------------------------------------------------------------------
# Forces and the conserved quantities of the full step
# --------------------------------------------------------------------------

def test_forces_are_minus_energy_gradient():
    """F = -dE_KS/dR at fixed orbitals (eq. new_EoM_b) by central differences.

    The projector is cut off at r_proj; with the default width the cut-off
    value is 3.7e-6 of the peak, and every grid point crossing the sphere
    during the +-dR displacement makes a jump that the difference quotient
    divides by 2 dR.  A narrower projector (cut-off value ~1e-15) removes
    those jumps, so the quotient tests the force formulas alone."""
    sp = I.Species(r_c=0.6)
    s = I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=31, species=sp)
    st = O.init_state(s)
    F = st.F
    dR = 1e-4

    def eks(R):
        t = O.atom_tables(R, s.species, s.n, s.h)
        g = O.ion_charge(t, s.species, s.n)
        st2 = O.State(**{**st.__dict__, "R": R, "tables": t, "g_ion": g,
                          "v_loc": O.poisson(-g, s.h)})
        return O.energies(st2)["ks"]

    for j in range(2):
        for ax in range(3):
            Rp = st.R.copy(); Rp[j, ax] += dR
            Rm = st.R.copy(); Rm[j, ax] -= dR
            fd = -(eks(Rp) - eks(Rm)) / (2 * dR)
            assert abs(fd - F[j, ax]) < 2e-6 * np.max(np.abs(F)) + 1e-8


def _energy_trace(s, dt, t_end):
    st = O.init_state(s)
    e0 = O.energies(st)["total"]
    dev = 0.0
    for _ in range(int(round(t_end / dt))):
        st = O.md_step(st, dt, s.mu)
        dev = max(dev, abs(O.energies(st)["total"] - e0))
    return dev, st


@pytest.mark.slow
def test_energy_conserved_and_converges_with_dt():
    """eq. E_new: E = sum M V^2/2 + E_KS is conserved by the dynamics; the
    discrete step's deviation shrinks at least ~second order in dt."""
    s = I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=41, n_orb=4)
    s.V = s.V * 30.0                      # hotter ions: forces and motion matter
    d1, _ = _energy_trace(s, 0.04, 0.8)
    d2, st = _energy_trace(s, 0.02, 0.8)
    e = abs(O.energies(st)["total"])
    assert d2 < 1e-5 * e
    assert d1 / d2 > 3.0


def test_orthonormality_preserved_without_constraints():
    """eq. escpro: overlaps stay constant with no explicit orthogonalisation;
    the only loss is Taylor-4 contraction, which shrinks fast with dt."""
    s = I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=51)
    errs = []
    for dt, nst in ((0.04, 10), (0.02, 20)):
        st = O.run(s, nst, dt=dt, mu=1.0)
        f = st.psi.reshape(st.psi.shape[0], -1)
        S = (f.conj() @ f.T) * s.h ** 3
        errs.append(np.max(np.abs(S - np.eye(S.shape[0]))))
    assert errs[1] < 1e-7
    assert errs[0] / errs[1] > 8.0


def test_first_step_with_fixed_ions_is_two_taylor_halves():
    """Step 0 with ions held: H(t+dt) = H(t) (constant extrapolation), so the
    step is T4(-i tau H)^2 psi with tau = dt / (2 mu) (eq. aetrs, eq. transf)."""
    s = I.small_system(n=16, h=0.35, fd_order=6, n_atoms=2, seed=61)
    st = O.init_state(s)
    dt, mu = 0.12, 3.0
    H = O.Hamiltonian(st.v_loc + st.vhxc_hist[0], st.tables, s.species, s.h, s.fd_order)
    tau = dt / (2 * mu)
    expect = O.taylor4(O.taylor4(st.psi, tau, H), tau, H)
    got = O.md_step(st, dt, mu, frozen_ions=True).psi
    assert np.max(np.abs(got - expect)) < 1e-14


def test_extrapolation_exact_on_quadratic_history():
    t = np.array([0.0, 1.0, 2.0])
    a, b, c = 0.3, -1.1, 2.5
    f = lambda tt: a * tt * tt + b * tt + c
    hist = [np.array([f(2.0)]), np.array([f(1.0)]), np.array([f(0.0)])]
    assert abs(O.extrapolate_vhxc(hist)[0] - f(3.0)) < 1e-13
    lin = [np.array([b * 1.0 + c]), np.array([c])]
    assert abs(O.extrapolate_vhxc(lin)[0] - (2 * b + c)) < 1e-13


def test_initial_density_is_neutralising():
    """rho = 2 sum |phi|^2 of orthonormal orbitals integrates to N_e = sum Z."""
    s = I.tiny_fp64()
    rho = O.density(s.psi, s.occ)
    assert abs(rho.sum() * s.h ** 3 - s.n_atoms * s.species.z) < 1e-10


def test_hamiltonian_is_functional_derivative_of_energy():
    """eq. new_EoM_a: H phi_A = dE_KS/d phi_A^* / f.  For a perturbation
    phi_A -> phi_A + eps chi, dE_KS/d eps = 2 f Re <chi|H[rho] phi_A>, with
    H built from the potentials of the unperturbed density."""
    s = I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=71, n_orb=3)
    st = O.init_state(s)
    rng = np.random.default_rng(3)
    chi = rng.normal(size=st.psi.shape[1:]) + 1j * rng.normal(size=st.psi.shape[1:])
    chi *= 0.05
    A = 1
    H = O.Hamiltonian(st.v_loc + st.v_h + st.v_xc, st.tables, s.species, s.h, s.fd_order)
    hphi = H.apply(st.psi)[A]
    ana = 2 * s.occ * s.h ** 3 * float(np.sum((np.conj(chi) * hphi).real))

    def eks(eps):
        psi = st.psi.copy()
        psi[A] = psi[A] + eps * chi
        rho, vh, ex, vx = O.electron_potentials(psi, s.occ, s.h)
        st2 = O.State(**{**st.__dict__, "psi": psi, "rho": rho, "v_h": vh,
                          "eps_xc": ex, "v_xc": vx})
        return O.energies(st2)["ks"]

    e = 1e-5
    num = (eks(e) - eks(-e)) / (2 * e)
    assert abs(num - ana) < 1e-6 * abs(ana)


def test_dipole_of_a_shifted_gaussian_cloud():
    """A Gaussian electron cloud of charge N at c (sigma = 0.5, tails at the
    box edge below 1e-15, sampling error of its moments ~e^-55) has
    electron dipole -N (c - L/2) along each axis (symmetry); shifting it by
    k grid points moves that by -N k h; a point ion of charge Z at the same
    centre cancels it when Z = N."""
    n, h = 32, 0.3
    L = n * h
    x = np.arange(n) * h
    c = np.array([4.2, 5.1, 4.8])           # cloud centre on no grid symmetry

    def cloud(cc):
        g = [np.exp(-(x - cc[a]) ** 2 / (2 * 0.5 ** 2)) for a in range(3)]
        rho = g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]
        return rho * 4.0 / (rho.sum() * h ** 3)    # 4 electrons

    D = O.dipole(cloud(c), np.zeros((0, 3)), 4.0, h)
    # discrete symmetric cloud: first moment equals the centre to ~1e-12
    assert np.allclose(D, -4.0 * (c - L / 2), atol=1e-9)
    D2 = O.dipole(cloud(c + np.array([0, 0, 2 * h])), np.zeros((0, 3)), 4.0, h)
    assert abs((D2[2] - D[2]) - (-4.0 * 2 * h)) < 1e-9
    assert np.allclose(O.dipole(cloud(c), c[None, :] + L, 4.0, h), 0.0, atol=1e-9)


# --------------------------------------------------------------------------
# Projector normalisation (Sec. 5, separable pseudopotential) from the
# continuum closed forms, and the length-gauge field against the dipole energy
# --------------------------------------------------------------------------

def test_projector_overlaps_match_continuum_gaussian_integrals():
    """The projector is a Gaussian of unit norm in the continuum.  Written
    from that definition, not from the oracle's formula: for two such
    Gaussians a distance d apart, int p_J p_K d^3r = exp(-d^2 / (4 r_c^2)),
    which is 1 at d = 0.  The grid sum h^3 sum_r p_J p_K differs from the
    integral by (i) aliasing, of order exp(-pi^2 r_c^2 / h^2) (Poisson
    summation of a Gaussian of variance r_c^2/2; here e^-120), and (ii) the
    cut-off at r_proj = 5 r_c.  The product p_J p_K is exp(-d^2/(4 r_c^2))
    times a unit Gaussian of variance r_c^2/2 centred midway, d/2 from each
    centre, so each cut-off removes at most its mass outside a ball of
    radius x r_c, x = (r_proj - d/2)/r_c: T(x) = erfc(x) + (2/sqrt(pi)) x
    e^(-x^2) (8e-11 at d = 0).  The test allows twice that plus 1e-12.
    r_c = 0.7 (not 1) so that a wrong power of r_c changes the result, and
    the supports stay inside the box (no image sums)."""
    rc = 0.7
    sp = I.Species(r_c=rc, r_proj=5.0 * rc)
    n, h = 44, 0.2
    L = n * h
    centre = np.array([0.5 * L + 0.013, 0.5 * L - 0.021, 0.5 * L + 0.007])
    for d in (0.0, 0.45, 1.1):
        shift = d * np.array([1.0, 2.0, 2.0]) / 3.0      # unit vector (1,2,2)/3
        R = np.stack([centre - 0.5 * shift, centre + 0.5 * shift])
        t = O.atom_tables(R, sp, n, h)
        pj = np.zeros(n ** 3)
        pk = np.zeros(n ** 3)
        pj[t.pmerged[0][0]] = t.pmerged[0][1]
        pk[t.pmerged[1][0]] = t.pmerged[1][1]
        ov = h ** 3 * float(pj @ pk)
        x = (sp.r_proj - 0.5 * d) / rc
        tail = math.erfc(x) + 2.0 / math.sqrt(math.pi) * x * math.exp(-x * x)
        exact = math.exp(-d * d / (4.0 * rc * rc))
        assert abs(ov - exact) < 2.0 * exact * tail + 1e-12, (d, ov, exact, tail)


def _field_system():
    sp = I.Species(r_c=0.6)                     # narrow projector: see the force pin
    s = I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=33, species=sp,
                       n_orb=3)
    return s


def test_field_hamiltonian_is_derivative_of_energy_with_dipole_term():
    """Length gauge (field along z): the energy of the electrons and ions in a
    uniform field e is -e D_z, with D_z the dipole of the pinned dipole
    read-out.  The step's Hamiltonian with a field must then be
    d(E_KS - e D_z)/d phi^* / f.  The test takes the first step of the oracle
    with ions held, where H(t+dt) = H(t) (constant extrapolation), and checks
    (1) that it equals two Taylor halves of H_KS + e s(z), and (2) that this
    H is the functional derivative of E_KS - e D_z by central differences
    along a random direction."""
    s = _field_system()
    st = O.init_state(s)
    e_f = 0.37                                   # large: the term must show
    H = O.Hamiltonian(st.v_loc + st.v_h + st.v_xc + e_f * O.sawtooth_z(s.n, s.h),
                      st.tables, s.species, s.h, s.fd_order)
    dt, mu = 0.05, 1.0
    tau = dt / (2 * mu)
    got = O.md_step(st, dt, mu, field=e_f, frozen_ions=True).psi
    assert np.max(np.abs(got - O.taylor4(O.taylor4(st.psi, tau, H), tau, H))) < 1e-14

    rng = np.random.default_rng(5)
    chi = 0.05 * (rng.normal(size=st.psi.shape[1:]) + 1j * rng.normal(size=st.psi.shape[1:]))
    A = 2
    ana = 2 * s.occ * s.h ** 3 * float(np.sum((np.conj(chi) * H.apply(st.psi)[A]).real))

    def energy(eps):
        psi = st.psi.copy()
        psi[A] = psi[A] + eps * chi
        rho, vh, ex, vx = O.electron_potentials(psi, s.occ, s.h)
        st2 = O.State(**{**st.__dict__, "psi": psi, "rho": rho, "v_h": vh,
                          "eps_xc": ex, "v_xc": vx})
        return O.energies(st2)["ks"] - e_f * O.dipole(rho, st.R, s.species.z, s.h)[2]

    eps = 1e-5
    num = (energy(eps) - energy(-eps)) / (2 * eps)
    assert abs(num - ana) < 1e-6 * abs(ana)


def test_field_forces_are_minus_gradient_of_energy_with_dipole_term():
    """With a field e the force on the ions is -d(E_KS - e D_z)/dR at fixed
    orbitals (the ion part of D_z is sum_J Z s(R_Jz)).  The forces the
    oracle's step computes with a field (F(t+dt) after one step with moving
    ions) are compared with central differences of that energy at the new
    state."""
    s = _field_system()
    s.V = s.V * 50.0
    st0 = O.init_state(s)
    e_f = 0.23
    st = O.md_step(st0, 0.05, 1.0, field=e_f)
    dR = 1e-4

    def energy(R):
        t = O.atom_tables(R, s.species, s.n, s.h)
        g = O.ion_charge(t, s.species, s.n)
        st2 = O.State(**{**st.__dict__, "R": R, "tables": t, "g_ion": g,
                          "v_loc": O.poisson(-g, s.h)})
        return O.energies(st2)["ks"] - e_f * O.dipole(st.rho, R, s.species.z, s.h)[2]

    scale = np.max(np.abs(st.F))
    assert scale > 0.5 * s.species.z * e_f       # the field term dominates
    for j in range(2):
        for ax in range(3):
            Rp = st.R.copy(); Rp[j, ax] += dR
            Rm = st.R.copy(); Rm[j, ax] -= dR
            fd = -(energy(Rp) - energy(Rm)) / (2 * dR)
            assert abs(fd - st.F[j, ax]) < 2e-6 * scale + 1e-8, (j, ax, fd, st.F[j, ax])


# --------------------------------------------------------------------------
# Several projectors per atom (l <= 2): the Gaussian-type separable terms
# against closed forms of Gaussian moments, and E / F / H consistency
# --------------------------------------------------------------------------

LM_SP = I.Species(r_c=0.7, r_proj=4.9, lmax=2, h_l=(0.7, -0.4))
LM_NAMES = ["s", "x", "y", "z", "xy", "yz", "zx", "x2-y2", "3z2-r2"]


def _lm_grid_projectors(R, n, h):
    """Every projector of the atoms at R on the full grid, [n_atoms * 9, n^3]."""
    t = O.atom_tables(R, LM_SP, n, h)
    P = np.zeros((len(t.pmerged), n ** 3))
    for k, (idx, p) in enumerate(t.pmerged):
        P[k, idx] = p
    return P


def test_lm_projectors_orthonormal_and_overlaps_closed_forms():
    """Written from the definitions, not from the oracle's formulas.  The 9
    projectors of one atom are orthonormal in the continuum (unit norm by
    the choice of N_l; the real solid harmonics are orthogonal on the
    sphere).  For two atoms a vector D apart, with s the position relative
    to their midpoint, the product of two Gaussians of width r_c is
    exp(-D^2/(4 r_c^2)) exp(-s^2/r_c^2), whose moments are <s_a^2> = r_c^2/2
    and <s_a^2 s_b^2> = r_c^4/4 (a != b): the s-s overlap is E =
    exp(-D^2/(4 r_c^2)); p_a-p_b is E (delta_ab - D_a D_b / (2 r_c^2)); s on
    J with p_a on K (K at J + D) is -E D_a / (sqrt(2) r_c); xy-xy is E (1 -
    D_x^2/(2 r_c^2)) (1 - D_y^2/(2 r_c^2)).  The grid sums differ by
    aliasing (~exp(-pi^2 r_c^2/h^2) = e^-121 here) and the cut-off at r_proj
    = 7 r_c (relative tails below 1e-16 for l <= 2)."""
    n, h = 56, 0.2
    L = n * h
    rc = LM_SP.r_c
    c0 = np.array([0.5 * L + 0.013, 0.5 * L - 0.021, 0.5 * L + 0.007])
    G = h ** 3 * (lambda P: P @ P.T)(_lm_grid_projectors(c0[None, :], n, h))
    assert np.max(np.abs(G - np.eye(9))) < 1e-10, np.round(G, 6)
    for d in (0.45, 1.1):
        D = d * np.array([1.0, 2.0, 2.0]) / 3.0
        P = _lm_grid_projectors(np.stack([c0 - 0.5 * D, c0 + 0.5 * D]), n, h)
        ov = h ** 3 * (P[:9] @ P[9:].T)          # [channel on J, channel on K]
        E = math.exp(-d * d / (4 * rc * rc))
        assert abs(ov[0, 0] - E) < 1e-10
        for a in range(3):
            assert abs(ov[0, 1 + a] - (-E * D[a] / (math.sqrt(2.0) * rc))) < 1e-10
            for b in range(3):
                exact = E * ((a == b) - D[a] * D[b] / (2 * rc * rc))
                assert abs(ov[1 + a, 1 + b] - exact) < 1e-10, (a, b)
        exact = E * (1 - D[0] ** 2 / (2 * rc * rc)) * (1 - D[1] ** 2 / (2 * rc * rc))
        assert abs(ov[4, 4] - exact) < 1e-10


def _lm_system(seed):
    sp = I.Species(r_c=0.6, lmax=2, h_l=(0.7, -0.4))
    return I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=seed, species=sp, n_orb=3)


def test_lm_forces_are_minus_energy_gradient():
    """F = -dE_KS/dR at fixed orbitals with s, p and d projectors, by central
    differences (narrow projectors as in the s-only test, so that no grid
    point crosses the cut-off sphere during the displacement)."""
    s = _lm_system(37)
    st = O.init_state(s)
    F = st.F
    dR = 1e-4

    def eks(R):
        t = O.atom_tables(R, s.species, s.n, s.h)
        g = O.ion_charge(t, s.species, s.n)
        st2 = O.State(**{**st.__dict__, "R": R, "tables": t, "g_ion": g,
                          "v_loc": O.poisson(-g, s.h)})
        return O.energies(st2)["ks"]

    for j in range(2):
        for ax in range(3):
            Rp = st.R.copy(); Rp[j, ax] += dR
            Rm = st.R.copy(); Rm[j, ax] -= dR
            fd = -(eks(Rp) - eks(Rm)) / (2 * dR)
            assert abs(fd - F[j, ax]) < 2e-6 * np.max(np.abs(F)) + 1e-8


def test_lm_hamiltonian_is_functional_derivative_of_energy():
    """H phi = dE_KS/d phi^* / f with s, p and d projectors (eq. new_EoM_a)."""
    s = _lm_system(71)
    st = O.init_state(s)
    rng = np.random.default_rng(3)
    chi = 0.05 * (rng.normal(size=st.psi.shape[1:]) + 1j * rng.normal(size=st.psi.shape[1:]))
    A = 1
    H = O.Hamiltonian(st.v_loc + st.v_h + st.v_xc, st.tables, s.species, s.h, s.fd_order)
    ana = 2 * s.occ * s.h ** 3 * float(np.sum((np.conj(chi) * H.apply(st.psi)[A]).real))

    def eks(eps):
        psi = st.psi.copy()
        psi[A] = psi[A] + eps * chi
        rho, vh, ex, vx = O.electron_potentials(psi, s.occ, s.h)
        st2 = O.State(**{**st.__dict__, "psi": psi, "rho": rho, "v_h": vh,
                          "eps_xc": ex, "v_xc": vx})
        return O.energies(st2)["ks"]

    e = 1e-5
    num = (eks(e) - eks(-e)) / (2 * e)
    assert abs(num - ana) < 1e-6 * abs(ana)


def test_lm_nonlocal_term_is_rotation_invariant():
    """Rotating the whole configuration (atoms and orbitals) by a cube
    symmetry of the grid (x -> y -> z -> x) leaves the nonlocal energy
    unchanged: the strength is shared by the m of an l, and the solid
    harmonics of one l span a rotation-invariant space.  A wrong
    normalisation of one m (e.g. without the sqrt(3) of xy) breaks it."""
    s = _lm_system(53)
    st = O.init_state(s)
    c = O.projections(st.psi, st.tables, s.species, s.h)
    e1 = float(np.sum(st.tables.hP[:, None] * np.abs(c) ** 2))
    # (x, y, z) -> (y, z, x): array axes are [z, y, x]
    psi_r = np.transpose(st.psi, (0, 2, 3, 1))
    R_r = st.R[:, [2, 0, 1]]
    t = O.atom_tables(R_r, s.species, s.n, s.h)
    c_r = O.projections(psi_r, t, s.species, s.h)
    e2 = float(np.sum(t.hP[:, None] * np.abs(c_r) ** 2))
    assert abs(e1 - e2) < 1e-12 * abs(e1)
