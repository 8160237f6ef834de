"""Pins of the ground-state oracle (Sec. 4.1, eqs. EoM_BO_a, EoM_BO_b).

The BO ground state is the minimum of E_KS over orthonormal orbital sets at
fixed ions; the checks below use only that definition, the KS equations it
implies and the aufbau order, not the oracle's iteration.
"""

import numpy as np
import pytest

from paper_0812_2801_gb300 import inputs as I
from oracle import emd_groundstate as G
from oracle import emd_oracle as O


@pytest.fixture(scope="module")
def system():
    return I.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=41, n_orb=4)


@pytest.fixture(scope="module")
def gs(system):
    return G.ground_state(system, tol=1e-11, alpha=0.3)


def _e_ks(st, psi):
    rho, v_h, eps, vxc = O.electron_potentials(psi, st.occ, st.h)
    st2 = O.State(**{**st.__dict__, "psi": psi, "rho": rho, "v_h": v_h,
                      "eps_xc": eps, "v_xc": vxc})
    return O.energies(st2)["ks"]


def _orthonormalise(psi, h):
    f = psi.reshape(psi.shape[0], -1)
    S = (f.conj() @ f.T) * h ** 3
    L = np.linalg.cholesky(S)
    return np.linalg.solve(L.conj(), f).reshape(psi.shape)


def test_ground_state_is_a_constrained_minimum(system, gs):
    """E_KS rises at second order along any orthonormality-preserving
    perturbation that leaves the occupied space: E(eps) - E(0) > 0 and
    shrinks ~100x when eps shrinks 10x (no first-order term).  The
    perturbations are smooth (Fourier modes |m_a| <= 2), where a wrong
    potential in H would show up at first order; white noise would be
    dominated by its large kinetic curvature."""
    st, h = gs.state, system.h
    e0 = _e_ks(st, gs.psi)
    f = gs.psi.reshape(gs.psi.shape[0], -1)
    n = system.n
    m = np.fft.fftfreq(n, d=1.0 / n)
    low = ((np.abs(m)[:, None, None] <= 2) & (np.abs(m)[None, :, None] <= 2)
           & (np.abs(m)[None, None, :] <= 2))
    rng = np.random.default_rng(7)
    for trial in range(3):
        d = rng.normal(size=gs.psi.shape) + 1j * rng.normal(size=gs.psi.shape)
        d = np.fft.ifftn(np.fft.fftn(d, axes=(1, 2, 3)) * low[None], axes=(1, 2, 3))
        dflat = d.reshape(d.shape[0], -1)
        dflat -= (dflat @ f.conj().T) @ f * h ** 3      # leave the occupied span
        d = dflat.reshape(d.shape)
        d /= np.sqrt(np.sum(np.abs(d) ** 2) * h ** 3)
        rises = []
        for eps in (1e-3, 1e-4):
            rises.append(_e_ks(st, _orthonormalise(gs.psi + eps * d, h)) - e0)
        assert rises[0] > 0 and rises[1] > 0, (trial, rises)
        assert 50.0 < rises[0] / rises[1] < 200.0, (trial, rises)


def test_ground_state_satisfies_ks_equations(system, gs):
    """H[rho] phi_A = sum_B phi_B Lambda_BA with rho from the phi themselves,
    Lambda = h^3 Phi^H H Phi Hermitian with the solver's eigenvalues."""
    st, h = gs.state, system.h
    H = O.Hamiltonian(st.v_loc + st.v_h + st.v_xc, st.tables, system.species, h,
                      system.fd_order)
    hp = H.apply(gs.psi)
    f = gs.psi.reshape(gs.psi.shape[0], -1)
    hf = hp.reshape(hp.shape[0], -1)
    lam = (f.conj() @ hf.T) * h ** 3
    assert np.max(np.abs(lam - lam.conj().T)) < 1e-10
    assert np.allclose(np.sort(np.linalg.eigvalsh(lam)), gs.eigenvalues, atol=1e-8)
    resid = hf - lam.T @ f
    scale = np.max(np.abs(hf))
    assert np.max(np.abs(resid)) < 1e-6 * scale


def test_ground_state_aufbau_and_normalisation(system, gs):
    assert np.all(np.diff(gs.eigenvalues) >= 0)
    assert gs.next_eigenvalue > gs.eigenvalues[-1] + 1e-3       # a gap
    f = gs.psi.reshape(gs.psi.shape[0], -1)
    S = (f.conj() @ f.T) * system.h ** 3
    assert np.max(np.abs(S - np.eye(S.shape[0]))) < 1e-10
    assert abs(gs.rho.sum() * system.h ** 3 - system.occ * system.n_orb) < 1e-9
    assert gs.residual < 1e-11


def test_ground_state_independent_of_mixing(system, gs):
    other = G.ground_state(system, tol=1e-11, alpha=0.5)
    assert abs(O.energies(other.state)["ks"] - O.energies(gs.state)["ks"]) < 1e-9
    assert np.max(np.abs(other.rho - gs.rho)) < 1e-7 * np.max(gs.rho)


# --------------------------------------------------------------------------
# Fractional (Fermi-Dirac) occupations.  The fixed point is the stationary
# point of the Mermin free energy F = E_KS - kT S over orthonormal orbitals
# and occupations summing to N_e; the checks use that definition, closed
# forms of the occupation rule and the kT -> 0 limit, not the iteration.
# --------------------------------------------------------------------------

KT = 0.05
N_E = 8.0


def _free_energy(st, phi, f, kT):
    """F = E_KS[rho = sum f |phi|^2] - kT S(f), through the oracle's
    energies on the orbitals sqrt(f / occ) phi."""
    occ = st.occ
    scaled = phi * np.sqrt(np.asarray(f) / occ)[:, None, None, None]
    rho, v_h, eps, vxc = O.electron_potentials(scaled, occ, st.h)
    st2 = O.State(**{**st.__dict__, "psi": scaled, "rho": rho, "v_h": v_h,
                      "eps_xc": eps, "v_xc": vxc})
    return O.energies(st2)["ks"] - kT * G.smearing_entropy(f, occ)


@pytest.fixture(scope="module")
def smeared_system(system):
    return I.with_extra_states(system, 2)          # 6 states for 8 electrons


@pytest.fixture(scope="module")
def gs_smeared(smeared_system):
    return G.ground_state(smeared_system, tol=1e-12, alpha=0.3, kT=KT, n_electrons=N_E)


def test_fermi_dirac_closed_forms():
    occ, kT = 2.0, 0.03
    # two levels symmetric about 0 holding occ electrons: mu = 0 by symmetry
    a = 0.02
    f, mu = G.fermi_dirac(np.array([-a, a]), occ, occ, kT)
    assert abs(mu) < 1e-14
    assert np.allclose(f, occ / (1.0 + np.exp(np.array([-a, a]) / kT)), rtol=0, atol=1e-14)
    # n degenerate levels share N_e equally; mu from g = N_e / (occ n)
    e0, n, ne = -0.3, 5, 3.0
    f, mu = G.fermi_dirac(np.full(n, e0), ne, occ, kT)
    g = ne / (occ * n)
    assert np.allclose(f, ne / n, rtol=0, atol=1e-14)
    assert abs(mu - (e0 + kT * np.log(g / (1.0 - g)))) < 1e-12
    # half filling of every state: S = n occ ln 2
    assert abs(G.smearing_entropy(np.full(4, 1.0), occ) - 4 * occ * np.log(2.0)) < 1e-14
    # a gapped spectrum at small kT fills the lowest states
    f, _ = G.fermi_dirac(np.array([-1.0, -0.9, 0.5, 0.6]), 4.0, occ, 0.005)
    assert np.allclose(f, [2.0, 2.0, 0.0, 0.0], atol=1e-30)
    with pytest.raises(ValueError):
        G.fermi_dirac(np.zeros(3), 6.0, occ, kT)


def test_smeared_occupations_and_charge(smeared_system, gs_smeared):
    gs, occ = gs_smeared, smeared_system.occ
    f_rule = occ / (1.0 + np.exp((gs.eigenvalues - gs.fermi_level) / KT))
    assert np.max(np.abs(gs.occupations - f_rule)) < 1e-13
    assert abs(gs.occupations.sum() - N_E) < 1e-12
    assert abs(gs.rho.sum() * smeared_system.h ** 3 - N_E) < 1e-10
    assert 0.05 < gs.occupations[-2] / occ < 0.95      # genuinely fractional
    assert gs.residual < 1e-12


def test_smeared_ground_state_satisfies_ks_equations(smeared_system, gs_smeared):
    st, h = gs_smeared.state, smeared_system.h
    H = O.Hamiltonian(st.v_loc + st.v_h + st.v_xc, st.tables, smeared_system.species, h,
                      smeared_system.fd_order)
    hp = H.apply(gs_smeared.psi).reshape(gs_smeared.psi.shape[0], -1)
    f = gs_smeared.psi.reshape(gs_smeared.psi.shape[0], -1)
    resid = hp - gs_smeared.eigenvalues[:, None] * f
    assert np.max(np.abs(resid)) < 1e-6 * np.max(np.abs(hp))


def test_free_energy_stationary_in_occupations(smeared_system, gs_smeared):
    """At fixed orbitals, dF/df_A = eps_A + kT ln(g / (1 - g)) is the same
    (mu_F) for every state at the Fermi-Dirac occupations, so a change of
    the occupations that keeps N_e has no first-order term: F(+e) - F(-e)
    is far below the second difference, which is positive."""
    st, gs = gs_smeared.state, gs_smeared
    rng = np.random.default_rng(3)
    for trial in range(3):
        d = rng.normal(size=gs.occupations.size)
        d -= d.mean()
        d /= np.max(np.abs(d))
        e = 1e-4
        fp = _free_energy(st, gs.psi, gs.occupations + e * d, KT)
        fm = _free_energy(st, gs.psi, gs.occupations - e * d, KT)
        f0 = _free_energy(st, gs.psi, gs.occupations, KT)
        d2 = fp + fm - 2.0 * f0
        assert d2 > 0.0, (trial, d2)
        assert abs(fp - fm) < 1e-2 * d2, (trial, fp - fm, d2)


def test_free_energy_stationary_in_orbitals(smeared_system, gs_smeared):
    """At the Fermi-Dirac occupations, F rises at second order under
    rotations among the states (states of different f mix at a cost
    (f_A - f_B)(eps_B - eps_A) > 0) and under smooth perturbations that
    leave their span."""
    st, gs, h = gs_smeared.state, gs_smeared, smeared_system.h
    f0 = _free_energy(st, gs.psi, gs.occupations, KT)
    k = gs.psi.shape[0]
    rng = np.random.default_rng(5)
    from scipy.linalg import expm
    A = rng.normal(size=(k, k)) + 1j * rng.normal(size=(k, k))
    A = A - A.conj().T
    rises = []
    for e in (1e-3, 1e-4):
        U = expm(e * A)
        phi = (U @ gs.psi.reshape(k, -1)).reshape(gs.psi.shape)
        rises.append(_free_energy(st, phi, gs.occupations, KT) - f0)
    assert rises[0] > 0 and rises[1] > 0, rises
    assert 50.0 < rises[0] / rises[1] < 200.0, rises
    n = smeared_system.n
    m = np.fft.fftfreq(n, d=1.0 / n)
    low = ((np.abs(m)[:, None, None] <= 2) & (np.abs(m)[None, :, None] <= 2)
           & (np.abs(m)[None, None, :] <= 2))
    d = rng.normal(size=gs.psi.shape) + 1j * rng.normal(size=gs.psi.shape)
    d = np.fft.ifftn(np.fft.fftn(d, axes=(1, 2, 3)) * low[None], axes=(1, 2, 3))
    f = gs.psi.reshape(k, -1)
    dflat = d.reshape(k, -1)
    dflat -= (dflat @ f.conj().T) @ f * h ** 3
    d = dflat.reshape(d.shape) / np.sqrt(np.sum(np.abs(dflat) ** 2) * h ** 3)
    rises = [_free_energy(st, _orthonormalise(gs.psi + e * d, h), gs.occupations, KT) - f0
             for e in (1e-3, 1e-4)]
    assert rises[0] > 0 and rises[1] > 0, rises
    assert 50.0 < rises[0] / rises[1] < 200.0, rises


def test_small_smearing_reduces_to_integer_ground_state(system, gs):
    """Across the aufbau gap (0.16 Ha) at kT = 0.003 the state above it
    holds ~1e-11 electrons: the smeared fixed point is the integer one."""
    five = I.with_extra_states(system, 1)
    sm = G.ground_state(five, tol=1e-12, alpha=0.3, kT=0.003, n_electrons=N_E)
    assert sm.occupations[-1] < 1e-10
    assert np.max(np.abs(sm.eigenvalues[:4] - gs.eigenvalues)) < 1e-8
    assert np.max(np.abs(sm.rho - gs.rho)) < 1e-8 * np.max(gs.rho)
    e_int = O.energies(gs.state)["ks"]
    assert abs(sm.free_energy - e_int) < 1e-9 * abs(e_int)


def test_kerker_factor_on_plane_waves():
    """Kerker's preconditioner multiplies a plane wave of wave vector G by
    |G|^2 / (|G|^2 + q0^2) and leaves a constant alone."""
    n, h, q0 = 12, 0.4, 0.7
    L = n * h
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    m = (1, 2, 3)
    k = 2 * np.pi * np.array(m) / L
    wave = np.cos(k[0] * X + k[1] * Y + k[2] * Z)
    g2 = float(k @ k)
    out = G.kerker(wave + 0.25, h, q0)
    assert np.max(np.abs(out - (g2 / (g2 + q0 * q0) * wave + 0.25))) < 1e-13
