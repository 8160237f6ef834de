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
