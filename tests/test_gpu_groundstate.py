"""emd_ground_state (Sec. 4.1, eqs. EoM_BO_a, EoM_BO_b) against the oracle's
self-consistent ground state, through the C ABI.

Both sides iterate to the same fixed point by different routes (dense
Lanczos with linear mixing on the CPU; Chebyshev-filtered subspace
iteration with Anderson mixing on the GPU), so the agreement is set by the
two convergence tolerances and, for complex64 orbitals, their precision.
"""

import numpy as np
import pytest

from paper_0812_2801_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emd():
    from paper_0812_2801_gb300 import emd as E
    E.load()
    return E


@pytest.fixture(scope="module")
def case():
    from oracle import emd_groundstate as G
    from oracle import emd_oracle as O
    s = inputs.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=41, n_orb=4)
    gs = G.ground_state(s, tol=1e-12, alpha=0.3)
    return s, gs, O.energies(gs.state)


def _run(emd, s, precision, tol, degree=16):
    h = emd.emd_init_system(emd.config_for(s, precision))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    w, info = emd.emd_ground_state(h, s.n_orb, max_scf=300, tol=tol, degree=degree)
    e = emd.emd_get_energy(h)
    F = emd.emd_get_forces(h, s.n_atoms)
    _, _, psi, rho = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n)
    return h, w, info, e, F, psi, rho


def test_ground_state_fp64_matches_oracle(emd, case):
    s, gs, eo = case
    h, w, info, e, F, psi, rho = _run(emd, s, emd.EMD_FP64, tol=1e-11)
    emd.emd_destroy(h)
    assert info["residual"] < 1e-11
    assert np.max(np.abs(w - gs.eigenvalues)) < 1e-8, (w, gs.eigenvalues)
    assert abs(info["gap"] - (gs.next_eigenvalue - gs.eigenvalues[-1])) < 1e-5
    assert abs(e["ks"] - eo["ks"]) < 1e-9 * abs(eo["ks"]), (e["ks"], eo["ks"])
    assert np.max(np.abs(rho - gs.rho)) < 1e-8 * np.max(gs.rho)
    scale = np.max(np.abs(gs.state.F))
    assert np.max(np.abs(F - gs.state.F)) < 1e-7 * scale
    # orthonormal Ritz vectors spanning the oracle's occupied space
    f = psi.reshape(s.n_orb, -1)
    S = (f.conj() @ f.T) * s.h ** 3
    assert np.max(np.abs(S - np.eye(s.n_orb))) < 1e-12
    g = gs.psi.reshape(s.n_orb, -1)
    P = (g.conj() @ f.T) * s.h ** 3                 # overlaps with the oracle's set
    assert np.max(np.abs(P.conj().T @ P - np.eye(s.n_orb))) < 1e-8


def test_ground_state_fp32_matches_oracle(emd, case):
    s, gs, eo = case
    h, w, info, e, F, psi, rho = _run(emd, s, emd.EMD_FP32_ORBITALS, tol=1e-6)
    emd.emd_destroy(h)
    assert info["residual"] < 1e-6
    assert np.max(np.abs(w - gs.eigenvalues)) < 1e-5, (w, gs.eigenvalues)
    assert abs(e["ks"] - eo["ks"]) < 1e-6 * abs(eo["ks"]), (e["ks"], eo["ks"])
    assert np.max(np.abs(rho - gs.rho)) < 1e-5 * np.max(gs.rho)


def test_ground_state_solves_ks_equations_through_the_abi(emd, case):
    """With the library's own H (emd_apply_hamiltonian at the new state):
    H phi_A = sum_B phi_B Lambda_BA, Lambda Hermitian with the returned
    eigenvalues."""
    s, _, _ = case
    h, w, info, e, F, psi, rho = _run(emd, s, emd.EMD_FP64, tol=1e-11)
    hp = emd.emd_apply_hamiltonian(h, psi)
    emd.emd_destroy(h)
    f = psi.reshape(s.n_orb, -1)
    hf = hp.reshape(s.n_orb, -1)
    lam = (f.conj() @ hf.T) * s.h ** 3
    assert np.max(np.abs(lam - np.diag(w))) < 1e-8
    assert np.max(np.abs(hf - lam.T @ f)) < 1e-6 * np.max(np.abs(hf))


def test_ground_state_reports_no_convergence(emd, case):
    s, _, _ = case
    h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP64))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    with pytest.raises(emd.EmdError) as ei:
        emd.emd_ground_state(h, s.n_orb, max_scf=2, tol=1e-14, degree=4)
    assert ei.value.code == emd.EMD_ENOTCONV
    # the last iterate is a usable orthonormal state
    _, _, psi, _ = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n, want_rho=False)
    f = psi.reshape(s.n_orb, -1)
    assert np.max(np.abs((f.conj() @ f.T) * s.h ** 3 - np.eye(s.n_orb))) < 1e-12
    emd.emd_propagate(h, 2, 0.05, 1.0)
    emd.emd_destroy(h)


def test_md_from_the_ground_state_stays_adiabatic(emd, case):
    """Started on the BO surface, the electrons stay near the instantaneous
    ground state: over 40 steps (mu = 10) the kinetic energy of the
    electrons changes by orders of magnitude less than from the atom-Gaussian
    start, and the total energy is conserved."""
    s = inputs.SystemInput(**{**case[0].__dict__, "mu": 10.0, "dt": 0.05 * 10.0 ** 0.5})
    runs = {}
    for start in ("gaussians", "ground"):
        h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP64))
        emd.emd_set_ions(h, s.R, s.V)
        emd.emd_set_orbitals(h, s.psi)
        if start == "ground":
            emd.emd_ground_state(h, s.n_orb, max_scf=300, tol=1e-9)
        e0 = emd.emd_get_energy(h)
        emd.emd_propagate(h, 40, s.dt, s.mu)
        e1 = emd.emd_get_energy(h)
        emd.emd_destroy(h)
        runs[start] = (e0, e1)
    for start, bound in (("ground", 1e-6), ("gaussians", 1e-4)):
        e0, e1 = runs[start]
        assert abs(e1["total"] - e0["total"]) < bound * abs(e0["total"]), start
    dk_g = abs(runs["gaussians"][1]["kin_e"] - runs["gaussians"][0]["kin_e"])
    dk_gs = abs(runs["ground"][1]["kin_e"] - runs["ground"][0]["kin_e"])
    assert runs["ground"][0]["ks"] < runs["gaussians"][0]["ks"]
    assert dk_gs < 1e-2 * dk_g, (dk_gs, dk_g)
