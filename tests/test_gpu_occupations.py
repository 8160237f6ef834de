"""Fractional occupations through the C ABI: emd_set_occupations (rho =
sum_A f_A |phi_A|^2, eq. density with a weight per orbital) and the smeared
ground state emd_ground_state_smeared (Fermi-Dirac occupations, Kerker-
preconditioned mixing), against the oracle.

The oracle computes energies, forces and MD steps with per-orbital weights
on the orbitals sqrt(f_A / occ) phi_A (every term of E_KS is quadratic in an
orbital with its weight, and the propagation is linear in each orbital).
"""
import numpy as np
import pytest

from oracle import emd_groundstate as G
from oracle import emd_oracle as O
from paper_0812_2801_gb300 import emd, inputs

pytestmark = pytest.mark.gpu

KT = 0.05
N_E = 8.0


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _scaled(sysin, f):
    w = np.sqrt(np.asarray(f) / sysin.occ)
    return inputs.SystemInput(**{**sysin.__dict__,
                                 "psi": np.ascontiguousarray(sysin.psi * w[:, None, None, None])})


@pytest.fixture(scope="module")
def six():
    s = inputs.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=41, n_orb=4)
    return inputs.with_extra_states(s, 2)


@pytest.fixture(scope="module")
def oracle_gs(six):
    return G.ground_state(six, tol=1e-12, alpha=0.3, kT=KT, n_electrons=N_E)


@pytest.mark.parametrize("precision,tol", [(emd.EMD_FP64, 1e-12), (emd.EMD_FP32_ORBITALS, 1e-6)])
def test_occupation_weights_match_oracle(six, precision, tol):
    """Set f, then orbitals: potentials, projections, energies and forces
    of sum f |phi|^2, and the orbitals read back unweighted."""
    s = six
    f = np.array([2.0, 1.9, 1.5, 1.0, 0.3, 1e-3])
    h = emd.emd_init_system(emd.config_for(s, precision))
    emd.emd_set_occupations(h, f)
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    assert np.array_equal(emd.emd_get_occupations(h, s.n_orb), f)
    st = O.init_state(_scaled(s, f))
    pot = emd.emd_get_potentials(h, s.n)
    assert rel(pot["v_h"], st.v_h) < tol
    assert rel(pot["v_xc"], st.v_xc) < tol
    c = emd.emd_get_projections(h, s.n_atoms, s.n_orb)
    assert rel(c, O.projections(s.psi, st.tables, s.species, s.h)) < 10 * tol
    _, _, psi, rho = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n)
    assert rel(psi, s.psi) < (1e-15 if precision == emd.EMD_FP64 else 1e-6)
    assert rel(rho, G.weighted_density(s.psi, f)) < tol
    e = emd.emd_get_energy(h)
    eo = O.energies(st)
    for k in ("kin_e", "nl", "es", "xc", "total"):
        assert abs(e[k] - eo[k]) <= 10 * tol * abs(eo[k]), k
    assert abs(e["n_elec"] - f.sum()) < max(tol, 1e-10) * f.sum()
    assert rel(emd.emd_get_forces(h, s.n_atoms), st.F) < 100 * tol
    # changing the occupations after the orbitals rescales them in place
    f2 = f[::-1].copy()
    emd.emd_set_occupations(h, f2)
    _, _, psi2, rho2 = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n)
    assert rel(psi2, s.psi) < (1e-15 if precision == emd.EMD_FP64 else 1e-6)
    assert rel(rho2, G.weighted_density(s.psi, f2)) < tol
    emd.emd_destroy(h)


def test_md_with_occupations_matches_oracle(six):
    """4 MD steps with fixed fractional occupations, FP64: orbitals, forces
    and energies at the method's FP64 tolerances."""
    s = six
    f = np.array([2.0, 1.9, 1.5, 1.0, 0.3, 1e-3])
    h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP64))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    emd.emd_set_occupations(h, f)
    emd.emd_propagate(h, 4, 0.04, 1.0)
    R, V, psi, rho = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n)
    F = emd.emd_get_forces(h, s.n_atoms)
    e = emd.emd_get_energy(h)
    emd.emd_destroy(h)
    st = O.run(_scaled(s, f), 4, dt=0.04, mu=1.0)
    w = np.sqrt(f / s.occ)[:, None, None, None]
    assert np.max(np.abs(psi * w - st.psi)) <= 1e-10
    assert rel(rho, st.rho) < 1e-10
    assert rel(R, st.R) < 1e-12
    assert rel(F, st.F) < 1e-9
    eo = O.energies(st)
    for k in ("kin_e", "nl", "es", "xc", "total"):
        assert abs(e[k] - eo[k]) <= 1e-9 * abs(eo[k]), k


def _smeared(s, precision, tol, q0):
    h = emd.emd_init_system(emd.config_for(s, precision))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    w, f, info = emd.emd_ground_state_smeared(h, s.n_orb, KT, N_E, kerker_q0=q0,
                                              max_scf=300, tol=tol)
    e = emd.emd_get_energy(h)
    F = emd.emd_get_forces(h, s.n_atoms)
    _, _, psi, rho = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n)
    fs = emd.emd_get_occupations(h, s.n_orb)
    return h, w, f, info, e, F, psi, rho, fs


@pytest.mark.parametrize("q0", [0.0, 0.8])
def test_smeared_ground_state_fp64_matches_oracle(six, oracle_gs, q0):
    s, gs = six, oracle_gs
    h, w, f, info, e, F, psi, rho, fs = _smeared(s, emd.EMD_FP64, 1e-11, q0)
    emd.emd_destroy(h)
    assert info["residual"] < 1e-11
    assert np.array_equal(f, fs)
    assert np.max(np.abs(w - gs.eigenvalues)) < 1e-8, (w, gs.eigenvalues)
    assert np.max(np.abs(f - gs.occupations)) < 1e-8, (f, gs.occupations)
    assert abs(info["fermi_level"] - gs.fermi_level) < 1e-8
    assert abs(info["entropy"] - gs.entropy) < 1e-8 * abs(gs.entropy)
    eo = O.energies(gs.state)
    assert abs(e["ks"] - eo["ks"]) < 1e-9 * abs(eo["ks"]), (e["ks"], eo["ks"])
    free = e["ks"] - KT * info["entropy"]
    assert abs(free - gs.free_energy) < 1e-9 * abs(gs.free_energy)
    assert abs(e["n_elec"] - N_E) < 1e-10
    assert np.max(np.abs(rho - gs.rho)) < 1e-8 * np.max(gs.rho)
    assert rel(F, gs.state.F) < 1e-7
    fl = psi.reshape(s.n_orb, -1)
    S = (fl.conj() @ fl.T) * s.h ** 3                # unweighted orbitals come back
    assert np.max(np.abs(S - np.eye(s.n_orb))) < 1e-12
    g = gs.psi.reshape(s.n_orb, -1)
    P = (g.conj() @ fl.T) * s.h ** 3                 # each state up to a phase
    assert np.max(np.abs(np.abs(np.diag(P)) - 1.0)) < 1e-7


def test_smeared_ground_state_fp32_matches_oracle(six, oracle_gs):
    s, gs = six, oracle_gs
    h, w, f, info, e, F, psi, rho, fs = _smeared(s, emd.EMD_FP32_ORBITALS, 1e-6, 0.8)
    emd.emd_destroy(h)
    assert info["residual"] < 1e-6
    assert np.max(np.abs(w - gs.eigenvalues)) < 1e-5
    assert np.max(np.abs(f - gs.occupations)) < 1e-4
    assert abs(e["ks"] - O.energies(gs.state)["ks"]) < 1e-6 * abs(gs.free_energy)
    assert np.max(np.abs(rho - gs.rho)) < 1e-5 * np.max(gs.rho)


def test_smeared_ground_state_refusals(six):
    s = six
    h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP64))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    for kT, ne, q0 in ((0.05, 12.0, 0.0), (0.05, 0.0, 0.0), (-0.1, 8.0, 0.0), (0.05, 8.0, -1.0)):
        with pytest.raises(emd.EmdError) as ei:
            emd.emd_ground_state_smeared(h, s.n_orb, kT, ne, kerker_q0=q0)
        assert ei.value.code == emd.EMD_EINVAL
    for bad in (np.array([2.0, 2.0, 2.0, 2.0, 0.0, 0.0]), np.full(6, 2.5)):
        with pytest.raises(emd.EmdError) as ei:
            emd.emd_set_occupations(h, bad)
        assert ei.value.code == emd.EMD_EINVAL
    # the integer ground state resets the occupations to occ
    emd.emd_set_occupations(h, np.full(6, 4.0 / 3.0))
    emd.emd_ground_state(h, s.n_orb, max_scf=300, tol=1e-9)
    assert np.array_equal(emd.emd_get_occupations(h, s.n_orb), np.full(6, 2.0))
    emd.emd_destroy(h)


def test_md_from_smeared_ground_state_conserves_energy(six):
    """From the smeared ground state, 40 steps at mu = 10 with the
    occupations fixed: the total energy is conserved and the orbitals stay
    orthonormal."""
    s = six
    h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP64))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    _, f, _ = emd.emd_ground_state_smeared(h, s.n_orb, KT, N_E, kerker_q0=0.8, tol=1e-10)
    e0 = emd.emd_get_energy(h)
    emd.emd_propagate(h, 40, 0.05 * 10 ** 0.5, 10.0)
    e1 = emd.emd_get_energy(h)
    _, _, psi, _ = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n, want_rho=False)
    assert np.array_equal(emd.emd_get_occupations(h, s.n_orb), f)
    emd.emd_destroy(h)
    assert abs(e1["total"] - e0["total"]) < 1e-6 * abs(e0["total"])
    assert abs(e1["n_elec"] - N_E) < 1e-8
    fl = psi.reshape(s.n_orb, -1)
    assert np.max(np.abs((fl.conj() @ fl.T) * s.h ** 3 - np.eye(s.n_orb))) < 1e-7


def _ks_residuals(sysin, psi_rows, eps, rho):
    """max_r |H[rho] phi - eps phi| / max |H phi| for the given orbitals,
    H the oracle's, built from the GPU's density."""
    sp, n, h = sysin.species, sysin.n, sysin.h
    tables = O.atom_tables(np.asarray(sysin.R, dtype=np.float64), sp, n, h)
    v_loc = O.poisson(-O.ion_charge(tables, sp, n), h)
    _, vxc = O.lda_pz81(rho)
    H = O.Hamiltonian(v_loc + O.poisson(rho, h) + vxc, tables, sp, h, sysin.fd_order)
    hp = H.apply(psi_rows)
    return [float(np.max(np.abs(hp[i] - eps[i] * psi_rows[i])) / np.max(np.abs(hp[i])))
            for i in range(psi_rows.shape[0])]


@pytest.mark.parametrize("name,n_extra,kT,q0", [("c48", 4, 0.01, 0.8)])
def test_smeared_ground_state_of_the_lattice_workloads(name, n_extra, kT, q0):
    """The nearly metallic 48^3 Si-like cell (8 atoms, 16 filled states),
    FP64, with extra states above the 2-per-atom filled ones: converged to
    1e-8 in density; Fermi-Dirac occupations of the returned eigenvalues
    summing to the valence charge; rho = sum f |phi|^2 of the returned
    orbitals; and, with the oracle's H of that density, the KS equations
    hold for the lowest state, the two around the Fermi level and the
    highest one holding more than 1e-3 electrons (a sample)."""
    base = inputs.conservation_c48()
    n_e = base.occ * base.n_orb
    s = inputs.with_extra_states(base, n_extra)
    h = emd.emd_init_system(emd.config_for(s, emd.EMD_FP64))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    w, f, info = emd.emd_ground_state_smeared(h, s.n_orb, kT, n_e, kerker_q0=q0,
                                              max_scf=400, tol=1e-8)
    _, _, psi, rho = emd.emd_get_state(h, s.n_atoms, s.n_orb, s.n)
    emd.emd_destroy(h)
    assert info["residual"] < 1e-8
    f_rule = s.occ / (1.0 + np.exp((w - info["fermi_level"]) / kT))
    assert np.max(np.abs(f - f_rule)) < 1e-12
    assert abs(f.sum() - n_e) < 1e-9 * n_e
    assert np.any((f > 0.02) & (f < 1.98))               # fractional near mu_F
    assert rel(rho, G.weighted_density(psi, f)) < 1e-10
    i_f = int(np.argmin(np.abs(w - info["fermi_level"])))
    i_top = int(np.max(np.nonzero(f > 1e-3)[0]))        # highest state that matters
    pick = sorted({0, max(i_f - 1, 0), i_f, i_top})
    res = _ks_residuals(s, psi[pick], w[pick], rho)
    assert max(res) < 1e-5, (pick, res)
