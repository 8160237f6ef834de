"""Spectral tools of the vibrational analysis against closed forms (host)."""

import numpy as np

from paper_0812_2801_gb300 import vibrations as vib


def test_power_spectrum_and_fit_find_a_known_frequency():
    w0, dt = 0.0123, 7.0
    t = np.arange(600) * dt                       # ~8 periods
    x = 1.7 + 0.3 * np.cos(w0 * t + 0.4)
    om, p = vib.power_spectrum(x, dt)
    assert abs(vib.peak(om, p) - w0) < 0.02 * w0
    assert abs(vib.fit_frequency(t, x, vib.peak(om, p)) - w0) < 1e-7 * w0


def test_vdos_weights_by_mass_and_ir_uses_the_dipole_derivative():
    dt = 5.0
    t = np.arange(2000) * dt
    wa, wb = 0.01, 0.02
    V = np.zeros((t.size, 2, 3))
    V[:, 0, 2] = np.cos(wa * t)                   # light atom, low frequency
    V[:, 1, 0] = np.cos(wb * t)                   # heavy atom, high frequency
    om, p = vib.vdos(V, [1.0, 10.0], dt)
    assert abs(vib.peak(om, p) - wb) < 0.01 * wb  # the heavy atom dominates
    om, p = vib.vdos(V, [10.0, 1.0], dt)
    assert abs(vib.peak(om, p) - wa) < 0.01 * wa
    D = np.zeros((t.size, 3))
    D[:, 1] = 0.2 * np.sin(wa * t) + 0.2 * np.sin(wb * t)
    om, p = vib.ir_spectrum(D, dt)
    # |FT dD/dt|^2 carries omega^2: the higher line is 4x stronger
    assert abs(vib.peak(om, p) - wb) < 0.01 * wb
    band = (0.5 * wa, 1.5 * wa)
    assert abs(vib.peak(om, p, *band) - wa) < 0.01 * wa


def test_wavenumber_conversion():
    # 1 E_h / hbar in cm^-1 (CODATA): E_h / (h c)
    assert abs(vib.HARTREE_CM1 - 2.1947463136e5) < 1e-3


def test_fit_frequency_from_a_far_guess_and_few_periods():
    """3.2 periods sampled 40 times each; the starting guess 20 % off (a
    typical error of a short record's Fourier peak)."""
    w0 = 0.0051
    t = np.linspace(0.0, 3.2 * 2 * np.pi / w0, 129)
    x = 3.35 + 0.05 * np.cos(w0 * t) + 0.002 * np.cos(2 * w0 * t)
    w = vib.fit_frequency(t, x, 1.2 * w0)
    assert abs(w - w0) < 2e-3 * w0


def test_study_systems_are_neutral_closed_shell_inputs():
    """The N-like dimer: 10 electrons in 5 orthonormal orbitals, bond along
    z through the box centre; the two-atom cell keeps its centre and sets
    the bond length."""
    s = vib.n_dimer(3.3)
    assert s.n_orb * s.occ == s.n_atoms * s.species.z == 10
    f = s.psi.reshape(s.n_orb, -1)
    S = (f.conj() @ f.T) * s.h ** 3
    assert np.max(np.abs(S - np.eye(s.n_orb))) < 1e-12
    assert abs(np.linalg.norm(s.R[1] - s.R[0]) - 3.3) < 1e-12
    assert np.allclose(s.V, 0.0)
    b = vib.pair_base()
    p = vib.pair(2.0, b)
    L = b.n * b.h
    assert abs(vib.bond_length(p.R[None], L)[0] - 2.0) < 1e-12
    mid_b = b.R[0] + 0.5 * ((b.R[1] - b.R[0]) - L * np.round((b.R[1] - b.R[0]) / L))
    assert np.allclose(0.5 * (p.R[0] + p.R[1]), mid_b)
