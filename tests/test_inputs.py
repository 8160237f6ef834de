"""Seeded input generators (host only)."""

import numpy as np

from paper_0812_2801_gb300 import inputs


def test_separable_orthonormalisation_equals_gram_schmidt():
    """The large-grid builder (Gram matrix from 1-D sums, planes by GEMM)
    reproduces Gram-Schmidt in index order of the full-grid orbitals, and
    its result is orthonormal under <a|b> = h^3 sum conj(a) b."""
    R = inputs.jitter(inputs.lattice_sites("sc", 2, 6.0), seed=1)
    h = 0.25
    a = inputs.orthonormalise(inputs.atom_gaussian_orbitals(48, h, R, 3), h)
    b = inputs.orthonormal_gaussian_orbitals(48, h, R, 3)
    assert np.max(np.abs(a - b)) < 1e-13
    f = b.reshape(b.shape[0], -1)
    S = (f.conj() @ f.T) * h ** 3
    assert np.max(np.abs(S - np.eye(S.shape[0]))) < 1e-13
    c = inputs.orthonormal_gaussian_orbitals(48, h, R, 3, dtype=np.complex64)
    assert c.dtype == np.complex64
    assert np.array_equal(c, b.astype(np.complex64))


def test_workloads_are_neutral_and_seeded():
    """N_orb * occ equals the ion charge, and a second build is bitwise equal."""
    for make in (inputs.tiny_fp64, inputs.conservation_c48):
        s1, s2 = make(), make()
        assert s1.n_orb * s1.occ == s1.n_atoms * s1.species.z
        assert np.array_equal(s1.psi, s2.psi) and np.array_equal(s1.R, s2.R)
        assert np.array_equal(s1.V, s2.V)
