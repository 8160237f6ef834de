"""Several Gaussian-type projectors per atom (l <= 2) on the GPU, FP64 form,
against the FP64 oracle (the separable term of Sec. 5's norm-conserving
pseudopotentials with one strength per angular momentum).

Tolerances as for the s-projector: single operators 1e-12 relative, forces
and energies 1e-10 at the initial state and 1e-9 after MD steps, psi 1e-10.
"""
import numpy as np
import pytest

from oracle import emd_oracle as O
from paper_0812_2801_gb300 import emd, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def lm_system(lmax, seed=41):
    sp = inputs.Species(r_c=0.8, r_proj=3.4, lmax=lmax, h_l=(0.6, -0.35))
    return inputs.small_system(n=24, h=0.3, fd_order=6, n_atoms=3, seed=seed, species=sp)


@pytest.mark.parametrize("lmax", [1, 2])
def test_initial_state_and_hamiltonian_match_oracle(lmax):
    s = lm_system(lmax)
    nch = (lmax + 1) ** 2
    st = O.init_state(s)
    g = emd.System(s, emd.EMD_FP64)
    c = emd.emd_get_projections(g.handle, s.n_atoms, s.n_orb, nch)
    assert c.shape[0] == len(st.tables.pmerged)
    assert rel(c, O.projections(st.psi, st.tables, s.species, s.h)) < 1e-12
    assert rel(g.forces(), st.F) < 1e-10
    eg, eo = g.energy(), O.energies(st)
    for k in ("nl", "kin_e", "es", "xc", "total"):
        assert abs(eg[k] - eo[k]) <= 1e-10 * max(abs(eo[k]), 1e-12), k
    rng = np.random.default_rng(7)
    u = rng.normal(size=(5, s.n, s.n, s.n)) + 1j * rng.normal(size=(5, s.n, s.n, s.n))
    H = O.Hamiltonian(st.v_loc + st.v_h + st.v_xc, st.tables, s.species, s.h, s.fd_order)
    assert rel(emd.emd_apply_hamiltonian(g.handle, u), H.apply(u)) < 1e-12
    g.close()


def test_md_steps_match_oracle():
    """10 MD steps with s, p and d projectors (moving ions: the channel
    tables are rebuilt every step)."""
    s = lm_system(2, seed=43)
    n_steps, dt, mu = 10, 0.04, 1.0
    st = O.run(s, n_steps, dt=dt, mu=mu)
    g = emd.System(s, emd.EMD_FP64)
    g.propagate(n_steps, dt=dt, mu=mu)
    R, V, psi, rho = g.state()
    assert np.max(np.abs(psi - st.psi)) < 1e-10
    assert rel(R, st.R) < 1e-12
    assert rel(g.forces(), st.F) < 1e-9
    eg, eo = g.energy(), O.energies(st)
    for k in ("nl", "total"):
        assert abs(eg[k] - eo[k]) <= 1e-9 * abs(eo[k]), k
    g.close()


def test_several_projectors_need_the_double_float_fp64_form():
    s = lm_system(1)
    for prec, bo in ((emd.EMD_FP32_ORBITALS, 0), (emd.EMD_FP64, 4), (emd.EMD_FP64, 1)):
        with pytest.raises(emd.EmdError) as ei:
            emd.emd_init_system(emd.config_for(s, prec, block_orbitals=bo))
        assert ei.value.code == emd.EMD_EINVAL
