"""Energy conservation of eq. E_new on the GPU.

E = sum_J M |V_J|^2 / 2 + E_KS is a constant of the modified Ehrenfest
motion (Sec. 4); the time-reversible discretisation (Sec. 5.1) leaves an
error that vanishes with dt.  The system used here has grid points whose
density crosses r_s = 1 during the run, where the two branches of the PZ81
correlation meet, so a functional that is not continuous there (and hence an
H that is not the derivative of E) would show a deviation independent of dt.
"""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emd():
    from paper_0812_2801_gb300 import emd as E
    E.load()
    return E


def _trace(emd, s, precision, dt, n_steps):
    sysg = emd.System(s, precision)
    E = [sysg.energy()["total"]]
    for _ in range(n_steps):
        sysg.propagate(1, dt=dt)
        E.append(sysg.energy()["total"])
    _, _, _, rho = sysg.state(want_psi=False, want_rho=True)
    sysg.close()
    return np.asarray(E), rho


def test_energy_deviation_converges_with_dt_across_rs_one(emd):
    from paper_0812_2801_gb300 import inputs
    s = inputs.conservation_c48(mu=10.0)
    rho1 = 3.0 / (4.0 * math.pi)
    from oracle import emd_oracle as O          # initial density only
    rho0 = O.density(s.psi, s.occ)
    E1, rho_end = _trace(emd, s, emd.EMD_FP64, s.dt, 12)
    E2, _ = _trace(emd, s, emd.EMD_FP64, 0.5 * s.dt, 24)
    crossed = int(np.sum((rho0 > rho1) != (rho_end > rho1)))
    assert crossed >= 20, crossed
    e0 = abs(E1[0])
    d1 = np.max(np.abs(E1 - E1[0])) / e0
    d2 = np.max(np.abs(E2 - E2[0])) / e0
    # second order in dt (measured ratio 3.5 in the oracle); a jump of
    # rho h^3 * 3.2e-5 Ha per crossing would put ~5e-7 into both
    assert d2 < 5e-8, (d1, d2)
    assert d1 / d2 > 2.8, (d1, d2)


def test_fp32_energy_changes_track_fp64(emd):
    from paper_0812_2801_gb300 import inputs
    s = inputs.conservation_c48(mu=10.0)
    E64, _ = _trace(emd, s, emd.EMD_FP64, s.dt, 24)
    E32, _ = _trace(emd, s, emd.EMD_FP32_ORBITALS, s.dt, 24)
    e0 = abs(E64[0])
    # the complex64 energy carries a fixed offset from the rounded orbitals
    assert abs(E32[0] - E64[0]) / e0 < 1e-5
    # its changes along the run follow the FP64 run's
    diff = np.abs((E32 - E32[0]) - (E64 - E64[0])) / e0
    assert np.max(diff) < 1e-7, np.max(diff)
