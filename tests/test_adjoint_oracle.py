"""Pins of the reference adjoint (reverse-mode differentiation of the
fixed-ion forward map restated in PyTorch): its forward pass equals the numpy
oracle's, and its gradients equal central finite differences of the numpy
oracle (which rebuilds every support at the displaced positions)."""
import numpy as np
import pytest
import torch

from oracle import emd_adjoint as A
from oracle import emd_oracle as O
from paper_0812_2801_gb300 import inputs

# narrow projector: support jumps at the cut-off are ~1e-15 of the peak, so
# finite differences see the smooth map (the default width is 3.7e-6)
SP = inputs.Species(r_c=0.6)


def small():
    s = inputs.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=81, n_orb=4,
                            species=SP)
    return s


def numpy_observable(s, R, field, n_steps, dt, mu, kind):
    s2 = inputs.SystemInput(**{**s.__dict__, "R": R})
    st = O.run(s2, n_steps, dt=dt, mu=mu, field=field, frozen_ions=True)
    if kind == "dipole":
        saw = O.sawtooth_z(s.n, s.h)
        zs = O.sawtooth_point(R[:, 2], s.n * s.h)
        return -s.h ** 3 * float(np.sum(st.rho * saw)) + s.species.z * float(np.sum(zs))
    return O.energies(st)["ks"]


def test_torch_forward_equals_numpy_oracle():
    s = small()
    field = np.array([0.01, -0.02, 0.005])
    st_np = O.run(s, 3, dt=0.05, mu=1.0, field=field, frozen_ions=True)
    T = A.TorchStep(s)
    psi, rho, g, v_loc, pv = T.run(torch.as_tensor(s.R), torch.as_tensor(field), 3, 0.05, 1.0)
    assert np.max(np.abs(psi.numpy() - st_np.psi)) < 1e-12
    for kind in ("dipole", "energy"):
        val = float(A.observable(s, torch.as_tensor(s.R), torch.as_tensor(field), 3, 0.05, 1.0, kind))
        ref = numpy_observable(s, s.R, field, 3, 0.05, 1.0, kind)
        assert abs(val - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("kind", ["dipole", "energy"])
def test_reference_adjoint_matches_finite_differences(kind):
    s = small()
    n_steps, dt, mu = 3, 0.05, 1.0
    field = np.array([0.01, -0.02, 0.005])
    L, gR, gf = A.gradients(s, field, n_steps, dt, mu, kind)
    h = 1e-4
    for i in range(n_steps):
        fp = field.copy(); fp[i] += h
        fm = field.copy(); fm[i] -= h
        fd = (numpy_observable(s, s.R, fp, n_steps, dt, mu, kind)
              - numpy_observable(s, s.R, fm, n_steps, dt, mu, kind)) / (2 * h)
        assert abs(fd - gf[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, gf[i])
    for j in range(s.n_atoms):
        for ax in range(3):
            Rp = s.R.copy(); Rp[j, ax] += h
            Rm = s.R.copy(); Rm[j, ax] -= h
            fd = (numpy_observable(s, Rp, field, n_steps, dt, mu, kind)
                  - numpy_observable(s, Rm, field, n_steps, dt, mu, kind)) / (2 * h)
            assert abs(fd - gR[j, ax]) <= 1e-5 * max(abs(fd), 1e-2), (j, ax, fd, gR[j, ax])


def numpy_md_observable(s, R, field, n_steps, dt, mu, kind):
    s2 = inputs.SystemInput(**{**s.__dict__, "R": R})
    st = O.run(s2, n_steps, dt=dt, mu=mu, field=field)
    if kind == "dipole":
        saw = O.sawtooth_z(s.n, s.h)
        zs = O.sawtooth_point(st.R[:, 2], s.n * s.h)
        return -s.h ** 3 * float(np.sum(st.rho * saw)) + s.species.z * float(np.sum(zs))
    return O.energies(st)["total"]


def test_torch_md_forward_equals_numpy_oracle():
    s = small()
    s.V = s.V * 200.0
    field = np.array([0.01, -0.02, 0.005])
    T = A.TorchMD(s, 3, 0.05, 1.0, field)
    psi, rho, g, v_loc, pv, R, V = T.run_md(torch.as_tensor(s.R), torch.as_tensor(s.V),
                                             torch.as_tensor(field))
    st = O.run(s, 3, dt=0.05, mu=1.0, field=field)
    assert np.max(np.abs(psi.numpy() - st.psi)) < 1e-12
    assert np.max(np.abs(R.numpy() - st.R)) < 1e-13
    assert np.max(np.abs(V.numpy() - st.V)) < 1e-13


@pytest.mark.parametrize("kind", ["dipole", "energy"])
def test_reference_md_adjoint_matches_finite_differences(kind):
    """Moving ions (fast, so positions change measurably in 3 steps)."""
    s = small()
    s.V = s.V * 200.0
    n_steps, dt, mu = 3, 0.05, 1.0
    field = np.array([0.01, -0.02, 0.005])
    L, gR, gf = A.gradients_md(s, field, n_steps, dt, mu, kind)
    h = 1e-4
    for i in range(n_steps):
        fp = field.copy(); fp[i] += h
        fm = field.copy(); fm[i] -= h
        fd = (numpy_md_observable(s, s.R, fp, n_steps, dt, mu, kind)
              - numpy_md_observable(s, s.R, fm, n_steps, dt, mu, kind)) / (2 * h)
        assert abs(fd - gf[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, gf[i])
    for j in range(s.n_atoms):
        for ax in range(3):
            Rp = s.R.copy(); Rp[j, ax] += h
            Rm = s.R.copy(); Rm[j, ax] -= h
            fd = (numpy_md_observable(s, Rp, field, n_steps, dt, mu, kind)
                  - numpy_md_observable(s, Rm, field, n_steps, dt, mu, kind)) / (2 * h)
            assert abs(fd - gR[j, ax]) <= 1e-5 * max(abs(fd), 1e-2), (j, ax, fd, gR[j, ax])
