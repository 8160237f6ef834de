"""Kohn-Sham ground state at fixed ions: plain CPU oracle.

TEST INFRASTRUCTURE ONLY, like ``emd_oracle``: imported by ``tests/`` alone;
it shares no code with the CUDA library.

The BO ground state of the paper (Sec. 4.1, eqs. EoM_BO_a and EoM_BO_b) is a
set of orthonormal orbitals phi_A that satisfy H_KS[rho] phi_A =
sum_B Lambda_AB phi_B with rho built from them, and that occupy the lowest
eigenstates of that H; it is the orbital set phi_gs(R) of eq. EoM_BO_2, the
minimum of E_KS (eq. E_KS) at fixed R under the orthonormality constraint.
The paper gives no algorithm for it.  Here it is found by the plainest
fixed-point iteration on the density:

    rho -> H[rho] -> its n_orb lowest eigenvectors (a library eigensolver on
    the matrix-free H of ``emd_oracle``) -> rho_out;
    rho <- rho + alpha (rho_out - rho)

until h^3 sum |rho_out - rho| / N_e < tol.  The fixed point does not depend
on the mixing; the solver does not enter the result.  The library
eigensolver (ARPACK through scipy, on the Hermitian operator) is one step.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import emd_oracle as O


@dataclasses.dataclass
class GroundState:
    psi: np.ndarray          # [n_orb][N][N][N], h^3-orthonormal eigenvectors
    eigenvalues: np.ndarray  # [n_orb] ascending
    next_eigenvalue: float   # the lowest unoccupied eigenvalue (aufbau check)
    rho: np.ndarray          # density of psi
    state: O.State           # oracle state at (R, psi), for energies/forces
    iterations: int
    residual: float          # h^3 sum |rho_out - rho_in| / N_e at the end


def lowest_eigenpairs(H: O.Hamiltonian, n: int, k: int, v0=None, tol: float = 1e-13):
    """The k lowest eigenpairs of the (Hermitian) grid Hamiltonian, with the
    eigenvectors normalised to h^3 sum |phi|^2 = 1."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    N = n ** 3

    def mv(x):
        return H.apply(x.reshape(1, n, n, n)).reshape(N)

    op = LinearOperator((N, N), matvec=mv, dtype=np.complex128)
    w, U = eigsh(op, k=k, which="SA", tol=tol, v0=v0, ncv=max(2 * k + 1, 20))
    order = np.argsort(w)
    w, U = w[order], U[:, order]
    psi = (U.T / np.sqrt(H.h ** 3)).reshape(k, n, n, n)
    return w, psi


def ground_state(sysin, tol: float = 1e-11, max_iter: int = 300,
                 alpha: float = 0.3) -> GroundState:
    """Self-consistent ground state at the ions of ``sysin`` (the orbitals of
    ``sysin`` only provide the starting density)."""
    st = O.init_state(sysin)
    n, h, sp = sysin.n, sysin.h, sysin.species
    n_orb = sysin.n_orb
    n_e = sysin.occ * n_orb
    rho = st.rho.copy()
    v0 = None
    res = np.inf
    for it in range(1, max_iter + 1):
        v_h = O.poisson(rho, h)
        _, vxc = O.lda_pz81(rho)
        H = O.Hamiltonian(st.v_loc + v_h + vxc, st.tables, sp, h, sysin.fd_order)
        w, psi = lowest_eigenpairs(H, n, n_orb + 1, v0=v0)
        v0 = psi[0].reshape(-1) * np.sqrt(h ** 3)
        rho_out = O.density(psi[:n_orb], sysin.occ)
        res = float(np.sum(np.abs(rho_out - rho))) * h ** 3 / n_e
        if res < tol:
            break
        rho = rho + alpha * (rho_out - rho)
    psi_occ = np.ascontiguousarray(psi[:n_orb])
    rho, v_h, eps, vxc = O.electron_potentials(psi_occ, sysin.occ, h)
    final = dataclasses.replace(st, psi=psi_occ, rho=rho, v_h=v_h, eps_xc=eps,
                                v_xc=vxc, vhxc_hist=[v_h + vxc])
    final.F = O.forces(final)
    return GroundState(psi=psi_occ, eigenvalues=w[:n_orb], next_eigenvalue=float(w[n_orb]),
                       rho=rho, state=final, iterations=it, residual=res)
