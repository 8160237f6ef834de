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

Fractional occupations (a reading: the paper's cells are gapped and it
needs none; nearly metallic cells do).  With a smearing width kT > 0 the
n_states lowest eigenstates carry Fermi-Dirac occupations

    f_i = occ / (1 + exp((eps_i - mu_F) / kT)),   sum_i f_i = N_e,

rho = sum_i f_i |phi_i|^2, and the fixed point is the stationary point of
the Mermin free energy F = E_KS - kT S with
S = -sum_i occ [g_i ln g_i + (1 - g_i) ln(1 - g_i)], g_i = f_i / occ.
E_KS is quadratic in each orbital with weight f_i, so it equals the energy
of the same formula with the single weight occ on the orbitals
sqrt(f_i / occ) phi_i; ``GroundState.state`` holds those, for the energies
and forces of ``emd_oracle``.

The mixing may be preconditioned by Kerker's factor G^2 / (G^2 + q0^2) on
the residual (factor 1 at G = 0, where the residual of two densities with
the same charge vanishes); q0 = 0 is plain linear mixing.  Neither choice
moves the fixed point.
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
    occupations: np.ndarray = None   # [n_states] f_i (occ each when kT = 0)
    fermi_level: float = float("nan")
    entropy: float = 0.0             # S (kT S is subtracted from E_KS in F)
    free_energy: float = float("nan")   # F = E_KS - kT S


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


def fermi_dirac(eps: np.ndarray, n_electrons: float, occ: float, kT: float,
                iters: int = 200):
    """Occupations f_i = occ / (1 + exp((eps_i - mu) / kT)) with mu found by
    bisection on sum_i f_i = n_electrons (monotone in mu); returns (f, mu).
    Needs 0 < n_electrons < occ * len(eps)."""
    from scipy.special import expit
    eps = np.asarray(eps, dtype=np.float64)
    if not (0.0 < n_electrons < occ * eps.size) or not kT > 0.0:
        raise ValueError("need kT > 0 and 0 < n_electrons < occ * n_states")
    lo = float(eps.min()) - 50.0 * kT - 1.0
    hi = float(eps.max()) + 50.0 * kT + 1.0
    for _ in range(iters):
        mu = 0.5 * (lo + hi)
        if occ * float(np.sum(expit(-(eps - mu) / kT))) < n_electrons:
            lo = mu
        else:
            hi = mu
    mu = 0.5 * (lo + hi)
    return occ * expit(-(eps - mu) / kT), mu


def smearing_entropy(f: np.ndarray, occ: float) -> float:
    """S = -sum_i occ [g ln g + (1 - g) ln(1 - g)], g = f / occ (0 ln 0 = 0)."""
    from scipy.special import xlogy
    g = np.asarray(f, dtype=np.float64) / occ
    return -occ * float(np.sum(xlogy(g, g) + xlogy(1.0 - g, 1.0 - g)))


def kerker(r: np.ndarray, h: float, q0: float) -> np.ndarray:
    """Kerker's preconditioner on a density residual: r(G) G^2 / (G^2 + q0^2)
    for G != 0, r(0) unchanged."""
    if q0 <= 0.0:
        return r
    n = r.shape[0]
    g = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / (n * h)
    G2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    fac = G2 / (G2 + q0 * q0)
    fac[0, 0, 0] = 1.0
    return np.fft.ifftn(np.fft.fftn(r) * fac).real


def weighted_density(psi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """rho = sum_i f_i |phi_i|^2 (eq. density with per-state weights)."""
    return np.einsum("i,ixyz->xyz", np.asarray(f, dtype=np.float64),
                     psi.real ** 2 + psi.imag ** 2)


def ground_state(sysin, tol: float = 1e-11, max_iter: int = 300,
                 alpha: float = 0.3, kT: float = 0.0, n_electrons=None,
                 kerker_q0: float = 0.0) -> GroundState:
    """Self-consistent ground state at the ions of ``sysin`` (the orbitals of
    ``sysin`` only provide the starting density).

    kT = 0: the n_orb lowest states filled with occ each.  kT > 0: the n_orb
    lowest states (n_orb of ``sysin``) with Fermi-Dirac occupations summing
    to n_electrons (< occ n_orb)."""
    st = O.init_state(sysin)
    n, h, sp = sysin.n, sysin.h, sysin.species
    n_orb = sysin.n_orb
    occ = sysin.occ
    n_e = occ * n_orb if kT <= 0.0 else float(n_electrons)
    rho = st.rho.copy() * (n_e / (occ * n_orb))
    v0 = None
    res = np.inf
    f = np.full(n_orb, occ)
    mu_f = float("nan")
    for it in range(1, max_iter + 1):
        v_h = O.poisson(rho, h)
        _, vxc = O.lda_pz81(rho)
        H = O.Hamiltonian(st.v_loc + v_h + vxc, st.tables, sp, h, sysin.fd_order)
        w, psi = lowest_eigenpairs(H, n, n_orb + 1, v0=v0)
        v0 = psi[0].reshape(-1) * np.sqrt(h ** 3)
        if kT > 0.0:
            f, mu_f = fermi_dirac(w[:n_orb], n_e, occ, kT)
        rho_out = weighted_density(psi[:n_orb], f)
        res = float(np.sum(np.abs(rho_out - rho))) * h ** 3 / n_e
        if res < tol:
            break
        rho = rho + alpha * kerker(rho_out - rho, h, kerker_q0)
    psi_occ = np.ascontiguousarray(psi[:n_orb])
    scaled = psi_occ * np.sqrt(f / occ)[:, None, None, None]
    rho, v_h, eps, vxc = O.electron_potentials(scaled, occ, h)
    final = dataclasses.replace(st, psi=scaled, rho=rho, v_h=v_h, eps_xc=eps,
                                v_xc=vxc, vhxc_hist=[v_h + vxc])
    final.F = O.forces(final)
    S = smearing_entropy(f, occ) if kT > 0.0 else 0.0
    return GroundState(psi=psi_occ, eigenvalues=w[:n_orb], next_eigenvalue=float(w[n_orb]),
                       rho=rho, state=final, iterations=it, residual=res,
                       occupations=f, fermi_level=mu_f, entropy=S,
                       free_energy=O.energies(final)["ks"] - kT * S)
