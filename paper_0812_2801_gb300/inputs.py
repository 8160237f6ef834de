"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module builds initial conditions only; it holds none of the propagation
arithmetic (no Hamiltonian, no propagator, no density, no forces).  What it
produces is the initial condition of the paper's equations of motion
(Sec. 2, eq. Ehr_ic: orbitals psi(0), positions R(0), velocities Rdot(0)) for
synthetic "Si-like" systems shaped like the paper's large runs (Sec. 6.3:
hundreds of atoms on a real-space grid).  The paper's own molecules need
Troullier-Martins pseudopotential data that is not part of this project, so a
synthetic species stands in (Sec. 5 uses norm-conserving pseudopotentials;
here: an erf-screened local part plus one Gaussian s-projector per atom).

Recipe (every draw is seeded, NumPy PCG64):
  * sites: simple-cubic n^3 lattice with spacing a_lat (site i at (i+1/2)a_lat)
    or bcc (two interpenetrating simple-cubic sublattices), each coordinate
    jittered by U[-0.2, 0.2] bohr (seed 1, or the replica seed);
  * velocities: Maxwell-Boltzmann at 300 K, N(0, k_B T / M) per component,
    centre-of-mass velocity removed (seed 2);
  * orbitals: two per atom, s = exp(-d^2 / (2 sigma^2)) and
    p_z = d_z exp(-d^2 / (2 sigma^2)) with sigma = 1.2 bohr, summed over the
    27 nearest periodic images, times exp(i theta_A) with theta_A ~ U[0, 2 pi)
    (seed 3), then orthonormalised in orbital-index order with the grid inner
    product <a|b> = h^3 sum_r conj(a) b (Cholesky factor of the Gram matrix,
    which is the Gram-Schmidt result in that order);
  * external field amplitudes (only for the field workload): U[-0.01, 0.01]
    a.u. per step (seed 4).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

AMU_IN_ME = 1822.888486          # atomic mass unit in electron masses
KB_HARTREE_PER_K = 3.166811563e-6  # Boltzmann constant in Ha/K


@dataclasses.dataclass(frozen=True)
class Species:
    """Synthetic pseudo-atom (all atomic units).

    z       valence charge Z_J
    mass    ionic mass M_J (electron masses)
    a_loc   width of the Gaussian ion charge, v_loc = -Z erf(r/a_loc)/r
    r_loc   support radius of that Gaussian charge on the grid
    r_c     width of the Gaussian projectors
    h_kb    strength of the separable (Kleinman-Bylander) term, l = 0
    r_proj  support radius of the projectors on the grid
    lmax    highest angular momentum of the separable term (0, 1 or 2):
            projectors p_lm = N_l S_lm(d) exp(-d^2/(2 r_c^2)) for l <= lmax
    h_l     strengths of the l = 1 and l = 2 terms
    """
    z: float = 4.0
    mass: float = 28.0 * AMU_IN_ME
    a_loc: float = 0.8
    r_loc: float = 5.0
    r_c: float = 1.0
    h_kb: float = 1.0
    r_proj: float = 5.0
    lmax: int = 0
    h_l: tuple = (0.0, 0.0)


SI_LIKE = Species()
# five valence electrons: a homonuclear dimer of it is closed-shell (the
# sigma and both pi bonding levels filled, like the paper's N2 example)
N_LIKE = Species(z=5.0, mass=14.0067 * AMU_IN_ME)


@dataclasses.dataclass
class SystemInput:
    """One periodic system: grid, species, ions and orbitals (canonical layout).

    psi has shape [n_orb, N, N, N] (axis order z, y, x; x fastest), complex128.
    R and V have shape [n_atoms, 3] (x, y, z), float64.
    """
    name: str
    n: int
    h: float
    fd_order: int
    species: Species
    R: np.ndarray
    V: np.ndarray
    psi: np.ndarray
    occ: float = 2.0
    mu: float = 1.0
    dt: float = 0.05
    n_steps: int = 1
    field: Optional[np.ndarray] = None

    @property
    def L(self) -> float:
        return self.n * self.h

    @property
    def n_atoms(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_orb(self) -> int:
        return int(self.psi.shape[0])


def lattice_sites(kind: str, n_cells: int, a_lat: float) -> np.ndarray:
    """Sites of a simple-cubic ('sc') or body-centred ('bcc') lattice."""
    idx = np.arange(n_cells, dtype=np.float64)
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    base = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    if kind == "sc":
        return (base + 0.5) * a_lat
    if kind == "bcc":
        return np.concatenate([(base + 0.25) * a_lat, (base + 0.75) * a_lat], axis=0)
    raise ValueError(f"unknown lattice kind {kind!r}")


def jitter(sites: np.ndarray, seed: int, amp: float = 0.2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return sites + rng.uniform(-amp, amp, size=sites.shape)


def maxwell_velocities(n_atoms: int, mass: float, seed: int,
                       temperature: float = 300.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    sigma = math.sqrt(KB_HARTREE_PER_K * temperature / mass)
    v = rng.normal(0.0, sigma, size=(n_atoms, 3))
    return v - v.mean(axis=0, keepdims=True)


def _periodic_gauss_1d(coord: np.ndarray, center: float, L: float, sigma: float,
                       moment: bool) -> np.ndarray:
    """sum over images n in {-1,0,1} of (d^moment) exp(-d^2/(2 sigma^2)), d = x - c - nL."""
    out = np.zeros_like(coord)
    for nimg in (-1, 0, 1):
        d = coord - center - nimg * L
        g = np.exp(-d * d / (2.0 * sigma * sigma))
        out += d * g if moment else g
    return out


def atom_gaussian_orbitals(n: int, h: float, R: np.ndarray, phase_seed: int,
                           sigma: float = 1.2) -> np.ndarray:
    """Two image-summed atom-centred Gaussians (s, p_z) per atom with random phases."""
    L = n * h
    coord = np.arange(n, dtype=np.float64) * h
    n_orb = 2 * R.shape[0]
    rng = np.random.default_rng(phase_seed)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n_orb)
    psi = np.empty((n_orb, n, n, n), dtype=np.complex128)
    for j, (x0, y0, z0) in enumerate(R):
        gx = _periodic_gauss_1d(coord, x0, L, sigma, False)
        gy = _periodic_gauss_1d(coord, y0, L, sigma, False)
        gz = _periodic_gauss_1d(coord, z0, L, sigma, False)
        gz1 = _periodic_gauss_1d(coord, z0, L, sigma, True)
        s = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        pz = gz1[:, None, None] * gy[None, :, None] * gx[None, None, :]
        psi[2 * j] = s * np.exp(1j * theta[2 * j])
        psi[2 * j + 1] = pz * np.exp(1j * theta[2 * j + 1])
    return psi


def orthonormalise(psi: np.ndarray, h: float) -> np.ndarray:
    """Orthonormalise in index order under <a|b> = h^3 sum conj(a) b.

    With the Gram matrix S = h^3 Phi^H Phi = L L^H (Cholesky), Phi L^{-H} is
    exactly what classical Gram-Schmidt in index order produces.
    """
    n_orb = psi.shape[0]
    flat = psi.reshape(n_orb, -1)
    S = (flat.conj() @ flat.T) * h ** 3    # S_AB = <phi_A|phi_B>
    Lc = np.linalg.cholesky(S)             # S = Lc Lc^H, Lc lower triangular
    # rows M Phi with M = conj(Lc)^{-1} (lower, positive diagonal) give
    # conj(M) S M^T = I, i.e. orthonormal rows
    out = np.linalg.solve(Lc.conj(), flat)
    return out.reshape(psi.shape)


def orthonormal_gaussian_orbitals(n: int, h: float, R: np.ndarray, phase_seed: int,
                                  sigma: float = 1.2, dtype=np.complex128,
                                  device=None) -> np.ndarray:
    """``orthonormalise(atom_gaussian_orbitals(...))`` for large grids.

    Each orbital of ``atom_gaussian_orbitals`` is a product
    e^{i theta_A} X_A(x) Y_A(y) Z_A(z) of image-summed 1-D factors, so the
    Gram matrix comes from 1-D sums, S_AB = h^3 e^{i(theta_B - theta_A)}
    (X_A.X_B)(Y_A.Y_B)(Z_A.Z_B), and with M = conj(Lc)^{-1} (S = Lc Lc^H) the
    orthonormal set is sum_B M_AB phi_B, assembled one z-plane at a time as
    (M diag(e^{i theta}) diag(Z(z))) @ (Y (x) X): N_orb^2 N^3 multiply-adds
    in GEMMs instead of Gram-Schmidt over the full grid.  Same result as the
    direct path up to rounding.  ``device``: a torch device for the GEMMs
    (complex128 arithmetic); None uses numpy.
    """
    L = n * h
    coord = np.arange(n, dtype=np.float64) * h
    n_orb = 2 * R.shape[0]
    rng = np.random.default_rng(phase_seed)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n_orb)
    X = np.empty((n_orb, n))
    Y = np.empty((n_orb, n))
    Z = np.empty((n_orb, n))
    for j, (x0, y0, z0) in enumerate(R):
        X[2 * j] = X[2 * j + 1] = _periodic_gauss_1d(coord, x0, L, sigma, False)
        Y[2 * j] = Y[2 * j + 1] = _periodic_gauss_1d(coord, y0, L, sigma, False)
        Z[2 * j] = _periodic_gauss_1d(coord, z0, L, sigma, False)
        Z[2 * j + 1] = _periodic_gauss_1d(coord, z0, L, sigma, True)
    ph = np.exp(1j * theta)
    S = (h ** 3) * (np.conj(ph)[:, None] * ph[None, :]) * (X @ X.T) * (Y @ Y.T) * (Z @ Z.T)
    Lc = np.linalg.cholesky(S)
    M = np.linalg.solve(Lc.conj(), np.eye(n_orb)) * ph[None, :]
    P = (Y[:, :, None] * X[:, None, :]).reshape(n_orb, n * n)     # [B, y n + x]
    out = np.empty((n_orb, n, n, n), dtype=dtype)
    if device is None:
        for z in range(n):
            out[:, z] = ((M * Z[:, z][None, :]) @ P).reshape(n_orb, n, n)
        return out
    import torch
    Mt = torch.from_numpy(M).to(device)
    Zt = torch.from_numpy(Z).to(device)
    Pt = torch.from_numpy(P).to(device=device, dtype=torch.complex128)
    tdt = torch.complex64 if np.dtype(dtype) == np.complex64 else torch.complex128
    for z in range(n):
        plane = (Mt * Zt[:, z][None, :]) @ Pt
        out[:, z] = plane.to(tdt).cpu().numpy().reshape(n_orb, n, n)
    return out


def build_system(name: str, n: int, h: float, fd_order: int, R: np.ndarray,
                 vel_seed: int, phase_seed: int, species: Species = SI_LIKE,
                 mu: float = 1.0, dt: float = 0.05, n_steps: int = 1,
                 field: Optional[np.ndarray] = None) -> SystemInput:
    R = np.ascontiguousarray(R, dtype=np.float64)
    V = maxwell_velocities(R.shape[0], species.mass, vel_seed)
    psi = orthonormalise(atom_gaussian_orbitals(n, h, R, phase_seed), h)
    return SystemInput(name=name, n=n, h=h, fd_order=fd_order, species=species,
                       R=R, V=V, psi=np.ascontiguousarray(psi), mu=mu, dt=dt,
                       n_steps=n_steps, field=field)


# --------------------------------------------------------------------------
# Named workloads.  Sizes follow the paper's large-run shapes (Sec. 6.3).
# --------------------------------------------------------------------------

def tiny_fp64() -> SystemInput:
    """8 atoms (sc 2^3, 4.8 bohr), 16 orbitals, 32^3 grid at 0.3 bohr, order 4."""
    R = jitter(lattice_sites("sc", 2, 4.8), seed=1)
    return build_system("tiny-8at-32^3", 32, 0.3, 4, R, 2, 3,
                        mu=1.0, dt=0.05, n_steps=50)


def precision_c96(mu: float = 10.0) -> SystemInput:
    """64 atoms (sc 4^3, 6.0 bohr), 128 orbitals, 96^3 grid at 0.25 bohr, order 8.

    dt = 0.05 sqrt(mu); mu = 1 uses dt = 0.025 because 0.05 lies outside the
    stability interval of the degree-4 Taylor polynomial on the imaginary axis.
    """
    R = jitter(lattice_sites("sc", 4, 6.0), seed=1)
    dt = 0.025 if mu == 1.0 else 0.05 * math.sqrt(mu)
    return build_system("precision-64at-96^3", 96, 0.25, 8, R, 2, 3,
                        mu=mu, dt=dt, n_steps=1000)


def conservation_c48(mu: float = 10.0) -> SystemInput:
    """8 atoms (sc 2^3, 6.0 bohr), 16 orbitals, 48^3 grid at 0.25 bohr, order 8:
    the 96^3 workload's local structure in a box of 2^3 sites; its density
    peaks near 0.25, so grid points cross r_s = 1 as the orbitals move."""
    R = jitter(lattice_sites("sc", 2, 6.0), seed=1)
    return build_system("conservation-8at-48^3", 48, 0.25, 8, R, 2, 3,
                        mu=mu, dt=0.05 * math.sqrt(mu), n_steps=24)


def field_c64(n_steps: int = 200) -> SystemInput:
    """16 atoms (bcc 2x2x2, a = 9.6), 32 orbitals, 64^3 at 0.3, order 6, field."""
    R = jitter(lattice_sites("bcc", 2, 9.6), seed=1)
    rng = np.random.default_rng(4)
    field = rng.uniform(-0.01, 0.01, size=n_steps)
    return build_system("field-16at-64^3", 64, 0.3, 6, R, 2, 3, mu=10.0,
                        dt=0.05 * math.sqrt(10.0), n_steps=n_steps, field=field)


def large_c160(device=None) -> SystemInput:
    """512 atoms (sc 8^3, 6.0 bohr), 1024 orbitals, 160^3 at 0.3, order 8.

    The orbitals are built by ``orthonormal_gaussian_orbitals`` and held as
    complex64 (33.5 GB; complex128 would be 67 GB on the host), for the
    complex64 form; ``device`` is passed on for the GEMMs."""
    R = jitter(lattice_sites("sc", 8, 6.0), seed=1)
    R = np.ascontiguousarray(R, dtype=np.float64)
    V = maxwell_velocities(R.shape[0], SI_LIKE.mass, 2)
    psi = orthonormal_gaussian_orbitals(160, 0.3, R, 3, dtype=np.complex64, device=device)
    return SystemInput(name="large-512at-160^3", n=160, h=0.3, fd_order=8,
                       species=SI_LIKE, R=R, V=V, psi=psi, mu=50.0,
                       dt=0.05 * math.sqrt(50.0), n_steps=100)


def replica_specs(n_replicas: int = 32, seed: int = 5):
    """Ragged replica shapes: N_a ~ U{8..64} on a random subset of a jittered
    n^3 lattice at 6.0 bohr, n = ceil(N_a^(1/3)); grid 48/64/80 for n = 2/3/4."""
    rng = np.random.default_rng(seed)
    grid_for = {2: (48, 0.25), 3: (64, 0.28125), 4: (80, 0.3)}
    specs = []
    for r in range(n_replicas):
        n_at = int(rng.integers(8, 65))
        nc = 2
        while nc ** 3 < n_at:
            nc += 1
        sites = lattice_sites("sc", nc, 6.0)
        pick = np.sort(rng.choice(sites.shape[0], size=n_at, replace=False))
        jit = rng.uniform(-0.2, 0.2, size=(n_at, 3))
        n, h = grid_for[nc]
        specs.append(dict(n=n, h=h, R=sites[pick] + jit, vel_seed=100 + r,
                          phase_seed=200 + r))
    return specs


def small_replica_specs(n_replicas: int = 16, seed: int = 6):
    """Replicas of the smallest shape of the ragged set: 8 atoms on the 2^3
    lattice at 6.0 bohr, each coordinate jittered by U[-0.2, 0.2], 48^3 at
    0.25 bohr (16 orbitals)."""
    rng = np.random.default_rng(seed)
    sites = lattice_sites("sc", 2, 6.0)
    return [dict(n=48, h=0.25, R=sites + rng.uniform(-0.2, 0.2, size=sites.shape),
                 vel_seed=300 + r, phase_seed=400 + r) for r in range(n_replicas)]


def replica(spec: dict, idx: int) -> SystemInput:
    return build_system(f"replica-{idx}", spec["n"], spec["h"], 8, spec["R"],
                        spec["vel_seed"], spec["phase_seed"], mu=10.0,
                        dt=0.05 * math.sqrt(10.0), n_steps=1)


def small_system(n: int = 16, h: float = 0.3, fd_order: int = 4,
                 n_atoms: int = 2, seed: int = 11, species: Species = SI_LIKE,
                 n_orb: Optional[int] = None) -> SystemInput:
    """A quick test system: atoms at seeded random positions in the box.

    n_orb defaults to 2 n_atoms (charge neutral for Z = 4 and occupation 2);
    a smaller value keeps only the first orbitals.
    """
    rng = np.random.default_rng(seed)
    L = n * h
    R = rng.uniform(0.0, L, size=(n_atoms, 3))
    sysin = build_system(f"small-{n_atoms}at-{n}^3", n, h, fd_order, R,
                         seed + 1, seed + 2, species=species)
    if n_orb is not None and n_orb < sysin.n_orb:
        sysin.psi = np.ascontiguousarray(sysin.psi[:n_orb])
    return sysin


def with_extra_states(sysin: SystemInput, n_extra: int, seed: int = 17) -> SystemInput:
    """``sysin`` with n_extra more orbitals: smooth random functions (complex
    normal noise keeping the Fourier modes |m_a| <= 2 on each axis),
    orthonormalised after the existing ones.  For a smeared ground state,
    whose partially occupied states sit above the n_orb filled ones."""
    n = sysin.n
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_extra, n, n, n)) + 1j * rng.normal(size=(n_extra, n, n, n))
    m = np.abs(np.fft.fftfreq(n, d=1.0 / n))
    low = (m[:, None, None] <= 2) & (m[None, :, None] <= 2) & (m[None, None, :] <= 2)
    d = np.fft.ifftn(np.fft.fftn(d, axes=(1, 2, 3)) * low[None], axes=(1, 2, 3))
    psi = orthonormalise(np.concatenate([sysin.psi, d]), sysin.h)
    return dataclasses.replace(sysin, name=f"{sysin.name}+{n_extra}",
                               psi=np.ascontiguousarray(psi))


WORKLOADS = {
    "tiny": tiny_fp64,
    "precision": precision_c96,
    "field": field_c64,
    "large": large_c160,
}
