"""Plain FP64 CPU oracle of the modified-Ehrenfest TDDFT MD step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
it is used by ``tests/``, by ``__graft_entry__.smoke()`` (to check one small
GPU run) and by the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py``.  It shares no code with the CUDA library; the only module both
sides use is the seeded input generator ``paper_0812_2801_gb300.inputs``.

Everything is written out directly from the paper (arXiv:0812.2801) and the
readings recorded for its silent points; each function names the passage it
follows.  The method computed here is:

* equations of motion (Sec. 4.1, eq. new_EoM): i mu dphi_A/dt = H_KS phi_A and
  M_J d^2R_J/dt^2 = -grad_J E_KS, with E_KS of eq. E_KS on a uniform periodic
  real-space grid with finite-difference derivatives (Sec. 5);
* electrons: AETRS (Sec. 5.1, eq. aetrs) with each exponential replaced by
  its degree-4 Taylor polynomial (Sec. 5.1), in the fictitious time of
  eq. transf, i.e. each half step is exp(-i tau H) with tau = dt / (2 mu);
  H(t+dt) uses the ionic part at R(t+dt) and a Hartree+xc potential
  extrapolated from the previous steps (Sec. 5.1 builds H(t+dt) from earlier
  steps without fixing the order; quadratic extrapolation);
* ions: velocity Verlet (Sec. 5.1) with F = -dE_KS/dR at fixed orbitals
  (eq. new_EoM_b), taken as the exact derivative of the discrete energy;
* density rho = 2 sum_A |phi_A|^2 (eq. density), Hartree potential from a
  periodic spectral Poisson solve, Perdew-Zunger LDA exchange-correlation
  (Sec. 5), ionic potential as a sum over atoms (eq. ionicpotential).

The Taylor polynomial is accumulated term by term (sum_k (-i tau H)^k / k!),
not in the nested (Horner) form the CUDA path uses: the same polynomial with a
different rounding order.  Library primitives used as single steps: numpy's
FFT (Poisson solve), numpy sums and dot products.

Conventions: grid arrays are [z, y, x] (x fastest), point i of an axis sits at
i*h, the box is [0, L)^3 with L = N h, inner product <a|b> = h^3 sum conj(a) b.
Positions R[J] = (x, y, z).  All arithmetic is float64 / complex128.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

FOUR_PI = 4.0 * math.pi

# --------------------------------------------------------------------------
# Finite differences (Sec. 5: real-space grid, finite-difference derivatives)
# --------------------------------------------------------------------------


def fd_coefficients(order: int) -> np.ndarray:
    """Central FD weights [c_0, c_1, ..., c_m] (m = order/2) for d^2/dx^2.

    Closed form of the maximal-order central scheme (Fornberg):
    c_k = 2 (-1)^(k+1) (m!)^2 / (k^2 (m-k)! (m+k)!) for k >= 1 and
    c_0 = -2 sum_k c_k (a constant is annihilated).
    """
    if order not in (2, 4, 6, 8, 10, 12):
        raise ValueError("order must be even, 2..12")
    m = order // 2
    fm = math.factorial(m)
    c = np.zeros(m + 1)
    for k in range(1, m + 1):
        c[k] = 2.0 * (-1.0) ** (k + 1) * fm * fm / (
            k * k * math.factorial(m - k) * math.factorial(m + k))
    c[0] = -2.0 * c[1:].sum()
    return c


def laplacian(u: np.ndarray, h: float, order: int) -> np.ndarray:
    """Periodic FD Laplacian over the last three axes of u."""
    c = fd_coefficients(order)
    out = 3.0 * c[0] * u
    for ax in (-1, -2, -3):
        for k in range(1, len(c)):
            t = np.roll(u, k, axis=ax)
            t += np.roll(u, -k, axis=ax)
            t *= c[k]
            out += t
    out /= h * h
    return out


def kinetic(u: np.ndarray, h: float, order: int) -> np.ndarray:
    """-1/2 nabla^2_FD u (eq. new_EoM_a, first term)."""
    return -0.5 * laplacian(u, h, order)


# --------------------------------------------------------------------------
# Geometry: atoms, periodic images, supports
# --------------------------------------------------------------------------


def wrap(R: np.ndarray, L: float) -> np.ndarray:
    """Positions folded into [0, L): X - L floor(X / L)."""
    return R - L * np.floor(R / L)


def sphere_entries(center: np.ndarray, r_cut: float, n: int, h: float):
    """All (grid point, periodic image) pairs with |d| < r_cut.

    d = (i h - X) - n_img L per axis, images n_img in {-1, 0, 1}^3 around a
    centre already folded into [0, L) (r_cut <= L is required, so no other
    image can reach the box).  Returns flat indices ((z N + y) N + x) and the
    three components of d; a point reached by two images appears twice.
    """
    L = n * h
    if r_cut > L:
        raise ValueError("support radius larger than the box")
    rc2 = r_cut * r_cut
    idx_out, dx_out, dy_out, dz_out = [], [], [], []
    ar = np.arange(n)
    coord = ar * h
    for nz in (-1, 0, 1):
        for ny in (-1, 0, 1):
            for nx in (-1, 0, 1):
                ds = []
                ok = True
                for c, nimg in ((center[0], nx), (center[1], ny), (center[2], nz)):
                    d1 = (coord - c) - nimg * L
                    sel = np.abs(d1) < r_cut
                    if not sel.any():
                        ok = False
                        break
                    ds.append((ar[sel], d1[sel]))
                if not ok:
                    continue
                (ix, dx), (iy, dy), (iz, dz) = ds
                DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
                IZ, IY, IX = np.meshgrid(iz, iy, ix, indexing="ij")
                d2 = DX * DX + DY * DY + DZ * DZ
                m = d2 < rc2
                idx_out.append(((IZ * n + IY) * n + IX)[m])
                dx_out.append(DX[m])
                dy_out.append(DY[m])
                dz_out.append(DZ[m])
    if not idx_out:
        e = np.zeros(0)
        return np.zeros(0, dtype=np.int64), e, e, e
    return (np.concatenate(idx_out), np.concatenate(dx_out),
            np.concatenate(dy_out), np.concatenate(dz_out))


@dataclasses.dataclass
class AtomTables:
    """Per-atom supports at one set of positions.

    loc, proj: [(idx, dx, dy, dz)] per atom, every (point, image) pair;
    pmerged:   [(idx, p)] per projector P = J n_ch + k (channel k of
               channels(sp); P = J for an s-projector only) with p_P(r)
               summed over images, idx unique;
    hP:        strength of projector P (h_kb for l = 0, h_l otherwise).
    """
    loc: list
    proj: list
    pmerged: list
    hP: Optional[np.ndarray] = None


def atom_tables(R: np.ndarray, sp, n: int, h: float) -> AtomTables:
    Rw = wrap(R, n * h)
    loc = [sphere_entries(Rw[j], sp.r_loc, n, h) for j in range(R.shape[0])]
    proj = [sphere_entries(Rw[j], sp.r_proj, n, h) for j in range(R.shape[0])]
    ch = channels(sp)
    pmerged, hP = [], []
    for (idx, dx, dy, dz) in proj:
        uidx, inv = np.unique(idx, return_inverse=True)
        for (l, m) in ch:
            p = np.bincount(inv, weights=projector_lm_values(sp, l, m, dx, dy, dz),
                            minlength=uidx.size)
            pmerged.append((uidx, p))
            hP.append(channel_strength(sp, l))
    return AtomTables(loc=loc, proj=proj, pmerged=pmerged, hP=np.array(hP))


def gaussian_charge_values(sp, dx, dy, dz) -> np.ndarray:
    """g(d) = Z pi^(-3/2) a^(-3) exp(-d^2/a^2): the ion charge whose potential
    is Z erf(d/a)/d, i.e. v_loc = -Z erf(r/a)/r per atom (eq. ionicpotential)."""
    d2 = dx * dx + dy * dy + dz * dz
    a = sp.a_loc
    return sp.z * math.pi ** -1.5 * a ** -3 * np.exp(-d2 / (a * a))


def projector_values(sp, dx, dy, dz) -> np.ndarray:
    """p(d) = pi^(-3/4) r_c^(-3/2) exp(-d^2/(2 r_c^2)) (unit norm in the continuum)."""
    d2 = dx * dx + dy * dy + dz * dz
    rc = sp.r_c
    return math.pi ** -0.75 * rc ** -1.5 * np.exp(-d2 / (2.0 * rc * rc))


# Several projectors per atom.  The paper's norm-conserving pseudopotentials
# (Sec. 5) carry one separable term per angular momentum l; here each l <=
# lmax has 2l + 1 Gaussian-type projectors p_lm(d) = N_l S_lm(d) exp(-d^2 /
# (2 r_c^2)) with the real solid harmonics S_lm normalised so that their
# square integrates over directions to 4 pi r^(2l) / (2l + 1), and one
# strength h_l shared by the m of an l (rotational invariance).

def channels(sp) -> list:
    """(l, m) of the projectors of one atom, in their order within the atom."""
    lmax = int(getattr(sp, "lmax", 0))
    return [(l, m) for l in range(lmax + 1) for m in range(2 * l + 1)]


def channel_strength(sp, l: int) -> float:
    return sp.h_kb if l == 0 else float(sp.h_l[l - 1])


def solid_harmonic(l: int, m: int, dx, dy, dz):
    """S_lm(d) and its gradient (three arrays)."""
    z0 = np.zeros_like(dx)
    one = np.ones_like(dx)
    s3 = math.sqrt(3.0)
    if l == 0:
        return one, (z0, z0, z0)
    if l == 1:
        d = (dx, dy, dz)[m]
        g = [z0, z0, z0]
        g[m] = one
        return d, tuple(g)
    if m == 0:
        return s3 * dx * dy, (s3 * dy, s3 * dx, z0)
    if m == 1:
        return s3 * dy * dz, (z0, s3 * dz, s3 * dy)
    if m == 2:
        return s3 * dz * dx, (s3 * dz, z0, s3 * dx)
    if m == 3:
        return 0.5 * s3 * (dx * dx - dy * dy), (s3 * dx, -s3 * dy, z0)
    return 0.5 * (2.0 * dz * dz - dx * dx - dy * dy), (-dx, -dy, 2.0 * dz)


def projector_norm(l: int, rc: float) -> float:
    """N_l with int p_lm^2 d^3r = 1: N_l^-2 = (4 pi/(2l+1)) int_0^inf
    r^(2l+2) exp(-r^2/r_c^2) dr = (2 pi/(2l+1)) Gamma(l + 3/2) r_c^(2l+3)."""
    return (2.0 * math.pi / (2 * l + 1) * math.gamma(l + 1.5) * rc ** (2 * l + 3)) ** -0.5


def projector_lm_values(sp, l: int, m: int, dx, dy, dz) -> np.ndarray:
    if l == 0:
        return projector_values(sp, dx, dy, dz)
    S, _ = solid_harmonic(l, m, dx, dy, dz)
    d2 = dx * dx + dy * dy + dz * dz
    rc = sp.r_c
    return projector_norm(l, rc) * S * np.exp(-d2 / (2.0 * rc * rc))


def projector_lm_gradient(sp, l: int, m: int, dx, dy, dz):
    """grad_d p_lm = N_l exp(-d^2/(2 r_c^2)) (grad S_lm - S_lm d / r_c^2)."""
    S, gS = solid_harmonic(l, m, dx, dy, dz)
    d2 = dx * dx + dy * dy + dz * dz
    rc = sp.r_c
    e = projector_norm(l, rc) * np.exp(-d2 / (2.0 * rc * rc))
    return tuple(e * (gS[a] - S * d / (rc * rc)) for a, d in enumerate((dx, dy, dz)))


def ion_charge(tables: AtomTables, sp, n: int) -> np.ndarray:
    """sum_J g_J(r) on the grid (eq. ionicpotential, as a charge density)."""
    g = np.zeros(n ** 3)
    for (idx, dx, dy, dz) in tables.loc:
        np.add.at(g, idx, gaussian_charge_values(sp, dx, dy, dz))
    return g.reshape(n, n, n)


# --------------------------------------------------------------------------
# Electrostatics and exchange-correlation (Sec. 5; eq. E_KS)
# --------------------------------------------------------------------------


def poisson(charge: np.ndarray, h: float) -> np.ndarray:
    """Periodic solution of nabla^2 v = -4 pi n: v(G) = 4 pi n(G) / |G|^2, v(0) = 0."""
    n = charge.shape[0]
    L = n * h
    m = np.fft.fftfreq(n, d=1.0 / n)            # integers in [-N/2, N/2)
    g = 2.0 * math.pi * m / L
    G2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    nk = np.fft.fftn(charge)
    G2[0, 0, 0] = 1.0
    vk = FOUR_PI * nk / G2
    vk[0, 0, 0] = 0.0
    return np.fft.ifftn(vk).real


PZ81 = dict(gamma=-0.1423, beta1=1.0529, beta2=0.3334,
            A=0.0311, B=-0.048, C=0.0020, D=-0.0116)


def pz81_continuous(P: dict = PZ81) -> dict:
    """PZ81 with C and D of the r_s < 1 branch fixed by continuity at r_s = 1.

    Matching the value and the first derivative of the two branches at
    r_s = 1 gives, with q = 1 + beta1 + beta2,
        B + D = gamma / q
        A + C + D = -gamma (beta1 / 2 + beta2) / q^2
    The published C and D are these values rounded to four decimals.  With
    the rounded values eps_c jumps by 3.2e-5 Ha at r_s = 1, so the discrete
    E_KS of eq. E_KS is not differentiable there: each grid point whose
    density crosses 3 / (4 pi) changes E by about rho h^3 * 3.2e-5 while H
    (its derivative elsewhere) does not see it, and the energy of eq. E_new
    drifts at a rate set by how often points cross, not by dt.  Continuous
    C and D make H the derivative of E_KS everywhere.
    """
    q = 1.0 + P["beta1"] + P["beta2"]
    D = P["gamma"] / q - P["B"]
    C = -P["gamma"] * (0.5 * P["beta1"] + P["beta2"]) / (q * q) - P["A"] - D
    return {**P, "C": C, "D": D}


PZ81_C1 = pz81_continuous(PZ81)


def lda_pz81(rho: np.ndarray):
    """Unpolarised Perdew-Zunger LDA (Sec. 5) with the continuous C, D of
    ``pz81_continuous``: returns (eps_xc, v_xc).

    eps_x = -(3/4)(3 rho/pi)^(1/3), v_x = (4/3) eps_x.
    r_s >= 1: eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)
    r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s
    v_c = eps_c - (r_s/3) d eps_c / d r_s, written out per branch.
    Points with rho < 1e-30 get eps = v = 0.
    """
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho >= 1e-30
    r = rho[m]
    ex = -0.75 * np.cbrt(3.0 * r / math.pi)
    vx = (4.0 / 3.0) * ex
    rs = np.cbrt(3.0 / (4.0 * math.pi * r))
    P = PZ81_C1
    ec = np.empty_like(r)
    vc = np.empty_like(r)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    q = 1.0 + P["beta1"] * s + P["beta2"] * rs[hi]
    ec[hi] = P["gamma"] / q
    vc[hi] = P["gamma"] * (1.0 + (7.0 / 6.0) * P["beta1"] * s
                           + (4.0 / 3.0) * P["beta2"] * rs[hi]) / (q * q)
    lo = ~hi
    x = rs[lo]
    lx = np.log(x)
    ec[lo] = P["A"] * lx + P["B"] + P["C"] * x * lx + P["D"] * x
    vc[lo] = (P["A"] * lx + (P["B"] - P["A"] / 3.0)
              + (2.0 / 3.0) * P["C"] * x * lx + ((2.0 * P["D"] - P["C"]) / 3.0) * x)
    eps[m] = ex + ec
    v[m] = vx + vc
    return eps, v


def sawtooth_z(n: int, h: float) -> np.ndarray:
    """s(z) = z - L/2 for z in [0, L): length-gauge coordinate of a uniform
    field along z in a periodic box (v_ext = e s(z))."""
    L = n * h
    z = np.arange(n) * h
    return np.broadcast_to((z - 0.5 * L)[:, None, None], (n, n, n)).copy()


def sawtooth_point(zc: np.ndarray, L: float) -> np.ndarray:
    zw = zc - L * np.floor(zc / L)
    return zw - 0.5 * L


def dipole(rho: np.ndarray, R: np.ndarray, z_ion: float, h: float) -> np.ndarray:
    """Dipole of the electrons and ions in the length gauge of a periodic box
    (the sawtooth coordinate of ``sawtooth_z`` along each axis):
    D_a = -h^3 sum_r rho(r) (r_a - L/2) + sum_J Z (R_Ja wrapped - L/2),
    with grid points r_a = i h in [0, L), axes (x, y, z)."""
    n = rho.shape[0]
    L = n * h
    s = np.arange(n) * h - 0.5 * L
    D = np.empty(3)
    # canonical layout rho[z][y][x]
    D[0] = -h ** 3 * np.sum(rho * s[None, None, :])
    D[1] = -h ** 3 * np.sum(rho * s[None, :, None])
    D[2] = -h ** 3 * np.sum(rho * s[:, None, None])
    for a in range(3):
        D[a] += z_ion * np.sum(sawtooth_point(R[:, a], L))
    return D


# --------------------------------------------------------------------------
# Hamiltonian (eq. new_EoM_a) and its pieces
# --------------------------------------------------------------------------


def projections(u: np.ndarray, tables: AtomTables, sp, h: float) -> np.ndarray:
    """c[P, A] = <p_P|u_A> = h^3 sum_r p_P(r) u_A(r) (p real; P = J with an
    s-projector only, J n_ch + k with several)."""
    n_orb = u.shape[0]
    flat = u.reshape(n_orb, -1)
    c = np.zeros((len(tables.pmerged), n_orb), dtype=np.complex128)
    for j, (idx, p) in enumerate(tables.pmerged):
        c[j] = (flat[:, idx] @ p) * h ** 3
    return c


def nonlocal_apply(c: np.ndarray, tables: AtomTables, sp, shape) -> np.ndarray:
    """sum_P h_P |p_P><p_P|u> = sum_P h_P c_P p_P(r)."""
    n_orb = c.shape[1]
    outT = np.zeros((int(np.prod(shape[1:])), n_orb), dtype=np.complex128)
    for j, (idx, p) in enumerate(tables.pmerged):
        outT[idx] += np.outer(p, tables.hP[j] * c[j])  # idx unique per projector
    return outT.T.reshape(shape)


@dataclasses.dataclass
class Hamiltonian:
    """H = -1/2 nabla^2_FD + v_eff(r) + sum_J h_J |p_J><p_J|."""
    v_eff: np.ndarray
    tables: AtomTables
    sp: object
    h: float
    order: int

    def apply(self, u: np.ndarray) -> np.ndarray:
        c = projections(u, self.tables, self.sp, self.h)
        return (kinetic(u, self.h, self.order) + self.v_eff[None] * u
                + nonlocal_apply(c, self.tables, self.sp, u.shape))


def taylor4(psi: np.ndarray, tau: float, H: Hamiltonian) -> np.ndarray:
    """exp(-i tau H) psi by its degree-4 Taylor polynomial (Sec. 5.1),
    accumulated term by term: sum_{k=0..4} (-i tau H)^k psi / k!."""
    out = psi.copy()
    term = psi
    for k in range(1, 5):
        term = (-1j * tau / k) * H.apply(term)
        out = out + term
    return out


def density(psi: np.ndarray, occ: float) -> np.ndarray:
    """rho = f sum_A |phi_A|^2 (eq. density, f = 2 closed shell)."""
    return occ * np.sum(psi.real ** 2 + psi.imag ** 2, axis=0)


# --------------------------------------------------------------------------
# Energy (eq. E_KS, eq. E_new) and forces (eq. new_EoM_b)
# --------------------------------------------------------------------------


def short_range_ion(R: np.ndarray, sp, L: float, r_cut: float = 12.0):
    """E_sr = 1/2 sum' Z_J Z_K erfc(d / (sqrt2 a)) / d over images with d < r_cut,
    and its force -dE_sr/dR_J.  Together with the Gaussian charges on the grid
    and the self term this is the ion-ion sum of eq. E_KS."""
    from scipy.special import erfc
    na = R.shape[0]
    s = math.sqrt(2.0) * sp.a_loc
    nmax = int(math.ceil(r_cut / L)) + 1
    Rw = wrap(R, L)
    rng = np.arange(-nmax, nmax + 1)
    img = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), axis=-1).reshape(-1, 3) * L
    E = 0.0
    F = np.zeros((na, 3))
    zz = sp.z * sp.z
    for j in range(na):
        dv = (Rw[j][None, None, :] - Rw[:, None, :] - img[None, :, :]).reshape(-1, 3)
        d = np.sqrt(np.sum(dv * dv, axis=1))
        keep = (d < r_cut) & (d > 0.0)
        dv, d = dv[keep], d[keep]
        e = erfc(d / s) / d
        E += 0.5 * zz * float(np.sum(e))
        fmag = zz * (e / d + 2.0 / (s * math.sqrt(math.pi)) * np.exp(-d * d / (s * s)) / d)
        F[j] = np.sum((fmag / d)[:, None] * dv, axis=0)
    return E, F


def ion_self_energy(n_atoms: int, sp) -> float:
    """Self energy of the Gaussian charges: sum_J Z_J^2 / (sqrt(2 pi) a)."""
    return n_atoms * sp.z * sp.z / (math.sqrt(2.0 * math.pi) * sp.a_loc)


@dataclasses.dataclass
class State:
    psi: np.ndarray
    R: np.ndarray
    V: np.ndarray
    F: np.ndarray
    tables: AtomTables
    g_ion: np.ndarray
    v_loc: np.ndarray
    rho: np.ndarray
    v_h: np.ndarray
    eps_xc: np.ndarray
    v_xc: np.ndarray
    vhxc_hist: List[np.ndarray]
    n: int
    h: float
    order: int
    sp: object
    occ: float
    step: int = 0
    last_field: float = 0.0


def electron_potentials(psi, occ, h):
    rho = density(psi, occ)
    v_h = poisson(rho, h)
    eps, vxc = lda_pz81(rho)
    return rho, v_h, eps, vxc


def forces(st: State) -> np.ndarray:
    """F_J = -dE_KS/dR_J at fixed orbitals, exact derivative of the discrete
    energy (eq. new_EoM_b; the local part of eq. ionicforces with the gradient
    moved onto the analytic ion charge)."""
    sp, h = st.sp, st.h
    na = st.R.shape[0]
    v_es = (st.v_h + st.v_loc).ravel()
    F = np.zeros((na, 3))
    a2 = sp.a_loc ** 2
    for j, (idx, dx, dy, dz) in enumerate(st.tables.loc):
        g = gaussian_charge_values(sp, dx, dy, dz)
        w = v_es[idx] * g * (2.0 / a2)
        F[j] += h ** 3 * np.array([w @ dx, w @ dy, w @ dz])
    c = projections(st.psi, st.tables, sp, h)
    flat = st.psi.reshape(st.psi.shape[0], -1)
    ch = channels(sp)
    for j, (idx, dx, dy, dz) in enumerate(st.tables.proj):
        u = flat[:, idx]
        for k, (l, m) in enumerate(ch):
            P = j * len(ch) + k
            # p_P depends on r - R_J: d p / d R_J = -grad_d p
            g = projector_lm_gradient(sp, l, m, dx, dy, dz)
            for ax in range(3):
                dc = (u @ (-g[ax])) * h ** 3            # d c_PA / d R_J,ax
                F[j, ax] += -2.0 * st.tables.hP[P] * st.occ * np.sum((np.conj(c[P]) * dc).real)
    _, Fsr = short_range_ion(st.R, sp, st.n * h)
    return F + Fsr


def energies(st: State, V: Optional[np.ndarray] = None) -> dict:
    """Components of E_KS (eq. E_KS) and the conserved E = T_ion + E_KS (eq. E_new)."""
    sp, h = st.sp, st.h
    psi = st.psi
    dv = h ** 3
    e_kin = st.occ * dv * float(np.sum((np.conj(psi) * kinetic(psi, h, st.order)).real))
    c = projections(psi, st.tables, sp, h)
    e_nl = st.occ * float(np.sum(st.tables.hP[:, None] * np.abs(c) ** 2))
    n_tot = st.rho - st.g_ion
    v_es = st.v_h + st.v_loc
    e_sr, _ = short_range_ion(st.R, sp, st.n * h)
    e_es = 0.5 * dv * float(np.sum(n_tot * v_es)) - ion_self_energy(st.R.shape[0], sp) + e_sr
    e_xc = dv * float(np.sum(st.rho * st.eps_xc))
    Vv = st.V if V is None else V
    t_ion = 0.5 * sp.mass * float(np.sum(Vv * Vv))
    e_ks = e_kin + e_nl + e_es + e_xc
    return dict(kin_e=e_kin, nl=e_nl, es=e_es, xc=e_xc, sr=e_sr, kin_ion=t_ion,
                ks=e_ks, total=e_ks + t_ion)


def init_state(sysin) -> State:
    """Initial condition (eq. Ehr_ic): psi(0), R(0), V(0); derived rho(0),
    v_Hxc(0) and F(0)."""
    n, h, sp = sysin.n, sysin.h, sysin.species
    R = np.array(sysin.R, dtype=np.float64)
    tables = atom_tables(R, sp, n, h)
    g = ion_charge(tables, sp, n)
    v_loc = poisson(-g, h)
    psi = np.array(sysin.psi, dtype=np.complex128)
    rho, v_h, eps, vxc = electron_potentials(psi, sysin.occ, h)
    st = State(psi=psi, R=R, V=np.array(sysin.V, dtype=np.float64),
               F=np.zeros_like(R), tables=tables, g_ion=g, v_loc=v_loc, rho=rho,
               v_h=v_h, eps_xc=eps, v_xc=vxc, vhxc_hist=[v_h + vxc], n=n, h=h,
               order=sysin.fd_order, sp=sp, occ=sysin.occ)
    st.F = forces(st)
    return st


def extrapolate_vhxc(hist: List[np.ndarray]) -> np.ndarray:
    """v_Hxc(t+dt) predicted from the stored exact values (most recent first):
    constant, then linear 2v_n - v_(n-1), then quadratic 3v_n - 3v_(n-1) + v_(n-2)."""
    if len(hist) == 1:
        return hist[0].copy()
    if len(hist) == 2:
        return 2.0 * hist[0] - hist[1]
    return 3.0 * hist[0] - 3.0 * hist[1] + hist[2]


def md_step(st: State, dt: float, mu: float, field: float = 0.0,
            frozen_ions: bool = False) -> State:
    """One step: velocity-Verlet positions, AETRS with Taylor-4 halves,
    new density and potentials, new forces, velocity-Verlet velocities
    (Sec. 5.1; eq. aetrs; eq. transf)."""
    sp, h, n = st.sp, st.h, st.n
    tau = 0.5 * (dt / mu)
    s_ext = sawtooth_z(n, h) if field != 0.0 else 0.0
    # H(t): current ionic part and the exact v_Hxc(t)
    H1 = Hamiltonian(st.v_loc + st.vhxc_hist[0] + field * s_ext, st.tables, sp, h, st.order)
    if frozen_ions:
        R_new, tables_new, g_new, v_loc_new = st.R, st.tables, st.g_ion, st.v_loc
    else:
        R_new = st.R + st.V * dt + st.F * (dt * dt / (2.0 * sp.mass))
        tables_new = atom_tables(R_new, sp, n, h)
        g_new = ion_charge(tables_new, sp, n)
        v_loc_new = poisson(-g_new, h)
    H2 = Hamiltonian(v_loc_new + extrapolate_vhxc(st.vhxc_hist) + field * s_ext,
                     tables_new, sp, h, st.order)
    psi = taylor4(taylor4(st.psi, tau, H1), tau, H2)
    rho, v_h, eps, vxc = electron_potentials(psi, st.occ, h)
    hist = [v_h + vxc] + st.vhxc_hist[:2]
    new = dataclasses.replace(st, psi=psi, R=R_new, tables=tables_new, g_ion=g_new,
                              v_loc=v_loc_new, rho=rho, v_h=v_h, eps_xc=eps,
                              v_xc=vxc, vhxc_hist=hist, step=st.step + 1,
                              last_field=field)
    if frozen_ions:
        return new
    F_new = forces(new)
    if field != 0.0:
        F_new = F_new.copy()
        F_new[:, 2] += sp.z * field
    new.V = st.V + (st.F + F_new) * (dt / (2.0 * sp.mass))
    new.F = F_new
    return new


def run(sysin, n_steps: int, dt: Optional[float] = None, mu: Optional[float] = None,
        field: Optional[np.ndarray] = None, frozen_ions: bool = False,
        record=None) -> State:
    dt = sysin.dt if dt is None else dt
    mu = sysin.mu if mu is None else mu
    st = init_state(sysin)
    for i in range(n_steps):
        e = 0.0 if field is None else float(field[i])
        st = md_step(st, dt, mu, e, frozen_ions)
        if record is not None:
            record(st)
    return st


# --------------------------------------------------------------------------
# Point-by-point evaluation for sampled parity at sizes too large to step
# --------------------------------------------------------------------------


def hamiltonian_at_points(u: np.ndarray, v_eff: np.ndarray, c: np.ndarray,
                          R: np.ndarray, sp, h: float, order: int,
                          points, orbitals) -> np.ndarray:
    """(H u)_A(r) at the listed points (z, y, x) and orbitals, one by one.

    u is [n_orb, N, N, N]; c are the projections <p_P|u_A> [n_proj, n_orb].
    """
    n = u.shape[1]
    L = n * h
    cf = fd_coefficients(order)
    Rw = wrap(R, L)
    ch = channels(sp)
    hP = np.array([channel_strength(sp, l) for _ in range(R.shape[0]) for (l, m) in ch])
    out = np.zeros((len(orbitals), len(points)), dtype=np.complex128)
    for pi_, (z, y, x) in enumerate(points):
        pv = np.zeros(R.shape[0] * len(ch))
        for j in range(R.shape[0]):
            for nz in (-1, 0, 1):
                for ny in (-1, 0, 1):
                    for nx in (-1, 0, 1):
                        dx = (x * h - Rw[j, 0]) - nx * L
                        dy = (y * h - Rw[j, 1]) - ny * L
                        dz = (z * h - Rw[j, 2]) - nz * L
                        d2 = dx * dx + dy * dy + dz * dz
                        if d2 < sp.r_proj * sp.r_proj:
                            for k, (l, m) in enumerate(ch):
                                pv[j * len(ch) + k] += projector_lm_values(
                                    sp, l, m, np.array(dx), np.array(dy), np.array(dz))
        for oi, a in enumerate(orbitals):
            lap = 3.0 * cf[0] * u[a, z, y, x]
            for k in range(1, len(cf)):
                lap += cf[k] * (u[a, z, y, (x + k) % n] + u[a, z, y, (x - k) % n]
                                + u[a, z, (y + k) % n, x] + u[a, z, (y - k) % n, x]
                                + u[a, (z + k) % n, y, x] + u[a, (z - k) % n, y, x])
            val = -0.5 * lap / (h * h) + v_eff[z, y, x] * u[a, z, y, x]
            val += np.sum(hP * c[:, a] * pv)
            out[oi, pi_] = val
    return out
