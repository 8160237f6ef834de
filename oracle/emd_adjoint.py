"""FP64 reference gradients for the adjoint (backward-in-time) propagation.

TEST INFRASTRUCTURE ONLY (used by tests/ like the rest of oracle/).

The forward map is the oracle's MD step with the ions held fixed (Sec. 5.1,
eq. aetrs with Taylor-4 halves, tau = dt/(2 mu) as in eq. transf; the density
of eq. density feeds the Hartree + LDA potential, whose value at t+dt is
extrapolated from the previous steps), restated in plain PyTorch CPU
operations in float64/complex128 so that reverse-mode differentiation gives
the exact discrete adjoint of the written forward map.  A uniform field e_n
along z acts through v_ext = e_n (z - L/2) during step n.

Observables of the final state (n steps):
  dipole  D_z = -h^3 sum_r rho(r) s(z) + sum_J Z s(R_J,z),  s = z - L/2 folded
  energy  E_KS of eq. E_KS (kinetic + nonlocal + electrostatic + xc), the
          field term excluded.
Gradients are taken with respect to the (fixed) ion positions R and every
field amplitude e_n.

The supports of the Gaussian charge and projector (which grid points lie
within r_loc / r_proj) are integer decisions taken once from the numpy
oracle's tables at R; the values on them are differentiable functions of R.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import emd_oracle as O


def _support_tensors(tables: O.AtomTables):
    loc = [(torch.as_tensor(idx), torch.as_tensor(np.stack([dx, dy, dz], 1)))
           for (idx, dx, dy, dz) in tables.loc]
    proj = [(torch.as_tensor(idx), torch.as_tensor(np.stack([dx, dy, dz], 1)))
            for (idx, dx, dy, dz) in tables.proj]
    return loc, proj


class TorchStep:
    """Differentiable restatement of the fixed-ion MD step."""

    def __init__(self, sysin):
        self.s = sysin
        self.n, self.h, self.sp = sysin.n, sysin.h, sysin.species
        if int(getattr(self.sp, "lmax", 0)) > 0:
            raise NotImplementedError("the adjoint reference covers the s-projector only")
        self.L = self.n * self.h
        self.order = sysin.fd_order
        self.c = torch.as_tensor(O.fd_coefficients(self.order))
        tables = O.atom_tables(sysin.R, self.sp, self.n, self.h)
        self.loc, self.proj = _support_tensors(tables)
        self.R0 = torch.as_tensor(np.array(sysin.R))
        n = self.n
        m = np.fft.fftfreq(n, d=1.0 / n)
        g = 2.0 * math.pi * m / self.L
        G2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
        G2[0, 0, 0] = 1.0
        kern = 4.0 * math.pi / G2
        kern[0, 0, 0] = 0.0
        self.kern = torch.as_tensor(kern)
        z = np.arange(n) * self.h
        self.saw = torch.as_tensor(np.broadcast_to((z - 0.5 * self.L)[:, None, None], (n, n, n)).copy())

    # displacement d = r - R_image on the fixed supports, differentiable in R
    def _disp(self, d0, R, J):
        return d0 - (R[J] - self.R0[J])

    def ion_charge(self, R):
        sp = self.sp
        out = torch.zeros(self.n ** 3, dtype=torch.float64)
        for J, (idx, d0) in enumerate(self.loc):
            d = self._disp(d0, R, J)
            d2 = (d * d).sum(1)
            val = sp.z * math.pi ** -1.5 * sp.a_loc ** -3 * torch.exp(-d2 / sp.a_loc ** 2)
            out = out.index_add(0, idx, val)
        return out.reshape(self.n, self.n, self.n)

    def projector_values(self, R):
        sp = self.sp
        vals = []
        for J, (idx, d0) in enumerate(self.proj):
            d = self._disp(d0, R, J)
            d2 = (d * d).sum(1)
            vals.append(math.pi ** -0.75 * sp.r_c ** -1.5 * torch.exp(-d2 / (2 * sp.r_c ** 2)))
        return vals

    def poisson(self, rho):
        return torch.fft.ifftn(torch.fft.fftn(rho) * self.kern).real

    def lda(self, rho):
        P = O.PZ81_C1
        r = torch.clamp(rho, min=1e-30)
        ex = -0.75 * (3.0 * r / math.pi) ** (1.0 / 3.0)
        vx = (4.0 / 3.0) * ex
        rs = (3.0 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
        hi = rs >= 1.0
        rs_hi = torch.where(hi, rs, torch.ones_like(rs))
        rs_lo = torch.where(hi, 0.5 * torch.ones_like(rs), rs)
        s = torch.sqrt(rs_hi)
        q = 1.0 + P["beta1"] * s + P["beta2"] * rs_hi
        ec_hi = P["gamma"] / q
        vc_hi = P["gamma"] * (1.0 + (7.0 / 6.0) * P["beta1"] * s + (4.0 / 3.0) * P["beta2"] * rs_hi) / (q * q)
        lx = torch.log(rs_lo)
        ec_lo = P["A"] * lx + P["B"] + P["C"] * rs_lo * lx + P["D"] * rs_lo
        vc_lo = (P["A"] * lx + (P["B"] - P["A"] / 3.0) + (2.0 / 3.0) * P["C"] * rs_lo * lx
                 + ((2.0 * P["D"] - P["C"]) / 3.0) * rs_lo)
        ec = torch.where(hi, ec_hi, ec_lo)
        vc = torch.where(hi, vc_hi, vc_lo)
        live = rho >= 1e-30
        eps = torch.where(live, ex + ec, torch.zeros_like(rho))
        v = torch.where(live, vx + vc, torch.zeros_like(rho))
        return eps, v

    def kinetic(self, u):
        c = self.c
        out = 3.0 * c[0] * u
        for ax in (-1, -2, -3):
            for k in range(1, len(c)):
                out = out + c[k] * (torch.roll(u, k, ax) + torch.roll(u, -k, ax))
        return -0.5 * out / self.h ** 2

    def projections(self, u, pvals):
        flat = u.reshape(u.shape[0], -1)
        cs = []
        for (idx, _), p in zip(self.proj, pvals):
            cs.append((flat[:, idx] * p.to(flat.dtype)).sum(1) * self.h ** 3)
        return cs

    def apply_h(self, u, v_eff, pvals):
        cs = self.projections(u, pvals)
        flat = torch.zeros(u.shape[0], self.n ** 3, dtype=u.dtype)
        for (idx, _), p, c in zip(self.proj, pvals, cs):
            flat = flat.index_add(1, idx, self.sp.h_kb * c[:, None] * p.to(u.dtype)[None, :])
        return self.kinetic(u) + v_eff[None].to(u.dtype) * u + flat.reshape(u.shape)

    def taylor4(self, psi, tau, v_eff, pvals):
        out = psi
        term = psi
        for k in range(1, 5):
            term = (-1j * tau / k) * self.apply_h(term, v_eff, pvals)
            out = out + term
        return out

    def density(self, psi):
        return self.s.occ * (psi.real ** 2 + psi.imag ** 2).sum(0)

    def run(self, R, field, n_steps, dt, mu):
        """Final (psi, rho, v_loc, pvals) after n_steps fixed-ion steps."""
        psi = torch.as_tensor(np.array(self.s.psi))
        g = self.ion_charge(R)
        v_loc = self.poisson(-g)
        pvals = self.projector_values(R)
        rho = self.density(psi)
        _, vxc = self.lda(rho)
        hist = [self.poisson(rho) + vxc]
        tau = 0.5 * (dt / mu)
        for i in range(n_steps):
            e = field[i]
            if len(hist) == 1:
                x = hist[0]
            elif len(hist) == 2:
                x = 2.0 * hist[0] - hist[1]
            else:
                x = 3.0 * hist[0] - 3.0 * hist[1] + hist[2]
            v1 = v_loc + hist[0] + e * self.saw
            v2 = v_loc + x + e * self.saw
            psi = self.taylor4(self.taylor4(psi, tau, v1, pvals), tau, v2, pvals)
            rho = self.density(psi)
            _, vxc = self.lda(rho)
            hist = [self.poisson(rho) + vxc] + hist[:2]
        return psi, rho, g, v_loc, pvals

    def dipole(self, R, rho):
        zw = R[:, 2] - self.L * torch.floor(R[:, 2] / self.L).detach()
        return -self.h ** 3 * (rho * self.saw).sum() + self.sp.z * (zw - 0.5 * self.L).sum()

    def energy_ks(self, R, psi, rho, g, v_loc, pvals):
        h3 = self.h ** 3
        e_kin = self.s.occ * h3 * (psi.conj() * self.kinetic(psi)).real.sum()
        cs = self.projections(psi, pvals)
        e_nl = self.s.occ * self.sp.h_kb * sum((c.real ** 2 + c.imag ** 2).sum() for c in cs)
        v_es = self.poisson(rho) + v_loc
        e_es = 0.5 * h3 * ((rho - g) * v_es).sum() - O.ion_self_energy(R.shape[0], self.sp)
        e_es = e_es + self.short_range(R)
        eps, _ = self.lda(rho)
        e_xc = h3 * (rho * eps).sum()
        return e_kin + e_nl + e_es + e_xc

    def short_range(self, R, r_cut=12.0):
        sp = self.sp
        L = self.L
        s = math.sqrt(2.0) * sp.a_loc
        nmax = int(math.ceil(r_cut / L)) + 1
        Rw = R - L * torch.floor(R / L).detach()
        rng = torch.arange(-nmax, nmax + 1, dtype=torch.float64)
        img = torch.stack(torch.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) * L
        E = torch.zeros((), dtype=torch.float64)
        na = R.shape[0]
        for j in range(na):
            dv = (Rw[j][None, None, :] - Rw[:, None, :] - img[None, :, :]).reshape(-1, 3)
            d2 = (dv * dv).sum(1)
            keep = (d2.detach() < r_cut * r_cut) & (d2.detach() > 0.0)
            dk = torch.sqrt(d2[keep])
            E = E + 0.5 * sp.z ** 2 * (torch.special.erfc(dk / s) / dk).sum()
        return E


def observable(sysin, R, field, n_steps, dt, mu, kind: str):
    st = TorchStep(sysin)
    psi, rho, g, v_loc, pvals = st.run(R, field, n_steps, dt, mu)
    if kind == "dipole":
        return st.dipole(R, rho)
    return st.energy_ks(R, psi, rho, g, v_loc, pvals)


def gradients(sysin, field, n_steps, dt, mu, kind: str):
    """(L, dL/dR [n_atoms, 3], dL/dfield [n_steps]) by reverse-mode
    differentiation of the fixed-ion forward map."""
    R = torch.as_tensor(np.array(sysin.R)).clone().requires_grad_(True)
    f = torch.as_tensor(np.array(field, dtype=np.float64)).clone().requires_grad_(True)
    L = observable(sysin, R, f, n_steps, dt, mu, kind)
    gR, gf = torch.autograd.grad(L, [R, f])
    return float(L.detach()), gR.numpy(), gf.numpy()


# --------------------------------------------------------------------------
# Moving ions: the full MD step (velocity Verlet, forces = -dE_KS/dR at fixed
# orbitals, Sec. 5.1 and eq. new_EoM_b) restated in PyTorch.  The supports at
# each step's positions are taken from the numpy oracle's own trajectory (the
# integer decisions), the values on them are differentiable.
# --------------------------------------------------------------------------

class TorchMD(TorchStep):
    def __init__(self, sysin, n_steps, dt, mu, field):
        super().__init__(sysin)
        self.n_steps, self.dt, self.mu = n_steps, dt, mu
        self.field_np = np.zeros(n_steps) if field is None else np.array(field, dtype=np.float64)
        # trajectory of the numpy oracle -> supports at every step
        self.sup = []
        st = O.init_state(sysin)
        self.sup.append(_support_tensors(st.tables) + (torch.as_tensor(np.array(st.R)),))
        for i in range(n_steps):
            st = O.md_step(st, dt, mu, float(self.field_np[i]))
            self.sup.append(_support_tensors(st.tables) + (torch.as_tensor(np.array(st.R)),))

    def _use(self, k):
        self.loc, self.proj, self.R0 = self.sup[k]

    def forces(self, R, psi, v_es, pvals):
        sp, h3 = self.sp, self.h ** 3
        na = R.shape[0]
        F = []
        vflat = v_es.reshape(-1)
        cs = self.projections(psi, pvals)
        flat = psi.reshape(psi.shape[0], -1)
        rc2 = sp.r_c ** 2
        for J in range(na):
            idx, d0 = self.loc[J]
            d = self._disp(d0, R, J)
            d2 = (d * d).sum(1)
            g = sp.z * math.pi ** -1.5 * sp.a_loc ** -3 * torch.exp(-d2 / sp.a_loc ** 2)
            floc = h3 * ((vflat[idx] * g * (2.0 / sp.a_loc ** 2))[:, None] * d).sum(0)
            pidx, pd0 = self.proj[J]
            pdd = self._disp(pd0, R, J)
            pp = math.pi ** -0.75 * sp.r_c ** -1.5 * torch.exp(-(pdd * pdd).sum(1) / (2 * rc2))
            u = flat[:, pidx]
            dc = h3 * (u[:, :, None] * (pp[:, None] * pdd / rc2)[None].to(u.dtype)).sum(1)
            fnl = -2.0 * sp.h_kb * self.s.occ * (cs[J].conj()[:, None] * dc).real.sum(0)
            F.append(floc + fnl)
        F = torch.stack(F)
        return F + self.short_range_force(R)

    def short_range_force(self, R, r_cut=12.0):
        sp = self.sp
        L = self.L
        s = math.sqrt(2.0) * sp.a_loc
        nmax = int(math.ceil(r_cut / L)) + 1
        Rw = R - L * torch.floor(R / L).detach()
        rng = torch.arange(-nmax, nmax + 1, dtype=torch.float64)
        img = torch.stack(torch.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) * L
        out = []
        zz = sp.z ** 2
        for j in range(R.shape[0]):
            dv = (Rw[j][None, None, :] - Rw[:, None, :] - img[None, :, :]).reshape(-1, 3)
            d2 = (dv * dv).sum(1)
            keep = (d2.detach() < r_cut * r_cut) & (d2.detach() > 0.0)
            dk = torch.sqrt(d2[keep])
            dvk = dv[keep]
            ef = torch.special.erfc(dk / s) / dk
            fm = zz * (ef / dk + 2.0 / (s * math.sqrt(math.pi)) * torch.exp(-dk * dk / (s * s)) / dk)
            out.append(((fm / dk)[:, None] * dvk).sum(0))
        return torch.stack(out)

    def run_md(self, R, V, field):
        sp, dt, mu = self.sp, self.dt, self.mu
        M = sp.mass
        tau = 0.5 * (dt / mu)
        psi = torch.as_tensor(np.array(self.s.psi))
        self._use(0)
        g = self.ion_charge(R)
        v_loc = self.poisson(-g)
        pv = self.projector_values(R)
        rho = self.density(psi)
        _, vxc = self.lda(rho)
        vh = self.poisson(rho)
        hist = [vh + vxc]
        F = self.forces(R, psi, vh + v_loc, pv)
        for i in range(self.n_steps):
            e = field[i]
            R_new = R + V * dt + F * (dt * dt / (2.0 * M))
            self._use(i + 1)
            g_new = self.ion_charge(R_new)
            v_loc_new = self.poisson(-g_new)
            pv_new = self.projector_values(R_new)
            if len(hist) == 1:
                x = hist[0]
            elif len(hist) == 2:
                x = 2.0 * hist[0] - hist[1]
            else:
                x = 3.0 * hist[0] - 3.0 * hist[1] + hist[2]
            self._use(i)
            psi1 = self.taylor4(psi, tau, v_loc + hist[0] + e * self.saw, pv)
            self._use(i + 1)
            psi = self.taylor4(psi1, tau, v_loc_new + x + e * self.saw, pv_new)
            rho = self.density(psi)
            _, vxc = self.lda(rho)
            vh = self.poisson(rho)
            hist = [vh + vxc] + hist[:2]
            F_new = self.forces(R_new, psi, vh + v_loc_new, pv_new)
            F_new = F_new + torch.stack([torch.zeros_like(e), torch.zeros_like(e), sp.z * e])[None, :]
            V = V + (F + F_new) * (dt / (2.0 * M))
            R, F, g, v_loc, pv = R_new, F_new, g_new, v_loc_new, pv_new
        return psi, rho, g, v_loc, pv, R, V

    def total_energy(self, psi, rho, g, v_loc, pv, R, V):
        return self.energy_ks(R, psi, rho, g, v_loc, pv) + 0.5 * self.sp.mass * (V * V).sum()


def gradients_md(sysin, field, n_steps, dt, mu, kind: str):
    """(L, dL/dR(0), dL/dfield) for the moving-ion dynamics; kind 'dipole'
    (final D_z) or 'energy' (final E_KS + sum M V^2 / 2)."""
    T = TorchMD(sysin, n_steps, dt, mu, field)
    R = torch.as_tensor(np.array(sysin.R)).clone().requires_grad_(True)
    V = torch.as_tensor(np.array(sysin.V))
    f = torch.as_tensor(np.array(T.field_np)).clone().requires_grad_(True)
    psi, rho, g, v_loc, pv, Rn, Vn = T.run_md(R, V, f)
    if kind == "dipole":
        L = T.dipole(Rn, rho)
    else:
        L = T.total_energy(psi, rho, g, v_loc, pv, Rn, Vn)
    gR, gf = torch.autograd.grad(L, [R, f])
    return float(L.detach()), gR.numpy(), gf.numpy()
