"""Vibrational analysis of trajectories: how the electronic mass-like
parameter mu shifts vibrational frequencies (the paper's accuracy check of
the modified Ehrenfest dynamics, Sec. 6, with the time-scale argument of
Sec. 4.3 behind the bound on mu).

A trajectory is recorded through the C ABI (positions, velocities and the
dipole of ``emd_get_dipole`` every ``every`` steps).  Spectra are Fourier
powers of the samples after removing the mean and applying a Hann window:

* vibrational density of states: sum_J M_J sum_a |FT v_Ja(t)|^2, the
  Fourier transform of the mass-weighted velocity autocorrelation function
  (Wiener-Khinchin);
* infrared: sum_a |FT dD_a/dt|^2, with the derivative by central
  differences.

Angular frequencies are in atomic units (E_h / hbar); ``HARTREE_CM1``
converts to wavenumbers.

``python -m paper_0812_2801_gb300.vibrations`` runs the study on a
closed-shell N-like dimer (the paper's N2 example with the synthetic
pseudopotential): the BO frequency of the bond from ground-state energies
along it, then MD from the ground state at several mu with dt = c mu (the
paper's time-step rule), each reporting its frequency against the BO one.
"""

from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

HARTREE_CM1 = 219474.6313705    # 1 E_h / hbar in cm^-1


def power_spectrum(x: np.ndarray, dt: float, weights=None):
    """Fourier power of real samples x[t, ...] spaced dt, summed over the
    trailing axes (optionally weighted, one weight per x[0, j] along the
    first trailing axis).  Returns (omega, power), omega >= 0."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[0]
    xs = (x - x.mean(axis=0)).reshape(T, -1)
    w = np.hanning(T)[:, None]
    f = np.fft.rfft(xs * w, axis=0)
    p = np.abs(f) ** 2
    if weights is not None:
        wt = np.repeat(np.asarray(weights, dtype=np.float64),
                       xs.shape[1] // len(weights))
        p = p * wt[None, :]
    omega = 2.0 * math.pi * np.fft.rfftfreq(T, d=dt)
    return omega, p.sum(axis=1)


def vdos(V: np.ndarray, masses, dt: float):
    """Vibrational density of states from velocities V[t, J, 3]."""
    return power_spectrum(V, dt, weights=masses)


def ir_spectrum(D: np.ndarray, dt: float):
    """Infrared spectrum from dipoles D[t, 3] (|FT dD/dt|^2)."""
    D = np.asarray(D, dtype=np.float64)
    dD = np.empty_like(D)
    dD[1:-1] = (D[2:] - D[:-2]) / (2.0 * dt)
    dD[0] = (D[1] - D[0]) / dt
    dD[-1] = (D[-1] - D[-2]) / dt
    return power_spectrum(dD, dt)


def peak(omega: np.ndarray, power: np.ndarray, lo: float = 0.0, hi: float = np.inf) -> float:
    """Frequency of the largest peak in [lo, hi], refined by a parabola
    through the three bins around the maximum of log(power)."""
    idx = np.nonzero((omega >= lo) & (omega <= hi))[0]
    if idx.size == 0:
        raise ValueError("no frequency bins in the requested band")
    k = idx[np.argmax(power[idx])]
    if 0 < k < len(omega) - 1 and np.all(power[k - 1:k + 2] > 0):
        a, b, c = np.log(power[k - 1:k + 2])
        den = a - 2.0 * b + c
        off = 0.5 * (a - c) / den if den != 0.0 else 0.0
        return float(omega[k] + off * (omega[1] - omega[0]))
    return float(omega[k])


def fit_frequency(t: np.ndarray, x: np.ndarray, omega0: float, rel: float = 0.3) -> float:
    """Angular frequency of a single-mode signal x(t): the omega within
    omega0 (1 +- rel) minimising the least-squares residual of
    x ~ a + b cos(omega t) + c sin(omega t) (the linear coefficients are
    solved exactly at each omega)."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)

    def resid(w):
        A = np.stack([np.ones_like(t), np.cos(w * t), np.sin(w * t)], axis=1)
        coef, *_ = np.linalg.lstsq(A, x, rcond=None)
        return float(np.sum((A @ coef - x) ** 2))

    # a grid first (the residual has sidelobes a main-lobe width apart),
    # then golden section within one grid step of the best point
    grid = omega0 * np.linspace(1.0 - rel, 1.0 + rel, 241)
    k = int(np.argmin([resid(w) for w in grid]))
    step = grid[1] - grid[0]
    lo, hi = grid[k] - step, grid[k] + step
    g = 0.5 * (math.sqrt(5.0) - 1.0)
    a, b = hi - g * (hi - lo), lo + g * (hi - lo)
    fa, fb = resid(a), resid(b)
    for _ in range(80):
        if fa < fb:
            hi, b, fb = b, a, fa
            a = hi - g * (hi - lo)
            fa = resid(a)
        else:
            lo, a, fa = a, b, fb
            b = lo + g * (hi - lo)
            fb = resid(b)
    return 0.5 * (lo + hi)


def record(h, n_atoms: int, n_steps: int, dt: float, mu: float, every: int = 1) -> dict:
    """Propagate n_steps MD steps, sampling R, V and the dipole every
    ``every`` steps (and at the start)."""
    from . import emd
    R, V, D, t = [], [], [], []
    done = 0
    while True:
        r, v, _, _ = emd.emd_get_state(h, n_atoms, 1, 1, want_psi=False, want_rho=False)
        R.append(r)
        V.append(v)
        D.append(emd.emd_get_dipole(h))
        t.append(done * dt)
        if done >= n_steps:
            break
        k = min(every, n_steps - done)
        emd.emd_propagate(h, k, dt, mu)
        done += k
    return {"t": np.asarray(t), "R": np.asarray(R), "V": np.asarray(V), "D": np.asarray(D)}


def pair_base():
    """The two-atom cell of the ground-state tests (16^3, h = 0.35, order 4,
    4 orbitals), whose closed-shell ground state has a gap of 0.16 E_h.  (A
    free homonuclear dimer with 8 electrons would leave its highest pair of
    degenerate pi orbitals half filled: no closed-shell gap.)"""
    from . import inputs
    return inputs.small_system(n=16, h=0.35, fd_order=4, n_atoms=2, seed=41, n_orb=4)


def pair(bond: float, base=None, mu: float = 10.0):
    """``base`` (two atoms) with both atoms moved symmetrically along their
    minimum-image bond direction to bond length ``bond``, at rest; the base
    orbitals are the starting guess."""
    import dataclasses
    base = pair_base() if base is None else base
    L = base.n * base.h
    d = base.R[1] - base.R[0]
    d -= L * np.round(d / L)
    u = d / np.linalg.norm(d)
    c = base.R[0] + 0.5 * d
    R = np.stack([c - 0.5 * bond * u, c + 0.5 * bond * u])
    return dataclasses.replace(base, R=R, V=np.zeros_like(base.V), mu=mu,
                               dt=0.05 * math.sqrt(mu))


def n_dimer(bond: float, n: int = 48, h: float = 0.3, fd_order: int = 8, mu: float = 10.0):
    """Two N-like atoms (Z = 5) on the z axis through the box centre, at
    rest: 10 electrons in 5 doubly occupied orbitals, a closed shell.  The
    starting guess is s and p_z on each atom plus p_x on the first,
    orthonormalised."""
    from . import inputs
    L = n * h
    c = 0.5 * L
    R = np.array([[c, c, c - 0.5 * bond], [c, c, c + 0.5 * bond]])
    sp = inputs.N_LIKE
    s = inputs.build_system(f"n-dimer-{bond:.3f}-{n}^3", n, h, fd_order, R, 2, 3,
                            species=sp, mu=mu, dt=0.05 * math.sqrt(mu), n_steps=1)
    x = np.arange(n) * h
    g = [np.exp(-(x - R[0, a]) ** 2 / (2 * 1.2 ** 2)) for a in range(3)]
    px = g[2][:, None, None] * g[1][None, :, None] * ((x - R[0, 0]) * g[0])[None, None, :]
    guess = np.concatenate([inputs.atom_gaussian_orbitals(n, h, R, 3), px[None] + 0j])
    s.psi = np.ascontiguousarray(inputs.orthonormalise(guess, h))
    s.V = np.zeros_like(s.V)
    return s


def bond_length(R: np.ndarray, L: float) -> np.ndarray:
    """Minimum-image distance between atoms 0 and 1 of R[t, 2, 3]."""
    d = R[:, 1] - R[:, 0]
    d -= L * np.round(d / L)
    return np.linalg.norm(d, axis=1)


def ground_state_energy(s, precision, tol: float = 1e-9):
    """E_KS of the ground state at the ions of s, and the handle (caller
    destroys it)."""
    from . import emd
    h = emd.emd_init_system(emd.config_for(s, precision))
    emd.emd_set_ions(h, s.R, s.V)
    emd.emd_set_orbitals(h, s.psi)
    _, info = emd.emd_ground_state(h, s.n_orb, max_scf=400, tol=tol)
    return emd.emd_get_energy(h)["ks"], info, h


def bo_frequency(precision, d0: float, build=None, coarse: float = 0.3, step: float = 0.05,
                 n_side: int = 3, mass: float = None):
    """Harmonic BO frequency of the pair: ground-state energies on a coarse
    bond grid around d0 (step ``coarse``) bracket the minimum, then a fine
    grid (step ``step``) around the coarse minimum gives the minimum and the
    curvature k from a quartic fit; omega = sqrt(k / m_red), m_red = M / 2.
    ``build(d)`` makes the system at bond length d (default ``n_dimer``)."""
    from . import emd
    build = n_dimer if build is None else build

    def energies(ds):
        es = []
        for d in ds:
            e, _, h = ground_state_energy(build(d), precision)
            emd.emd_destroy(h)
            es.append(e)
        return np.asarray(es)

    dc = d0 + coarse * np.arange(-4, 5)
    ec = energies(dc)
    d0 = float(dc[int(np.argmin(ec))])
    ds = d0 + step * np.arange(-n_side, n_side + 1)
    es = energies(ds)
    c = np.polyfit(ds - d0, es, 4)
    p = np.poly1d(c)
    span = n_side * step
    crit = [r.real for r in np.roots(np.polyder(p))
            if abs(r.imag) < 1e-12 and abs(r.real) <= span]
    if not crit:
        raise RuntimeError("no energy minimum inside the bond scan")
    x_eq = min(crit, key=lambda x: p(x))
    k = np.polyder(p, 2)(x_eq)
    m_red = 0.5 * build(d0).species.mass
    omega = math.sqrt(k / m_red) if k > 0 else float("nan")
    return {"bond": d0 + x_eq, "k": float(k), "omega": omega,
            "cm1": omega * HARTREE_CM1,
            "scan": {"d": dc.tolist() + ds.tolist(), "E": ec.tolist() + es.tolist()}}


def study(mus, precision, bond: float, stretch: float = 0.1, periods: float = 4.0,
          omega_bo: float = None, dt_per_mu: float = 0.04, samples_per_period: int = 64,
          build=None):
    """MD of the pair from its ground state at bond + stretch, for each mu
    with dt = dt_per_mu * mu, long enough for ``periods`` BO periods;
    returns the VDOS peak and the fitted frequency of the bond length."""
    from . import emd
    out = []
    for mu in mus:
        dt = dt_per_mu * mu
        T = 2.0 * math.pi / omega_bo
        n_steps = int(math.ceil(periods * T / dt))
        every = max(1, int(T / dt / samples_per_period))
        s = (n_dimer if build is None else build)(bond + stretch)
        s.mu, s.dt = mu, dt
        _, info, h = ground_state_energy(s, precision)
        e0 = emd.emd_get_energy(h)["total"]
        t0 = time.perf_counter()
        tr = record(h, s.n_atoms, n_steps, dt, mu, every)
        wall = time.perf_counter() - t0
        e1 = emd.emd_get_energy(h)["total"]
        emd.emd_destroy(h)
        ds = dt * every
        om, pv = vdos(tr["V"], [s.species.mass] * s.n_atoms, ds)
        band = (0.3 * omega_bo, 3.0 * omega_bo)
        bondlen = bond_length(tr["R"], s.n * s.h)
        w_v = peak(om, pv, *band)
        w_b = fit_frequency(tr["t"], bondlen, w_v)
        out.append({"mu": mu, "dt": dt, "steps": n_steps, "sample_every": every,
                    "omega_vdos_peak": w_v, "omega_bond_fit": w_b,
                    "ratio_to_bo": w_b / omega_bo, "cm1": w_b * HARTREE_CM1,
                    "bond_amplitude": float(0.5 * (bondlen.max() - bondlen.min())),
                    "energy_change_rel": abs(e1 - e0) / abs(e0),
                    "gs_iterations": info["iterations"], "wall_s": wall,
                    "ms_per_step": 1e3 * wall / n_steps})
    return out


def main(argv=None) -> int:
    from . import emd
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--mu", type=float, nargs="+", default=[5.0, 10.0, 20.0])
    ap.add_argument("--system", choices=["n2", "pair"], default="n2",
                    help="N-like dimer in a 48^3 box, or the two-atom 16^3 cell")
    ap.add_argument("--bond", type=float, default=None, help="starting guess of the bond")
    ap.add_argument("--periods", type=float, default=4.0)
    ap.add_argument("--fp32", action="store_true", help="complex64 orbitals")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    emd.load()
    prec = emd.EMD_FP32_ORBITALS if args.fp32 else emd.EMD_FP64
    if args.system == "n2":
        build, d0 = n_dimer, args.bond or 3.3
    else:
        base = pair_base()
        build = lambda d: pair(d, base)                       # noqa: E731
        d0 = args.bond or float(bond_length(base.R[None], base.n * base.h)[0])
    bo = bo_frequency(prec, d0, build)
    print(json.dumps({"bo": bo}), flush=True)
    res = study(args.mu, prec, bo["bond"], omega_bo=bo["omega"], periods=args.periods,
                build=build)
    for r in res:
        print(json.dumps(r), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"bo": bo, "runs": res}, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
