"""Thin ctypes binding of libemd (see include/emd.h for the contract).

Argument marshalling only: every step of the propagation runs in the CUDA
library.  Loading fails loudly if ``libemd.so`` has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libemd.so")

EMD_OK, EMD_EINVAL, EMD_ENOMEM, EMD_ECUDA, EMD_EUNSTABLE, EMD_ESTATE, EMD_ETABLE = range(7)
EMD_ENOTCONV = 7
EMD_ETIMEOUT = 8
EMD_FP64, EMD_FP32_ORBITALS = 0, 1
EMD_OPT_FROZEN_IONS, EMD_OPT_PROFILE, EMD_OPT_CHECK_STABLE, EMD_OPT_STAGE_VARIANT = 1, 2, 3, 4
EMD_OPT_PROJECTION = 5
EMD_OPT_ZCHUNK = 6
EMD_KERNEL_HORNER, EMD_KERNEL_ALL = 0, 1
EMD_OBS_ENERGY, EMD_OBS_DIPOLE_Z = 0, 1


class EmdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libemd error {code}: {msg}")
        self.code = code


class emd_species(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("z", "mass", "a_loc", "r_loc", "r_c", "h_kb", "r_proj")] + [
                ("lmax", ctypes.c_int), ("h_l", ctypes.c_double * 2)]


class emd_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("h", ctypes.c_double),
                ("fd_order", ctypes.c_int), ("n_orb", ctypes.c_int),
                ("occ", ctypes.c_double), ("precision", ctypes.c_int),
                ("n_atoms", ctypes.c_int), ("species", emd_species),
                ("cuda_stream", ctypes.c_void_p),
                ("block_orbitals", ctypes.c_int)]


class emd_energy(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("kin_e", "nl", "es", "xc", "sr", "kin_ion", "ks", "total", "n_elec")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class emd_gs_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("residual", ctypes.c_double),
                ("band_energy", ctypes.c_double), ("gap", ctypes.c_double),
                ("fermi_level", ctypes.c_double), ("entropy", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_DPTR = ctypes.POINTER(ctypes.c_double)


def load() -> ctypes.CDLL:
    """Load libemd.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.emd_init_system.argtypes = [ctypes.POINTER(emd_config), ctypes.POINTER(vp)]
    lib.emd_set_ions.argtypes = [vp, ip, _DPTR, _DPTR]
    lib.emd_set_orbitals.argtypes = [vp, _DPTR]
    lib.emd_set_orbitals_c64.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.emd_get_orbitals_c64.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.emd_propagate.argtypes = [vp, ip, dp, dp, _DPTR]
    lib.emd_get_forces.argtypes = [vp, _DPTR]
    lib.emd_get_energy.argtypes = [vp, ctypes.POINTER(emd_energy)]
    lib.emd_get_state.argtypes = [vp, _DPTR, _DPTR, _DPTR, _DPTR]
    lib.emd_get_potentials.argtypes = [vp, _DPTR, _DPTR, _DPTR, _DPTR]
    lib.emd_get_projections.argtypes = [vp, _DPTR]
    lib.emd_apply_hamiltonian.argtypes = [vp, ip, _DPTR, _DPTR]
    lib.emd_set_option.argtypes = [vp, ip, dp]
    lib.emd_kernel_stats.argtypes = [vp, ip, _DPTR, ctypes.POINTER(ctypes.c_longlong)]
    lib.emd_poisson_static.argtypes = [ip, dp, vp, vp, vp]
    lib.emd_poisson_static.restype = ctypes.c_int
    lib.emd_propagate_adjoint.argtypes = [vp, ip, dp, dp, _DPTR, ip, ip, _DPTR, _DPTR, _DPTR]
    lib.emd_propagate_adjoint.restype = ctypes.c_int
    lib.emd_batch_create.argtypes = [ip, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.emd_batch_create.restype = ctypes.c_int
    lib.emd_batch_propagate.argtypes = [vp, ip, dp, dp]
    lib.emd_batch_propagate.restype = ctypes.c_int
    lib.emd_batch_destroy.argtypes = [vp]
    lib.emd_batch_destroy.restype = None
    lib.emd_get_dipole.argtypes = [vp, _DPTR]
    lib.emd_get_dipole.restype = ctypes.c_int
    lib.emd_ground_state.argtypes = [vp, ip, dp, ip, dp, _DPTR, ctypes.POINTER(emd_gs_info)]
    lib.emd_ground_state.restype = ctypes.c_int
    lib.emd_ground_state_smeared.argtypes = [vp, ip, dp, ip, dp, dp, dp, dp, _DPTR, _DPTR,
                                             ctypes.POINTER(emd_gs_info)]
    lib.emd_ground_state_smeared.restype = ctypes.c_int
    lib.emd_set_occupations.argtypes = [vp, _DPTR]
    lib.emd_set_occupations.restype = ctypes.c_int
    lib.emd_get_occupations.argtypes = [vp, _DPTR]
    lib.emd_get_occupations.restype = ctypes.c_int
    lib.emd_destroy.argtypes = [vp]
    lib.emd_destroy.restype = None
    lib.emd_last_error.restype = ctypes.c_char_p
    lib.emd_version.restype = ctypes.c_char_p
    for name in ("emd_init_system", "emd_set_ions", "emd_set_orbitals",
                 "emd_propagate", "emd_get_forces", "emd_get_energy",
                 "emd_get_state", "emd_get_potentials", "emd_get_projections",
                 "emd_apply_hamiltonian", "emd_set_option", "emd_kernel_stats"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int) -> None:
    if code != EMD_OK:
        raise EmdError(code, load().emd_last_error().decode())


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_DPTR)


def _c128(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


# ---- one-to-one wrappers of the C entry points -----------------------------

def emd_init_system(cfg: emd_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().emd_init_system(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def emd_set_ions(h, R: np.ndarray, V: np.ndarray) -> None:
    R = np.ascontiguousarray(R, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    _check(load().emd_set_ions(h, R.shape[0], _dptr(R), _dptr(V)))


def emd_set_orbitals(h, psi: np.ndarray) -> None:
    psi = _c128(psi)
    _check(load().emd_set_orbitals(h, psi.view(np.float64).ctypes.data_as(_DPTR)))


def emd_set_orbitals_c64(h, psi: np.ndarray) -> None:
    """Orbitals from a complex64 array [n_orb, N, N, N]."""
    psi = np.ascontiguousarray(psi, dtype=np.complex64)
    _check(load().emd_set_orbitals_c64(
        h, psi.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def emd_get_orbitals_c64(h, n_orb: int, n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Orbitals of the current state as complex64 [n_orb, N, N, N] (into out
    if given, which must be C-contiguous complex64 of that shape)."""
    if out is None:
        out = np.empty((n_orb, n, n, n), dtype=np.complex64)
    _check(load().emd_get_orbitals_c64(
        h, out.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def emd_propagate(h, n_steps: int, dt: float, mu: float,
                  field: Optional[np.ndarray] = None) -> None:
    f = None if field is None else np.ascontiguousarray(field, dtype=np.float64)
    _check(load().emd_propagate(h, int(n_steps), float(dt), float(mu), _dptr(f)))


def emd_get_forces(h, n_atoms: int) -> np.ndarray:
    F = np.zeros((n_atoms, 3))
    _check(load().emd_get_forces(h, _dptr(F)))
    return F


def emd_get_energy(h) -> dict:
    e = emd_energy()
    _check(load().emd_get_energy(h, ctypes.byref(e)))
    return e.as_dict()


def emd_get_dipole(h) -> np.ndarray:
    D = np.zeros(3)
    _check(load().emd_get_dipole(h, _dptr(D)))
    return D


def emd_ground_state(h, n_orb: int, max_scf: int = 200, tol: float = 1e-10,
                     degree: int = 16, mix: float = 0.5):
    """Ground state at the current ions (see include/emd.h).  Returns
    (eigenvalues [n_orb], info dict); raises EmdError, with code
    EMD_ENOTCONV if the tolerance was not reached."""
    w = np.zeros(n_orb)
    info = emd_gs_info()
    _check(load().emd_ground_state(h, max_scf, tol, degree, mix, _dptr(w), ctypes.byref(info)))
    return w, info.as_dict()


def emd_ground_state_smeared(h, n_orb: int, kT: float, n_electrons: float,
                             kerker_q0: float = 0.0, max_scf: int = 200,
                             tol: float = 1e-10, degree: int = 16, mix: float = 0.5):
    """Ground state with Fermi-Dirac occupations (see include/emd.h).
    Returns (eigenvalues [n_orb], occupations [n_orb], info dict)."""
    w = np.zeros(n_orb)
    f = np.zeros(n_orb)
    info = emd_gs_info()
    _check(load().emd_ground_state_smeared(h, max_scf, tol, degree, mix, kT, n_electrons,
                                           kerker_q0, _dptr(w), _dptr(f), ctypes.byref(info)))
    return w, f, info.as_dict()


def emd_set_occupations(h, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().emd_set_occupations(h, _dptr(f)))


def emd_get_occupations(h, n_orb: int) -> np.ndarray:
    f = np.zeros(n_orb)
    _check(load().emd_get_occupations(h, _dptr(f)))
    return f


def emd_get_state(h, n_atoms: int, n_orb: int, n: int, want_psi=True, want_rho=True):
    R = np.zeros((n_atoms, 3))
    V = np.zeros((n_atoms, 3))
    psi = np.zeros((n_orb, n, n, n), dtype=np.complex128) if want_psi else None
    rho = np.zeros((n, n, n)) if want_rho else None
    _check(load().emd_get_state(
        h, _dptr(R), _dptr(V),
        None if psi is None else psi.view(np.float64).ctypes.data_as(_DPTR),
        _dptr(rho)))
    return R, V, psi, rho


def emd_get_potentials(h, n: int):
    out = [np.zeros((n, n, n)) for _ in range(4)]
    _check(load().emd_get_potentials(h, *[_dptr(a) for a in out]))
    return dict(zip(("v_loc", "v_h", "v_xc", "g_ion"), out))


def emd_get_projections(h, n_atoms: int, n_orb: int, n_ch: int = 1) -> np.ndarray:
    """Projections [n_atoms * n_ch, n_orb]; n_ch = (lmax + 1)^2 projectors per atom."""
    c = np.zeros((n_atoms * n_ch, n_orb), dtype=np.complex128)
    _check(load().emd_get_projections(h, c.view(np.float64).ctypes.data_as(_DPTR)))
    return c


def emd_apply_hamiltonian(h, psi: np.ndarray) -> np.ndarray:
    psi = _c128(psi)
    out = np.zeros_like(psi)
    _check(load().emd_apply_hamiltonian(
        h, psi.shape[0], psi.view(np.float64).ctypes.data_as(_DPTR),
        out.view(np.float64).ctypes.data_as(_DPTR)))
    return out


def emd_set_option(h, option: int, value: float) -> None:
    _check(load().emd_set_option(h, int(option), float(value)))


def emd_kernel_stats(h, kernel: int = EMD_KERNEL_HORNER):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(load().emd_kernel_stats(h, int(kernel), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def emd_poisson_static(n: int, h: float, charge_dev: int, v_dev: int,
                       stream: int = 0) -> None:
    """Periodic Poisson solve on device buffers without any allocation
    (see include/emd.h); charge_dev and v_dev are device addresses."""
    _check(load().emd_poisson_static(int(n), float(h), ctypes.c_void_p(charge_dev),
                                     ctypes.c_void_p(v_dev),
                                     ctypes.c_void_p(stream) if stream else None))


def emd_destroy(h) -> None:
    if h:
        load().emd_destroy(h)


def emd_propagate_adjoint(h, n_steps: int, dt: float, mu: float,
                          field: Optional[np.ndarray], ckpt_every: int,
                          observable: int, n_atoms: int):
    """Returns (L, dL/dR [n_atoms, 3], dL/dfield [n_steps] or None)."""
    f = None if field is None else np.ascontiguousarray(field, dtype=np.float64)
    L = ctypes.c_double()
    dR = np.zeros((n_atoms, 3))
    df = None if f is None else np.zeros(n_steps)
    _check(load().emd_propagate_adjoint(h, int(n_steps), float(dt), float(mu), _dptr(f),
                                        int(ckpt_every), int(observable),
                                        ctypes.cast(ctypes.pointer(L), _DPTR),
                                        _dptr(dR), _dptr(df)))
    return L.value, dR, df


def emd_batch_create(handles) -> ctypes.c_void_p:
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                              for h in handles])
    b = ctypes.c_void_p()
    _check(load().emd_batch_create(len(handles), arr, ctypes.byref(b)))
    return b


def emd_batch_propagate(b, n_steps: int, dt: float, mu: float) -> None:
    _check(load().emd_batch_propagate(b, int(n_steps), float(dt), float(mu)))


def emd_batch_destroy(b) -> None:
    if b:
        load().emd_batch_destroy(b)


# ---- convenience -----------------------------------------------------------

def config_for(sysin, precision: int = EMD_FP64, stream: int = 0,
               block_orbitals: int = 0) -> emd_config:
    sp = sysin.species
    return emd_config(n=sysin.n, h=sysin.h, fd_order=sysin.fd_order,
                      n_orb=sysin.n_orb, occ=sysin.occ, precision=precision,
                      n_atoms=sysin.n_atoms,
                      species=emd_species(sp.z, sp.mass, sp.a_loc, sp.r_loc,
                                          sp.r_c, sp.h_kb, sp.r_proj,
                                          int(getattr(sp, "lmax", 0)),
                                          (ctypes.c_double * 2)(*getattr(sp, "h_l", (0.0, 0.0)))),
                      cuda_stream=stream or None,
                      block_orbitals=block_orbitals)


class System:
    """Owns one libemd handle for a ``SystemInput``."""

    def __init__(self, sysin, precision: int = EMD_FP64, stream: int = 0,
                 block_orbitals: int = 0):
        self.sysin = sysin
        self.handle = emd_init_system(config_for(sysin, precision, stream, block_orbitals))
        emd_set_ions(self.handle, sysin.R, sysin.V)
        emd_set_orbitals(self.handle, sysin.psi)

    def propagate(self, n_steps, dt=None, mu=None, field=None):
        emd_propagate(self.handle, n_steps, self.sysin.dt if dt is None else dt,
                      self.sysin.mu if mu is None else mu, field)

    def forces(self):
        return emd_get_forces(self.handle, self.sysin.n_atoms)

    def energy(self):
        return emd_get_energy(self.handle)

    def state(self, want_psi=True, want_rho=True):
        s = self.sysin
        return emd_get_state(self.handle, s.n_atoms, s.n_orb, s.n, want_psi, want_rho)

    def occupations(self):
        return emd_get_occupations(self.handle, self.sysin.n_orb)

    def set_occupations(self, f):
        emd_set_occupations(self.handle, f)

    def ground_state(self, kT: float = 0.0, n_electrons: Optional[float] = None,
                     kerker_q0: float = 0.0, **kw):
        """Ground state at the current ions: integer occupations (kT = 0) or
        Fermi-Dirac ones holding n_electrons (default: the valence charge
        Z n_atoms).
        Returns (eigenvalues, occupations, info)."""
        s = self.sysin
        if kT <= 0.0:
            w, info = emd_ground_state(self.handle, s.n_orb, **kw)
            return w, self.occupations(), info
        if n_electrons is None:
            n_electrons = s.species.z * s.n_atoms
        return emd_ground_state_smeared(self.handle, s.n_orb, kT, n_electrons,
                                        kerker_q0=kerker_q0, **kw)

    def close(self):
        emd_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                self.close()
        except Exception:
            pass
