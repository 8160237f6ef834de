"""The ground-state solver's host steps (csrc/gs_host.h), compiled with the
host C++ compiler and checked without a GPU:

* the Rayleigh-Ritz generalized Hermitian eigenproblem H v = lambda S v
  against scipy's eigh, and by its defining properties (residual, S-
  orthonormality), including degenerate, diagonal and 1 x 1 cases and a
  non-positive-definite S;
* the Anderson coefficients against the constrained least-squares problem
  they solve (min |sum c_i F_i| with sum c_i = 1), solved with numpy;
* the Fermi-Dirac occupations and entropy against closed forms.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_0812_2801_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("gs_host") / "gs_host_driver")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC,
                    os.path.join(HERE, "host", "gs_host_driver.cpp"), "-o", exe], check=True)
    return exe


def _run(exe, text):
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    return out.split("\n")


def _cplx_lines(M):
    return "\n".join(f"{float(z.real)!r} {float(z.imag)!r}" for z in M.flatten(order="F"))


def geig(exe, H, S):
    m = H.shape[0]
    lines = _run(exe, f"eig {m}\n{_cplx_lines(H)}\n{_cplx_lines(S)}\n")
    if lines[0] == "0":
        return None
    w = np.array([float(x) for x in lines[1:1 + m]])
    v = np.array([complex(*map(float, l.split())) for l in lines[1 + m:1 + m + m * m]])
    return w, v.reshape(m, m, order="F")


def _hermitian(rng, m):
    X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    return 0.5 * (X + X.conj().T)


def _spd(rng, m):
    X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    return X @ X.conj().T / m + np.eye(m)


def _check_pairs(H, S, w, V, tol):
    scale = max(np.max(np.abs(H)), 1.0)
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(H @ V - S @ V * w[None, :])) < tol * scale
    assert np.max(np.abs(V.conj().T @ S @ V - np.eye(H.shape[0]))) < tol


@pytest.mark.parametrize("m", [1, 2, 3, 7, 40])
def test_generalized_eig_random(driver, m):
    from scipy.linalg import eigh
    rng = np.random.default_rng(m)
    H, S = _hermitian(rng, m), _spd(rng, m)
    w, V = geig(driver, H, S)
    assert np.max(np.abs(w - eigh(H, S, eigvals_only=True))) < 1e-12 * max(np.max(np.abs(w)), 1)
    _check_pairs(H, S, w, V, 1e-11)


def test_generalized_eig_degenerate_and_diagonal(driver):
    rng = np.random.default_rng(3)
    m = 12
    # H = S U diag(lam) U^H S with triple and double eigenvalues: H v = lam S v
    lam = np.array([-1.0, -1.0, -1.0, 0.0, 0.5, 0.5, 1.0, 2.0, 2.0, 3.0, 4.0, 5.0])
    S = _spd(rng, m)
    Ls = np.linalg.cholesky(S)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    A = Q @ np.diag(lam) @ Q.conj().T
    H = Ls @ A @ Ls.conj().T
    H = 0.5 * (H + H.conj().T)
    w, V = geig(driver, H, S)
    assert np.max(np.abs(w - lam)) < 1e-12 * 5
    _check_pairs(H, S, w, V, 1e-11)
    # already diagonal (the state of a converged subspace), with a zero
    Hd = np.diag([0.3, -0.2, 0.0, 0.1]).astype(complex)
    w, V = geig(driver, Hd, np.eye(4, dtype=complex))
    assert np.array_equal(w, np.sort(np.diag(Hd).real))
    _check_pairs(Hd, np.eye(4), w, V, 1e-15)


def test_generalized_eig_nearly_diagonal(driver):
    """The Rayleigh-Ritz matrices near convergence: a diagonal with
    clustered entries plus 1e-9 couplings."""
    rng = np.random.default_rng(11)
    m = 30
    H = np.diag(np.sort(rng.normal(size=m)) * 0.01).astype(complex) + 1e-9 * _hermitian(rng, m)
    S = np.eye(m) + 1e-9 * _hermitian(rng, m)
    w, V = geig(driver, H, S)
    from scipy.linalg import eigh
    assert np.max(np.abs(w - eigh(H, S, eigvals_only=True))) < 1e-15
    _check_pairs(H, S, w, V, 1e-12)


def test_generalized_eig_rejects_indefinite_overlap(driver):
    rng = np.random.default_rng(5)
    S = np.diag([1.0, 1.0, -1e-3, 1.0]).astype(complex)
    assert geig(driver, _hermitian(rng, 4), S) is None


def anderson(exe, B, act, newest):
    K = B.shape[0]
    text = (f"anderson {K} {len(act)} {newest}\n" + " ".join(map(str, act)) + "\n"
            + " ".join(repr(float(x)) for x in B.flatten()) + "\n")
    return np.array([float(x) for x in _run(exe, text) if x])


def test_anderson_solves_the_constrained_least_squares(driver):
    rng = np.random.default_rng(8)
    K, n = 6, 50
    F = rng.normal(size=(K, n))
    B = F @ F.T
    act = [3, 5, 0, 1]
    c = anderson(driver, B, act, newest=1)
    # KKT system of min |sum c_i F_i|^2 subject to sum c_i = 1
    Fa = F[act]
    M = np.zeros((5, 5))
    M[:4, :4] = 2 * Fa @ Fa.T
    M[:4, 4] = M[4, :4] = 1.0
    sol = np.linalg.solve(M, np.r_[np.zeros(4), 1.0])
    assert abs(c.sum() - 1.0) < 1e-14
    assert np.max(np.abs(c - sol[:4])) < 1e-9
    # no history to combine: plain mixing with the newest pair
    c0 = anderson(driver, np.zeros((K, K)), [2, 4], newest=4)
    assert np.array_equal(c0, [0.0, 1.0])


def fd(exe, eps, ne, occ, kT):
    text = f"fd {len(eps)} {ne!r} {occ!r} {kT!r}\n" + " ".join(repr(float(e)) for e in eps) + "\n"
    out = [float(x) for x in _run(exe, text) if x]
    return out[0], out[1], np.array(out[2:])


def test_fermi_dirac_closed_forms(driver):
    occ, kT = 2.0, 0.03
    mu, S, f = fd(driver, [-0.02, 0.02], occ, occ, kT)
    assert abs(mu) < 1e-14
    assert np.max(np.abs(f - occ / (1 + np.exp(np.array([-0.02, 0.02]) / kT)))) < 1e-14
    g = f / occ
    assert abs(S + occ * np.sum(g * np.log(g) + (1 - g) * np.log(1 - g))) < 1e-13
    mu, S, f = fd(driver, [-0.3] * 5, 3.0, occ, kT)
    g = 3.0 / (occ * 5)
    assert np.max(np.abs(f - 0.6)) < 1e-14
    assert abs(mu - (-0.3 + kT * np.log(g / (1 - g)))) < 1e-12
    mu, S, f = fd(driver, [0.1] * 4, 4.0, occ, kT)          # half filling
    assert abs(S - 4 * occ * np.log(2.0)) < 1e-13
    mu, S, f = fd(driver, [-1.0, -0.9, 0.5, 0.6], 4.0, occ, 0.005)
    # any mu inside the 1.4 Ha gap holds the charge to rounding: the filled
    # states keep 1 - g below ~e^-30 and S is at rounding level
    assert np.all(np.abs(f[:2] - 2.0) < 1e-12) and np.all(f[2:] < 1e-12) and abs(S) < 1e-12
    rng = np.random.default_rng(2)
    eps = np.sort(rng.normal(size=30)) * 0.1
    mu, S, f = fd(driver, eps, 37.5, occ, 0.01)
    assert abs(f.sum() - 37.5) < 1e-12
    assert np.max(np.abs(f - occ / (1 + np.exp((eps - mu) / 0.01)))) < 1e-15
