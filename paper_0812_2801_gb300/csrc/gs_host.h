// Host-side dense steps of the ground-state solver (the KS equations at
// fixed ions, Sec. 4.1, eqs. EoM_BO_a and EoM_BO_b): the m x m generalized
// eigenproblem of the Rayleigh-Ritz step, the Anderson mixing
// coefficients, and Fermi-Dirac occupations with their entropy.  Plain
// C++17 with no CUDA, so that host tests compile and check it on their own.

#ifndef EMD_GS_HOST_H
#define EMD_GS_HOST_H

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace emd_host {

// Eigenvalues lam[n] (unordered) and orthonormal eigenvectors Z (columns,
// n x n column-major) of the Hermitian matrix A (column-major; overwritten).
//  1. Householder reflections P_k = I - 2 v v^H, v over rows k+1..n-1 and
//     |v| = 1, reduce A to a Hermitian tridiagonal T = Q^H A Q, Q = P_0 P_1
//     ...  Each maps the column x below the diagonal to alpha e_1 with
//     alpha = -(x_0/|x_0|) |x| (x^H alpha e_1 real, so the map exists);
//     with p = A v and w = p - (v^H p) v the update is
//     A <- A - 2 v w^H - 2 w v^H on the trailing block.
//  2. The phases phi_0 = 1, phi_{k+1} = phi_k t_k / |t_k| (t_k the
//     subdiagonal) make D^H T D real symmetric with off-diagonal |t_k|.
//  3. Implicit QR steps with Wilkinson's shift (the eigenvalue of the
//     trailing 2 x 2 block nearer its last diagonal entry) on that real
//     tridiagonal: each step is a chain of plane rotations that starts from
//     (d_lo - shift, e_lo) and chases the off-tridiagonal bulge down the
//     block; a subdiagonal entry below 2^-52 (|d_i| + |d_i+1|) splits the
//     matrix.  The rotations are accumulated into Z = Q D, so Z holds the
//     eigenvectors of A at the end.
// Returns false if the QR steps did not converge within 60 n steps.
inline bool hermitian_eig(int n, std::vector<std::complex<double>> &A, std::vector<double> &lam,
                          std::vector<std::complex<double>> &Z) {
  typedef std::complex<double> cd;
  auto at = [n](std::vector<cd> &M, int i, int j) -> cd & { return M[(size_t)j * n + i]; };
  std::vector<std::vector<cd>> refl;            // v of each reflection (rows k+1..n-1)
  std::vector<cd> p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int len = n - k - 1;
    double xn = 0.0;
    for (int i = 0; i < len; ++i) xn += std::norm(at(A, k + 1 + i, k));
    xn = std::sqrt(xn);
    std::vector<cd> v(len);
    const cd x0 = at(A, k + 1, k);
    const double ax0 = std::abs(x0);
    if (xn == 0.0 || (ax0 == xn && len == 1)) {
      refl.push_back(std::vector<cd>());        // already reduced: P_k = I
      continue;
    }
    const cd ph = ax0 > 0.0 ? x0 / ax0 : cd(1.0, 0.0);
    const cd alpha = -ph * xn;
    for (int i = 0; i < len; ++i) v[i] = at(A, k + 1 + i, k);
    v[0] -= alpha;
    double vn = 0.0;
    for (int i = 0; i < len; ++i) vn += std::norm(v[i]);
    vn = std::sqrt(vn);
    for (int i = 0; i < len; ++i) v[i] /= vn;
    // p = A_sub v, K = v^H p (real), w = p - K v
    for (int i = 0; i < len; ++i) {
      cd t = 0.0;
      for (int j = 0; j < len; ++j) t += at(A, k + 1 + i, k + 1 + j) * v[j];
      p[i] = t;
    }
    double K = 0.0;
    for (int i = 0; i < len; ++i) K += (std::conj(v[i]) * p[i]).real();
    for (int i = 0; i < len; ++i) w[i] = p[i] - K * v[i];
    for (int j = 0; j < len; ++j)
      for (int i = 0; i < len; ++i)
        at(A, k + 1 + i, k + 1 + j) -=
            2.0 * (v[i] * std::conj(w[j]) + w[i] * std::conj(v[j]));
    at(A, k + 1, k) = alpha;
    at(A, k, k + 1) = std::conj(alpha);
    for (int i = 1; i < len; ++i) at(A, k + 1 + i, k) = at(A, k, k + 1 + i) = 0.0;
    refl.push_back(v);
  }
  // Z = Q = P_0 P_1 ... (applied from the right to the identity), then Q D
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) at(Z, i, i) = 1.0;
  for (int k = 0; k < (int)refl.size(); ++k) {
    const std::vector<cd> &v = refl[k];
    if (v.empty()) continue;
    const int len = (int)v.size();
    for (int r = 0; r < n; ++r) {               // row r of Z: z <- z - 2 (z v) v^H
      cd t = 0.0;
      for (int i = 0; i < len; ++i) t += at(Z, r, k + 1 + i) * v[i];
      for (int i = 0; i < len; ++i) at(Z, r, k + 1 + i) -= 2.0 * t * std::conj(v[i]);
    }
  }
  std::vector<double> d(n), e(n > 1 ? n - 1 : 1, 0.0);
  cd phi = 1.0;
  for (int i = 0; i < n; ++i) {
    d[i] = at(A, i, i).real();
    if (i > 0) {
      const cd t = at(A, i, i - 1);
      const double at_ = std::abs(t);
      e[i - 1] = at_;
      if (at_ > 0.0) phi *= t / at_;
      for (int r = 0; r < n; ++r) at(Z, r, i) *= phi;
    }
  }
  // implicit QR on the real tridiagonal (d, e), rotations into Z's columns
  const double eps = std::ldexp(1.0, -52);
  int steps = 0;
  int hi = n - 1;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo])))
      --lo;
    if (++steps > 60 * n) return false;
    const double delta = 0.5 * (d[hi - 1] - d[hi]);
    const double b = e[hi - 1];
    const double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * std::hypot(delta, b);
    const double shift = d[hi] - b * b / den;
    double x = d[lo] - shift, z = e[lo], bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      if (k > lo) {
        x = e[k - 1];
        z = bulge;
      }
      const double r = std::hypot(x, z);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
      // the window of T touched by a rotation of rows/columns k, k + 1
      const int a0 = k > lo ? k - 1 : k, a1 = std::min(k + 2, hi);
      const int wn = a1 - a0 + 1, pk = k - a0;
      double W[4][4] = {};
      for (int i = a0; i <= a1; ++i) W[i - a0][i - a0] = d[i];
      for (int i = a0; i < a1; ++i) W[i - a0][i + 1 - a0] = W[i + 1 - a0][i - a0] = e[i];
      if (k > lo) W[0][2] = W[2][0] = bulge;
      for (int j = 0; j < wn; ++j) {            // rows: G^T W
        const double u = W[pk][j], t = W[pk + 1][j];
        W[pk][j] = c * u + s * t;
        W[pk + 1][j] = -s * u + c * t;
      }
      for (int i = 0; i < wn; ++i) {            // columns: W G
        const double u = W[i][pk], t = W[i][pk + 1];
        W[i][pk] = c * u + s * t;
        W[i][pk + 1] = -s * u + c * t;
      }
      for (int i = a0; i <= a1; ++i) d[i] = W[i - a0][i - a0];
      for (int i = a0; i < a1; ++i) e[i] = W[i - a0][i + 1 - a0];
      bulge = k + 2 <= hi ? W[pk][pk + 2] : 0.0;
      for (int r2 = 0; r2 < n; ++r2) {          // Z <- Z G
        const cd u = at(Z, r2, k), t = at(Z, r2, k + 1);
        at(Z, r2, k) = c * u + s * t;
        at(Z, r2, k + 1) = -s * u + c * t;
      }
    }
  }
  lam = d;
  return true;
}

// The m x m generalized Hermitian eigenproblem H v = lambda S v of the
// Rayleigh-Ritz step, on the host (column-major): the Cholesky factor S = L
// L^H, A = L^-1 H L^-H, its eigenpairs (A w = lambda w, hermitian_eig),
// then v = L^-H w.  Returns the eigenvalues ascending with their
// S-orthonormal vectors; false if S is not positive definite or the QR
// iteration did not converge.
inline bool hermitian_generalized_eig(int m, const std::vector<std::complex<double>> &H,
                               const std::vector<std::complex<double>> &S,
                               std::vector<double> &w,
                               std::vector<std::complex<double>> &V) {
  typedef std::complex<double> cd;
  auto at = [m](std::vector<cd> &M, int i, int j) -> cd & { return M[(size_t)j * m + i]; };
  std::vector<cd> L((size_t)m * m, 0.0), Sc(S), Hc(H);
  for (int j = 0; j < m; ++j) {                 // Cholesky, lower
    double d = at(Sc, j, j).real();
    for (int k = 0; k < j; ++k) d -= std::norm(at(L, j, k));
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    at(L, j, j) = ljj;
    for (int i = j + 1; i < m; ++i) {
      cd v = at(Sc, i, j);
      for (int k = 0; k < j; ++k) v -= at(L, i, k) * std::conj(at(L, j, k));
      at(L, i, j) = v / ljj;
    }
  }
  // Y = L^-1 H (forward substitution per column), then A = L^-1 Y^H (= (Y L^-H)^H)
  std::vector<cd> Y((size_t)m * m), A((size_t)m * m);
  auto lsolve = [&](std::vector<cd> &B, std::vector<cd> &X) {
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < m; ++i) {
        cd v = at(B, i, c);
        for (int k = 0; k < i; ++k) v -= at(L, i, k) * at(X, k, c);
        at(X, i, c) = v / at(L, i, i);
      }
  };
  lsolve(Hc, Y);
  std::vector<cd> Yh((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) at(Yh, i, j) = std::conj(at(Y, j, i));
  lsolve(Yh, A);
  for (int i = 0; i < m; ++i) {                 // A is Hermitian up to rounding
    at(A, i, i) = at(A, i, i).real();
    for (int j = i + 1; j < m; ++j) {
      const cd v = 0.5 * (at(A, i, j) + std::conj(at(A, j, i)));
      at(A, i, j) = v;
      at(A, j, i) = std::conj(v);
    }
  }
  std::vector<cd> W;
  std::vector<double> lam;
  if (!hermitian_eig(m, A, lam, W)) return false;
  std::vector<int> ord(m);
  for (int i = 0; i < m; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return lam[a] < lam[b];
  });
  w.resize(m);
  V.assign((size_t)m * m, 0.0);
  for (int c = 0; c < m; ++c) {
    const int k = ord[c];
    w[c] = lam[k];
    for (int i = m - 1; i >= 0; --i) {          // v = L^-H w_k (back substitution)
      cd v = at(W, i, k);
      for (int j = i + 1; j < m; ++j) v -= std::conj(at(L, j, i)) * at(V, j, c);
      at(V, i, c) = v / at(L, i, i);
    }
  }
  return true;
}

// Anderson mixing: with F_i = rho_out_i - rho_in_i over the stored
// iterations, c minimises |sum c_i F_i| subject to sum c_i = 1, and
// rho_in <- sum c_i (rho_in_i + mix F_i).  B (K x K, row-major) holds
// <F_i, F_j> for the history slots; act lists the slots in use, newest the
// latest (the fallback when the system is singular).
inline void anderson_coefficients(int K, const double *B, const std::vector<int> &act,
                                  int newest, std::vector<double> &c) {
  const int m = (int)act.size();
  std::vector<double> M(m * m), x(m, 1.0);
  double dmax = 0.0;
  for (int i = 0; i < m; ++i) dmax = std::max(dmax, B[act[i] * K + act[i]]);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      M[i * m + j] = B[act[i] * K + act[j]] + (i == j ? 1e-12 * dmax : 0.0);
  bool ok = dmax > 0.0;
  for (int k = 0; ok && k < m; ++k) {       // Gaussian elimination, partial pivoting
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (std::fabs(M[i * m + k]) > std::fabs(M[p * m + k])) p = i;
    if (!(std::fabs(M[p * m + k]) > 0.0)) {
      ok = false;
      break;
    }
    if (p != k) {
      for (int j = 0; j < m; ++j) std::swap(M[k * m + j], M[p * m + j]);
      std::swap(x[k], x[p]);
    }
    for (int i = k + 1; i < m; ++i) {
      const double f = M[i * m + k] / M[k * m + k];
      for (int j = k; j < m; ++j) M[i * m + j] -= f * M[k * m + j];
      x[i] -= f * x[k];
    }
  }
  for (int k = m - 1; ok && k >= 0; --k) {
    double v = x[k];
    for (int j = k + 1; j < m; ++j) v -= M[k * m + j] * x[j];
    x[k] = v / M[k * m + k];
  }
  double sum = 0.0;
  for (int i = 0; ok && i < m; ++i) sum += x[i];
  ok = ok && std::isfinite(sum) && std::fabs(sum) > 0.0;
  c.assign(m, 0.0);
  if (!ok) {                                // plain mixing with the newest pair
    for (int i = 0; i < m; ++i) c[i] = act[i] == newest ? 1.0 : 0.0;
    return;
  }
  for (int i = 0; i < m; ++i) c[i] = x[i] / sum;
}

// Fermi-Dirac occupations of the n lowest Ritz values, f_i = occ / (1 +
// exp((eps_i - mu) / kT)), with mu bisected (sum f is increasing in mu)
// until sum f = n_e; returns mu.  Needs 0 < n_e < occ n.
inline double fermi_dirac(const std::vector<double> &eps, int n, double n_e, double occ,
                      double kT, std::vector<double> &f) {
  double lo = eps[0], hi = eps[0];
  for (int i = 0; i < n; ++i) {
    lo = std::min(lo, eps[i]);
    hi = std::max(hi, eps[i]);
  }
  lo -= 50.0 * kT + 1.0;                    // sum f ~ 0 here
  hi += 50.0 * kT + 1.0;                    // sum f ~ occ n here
  f.assign(n, 0.0);
  auto fill = [&](double mu) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) {
      f[i] = occ / (1.0 + std::exp((eps[i] - mu) / kT));
      t += f[i];
    }
    return t;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (fill(mid) < n_e) lo = mid;
    else hi = mid;
  }
  const double mu = 0.5 * (lo + hi);
  fill(mu);
  return mu;
}

// S = -sum_i occ [g ln g + (1 - g) ln(1 - g)], g = 1 / (1 + e^x) and
// 1 - g = 1 / (1 + e^-x), x = (eps_i - mu) / kT (0 ln 0 = 0)
inline double smearing_entropy(const std::vector<double> &eps, int n, double mu, double occ, double kT) {
  auto xlx = [](double v) { return v > 0.0 ? v * std::log(v) : 0.0; };
  double t = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = (eps[i] - mu) / kT;
    t += xlx(1.0 / (1.0 + std::exp(x))) + xlx(1.0 / (1.0 + std::exp(-x)));
  }
  return -occ * t;
}

}  // namespace emd_host

#endif  // EMD_GS_HOST_H
