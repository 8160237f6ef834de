// Test driver for the ground-state solver's host steps (gs_host.h): reads
// one problem from stdin, writes the library's answer to stdout (%.17g).
//   eig m  H S       -> ok, w[m], V[m x m] (complex as re im, column-major)
//   fd n n_e occ kT eps[n]  -> mu, S, f[n]
//   anderson K n_act newest act[n_act] B[K x K]  -> c[n_act]
#include <cstdio>
#include <cstring>
#include "gs_host.h"

int main() {
  char mode[32];
  if (std::scanf("%31s", mode) != 1) return 2;
  if (!std::strcmp(mode, "eig")) {
    int m;
    if (std::scanf("%d", &m) != 1) return 2;
    std::vector<std::complex<double>> H((size_t)m * m), S((size_t)m * m), V;
    for (auto *M : {&H, &S})
      for (auto &z : *M) {
        double re, im;
        if (std::scanf("%lf %lf", &re, &im) != 2) return 2;
        z = {re, im};
      }
    std::vector<double> w;
    const bool ok = emd_host::hermitian_generalized_eig(m, H, S, w, V);
    std::printf("%d\n", ok ? 1 : 0);
    if (!ok) return 0;
    for (double x : w) std::printf("%.17g\n", x);
    for (auto &z : V) std::printf("%.17g %.17g\n", z.real(), z.imag());
  } else if (!std::strcmp(mode, "fd")) {
    int n;
    double ne, occ, kT;
    if (std::scanf("%d %lf %lf %lf", &n, &ne, &occ, &kT) != 4) return 2;
    std::vector<double> eps(n), f;
    for (auto &x : eps)
      if (std::scanf("%lf", &x) != 1) return 2;
    const double mu = emd_host::fermi_dirac(eps, n, ne, occ, kT, f);
    std::printf("%.17g\n%.17g\n", mu, emd_host::smearing_entropy(eps, n, mu, occ, kT));
    for (double x : f) std::printf("%.17g\n", x);
  } else if (!std::strcmp(mode, "anderson")) {
    int K, na, newest;
    if (std::scanf("%d %d %d", &K, &na, &newest) != 3) return 2;
    std::vector<int> act(na);
    for (auto &a : act)
      if (std::scanf("%d", &a) != 1) return 2;
    std::vector<double> B((size_t)K * K), c;
    for (auto &x : B)
      if (std::scanf("%lf", &x) != 1) return 2;
    emd_host::anderson_coefficients(K, B.data(), act, newest, c);
    for (double x : c) std::printf("%.17g\n", x);
  } else {
    return 2;
  }
  return 0;
}
