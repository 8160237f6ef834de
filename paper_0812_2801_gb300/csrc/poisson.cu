// Hartree/ionic electrostatics by a periodic spectral Poisson solve, the
// Perdew-Zunger LDA, the effective potential of each AETRS half and
// deterministic grid reductions.
//
// Paper: the Hartree term of E_KS (eq. E_KS) and the ionic potential
// (eq. ionicpotential) are electrostatic potentials; the paper's finite
// systems use an interpolating-scaling-function Poisson solver (Sec. 5), the
// periodic boxes here solve nabla^2 v = -4 pi n in Fourier space with the
// G = 0 component set to zero.  XC: Perdew-Zunger LDA (Sec. 5), adiabatic
// (instantaneous density, Sec. 4.1).  H(t+dt) of AETRS uses a v_Hxc
// extrapolated from previous steps (Sec. 5.1, eq. aetrs).
//
// The 3-D FFT is three passes of batched 1-D FFTs along the contiguous axis;
// each pass writes its output transposed ([a][b][k] -> [k][a][b]) so the
// next axis becomes contiguous and three passes restore the layout.  Each
// 1-D FFT is a mixed-radix Stockham autosort transform in shared memory
// (radix 4, 2, 3, 5 and a direct DFT for other small primes) with twiddles
// precomputed once per grid size.
#include <cmath>
#include <mutex>
#include <vector>
#include "emd_internal.cuh"

namespace {

constexpr int kMaxStages = 16;
constexpr int kMaxRadix = 13;

struct FftPlan {
  int n, ns, lines;
  int rad[kMaxStages];
  int tw_off[kMaxStages];   // twiddles exp(-2 pi i jm r / (Ns R)), [jm][r]
  int root_off[kMaxStages]; // roots exp(-2 pi i m / R), m < R
};

// exp(-2 pi i num / den) evaluated in extended precision on the host.
double2 unit_root(long num, long den) {
  const long double PI_L = 3.141592653589793238462643383279502884L;
  const long double ang = -2.0L * PI_L * (long double)num / (long double)den;
  return make_double2((double)cosl(ang), (double)sinl(ang));
}

bool make_plan(int n, FftPlan &p, std::vector<double2> &tab) {
  p.n = n;
  p.ns = 0;
  int m = n;
  const int order[] = {4, 2, 3, 5, 7, 11, 13};
  for (int r : order) {
    while (m % r == 0) {
      if (p.ns >= kMaxStages) return false;
      p.rad[p.ns++] = r;
      m /= r;
    }
  }
  if (m != 1) return false;
  tab.clear();
  int Ns = 1;
  for (int s = 0; s < p.ns; ++s) {
    const int R = p.rad[s];
    p.tw_off[s] = (int)tab.size();
    for (int jm = 0; jm < Ns; ++jm)
      for (int r = 0; r < R; ++r) {
        // angle = -2 pi jm r / (Ns R), reduced exactly as a rational
        const long num = (long)jm * r % ((long)Ns * R);
        tab.push_back(unit_root(num, (long)Ns * R));
      }
    p.root_off[s] = (int)tab.size();
    for (int q = 0; q < R; ++q) tab.push_back(unit_root(q, R));
    Ns *= R;
  }
  p.lines = n >= 1280 ? 1 : (1280 / n > 8 ? 8 : 1280 / n);
  return true;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
// multiply by sign * i
__device__ __forceinline__ double2 cmuli(double2 a, int sign) {
  return sign > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// One radix-R Stockham stage on L lines of length n in shared memory (x -> y),
// R a compile-time constant so the R inputs of a butterfly stay in registers.
template <int R>
__device__ __forceinline__ void fft_stage(const double2 *b0, double2 *b1, int n, int L,
                                          int Ns, const double2 *tw, const double2 *root,
                                          int sign, int stride) {
  const int m = n / R;
  for (int t = threadIdx.x; t < L * m; t += blockDim.x) {
    const int l = t / m, j = t - l * m;
    const double2 *x = b0 + l * stride;
    double2 *y = b1 + l * stride;
    const int jm = j % Ns;
    const int base = (j / Ns) * Ns * R + jm;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double2 a = x[j + r * m];
      if (r > 0 && jm > 0) {
        double2 w = tw[jm * R + r];
        if (sign > 0) w.y = -w.y;
        a = cmul(a, w);
      }
      v[r] = a;
    }
    if (R == 4) {
      const double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
      const double2 t2 = cadd(v[1], v[3]), t3 = cmuli(csub(v[1], v[3]), sign);
      y[base] = cadd(t0, t2);
      y[base + Ns] = cadd(t1, t3);
      y[base + 2 * Ns] = csub(t0, t2);
      y[base + 3 * Ns] = csub(t1, t3);
    } else if (R == 2) {
      y[base] = cadd(v[0], v[1]);
      y[base + Ns] = csub(v[0], v[1]);
    } else if (R == 3) {
      const double c3 = 0.86602540378443864676;  // sqrt(3)/2
      const double2 sm_ = cadd(v[1], v[2]), df = csub(v[1], v[2]);
      const double2 a = make_double2(v[0].x - 0.5 * sm_.x, v[0].y - 0.5 * sm_.y);
      double2 b = cmuli(df, sign);
      b.x *= c3;
      b.y *= c3;
      y[base] = cadd(v[0], sm_);
      y[base + Ns] = cadd(a, b);
      y[base + 2 * Ns] = csub(a, b);
    } else {
#pragma unroll
      for (int k = 0; k < R; ++k) {
        double2 acc = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) {
          double2 w = root[(r * k) % R];
          if (sign > 0) w.y = -w.y;
          acc = cadd(acc, cmul(v[r], w));
        }
        y[base + k * Ns] = acc;
      }
    }
  }
}

// Any other radix (7, 11, 13): the same stage with the R inputs in a local
// array (rare grid sizes; keeps the common radices' register use low).
__device__ __noinline__ void fft_stage_any(int R, const double2 *b0, double2 *b1, int n,
                                           int L, int Ns, const double2 *tw,
                                           const double2 *root, int sign, int stride) {
  const int m = n / R;
  for (int t = threadIdx.x; t < L * m; t += blockDim.x) {
    const int l = t / m, j = t - l * m;
    const double2 *x = b0 + l * stride;
    double2 *y = b1 + l * stride;
    const int jm = j % Ns;
    const int base = (j / Ns) * Ns * R + jm;
    double2 v[kMaxRadix];
    for (int r = 0; r < R; ++r) {
      double2 a = x[j + r * m];
      if (r > 0 && jm > 0) {
        double2 w = tw[jm * R + r];
        if (sign > 0) w.y = -w.y;
        a = cmul(a, w);
      }
      v[r] = a;
    }
    for (int k = 0; k < R; ++k) {
      double2 acc = v[0];
      for (int r = 1; r < R; ++r) {
        double2 w = root[(r * k) % R];
        if (sign > 0) w.y = -w.y;
        acc = cadd(acc, cmul(v[r], w));
      }
      y[base + k * Ns] = acc;
    }
  }
}

// One pass: 1-D FFTs of length n along the contiguous axis of [a][b][n],
// output transposed to [k][a][b].  IN_REAL: input is a real array.
// OUT_REAL: write the real part times `scale` to a real array.
template <bool IN_REAL, bool OUT_REAL>
__global__ void __launch_bounds__(256)
k_fft_pass(const void *in, void *out, FftPlan pl, const double2 *tab,
           int sign, double scale) {
  extern __shared__ double2 sm[];
  const int n = pl.n, L = pl.lines;
  const int nlines = n * n;
  const int l0 = blockIdx.x * L;
  double2 *b0 = sm, *b1 = sm + L * n;
  for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
    const int l = t / n, i = t - l * n, line = l0 + l;
    double2 v = make_double2(0.0, 0.0);
    if (line < nlines) {
      if (IN_REAL)
        v.x = static_cast<const double *>(in)[(size_t)line * n + i];
      else
        v = static_cast<const double2 *>(in)[(size_t)line * n + i];
    }
    b0[t] = v;
  }
  __syncthreads();
  int Ns = 1;
  for (int s = 0; s < pl.ns; ++s) {
    const int R = pl.rad[s];
    const double2 *tw = tab + pl.tw_off[s];
    const double2 *root = tab + pl.root_off[s];
    switch (R) {
      case 4: fft_stage<4>(b0, b1, n, L, Ns, tw, root, sign, n); break;
      case 2: fft_stage<2>(b0, b1, n, L, Ns, tw, root, sign, n); break;
      case 3: fft_stage<3>(b0, b1, n, L, Ns, tw, root, sign, n); break;
      case 5: fft_stage<5>(b0, b1, n, L, Ns, tw, root, sign, n); break;
      default: fft_stage_any(R, b0, b1, n, L, Ns, tw, root, sign, n); break;
    }
    __syncthreads();
    double2 *tmp = b0;
    b0 = b1;
    b1 = tmp;
    Ns *= R;
  }
  for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
    const int k = t / L, l = t - k * L, line = l0 + l;
    if (line >= nlines) continue;
    const int a = line / n, b = line - a * n;
    const size_t o = ((size_t)k * n + a) * n + b;
    const double2 v = b0[l * n + k];
    if (OUT_REAL)
      static_cast<double *>(out)[o] = v.x * scale;
    else
      static_cast<double2 *>(out)[o] = v;
  }
}

// Real-data passes for even grids (n = 2m).  A pass transforms the A x B
// lines of an [A][B][len] array along the contiguous axis and writes the
// result transposed, [k][A][B].  MODE 0: complex to complex, length pl.n.
// MODE 1 (real to complex): a real line x of length 2m is read as the m
// complex values z_j = x_2j + i x_2j+1, transformed with the length-m plan,
// and untangled into the half spectrum X_k, k = 0..m:
//   X_k = E_k + W^k O_k,  E_k = (Z_k + conj Z_{m-k}) / 2,
//   O_k = (Z_k - conj Z_{m-k}) / (2i),  W = exp(-2 pi i / 2m),  Z_m = Z_0.
// MODE 2 (complex to real, the unnormalised inverse of a Hermitian spectrum
// given by X_0..X_m): Z''_k = (X_k + conj X_{m-k}) + i conj(W^k) (X_k -
// conj X_{m-k}) for k < m, an inverse length-m transform gives z, and
// x_2j = Re z_j, x_2j+1 = Im z_j are written to the real array [B][A][x].
template <int MODE>
__global__ void __launch_bounds__(256)
k_fft_pass_r(const void *in, void *out, FftPlan pl, const double2 *tab,
             const double2 *rtw, int A, int B, int sign) {
  extern __shared__ double2 sm[];
  const int n = pl.n, L = pl.lines;
  const int m = n;                        // MODE 1/2: the half length
  const int lin = MODE == 2 ? m + 1 : n;  // complex values read per line
  const int nlines = A * B;
  const int l0 = blockIdx.x * L;
  double2 *b0 = sm, *b1 = sm + L * (n + 1);
  const int stride = n + 1;
  if (MODE == 2) {
    for (int t = threadIdx.x; t < L * lin; t += blockDim.x) {
      const int l = t / lin, i = t - l * lin, line = l0 + l;
      b1[l * stride + i] = line < nlines
                               ? static_cast<const double2 *>(in)[(size_t)line * lin + i]
                               : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < L * m; t += blockDim.x) {
      const int l = t / m, k = t - l * m;
      const double2 xk = b1[l * stride + k], xr = b1[l * stride + (m - k)];
      const double2 cr = make_double2(xr.x, -xr.y);            // conj X_{m-k}
      const double2 sp = cadd(xk, cr), df = csub(xk, cr);
      const double2 w = rtw[k];                                 // W^k
      const double2 wc = make_double2(w.x, -w.y);               // conj W^k
      const double2 t2 = cmul(wc, df);
      b0[l * stride + k] = make_double2(sp.x - t2.y, sp.y + t2.x);   // sp + i t2
    }
  } else {
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
      const int l = t / n, i = t - l * n, line = l0 + l;
      b0[l * stride + i] = line < nlines
                               ? static_cast<const double2 *>(in)[(size_t)line * n + i]
                               : make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  int Ns = 1;
  for (int s = 0; s < pl.ns; ++s) {
    const int R = pl.rad[s];
    const double2 *tw = tab + pl.tw_off[s];
    const double2 *root = tab + pl.root_off[s];
    switch (R) {
      case 4: fft_stage<4>(b0, b1, n, L, Ns, tw, root, sign, stride); break;
      case 2: fft_stage<2>(b0, b1, n, L, Ns, tw, root, sign, stride); break;
      case 3: fft_stage<3>(b0, b1, n, L, Ns, tw, root, sign, stride); break;
      case 5: fft_stage<5>(b0, b1, n, L, Ns, tw, root, sign, stride); break;
      default: fft_stage_any(R, b0, b1, n, L, Ns, tw, root, sign, stride); break;
    }
    __syncthreads();
    double2 *tmp = b0;
    b0 = b1;
    b1 = tmp;
    Ns *= R;
  }
  if (MODE == 0) {
    for (int t = threadIdx.x; t < L * n; t += blockDim.x) {
      const int k = t / L, l = t - k * L, line = l0 + l;
      if (line >= nlines) continue;
      const int a = line / B, b = line - a * B;
      static_cast<double2 *>(out)[((size_t)k * A + a) * B + b] = b0[l * stride + k];
    }
  } else if (MODE == 1) {
    for (int t = threadIdx.x; t < L * (m + 1); t += blockDim.x) {
      const int k = t / L, l = t - k * L, line = l0 + l;
      if (line >= nlines) continue;
      const double2 zk = b0[l * stride + (k == m ? 0 : k)];
      const double2 zr = b0[l * stride + (k == 0 ? 0 : m - k)];
      const double2 cr = make_double2(zr.x, -zr.y);            // conj Z_{m-k}
      const double2 e = make_double2(0.5 * (zk.x + cr.x), 0.5 * (zk.y + cr.y));
      const double2 dd = csub(zk, cr);
      const double2 o = make_double2(0.5 * dd.y, -0.5 * dd.x);  // dd / (2i)
      const double2 xk = cadd(e, cmul(rtw[k], o));
      const int a = line / B, b = line - a * B;
      static_cast<double2 *>(out)[((size_t)k * A + a) * B + b] = xk;
    }
  } else {
    for (int t = threadIdx.x; t < L * m; t += blockDim.x) {
      const int l = t / m, j = t - l * m, line = l0 + l;
      if (line >= nlines) continue;
      const int a = line / B, b = line - a * B;
      static_cast<double2 *>(out)[((size_t)b * A + a) * m + j] = b0[l * stride + j];
    }
  }
}

// The spectral factor of the integer s = mx^2 + my^2 + mz^2 (|G|^2 = (2 pi /
// L)^2 s): the Poisson kernel c inv_s[s] when kappa < 0; otherwise Kerker's
// c s / (s + kappa), kappa = (q0 L / 2 pi)^2, with c at s = 0
__device__ __forceinline__ double spectral_factor(int s, double c, double kappa,
                                                  const double *__restrict__ inv_s) {
  if (kappa < 0.0) return c * inv_s[s];
  return s == 0 ? c : c * (double)s / ((double)s + kappa);
}

// [kz][ky][kx] (kx in 0..m) -> v(G) = factor(s) n(G) written to
// [kx][ky][kz], through 32 x 32 shared-memory tiles of each (kz, kx) plane
__global__ void __launch_bounds__(256)
k_poisson_transpose(const double2 *__restrict__ a, double2 *__restrict__ b, int n, int nh,
                    double c, double kappa, const double *__restrict__ inv_s) {
  __shared__ double2 tile[32][33];
  const int ky = blockIdx.z;
  const int kx0 = blockIdx.x * 32, kz0 = blockIdx.y * 32;
  const int my = 2 * ky < n ? ky : ky - n;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int kz = kz0 + r, kx = kx0 + threadIdx.x;
    if (kz < n && kx < nh) {
      const int mz = 2 * kz < n ? kz : kz - n;
      const int mx = kx;   // kx <= n / 2 (the Nyquist plane has |mx| = n / 2 either way)
      const double f = spectral_factor(mx * mx + my * my + mz * mz, c, kappa, inv_s);
      const double2 v = a[((size_t)kz * n + ky) * nh + kx];
      tile[r][threadIdx.x] = make_double2(f * v.x, f * v.y);
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int kx = kx0 + r, kz = kz0 + threadIdx.x;
    if (kz < n && kx < nh) b[((size_t)kx * n + ky) * n + kz] = tile[threadIdx.x][r];
  }
}

// v(G) = 4 pi n(G) / |G|^2 (G != 0), v(0) = 0; also folds in 1/N^3 of the
// unnormalised inverse transform.  |G|^2 = (2 pi / L)^2 s with the integer
// s = mx^2 + my^2 + mz^2, and inv_s[s] = 1 / s (inv_s[0] = 0) is a table per
// grid size, so v(G) = c inv_s[s] n(G), c = 4 pi / ((2 pi / L)^2 N^3).
__global__ void k_poisson_kernel(double2 *a, int n, double c, double kappa, const double *inv_s) {
  const size_t n3 = (size_t)n * n * n;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int kx = i % n, ky = (i / n) % n, kz = i / ((size_t)n * n);
  const int mx = 2 * kx < n ? kx : kx - n;
  const int my = 2 * ky < n ? ky : ky - n;
  const int mz = 2 * kz < n ? kz : kz - n;
  const double f = spectral_factor(mx * mx + my * my + mz * mz, c, kappa, inv_s);
  double2 v = a[i];
  v.x *= f;
  v.y *= f;
  a[i] = v;
}

// The same multiplication with 4 pi / |G|^2 evaluated in place (no table):
// used by the allocation-free entry point.
__global__ void k_poisson_kernel_direct(double2 *a, int n, double L) {
  const size_t n3 = (size_t)n * n * n;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int kx = i % n, ky = (i / n) % n, kz = i / ((size_t)n * n);
  const int mx = 2 * kx < n ? kx : kx - n;
  const int my = 2 * ky < n ? ky : ky - n;
  const int mz = 2 * kz < n ? kz : kz - n;
  const double g = 2.0 * M_PI / L;
  const double gx = g * mx, gy = g * my, gz = g * mz;
  const double G2 = gz * gz + gy * gy + gx * gx;
  double2 v = a[i];
  if (mx == 0 && my == 0 && mz == 0) {
    v = make_double2(0.0, 0.0);
  } else {
    const double f = 4.0 * M_PI / G2 / (double)n3;
    v.x *= f;
    v.y *= f;
  }
  a[i] = v;
}

// Perdew-Zunger LDA (unpolarised): eps_xc, v_xc; vhxc = v_h + v_xc.
__global__ void k_lda(int n3, const double *rho, const double *vh,
                      double *eps, double *vxc, double *vhxc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double r = rho[i];
  double e = 0.0, v = 0.0;
  if (r >= 1e-30) {
    // one cube root: (3 r / pi)^(1/3) = c1 r^(1/3), r_s = c2 / r^(1/3)
    const double t = cbrt(r);
    const double ex = -0.75 * (0.98474502184269654115 * t);   // (3/pi)^(1/3)
    const double vx = (4.0 / 3.0) * ex;
    const double rs = 0.62035049089940001667 / t;             // (3/(4 pi))^(1/3)
    double ec, vc;
    if (rs >= 1.0) {
      using namespace pz81;
      const double s = sqrt(rs);
      const double q = 1.0 + b1 * s + b2 * rs;
      ec = gam / q;
      vc = gam * (1.0 + (7.0 / 6.0) * b1 * s + (4.0 / 3.0) * b2 * rs) / (q * q);
    } else {
      using namespace pz81;
      const double lx = log(rs);
      ec = A * lx + B + C * rs * lx + D * rs;
      vc = A * lx + (B - A / 3.0) + (2.0 / 3.0) * C * rs * lx +
           ((2.0 * D - C) / 3.0) * rs;
    }
    e = ex + ec;
    v = vx + vc;
  }
  eps[i] = e;
  vxc[i] = v;
  vhxc[i] = vh[i] + v;
}

// v_eff = v_loc + extrapolated v_Hxc + field * (z - L/2).
__global__ void k_veff(int n, double h, double L, const double *vloc,
                       const double *h0, const double *h1, const double *h2,
                       int hist_len, double field, double *ve, float *vef,
                       float4 *vdiag, double w0) {
  const int n3 = n * n * n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double x;
  if (hist_len <= 1)
    x = h0[i];
  else if (hist_len == 2)
    x = 2.0 * h0[i] - h1[i];
  else
    x = 3.0 * h0[i] - 3.0 * h1[i] + h2[i];
  double v = vloc[i] + x;
  if (field != 0.0) {
    const int z = i / (n * n);
    v += field * (z * h - 0.5 * L);
  }
  ve[i] = v;
  if (vef) vef[i] = (float)v;
  if (vdiag) {
    const float d = (float)(w0 + v);
    vdiag[i] = make_float4(d, d, d, d);
  }
}

// partial[b] = sum over block b of (a - c)(b + d) (c, d optional).
__global__ void __launch_bounds__(256)
k_dot4(int n, const double *a, const double *b, const double *c,
       const double *d, double *part) {
  __shared__ double red[8];
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const double x = c ? a[i] - c[i] : a[i];
    const double y = b ? (d ? b[i] + d[i] : b[i]) : 1.0;
    acc[0] += x * y;
  }
  emd_block_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

__global__ void __launch_bounds__(256)
k_sum(const double *part, int n, double *out) {
  __shared__ double red[8];
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc[0] += part[i];
  emd_block_sum<1>(acc, red);
  if (threadIdx.x == 0) *out = acc[0];
}

// FFT plans with their device twiddle tables, one per (device, grid size),
// created on first use and kept for the life of the process.
struct PlanCache {
  int dev = -1, n = -1;
  FftPlan plan;
  double2 *tab = nullptr;
  double *inv_s = nullptr;   // 1 / s for s = 0 .. 3 (n/2)^2, inv_s[0] = 0
  double2 *rtw = nullptr;    // even n: W^k = exp(-2 pi i k / n), k = 0 .. n/2
};
std::mutex g_plan_mu;
std::vector<PlanCache *> g_plans;

const PlanCache *get_plan(int n) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (PlanCache *c : g_plans)
    if (c->n == n && c->dev == dev) return c;
  PlanCache *c = new PlanCache();
  std::vector<double2> tab;
  if (!make_plan(n, c->plan, tab) ||
      cudaMalloc(&c->tab, tab.size() * sizeof(double2)) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  if (cudaMemcpy(c->tab, tab.data(), tab.size() * sizeof(double2),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(c->tab);
    delete c;
    return nullptr;
  }
  if (n % 2 == 0) {
    std::vector<double2> w(n / 2 + 1);
    for (int k = 0; k <= n / 2; ++k) w[k] = unit_root(k, n);
    if (cudaMalloc(&c->rtw, w.size() * sizeof(double2)) != cudaSuccess ||
        cudaMemcpy(c->rtw, w.data(), w.size() * sizeof(double2), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaFree(c->tab);
      if (c->rtw) cudaFree(c->rtw);
      delete c;
      return nullptr;
    }
  }
  const int smax = 3 * (n / 2) * (n / 2);
  std::vector<double> inv(smax + 1);
  inv[0] = 0.0;
  for (int q = 1; q <= smax; ++q) inv[q] = 1.0 / (double)q;
  if (cudaMalloc(&c->inv_s, inv.size() * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(c->inv_s, inv.data(), inv.size() * sizeof(double),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(c->tab);
    if (c->inv_s) cudaFree(c->inv_s);
    delete c;
    return nullptr;
  }
  c->n = n;
  c->dev = dev;
  g_plans.push_back(c);
  return c;
}

}  // namespace

void emd_fft_plan_check(int n, int *ok) {
  FftPlan p;
  std::vector<double2> t;
  *ok = make_plan(n, p, t);
}

int emd_fft_prepare(int n) {
  if (get_plan(n) == nullptr) return 1;
  if (n % 2 == 0 && get_plan(n / 2) == nullptr) return 1;
  return 0;
}

namespace {

// v = the inverse transform of factor(s) times the transform of the real grid
// `charge` (spectral_factor; cpois includes the 1/N^3 of the inverse);
// `charge` is read by the first pass only, so v may alias it
void spectral_multiply(const GridInfo &g, const double *charge, double *v, double2 *wa,
                       double2 *wb, double cpois, double kappa, cudaStream_t st) {
  const PlanCache *pc = get_plan(g.n);
  const int n = g.n;
  if (n % 2 == 0) {
    // real data: half-length transforms along x, half spectrum in kx
    emd_note_launches(7);
    const int m = n / 2, nh = m + 1;
    const PlanCache *ph = get_plan(m);
    const FftPlan &pf = pc->plan, &pm = ph->plan;
    const size_t smf = 2 * (size_t)pf.lines * (n + 1) * sizeof(double2);
    const size_t smm = 2 * (size_t)pm.lines * (m + 1) * sizeof(double2);
    const int bx = (n * n + pm.lines - 1) / pm.lines;     // lines along x
    const int bh = (nh * n + pf.lines - 1) / pf.lines;    // lines along y or z
    k_fft_pass_r<1><<<bx, 256, smm, st>>>(charge, wa, pm, ph->tab, pc->rtw, n, n, -1);
    k_fft_pass_r<0><<<bh, 256, smf, st>>>(wa, wb, pf, pc->tab, nullptr, nh, n, -1);
    k_fft_pass_r<0><<<bh, 256, smf, st>>>(wb, wa, pf, pc->tab, nullptr, n, nh, -1);
    k_poisson_transpose<<<dim3((nh + 31) / 32, (n + 31) / 32, n), dim3(32, 8), 0, st>>>(
        wa, wb, n, nh, cpois, kappa, pc->inv_s);
    k_fft_pass_r<0><<<bh, 256, smf, st>>>(wb, wa, pf, pc->tab, nullptr, nh, n, +1);
    k_fft_pass_r<0><<<bh, 256, smf, st>>>(wa, wb, pf, pc->tab, nullptr, n, nh, +1);
    k_fft_pass_r<2><<<bx, 256, smm, st>>>(wb, v, pm, ph->tab, pc->rtw, n, n, +1);
    return;
  }
  emd_note_launches(7);
  const FftPlan &p = pc->plan;
  const int blocks = (g.n * g.n + p.lines - 1) / p.lines;
  const size_t smem = 2 * (size_t)p.lines * g.n * sizeof(double2);
  k_fft_pass<true, false><<<blocks, 256, smem, st>>>(charge, wa, p, pc->tab, -1, 1.0);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wa, wb, p, pc->tab, -1, 1.0);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wb, wa, p, pc->tab, -1, 1.0);
  k_poisson_kernel<<<(g.n3 + 255) / 256, 256, 0, st>>>(wa, g.n, cpois, kappa, pc->inv_s);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wa, wb, p, pc->tab, +1, 1.0);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wb, wa, p, pc->tab, +1, 1.0);
  k_fft_pass<false, true><<<blocks, 256, smem, st>>>(wa, v, p, pc->tab, +1, 1.0);
}

}  // namespace

void emd_launch_poisson(const GridInfo &g, const double *charge, double *v,
                        double2 *wa, double2 *wb, cudaStream_t st) {
  const double gq = 2.0 * M_PI / g.L;
  spectral_multiply(g, charge, v, wa, wb, 4.0 * M_PI / (gq * gq) / (double)g.n3, -1.0, st);
}

void emd_launch_kerker(const GridInfo &g, double q0, const double *r, double *out,
                       double2 *wa, double2 *wb, cudaStream_t st) {
  const double k = q0 * g.L / (2.0 * M_PI);
  spectral_multiply(g, r, out, wa, wb, 1.0 / (double)g.n3, k * k, st);
}

void emd_launch_lda(int n3, const double *rho, const double *v_h,
                    double *eps_xc, double *v_xc, double *vhxc,
                    cudaStream_t st) {
  emd_note_launches(1);
  k_lda<<<(n3 + 255) / 256, 256, 0, st>>>(n3, rho, v_h, eps_xc, v_xc, vhxc);
}

void emd_launch_veff(const GridInfo &g, const double *v_loc,
                     const double *const *hist, int hist_len, double field,
                     double *v_eff, float *v_eff_f, cudaStream_t st,
                     float4 *v_diag, double w0) {
  emd_note_launches(1);
  k_veff<<<(g.n3 + 255) / 256, 256, 0, st>>>(
      g.n, g.h, g.L, v_loc, hist[0], hist_len > 1 ? hist[1] : hist[0],
      hist_len > 2 ? hist[2] : hist[0], hist_len, field, v_eff, v_eff_f, v_diag, w0);
}

void emd_launch_dot_partials(int n3, const double *a, const double *b,
                             const double *c, const double *d,
                             double *partials, int nblocks, cudaStream_t st) {
  emd_note_launches(1);
  k_dot4<<<nblocks, 256, 0, st>>>(n3, a, b, c, d, partials);
}

void emd_launch_sum(const double *partials, int n, double *out,
                    cudaStream_t st) {
  emd_note_launches(1);
  k_sum<<<1, 256, 0, st>>>(partials, n, out);
}

// ===========================================================================
// Poisson solve that allocates nothing (emd_poisson_static).
//
// For callers that cannot allocate device memory: code that runs while a
// CUDA graph is being captured (cudaMalloc is not capturable), applications
// whose device memory is owned by another allocator or a fixed budget, and
// latency-critical loops where cudaMalloc/cudaFree would synchronise the
// device.  The FFT work arrays and the twiddle table live in one file-scope
// __device__ array of fixed size, present on every GPU that loads the
// library until the process exits.
// ===========================================================================
namespace {

constexpr int kStaticMaxN = 64;                       // largest grid edge
constexpr size_t kStaticN3 = (size_t)kStaticMaxN * kStaticMaxN * kStaticMaxN;
constexpr int kStaticTab = 2048;                      // twiddle entries
// [0, N^3): work a, [N^3, 2 N^3): work b, then the twiddle table
__device__ __align__(256) double2 g_static_scratch[2 * kStaticN3 + kStaticTab];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double2 *g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set-up on the
// first call per device).  In host code the symbol is only a stand-in.
cudaError_t static_scratch(double2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = static_cast<double2 *>(p);
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

// Plan offsets only (no table, no heap): same radix order as make_plan.
bool plan_offsets(int n, FftPlan &p) {
  p.n = n;
  p.ns = 0;
  int m = n;
  const int order[] = {4, 2, 3, 5, 7, 11, 13};
  for (int r : order) {
    while (m % r == 0) {
      if (p.ns >= kMaxStages) return false;
      p.rad[p.ns++] = r;
      m /= r;
    }
  }
  if (m != 1) return false;
  int off = 0, Ns = 1;
  for (int s = 0; s < p.ns; ++s) {
    p.tw_off[s] = off;
    off += Ns * p.rad[s];
    p.root_off[s] = off;
    off += p.rad[s];
    Ns *= p.rad[s];
  }
  if (off > kStaticTab) return false;
  p.lines = n >= 1280 ? 1 : (1280 / n > 8 ? 8 : 1280 / n);
  return true;
}

// Twiddles and roots of the plan, computed on the device with sincospi.
__global__ void k_fill_twiddles(FftPlan p, double2 *tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int Ns = 1;
  for (int s = 0; s < p.ns; ++s) {
    const int R = p.rad[s];
    if (i >= p.tw_off[s] && i < p.tw_off[s] + Ns * R) {
      const int k = i - p.tw_off[s];
      const int jm = k / R, r = k % R;
      const long num = (long)jm * r % ((long)Ns * R);
      double sn, cs;
      sincospi(-2.0 * (double)num / (double)(Ns * R), &sn, &cs);
      tab[i] = make_double2(cs, sn);
    } else if (i >= p.root_off[s] && i < p.root_off[s] + R) {
      const int q = i - p.root_off[s];
      double sn, cs;
      sincospi(-2.0 * (double)q / (double)R, &sn, &cs);
      tab[i] = make_double2(cs, sn);
    }
    Ns *= R;
  }
}

}  // namespace

extern "C" int emd_poisson_static(int n, double h, const double *charge,
                                  double *v, void *cuda_stream) {
  if (!charge || !v || !(h > 0.0) || n < 2)
    return emd_set_error(EMD_EINVAL, "emd_poisson_static: NULL pointer, h <= 0 or n < 2");
  if (n > kStaticMaxN)
    return emd_set_error(EMD_EINVAL, "emd_poisson_static: n exceeds the static "
                                     "scratch limit of 64 points per axis");
  FftPlan p;
  if (!plan_offsets(n, p))
    return emd_set_error(EMD_EINVAL, "emd_poisson_static: n has a prime factor above 13");
  double2 *base = nullptr;
  if (static_scratch(&base) != cudaSuccess)
    return emd_set_error(EMD_ECUDA, "emd_poisson_static: cudaGetSymbolAddress of "
                                    "the static scratch failed");
  const size_t n3 = (size_t)n * n * n;
  double2 *wa = base, *wb = base + kStaticN3, *tab = base + 2 * kStaticN3;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_fill_twiddles<<<(kStaticTab + 255) / 256, 256, 0, st>>>(p, tab);
  const int blocks = (n * n + p.lines - 1) / p.lines;
  const size_t smem = 2 * (size_t)p.lines * n * sizeof(double2);
  const double L = n * h;
  k_fft_pass<true, false><<<blocks, 256, smem, st>>>(charge, wa, p, tab, -1, 1.0);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wa, wb, p, tab, -1, 1.0);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wb, wa, p, tab, -1, 1.0);
  k_poisson_kernel_direct<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(wa, n, L);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wa, wb, p, tab, +1, 1.0);
  k_fft_pass<false, false><<<blocks, 256, smem, st>>>(wb, wa, p, tab, +1, 1.0);
  k_fft_pass<false, true><<<blocks, 256, smem, st>>>(wa, v, p, tab, +1, 1.0);
  if (cudaGetLastError() != cudaSuccess)
    return emd_set_error(EMD_ECUDA, "emd_poisson_static: kernel launch failed");
  return emd_set_error(EMD_OK, "");
}
