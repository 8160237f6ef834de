// Element-wise kernels of the ground-state solver (the KS equations at fixed
// ions, Sec. 4.1, eqs. EoM_BO_a and EoM_BO_b): one step of the Chebyshev
// three-term recurrence over an orbital set, weighted sums of density grids
// (Anderson mixing) and the L1 distance of two densities.  The driver, with
// the subspace GEMMs and the dense generalized eigenproblem, is in
// emd_api.cu.

#include "emd_internal.cuh"

namespace {

// out = alpha (w - c y) - beta out; with beta = 0 out is only written.
// out may alias neither w nor y.
template <typename T, typename V>
__global__ void k_cheb(size_t n, const V *__restrict__ w, const V *__restrict__ y,
                       V *out, T alpha, T c, T beta) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V a = w[i], b = y[i];
  V r;
  r.x = alpha * (a.x - c * b.x);
  r.y = alpha * (a.y - c * b.y);
  if (beta != (T)0) {
    const V z = out[i];
    r.x -= beta * z.x;
    r.y -= beta * z.y;
  }
  out[i] = r;
}

__global__ void k_comb(int n3, EmdComb cb, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double s = 0.0;
  for (int k = 0; k < cb.m; ++k) s += cb.w[k] * cb.p[k][i];
  out[i] = s;
}

__global__ void __launch_bounds__(256)
k_absdiff(int n, const double *__restrict__ a, const double *__restrict__ b,
          double *__restrict__ part) {
  __shared__ double red[8];
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc[0] += fabs(a[i] - b[i]);
  emd_block_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

__global__ void k_widen(size_t n, const float2 *__restrict__ a, double2 *__restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

__global__ void k_narrow(size_t n, const double2 *__restrict__ a, float2 *__restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// columns c0 .. c1-1 of a canonical (column-major n3 x m) set: uniform
// values in [-1, 1) from a counter hash of (seed, element index)
template <typename V>
__global__ void k_fill_random(V *x, size_t n3, int c0, int c1, unsigned seed) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = n3 * (size_t)(c1 - c0);
  if (i >= total) return;
  const size_t e = (size_t)c0 * n3 + i;
  uint64_t z = (uint64_t)e * 2ull + ((uint64_t)seed << 40);
  V v;
  for (int k = 0; k < 2; ++k) {
    uint64_t q = z + (uint64_t)k + 0x9E3779B97F4A7C15ull;   // splitmix64
    q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
    q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
    q ^= q >> 31;
    const double u = (double)(q >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    if (k == 0) v.x = u;
    else v.y = u;
  }
  x[e] = v;
}

inline unsigned blocks(size_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void emd_launch_cheb(int prec, size_t n, const void *w, const void *y, void *out,
                     double alpha, double c, double beta, cudaStream_t st) {
  emd_note_launches(1);
  if (prec == EMD_FP64)
    k_cheb<double, double2><<<blocks(n), 256, 0, st>>>(
        n, (const double2 *)w, (const double2 *)y, (double2 *)out, alpha, c, beta);
  else
    k_cheb<float, float2><<<blocks(n), 256, 0, st>>>(
        n, (const float2 *)w, (const float2 *)y, (float2 *)out, (float)alpha, (float)c,
        (float)beta);
}

void emd_launch_comb(int n3, const EmdComb &cb, double *out, cudaStream_t st) {
  emd_note_launches(1);
  k_comb<<<blocks(n3), 256, 0, st>>>(n3, cb, out);
}

void emd_launch_absdiff_partials(int n3, const double *a, const double *b, double *part,
                                 int nblocks, cudaStream_t st) {
  emd_note_launches(1);
  k_absdiff<<<nblocks, 256, 0, st>>>(n3, a, b, part);
}

void emd_launch_widen(size_t n, const float2 *a, double2 *b, cudaStream_t st) {
  emd_note_launches(1);
  k_widen<<<blocks(n), 256, 0, st>>>(n, a, b);
}

void emd_launch_narrow(size_t n, const double2 *a, float2 *b, cudaStream_t st) {
  emd_note_launches(1);
  k_narrow<<<blocks(n), 256, 0, st>>>(n, a, b);
}

void emd_launch_fill_random(int prec, void *canon, size_t n3, int c0, int c1, unsigned seed,
                            cudaStream_t st) {
  if (c1 <= c0) return;
  emd_note_launches(1);
  const size_t total = n3 * (size_t)(c1 - c0);
  if (prec == EMD_FP64)
    k_fill_random<double2><<<blocks(total), 256, 0, st>>>((double2 *)canon, n3, c0, c1, seed);
  else
    k_fill_random<float2><<<blocks(total), 256, 0, st>>>((float2 *)canon, n3, c0, c1, seed);
}
