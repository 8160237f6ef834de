// Kernels of the ground-state solver (the KS equations at fixed ions, Sec.
// 4.1, eqs. EoM_BO_a and EoM_BO_b): one step of the Chebyshev three-term
// recurrence over an orbital set, weighted sums of density grids (Anderson
// mixing), the L1 distance of two densities, and the Rayleigh-Ritz subspace
// products (the overlap and Hamiltonian matrices X^H Y of two tall n3 x m
// sets, and the rotation X V).  The driver, with the dense m x m generalized
// eigenproblem on the host, is in emd_api.cu.

#include <algorithm>

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

// ---- per-orbital weights ----------------------------------------------------
// u_A <- w_A u_A for the orbitals A < n_orb of a packed set (element i of
// [n_blk][n3][bo] belongs to orbital (i / (bo n3)) bo + i % bo); the padding
// orbitals are left alone.  The product is formed in FP64.
template <typename V>
__global__ void k_scale_packed(V *u, size_t n3, int bo, int n_orb, size_t tot,
                               const double *__restrict__ w) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int A = (int)(i / ((size_t)bo * n3)) * bo + (int)(i % (size_t)bo);
  if (A >= n_orb) return;
  const double f = w[A];
  V v = u[i];
  v.x = (double)v.x * f;
  v.y = (double)v.y * f;
  u[i] = v;
}

// c_A <- w_A c_A over the n_vec columns of a canonical set (column A at c + A n3)
template <typename V>
__global__ void k_scale_canon(V *c, size_t n3, size_t tot, const double *__restrict__ w) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const double f = w[i / n3];
  V v = c[i];
  v.x = (double)v.x * f;
  v.y = (double)v.y * f;
  c[i] = v;
}

// ---- subspace products ----------------------------------------------------
// X, Y: canonical column-major sets, column i at X + i n3 (complex128, or
// complex64 read into FP64 sums).  G = h^3 X^H Y, m x m, column-major FP64.
// k_gram: CTA (row chunk, 16 x 16 tile of G); the chunk's rows pass through
// shared memory 32 at a time; complex64 products are summed in FP32 over
// those 32 rows and added to the FP64 sums; the chunks' partial tiles are
// added in chunk order by k_gram_sum (deterministic).
template <typename C> struct GramT;
template <> struct GramT<double2> {
  __device__ static double2 load(const double2 *p) { return *p; }
};
template <> struct GramT<float2> {
  __device__ static double2 load(const float2 *p) {
    const float2 v = *p;
    return make_double2((double)v.x, (double)v.y);
  }
};

template <typename C>
__global__ void __launch_bounds__(256)
k_gram(const C *__restrict__ X, const C *__restrict__ Y, int n3, int m, int rows,
       double2 *__restrict__ part) {
  __shared__ C xs[32][17], ys[32][17];
  const int chunk = blockIdx.x, i0 = blockIdx.y * 16, j0 = blockIdx.z * 16;
  const int a = threadIdx.x & 15, b = threadIdx.x >> 4;     // G entry (i0 + a, j0 + b)
  const int r0 = chunk * rows, r1 = min(n3, r0 + rows);
  double sr = 0.0, si = 0.0;
  for (int rb = r0; rb < r1; rb += 32) {
    // stage rows rb .. rb + 31 of the 16 columns of X and of Y: thread
    // (row, column pair) loads two values of each
    for (int q = threadIdx.x; q < 32 * 16; q += 256) {
      const int r = q & 31, c = q >> 5;
      const bool okx = rb + r < r1 && i0 + c < m, oky = rb + r < r1 && j0 + c < m;
      C zero;
      zero.x = 0;
      zero.y = 0;
      xs[r][c] = okx ? X[(size_t)(i0 + c) * n3 + rb + r] : zero;
      ys[r][c] = oky ? Y[(size_t)(j0 + c) * n3 + rb + r] : zero;
    }
    __syncthreads();
    if (sizeof(C) == 16) {
      for (int r = 0; r < 32; ++r) {
        const double2 x = GramT<C>::load(&xs[r][a]), y = GramT<C>::load(&ys[r][b]);
        sr = fma(x.x, y.x, fma(x.y, y.y, sr));           // conj(x) y
        si = fma(x.x, y.y, fma(-x.y, y.x, si));
      }
    } else {
      float fr = 0.f, fi = 0.f;
      for (int r = 0; r < 32; ++r) {
        const float2 x = *reinterpret_cast<const float2 *>(&xs[r][a]);
        const float2 y = *reinterpret_cast<const float2 *>(&ys[r][b]);
        fr = fmaf(x.x, y.x, fmaf(x.y, y.y, fr));
        fi = fmaf(x.x, y.y, fmaf(-x.y, y.x, fi));
      }
      sr += (double)fr;
      si += (double)fi;
    }
    __syncthreads();
  }
  if (i0 + a < m && j0 + b < m)
    part[((size_t)chunk * m + (j0 + b)) * m + i0 + a] = make_double2(sr, si);
}

__global__ void k_gram_sum(const double2 *__restrict__ part, int nchunk, int m, double scale,
                           double2 *__restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * m) return;
  double sr = 0.0, si = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double2 v = part[(size_t)c * m * m + i];
    sr += v.x;
    si += v.y;
  }
  G[i] = make_double2(scale * sr, scale * si);
}

// B = X V: X canonical n3 x m, V column-major m x m (FP64), B canonical.
// CTA: 64 rows x 16 columns of B; k in steps of 16 through shared memory;
// FP64 sums (complex64 X widened on load, the result rounded to complex64).
template <typename C>
__global__ void __launch_bounds__(256)
k_rotate(const C *__restrict__ X, const double2 *__restrict__ V, int n3, int m,
         C *__restrict__ B) {
  __shared__ double2 xs[16][65], vs[16][17];
  const int r0 = blockIdx.x * 64, j0 = blockIdx.y * 16;
  const int rr = threadIdx.x & 63, jq = threadIdx.x >> 6;   // 4 columns per thread
  double2 acc[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) acc[t] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < m; k0 += 16) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int r = q & 63, k = q >> 6;
      xs[k][r] = (r0 + r < n3 && k0 + k < m) ? GramT<C>::load(X + (size_t)(k0 + k) * n3 + r0 + r)
                                              : make_double2(0.0, 0.0);
    }
    {
      const int k = threadIdx.x & 15, j = threadIdx.x >> 4;
      vs[k][j] = (k0 + k < m && j0 + j < m) ? V[(size_t)(j0 + j) * m + k0 + k]
                                            : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
      const double2 x = xs[k][rr];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const double2 v = vs[k][4 * jq + t];
        acc[t].x = fma(x.x, v.x, fma(-x.y, v.y, acc[t].x));
        acc[t].y = fma(x.x, v.y, fma(x.y, v.x, acc[t].y));
      }
    }
    __syncthreads();
  }
  if (r0 + rr < n3)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = j0 + 4 * jq + t;
      if (j < m) {
        C o;
        o.x = acc[t].x;
        o.y = acc[t].y;
        B[(size_t)j * n3 + r0 + rr] = o;
      }
    }
}

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

// G = scale X^H Y (m x m, column-major FP64); part: scratch of
// emd_gram_scratch(n3, m) double2
int emd_gram_chunks(int n3) { return std::max(1, std::min(64, n3 / 4096)); }
size_t emd_gram_scratch(int n3, int m) { return (size_t)emd_gram_chunks(n3) * m * m; }

void emd_launch_gram(int prec, const void *X, const void *Y, int n3, int m, double scale,
                     double2 *part, double2 *G, cudaStream_t st) {
  emd_note_launches(2);
  const int nchunk = emd_gram_chunks(n3);
  const int rows = (n3 + nchunk - 1) / nchunk;
  const dim3 grid(nchunk, (m + 15) / 16, (m + 15) / 16);
  if (prec == EMD_FP64)
    k_gram<double2><<<grid, 256, 0, st>>>((const double2 *)X, (const double2 *)Y, n3, m, rows, part);
  else
    k_gram<float2><<<grid, 256, 0, st>>>((const float2 *)X, (const float2 *)Y, n3, m, rows, part);
  k_gram_sum<<<(m * m + 255) / 256, 256, 0, st>>>(part, nchunk, m, scale, G);
}

void emd_launch_rotate(int prec, const void *X, const double2 *V, int n3, int m, void *B,
                       cudaStream_t st) {
  emd_note_launches(1);
  const dim3 grid((n3 + 63) / 64, (m + 15) / 16);
  if (prec == EMD_FP64)
    k_rotate<double2><<<grid, 256, 0, st>>>((const double2 *)X, V, n3, m, (double2 *)B);
  else
    k_rotate<float2><<<grid, 256, 0, st>>>((const float2 *)X, V, n3, m, (float2 *)B);
}

void emd_launch_scale_orbitals(const OrbLayout &o, void *u, int n_orb, const double *w,
                               cudaStream_t st) {
  emd_note_launches(1);
  const size_t tot = (size_t)((n_orb + o.bo - 1) / o.bo) * o.n3 * o.bo;
  if (o.prec == EMD_FP64)
    k_scale_packed<double2><<<blocks(tot), 256, 0, st>>>((double2 *)u, (size_t)o.n3, o.bo,
                                                          n_orb, tot, w);
  else
    k_scale_packed<float2><<<blocks(tot), 256, 0, st>>>((float2 *)u, (size_t)o.n3, o.bo,
                                                         n_orb, tot, w);
}

void emd_launch_scale_canon(bool c64, void *c, size_t n3, int n_vec, const double *w,
                            cudaStream_t st) {
  if (n_vec <= 0) return;
  emd_note_launches(1);
  const size_t tot = n3 * (size_t)n_vec;
  if (c64)
    k_scale_canon<float2><<<blocks(tot), 256, 0, st>>>((float2 *)c, n3, tot, w);
  else
    k_scale_canon<double2><<<blocks(tot), 256, 0, st>>>((double2 *)c, n3, tot, w);
}
