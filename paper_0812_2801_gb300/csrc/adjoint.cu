// Kernels of the discrete adjoint (backward-in-time) propagation, FP64.
//
// The forward map is the MD step of the modified Ehrenfest scheme with the
// ions held fixed (paper Sec. 5.1: AETRS, eq. aetrs, with Taylor-4 halves in
// nested form; tau = dt/(2 mu), eq. transf; the density of eq. density feeds
// Hartree + LDA, extrapolated for H(t+dt)).  With the convention
// dL = Re sum_{A,r} conj(lambda_A(r)) dpsi_A(r), the reverse of one nested
// stage u_k = psi0 + a_k H u_{k+1}, a_k = -i tau/k, is
//   lambda_psi0 += mu_k,   mu_{k+1} = conj(a_k) H mu_k           (H Hermitian)
//   g_v(r)      += (tau/k) Im sum_A conj(mu_k,A(r)) u_{k+1,A}(r)  (dL/dv_eff)
//   g_R[J]      += (h_kb tau/(k h^3)) Im sum_A [conj(dc_J(mu)) c_J(u)
//                                              + conj(c_J(mu)) dc_J(u)]
// where c_J(x) = h^3 sum p_J x and dc_J(x) = h^3 sum dp_J/dR_J x.
#include "emd_internal.cuh"

namespace {

// y += x over n complex values
__global__ void k_axpy(double2 *y, const double2 *x, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 a = y[i], b = x[i];
    y[i] = make_double2(a.x + b.x, a.y + b.y);
  }
}

// g[p] += b * Im sum_{blk, j} conj(mu) u
template <int BO>
__global__ void k_gv_accum(const double2 *__restrict__ mu,
                           const double2 *__restrict__ u, size_t n3, int n_blk,
                           double b, double *g) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n3) return;
  double s = 0.0;
  for (int k = 0; k < n_blk; ++k) {
    const size_t o = ((size_t)k * n3 + p) * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const double2 m = mu[o + j], v = u[o + j];
      s += m.x * v.y - m.y * v.x;   // Im(conj(m) v)
    }
  }
  g[p] += b * s;
}

// c = h^3 sum p x, dc_a = h^3 sum p d_a / r_c^2 x per (atom, orbital);
// hc = h_kb c.  One block per (atom, orbital block), fixed-order sums.
template <int BO>
__global__ void __launch_bounds__(256)
k_project_grad(const double2 *__restrict__ x, size_t n3, const int *at_cnt,
               const int *at_pt, const double *at_p, const double *at_d,
               int cap, double h3, double h_kb, double inv_rc2, int n_orb_pad,
               double2 *c, double2 *hc, double2 *dc) {
  __shared__ double red[8 * 8 * BO];
  const int J = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[J];
  const double2 *xb = x + (size_t)blk * n3 * BO;
  double acc[8 * BO];
#pragma unroll
  for (int k = 0; k < 8 * BO; ++k) acc[k] = 0.0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const size_t idx = (size_t)J * cap + e;
    const int pt = at_pt[idx];
    const double pv = at_p[idx];
    const double q = pv * inv_rc2;
    const double d0 = at_d[3 * idx], d1 = at_d[3 * idx + 1], d2 = at_d[3 * idx + 2];
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const double2 v = xb[(size_t)pt * BO + j];
      acc[8 * j + 0] += pv * v.x;
      acc[8 * j + 1] += pv * v.y;
      acc[8 * j + 2] += q * d0 * v.x;
      acc[8 * j + 3] += q * d0 * v.y;
      acc[8 * j + 4] += q * d1 * v.x;
      acc[8 * j + 5] += q * d1 * v.y;
      acc[8 * j + 6] += q * d2 * v.x;
      acc[8 * j + 7] += q * d2 * v.y;
    }
  }
  emd_block_sum<8 * BO>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const size_t o = (size_t)J * n_orb_pad + (size_t)blk * BO + j;
      c[o] = make_double2(h3 * acc[8 * j], h3 * acc[8 * j + 1]);
      hc[o] = make_double2(h_kb * h3 * acc[8 * j], h_kb * h3 * acc[8 * j + 1]);
      for (int a = 0; a < 3; ++a)
        dc[3 * o + a] = make_double2(h3 * acc[8 * j + 2 + 2 * a], h3 * acc[8 * j + 3 + 2 * a]);
    }
  }
}

// gR[J][a] += coef * Im sum_A [conj(dcm) cu + conj(cm) dcu]
__global__ void k_proj_sens(const double2 *cm, const double2 *dcm,
                            const double2 *cu, const double2 *dcu, int n_atoms,
                            int n_orb, int n_orb_pad, double coef, double *gR) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n_atoms) return;
  const int J = i / 3, a = i % 3;
  double s = 0.0;
  for (int A = 0; A < n_orb; ++A) {
    const size_t o = (size_t)J * n_orb_pad + A;
    const double2 dm = dcm[3 * o + a], m = cm[o], u = cu[o], du = dcu[3 * o + a];
    // Im(conj(dm) u) + Im(conj(m) du)
    s += (dm.x * u.y - dm.y * u.x) + (m.x * du.y - m.y * du.x);
  }
  gR[i] += coef * s;
}

// f_xc = d v_xc / d rho of the Perdew-Zunger LDA (derivative of the
// potential formulas used by the forward step).
__device__ double fxc_pz81(double r) {
  if (r < 1e-30) return 0.0;
  const double vx = -(cbrt(3.0 * r / M_PI));          // (4/3) eps_x
  const double dvx = vx / (3.0 * r);
  const double rs = cbrt(3.0 / (4.0 * M_PI * r));
  const double drs = -rs / (3.0 * r);
  double dvc;
  if (rs >= 1.0) {
    const double gam = -0.1423, b1 = 1.0529, b2 = 0.3334;
    const double s = sqrt(rs);
    const double q = 1.0 + b1 * s + b2 * rs;
    const double nn = 1.0 + (7.0 / 6.0) * b1 * s + (4.0 / 3.0) * b2 * rs;
    const double dq = b1 / (2.0 * s) + b2;
    const double dn = (7.0 / 6.0) * b1 / (2.0 * s) + (4.0 / 3.0) * b2;
    dvc = gam * (dn * q - 2.0 * nn * dq) / (q * q * q);
  } else {
    const double A = 0.0311, C = 0.0020, D = -0.0116;
    dvc = A / rs + (2.0 / 3.0) * C * (log(rs) + 1.0) + (2.0 * D - C) / 3.0;
  }
  return dvx + dvc * drs;
}

// lam_rho = pois + f_xc(rho) lam_v  (pois = Poisson(lam_v), computed before)
__global__ void k_rho_adjoint(int n3, const double *rho, const double *lam_v,
                              double *pois_inout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) pois_inout[i] += fxc_pz81(rho[i]) * lam_v[i];
}

// lam[A](r) += scale * w(r) * psi[A](r)  (w real grid)
template <int BO>
__global__ void k_scale_add(double2 *lam, const double2 *psi, const double *w,
                            size_t n3, int n_blk, double scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n_blk * n3 * BO) return;
  const size_t p = (i / BO) % n3;
  const double f = scale * w[p];
  const double2 v = psi[i], l = lam[i];
  lam[i] = make_double2(l.x + f * v.x, l.y + f * v.y);
}

// out = a0 x0 + a1 x1 + a2 x2 + a3 x3 (grids; NULL inputs skipped)
__global__ void k_lincomb(int n, double *out, double a0, const double *x0,
                          double a1, const double *x1, double a2,
                          const double *x2, double a3, const double *x3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  if (x0) s += a0 * x0[i];
  if (x1) s += a1 * x1[i];
  if (x2) s += a2 * x2[i];
  if (x3) s += a3 * x3[i];
  out[i] = s;
}

}  // namespace

void emd_adj_axpy(double2 *y, const double2 *x, size_t n, cudaStream_t st) {
  emd_note_launches(1);
  k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, x, n);
}

void emd_adj_gv(const OrbLayout &o, const double2 *mu, const double2 *u, double b,
                double *g, cudaStream_t st) {
  emd_note_launches(1);
  const unsigned nb = (unsigned)((o.n3 + 255) / 256);
  switch (o.bo) {
    case 1: k_gv_accum<1><<<nb, 256, 0, st>>>(mu, u, (size_t)o.n3, o.n_blk, b, g); break;
    case 2: k_gv_accum<2><<<nb, 256, 0, st>>>(mu, u, (size_t)o.n3, o.n_blk, b, g); break;
    case 4: k_gv_accum<4><<<nb, 256, 0, st>>>(mu, u, (size_t)o.n3, o.n_blk, b, g); break;
  }
}

void emd_adj_project_grad(const OrbLayout &o, const TableSet &t, int n_atoms,
                          const double2 *x, double h3, double h_kb,
                          double inv_rc2, double2 *c, double2 *hc, double2 *dc,
                          cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  dim3 grid(n_atoms, o.n_blk);
  switch (o.bo) {
    case 1: k_project_grad<1><<<grid, 256, 0, st>>>(x, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, h_kb, inv_rc2, o.n_orb_pad, c, hc, dc); break;
    case 2: k_project_grad<2><<<grid, 256, 0, st>>>(x, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, h_kb, inv_rc2, o.n_orb_pad, c, hc, dc); break;
    case 4: k_project_grad<4><<<grid, 256, 0, st>>>(x, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, h_kb, inv_rc2, o.n_orb_pad, c, hc, dc); break;
  }
}

void emd_adj_proj_sens(const double2 *cm, const double2 *dcm, const double2 *cu,
                       const double2 *dcu, int n_atoms, int n_orb, int n_orb_pad,
                       double coef, double *gR, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  const int m = 3 * n_atoms;
  k_proj_sens<<<(m + 127) / 128, 128, 0, st>>>(cm, dcm, cu, dcu, n_atoms, n_orb,
                                               n_orb_pad, coef, gR);
}

void emd_adj_rho(int n3, const double *rho, const double *lam_v, double *pois,
                 cudaStream_t st) {
  emd_note_launches(1);
  k_rho_adjoint<<<(n3 + 255) / 256, 256, 0, st>>>(n3, rho, lam_v, pois);
}

void emd_adj_scale_add(const OrbLayout &o, double2 *lam, const double2 *psi,
                       const double *w, double scale, cudaStream_t st) {
  emd_note_launches(1);
  const size_t tot = (size_t)o.n_blk * o.n3 * o.bo;
  const unsigned nb = (unsigned)((tot + 255) / 256);
  switch (o.bo) {
    case 1: k_scale_add<1><<<nb, 256, 0, st>>>(lam, psi, w, (size_t)o.n3, o.n_blk, scale); break;
    case 2: k_scale_add<2><<<nb, 256, 0, st>>>(lam, psi, w, (size_t)o.n3, o.n_blk, scale); break;
    case 4: k_scale_add<4><<<nb, 256, 0, st>>>(lam, psi, w, (size_t)o.n3, o.n_blk, scale); break;
  }
}

void emd_adj_lincomb(int n, double *out, double a0, const double *x0, double a1,
                     const double *x1, double a2, const double *x2, double a3,
                     const double *x3, cudaStream_t st) {
  emd_note_launches(1);
  k_lincomb<<<(n + 255) / 256, 256, 0, st>>>(n, out, a0, x0, a1, x1, a2, x2, a3, x3);
}
