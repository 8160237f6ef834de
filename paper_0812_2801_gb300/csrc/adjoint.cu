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

// complex128, bo = 2: the same sums (c, h_kb c and the three moments dc) in
// double-float arithmetic on the FP32 pipes from the pre-split atom records
// (p and p d / r_c^2 as (hi, lo) pairs, as the forward projections and
// moments use), two entries of a thread in flight; widened to FP64 once and
// added by the fixed-tree block sum.
__global__ void __launch_bounds__(256)
k_project_grad_df(const double2 *__restrict__ x, size_t n3, const int *__restrict__ at_cnt,
                  const uint4 *__restrict__ at_rec, const float4 *__restrict__ at_w, int cap,
                  double h3, double h_kb, int n_orb_pad, double2 *c, double2 *hc, double2 *dc) {
  constexpr int BO = 2, EU = 2;
  __shared__ double red[8 * 8 * BO];
  const int J = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[J];
  const double2 *xb = x + (size_t)blk * n3 * BO;
  const uint4 *rec = at_rec + (size_t)J * cap;
  const float4 *wr = at_w + (size_t)J * cap * 2;
  float2 ah[4 * BO], al[4 * BO];     // [orbital][c, dc_x, dc_y, dc_z]
#pragma unroll
  for (int k = 0; k < 4 * BO; ++k) ah[k] = al[k] = make_float2(0.f, 0.f);
  for (int e0 = threadIdx.x; e0 < cnt; e0 += EU * 256) {
    uint4 r[EU];
    float4 w0[EU], w1[EU];
#pragma unroll
    for (int v = 0; v < EU; ++v) {        // past the end: point 0, zero weights
      const int e = e0 + 256 * v;
      const bool ok = e < cnt;
      r[v] = ok ? __ldg(rec + e) : make_uint4(0u, 0u, 0u, 0u);
      w0[v] = ok ? __ldg(wr + 2 * e) : make_float4(0.f, 0.f, 0.f, 0.f);
      w1[v] = ok ? __ldg(wr + 2 * e + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    double2 xv[EU][BO];
#pragma unroll
    for (int v = 0; v < EU; ++v)
#pragma unroll
      for (int j = 0; j < BO; ++j) xv[v][j] = xb[(size_t)r[v].x * BO + j];
#pragma unroll
    for (int v = 0; v < EU; ++v)
#pragma unroll
      for (int j = 0; j < BO; ++j) {
        const float4 xs = df_split2(xv[v][j]);
        dfp_add_prod(ah[4 * j + 0], al[4 * j + 0], __uint_as_float(r[v].y),
                     __uint_as_float(r[v].z), f4hi(xs), f4lo(xs));
        dfp_add_prod(ah[4 * j + 1], al[4 * j + 1], w0[v].x, w0[v].y, f4hi(xs), f4lo(xs));
        dfp_add_prod(ah[4 * j + 2], al[4 * j + 2], w0[v].z, w0[v].w, f4hi(xs), f4lo(xs));
        dfp_add_prod(ah[4 * j + 3], al[4 * j + 3], w1[v].x, w1[v].y, f4hi(xs), f4lo(xs));
      }
  }
  double acc[8 * BO];
#pragma unroll
  for (int k = 0; k < 4 * BO; ++k) {
    acc[2 * k] = __dadd_rn(df_widen(ah[k].x), df_widen(al[k].x));
    acc[2 * k + 1] = __dadd_rn(df_widen(ah[k].y), df_widen(al[k].y));
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
    using namespace pz81;
    const double s = sqrt(rs);
    const double q = 1.0 + b1 * s + b2 * rs;
    const double nn = 1.0 + (7.0 / 6.0) * b1 * s + (4.0 / 3.0) * b2 * rs;
    const double dq = b1 / (2.0 * s) + b2;
    const double dn = (7.0 / 6.0) * b1 / (2.0 * s) + (4.0 / 3.0) * b2;
    dvc = gam * (dn * q - 2.0 * nn * dq) / (q * q * q);
  } else {
    using namespace pz81;
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
    case 2:
      if (t.at_rec)
        k_project_grad_df<<<grid, 256, 0, st>>>(x, (size_t)o.n3, t.at_cnt, t.at_rec, t.at_w,
                                                t.cap, h3, h_kb, o.n_orb_pad, c, hc, dc);
      else
        k_project_grad<2><<<grid, 256, 0, st>>>(x, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, h_kb, inv_rc2, o.n_orb_pad, c, hc, dc);
      break;
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

// ===========================================================================
// Moving ions: reverse of the force F(psi, R, v_es) (eq. new_EoM_b) used by
// velocity Verlet.  With lam_F the adjoint of the forces:
//   splat   w(r)   = h^3 sum_J lam_J . g_J(r) 2 d / a^2      (dL/dv_es)
//   loc HVP dL/dR_J += h^3 sum_r v_es g_J (-2/a^2) [lam_J - 2 d (d.lam_J)/a^2]
//   nl orb  Lam(r) += -2 h_kb f h^3 sum_J [p_J alpha_J + (lam_J . dp_J) c_J]
//           alpha_J = lam_J . dc_J,  dp_J = p_J d / r_c^2
//   nl R    second moments m_b = h^3 sum p [(lam.d) d_b / r_c^4 - lam_b / r_c^2] u
//   sr HVP  dL/dR_m += sum_{K,n} Jac(D_mKn) (lam_m - lam_K)
// ===========================================================================
namespace {

// w(r) for every grid point from the (atom, image) candidates of its tile.
__global__ void __launch_bounds__(512)
k_force_splat(int n, double h, double L, const double *Rw, SpeciesDev sp,
              const int *tile_cnt, const int *tile_ent, const double *lamF,
              double *w) {
  __shared__ int cand[EMD_TILE_CAND_MAX];
  const int nt = (n + EMD_TILE - 1) / EMD_TILE;
  const int t = blockIdx.x;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  const int nc = tile_cnt[t];
  for (int i = threadIdx.x; i < nc; i += blockDim.x)
    cand[i] = tile_ent[t * EMD_TILE_CAND_MAX + i];
  __syncthreads();
  const int x = tx * EMD_TILE + (threadIdx.x & 7);
  const int y = ty * EMD_TILE + ((threadIdx.x >> 3) & 7);
  const int z = tz * EMD_TILE + (threadIdx.x >> 6);
  if (x >= n || y >= n || z >= n) return;
  const double rl2 = __dmul_rn(sp.r_loc, sp.r_loc);
  const double h3 = h * h * h;
  double acc = 0.0;
  for (int e = 0; e < nc; ++e) {
    const int J = cand[e] / 27, img = cand[e] % 27;
    const double dx = emd_disp(x, h, Rw[3 * J + 0], img % 3 - 1, L);
    const double dy = emd_disp(y, h, Rw[3 * J + 1], (img / 3) % 3 - 1, L);
    const double dz = emd_disp(z, h, Rw[3 * J + 2], img / 9 - 1, L);
    const double d2 = emd_norm2(dx, dy, dz);
    if (d2 < rl2) {
      const double g = sp.c_g * exp(-d2 * sp.inv_a2) * (2.0 * sp.inv_a2);
      acc += g * (lamF[3 * J] * dx + lamF[3 * J + 1] * dy + lamF[3 * J + 2] * dz);
    }
  }
  w[((size_t)z * n + y) * n + x] = h3 * acc;
}

// Orbital term of the nonlocal-force adjoint, added to lam (orbital layout).
// coef = -2 h_kb f h^3; cc[J][A] = c_JA, dc[J][A][b] = dc_JA,b, and
// alpha_JA = lam_J . dc_JA is formed on the fly.
template <int BO>
__global__ void __launch_bounds__(512)
k_nl_force_adj_orb(int n, double h, double L, const double *Rw, SpeciesDev sp,
                   const int *tile_cnt, const int *tile_ent, const double *lamF,
                   const double2 *dc, const double2 *cc, int n_orb_pad,
                   double coef, double2 *lam) {
  __shared__ int cand[EMD_TILE_CAND_MAX];
  const int nt = (n + EMD_TILE - 1) / EMD_TILE;
  const int t = blockIdx.x, blk = blockIdx.y;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  const int nc = tile_cnt[t];
  for (int i = threadIdx.x; i < nc; i += blockDim.x)
    cand[i] = tile_ent[t * EMD_TILE_CAND_MAX + i];
  __syncthreads();
  const int x = tx * EMD_TILE + (threadIdx.x & 7);
  const int y = ty * EMD_TILE + ((threadIdx.x >> 3) & 7);
  const int z = tz * EMD_TILE + (threadIdx.x >> 6);
  if (x >= n || y >= n || z >= n) return;
  const double rp2 = __dmul_rn(sp.r_proj, sp.r_proj);
  double2 acc[BO];
#pragma unroll
  for (int j = 0; j < BO; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int e = 0; e < nc; ++e) {
    const int J = cand[e] / 27, img = cand[e] % 27;
    const double dx = emd_disp(x, h, Rw[3 * J + 0], img % 3 - 1, L);
    const double dy = emd_disp(y, h, Rw[3 * J + 1], (img / 3) % 3 - 1, L);
    const double dz = emd_disp(z, h, Rw[3 * J + 2], img / 9 - 1, L);
    const double d2 = emd_norm2(dx, dy, dz);
    if (d2 < rp2) {
      const double p = sp.c_p * exp(-d2 * sp.inv_2rc2);
      const double ld = p * sp.inv_rc2 *
                        (lamF[3 * J] * dx + lamF[3 * J + 1] * dy + lamF[3 * J + 2] * dz);
#pragma unroll
      for (int j = 0; j < BO; ++j) {
        const size_t o = (size_t)J * n_orb_pad + (size_t)blk * BO + j;
        const double2 d0 = dc[3 * o], d1 = dc[3 * o + 1], d2v = dc[3 * o + 2];
        const double2 a = make_double2(
            lamF[3 * J] * d0.x + lamF[3 * J + 1] * d1.x + lamF[3 * J + 2] * d2v.x,
            lamF[3 * J] * d0.y + lamF[3 * J + 1] * d1.y + lamF[3 * J + 2] * d2v.y);
        const double2 c = cc[o];
        acc[j].x += p * a.x + ld * c.x;
        acc[j].y += p * a.y + ld * c.y;
      }
    }
  }
  const size_t n3 = (size_t)n * n * n;
  const size_t pidx = ((size_t)z * n + y) * n + x;
  double2 *lb = lam + ((size_t)blk * n3 + pidx) * BO;
#pragma unroll
  for (int j = 0; j < BO; ++j) {
    lb[j].x += coef * acc[j].x;
    lb[j].y += coef * acc[j].y;
  }
}

// m[J][A][b] = h^3 sum_e p_e [(lam_J . d) d_b / r_c^4 - lam_J,b / r_c^2] u_A
template <int BO>
__global__ void __launch_bounds__(256)
k_nl_second_moment(const double2 *__restrict__ u, size_t n3, const int *at_cnt,
                   const int *at_pt, const double *at_p, const double *at_d,
                   int cap, double h3, double inv_rc2, const double *lamF,
                   int n_orb_pad, double2 *m) {
  __shared__ double red[8 * 6 * BO];
  const int J = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[J];
  const double2 *ub = u + (size_t)blk * n3 * BO;
  const double l0 = lamF[3 * J], l1 = lamF[3 * J + 1], l2 = lamF[3 * J + 2];
  double acc[6 * BO];
#pragma unroll
  for (int k = 0; k < 6 * BO; ++k) acc[k] = 0.0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const size_t idx = (size_t)J * cap + e;
    const int pt = at_pt[idx];
    const double pv = at_p[idx];
    const double d0 = at_d[3 * idx], d1 = at_d[3 * idx + 1], d2 = at_d[3 * idx + 2];
    const double ld = (l0 * d0 + l1 * d1 + l2 * d2) * inv_rc2 * inv_rc2;
    const double w0 = pv * (ld * d0 - l0 * inv_rc2);
    const double w1 = pv * (ld * d1 - l1 * inv_rc2);
    const double w2 = pv * (ld * d2 - l2 * inv_rc2);
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const double2 v = ub[(size_t)pt * BO + j];
      acc[6 * j + 0] += w0 * v.x;
      acc[6 * j + 1] += w0 * v.y;
      acc[6 * j + 2] += w1 * v.x;
      acc[6 * j + 3] += w1 * v.y;
      acc[6 * j + 4] += w2 * v.x;
      acc[6 * j + 5] += w2 * v.y;
    }
  }
  emd_block_sum<6 * BO>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const size_t o = (size_t)J * n_orb_pad + (size_t)blk * BO + j;
      for (int b = 0; b < 3; ++b)
        m[3 * o + b] = make_double2(h3 * acc[6 * j + 2 * b], h3 * acc[6 * j + 2 * b + 1]);
    }
  }
}

// Position term of the nonlocal-force adjoint:
// out[J][b] = coef Re sum_A [conj(dc_JA,b) alpha_JA + conj(c_JA) m_JA,b],
// coef = -2 h_kb f, alpha_JA = lam_J . dc_JA.  One thread per (J, b), the
// orbital sum in fixed order.
__global__ void k_nl_force_adj_r(const double2 *cc, const double2 *dc,
                                 const double2 *m, const double *lamF,
                                 int n_atoms, int n_orb, int n_orb_pad,
                                 double coef, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n_atoms) return;
  const int J = i / 3, b = i % 3;
  const double l0 = lamF[3 * J], l1 = lamF[3 * J + 1], l2 = lamF[3 * J + 2];
  double s = 0.0;
  for (int A = 0; A < n_orb; ++A) {
    const size_t o = (size_t)J * n_orb_pad + A;
    const double2 d0 = dc[3 * o], d1 = dc[3 * o + 1], d2 = dc[3 * o + 2];
    const double ax = l0 * d0.x + l1 * d1.x + l2 * d2.x;
    const double ay = l0 * d0.y + l1 * d1.y + l2 * d2.y;
    const double2 db = dc[3 * o + b], c = cc[o], mb = m[3 * o + b];
    s += (db.x * ax + db.y * ay) + (c.x * mb.x + c.y * mb.y);
  }
  out[i] = coef * s;
}

// sum_{K,n} Jac(D)(lam_m - lam_K), Jac = Z^2 [psi(d) I + psi'(d) D D^T / d],
// psi = phi / d, phi(d) = erfc(d/s)/d^2 + 2/(s sqrt(pi)) exp(-d^2/s^2)/d.
__global__ void __launch_bounds__(256)
k_sr_hvp(SpeciesDev sp, int n_atoms, const double *Rw, double L, int nmax,
         const double *lamF, double *out) {
  __shared__ double red[8 * 3];
  const int m = blockIdx.x;
  const double s = sqrt(2.0) * sp.a_loc;
  const double zz = sp.z * sp.z;
  const double k2 = 2.0 / (s * sqrt(M_PI));
  const int side = 2 * nmax + 1, nimg = side * side * side;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < n_atoms * nimg; q += blockDim.x) {
    const int K = q / nimg, im = q % nimg;
    const int nx = im % side - nmax, ny = (im / side) % side - nmax,
              nz = im / (side * side) - nmax;
    if (K == m && nx == 0 && ny == 0 && nz == 0) continue;
    const double D0 = Rw[3 * m] - Rw[3 * K] - nx * L;
    const double D1 = Rw[3 * m + 1] - Rw[3 * K + 1] - ny * L;
    const double D2 = Rw[3 * m + 2] - Rw[3 * K + 2] - nz * L;
    const double d2 = D0 * D0 + D1 * D1 + D2 * D2;
    if (d2 >= 144.0 || d2 <= 0.0) continue;
    const double d = sqrt(d2);
    const double ex = exp(-d2 / (s * s));
    const double ef = erfc(d / s);
    const double phi = ef / d2 + k2 * ex / d;
    const double dphi = -k2 * ex / d2 - 2.0 * ef / (d2 * d) + k2 * ex * (-2.0 / (s * s) - 1.0 / d2);
    const double psi = phi / d;
    const double dpsi = (dphi * d - phi) / d2;
    const double l0 = lamF[3 * m] - lamF[3 * K], l1 = lamF[3 * m + 1] - lamF[3 * K + 1],
                 l2 = lamF[3 * m + 2] - lamF[3 * K + 2];
    const double Dl = (D0 * l0 + D1 * l1 + D2 * l2) * dpsi / d;
    acc[0] += zz * (psi * l0 + Dl * D0);
    acc[1] += zz * (psi * l1 + Dl * D1);
    acc[2] += zz * (psi * l2 + Dl * D2);
  }
  emd_block_sum<3>(acc, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) out[3 * m + a] = acc[a];
}

}  // namespace

void emd_adj_force_splat(const GridInfo &g, const SpeciesDev &sp, const TableSet &t,
                         const double *lamF, double *w, cudaStream_t st) {
  const int nt = (g.n + EMD_TILE - 1) / EMD_TILE;
  emd_note_launches(1);
  k_force_splat<<<nt * nt * nt, 512, 0, st>>>(g.n, g.h, g.L, t.Rw, sp, t.tile_cnt,
                                              t.tile_ent, lamF, w);
}

void emd_adj_nl_force_orb(const OrbLayout &o, const GridInfo &g, const SpeciesDev &sp,
                          const TableSet &t, const double *lamF, const double2 *dc,
                          const double2 *cc, double coef, double2 *lam,
                          cudaStream_t st) {
  const int nt = (g.n + EMD_TILE - 1) / EMD_TILE;
  dim3 grid(nt * nt * nt, o.n_blk);
  emd_note_launches(1);
  switch (o.bo) {
    case 1: k_nl_force_adj_orb<1><<<grid, 512, 0, st>>>(g.n, g.h, g.L, t.Rw, sp, t.tile_cnt, t.tile_ent, lamF, dc, cc, o.n_orb_pad, coef, lam); break;
    case 2: k_nl_force_adj_orb<2><<<grid, 512, 0, st>>>(g.n, g.h, g.L, t.Rw, sp, t.tile_cnt, t.tile_ent, lamF, dc, cc, o.n_orb_pad, coef, lam); break;
    case 4: k_nl_force_adj_orb<4><<<grid, 512, 0, st>>>(g.n, g.h, g.L, t.Rw, sp, t.tile_cnt, t.tile_ent, lamF, dc, cc, o.n_orb_pad, coef, lam); break;
  }
}

void emd_adj_nl_second_moment(const OrbLayout &o, const TableSet &t, int n_atoms,
                              const double2 *u, double h3, double inv_rc2,
                              const double *lamF, double2 *m, cudaStream_t st) {
  if (n_atoms <= 0) return;
  dim3 grid(n_atoms, o.n_blk);
  emd_note_launches(1);
  switch (o.bo) {
    case 1: k_nl_second_moment<1><<<grid, 256, 0, st>>>(u, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, inv_rc2, lamF, o.n_orb_pad, m); break;
    case 2: k_nl_second_moment<2><<<grid, 256, 0, st>>>(u, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, inv_rc2, lamF, o.n_orb_pad, m); break;
    case 4: k_nl_second_moment<4><<<grid, 256, 0, st>>>(u, (size_t)o.n3, t.at_cnt, t.at_pt, t.at_p, t.at_d, t.cap, h3, inv_rc2, lamF, o.n_orb_pad, m); break;
  }
}

void emd_adj_sr_hvp(const SpeciesDev &sp, int n_atoms, const double *Rw, double L,
                    const double *lamF, double *out, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  const int nmax = (int)ceil(12.0 / L) + 1;
  k_sr_hvp<<<n_atoms, 256, 0, st>>>(sp, n_atoms, Rw, L, nmax, lamF, out);
}

void emd_adj_nl_force_r(const double2 *cc, const double2 *dc, const double2 *m,
                        const double *lamF, int n_atoms, int n_orb, int n_orb_pad,
                        double coef, double *out, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  const int k = 3 * n_atoms;
  k_nl_force_adj_r<<<(k + 127) / 128, 128, 0, st>>>(cc, dc, m, lamF, n_atoms, n_orb,
                                                     n_orb_pad, coef, out);
}
