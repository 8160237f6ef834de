// Atom-dependent grid data for one set of ion positions: folded positions,
// per-tile atom candidates, the point-major projector table with the Gaussian
// ion charge, the atom-major projector table, and the ionic force terms.
//
// Paper: ionic potential as a sum of per-atom terms (Sec. 5.2,
// eq. ionicpotential); Hellmann-Feynman forces (eq. new_EoM_b) whose local
// part (eq. ionicforces) is taken here as the exact derivative of the
// discrete electrostatic energy with respect to R_J (the gradient acts on the
// analytic Gaussian charge, not on the grid density); velocity Verlet for the
// ions (Sec. 5.1).
#include "emd_internal.cuh"

#include <cmath>

// Bound on |d^2_FP32 - d^2| for a point of the image boxes of a sphere of
// radius r in a box of side L: each coordinate difference (i h - (R + n L),
// all terms below 2L + r in size) is off by at most ~4 FP32 roundings of
// 2L + r, and d^2 near r^2 amplifies that by 2 sqrt(3) r, plus the roundings
// of the squares and sums; a factor 8 on top.
float emd_fp32_d2_margin(double L, double r) {
  const double ex = 4.0 * 5.97e-8 * (2.0 * L + r + 1.0);
  return (float)(8.0 * (2.0 * std::sqrt(3.0) * r * ex + ex * ex + 4.0 * 5.97e-8 * r * r));
}

namespace {

__global__ void k_wrap(const double *R, double *Rw, int n, double L) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Rw[i] = emd_wrap_pos(R[i], L);
}

// Conservative (atom, image) candidates per tile of EMD_TILE^3 points: every
// pair whose support sphere can reach a point of the tile.  The exact
// per-point decision is taken later in FP64.  One block per tile; pairs are
// scanned in (J, image) order and compacted in that order.
__global__ void __launch_bounds__(256)
k_tile_candidates(int n, double h, double L, const double *Rw, int n_atoms,
                  float r_max, int *tile_cnt, int *tile_ent, int *err) {
  __shared__ int warp_tot[8];
  __shared__ int s_base;
  const int nt = (n + EMD_TILE - 1) / EMD_TILE;
  const int t = blockIdx.x;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  const float lo[3] = {(float)(tx * EMD_TILE * h), (float)(ty * EMD_TILE * h),
                       (float)(tz * EMD_TILE * h)};
  const float hi[3] = {(float)(min(tx * EMD_TILE + EMD_TILE - 1, n - 1) * h),
                       (float)(min(ty * EMD_TILE + EMD_TILE - 1, n - 1) * h),
                       (float)(min(tz * EMD_TILE + EMD_TILE - 1, n - 1) * h)};
  const float rr = (r_max + 0.05f) * (r_max + 0.05f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const int total = n_atoms * 27;
  for (int b0 = 0; b0 < total; b0 += blockDim.x) {
    const int q = b0 + threadIdx.x;
    bool hit = false;
    if (q < total) {
      const int J = q / 27, img = q % 27;
      const int ni[3] = {img % 3 - 1, (img / 3) % 3 - 1, img / 9 - 1};
      float d2 = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float c = (float)Rw[3 * J + a] + (float)(ni[a] * L);
        const float d = fmaxf(fmaxf(lo[a] - c, c - hi[a]), 0.f);
        d2 += d * d;
      }
      hit = d2 < rr;
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int off = s_base, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) off += warp_tot[w];
      tot += warp_tot[w];
    }
    if (hit) {
      const int e = off + __popc(m & ((1u << lane) - 1u));
      if (e < EMD_TILE_CAND_MAX)
        tile_ent[t * EMD_TILE_CAND_MAX + e] = q;   // q = J * 27 + image
      else
        atomicOr(err, EMD_ERRBIT_TILE);
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_cnt[t] = min(s_base, EMD_TILE_CAND_MAX);
}

// Point-major table: for each grid point the atoms whose projector reaches it
// (p summed over that atom's images), in increasing atom order; and the total
// Gaussian ion charge at the point.  One block = one tile, one thread = one
// point.  FP32 distances settle the support decisions away from a thin shell
// around each radius; FP64 computes the decisions inside it and every stored
// FP64 value (the ion charge always, p when F32 = false).  With F32 = true
// (complex64 path) p is evaluated in FP32, the precision its readers use,
// and the block also writes the tile's entries grouped by atom (te_*): the
// tile's distinct atoms (slots) are the runs of equal J in its candidate
// list, and the points of each slot are compacted in point order.
template <bool F32>
__global__ void __launch_bounds__(512)
k_point_table(int n, int n3, double h, double L, const double *Rw,
              SpeciesDev sp, float margin, const int *tile_cnt, const int *tile_ent,
              const double *gtab, const int *glo,
              int *pt_cnt, int *pt_J, double *pt_p, float *pt_pf, int2 *pt4, int4 *pt4d,
              double *g_ion, int *te_off, uint2 *te_pp, float4 *te_q, int kmax, int4 *pt_rec,
              int *err) {
  __shared__ int cand[EMD_TILE_CAND_MAX];
  __shared__ float cfs[EMD_TILE_CAND_MAX][3];
  __shared__ float cfl[F32 ? EMD_TILE_CAND_MAX : 1][3];   // low parts of the centres
  __shared__ int run_start[EMD_TILE_ATOM_MAX + 1];
  __shared__ int s_nrun;
  __shared__ int warp_tot[16];
  const int nt = (n + EMD_TILE - 1) / EMD_TILE;
  const int t = blockIdx.x;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  const int nc = tile_cnt[t];
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int code = tile_ent[t * EMD_TILE_CAND_MAX + i];
    const int J = code / 27, img = code % 27;
    cand[i] = code;
    const double c[3] = {Rw[3 * J + 0] + (img % 3 - 1) * L,
                         Rw[3 * J + 1] + ((img / 3) % 3 - 1) * L,
                         Rw[3 * J + 2] + (img / 9 - 1) * L};
    for (int a = 0; a < 3; ++a) {
      cfs[i][a] = (float)c[a];
      if (F32) cfl[i][a] = (float)(c[a] - (double)cfs[i][a]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // runs of equal atom in the (atom, image)-ordered candidate list
    int r = 0, last = -1;
    for (int i = 0; i < nc; ++i) {
      const int J = cand[i] / 27;
      if (J != last) {
        if (r < EMD_TILE_ATOM_MAX) run_start[r] = i;
        ++r;
        last = J;
      }
    }
    if (r > EMD_TILE_ATOM_MAX) {
      if (F32) atomicOr(err, EMD_ERRBIT_TILE);
      r = EMD_TILE_ATOM_MAX;   // (F32 = false: the runs are only a loop structure)
    }
    // with F32 = false every candidate must still be visited: one run per
    // slot is kept and the last run extends to the end of the list
    run_start[r] = nc;
    s_nrun = r;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = tx * EMD_TILE + (threadIdx.x & 7);
  const int y = ty * EMD_TILE + ((threadIdx.x >> 3) & 7);
  const int z = tz * EMD_TILE + (threadIdx.x >> 6);
  const bool in = x < n && y < n && z < n;
  const int p = in ? (z * n + y) * n + x : 0;
  const double rp2 = __dmul_rn(sp.r_proj, sp.r_proj);
  const double rl2 = __dmul_rn(sp.r_loc, sp.r_loc);
  const float rp2f = (float)rp2, rl2f = (float)rl2, hf = (float)h;
  const float rmax2f = fmaxf(rp2f, rl2f) + margin;
  const float xf = (float)x * hf, yf = (float)y * hf, zf = (float)z * hf;
  // the grid coordinate as float hi + lo (complex64 projector values)
  const double gx = (double)x * h, gy = (double)y * h, gz = (double)z * h;
  const float gxh = (float)gx, gyh = (float)gy, gzh = (float)gz;
  const float gxl = (float)(gx - (double)gxh), gyl = (float)(gy - (double)gyh),
              gzl = (float)(gz - (double)gzh);
  const int nrun = s_nrun;
  int cnt = 0;
  double gsum = 0.0;
  int te_base = 0;
  // complex128 with several projectors per atom: channel k >= 1 sums
  double pch[9];
  // the entries of atom J at this point: one per projector (channel)
  auto close_atom = [&](int J, double psum) {
    for (int k = 0; k < sp.nch; ++k) {
      if (cnt < kmax) {
        const double v = k == 0 ? psum : pch[k];
        pt_J[cnt * n3 + p] = J * sp.nch + k;
        pt_p[cnt * n3 + p] = v;
        pt_pf[cnt * n3 + p] = (float)v;
        if (pt_rec) {
          const float2 vs = emd_df_split(v);
          pt_rec[(size_t)cnt * n3 + p] =
              make_int4(J * sp.nch + k, __float_as_int(vs.x), __float_as_int(vs.y), 0);
        }
        ++cnt;
      } else {
        atomicOr(err, EMD_ERRBIT_PT);
      }
    }
  };
  for (int r = 0; r < nrun; ++r) {
    double psum = 0.0;
    float psumf = 0.f, pdx = 0.f, pdy = 0.f, pdz = 0.f;
    bool hit = false;
    int J = -1;
    if (!F32)
      for (int k = 1; k < sp.nch; ++k) pch[k] = 0.0;
    for (int e = run_start[r]; e < run_start[r + 1]; ++e) {
      const int code = cand[e];
      const int Je = code / 27, img = code % 27;
      if (!F32 && Je != J && hit) {
        // F32 = false with more than EMD_TILE_ATOM_MAX atoms: the last run
        // holds several atoms; close the previous one
        close_atom(J, psum);
        psum = 0.0;
        for (int k = 1; k < sp.nch; ++k) pch[k] = 0.0;
        hit = false;
      }
      J = Je;
      if (!in) continue;
      const float dxf = xf - cfs[e][0], dyf = yf - cfs[e][1], dzf = zf - cfs[e][2];
      const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
      if (d2f > rmax2f) continue;
      // decisions: FP32 where it is certain, FP64 in the shells
      bool in_p, in_l;
      double d2 = 0.0, dx = 0.0, dy = 0.0, dz = 0.0;
      bool have64 = false;
      if (d2f < rp2f - margin) {
        in_p = true;
      } else if (d2f > rp2f + margin) {
        in_p = false;
      } else {
        dx = emd_disp(x, h, Rw[3 * J + 0], img % 3 - 1, L);
        dy = emd_disp(y, h, Rw[3 * J + 1], (img / 3) % 3 - 1, L);
        dz = emd_disp(z, h, Rw[3 * J + 2], img / 9 - 1, L);
        d2 = emd_norm2(dx, dy, dz);
        have64 = true;
        in_p = d2 < rp2;
      }
      if (d2f < rl2f - margin) {
        in_l = true;
      } else if (d2f > rl2f + margin) {
        in_l = false;
      } else {
        if (!have64) {
          dx = emd_disp(x, h, Rw[3 * J + 0], img % 3 - 1, L);
          dy = emd_disp(y, h, Rw[3 * J + 1], (img / 3) % 3 - 1, L);
          dz = emd_disp(z, h, Rw[3 * J + 2], img / 9 - 1, L);
          d2 = emd_norm2(dx, dy, dz);
          have64 = true;
        }
        in_l = d2 < rl2;
      }
      // the ion charge from the separable tables (g = c_g T_x T_y T_z)
      bool g_tab = false;
      double g_val = 0.0;
      if (in_l && gtab) {
        const int *lo = glo + ((size_t)J * 27 + img) * 3;
        const int kx = x - lo[0], ky = y - lo[1], kz = z - lo[2];
        if (kx >= 0 && ky >= 0 && kz >= 0 && kx < EMD_GT_EXT && ky < EMD_GT_EXT &&
            kz < EMD_GT_EXT) {
          const double *T = gtab + ((size_t)J * 27 + img) * 3 * EMD_GT_EXT;
          g_val = sp.c_g * (T[kx] * (T[EMD_GT_EXT + ky] * T[2 * EMD_GT_EXT + kz]));
          g_tab = true;
        }
      }
      if (!have64 && ((in_l && !g_tab) || (in_p && !F32))) {
        dx = emd_disp(x, h, Rw[3 * J + 0], img % 3 - 1, L);
        dy = emd_disp(y, h, Rw[3 * J + 1], (img / 3) % 3 - 1, L);
        dz = emd_disp(z, h, Rw[3 * J + 2], img / 9 - 1, L);
        d2 = emd_norm2(dx, dy, dz);
      }
      if (in_p) {
        if (F32) {
          // displacement from hi + lo parts of both coordinates: the hi
          // difference is rounded once from the exact one, so the result is
          // the displacement to an ulp or two.  A plain float atom coordinate
          // (float)(R + image L) is off by up to half an ulp of L, the same
          // shift for every point of the sphere, and the projector force
          // sum_r p d psi cancels strongly: that shift showed up at ~1e-4 of
          // the forces.
          const float ex = (gxh - cfs[e][0]) + (gxl - cfl[e][0]);
          const float ey = (gyh - cfs[e][1]) + (gyl - cfl[e][1]);
          const float ez = (gzh - cfs[e][2]) + (gzl - cfl[e][2]);
          const float pv = (float)sp.c_p *
                           expf(-(ex * ex + ey * ey + ez * ez) * (float)sp.inv_2rc2);
          const float w = pv * (float)sp.inv_rc2;
          psumf += pv;
          pdx += w * ex;
          pdy += w * ey;
          pdz += w * ez;
        } else {
          const double ex = exp(-d2 * sp.inv_2rc2);
          psum += sp.c_p * ex;
          if (sp.nch > 1) {
            double pk[9];
            emd_channel_values(sp, dx, dy, dz, ex, pk, nullptr);
            for (int k = 1; k < sp.nch; ++k) pch[k] += pk[k];
          }
        }
        hit = true;
      }
      if (in_l) gsum += g_tab ? g_val : sp.c_g * exp(-d2 * sp.inv_a2);
    }
    if (hit) {
      if (!F32) {
        close_atom(J, psum);
      } else if (cnt < kmax) {
        pt_J[cnt * n3 + p] = J;
        pt_p[cnt * n3 + p] = (double)psumf;
        pt_pf[cnt * n3 + p] = psumf;
        ++cnt;
      } else {
        atomicOr(err, EMD_ERRBIT_PT);
      }
    }
    if (F32) {
      // compaction of this slot's points, in point order
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) warp_tot[warp] = __popc(m);
      __syncthreads();
      int off = te_base, tot = 0;
      for (int w = 0; w < 16; ++w) {
        if (w < warp) off += warp_tot[w];
        tot += warp_tot[w];
      }
      if (hit) {
        const int e = off + __popc(m & ((1u << lane) - 1u));
        if (e < EMD_TE_CAP) {
          const size_t q = (size_t)t * EMD_TE_CAP + e;
          te_pp[q] = make_uint2(threadIdx.x, __float_as_uint(psumf));
          te_q[q] = make_float4(pdx, pdy, pdz, __int_as_float((int)threadIdx.x));
        } else {
          atomicOr(err, EMD_ERRBIT_TILE);
        }
      }
      if (threadIdx.x == 0) te_off[t * (EMD_TILE_ATOM_MAX + 1) + r] = min(te_base, EMD_TE_CAP);
      te_base += tot;
      __syncthreads();
    }
  }
  if (F32 && threadIdx.x == 0) {
    for (int r = nrun; r <= EMD_TILE_ATOM_MAX; ++r)
      te_off[t * (EMD_TILE_ATOM_MAX + 1) + r] = min(te_base, EMD_TE_CAP);
  }
  if (!in) return;
  pt_cnt[p] = cnt;
  g_ion[p] = gsum;
  for (int e = 0; e < 4; ++e) {
    int2 q = make_int2(0, 0);
    if (e < cnt) q = make_int2(pt_J[e * n3 + p], __float_as_int(pt_pf[e * n3 + p]));
    if (e == 0) q.x |= cnt << 16;
    pt4[(size_t)p * 4 + e] = q;
  }
  if (pt4d) {
    int J[4];
    float2 pv[4];
    for (int e = 0; e < 4; ++e) {
      J[e] = e < cnt ? pt_J[e * n3 + p] : 0;
      pv[e] = e < cnt ? emd_df_split(pt_p[e * n3 + p]) : make_float2(0.f, 0.f);
    }
    int4 *r = pt4d + (size_t)p * 3;
    r[0] = make_int4(J[0] | (cnt << 16), J[1], J[2], J[3]);
    r[1] = make_int4(__float_as_int(pv[0].x), __float_as_int(pv[0].y), __float_as_int(pv[1].x),
                     __float_as_int(pv[1].y));
    r[2] = make_int4(__float_as_int(pv[2].x), __float_as_int(pv[2].y), __float_as_int(pv[3].x),
                     __float_as_int(pv[3].y));
  }
}

// Index box of the grid points an image sphere can reach along one axis.
__device__ __forceinline__ void axis_range(double c, int nimg, double L,
                                           double h, double r, int n, int &lo,
                                           int &hi) {
  const double cc = c + nimg * L;
  lo = max(0, (int)floor((cc - r) / h) - 1);
  hi = min(n - 1, (int)ceil((cc + r) / h) + 1);
}

// Boxes of the 27 images of atom J's support sphere, flattened in image
// order then box order (x fastest): the enumeration order of the atom table.
struct ImageBoxes {
  int lo[27][3], ext[27][3], start[28];
};
// Called by every thread of the block (contains barriers): threads 0..80
// compute one (image, axis) range each, thread 0 then the flattened starts.
__device__ void image_boxes(const double *c, double L, double h, double r,
                            int n, ImageBoxes &B) {
  if (threadIdx.x < 81) {
    const int img = threadIdx.x / 3, a = threadIdx.x % 3;
    const int ni = a == 0 ? img % 3 - 1 : a == 1 ? (img / 3) % 3 - 1 : img / 9 - 1;
    int lo, hi;
    axis_range(c[a], ni, L, h, r, n, lo, hi);
    B.lo[img][a] = lo;
    B.ext[img][a] = hi >= lo ? hi - lo + 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int img = 0; img < 27; ++img) {
      B.start[img] = acc;
      acc += B.ext[img][0] * B.ext[img][1] * B.ext[img][2];
    }
    B.start[27] = acc;
  }
  __syncthreads();
}

// Atom-major projector table: every (point, image) pair within r_proj of atom
// J, in image order then box order (deterministic), with p and d = r - R_img.
// Grid (atom, split): the flattened box space of the atom is cut into
// `nsplit` contiguous ranges.  Pass 0 counts the hits of each range; pass 1
// writes them at the offset given by the counts of the earlier ranges.
// The decision d^2 < r^2 is the FP64 one; FP32 settles it wherever the FP32
// d^2 is farther than `margin` (a bound on its error, set by the host) from
// r^2, so FP64 arithmetic runs only in a thin shell (and for the stored
// FP64 values of the hits).  Built for the complex128 path
// only (the complex64 kernels read the per-tile entries of the point table).
__global__ void __launch_bounds__(256)
k_atom_table(int pass, int n, double h, double L, const double *Rw,
             SpeciesDev sp, int cap, float margin, int *split_cnt, int *at_cnt,
             int *at_pt, double *at_p, double *at_d, uint4 *at_rec, float4 *at_w,
             int *err) {
  __shared__ ImageBoxes B;
  __shared__ float cf[27][3];
  __shared__ int warp_tot[8];
  __shared__ int s_base;
  const int J = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double c[3] = {Rw[3 * J], Rw[3 * J + 1], Rw[3 * J + 2]};
  const double rp2 = __dmul_rn(sp.r_proj, sp.r_proj);
  const float rp2f = (float)rp2, hf = (float)h;
  image_boxes(c, L, h, sp.r_proj, n, B);
  if (threadIdx.x == 0) {
    int base = 0;
    if (pass == 1)
      for (int s2 = 0; s2 < split; ++s2) base += split_cnt[J * nsplit + s2];
    s_base = base;
  }
  if (threadIdx.x < 81) {
    const int img = threadIdx.x / 3, a = threadIdx.x % 3;
    const int ni = a == 0 ? img % 3 - 1 : a == 1 ? (img / 3) % 3 - 1 : img / 9 - 1;
    cf[img][a] = (float)(c[a] + ni * L);
  }
  __syncthreads();
  const int total = B.start[27];
  const int per = (total + nsplit - 1) / nsplit;
  const int f0 = split * per, f1 = min(total, f0 + per);
  int img = 0;
  for (int b0 = f0; b0 < f1; b0 += blockDim.x) {
    const int f = b0 + threadIdx.x;
    bool flag = false;
    int ix = 0, iy = 0, iz = 0;
    float dxf = 0.f, dyf = 0.f, dzf = 0.f, d2f = 0.f;
    if (f < f1) {
      while (img < 26 && f >= B.start[img + 1]) ++img;
      const int k = f - B.start[img];
      const int ex = B.ext[img][0], ey = B.ext[img][1];
      ix = B.lo[img][0] + k % ex;
      iy = B.lo[img][1] + (k / ex) % ey;
      iz = B.lo[img][2] + k / (ex * ey);
      dxf = (float)ix * hf - cf[img][0];
      dyf = (float)iy * hf - cf[img][1];
      dzf = (float)iz * hf - cf[img][2];
      d2f = dxf * dxf + dyf * dyf + dzf * dzf;
      if (d2f < rp2f - margin) {
        flag = true;
      } else if (d2f <= rp2f + margin) {
        const int ni[3] = {img % 3 - 1, (img / 3) % 3 - 1, img / 9 - 1};
        const double dx = emd_disp(ix, h, c[0], ni[0], L);
        const double dy = emd_disp(iy, h, c[1], ni[1], L);
        const double dz = emd_disp(iz, h, c[2], ni[2], L);
        flag = emd_norm2(dx, dy, dz) < rp2;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int off = s_base, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) off += warp_tot[w];
      tot += warp_tot[w];
    }
    if (pass == 1 && flag) {
      const int e = off + __popc(m & ((1u << lane) - 1u));
      if (e < cap) {
        const size_t q = (size_t)J * cap + e;
        const int pidx = (iz * n + iy) * n + ix;
        at_pt[q] = pidx;
        const int ni[3] = {img % 3 - 1, (img / 3) % 3 - 1, img / 9 - 1};
        const double dx = emd_disp(ix, h, c[0], ni[0], L);
        const double dy = emd_disp(iy, h, c[1], ni[1], L);
        const double dz = emd_disp(iz, h, c[2], ni[2], L);
        const double ex = exp(-emd_norm2(dx, dy, dz) * sp.inv_2rc2);
        const double pv = sp.c_p * ex;
        at_p[q] = pv;
        double *dd = at_d + 3 * q;
        dd[0] = dx;
        dd[1] = dy;
        dd[2] = dz;
        if (at_rec) {
          // channel 0 (s): p and dp/dR = p d / r_c^2; channels k >= 1 from
          // the solid harmonics, in list J nch + k at the same position
          double pk[9], gk[9][3];
          pk[0] = pv;
          const double pw = pv * sp.inv_rc2;
          gk[0][0] = pw * dx;
          gk[0][1] = pw * dy;
          gk[0][2] = pw * dz;
          if (sp.nch > 1) emd_channel_values(sp, dx, dy, dz, ex, pk, gk);
          for (int k = 0; k < sp.nch; ++k) {
            const size_t qk = ((size_t)J * sp.nch + k) * cap + e;
            const float2 ps = emd_df_split(pk[k]);
            const float2 wx = emd_df_split(gk[k][0]), wy = emd_df_split(gk[k][1]),
                         wz = emd_df_split(gk[k][2]);
            at_rec[qk] = make_uint4((unsigned)pidx, __float_as_uint(ps.x), __float_as_uint(ps.y), 0u);
            at_w[2 * qk] = make_float4(wx.x, wx.y, wy.x, wy.y);
            at_w[2 * qk + 1] = make_float4(wz.x, wz.y, 0.f, 0.f);
          }
        }
      } else {
        atomicOr(err, EMD_ERRBIT_AT);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (pass == 0) split_cnt[J * nsplit + split] = s_base;
    else if (split == nsplit - 1) at_cnt[J] = min(s_base, cap);
  }
}

// 1-D factors of the ion Gaussian along each image box of atom J's r_loc
// sphere: exp(-d^2 / a^2) with d the FP64 displacement of grid index
// lo + i (the same operations as every displacement here), so that
// g = c_g T_x T_y T_z (three roundings from exp(-|d|^2 / a^2)).  One block
// per atom.
__global__ void __launch_bounds__(256)
k_gauss_tables(int n, double h, double L, const double *Rw, SpeciesDev sp, double *gtab,
               double *gtabd, int *glo) {
  __shared__ ImageBoxes B;
  const int J = blockIdx.x;
  const double c[3] = {Rw[3 * J], Rw[3 * J + 1], Rw[3 * J + 2]};
  image_boxes(c, L, h, sp.r_loc, n, B);
  __syncthreads();
  if (threadIdx.x < 81)
    glo[(size_t)J * 81 + threadIdx.x] = B.lo[threadIdx.x / 3][threadIdx.x % 3];
  double *T = gtab + (size_t)J * 27 * 3 * EMD_GT_EXT;
  for (int q = threadIdx.x; q < 27 * 3 * EMD_GT_EXT; q += blockDim.x) {
    const int img = q / (3 * EMD_GT_EXT), a = (q / EMD_GT_EXT) % 3, i = q % EMD_GT_EXT;
    if (i >= B.ext[img][a] || B.start[img + 1] == B.start[img]) continue;
    const int ni = a == 0 ? img % 3 - 1 : a == 1 ? (img / 3) % 3 - 1 : img / 9 - 1;
    const double d = emd_disp(B.lo[img][a] + i, h, c[a], ni, L);
    const double t = exp(-__dmul_rn(d, d) * sp.inv_a2);
    T[q] = t;
    if (a == 0) gtabd[((size_t)J * 27 + img) * EMD_GT_EXT + i] = t * d;
  }
}

// F_J^loc = h^3 sum_r v_es(r) g_J(d) 2 d / a^2 over the Gaussian support
// (-dE_es/dR_J of 1/2 h^3 sum n_tot v_es, n_tot = rho - sum g).  Grid
// (atom, split) over contiguous ranges of the flattened box space; partials
// are summed in split order by k_local_force_sum.  FP32 distances discard
// the box points certainly outside the sphere; the others get the exact FP64
// decision, and g comes from the separable tables (when present).
// HVP = true gives instead, for a direction lam per atom, the derivative
// d/dR_J of lam_J . F_loc,J at fixed potential:
//   h^3 sum v_es g_J (-2/a^2) [lam_J - 2 d (d . lam_J) / a^2].
template <bool HVP>
__global__ void __launch_bounds__(256)
k_local_force(int n, double h, double L, const double *Rw, const double *gtab,
              SpeciesDev sp, float margin, const double *va, const double *vb,
              const double *lam, double *part) {
  __shared__ ImageBoxes B;
  __shared__ float cf[27][3];
  __shared__ double red[8 * 3];
  const int J = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
  const double c[3] = {Rw[3 * J], Rw[3 * J + 1], Rw[3 * J + 2]};
  const double rl2 = __dmul_rn(sp.r_loc, sp.r_loc);
  const float rl2f = (float)rl2, hf = (float)h;
  image_boxes(c, L, h, sp.r_loc, n, B);
  if (threadIdx.x < 81) {
    const int img = threadIdx.x / 3, a = threadIdx.x % 3;
    const int ni = a == 0 ? img % 3 - 1 : a == 1 ? (img / 3) % 3 - 1 : img / 9 - 1;
    cf[img][a] = (float)(c[a] + ni * L);
  }
  __syncthreads();
  const double *T = gtab ? gtab + (size_t)J * 27 * 3 * EMD_GT_EXT : nullptr;
  const int total = B.start[27];
  const int per = (total + nsplit - 1) / nsplit;
  const int f0 = split * per, f1 = min(total, f0 + per);
  double acc[3] = {0.0, 0.0, 0.0};
  int img = 0;
  for (int f = f0 + threadIdx.x; f < f1; f += blockDim.x) {
    while (img < 26 && f >= B.start[img + 1]) ++img;
    const int k = f - B.start[img];
    const int ex = B.ext[img][0], ey = B.ext[img][1];
    const int kx = k % ex, ky = (k / ex) % ey, kz = k / (ex * ey);
    const int ix = B.lo[img][0] + kx, iy = B.lo[img][1] + ky, iz = B.lo[img][2] + kz;
    const float dxf = (float)ix * hf - cf[img][0], dyf = (float)iy * hf - cf[img][1],
                dzf = (float)iz * hf - cf[img][2];
    if (dxf * dxf + dyf * dyf + dzf * dzf > rl2f + margin) continue;
    const int ni[3] = {img % 3 - 1, (img / 3) % 3 - 1, img / 9 - 1};
    const double dx = emd_disp(ix, h, c[0], ni[0], L);
    const double dy = emd_disp(iy, h, c[1], ni[1], L);
    const double dz = emd_disp(iz, h, c[2], ni[2], L);
    const double d2 = emd_norm2(dx, dy, dz);
    if (d2 < rl2) {
      const int p = (iz * n + iy) * n + ix;
      const double *Ti = T ? T + (size_t)img * 3 * EMD_GT_EXT : nullptr;
      const bool tab = T && kx < EMD_GT_EXT && ky < EMD_GT_EXT && kz < EMD_GT_EXT;
      const double g = tab ? sp.c_g * (Ti[kx] * Ti[EMD_GT_EXT + ky] * Ti[2 * EMD_GT_EXT + kz])
                           : sp.c_g * exp(-d2 * sp.inv_a2);
      if (HVP) {
        const double l0 = lam[3 * J], l1 = lam[3 * J + 1], l2 = lam[3 * J + 2];
        const double w = (va[p] + vb[p]) * g * (-2.0 * sp.inv_a2);
        const double dl = (dx * l0 + dy * l1 + dz * l2) * (2.0 * sp.inv_a2);
        acc[0] += w * (l0 - dx * dl);
        acc[1] += w * (l1 - dy * dl);
        acc[2] += w * (l2 - dz * dl);
      } else {
        const double w = (va[p] + vb[p]) * g * (2.0 * sp.inv_a2);
        acc[0] += w * dx;
        acc[1] += w * dy;
        acc[2] += w * dz;
      }
    }
  }
  emd_block_sum<3>(acc, red);
  if (threadIdx.x == 0) {
    const double h3 = h * h * h;
    for (int a = 0; a < 3; ++a) part[((size_t)J * nsplit + split) * 3 + a] = h3 * acc[a];
  }
}

// The same force with one thread per row (y, z) of the image boxes and the
// Gaussian factored, g = c_g T_x(x) T_y(y) T_z(z):
//   F_x += c_g T_y T_z sum_x v T_x d_x,  F_{y,z} += c_g T_y T_z d_{y,z} sum_x v T_x
// over the row's chord through the sphere.  The chord is a contiguous run of
// x (the FP64 distance is monotone in x on each side of the centre); its
// exact ends are found by the FP64 decision, starting from an FP32 estimate,
// so the per-point work is two multiply-adds.  Tables T_x and T_x d_x come
// from k_gauss_tables.  Used for the forward force when the tables exist.
__global__ void __launch_bounds__(256)
k_local_force_rows(int n, double h, double L, const double *Rw, const double *gtab,
                   const double *gtabd, SpeciesDev sp, const double *va,
                   const double *vb, double *part) {
  __shared__ ImageBoxes B;
  __shared__ int rstart[28];
  __shared__ float cf[27][3];
  __shared__ double red[8 * 3];
  const int J = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
  const double c[3] = {Rw[3 * J], Rw[3 * J + 1], Rw[3 * J + 2]};
  const double rl2 = __dmul_rn(sp.r_loc, sp.r_loc);
  const float rl2f = (float)rl2, hf = (float)h, ihf = (float)(1.0 / h);
  image_boxes(c, L, h, sp.r_loc, n, B);
  if (threadIdx.x == 0) {
    int acc = 0;   // rows (y, z) per image, boxes with no point skipped
    for (int img = 0; img < 27; ++img) {
      rstart[img] = acc;
      if (B.start[img + 1] > B.start[img]) acc += B.ext[img][1] * B.ext[img][2];
    }
    rstart[27] = acc;
  }
  if (threadIdx.x < 81) {
    const int img = threadIdx.x / 3, a = threadIdx.x % 3;
    const int ni = a == 0 ? img % 3 - 1 : a == 1 ? (img / 3) % 3 - 1 : img / 9 - 1;
    cf[img][a] = (float)(c[a] + ni * L);
  }
  __syncthreads();
  const double *TJ = gtab + (size_t)J * 27 * 3 * EMD_GT_EXT;
  const double *DJ = gtabd + (size_t)J * 27 * EMD_GT_EXT;
  const int nrows = rstart[27];
  const int per = (nrows + nsplit - 1) / nsplit;
  const int q0 = split * per, q1 = min(nrows, q0 + per);
  double acc[3] = {0.0, 0.0, 0.0};
  int img = 0;
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    while (img < 26 && q >= rstart[img + 1]) ++img;
    const int k = q - rstart[img];
    const int ey = B.ext[img][1];
    const int ky = k % ey, kz = k / ey;
    const int iy = B.lo[img][1] + ky, iz = B.lo[img][2] + kz;
    const float dyf = (float)iy * hf - cf[img][1], dzf = (float)iz * hf - cf[img][2];
    const float remf = rl2f - (dyf * dyf + dzf * dzf);
    if (remf < -4.0f * hf * hf - 1e-3f * rl2f) continue;   // far from the sphere
    const int ni[3] = {img % 3 - 1, (img / 3) % 3 - 1, img / 9 - 1};
    const int lo0 = B.lo[img][0], hi0 = lo0 + B.ext[img][0] - 1;
    const float wf = sqrtf(fmaxf(remf, 0.f));
    // the exact chord lies within two points of the FP32 estimate (FP32
    // errors are far below a grid step); scan in from both ends of that range
    const int xa = max(lo0, (int)ceilf((cf[img][0] - wf) * ihf) - 2);
    const int xb = min(hi0, (int)floorf((cf[img][0] + wf) * ihf) + 2);
    const double dy = emd_disp(iy, h, c[1], ni[1], L);
    const double dz = emd_disp(iz, h, c[2], ni[2], L);
    auto inside = [&](int x) {
      return emd_norm2(emd_disp(x, h, c[0], ni[0], L), dy, dz) < rl2;
    };
    int xs = xa;
    while (xs <= xb && !inside(xs)) ++xs;
    if (xs > xb) continue;                                   // row misses the sphere
    int xe = xb;
    while (xe > xs && !inside(xe)) --xe;
    const double *Tx = TJ + (size_t)img * 3 * EMD_GT_EXT;
    const double *Dx = DJ + (size_t)img * EMD_GT_EXT;
    const double tyz = Tx[EMD_GT_EXT + ky] * Tx[2 * EMD_GT_EXT + kz];
    const size_t rowp = ((size_t)iz * n + iy) * n;
    double s0 = 0.0, s1 = 0.0;
    for (int x = xs; x <= xe; ++x) {
      const double v = va[rowp + x] + vb[rowp + x];
      s0 += v * Tx[x - lo0];
      s1 += v * Dx[x - lo0];
    }
    const double w = sp.c_g * tyz * (2.0 * sp.inv_a2);
    acc[0] += w * s1;
    acc[1] += w * dy * s0;
    acc[2] += w * dz * s0;
  }
  emd_block_sum<3>(acc, red);
  if (threadIdx.x == 0) {
    const double h3 = h * h * h;
    for (int a = 0; a < 3; ++a) part[((size_t)J * nsplit + split) * 3 + a] = h3 * acc[a];
  }
}

__global__ void k_local_force_sum(const double *part, int n_atoms, int nsplit,
                                  double *F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n_atoms) return;
  const int J = i / 3, a = i % 3;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[((size_t)J * nsplit + k) * 3 + a];
  F[i] = s;
}

// Short-range ion-ion term E_sr = 1/2 sum' Z^2 erfc(d/s)/d (s = sqrt2 a, d <
// 12 bohr, all images) and its force.  Grid (atom J, split): the (atom K,
// image) pairs of J are cut into EMD_SR_SPLIT contiguous ranges, each CTA
// writes an FP64 partial (fixed-order block sum), and k_short_range_sum adds
// the partials in split order.
__global__ void __launch_bounds__(256)
k_short_range(SpeciesDev sp, int n_atoms, const double *Rw, double L, int nmax,
              double *part) {
  __shared__ double red[8 * 4];
  const int J = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
  const double s = sqrt(2.0) * sp.a_loc;
  const double zz = sp.z * sp.z;
  const double rcut = 12.0;
  const double k2 = 2.0 / (s * sqrt(M_PI));
  const int side = 2 * nmax + 1, nimg = side * side * side;
  const int total = n_atoms * nimg, per = (total + nsplit - 1) / nsplit;
  const int q0 = split * per, q1 = min(total, q0 + per);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int K = q / nimg, im = q % nimg;
    const int nx = im % side - nmax, ny = (im / side) % side - nmax,
              nz = im / (side * side) - nmax;
    if (K == J && nx == 0 && ny == 0 && nz == 0) continue;
    const double dv0 = Rw[3 * J] - Rw[3 * K] - nx * L;
    const double dv1 = Rw[3 * J + 1] - Rw[3 * K + 1] - ny * L;
    const double dv2 = Rw[3 * J + 2] - Rw[3 * K + 2] - nz * L;
    const double d2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2;
    if (d2 >= rcut * rcut || d2 <= 0.0) continue;
    const double d = sqrt(d2);
    const double ef = erfc(d / s) / d;
    acc[0] += ef;
    const double fm = zz * (ef / d + k2 * exp(-d2 / (s * s)) / d) / d;
    acc[1] += fm * dv0;
    acc[2] += fm * dv1;
    acc[3] += fm * dv2;
  }
  emd_block_sum<4>(acc, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) part[((size_t)J * nsplit + split) * 4 + k] = acc[k];
}

__global__ void k_short_range_sum(const double *part, int n_atoms, int nsplit, double zz,
                                  double *F, double *e_part) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= n_atoms) return;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < nsplit; ++k)
    for (int c = 0; c < 4; ++c) a[c] += part[((size_t)J * nsplit + k) * 4 + c];
  e_part[J] = 0.5 * zz * a[0];
  F[3 * J] = a[1];
  F[3 * J + 1] = a[2];
  F[3 * J + 2] = a[3];
}

// R(t+dt) = R + V dt + F dt^2 / (2M), in the reference's rounding order.
__global__ void k_vv_positions(int n, const double *R, const double *V,
                               const double *F, double dt, double c2,
                               double *Rn) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    Rn[i] = __dadd_rn(__dadd_rn(R[i], __dmul_rn(V[i], dt)), __dmul_rn(F[i], c2));
}

// F_new = (F_loc + F_nl) + F_sr (+ Z e on z); V += (F_old + F_new) dt/(2M).
__global__ void k_vv_velocities(int n_atoms, const double *Fl,
                                const double *Fn, const double *Fs,
                                double fz, double *F, double *V, double c1,
                                int update_v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n_atoms) return;
  double f = __dadd_rn(__dadd_rn(Fl[i], Fn[i]), Fs[i]);
  if (i % 3 == 2) f = __dadd_rn(f, fz);
  if (update_v) V[i] = __dadd_rn(V[i], __dmul_rn(__dadd_rn(F[i], f), c1));
  F[i] = f;
}

}  // namespace

void emd_launch_wrap(const double *R, double *Rw, int n_atoms, double L,
                     cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  int n = 3 * n_atoms;
  k_wrap<<<(n + 127) / 128, 128, 0, st>>>(R, Rw, n, L);
}

void emd_launch_tables(const GridInfo &g, const SpeciesDev &sp, int n_atoms,
                       TableSet &t, int *err, cudaStream_t st) {
  emd_note_launches(2 + 2 * (n_atoms > 0));
  const int nt = (g.n + EMD_TILE - 1) / EMD_TILE;
  const int ntiles = nt * nt * nt;
  const float rmax = (float)fmax(sp.r_proj, sp.r_loc);
  k_tile_candidates<<<ntiles, 256, 0, st>>>(
      g.n, g.h, g.L, t.Rw, n_atoms, rmax, t.tile_cnt, t.tile_ent, err);
  if (t.gtab && n_atoms > 0) {
    emd_note_launches(1);
    k_gauss_tables<<<n_atoms, 256, 0, st>>>(g.n, g.h, g.L, t.Rw, sp, t.gtab, t.gtabd,
                                            t.glo);
  }
  const float margin_pt = emd_fp32_d2_margin(g.L, fmax(sp.r_proj, sp.r_loc));
  if (t.te_off)
    k_point_table<true><<<ntiles, 512, 0, st>>>(g.n, g.n3, g.h, g.L, t.Rw, sp, margin_pt,
                                                t.tile_cnt, t.tile_ent, t.gtab, t.glo,
                                                t.pt_cnt, t.pt_J, t.pt_p, t.pt_pf, t.pt4, t.pt4d,
                                                t.g_ion, t.te_off, t.te_pp, t.te_q,
                                                t.kmax, nullptr, err);
  else
    k_point_table<false><<<ntiles, 512, 0, st>>>(g.n, g.n3, g.h, g.L, t.Rw, sp, margin_pt,
                                                 t.tile_cnt, t.tile_ent, t.gtab, t.glo,
                                                 t.pt_cnt, t.pt_J, t.pt_p, t.pt_pf, t.pt4, t.pt4d,
                                                 t.g_ion, t.te_off, t.te_pp, t.te_q,
                                                 t.kmax, t.pt_rec, err);
  if (n_atoms > 0 && !t.te_off) {
    dim3 grid(n_atoms, EMD_SPLIT);
    const float margin = emd_fp32_d2_margin(g.L, sp.r_proj);
    for (int pass = 0; pass < 2; ++pass)
      k_atom_table<<<grid, 256, 0, st>>>(pass, g.n, g.h, g.L, t.Rw, sp, t.cap, margin,
                                         t.split_cnt, t.at_cnt, t.at_pt, t.at_p, t.at_d,
                                         t.at_rec, t.at_w, err);
  }
}

void emd_launch_local_force(const GridInfo &g, const SpeciesDev &sp,
                            int n_atoms, const TableSet &t, const double *v_es_a,
                            const double *v_es_b, double *part, double *F,
                            cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  dim3 grid(n_atoms, EMD_SPLIT);
  if (t.gtab)
    k_local_force_rows<<<grid, 256, 0, st>>>(g.n, g.h, g.L, t.Rw, t.gtab, t.gtabd, sp,
                                             v_es_a, v_es_b, part);
  else
    k_local_force<false><<<grid, 256, 0, st>>>(g.n, g.h, g.L, t.Rw, t.gtab, sp,
                                               emd_fp32_d2_margin(g.L, sp.r_loc), v_es_a,
                                               v_es_b, nullptr, part);
  const int m = 3 * n_atoms;
  k_local_force_sum<<<(m + 127) / 128, 128, 0, st>>>(part, n_atoms, EMD_SPLIT, F);
}

void emd_launch_local_force_hvp(const GridInfo &g, const SpeciesDev &sp,
                                int n_atoms, const TableSet &t,
                                const double *v_es_a, const double *v_es_b,
                                const double *lam, double *part, double *out,
                                cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  dim3 grid(n_atoms, EMD_SPLIT);
  k_local_force<true><<<grid, 256, 0, st>>>(g.n, g.h, g.L, t.Rw, t.gtab, sp,
                                            emd_fp32_d2_margin(g.L, sp.r_loc), v_es_a,
                                            v_es_b, lam, part);
  const int m = 3 * n_atoms;
  k_local_force_sum<<<(m + 127) / 128, 128, 0, st>>>(part, n_atoms, EMD_SPLIT, out);
}

void emd_launch_short_range(const SpeciesDev &sp, int n_atoms, const double *Rw,
                            double L, double *F, double *e_part, double *part,
                            cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  // pairs within 12 bohr: wrapped positions differ by less than L, so image
  // shifts up to (12 + L) / L box lengths suffice
  const int nmax = (int)floor((12.0 + L) / L);
  dim3 grid(n_atoms, EMD_SR_SPLIT);
  k_short_range<<<grid, 256, 0, st>>>(sp, n_atoms, Rw, L, nmax, part);
  k_short_range_sum<<<(n_atoms + 127) / 128, 128, 0, st>>>(part, n_atoms, EMD_SR_SPLIT,
                                                          sp.z * sp.z, F, e_part);
}

void emd_launch_vv_positions(int n_atoms, const double *R, const double *V,
                             const double *F, double dt, double mass,
                             double *R_new, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  const double c2 = (dt * dt) / (2.0 * mass);
  int n = 3 * n_atoms;
  k_vv_positions<<<(n + 127) / 128, 128, 0, st>>>(n, R, V, F, dt, c2, R_new);
}

void emd_launch_vv_velocities(int n_atoms, const double *F_loc,
                              const double *F_nl, const double *F_sr,
                              double field_z, double z, double *F, double *V,
                              double dt, double mass, int update_v,
                              cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  const double c1 = dt / (2.0 * mass);
  const double fz = z * field_z;
  int n = 3 * n_atoms;
  k_vv_velocities<<<(n + 127) / 128, 128, 0, st>>>(n_atoms, F_loc, F_nl, F_sr,
                                                    fz, F, V, c1, update_v);
}
