// Internal declarations shared by the libemd translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "emd.h"

#define EMD_PT_KMAX 16          // atoms per grid point in the point-major table
#define EMD_TILE 8              // edge of the tiles that carry atom candidates
#define EMD_TILE_CAND_MAX 160   // (atom, image) candidates per tile
#define EMD_TILE_ATOM_MAX 32    // distinct atoms per tile (point-major projections)
#define EMD_MAX_HALF_ORDER 6    // fd_order / 2 <= 6
#define EMD_TE_CAP (EMD_TILE * EMD_TILE * EMD_TILE * EMD_PT_KMAX)
#define EMD_GT_EXT 64
#define EMD_SR_SPLIT 8          // CTAs per atom for the short-range ion term
#define EMD_SPLIT 16            // CTAs per atom for table building and local forces

// error bits raised by kernels (device flag, read by emd_get_*)
// Perdew-Zunger (1981) correlation of the unpolarised uniform gas, the LDA
// of Sec. 5: eps_c = gam / (1 + b1 sqrt(r_s) + b2 r_s) for r_s >= 1 and
// A ln r_s + B + C r_s ln r_s + D r_s below.  C and D follow from continuity
// of eps_c and d eps_c / d r_s at r_s = 1 (the published four-decimal values
// are these rounded); with the rounded ones eps_c jumps by 3.2e-5 Ha at
// r_s = 1 and E_KS is not differentiable where a grid point's density
// crosses 3 / (4 pi), which shows up as an energy drift independent of dt.
namespace pz81 {
constexpr double gam = -0.1423, b1 = 1.0529, b2 = 0.3334;
constexpr double A = 0.0311, B = -0.048;
constexpr double q1 = 1.0 + b1 + b2;
constexpr double D = gam / q1 - B;                                  // eps_c
constexpr double C = -gam * (0.5 * b1 + b2) / (q1 * q1) - A - D;    // slope
}  // namespace pz81

#define EMD_ERRBIT_PT   1       // per-point list overflow
#define EMD_ERRBIT_TILE 2       // per-tile candidate overflow
#define EMD_ERRBIT_AT   4       // per-atom table overflow
#define EMD_ERRBIT_WAIT 8       // a bounded device wait gave up

template <typename T> struct cplx;
template <> struct cplx<double> { typedef double2 type; };
template <> struct cplx<float> { typedef float2 type; };

struct SpeciesDev {
  double z, mass, a_loc, r_loc, r_c, h_kb, r_proj;
  double c_g;      // Z pi^-3/2 a^-3
  double c_p;      // pi^-3/4 r_c^-3/2
  double inv_a2;   // 1 / a^2
  double inv_2rc2; // 1 / (2 r_c^2)
  double inv_rc2;  // 1 / r_c^2
  // several projectors per atom: channels k = 0 .. nch - 1 = (lmax + 1)^2 - 1
  // (s; x, y, z; sqrt3 xy, sqrt3 yz, sqrt3 zx, sqrt3/2 (x^2 - y^2),
  // (3z^2 - d^2)/2), strengths hl[l] (hl[0] = h_kb) and norms nl[l] (nl[0] = c_p)
  int lmax, nch;
  double hl[3], nl[3];
};

// angular momentum of channel k
__host__ __device__ __forceinline__ int emd_channel_l(int k) { return k == 0 ? 0 : k < 4 ? 1 : 2; }

// The projector values of channels 1 .. nch - 1 at displacement d (channel 0,
// the s-projector, is computed by the callers as before), and optionally
// their derivatives with respect to the atom position, -grad_d p =
// N_l e (S d / r_c^2 - grad S), e = exp(-d^2 / (2 r_c^2)).
__device__ __forceinline__ void emd_channel_values(const SpeciesDev &sp, double dx, double dy,
                                                   double dz, double e, double *pk,
                                                   double (*gk)[3]) {
  const double s3 = 1.7320508075688772;
  double S[9], G[9][3];
  S[1] = dx; G[1][0] = 1.0; G[1][1] = 0.0; G[1][2] = 0.0;
  S[2] = dy; G[2][0] = 0.0; G[2][1] = 1.0; G[2][2] = 0.0;
  S[3] = dz; G[3][0] = 0.0; G[3][1] = 0.0; G[3][2] = 1.0;
  S[4] = s3 * dx * dy; G[4][0] = s3 * dy; G[4][1] = s3 * dx; G[4][2] = 0.0;
  S[5] = s3 * dy * dz; G[5][0] = 0.0; G[5][1] = s3 * dz; G[5][2] = s3 * dy;
  S[6] = s3 * dz * dx; G[6][0] = s3 * dz; G[6][1] = 0.0; G[6][2] = s3 * dx;
  S[7] = 0.5 * s3 * (dx * dx - dy * dy); G[7][0] = s3 * dx; G[7][1] = -s3 * dy; G[7][2] = 0.0;
  S[8] = 0.5 * (2.0 * dz * dz - dx * dx - dy * dy); G[8][0] = -dx; G[8][1] = -dy; G[8][2] = 2.0 * dz;
  for (int k = 1; k < sp.nch; ++k) {
    const double ne = sp.nl[emd_channel_l(k)] * e;
    pk[k] = ne * S[k];
    if (gk) {
      gk[k][0] = ne * (S[k] * dx * sp.inv_rc2 - G[k][0]);
      gk[k][1] = ne * (S[k] * dy * sp.inv_rc2 - G[k][1]);
      gk[k][2] = ne * (S[k] * dz * sp.inv_rc2 - G[k][2]);
    }
  }
}

// One set of ion positions and every table derived from it.
struct TableSet {
  double *R;        // [n_atoms][3] positions as given (unwrapped)
  double *Rw;       // [n_atoms][3] folded into [0, L)
  int *tile_cnt;    // [n_tiles]
  int *tile_ent;    // [n_tiles][EMD_TILE_CAND_MAX], J*27 + image
  int *pt_cnt;      // [n3]
  int kmax;         // entries per point: EMD_PT_KMAX x projectors per atom
  int *pt_J;        // [kmax][n3] projector P = J n_ch + k (atom J if n_ch = 1)
  double *pt_p;     // [EMD_PT_KMAX][n3] p_J(r) summed over images
  float *pt_pf;     // [EMD_PT_KMAX][n3] the same in FP32 (complex64 path)
  int2 *pt4;        // [n3][4] first four (atom, FP32 p bits) per point, unused
                    // slots (0, 0.0f); entry 0's atom carries count << 16
  // complex128, bo = 2 (double-float stage): per point 3 x int4 = (J_0 |
  // count << 16, J_1, J_2, J_3), (p_0 hi, p_0 lo, p_1 hi, p_1 lo), (p_2 hi,
  // p_2 lo, p_3 hi, p_3 lo) with p in double-float (unused entries 0);
  // NULL for other layouts
  int4 *pt4d;
  // complex128 with several projectors per atom: every entry as (P, p hi,
  // p lo, 0), [kmax][n3], for the stage's entries past the first four;
  // NULL otherwise
  int4 *pt_rec;
  int *at_cnt;      // [n_atoms] (projector P's list: at_cnt[P / n_ch])
  int *split_cnt;   // [n_atoms][EMD_SPLIT] hits per range (table building)
  int *at_pt;       // [n_atoms][cap] flat grid index
  double *at_p;     // [n_atoms][cap] p value of that (point, image)
  double *at_d;     // [n_atoms][cap][3] displacement r - R_image
  // complex128 with bo = 2 (double-float projections and moments): the same
  // entries pre-split, (point, p hi, p lo, 0) and (w_x hi, w_x lo, w_y hi,
  // w_y lo), (w_z hi, w_z lo, 0, 0) with w = p d / r_c^2; NULL otherwise
  // (with several projectors per atom, lists per projector P, [n_proj][cap],
  // the entries of P at the positions of atom P / n_ch's entries; w = the
  // derivative of p_P with respect to the atom position)
  uint4 *at_rec;    // [n_proj][cap]
  float4 *at_w;     // [n_proj][cap][2]
  // complex64 path: per 8^3 tile, the (point, atom) pairs of the projectors
  // grouped by the tile's atoms (slots, in tile_atoms order): te_off[t][s]
  // is the first entry of slot s (te_off[t][S] the end), an entry holds the
  // point's index in the tile, p summed over images, and sum p d / r_c^2
  int *te_off;             // [n_tiles][EMD_TILE_ATOM_MAX + 1]
  uint2 *te_pp;            // [n_tiles][EMD_TE_CAP] (point index, bits of p)
  float4 *te_q;            // [n_tiles][EMD_TE_CAP] (sum p d / r_c^2, bits of
                           // the point index)
  int *tile_nat;    // [n_tiles] distinct atoms per tile
  int *tile_atoms;  // [n_tiles][EMD_TILE_ATOM_MAX] in atom order
  int *tile_off;    // [n_tiles] exclusive prefix sum of tile_nat
  int *at_ntiles;   // [n_atoms] tiles listing the atom
  int2 *at_tiles;   // [n_atoms][n_tiles] (tile, slot) in tile order
  int n_slots_cap;  // n_tiles * EMD_TILE_ATOM_MAX
  double *g_ion;    // [n3] sum of Gaussian ion charges
  // separable ion Gaussian: exp(-d_a^2 / a^2) per atom, image and axis along
  // the image box of the r_loc sphere, [n_atoms][27][3][EMD_GT_EXT]; NULL if
  // a box is longer than EMD_GT_EXT points (the kernels then call exp)
  double *gtab;
  int *glo;         // [n_atoms][27][3] first grid index of each table
  double *gtabd;    // [n_atoms][27][EMD_GT_EXT] T_x d_x along x
  double *v_loc;    // [n3] Poisson(-g_ion)
  int cap;
};

// ---------------------------------------------------------------------------
// Double-float split of a double from its bits: x = hi + lo, hi = x truncated
// to 24 significant bits (sign, exponent rebased from 1023 to 127 and the
// top 23 stored mantissa bits, moved into place by one funnel shift), lo =
// the remaining 29 mantissa bits converted to float with rounding to nearest
// and scaled by 2^(e - 1075), so |x - hi - lo| <= 2^-48 |x|.  |x| < 2^-126
// gives hi = 0, and lo is dropped below |x| < 2^-74 (an absolute error under
// 1e-29).  No FP64 instruction; the one conversion runs on the conversion
// unit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 emd_df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const unsigned e = (h >> 20) & 0x7ffu;
  const unsigned s = h & 0x80000000u;
  // (h - 896 << 20) << 3 | l >> 29: the rebased exponent fits 8 bits, so the
  // sign position receives a zero and is set from s
  const unsigned hb = s | __funnelshift_l(l, (h & 0x7fffffffu) - (896u << 20), 3);
  const float r = __uint2float_rn(l & 0x1fffffffu);
  const float sc = __uint_as_float(s | ((max(e, 948u) - 948u) << 23));   // 2^(e-1075) or 0
  return make_float2(e >= 897u ? __uint_as_float(hb) : 0.f, __fmul_rn(r, sc));
}

// Double-float arithmetic on the FP32 pipes (the complex128 stage,
// projections and nonlocal-force moments).
__device__ __forceinline__ float2 df_split(double x) { return emd_df_split(x); }

// exact widening of a float (normal or zero; float subnormals, below 2^-126,
// become 0) by integer operations
__device__ __forceinline__ double df_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned hw = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  const double d = __hiloint2double((int)hw, (int)(u << 29));
  return ex == 0u ? 0.0 : d;
}

// Double-float pairs for a complex value, packed so that both components go
// through one FP32x2 instruction: hi = (re_hi, im_hi), lo = (re_lo, im_lo);
// the packed operations round each lane as the scalar ones would.
__device__ __forceinline__ float2 f2neg_sub(float2 a, float2 b) {   // a - b
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// Knuth's TwoSum, per lane: s + e = a + b exactly
__device__ __forceinline__ void dfp_two_sum(float2 a, float2 b, float2 &s, float2 &e) {
  s = __fadd2_rn(a, b);
  const float2 bb = f2neg_sub(s, a);
  e = __fadd2_rn(f2neg_sub(a, f2neg_sub(s, bb)), f2neg_sub(b, bb));
}
// (hi, lo) += (p, q), p the leading part
__device__ __forceinline__ void dfp_add(float2 &hi, float2 &lo, float2 p, float2 q) {
  float2 s, e;
  dfp_two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd2_rn(lo, __fadd2_rn(e, q));
}
// TwoProduct of a scalar pair (w, w) and x, per lane: p + pe = w x exactly
__device__ __forceinline__ void dfp_two_prod(float2 w, float2 x, float2 &p, float2 &pe) {
  p = __fmul2_rn(w, x);
  pe = __ffma2_rn(w, x, __fmul2_rn(make_float2(-w.x, -w.y), x));
}
// (hi, lo) += (wh + wl)(xh + xl) for a real double-float w, dropping wl xl
__device__ __forceinline__ void dfp_add_prod(float2 &hi, float2 &lo, float wh, float wl,
                                             float2 xh, float2 xl) {
  const float2 w2 = make_float2(wh, wh);
  float2 p, pe;
  dfp_two_prod(w2, xh, p, pe);
  dfp_add(hi, lo, p, __ffma2_rn(w2, xl, __ffma2_rn(make_float2(wl, wl), xh, pe)));
}

// a complex double-float: (re_hi, im_hi, re_lo, im_lo)
__device__ __forceinline__ float4 df_split2(double2 v) {
  const float2 r = df_split(v.x), i = df_split(v.y);
  return make_float4(r.x, i.x, r.y, i.y);
}
__device__ __forceinline__ float2 f4hi(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f4lo(float4 v) { return make_float2(v.z, v.w); }

// ---------------------------------------------------------------------------
// Exact displacement arithmetic.  The support decision d^2 < r^2 is an
// integer decision taken in FP64 from the same operations, in the same
// order and rounding, as the reference definition: no contraction into FMA.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double emd_wrap_pos(double X, double L) {
  return __dsub_rn(X, __dmul_rn(L, floor(__ddiv_rn(X, L))));
}
__device__ __forceinline__ double emd_disp(int i, double h, double c, int nimg,
                                           double L) {
  return __dsub_rn(__dsub_rn(__dmul_rn((double)i, h), c),
                   __dmul_rn((double)nimg, L));
}
__device__ __forceinline__ double emd_norm2(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                   __dmul_rn(dz, dz));
}

// Deterministic block reduction of NV doubles per thread (fixed tree order).
// Requires blockDim.x a multiple of 32 and <= 1024.  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void emd_block_sum(double (&v)[NV], double *smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    v[k] = a;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int w = 0; w < nwarp; ++w) a += smem[w * NV + k];
      v[k] = a;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files).  All take the stream to issue on.
// ---------------------------------------------------------------------------
struct GridInfo {
  int n, n3;
  double h, L;
};

// Process-wide count of kernel launches issued by the library (for the
// benchmark's launch count); defined in emd_api.cu.
void emd_note_launches(int k);
// Set the calling thread's error message (emd_last_error) and return code.
int emd_set_error(int code, const char *msg);

// tables.cu
void emd_launch_wrap(const double *R, double *Rw, int n_atoms, double L,
                     cudaStream_t st);
void emd_launch_tables(const GridInfo &g, const SpeciesDev &sp, int n_atoms,
                       TableSet &t, int *err, cudaStream_t st);
// part: [n_atoms][EMD_SPLIT][3] scratch
void emd_launch_local_force(const GridInfo &g, const SpeciesDev &sp,
                            int n_atoms, const TableSet &t, const double *v_es_a,
                            const double *v_es_b, double *part, double *F,
                            cudaStream_t st);
void emd_launch_short_range(const SpeciesDev &sp, int n_atoms, const double *Rw,
                            double L, double *F, double *e_part, double *part,
                            cudaStream_t st);
void emd_launch_vv_positions(int n_atoms, const double *R, const double *V,
                             const double *F, double dt, double mass,
                             double *R_new, cudaStream_t st);
void emd_launch_vv_velocities(int n_atoms, const double *F_loc,
                              const double *F_nl, const double *F_sr,
                              double field_z, double z, double *F,
                              double *V, double dt, double mass, int update_v,
                              cudaStream_t st);

// poisson.cu
void emd_fft_plan_check(int n, int *ok);   // host-only factor check
int emd_fft_prepare(int n);                 // twiddle tables on the device
void emd_launch_poisson(const GridInfo &g, const double *charge, double *v,
                        double2 *work_a, double2 *work_b, cudaStream_t st);
// out = the inverse transform of K(G) r(G), Kerker's K = |G|^2 / (|G|^2 +
// q0^2) for G != 0 and K(0) = 1; out may alias r
void emd_launch_kerker(const GridInfo &g, double q0, const double *r, double *out,
                       double2 *work_a, double2 *work_b, cudaStream_t st);
void emd_launch_lda(int n3, const double *rho, const double *v_h,
                    double *eps_xc, double *v_xc, double *vhxc,
                    cudaStream_t st);
// v_eff = v_loc + extrapolated v_Hxc + field term (FP64 and, if v_eff_f,
// FP32); if v_diag, also (d, d, d, d) with d = w0 + v_eff in FP32
void emd_launch_veff(const GridInfo &g, const double *v_loc,
                     const double *const *hist, int hist_len, double field,
                     double *v_eff, float *v_eff_f, cudaStream_t st,
                     float4 *v_diag = nullptr, double w0 = 0.0);
// partials[b] = block sums of (a - c)(b + d); c, d, b may be NULL
void emd_launch_dot_partials(int n3, const double *a, const double *b,
                             const double *c, const double *d,
                             double *partials, int nblocks, cudaStream_t st);
void emd_launch_sum(const double *partials, int n, double *out,
                    cudaStream_t st);

// groundstate.cu
// out = alpha (w - c y) - beta out over n complex values of the orbital
// precision (beta = 0: out only written); out aliases neither w nor y
void emd_launch_cheb(int prec, size_t n, const void *w, const void *y, void *out,
                     double alpha, double c, double beta, cudaStream_t st);
struct EmdComb {
  const double *p[16];
  double w[16];
  int m;
};
// out = sum_k w_k p_k over n3 points
void emd_launch_comb(int n3, const EmdComb &cb, double *out, cudaStream_t st);
// part[b] = block sums of |a - b|
void emd_launch_absdiff_partials(int n3, const double *a, const double *b, double *part,
                                 int nblocks, cudaStream_t st);
// Rayleigh-Ritz products over canonical column-major sets (column i at
// X + i n3; complex128 for EMD_FP64, complex64 otherwise): G = scale X^H Y
// (m x m, column-major FP64, summed in FP64 in a fixed order; part holds
// emd_gram_scratch(n3, m) double2), and B = X V (V column-major FP64)
int emd_gram_chunks(int n3);
size_t emd_gram_scratch(int n3, int m);
void emd_launch_gram(int prec, const void *X, const void *Y, int n3, int m, double scale,
                     double2 *part, double2 *G, cudaStream_t st);
void emd_launch_rotate(int prec, const void *X, const double2 *V, int n3, int m, void *B,
                       cudaStream_t st);
// columns c0 .. c1-1 of a canonical (n3 x m, column-major) orbital array
// filled with uniform values in [-1, 1) (counter hash of seed and index)
void emd_launch_fill_random(int prec, void *canon, size_t n3, int c0, int c1, unsigned seed,
                            cudaStream_t st);

// observables.cu
// part[a * nblocks + b]: block sums of rho (r_a - L/2), a = x, y, z
void emd_launch_dipole_partials(int n, double h, const double *rho, double *part, int nblocks,
                                cudaStream_t st);

// hpsi.cu
struct StageArgs {
  const void *u_in;
  const void *psi0;
  void *u_out;
  const void *v_eff;       // double* (FP64) or float* (FP32)
  const void *v_diag = nullptr;   // FP32: float4 (d, d, d, d), d = w_0 + v_eff
  const TableSet *tab;
  const void *hc;          // [n_atoms][n_orb_pad] h_kb*c in orbital precision
  double a;                // tau / k ; u_out = psi0 + (-i a) H u_in
  int apply_only;          // 1: u_out = H u_in (psi0 unused)
  int *err = nullptr;      // device error bits (EMD_ERRBIT_*), may be NULL
};
struct OrbLayout {
  int n, n3, bo, n_blk, n_orb, n_orb_pad, prec, half_order, n_atoms;
  // projectors: nch per atom, n_proj = n_atoms nch rows of c and hc; hl[l]
  // the strength of channel l (hl[0] = h_kb)
  int nch = 1, n_proj = 0;
  double hl[3] = {0.0, 0.0, 0.0};
  int stage_variant;   // Horner-stage kernel (EMD_OPT_STAGE_VARIANT)
  int zchunk;          // planes per z-chunk of the marching stage kernels, 0 = automatic
  double h;
  double w[EMD_MAX_HALF_ORDER + 1];   // w_0 = -3 c_0 / (2 h^2), w_k = -c_k/(2 h^2)
  // the same stencil as integers over a common denominator: c_k = num_k / den
  // (the double-float FP64 stage accumulates with these, exact in FP32)
  double num[EMD_MAX_HALF_ORDER + 1], den;
};
void emd_launch_stage(const OrbLayout &o, const StageArgs &a, cudaStream_t st);
void emd_launch_project(const OrbLayout &o, const TableSet &t, int n_atoms,
                        const void *u, double h3, double h_kb, double2 *c,
                        void *hc, cudaStream_t st);
void emd_launch_density(const OrbLayout &o, const void *u, double occ,
                        double *rho, cudaStream_t st);
void emd_launch_kinetic_partials(const OrbLayout &o, const void *u,
                                 double *partials, int *nparts,
                                 cudaStream_t st);
// coef = -2 h_kb occ; coef_unit = -2 occ (times each channel's strength when
// the atoms carry several projectors)
void emd_launch_nl_force(const OrbLayout &o, const TableSet &t, int n_atoms,
                         const void *u, const double2 *c, double h3,
                         double coef, double coef_unit, double inv_rc2, double *part,
                         double *F_nl, cudaStream_t st);
// groundstate.cu, per-orbital weights: u_A <- w_A u_A for the orbitals A < n_orb of a
// packed set (layout o), and for the n_vec columns of a canonical set
// (complex64 when c64, else complex128)
void emd_launch_scale_orbitals(const OrbLayout &o, void *u, int n_orb, const double *w,
                               cudaStream_t st);
void emd_launch_scale_canon(bool c64, void *c, size_t n3, int n_vec, const double *w,
                            cudaStream_t st);
void emd_launch_pack(const OrbLayout &o, const double2 *canon, void *u,
                     int n_vec, cudaStream_t st);
void emd_launch_unpack(const OrbLayout &o, const void *u, double2 *canon,
                       int n_vec, cudaStream_t st);
// the same with complex64 host-side canonical arrays
void emd_launch_pack_c64(const OrbLayout &o, const float2 *canon, void *u, int n_vec,
                         cudaStream_t st);
void emd_launch_unpack_c64(const OrbLayout &o, const void *u, float2 *canon, int n_vec,
                           cudaStream_t st);
// sum |c|^2 over n entries; rows of `row` entries, row r weighted by w[l] of
// its channel l = emd_channel_l(r % nch) (w = {1, ...} with nch = 1)
void emd_launch_abs2_sum(const double2 *c, int n, int row, int nch, const double *w, double *out,
                         cudaStream_t st);

// project_pm.cu
void emd_launch_tile_atoms(const GridInfo &g, int n_atoms, TableSet &t, int *err,
                           cudaStream_t st);
// partial: [n_blk][n_slots_cap][bo] complex FP64 scratch
void emd_launch_project_pm(const OrbLayout &o, const TableSet &t, int n_atoms,
                           const void *u, double h3, double h_kb, double2 *c,
                           void *hc, double2 *partial, cudaStream_t st);

// adjoint.cu (FP64 orbitals)
void emd_adj_axpy(double2 *y, const double2 *x, size_t n, cudaStream_t st);
void emd_adj_gv(const OrbLayout &o, const double2 *mu, const double2 *u, double b,
                double *g, cudaStream_t st);
void emd_adj_project_grad(const OrbLayout &o, const TableSet &t, int n_atoms,
                          const double2 *x, double h3, double h_kb,
                          double inv_rc2, double2 *c, double2 *hc, double2 *dc,
                          cudaStream_t st);
void emd_adj_proj_sens(const double2 *cm, const double2 *dcm, const double2 *cu,
                       const double2 *dcu, int n_atoms, int n_orb, int n_orb_pad,
                       double coef, double *gR, cudaStream_t st);
void emd_adj_rho(int n3, const double *rho, const double *lam_v, double *pois,
                 cudaStream_t st);
void emd_adj_scale_add(const OrbLayout &o, double2 *lam, const double2 *psi,
                       const double *w, double scale, cudaStream_t st);
void emd_adj_lincomb(int n, double *out, double a0, const double *x0, double a1,
                     const double *x1, double a2, const double *x2, double a3,
                     const double *x3, cudaStream_t st);
void emd_adj_force_splat(const GridInfo &g, const SpeciesDev &sp, const TableSet &t,
                         const double *lamF, double *w, cudaStream_t st);
void emd_adj_nl_force_orb(const OrbLayout &o, const GridInfo &g, const SpeciesDev &sp,
                          const TableSet &t, const double *lamF, const double2 *dc,
                          const double2 *cc, double coef, double2 *lam,
                          cudaStream_t st);
void emd_adj_nl_second_moment(const OrbLayout &o, const TableSet &t, int n_atoms,
                              const double2 *u, double h3, double inv_rc2,
                              const double *lamF, double2 *m, cudaStream_t st);
void emd_launch_local_force_hvp(const GridInfo &g, const SpeciesDev &sp,
                                int n_atoms, const TableSet &t,
                                const double *v_es_a, const double *v_es_b,
                                const double *lam, double *part, double *out,
                                cudaStream_t st);
void emd_adj_sr_hvp(const SpeciesDev &sp, int n_atoms, const double *Rw, double L,
                    const double *lamF, double *out, cudaStream_t st);
void emd_adj_nl_force_r(const double2 *cc, const double2 *dc, const double2 *m,
                        const double *lamF, int n_atoms, int n_orb, int n_orb_pad,
                        double coef, double *out, cudaStream_t st);
float emd_fp32_d2_margin(double L, double r);
void emd_launch_project_tile(const OrbLayout &o, const TableSet &t, int n_atoms,
                             const void *u, double h3, double h_kb, double2 *c,
                             void *hc, double2 *partial, cudaStream_t st);
void emd_launch_nl_force_tile(const OrbLayout &o, const TableSet &t, int n_atoms,
                              const void *u, const double2 *c, double h3, double coef,
                              double2 *partial, double *F_nl, cudaStream_t st);
// partial sums of Re(conj(a) b) over complex64 orbital arrays (double-float
// per point, FP64 across points)
void emd_launch_cdot_re_c64(const OrbLayout &o, const void *a, const void *b,
                            double *partials, int *nparts, cudaStream_t st);
