// The hot loop: one Taylor/Horner stage u_out = psi0 + (-i a) H u_in with
//   H = -1/2 nabla^2_FD + v_eff + sum_J h_kb |p_J><p_J|     (eq. new_EoM_a)
// on a periodic grid, plus the projections c_JA = <p_J|u_A>, the density
// rho = f sum_A |phi_A|^2 (eq. density), the kinetic energy of eq. E_KS and
// the nonlocal part of the Hellmann-Feynman force (eq. new_EoM_b).
//
// The degree-4 Taylor polynomial of exp(-i tau H) (Sec. 5.1) is evaluated in
// nested form: u4 = psi0 + (-i tau/4) H psi0, u_k = psi0 + (-i tau/k) H u_{k+1},
// k = 3, 2, 1, result u1.  Four stages per exponential, two exponentials per
// AETRS step (eq. aetrs).
//
// Orbital layout: [block][n^3][bo] complex, bo orbitals of a block interleaved
// per grid point, so one thread updates bo orbitals at one point and shares
// the potential, the projector list and the index arithmetic between them.
#include <algorithm>
#include <cstring>
#include <cuda.h>
#include <map>
#include <mutex>
#include <tuple>

#include "emd_internal.cuh"

namespace {

// Stencil weights passed by value (kernel parameter space): w_0 = -3 c_0/(2h^2),
// w_k = -c_k/(2h^2), so the kinetic term is w_0 u + sum_k w_k (6 neighbours).
template <typename T> struct Weights { T w[EMD_MAX_HALF_ORDER + 1]; };

template <typename T> Weights<T> weights_of(const OrbLayout &o) {
  Weights<T> r;
  for (int k = 0; k <= EMD_MAX_HALF_ORDER; ++k) r.w[k] = (T)o.w[k];
  return r;
}

template <typename T, int BO, int M>
__global__ void __launch_bounds__(128)
k_stage(const typename cplx<T>::type *__restrict__ u_in,
        const typename cplx<T>::type *__restrict__ psi0,
        typename cplx<T>::type *__restrict__ u_out, const T *__restrict__ v_eff,
        const int *__restrict__ pt_cnt, const int *__restrict__ pt_J,
        const double *__restrict__ pt_p,
        const typename cplx<T>::type *__restrict__ hc, int n, int ntx,
        int n_orb_pad, T a, int apply_only, Weights<T> W) {
  typedef typename cplx<T>::type V;
  const int x = (blockIdx.x % ntx) * 32 + threadIdx.x;
  const int y = (blockIdx.x / ntx) * 4 + threadIdx.y;
  const int z = blockIdx.y;
  const int blk = blockIdx.z;
  if (x >= n || y >= n) return;
  const size_t n3 = (size_t)n * n * n;
  const int p = (z * n + y) * n + x;
  const V *ub = u_in + (size_t)blk * n3 * BO;

  V c0[BO], acc[BO];
#pragma unroll
  for (int j = 0; j < BO; ++j) {
    c0[j] = ub[(size_t)p * BO + j];
    acc[j].x = W.w[0] * c0[j].x;
    acc[j].y = W.w[0] * c0[j].y;
  }
#pragma unroll
  for (int k = 1; k <= M; ++k) {
    int xp = x + k, xm = x - k, yp = y + k, ym = y - k, zp = z + k, zm = z - k;
    if (xp >= n) xp -= n;
    if (xm < 0) xm += n;
    if (yp >= n) yp -= n;
    if (ym < 0) ym += n;
    if (zp >= n) zp -= n;
    if (zm < 0) zm += n;
    const size_t row = (size_t)(z * n + y) * n;
    const size_t q[6] = {row + xp, row + xm, (size_t)(z * n + yp) * n + x,
                         (size_t)(z * n + ym) * n + x, (size_t)(zp * n + y) * n + x,
                         (size_t)(zm * n + y) * n + x};
    const T w = W.w[k];
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const V v0 = ub[q[0] * BO + j];
      T sx = v0.x, sy = v0.y;
#pragma unroll
      for (int e = 1; e < 6; ++e) {
        const V v = ub[q[e] * BO + j];
        sx += v.x;
        sy += v.y;
      }
      acc[j].x += w * sx;
      acc[j].y += w * sy;
    }
  }
  const T ve = v_eff[p];
#pragma unroll
  for (int j = 0; j < BO; ++j) {
    acc[j].x += ve * c0[j].x;
    acc[j].y += ve * c0[j].y;
  }
  const int cnt = pt_cnt[p];
  for (int e = 0; e < cnt; ++e) {
    const int J = pt_J[(size_t)e * n3 + p];
    const T pv = (T)pt_p[(size_t)e * n3 + p];
    const V *hcj = hc + (size_t)J * n_orb_pad + (size_t)blk * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const V c = hcj[j];
      acc[j].x += pv * c.x;
      acc[j].y += pv * c.y;
    }
  }
  V *ob = u_out + (size_t)blk * n3 * BO + (size_t)p * BO;
  if (apply_only) {
#pragma unroll
    for (int j = 0; j < BO; ++j) ob[j] = acc[j];
  } else {
    const V *pb = psi0 + (size_t)blk * n3 * BO + (size_t)p * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const V s = pb[j];
      V o;
      o.x = s.x + a * acc[j].y;
      o.y = s.y - a * acc[j].x;
      ob[j] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 Horner stage, 2.5-D: a CTA owns a tile of TX x TY points (all BO
// orbitals of a block) and marches through a chunk of z-planes.  Each input
// plane (tile + periodic halo of M points in x and y) is copied to shared
// memory with cp.async, double-buffered.  Every arriving plane z' contributes
//   - its x/y stencil part and v_eff u to output plane z',
//   - w_k u(z') to output planes z' - k and z' + k (k = 1..M),
// through a delay line of 2M+1 register accumulators per output point, so
// only one plane is ever resident in shared memory.  Plane z' completes output
// plane z' - M, which then gets the projector term and the Taylor update and
// is stored.  Each thread owns one orbital column (x, j) and RY consecutive
// rows, so y-neighbours come from a register window (RY + 2M loads for RY
// outputs) and x-neighbours from shared memory (2M loads per output).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int BO, int M> struct ZTile {
  static constexpr int NC = 64;                 // orbital columns = threads in x
  static constexpr int TX = NC / BO;            // points per tile in x
  static constexpr int NT = 512;                // threads per CTA
  static constexpr int TYT = NT / NC;           // thread rows
  static constexpr int RY = 2;                  // grid rows per thread
  static constexpr int TY = TYT * RY;           // grid rows per tile
  static constexpr int SW = TX + 2 * M;         // staged points per row
  static constexpr int SH = TY + 2 * M;         // staged rows
  static constexpr int PLANE = SH * SW * BO;    // float2 per staged u-plane
  static constexpr int CH = BO / 2;             // 16-byte chunks per point
  static constexpr int NCHUNK = SH * SW * CH;   // u chunks per plane
  static constexpr int CPT = (NCHUNK + NT - 1) / NT;
  static constexpr int NV = TX * TY;            // tile points
  static constexpr int QPT = (2 * NV + NT - 1) / NT;        // pt4 chunks / thread
  static constexpr int SPT = (NV * CH + NT - 1) / NT;       // psi0 chunks / thread
  static constexpr int NS = 2 * M + 1;          // delay-line slots
  static constexpr int NB = 3;                  // ring depth (prefetch 2)
  // one ring slot: u-plane | v_eff | projector records | psi0 of the output plane
  static constexpr int UB = PLANE * 8, VB = NV * 4, QB = NV * 32, SB = NV * BO * 8;
  static constexpr int SLOT = UB + VB + QB + SB;
  static constexpr size_t SMEM_FIXED = (size_t)NB * SLOT;
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem)
               : "memory");
}

// The complex arithmetic uses the packed FP32x2 operations of sm_10x
// (__fadd2_rn, __ffma2_rn, __fmul2_rn): one instruction per complex add or
// real-times-complex multiply-add.
template <int BO, int M>
__global__ void __launch_bounds__(512, 1)
k_stage_z(const float2 *__restrict__ u_in, const float2 *__restrict__ psi0,
          float2 *__restrict__ u_out, const float *__restrict__ v_eff,
          const int2 *__restrict__ pt4, const int *__restrict__ pt_J,
          const float *__restrict__ pt_pf, const float2 *__restrict__ hc,
          int n, int ntx, int zc, int n_orb_pad, int n_atoms, int hc_in_smem,
          float a, int apply_only, Weights<float> W) {
  typedef ZTile<BO, M> Z;
  constexpr int RY = Z::RY;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2 *hcs = reinterpret_cast<float2 *>(smraw + Z::NB * Z::SLOT);
  const int tid = threadIdx.x;
  const int col = tid % Z::NC, tyr = tid / Z::NC;
  const int xl = col / BO, j = col % BO;
  const int tx0 = (blockIdx.x % ntx) * Z::TX, ty0 = (blockIdx.x / ntx) * Z::TY;
  const int z0 = blockIdx.y * zc;
  const int zcount = min(zc, n - z0);
  const int total = zcount + 2 * M;
  const int blk = blockIdx.z;
  const int n2 = n * n;
  const size_t n3 = (size_t)n2 * n;
  const float2 *ub = u_in + (size_t)blk * n3 * BO;
  const float2 *pb = psi0 + (size_t)blk * n3 * BO;
  float2 *ob = u_out + (size_t)blk * n3 * BO;
  const int x = tx0 + xl;

  // staging offsets within a plane (the same for every plane)
  int src_off[Z::CPT], dst_off[Z::CPT];
#pragma unroll
  for (int i = 0; i < Z::CPT; ++i) {
    const int q = tid + i * Z::NT;
    src_off[i] = -1;
    dst_off[i] = 0;
    if (q < Z::NCHUNK) {
      const int hh = q % Z::CH, pnt = q / Z::CH;
      const int c = pnt % Z::SW, rr = pnt / Z::SW;
      const int xx = (tx0 - M + c + 2 * n) % n;
      const int yy = (ty0 - M + rr + 2 * n) % n;
      src_off[i] = (yy * n + xx) * BO + 2 * hh;
      dst_off[i] = (rr * Z::SW + c) * BO + 2 * hh;
    }
  }
  int v_src = -1;
  if (tid < Z::NV) {
    const int vx = tid % Z::TX, vy = tid / Z::TX;
    v_src = ((ty0 + vy) % n) * n + (tx0 + vx) % n;
  }
  int q_src[Z::QPT], q_dst[Z::QPT];
#pragma unroll
  for (int i = 0; i < Z::QPT; ++i) {
    const int q = tid + i * Z::NT;
    q_src[i] = -1;
    q_dst[i] = 0;
    if (q < 2 * Z::NV) {
      const int pnt = q >> 1, half = q & 1;
      const int xx = min(tx0 + pnt % Z::TX, n - 1), yy = min(ty0 + pnt / Z::TX, n - 1);
      q_src[i] = (yy * n + xx) * 4 + 2 * half;
      q_dst[i] = pnt * 4 + 2 * half;
    }
  }
  int s_src[Z::SPT], s_dst[Z::SPT];
#pragma unroll
  for (int i = 0; i < Z::SPT; ++i) {
    const int q = tid + i * Z::NT;
    s_src[i] = -1;
    s_dst[i] = 0;
    if (q < Z::NV * Z::CH) {
      const int pnt = q / Z::CH, hh = q % Z::CH;
      const int xx = min(tx0 + pnt % Z::TX, n - 1), yy = min(ty0 + pnt / Z::TX, n - 1);
      s_src[i] = (yy * n + xx) * BO + 2 * hh;
      s_dst[i] = pnt * BO + 2 * hh;
    }
  }
  if (hc_in_smem) {
    for (int i = tid; i < n_atoms * BO; i += Z::NT)
      hcs[i] = hc[(size_t)(i / BO) * n_orb_pad + (size_t)blk * BO + i % BO];
  }

  auto issue = [&](int zi, int slot) {
    unsigned char *base = smraw + slot * Z::SLOT;
    float2 *U = reinterpret_cast<float2 *>(base);
    float *V = reinterpret_cast<float *>(base + Z::UB);
    int2 *Q = reinterpret_cast<int2 *>(base + Z::UB + Z::VB);
    float2 *S = reinterpret_cast<float2 *>(base + Z::UB + Z::VB + Z::QB);
    int zz = z0 - M + zi;
    if (zz < 0) zz += n;
    if (zz >= n) zz -= n;
    const float2 *src = ub + (size_t)zz * n2 * BO;
#pragma unroll
    for (int i = 0; i < Z::CPT; ++i)
      if (src_off[i] >= 0) cp_async16(U + dst_off[i], src + src_off[i]);
    if (v_src >= 0) cp_async4(V + tid, v_eff + (size_t)zz * n2 + v_src);
    if (zi >= 2 * M) {
      const int zo = z0 + zi - 2 * M;
      const int2 *qs = pt4 + (size_t)zo * n2 * 4;
#pragma unroll
      for (int i = 0; i < Z::QPT; ++i)
        if (q_src[i] >= 0) cp_async16(Q + q_dst[i], qs + q_src[i]);
      if (!apply_only) {
        const float2 *ss = pb + (size_t)zo * n2 * BO;
#pragma unroll
        for (int i = 0; i < Z::SPT; ++i)
          if (s_src[i] >= 0) cp_async16(S + s_dst[i], ss + s_src[i]);
      }
    }
    cp_async_commit();
  };

  float2 w2[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) w2[k] = make_float2(W.w[k], W.w[k]);
  const float2 a2 = make_float2(a, -a);

  float2 acc[RY][Z::NS];
#pragma unroll
  for (int r = 0; r < RY; ++r)
#pragma unroll
    for (int q = 0; q < Z::NS; ++q) acc[r][q] = make_float2(0.f, 0.f);

  issue(0, 0);
  if (total > 1) issue(1, 1);
  int sb = 0;   // ring slot of plane zi
  for (int g = 0; g * Z::NS < total; ++g) {
#pragma unroll
    for (int ph = 0; ph < Z::NS; ++ph) {
      const int zi = g * Z::NS + ph;
      if (zi >= total) break;
      if (zi + 2 < total) {
        issue(zi + 2, sb == 0 ? 2 : sb - 1);
        cp_async_wait<2>();
      } else if (zi + 1 < total) {
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const unsigned char *base = smraw + sb * Z::SLOT;
      const float2 *P = reinterpret_cast<const float2 *>(base);
      const float *VP = reinterpret_cast<const float *>(base + Z::UB);
      float2 win[RY + 2 * M];
#pragma unroll
      for (int w = 0; w < RY + 2 * M; ++w)
        win[w] = P[((tyr * RY + w) * Z::SW + xl + M) * BO + j];
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const float2 c = win[r + M];
        const float2 *row = P + ((tyr * RY + r + M) * Z::SW + xl + M) * BO + j;
        float2 s2 = __fmul2_rn(w2[0], c);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
          const float2 t = __fadd2_rn(__fadd2_rn(row[k * BO], row[-k * BO]),
                                      __fadd2_rn(win[r + M + k], win[r + M - k]));
          s2 = __ffma2_rn(w2[k], t, s2);
        }
        const float ve = VP[(tyr * RY + r) * Z::TX + xl];
        s2 = __ffma2_rn(make_float2(ve, ve), c, s2);
        acc[r][ph] = __fadd2_rn(acc[r][ph], s2);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
          acc[r][(ph + k) % Z::NS] = __ffma2_rn(w2[k], c, acc[r][(ph + k) % Z::NS]);
          if (g > 0 || ph - k >= 0)
            acc[r][(ph - k + Z::NS) % Z::NS] =
                __ffma2_rn(w2[k], c, acc[r][(ph - k + Z::NS) % Z::NS]);
        }
      }
      if (zi >= M) {
        const int slot = (ph - M + Z::NS) % Z::NS;
        if (zi >= 2 * M) {
          const int zo = z0 + zi - 2 * M;
          const int4 *Q4 = reinterpret_cast<const int4 *>(base + Z::UB + Z::VB);
          const float2 *S = reinterpret_cast<const float2 *>(base + Z::UB + Z::VB + Z::QB);
#pragma unroll
          for (int r = 0; r < RY; ++r) {
            const int vy = tyr * RY + r, y = ty0 + vy;
            if (x < n && y < n) {
              const int pnt = vy * Z::TX + xl;
              const int4 q01 = Q4[2 * pnt], q23 = Q4[2 * pnt + 1];
              const int cnt = q01.x >> 16;
              const int J[4] = {q01.x & 0xffff, q01.z, q23.x, q23.z};
              const float pv[4] = {__int_as_float(q01.y), __int_as_float(q01.w),
                                   __int_as_float(q23.y), __int_as_float(q23.w)};
              float2 hv = acc[r][slot];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 hcv = hc_in_smem
                    ? hcs[J[e] * BO + j]
                    : __ldg(hc + (size_t)J[e] * n_orb_pad + (size_t)blk * BO + j);
                hv = __ffma2_rn(make_float2(pv[e], pv[e]), hcv, hv);
              }
              const size_t p = (size_t)zo * n2 + (size_t)y * n + x;
              for (int e = 4; e < cnt; ++e) {
                const int Je = __ldg(pt_J + (size_t)e * n3 + p);
                const float pe = __ldg(pt_pf + (size_t)e * n3 + p);
                const float2 hcv = hc_in_smem
                    ? hcs[Je * BO + j]
                    : __ldg(hc + (size_t)Je * n_orb_pad + (size_t)blk * BO + j);
                hv = __ffma2_rn(make_float2(pe, pe), hcv, hv);
              }
              float2 out = hv;
              if (!apply_only)
                out = __ffma2_rn(a2, make_float2(hv.y, hv.x), S[pnt * BO + j]);
              ob[p * BO + j] = out;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
#pragma unroll
          for (int q = 0; q < Z::NS; ++q)
            if (q == slot) acc[r][q] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      sb = sb == 2 ? 0 : sb + 1;
    }
  }
}

// ---------------------------------------------------------------------------
// Lean column kernel: the tile, ring and delay line of k_stage_z, arranged so
// that the per-update work is the arithmetic itself.  The ring depth (3)
// divides the delay-line length (2M+1 = 9 for M = 4, 7 for M = 3 ...) only
// for M = 1 and M = 4, so the group of planes unrolled at once is lcm-sized:
// the ring slot of every plane is a compile-time constant.  Weight pairs are
// kernel parameters, the shared-memory hc path is a template flag, output
// and staging addresses are per-thread constants plus one plane offset, and
// the centre term starts from the delay-line accumulator.
// ---------------------------------------------------------------------------
template <typename T> struct WPairs { float2 w[EMD_MAX_HALF_ORDER + 1]; };
inline WPairs<float> wpairs_of(const OrbLayout &o) {
  WPairs<float> r;
  for (int k = 0; k <= EMD_MAX_HALF_ORDER; ++k) r.w[k] = make_float2((float)o.w[k], (float)o.w[k]);
  return r;
}

// ---- tensor copies (TMA) completing on an mbarrier -------------------------
__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(addr), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}\n"
               : "=r"(ok)
               : "r"(addr), "r"(parity)
               : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier; gives up after 2^31 SM cycles
// (about a second at 2 GHz) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned addr, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(addr, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *tm, int c0, int c1,
                                            int c2, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}

template <int M> struct LeanGroup {
  // planes unrolled per group: a multiple of both the ring depth 3 and 2M+1
  static constexpr int NS = 2 * M + 1;
  static constexpr int G = NS % 3 == 0 ? NS : 3 * NS;
};

// Lean kernel's tile: as ZTile, with the diagonal d = w_0 + v_eff staged as
// (d, d, d, d) per point (16 bytes) instead of v_eff (4 bytes).
template <int BO, int M> struct ZCTile : ZTile<BO, M> {
  typedef ZTile<BO, M> B;
  static constexpr int VB = B::NV * 16;
  static constexpr int SLOT = B::UB + VB + B::QB + B::SB;
  static constexpr size_t SMEM_FIXED = (size_t)B::NB * SLOT;
};

// TMA (bo = 4): the diagonal, the projector records and psi0 of a plane,
// which never wrap around the grid, arrive as three tensor copies issued by
// one thread and completing on the ring slot's mbarrier; the orbital plane
// with its periodic halo keeps the per-thread cp.async chunks.
template <int BO, int M, bool HCS, bool TMA>
__global__ void __launch_bounds__(512, 1)
k_stage_c(const float2 *__restrict__ u_in, const float2 *__restrict__ psi0,
          float2 *__restrict__ u_out, const float4 *__restrict__ diag,
          const int2 *__restrict__ pt4, const int *__restrict__ pt_J,
          const float *__restrict__ pt_pf, const float2 *__restrict__ hc,
          int n, int ntx, int zc, int n_orb_pad, int n_atoms, float a,
          int apply_only, WPairs<float> W, const __grid_constant__ CUtensorMap tm_diag,
          const __grid_constant__ CUtensorMap tm_pt4, const __grid_constant__ CUtensorMap tm_psi,
          int *err) {
  static_assert(!TMA || BO == 4, "tensor copies are laid out for bo = 4");
  typedef ZCTile<BO, M> Z;
  constexpr int RY = Z::RY;
  constexpr int NS = Z::NS;
  constexpr int G = LeanGroup<M>::G;
  extern __shared__ __align__(128) unsigned char smdyn[];
  // tensor copies land on 128-byte boundaries: align the ring (the launch
  // reserves 128 bytes of slack)
  unsigned char *smraw =
      smdyn + ((128u - ((unsigned)__cvta_generic_to_shared(smdyn) & 127u)) & 127u);
  float2 *hcs = reinterpret_cast<float2 *>(smraw + Z::NB * Z::SLOT);
  const int tid = threadIdx.x;
  const int col = tid % Z::NC, tyr = tid / Z::NC;
  const int xl = col / BO, j = col % BO;
  const int tx0 = (blockIdx.x % ntx) * Z::TX, ty0 = (blockIdx.x / ntx) * Z::TY;
  const int z0 = blockIdx.y * zc;
  const int zcount = min(zc, n - z0);
  const int total = zcount + 2 * M;
  const int n2 = n * n;
  const size_t n3 = (size_t)n2 * n;
  const size_t boff = (size_t)blockIdx.z * n3 * BO;
  const float2 *ub = u_in + boff;
  const float2 *pb = psi0 + boff;
  float2 *ob = u_out + boff;
  const int x = tx0 + xl;

  // staging: per-thread (global element offset within a plane, shared byte
  // offset within a ring slot); -1 = nothing to copy
  int src_off[Z::CPT];
  unsigned dst_b[Z::CPT];
#pragma unroll
  for (int i = 0; i < Z::CPT; ++i) {
    const int q = tid + i * Z::NT;
    src_off[i] = -1;
    dst_b[i] = 0;
    if (q < Z::NCHUNK) {
      const int hh = q % Z::CH, pnt = q / Z::CH;
      const int c = pnt % Z::SW, rr = pnt / Z::SW;
      const int xx = (tx0 - M + c + 2 * n) % n;
      const int yy = (ty0 - M + rr + 2 * n) % n;
      src_off[i] = (yy * n + xx) * BO + 2 * hh;
      dst_b[i] = ((rr * Z::SW + c) * BO + 2 * hh) * 8;
    }
  }
  int v_src = -1, s_src = -1, q_src[Z::QPT];
  unsigned s_dst = 0, q_dst[Z::QPT];
  if (tid < Z::NV) {
    const int vx = tid % Z::TX, vy = tid / Z::TX;
    v_src = ((ty0 + vy) % n) * n + (tx0 + vx) % n;
  }
  static_assert(Z::SPT <= 1, "one psi0 chunk per thread");
#pragma unroll
  for (int i = 0; i < Z::QPT; ++i) {
    const int q = tid + i * Z::NT;
    q_src[i] = -1;
    q_dst[i] = 0;
    if (q < 2 * Z::NV) {
      const int pnt = q >> 1, half = q & 1;
      const int xx = min(tx0 + pnt % Z::TX, n - 1), yy = min(ty0 + pnt / Z::TX, n - 1);
      q_src[i] = (yy * n + xx) * 4 + 2 * half;
      q_dst[i] = (pnt * 4 + 2 * half) * 8;
    }
  }
  if (tid < Z::NV * Z::CH) {
    const int pnt = tid / Z::CH, hh = tid % Z::CH;
    const int xx = min(tx0 + pnt % Z::TX, n - 1), yy = min(ty0 + pnt / Z::TX, n - 1);
    s_src = (yy * n + xx) * BO + 2 * hh;
    s_dst = (pnt * BO + 2 * hh) * 8;
  }
  if (HCS) {
    for (int i = tid; i < n_atoms * BO; i += Z::NT)
      hcs[i] = hc[(size_t)(i / BO) * n_orb_pad + (size_t)blockIdx.z * BO + i % BO];
  }
  const unsigned sm0 = (unsigned)__cvta_generic_to_shared(smraw);
  // one mbarrier per ring slot (after the h_kb c copy, 8-byte aligned)
  const unsigned mb0 = (sm0 + Z::NB * Z::SLOT + (HCS ? n_atoms * BO * 8 : 0) + 7u) & ~7u;
  bool timed_out = false;
  if (TMA) {
    if (tid == 0) {
      for (int k = 0; k < Z::NB; ++k) mbar_init(mb0 + 8 * k, 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
  }

  auto issue = [&](int zi, int slot) {
    const unsigned base = sm0 + slot * Z::SLOT;
    int zz = z0 - M + zi;
    zz += zz < 0 ? n : 0;
    zz -= zz >= n ? n : 0;
    const size_t poff = (size_t)zz * n2;
    const float2 *src = ub + poff * BO;
#pragma unroll
    for (int i = 0; i < Z::CPT; ++i)
      if (src_off[i] >= 0)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + dst_b[i]),
                     "l"(src + src_off[i]) : "memory");
    if (TMA) {
      if (tid == 0) {
        const bool out = zi >= 2 * M;
        const unsigned bytes = Z::NV * 16 + (out ? Z::NV * 32 + (apply_only ? 0 : Z::NV * 32) : 0);
        const unsigned mb = mb0 + 8 * slot;
        // the slot's previous contents were read through the generic proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_expect_tx(mb, bytes);
        tma_load_3d(base + Z::UB, &tm_diag, 0, tx0, zz * n + ty0, mb);
        if (out) {
          const int zo = z0 + zi - 2 * M;
          tma_load_3d(base + Z::UB + Z::VB, &tm_pt4, 0, tx0, zo * n + ty0, mb);
          if (!apply_only)
            tma_load_3d(base + Z::UB + Z::VB + Z::QB, &tm_psi, 0, tx0,
                        ((int)blockIdx.z * n + zo) * n + ty0, mb);
        }
      }
      cp_async_commit();
      return;
    }
    if (v_src >= 0)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + Z::UB + tid * 16),
                   "l"(diag + poff + v_src) : "memory");
    if (zi >= 2 * M) {
      const size_t zo = (size_t)(z0 + zi - 2 * M) * n2;
#pragma unroll
      for (int i = 0; i < Z::QPT; ++i)
        if (q_src[i] >= 0)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + Z::UB + Z::VB + q_dst[i]),
                       "l"(pt4 + zo * 4 + q_src[i]) : "memory");
      if (!apply_only && s_src >= 0)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + Z::UB + Z::VB + Z::QB + s_dst),
                     "l"(pb + zo * BO + s_src) : "memory");
    }
    cp_async_commit();
  };

  // per-thread output constants
  int orow[RY];
  bool oval[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int y = ty0 + tyr * RY + r;
    oval[r] = x < n && y < n;
    orow[r] = (y * n + x) * BO + j;
  }
  const int win0 = ((tyr * RY) * Z::SW + xl + M) * BO + j;     // float2 index
  const int pnt0 = (tyr * RY) * Z::TX + xl;

  float2 acc[RY][NS];
#pragma unroll
  for (int r = 0; r < RY; ++r)
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[r][q] = make_float2(0.f, 0.f);

  issue(0, 0);
  if (total > 1) issue(1, 1);
  for (int g = 0; g * G < total; ++g) {
#pragma unroll
    for (int ph = 0; ph < G; ++ph) {
      const int zi = g * G + ph;
      if (zi >= total) break;
      const int sb = ph % 3;
      const int dl = ph % NS;             // delay-line slot of this plane
      // planes zi (and zi + 1) are in flight: wait for zi, then one barrier
      // makes every thread's copies visible and proves that every thread has
      // finished plane zi - 1, whose ring slot the prefetch of zi + 2 reuses
      if (zi + 1 < total) cp_async_wait<1>();
      else cp_async_wait<0>();
      if (TMA && !mbar_wait_bounded(mb0 + 8 * sb, (unsigned)(zi / 3) & 1u)) timed_out = true;
      __syncthreads();
      if (zi + 2 < total) issue(zi + 2, (ph + 2) % 3);
      const unsigned char *base = smraw + sb * Z::SLOT;
      const float2 *P = reinterpret_cast<const float2 *>(base);
      const float2 *DP = reinterpret_cast<const float2 *>(base + Z::UB);   // (d, d) at 2 pnt
      float2 win[RY + 2 * M];
#pragma unroll
      for (int w = 0; w < RY + 2 * M; ++w) win[w] = P[win0 + w * Z::SW * BO];
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const float2 c = win[r + M];
        const float2 *row = P + win0 + (r + M) * Z::SW * BO;
        float2 s2 = __ffma2_rn(DP[2 * (pnt0 + r * Z::TX)], c, acc[r][dl]);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
          const float2 t = __fadd2_rn(__fadd2_rn(row[k * BO], row[-k * BO]),
                                      __fadd2_rn(win[r + M + k], win[r + M - k]));
          s2 = __ffma2_rn(W.w[k], t, s2);
        }
        acc[r][dl] = s2;
#pragma unroll
        for (int k = 1; k <= M; ++k) {
          acc[r][(ph + k) % NS] = __ffma2_rn(W.w[k], c, acc[r][(ph + k) % NS]);
          if (g > 0 || ph - k >= 0)
            acc[r][(ph - k + G) % NS] = __ffma2_rn(W.w[k], c, acc[r][(ph - k + G) % NS]);
        }
      }
      if (zi >= M) {
        const int slot = (ph - M + G) % NS;
        if (zi >= 2 * M) {
          const size_t zo = (size_t)(z0 + zi - 2 * M) * n2;
          const int4 *Q4 = reinterpret_cast<const int4 *>(base + Z::UB + Z::VB);
          const float2 *S = reinterpret_cast<const float2 *>(base + Z::UB + Z::VB + Z::QB);
          float2 *obz = ob + zo * BO;
#pragma unroll
          for (int r = 0; r < RY; ++r) {
            if (oval[r]) {
              const int pnt = pnt0 + r * Z::TX;
              const int4 q01 = Q4[2 * pnt], q23 = Q4[2 * pnt + 1];
              const int cnt = q01.x >> 16;
              const int J[4] = {q01.x & 0xffff, q01.z, q23.x, q23.z};
              const float pv[4] = {__int_as_float(q01.y), __int_as_float(q01.w),
                                   __int_as_float(q23.y), __int_as_float(q23.w)};
              float2 hv = acc[r][slot];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 hcv = HCS ? hcs[J[e] * BO + j]
                                       : __ldg(hc + (size_t)J[e] * n_orb_pad +
                                               (size_t)blockIdx.z * BO + j);
                hv = __ffma2_rn(make_float2(pv[e], pv[e]), hcv, hv);
              }
              if (cnt > 4) {
                const size_t p = zo + (size_t)(orow[r] - j) / BO;
                for (int e = 4; e < cnt; ++e) {
                  const int Je = __ldg(pt_J + (size_t)e * n3 + p);
                  const float pe = __ldg(pt_pf + (size_t)e * n3 + p);
                  const float2 hcv = HCS ? hcs[Je * BO + j]
                                         : __ldg(hc + (size_t)Je * n_orb_pad +
                                                 (size_t)blockIdx.z * BO + j);
                  hv = __ffma2_rn(make_float2(pe, pe), hcv, hv);
                }
              }
              float2 out = hv;
              if (!apply_only) {
                const float2 sv = S[pnt * BO + j];
                out.x = __fmaf_rn(a, hv.y, sv.x);
                out.y = __fmaf_rn(-a, hv.x, sv.y);
              }
              obz[orow[r]] = out;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) acc[r][slot] = make_float2(0.f, 0.f);
      }
    }
  }
  if (TMA && timed_out) {
    if (err) atomicOr(err, EMD_ERRBIT_WAIT);
    // copies of a slot that never completed may still be in flight: give
    // them one more bounded wait before the shared memory is released
    if (tid == 0)
      for (int k = 0; k < Z::NB && k < total; ++k) {
        const int last = k + 3 * ((total - 1 - k) / 3);   // last plane staged in slot k
        mbar_wait_bounded(mb0 + 8 * k, (unsigned)(last / 3) & 1u);
      }
  }
}

// ---------------------------------------------------------------------------
// Point-per-thread variant: each thread owns one grid point of a 32 x 16 tile
// and all bo orbitals of the block there, so the per-point work (staging
// offsets, v_eff, projector records, index arithmetic) is shared by the bo
// orbitals and shared memory is read 16 bytes at a time.  Same 3-deep ring
// and (2M+1)-slot delay line as k_stage_z.
// ---------------------------------------------------------------------------
template <int BO, int M, int RY> struct ZPTile {
  static constexpr int TX = 32;                      // points per tile row
  static constexpr int NT = RY == 1 ? 512 : 256;     // threads per CTA
  static constexpr int TYT = NT / TX;                // thread rows
  static constexpr int TY = TYT * RY;                // grid rows per tile
  static constexpr int SW = TX + 2 * M, SH = TY + 2 * M;
  static constexpr int PLANE = SH * SW * BO;
  static constexpr int CH = BO / 2;
  static constexpr int NCHUNK = SH * SW * CH;
  static constexpr int CPT = (NCHUNK + NT - 1) / NT;
  static constexpr int NV = TX * TY;
  static constexpr int VPT = (NV + NT - 1) / NT;             // v_eff values / thread
  static constexpr int QPT = (2 * NV + NT - 1) / NT;
  static constexpr int SPT = (NV * CH + NT - 1) / NT;
  static constexpr int NS = 2 * M + 1, NB = 3;
  static constexpr int UB = PLANE * 8, VB = NV * 4, QB = NV * 32, SB = NV * BO * 8;
  static constexpr int SLOT = UB + VB + QB + SB;
  static constexpr size_t SMEM_FIXED = (size_t)NB * SLOT;
};

template <int BO>
__device__ __forceinline__ void lds_point(const float2 *p, float2 (&v)[BO]) {
#pragma unroll
  for (int h = 0; h < BO / 2; ++h) {
    const float4 q = reinterpret_cast<const float4 *>(p)[h];
    v[2 * h] = make_float2(q.x, q.y);
    v[2 * h + 1] = make_float2(q.z, q.w);
  }
}

// Each thread owns the bo orbitals of one grid column over RY consecutive
// rows: y-neighbours come from a register window of RY + 2M points, x
// neighbours from shared memory, 16 bytes at a time.
template <int BO, int M, int RY>
__global__ void __launch_bounds__(ZPTile<BO, M, RY>::NT, 1)
k_stage_zp(const float2 *__restrict__ u_in, const float2 *__restrict__ psi0,
           float2 *__restrict__ u_out, const float *__restrict__ v_eff,
           const int2 *__restrict__ pt4, const int *__restrict__ pt_J,
           const float *__restrict__ pt_pf, const float2 *__restrict__ hc,
           int n, int ntx, int zc, int n_orb_pad, int n_atoms, int hc_in_smem,
           float a, int apply_only, Weights<float> W) {
  typedef ZPTile<BO, M, RY> Z;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2 *hcs = reinterpret_cast<float2 *>(smraw + Z::NB * Z::SLOT);
  const int tid = threadIdx.x;
  const int xl = tid % Z::TX, tyr = tid / Z::TX;
  const int tx0 = (blockIdx.x % ntx) * Z::TX, ty0 = (blockIdx.x / ntx) * Z::TY;
  const int x = tx0 + xl;
  const int z0 = blockIdx.y * zc;
  const int zcount = min(zc, n - z0);
  const int total = zcount + 2 * M;
  const int blk = blockIdx.z;
  const int n2 = n * n;
  const size_t n3 = (size_t)n2 * n;
  const float2 *ub = u_in + (size_t)blk * n3 * BO;
  const float2 *pb = psi0 + (size_t)blk * n3 * BO;
  float2 *ob = u_out + (size_t)blk * n3 * BO;

  int src_off[Z::CPT], dst_off[Z::CPT];
#pragma unroll
  for (int i = 0; i < Z::CPT; ++i) {
    const int q = tid + i * Z::NT;
    src_off[i] = -1;
    dst_off[i] = 0;
    if (q < Z::NCHUNK) {
      const int hh = q % Z::CH, pnt = q / Z::CH;
      const int c = pnt % Z::SW, rr = pnt / Z::SW;
      const int xx = (tx0 - M + c + 2 * n) % n;
      const int yy = (ty0 - M + rr + 2 * n) % n;
      src_off[i] = (yy * n + xx) * BO + 2 * hh;
      dst_off[i] = (rr * Z::SW + c) * BO + 2 * hh;
    }
  }
  int v_src[Z::VPT];
#pragma unroll
  for (int i = 0; i < Z::VPT; ++i) {
    const int q = tid + i * Z::NT;
    v_src[i] = -1;
    if (q < Z::NV) {
      const int vx = q % Z::TX, vy = q / Z::TX;
      v_src[i] = ((ty0 + vy) % n) * n + (tx0 + vx) % n;
    }
  }
  int q_src[Z::QPT], q_dst[Z::QPT];
#pragma unroll
  for (int i = 0; i < Z::QPT; ++i) {
    const int q = tid + i * Z::NT;
    q_src[i] = -1;
    q_dst[i] = 0;
    if (q < 2 * Z::NV) {
      const int pnt = q >> 1, half = q & 1;
      const int xx = min(tx0 + pnt % Z::TX, n - 1), yy = min(ty0 + pnt / Z::TX, n - 1);
      q_src[i] = (yy * n + xx) * 4 + 2 * half;
      q_dst[i] = pnt * 4 + 2 * half;
    }
  }
  int s_src[Z::SPT], s_dst[Z::SPT];
#pragma unroll
  for (int i = 0; i < Z::SPT; ++i) {
    const int q = tid + i * Z::NT;
    s_src[i] = -1;
    s_dst[i] = 0;
    if (q < Z::NV * Z::CH) {
      const int pnt = q / Z::CH, hh = q % Z::CH;
      const int xx = min(tx0 + pnt % Z::TX, n - 1), yy = min(ty0 + pnt / Z::TX, n - 1);
      s_src[i] = (yy * n + xx) * BO + 2 * hh;
      s_dst[i] = pnt * BO + 2 * hh;
    }
  }
  if (hc_in_smem) {
    for (int i = tid; i < n_atoms * BO; i += Z::NT)
      hcs[i] = hc[(size_t)(i / BO) * n_orb_pad + (size_t)blk * BO + i % BO];
  }

  auto issue = [&](int zi, int slot) {
    unsigned char *base = smraw + slot * Z::SLOT;
    float2 *U = reinterpret_cast<float2 *>(base);
    float *V = reinterpret_cast<float *>(base + Z::UB);
    int2 *Q = reinterpret_cast<int2 *>(base + Z::UB + Z::VB);
    float2 *S = reinterpret_cast<float2 *>(base + Z::UB + Z::VB + Z::QB);
    int zz = z0 - M + zi;
    if (zz < 0) zz += n;
    if (zz >= n) zz -= n;
    const float2 *src = ub + (size_t)zz * n2 * BO;
#pragma unroll
    for (int i = 0; i < Z::CPT; ++i)
      if (src_off[i] >= 0) cp_async16(U + dst_off[i], src + src_off[i]);
    const float *vsrc = v_eff + (size_t)zz * n2;
#pragma unroll
    for (int i = 0; i < Z::VPT; ++i)
      if (v_src[i] >= 0) cp_async4(V + tid + i * Z::NT, vsrc + v_src[i]);
    if (zi >= 2 * M) {
      const int zo = z0 + zi - 2 * M;
      const int2 *qs = pt4 + (size_t)zo * n2 * 4;
#pragma unroll
      for (int i = 0; i < Z::QPT; ++i)
        if (q_src[i] >= 0) cp_async16(Q + q_dst[i], qs + q_src[i]);
      if (!apply_only) {
        const float2 *ss = pb + (size_t)zo * n2 * BO;
#pragma unroll
        for (int i = 0; i < Z::SPT; ++i)
          if (s_src[i] >= 0) cp_async16(S + s_dst[i], ss + s_src[i]);
      }
    }
    cp_async_commit();
  };

  float2 w2[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) w2[k] = make_float2(W.w[k], W.w[k]);
  const float2 a2 = make_float2(a, -a);

  float2 acc[RY][BO][Z::NS];
#pragma unroll
  for (int r = 0; r < RY; ++r)
#pragma unroll
    for (int j = 0; j < BO; ++j)
#pragma unroll
      for (int q = 0; q < Z::NS; ++q) acc[r][j][q] = make_float2(0.f, 0.f);

  const int cidx = ((tyr * RY + M) * Z::SW + xl + M) * BO;   // own row 0
  issue(0, 0);
  if (total > 1) issue(1, 1);
  int sb = 0;
  for (int g = 0; g * Z::NS < total; ++g) {
#pragma unroll
    for (int ph = 0; ph < Z::NS; ++ph) {
      const int zi = g * Z::NS + ph;
      if (zi >= total) break;
      if (zi + 2 < total) {
        issue(zi + 2, sb == 0 ? 2 : sb - 1);
        cp_async_wait<2>();
      } else if (zi + 1 < total) {
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const unsigned char *base = smraw + sb * Z::SLOT;
      const float2 *P = reinterpret_cast<const float2 *>(base) + cidx;
      const float *VP = reinterpret_cast<const float *>(base + Z::UB);
      float2 win[RY + 2 * M][BO];
#pragma unroll
      for (int w = 0; w < RY + 2 * M; ++w) lds_point<BO>(P + (w - M) * Z::SW * BO, win[w]);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const float2 *Pr = P + r * Z::SW * BO;
        float2 s2[BO];
#pragma unroll
        for (int j = 0; j < BO; ++j) s2[j] = __fmul2_rn(w2[0], win[r + M][j]);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
#pragma unroll
          for (int h = 0; h < BO / 2; ++h) {
            const float4 xp = reinterpret_cast<const float4 *>(Pr + k * BO)[h];
            const float4 xm = reinterpret_cast<const float4 *>(Pr - k * BO)[h];
            const float2 t0 = __fadd2_rn(__fadd2_rn(make_float2(xp.x, xp.y), make_float2(xm.x, xm.y)),
                                         __fadd2_rn(win[r + M + k][2 * h], win[r + M - k][2 * h]));
            const float2 t1 = __fadd2_rn(__fadd2_rn(make_float2(xp.z, xp.w), make_float2(xm.z, xm.w)),
                                         __fadd2_rn(win[r + M + k][2 * h + 1], win[r + M - k][2 * h + 1]));
            s2[2 * h] = __ffma2_rn(w2[k], t0, s2[2 * h]);
            s2[2 * h + 1] = __ffma2_rn(w2[k], t1, s2[2 * h + 1]);
          }
        }
        const float ve = VP[(tyr * RY + r) * Z::TX + xl];
        const float2 ve2 = make_float2(ve, ve);
#pragma unroll
        for (int j = 0; j < BO; ++j) {
          const float2 c = win[r + M][j];
          s2[j] = __ffma2_rn(ve2, c, s2[j]);
          acc[r][j][ph] = __fadd2_rn(acc[r][j][ph], s2[j]);
#pragma unroll
          for (int k = 1; k <= M; ++k) {
            acc[r][j][(ph + k) % Z::NS] = __ffma2_rn(w2[k], c, acc[r][j][(ph + k) % Z::NS]);
            if (g > 0 || ph - k >= 0)
              acc[r][j][(ph - k + Z::NS) % Z::NS] =
                  __ffma2_rn(w2[k], c, acc[r][j][(ph - k + Z::NS) % Z::NS]);
          }
        }
      }
      if (zi >= M) {
        const int slot = (ph - M + Z::NS) % Z::NS;
        if (zi >= 2 * M) {
          const int zo = z0 + zi - 2 * M;
          const int4 *Q4 = reinterpret_cast<const int4 *>(base + Z::UB + Z::VB);
          const float2 *Sb = reinterpret_cast<const float2 *>(base + Z::UB + Z::VB + Z::QB);
#pragma unroll
          for (int r = 0; r < RY; ++r) {
            const int vy = tyr * RY + r, y = ty0 + vy;
            if (x < n && y < n) {
              const int pnt = vy * Z::TX + xl;
              const int4 q01 = Q4[2 * pnt], q23 = Q4[2 * pnt + 1];
              const int cnt = q01.x >> 16;
              const int J[4] = {q01.x & 0xffff, q01.z, q23.x, q23.z};
              const float pv[4] = {__int_as_float(q01.y), __int_as_float(q01.w),
                                   __int_as_float(q23.y), __int_as_float(q23.w)};
              float2 hv[BO];
#pragma unroll
              for (int j = 0; j < BO; ++j) hv[j] = acc[r][j][slot];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                float2 hcv[BO];
                if (hc_in_smem) {
                  lds_point<BO>(hcs + J[e] * BO, hcv);
                } else {
#pragma unroll
                  for (int j = 0; j < BO; ++j)
                    hcv[j] = __ldg(hc + (size_t)J[e] * n_orb_pad + (size_t)blk * BO + j);
                }
                const float2 p2 = make_float2(pv[e], pv[e]);
#pragma unroll
                for (int j = 0; j < BO; ++j) hv[j] = __ffma2_rn(p2, hcv[j], hv[j]);
              }
              const size_t p = (size_t)zo * n2 + (size_t)y * n + x;
              for (int e = 4; e < cnt; ++e) {
                const int Je = __ldg(pt_J + (size_t)e * n3 + p);
                const float pe = __ldg(pt_pf + (size_t)e * n3 + p);
                const float2 p2 = make_float2(pe, pe);
#pragma unroll
                for (int j = 0; j < BO; ++j) {
                  const float2 hcv = hc_in_smem ? hcs[Je * BO + j]
                      : __ldg(hc + (size_t)Je * n_orb_pad + (size_t)blk * BO + j);
                  hv[j] = __ffma2_rn(p2, hcv, hv[j]);
                }
              }
              float2 out[BO];
              if (apply_only) {
#pragma unroll
                for (int j = 0; j < BO; ++j) out[j] = hv[j];
              } else {
                float2 s0[BO];
                lds_point<BO>(Sb + pnt * BO, s0);
#pragma unroll
                for (int j = 0; j < BO; ++j)
                  out[j] = __ffma2_rn(a2, make_float2(hv[j].y, hv[j].x), s0[j]);
              }
              float4 *dst = reinterpret_cast<float4 *>(ob + p * BO);
#pragma unroll
              for (int h = 0; h < BO / 2; ++h)
                dst[h] = make_float4(out[2 * h].x, out[2 * h].y, out[2 * h + 1].x, out[2 * h + 1].y);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
          for (int j = 0; j < BO; ++j)
#pragma unroll
            for (int q = 0; q < Z::NS; ++q)
              if (q == slot) acc[r][j][q] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      sb = sb == 2 ? 0 : sb + 1;
    }
  }
}

// c[J][A] = h^3 sum_e p_e u_A(pt_e) over atom J's (point, image) entries;
// hc = h_kb c in orbital precision.  One block per (atom, orbital block).
// Each thread accumulates its strided share of the entries in T (FP32 for
// complex64 orbitals: GB300's FP64 rate is 1/64 of FP32), the block sum
// across threads is FP64 in a fixed tree order.
template <typename T, int BO>
__global__ void __launch_bounds__(256)
k_project(const typename cplx<T>::type *__restrict__ u, size_t n3,
          const int *__restrict__ at_cnt, const int *__restrict__ at_pt,
          const double *__restrict__ at_p, int cap, double h3, double h_kb,
          int n_orb_pad, double2 *c, typename cplx<T>::type *hc) {
  typedef typename cplx<T>::type V;
  __shared__ double red[8 * 2 * BO];
  const int J = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[J];
  const V *ub = u + (size_t)blk * n3 * BO;
  T tacc[2 * BO];
#pragma unroll
  for (int k = 0; k < 2 * BO; ++k) tacc[k] = 0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const size_t idx = (size_t)J * cap + e;
    const int pt = at_pt[idx];
    const T pv = (T)at_p[idx];
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const V v = ub[(size_t)pt * BO + j];
      tacc[2 * j] += pv * v.x;
      tacc[2 * j + 1] += pv * v.y;
    }
  }
  double acc[2 * BO];
#pragma unroll
  for (int k = 0; k < 2 * BO; ++k) acc[k] = (double)tacc[k];
  emd_block_sum<2 * BO>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const size_t o = (size_t)J * n_orb_pad + (size_t)blk * BO + j;
      const double re = h3 * acc[2 * j], im = h3 * acc[2 * j + 1];
      c[o] = make_double2(re, im);
      V w;
      w.x = (T)(h_kb * re);
      w.y = (T)(h_kb * im);
      hc[o] = w;
    }
  }
}

// partial[b] = sum over the points of block b and all orbitals of
// Re(conj(a) b) for complex64 arrays: per point in double-float arithmetic
// (exact FP32 products, TwoSum accumulation, as the density), converted to
// FP64 once per point, then a fixed-tree FP64 block sum.
template <int BO>
__global__ void __launch_bounds__(256)
k_cdot_re_c64(const float2 *__restrict__ a, const float2 *__restrict__ b, size_t n3,
              int n_blk, double *part) {
  __shared__ double red[8];
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (p < n3) {
    float hi = 0.f, lo = 0.f;
    for (int k = 0; k < n_blk; ++k) {
      const size_t o = ((size_t)k * n3 + p) * BO;
#pragma unroll
      for (int j = 0; j < BO; ++j) {
        const float2 x = a[o + j], y = b[o + j];
        const float px = __fmul_rn(x.x, y.x), py = __fmul_rn(x.y, y.y);
        lo = __fadd_rn(lo, __fadd_rn(__fmaf_rn(x.x, y.x, -px), __fmaf_rn(x.y, y.y, -py)));
        float t = px;
        float s2 = __fadd_rn(hi, t), bb = __fsub_rn(s2, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s2, bb)), __fsub_rn(t, bb)));
        hi = s2;
        t = py;
        s2 = __fadd_rn(hi, t);
        bb = __fsub_rn(s2, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s2, bb)), __fsub_rn(t, bb)));
        hi = s2;
      }
    }
    acc[0] = (double)hi + (double)lo;
  }
  emd_block_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

template <typename T, int BO>
__global__ void k_density(const typename cplx<T>::type *__restrict__ u,
                          size_t n3, int n_blk, double occ, double *rho) {
  typedef typename cplx<T>::type V;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n3) return;
  double acc = 0.0;
  for (int b = 0; b < n_blk; ++b) {
    const V *ub = u + ((size_t)b * n3 + p) * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const double re = (double)ub[j].x, im = (double)ub[j].y;
      acc += re * re + im * im;
    }
  }
  rho[p] = occ * acc;
}

// complex64 orbitals: sum |u|^2 in double-float arithmetic on the FP32
// pipes.  Each square is split exactly into p + e (e = fma(v, v, -p)); the
// running sum is a (hi, lo) pair updated with Knuth's TwoSum, and converted to
// FP64 once per point (~1e-13 relative, without FP64 instructions per term).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float t) {
  // rounded-to-nearest intrinsics: never contracted into FMAs
  const float s = __fadd_rn(hi, t);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb)));
  hi = s;
}

template <int BO>
__global__ void k_density_c64(const float2 *__restrict__ u, size_t n3, int n_blk,
                              double occ, double *rho) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n3) return;
  float hi = 0.f, lo = 0.f;
  for (int b = 0; b < n_blk; ++b) {
    const float2 *ub = u + ((size_t)b * n3 + p) * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const float2 v = ub[j];
      const float px = __fmul_rn(v.x, v.x), py = __fmul_rn(v.y, v.y);
      lo = __fadd_rn(lo, __fadd_rn(__fmaf_rn(v.x, v.x, -px), __fmaf_rn(v.y, v.y, -py)));
      two_sum_acc(hi, lo, px);
      two_sum_acc(hi, lo, py);
    }
  }
  rho[p] = occ * ((double)hi + (double)lo);
}

// complex128 orbitals: sum |u|^2 in double-float arithmetic on the FP32
// pipes (an FP64 multiply-add per component would bound the kernel by
// GB300's FP64 rate).  Each component splits into hi + lo (48 bits); its
// square is hi^2 (TwoProduct: p + e exactly) + 2 hi lo, the lo^2 term lying
// below 2^-47 of the square; the real and imaginary squares accumulate as
// packed (hi, lo) pairs with TwoSum and are widened and added once per point
// (relative error ~1e-14).
template <int BO>
__global__ void k_density_df(const double2 *__restrict__ u, size_t n3, int n_blk, double occ,
                             double *rho) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n3) return;
  float2 ah = make_float2(0.f, 0.f), al = ah;
#pragma unroll 4
  for (int b = 0; b < n_blk; ++b) {
    const double2 *ub = u + ((size_t)b * n3 + p) * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const float4 v = df_split2(ub[j]);
      const float2 h = f4hi(v), l = f4lo(v);
      float2 sq, e;
      dfp_two_prod(h, h, sq, e);
      dfp_add(ah, al, sq, __ffma2_rn(__fadd2_rn(h, h), l, e));
    }
  }
  const double re = __dadd_rn(df_widen(ah.x), df_widen(al.x));
  const double im = __dadd_rn(df_widen(ah.y), df_widen(al.y));
  rho[p] = occ * (re + im);
}

// partial[b] = sum over the points of block b and all orbitals of
// Re(conj(u) (-1/2 nabla^2_FD u)), FP64.
template <typename T, int BO, int M>
__global__ void __launch_bounds__(256)
k_kinetic(const typename cplx<T>::type *__restrict__ u, int n, int n_blk,
          double *part, Weights<double> W) {
  typedef typename cplx<T>::type V;
  __shared__ double red[8];
  const size_t n3 = (size_t)n * n * n;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (p < n3) {
    const int x = p % n, y = (p / n) % n, z = p / ((size_t)n * n);
    for (int b = 0; b < n_blk; ++b) {
      const V *ub = u + (size_t)b * n3 * BO;
      for (int j = 0; j < BO; ++j) {
        const V c0 = ub[p * BO + j];
        double lx = W.w[0] * (double)c0.x, ly = W.w[0] * (double)c0.y;
        for (int k = 1; k <= M; ++k) {
          const int xp = (x + k) % n, xm = (x - k + n) % n;
          const int yp = (y + k) % n, ym = (y - k + n) % n;
          const int zp = (z + k) % n, zm = (z - k + n) % n;
          const size_t q[6] = {(size_t)(z * n + y) * n + xp, (size_t)(z * n + y) * n + xm,
                               (size_t)(z * n + yp) * n + x, (size_t)(z * n + ym) * n + x,
                               (size_t)(zp * n + y) * n + x, (size_t)(zm * n + y) * n + x};
          double sx = 0, sy = 0;
          for (int e = 0; e < 6; ++e) {
            const V v = ub[q[e] * BO + j];
            sx += (double)v.x;
            sy += (double)v.y;
          }
          lx += W.w[k] * sx;
          ly += W.w[k] * sy;
        }
        acc[0] += (double)c0.x * lx + (double)c0.y * ly;
      }
    }
  }
  emd_block_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

// Nonlocal force partials: for atom J and orbital block blk,
// part[J][blk][a] = coef * sum_j Re(conj(c_JA) dc_JA,a),
// dc_JA,a = h^3 sum_e p_e d_e,a / r_c^2 u_A(pt_e)  (= d c_JA / d R_J,a).
template <typename T, int BO>
__global__ void __launch_bounds__(256)
k_nl_force(const typename cplx<T>::type *__restrict__ u, size_t n3, int n_blk,
           const int *__restrict__ at_cnt, const int *__restrict__ at_pt,
           const double *__restrict__ at_p, const double *__restrict__ at_d,
           int cap, const double2 *__restrict__ c, int n_orb_pad, int n_orb,
           double h3, double coef, double inv_rc2, double *part) {
  typedef typename cplx<T>::type V;
  __shared__ double red[8 * 6 * BO];
  const int J = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[J];
  const V *ub = u + (size_t)blk * n3 * BO;
  T tacc[6 * BO];
#pragma unroll
  for (int k = 0; k < 6 * BO; ++k) tacc[k] = 0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const size_t idx = (size_t)J * cap + e;
    const int pt = at_pt[idx];
    const T pv = (T)(at_p[idx] * inv_rc2);
    const T d0 = (T)at_d[3 * idx], d1 = (T)at_d[3 * idx + 1], d2 = (T)at_d[3 * idx + 2];
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const V v = ub[(size_t)pt * BO + j];
      const T wr = pv * v.x, wi = pv * v.y;
      tacc[6 * j + 0] += wr * d0;
      tacc[6 * j + 1] += wi * d0;
      tacc[6 * j + 2] += wr * d1;
      tacc[6 * j + 3] += wi * d1;
      tacc[6 * j + 4] += wr * d2;
      tacc[6 * j + 5] += wi * d2;
    }
  }
  double acc[6 * BO];
#pragma unroll
  for (int k = 0; k < 6 * BO; ++k) acc[k] = (double)tacc[k];
  emd_block_sum<6 * BO>(acc, red);
  if (threadIdx.x == 0) {
    double f[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < BO; ++j) {
      const int A = blk * BO + j;
      if (A >= n_orb) continue;
      const double2 cj = c[(size_t)J * n_orb_pad + A];
      for (int a = 0; a < 3; ++a) {
        const double dr = h3 * acc[6 * j + 2 * a], di = h3 * acc[6 * j + 2 * a + 1];
        f[a] += cj.x * dr + cj.y * di;   // Re(conj(c) dc)
      }
    }
    for (int a = 0; a < 3; ++a)
      part[((size_t)J * n_blk + blk) * 3 + a] = coef * f[a];
  }
}

__global__ void k_nl_force_sum(const double *part, int n_atoms, int n_blk,
                               double *F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n_atoms) return;
  const int J = i / 3, a = i % 3;
  double s = 0.0;
  for (int b = 0; b < n_blk; ++b) s += part[((size_t)J * n_blk + b) * 3 + a];
  F[i] = s;
}

// canonical [n_vec][n3] complex (C = double2 or float2) <-> orbital layout
template <typename T, int BO, typename C>
__global__ void k_pack(const C *__restrict__ canon,
                       typename cplx<T>::type *__restrict__ u, size_t n3,
                       int n_vec, int n_blk_vec) {
  typedef typename cplx<T>::type V;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t tot = (size_t)n_blk_vec * n3 * BO;
  if (i >= tot) return;
  const int j = i % BO;
  const size_t p = (i / BO) % n3;
  const int b = i / (BO * n3);
  const int A = b * BO + j;
  V v;
  if (A < n_vec) {
    const C s = canon[(size_t)A * n3 + p];
    v.x = (T)s.x;
    v.y = (T)s.y;
  } else {
    v.x = 0;
    v.y = 0;
  }
  u[i] = v;
}

template <typename T, int BO, typename C>
__global__ void k_unpack(const typename cplx<T>::type *__restrict__ u,
                         C *__restrict__ canon, size_t n3, int n_vec) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n_vec * n3) return;
  const int A = i / n3;
  const size_t p = i % n3;
  const int b = A / BO, j = A % BO;
  const typename cplx<T>::type v = u[((size_t)b * n3 + p) * BO + j];
  C c;
  c.x = v.x;
  c.y = v.y;
  canon[i] = c;
}

__global__ void __launch_bounds__(256)
k_abs2_sum(const double2 *c, int n, int row, int nch, double3 w, double *out) {
  __shared__ double red[8];
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a2 = c[i].x * c[i].x + c[i].y * c[i].y;
    if (nch == 1) {
      acc[0] += a2;
    } else {
      const int l = emd_channel_l((i / row) % nch);
      acc[0] += (l == 0 ? w.x : l == 1 ? w.y : w.z) * a2;
    }
  }
  emd_block_sum<1>(acc, red);
  if (threadIdx.x == 0) *out = acc[0];
}

// ---------------------------------------------------------------------------
// FP64 Horner stage in double-float arithmetic (complex128 orbitals, bo = 2).
// GB300 issues one FP64 warp instruction per 16 SM cycles, and the plain FP64
// stage spends ~59 FP64 instructions per update.  Here every value of a
// staged plane is split once into two floats, x = hi + lo (hi: the top 24
// significand bits, lo: the rest rounded to 24 bits; 48 bits in all), by
// integer operations on its bits, and the stencil runs on the FP32 pipes:
// products by the integer FD numerators num_k (exact in FP32) through
// TwoProduct with an FMA, sums through Knuth's TwoSum, the rounding errors
// gathered in the low word.  The accumulated K = dv u + sum_k num_k S_k,
// dv = 3 num_0 - 2 h^2 den v_eff, gives H u = -K / (2 h^2 den) + V_nl u; only
// the conversion of H u back to double and the Taylor update use FP64
// instructions (four per update).  The tile marches through z like the
// complex64 column kernels; each thread owns one orbital of one point, the
// z-direction accumulates in a (2M+1)-slot shift register, and planes are
// staged through registers (load, split, store) one plane ahead.
// ---------------------------------------------------------------------------
struct DFWeights {
  float num[EMD_MAX_HALF_ORDER + 1];   // FD numerators, exact in FP32
  float sk_hi, sk_lo;                  // -1 / (2 h^2 den) as double-float
  double dvs, dv0;                     // dv = dv0 + dvs v_eff
};

template <int M> struct DFTile {
  static constexpr int BO = 2;
  static constexpr int NC = 64;                 // orbital columns = threads in x
  static constexpr int TX = NC / BO;            // points per tile row
  static constexpr int NT = 512;
  static constexpr int TY = NT / NC;            // rows, one per thread row
  static constexpr int SW = TX + 2 * M, SH = TY + 2 * M;
  static constexpr int NCH = SH * SW * BO;      // complex values per staged plane
  static constexpr int CPT = (NCH + NT - 1) / NT;
  static constexpr int NV = TX * TY;            // tile points
  static constexpr int NS = 2 * M + 1;          // shift-register slots
  // raw slot (3, cp.async, two planes ahead): plane as complex128 | v_eff of
  // the tile points | records and psi0 of the output plane completed by it
  static constexpr int RU = NCH * 16, RV = NV * 8, RQ = NV * 48, RP = NV * BO * 16;
  static constexpr int RSLOT = RU + RV + RQ + RP;
  // split slot (2): plane as double-float complex | dv of the tile points
  static constexpr int DU = NCH * 16, DD = NV * 8;
  static constexpr int DSLOT = DU + DD;
  static constexpr size_t SMEM_FIXED = 3 * (size_t)RSLOT + 2 * (size_t)DSLOT;
};

// MP: several projectors per atom (the pre-split records past the first four
// are read with four in flight); a separate instantiation keeps the
// s-projector kernel's registers as they were
template <int M, bool HCS, bool MP>
__global__ void __launch_bounds__(512, 1)
k_stage_df(const double2 *__restrict__ u_in, const double2 *__restrict__ psi0,
           double2 *__restrict__ u_out, const double *__restrict__ v_eff,
           const int4 *__restrict__ pt4d, const int *__restrict__ pt_J,
           const double *__restrict__ pt_p, const int4 *__restrict__ pt_rec,
           const double2 *__restrict__ hc, int n,
           int ntx, int zc, int n_orb_pad, int n_atoms, double a, int apply_only,
           DFWeights W) {
  typedef DFTile<M> Z;
  constexpr int BO = Z::BO, NS = Z::NS, SW = Z::SW, NT = Z::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char *dfbase = smraw + 3 * Z::RSLOT;
  float4 *hcs = reinterpret_cast<float4 *>(smraw + Z::SMEM_FIXED);
  const int tid = threadIdx.x;
  const int col = tid % Z::NC, tyr = tid / Z::NC;
  const int xl = col / BO, j = col % BO;
  const int tx0 = (blockIdx.x % ntx) * Z::TX, ty0 = (blockIdx.x / ntx) * Z::TY;
  const int z0 = blockIdx.y * zc;
  const int zcount = min(zc, n - z0);
  const int total = zcount + 2 * M;
  const int n2 = n * n;
  const size_t n3 = (size_t)n2 * n;
  const size_t boff = (size_t)blockIdx.z * n3 * BO;
  const double2 *ub = u_in + boff;
  const double2 *pb = psi0 + boff;
  double2 *ob = u_out + boff;
  const int x = tx0 + xl, y = ty0 + tyr;
  const bool valid = x < n && y < n;
  const size_t pxy = (size_t)min(y, n - 1) * n + min(x, n - 1);

  // staging map of the plane values: source index within a plane, -1 = none
  int src[Z::CPT];
#pragma unroll
  for (int i = 0; i < Z::CPT; ++i) {
    const int q = tid + i * NT;
    src[i] = -1;
    if (q < Z::NCH) {
      const int jj = q % BO, pnt = q / BO;
      const int c = pnt % SW, rr = pnt / SW;
      const int xx = (tx0 - M + c + 2 * n) % n;
      const int yy = (ty0 - M + rr + 2 * n) % n;
      src[i] = (yy * n + xx) * BO + jj;
    }
  }
  // tile point of this thread in the per-point stagings (v_eff, records)
  const int vp = tid < Z::NV ? min(ty0 + tid / Z::TX, n - 1) * n + min(tx0 + tid % Z::TX, n - 1)
                             : -1;
  if (HCS) {
    for (int i = tid; i < n_atoms * BO; i += NT)
      hcs[i] = df_split2(hc[(size_t)(i / BO) * n_orb_pad + (size_t)blockIdx.z * BO + i % BO]);
  }
  const unsigned sm0 = (unsigned)__cvta_generic_to_shared(smraw);

  auto issue = [&](int zi) {
    const unsigned base = sm0 + (zi % 3) * Z::RSLOT;
    int zz = z0 - M + zi;
    zz += zz < 0 ? n : 0;
    zz -= zz >= n ? n : 0;
    const size_t poff = (size_t)zz * n2;
#pragma unroll
    for (int i = 0; i < Z::CPT; ++i)
      if (src[i] >= 0)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + (tid + i * NT) * 16),
                     "l"(ub + poff * BO + src[i]) : "memory");
    if (vp >= 0)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(base + Z::RU + tid * 8),
                   "l"(v_eff + poff + vp) : "memory");
    if (zi >= 2 * M && vp >= 0) {
      const size_t po = (size_t)(z0 + zi - 2 * M) * n2 + vp;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                         base + Z::RU + Z::RV + (tid * 3 + k) * 16),
                     "l"(pt4d + po * 3 + k) : "memory");
      if (!apply_only) {
#pragma unroll
        for (int jj = 0; jj < BO; ++jj)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                           base + Z::RU + Z::RV + Z::RQ + (tid * BO + jj) * 16),
                       "l"(pb + po * BO + jj) : "memory");
      }
    }
    cp_async_commit();
  };
  // split the raw plane zi into double-float slot zi & 1
  auto convert = [&](int zi) {
    const unsigned char *raw = smraw + (zi % 3) * Z::RSLOT;
    unsigned char *dst = dfbase + (zi & 1) * Z::DSLOT;
    const double2 *R = reinterpret_cast<const double2 *>(raw);
    float4 *D = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < Z::CPT; ++i)
      if (src[i] >= 0) D[tid + i * NT] = df_split2(R[tid + i * NT]);
    if (vp >= 0)
      reinterpret_cast<float2 *>(dst + Z::DU)[tid] =
          df_split(__fma_rn(W.dvs, reinterpret_cast<const double *>(raw + Z::RU)[tid], W.dv0));
  };

  // ah, al [s]: output plane zi - M + s, K as hi = (re, im), lo = (re, im)
  float2 ah[NS], al[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) ah[s] = al[s] = make_float2(0.f, 0.f);
  const int ci = ((tyr + M) * SW + xl + M) * BO + j;       // centre, float4 index
  const int pt = tyr * Z::TX + xl;                         // tile point index
  const char *hcj = reinterpret_cast<const char *>(hcs + j);
  const double2 *hcg = hc + (size_t)blockIdx.z * BO + j;

  issue(0);
  if (total > 1) issue(1);
  if (total > 1) cp_async_wait<1>();
  else cp_async_wait<0>();
  __syncthreads();
  convert(0);
  for (int zi = 0; zi < total; ++zi) {
    // raw plane zi + 1 (issued one iteration ago) is the only group in flight
    cp_async_wait<0>();
    // one barrier: raw zi + 1 visible; split zi (converted last iteration)
    // visible; every thread has finished iteration zi - 1, so split slot
    // (zi + 1) & 1 and raw slot (zi + 2) % 3 are free
    __syncthreads();
    if (zi + 2 < total) issue(zi + 2);
    if (zi + 1 < total) convert(zi + 1);
    const unsigned char *base = dfbase + (zi & 1) * Z::DSLOT;
    const float4 *P = reinterpret_cast<const float4 *>(base) + ci;
    const float2 d = reinterpret_cast<const float2 *>(base + Z::DU)[pt];
    const float4 c = P[0];
    const float2 ch = f4hi(c), cl = f4lo(c);
    // own plane: dv u + the x/y shells
    dfp_add_prod(ah[M], al[M], d.x, d.y, ch, cl);
#pragma unroll
    for (int k = 1; k <= M; ++k) {
      const float4 v1 = P[k * BO], v2 = P[-k * BO], v3 = P[k * SW * BO], v4 = P[-k * SW * BO];
      float2 sh = f4hi(v1), sl = f4lo(v1);
      dfp_add(sh, sl, f4hi(v2), f4lo(v2));
      dfp_add(sh, sl, f4hi(v3), f4lo(v3));
      dfp_add(sh, sl, f4hi(v4), f4lo(v4));
      const float2 w2 = make_float2(W.num[k], W.num[k]);
      float2 p, pe;
      dfp_two_prod(w2, sh, p, pe);
      dfp_add(ah[M], al[M], p, __ffma2_rn(w2, sl, pe));
    }
    // z-direction: this plane is neighbour k of output planes zi +- k
#pragma unroll
    for (int k = 1; k <= M; ++k) {
      const float2 w2 = make_float2(W.num[k], W.num[k]);
      float2 p, pe;
      dfp_two_prod(w2, ch, p, pe);
      const float2 q = __ffma2_rn(w2, cl, pe);
      dfp_add(ah[M + k], al[M + k], p, q);
      if (zi >= k) dfp_add(ah[M - k], al[M - k], p, q);
    }
    if (zi >= 2 * M && valid) {   // output plane z0 + zi - 2M is complete in slot 0
      const unsigned char *raw = smraw + (zi % 3) * Z::RSLOT;
      const int4 *Q = reinterpret_cast<const int4 *>(raw + Z::RU + Z::RV) + pt * 3;
      const int4 q0 = Q[0], q1 = Q[1], q2 = Q[2];
      float2 hh = make_float2(0.f, 0.f), hl = make_float2(0.f, 0.f);
      dfp_add_prod(hh, hl, W.sk_hi, W.sk_lo, ah[0], al[0]);
      // four entries (unused ones have p = 0 and add exactly zero)
      const int Je[4] = {q0.x & 0xffff, q0.y, q0.z, q0.w};
      const float ph[4] = {__int_as_float(q1.x), __int_as_float(q1.z), __int_as_float(q2.x),
                           __int_as_float(q2.z)};
      const float pl[4] = {__int_as_float(q1.y), __int_as_float(q1.w), __int_as_float(q2.y),
                           __int_as_float(q2.w)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float4 h4 = HCS ? *reinterpret_cast<const float4 *>(hcj + Je[e] * (BO * 16))
                              : df_split2(hcg[(size_t)Je[e] * n_orb_pad]);
        dfp_add_prod(hh, hl, ph[e], pl[e], f4hi(h4), f4lo(h4));
      }
      const int cnt = q0.x >> 16;
      if (cnt > 4) {
        const size_t p = (size_t)(z0 + zi - 2 * M) * n2 + pxy;
        if (MP) {
          // several projectors per atom: pre-split 16-byte records, four in
          // flight, summed into four independent pairs (combined in a fixed
          // order) so that the TwoSum chains overlap
          float2 xh[4], xl[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) xh[v] = xl[v] = make_float2(0.f, 0.f);
          for (int e = 4; e < cnt; e += 4) {
            int4 q[4];
#pragma unroll
            for (int v = 0; v < 4; ++v)
              q[v] = e + v < cnt ? __ldg(pt_rec + (size_t)(e + v) * n3 + p) : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const float4 h4 = HCS ? *reinterpret_cast<const float4 *>(hcj + q[v].x * (BO * 16))
                                    : df_split2(hcg[(size_t)q[v].x * n_orb_pad]);
              dfp_add_prod(xh[v], xl[v], __int_as_float(q[v].y), __int_as_float(q[v].z),
                           f4hi(h4), f4lo(h4));
            }
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) dfp_add(hh, hl, xh[v], xl[v]);
        } else {
          for (int e = 4; e < cnt; ++e) {
            const int J = pt_J[(size_t)e * n3 + p];
            const float2 pv = df_split(pt_p[(size_t)e * n3 + p]);
            const float4 h4 = HCS ? *reinterpret_cast<const float4 *>(hcj + J * (BO * 16))
                                  : df_split2(hcg[(size_t)J * n_orb_pad]);
            dfp_add_prod(hh, hl, pv.x, pv.y, f4hi(h4), f4lo(h4));
          }
        }
      }
      const double Hr = __dadd_rn(df_widen(hh.x), df_widen(hl.x));
      const double Hi = __dadd_rn(df_widen(hh.y), df_widen(hl.y));
      double2 out;
      if (apply_only) {
        out = make_double2(Hr, Hi);
      } else {
        const double2 sv =
            reinterpret_cast<const double2 *>(raw + Z::RU + Z::RV + Z::RQ)[pt * BO + j];
        out.x = __fma_rn(a, Hi, sv.x);
        out.y = __fma_rn(-a, Hr, sv.y);
      }
      ob[((size_t)(z0 + zi - 2 * M) * n2 + pxy) * BO + j] = out;
    }
    // shift the register line: output plane zi - M + 1 moves to slot 0
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
      ah[s] = ah[s + 1];
      al[s] = al[s + 1];
    }
    ah[NS - 1] = al[NS - 1] = make_float2(0.f, 0.f);
  }
}

// complex128 projections and nonlocal-force moments (bo = 2) in double-float
// arithmetic on the FP32 pipes: the FP64 forms spend 2 (projection) and 8
// (moments) FP64 instructions per table entry and orbital, which bounds them
// by GB300's FP64 rate.  Each thread takes the atom's entries tid, tid + 256,
// ... from the pre-split records (point, p as (hi, lo), and for the moments
// p d / r_c^2 as (hi, lo) per axis), DF_EU of them in flight at a time (the
// loads of an entry's orbital values wait on its record), splits the
// orbital values and accumulates (hi, lo) pairs with TwoProduct and TwoSum,
// real and imaginary parts packed; the sums are widened to FP64 once and
// join the fixed-tree FP64 block sum.
#define DF_EU 4

__global__ void __launch_bounds__(256)
k_project_df(const double2 *__restrict__ u, size_t n3, const int *__restrict__ at_cnt,
             const uint4 *__restrict__ at_rec, int cap, int nch, double h3, double3 hl,
             int n_orb_pad, double2 *c, double2 *hc) {
  constexpr int BO = 2;
  __shared__ double red[8 * 2 * BO];
  // one CTA per (projector P = J nch + k, block): atom J's entries, channel k
  const int P = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[P / nch];
  const int l = emd_channel_l(P % nch);
  const double h_kb = l == 0 ? hl.x : l == 1 ? hl.y : hl.z;
  const double2 *ub = u + (size_t)blk * n3 * BO;
  const uint4 *rec = at_rec + (size_t)P * cap;
  float2 ah[BO], al[BO];
#pragma unroll
  for (int j = 0; j < BO; ++j) ah[j] = al[j] = make_float2(0.f, 0.f);
  for (int e0 = threadIdx.x; e0 < cnt; e0 += DF_EU * 256) {
    uint4 r[DF_EU];
#pragma unroll
    for (int v = 0; v < DF_EU; ++v)       // past the end: point 0, p = 0 (adds zero)
      r[v] = e0 + 256 * v < cnt ? __ldg(rec + e0 + 256 * v) : make_uint4(0u, 0u, 0u, 0u);
    double2 x[DF_EU][BO];
#pragma unroll
    for (int v = 0; v < DF_EU; ++v)
#pragma unroll
      for (int j = 0; j < BO; ++j) x[v][j] = ub[(size_t)r[v].x * BO + j];
#pragma unroll
    for (int v = 0; v < DF_EU; ++v)
#pragma unroll
      for (int j = 0; j < BO; ++j) {
        const float4 xs = df_split2(x[v][j]);
        dfp_add_prod(ah[j], al[j], __uint_as_float(r[v].y), __uint_as_float(r[v].z), f4hi(xs),
                     f4lo(xs));
      }
  }
  double acc[2 * BO];
#pragma unroll
  for (int j = 0; j < BO; ++j) {
    acc[2 * j] = __dadd_rn(df_widen(ah[j].x), df_widen(al[j].x));
    acc[2 * j + 1] = __dadd_rn(df_widen(ah[j].y), df_widen(al[j].y));
  }
  emd_block_sum<2 * BO>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < BO; ++j) {
      const size_t o = (size_t)P * n_orb_pad + (size_t)blk * BO + j;
      const double re = h3 * acc[2 * j], im = h3 * acc[2 * j + 1];
      c[o] = make_double2(re, im);
      hc[o] = make_double2(h_kb * re, h_kb * im);
    }
  }
}

// part[(P n_blk + blk) 3 + a]: projector P's share of the nonlocal force of
// block blk's orbitals on atom P / nch (coef for P's strength: coef3.x for
// l = 0, .y for l = 1, .z for l = 2)
__global__ void __launch_bounds__(256)
k_nl_force_df(const double2 *__restrict__ u, size_t n3, int n_blk,
              const int *__restrict__ at_cnt, const uint4 *__restrict__ at_rec,
              const float4 *__restrict__ at_w, int cap, int nch, const double2 *__restrict__ c,
              int n_orb_pad, int n_orb, double h3, double3 coef3, double *part) {
  constexpr int BO = 2, EU = DF_EU;
  __shared__ double red[8 * 6 * BO];
  const int P = blockIdx.x, blk = blockIdx.y;
  const int cnt = at_cnt[P / nch];
  const int l = emd_channel_l(P % nch);
  const double coef = l == 0 ? coef3.x : l == 1 ? coef3.y : coef3.z;
  const double2 *ub = u + (size_t)blk * n3 * BO;
  const uint4 *rec = at_rec + (size_t)P * cap;
  const float4 *wr = at_w + (size_t)P * cap * 2;
  float2 ah[3 * BO], al[3 * BO];      // [orbital][axis] complex moments
#pragma unroll
  for (int k = 0; k < 3 * BO; ++k) ah[k] = al[k] = make_float2(0.f, 0.f);
  for (int e0 = threadIdx.x; e0 < cnt; e0 += EU * 256) {
    int pt[EU];
    float4 w0[EU], w1[EU];
#pragma unroll
    for (int v = 0; v < EU; ++v) {        // past the end: point 0, w = 0 (adds zero)
      const int e = e0 + 256 * v;
      const bool ok = e < cnt;
      pt[v] = ok ? (int)__ldg(&rec[e].x) : 0;
      w0[v] = ok ? __ldg(wr + 2 * e) : make_float4(0.f, 0.f, 0.f, 0.f);
      w1[v] = ok ? __ldg(wr + 2 * e + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    double2 x[EU][BO];
#pragma unroll
    for (int v = 0; v < EU; ++v)
#pragma unroll
      for (int j = 0; j < BO; ++j) x[v][j] = ub[(size_t)pt[v] * BO + j];
#pragma unroll
    for (int v = 0; v < EU; ++v)
#pragma unroll
      for (int j = 0; j < BO; ++j) {
        const float4 xs = df_split2(x[v][j]);
        dfp_add_prod(ah[3 * j + 0], al[3 * j + 0], w0[v].x, w0[v].y, f4hi(xs), f4lo(xs));
        dfp_add_prod(ah[3 * j + 1], al[3 * j + 1], w0[v].z, w0[v].w, f4hi(xs), f4lo(xs));
        dfp_add_prod(ah[3 * j + 2], al[3 * j + 2], w1[v].x, w1[v].y, f4hi(xs), f4lo(xs));
      }
  }
  double acc[6 * BO];
#pragma unroll
  for (int j = 0; j < BO; ++j)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[6 * j + 2 * a] = __dadd_rn(df_widen(ah[3 * j + a].x), df_widen(al[3 * j + a].x));
      acc[6 * j + 2 * a + 1] = __dadd_rn(df_widen(ah[3 * j + a].y), df_widen(al[3 * j + a].y));
    }
  emd_block_sum<6 * BO>(acc, red);
  if (threadIdx.x == 0) {
    double f[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < BO; ++j) {
      const int A = blk * BO + j;
      if (A >= n_orb) continue;
      const double2 cj = c[(size_t)P * n_orb_pad + A];
      for (int a = 0; a < 3; ++a) {
        const double dr = h3 * acc[6 * j + 2 * a], di = h3 * acc[6 * j + 2 * a + 1];
        f[a] += cj.x * dr + cj.y * di;   // Re(conj(c) dc)
      }
    }
    for (int a = 0; a < 3; ++a)
      part[((size_t)P * n_blk + blk) * 3 + a] = coef * f[a];
  }
}

// ---- dispatch -------------------------------------------------------------

// planes per z-chunk of a marching stage launch: the caller's choice, else
// whole columns unless the columns alone would leave SMs idle (each chunk
// restages and re-stencils 2M halo planes)
inline int stage_zchunk(const OrbLayout &o, int cols, int min_ctas) {
  if (o.zchunk > 0) return std::min(o.zchunk, o.n);
  const int nz = std::max(1, std::min((min_ctas + cols - 1) / cols, o.n / 16));
  return (o.n + nz - 1) / nz;
}

template <typename T, int BO, int M>
void stage_t(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  typedef typename cplx<T>::type V;
  const int ntx = (o.n + 31) / 32, nty = (o.n + 3) / 4;
  dim3 grid(ntx * nty, o.n, o.n_blk), block(32, 4);
  k_stage<T, BO, M><<<grid, block, 0, st>>>(
      (const V *)a.u_in, (const V *)a.psi0, (V *)a.u_out, (const T *)a.v_eff,
      a.tab->pt_cnt, a.tab->pt_J, a.tab->pt_p, (const V *)a.hc, o.n, ntx,
      o.n_orb_pad, (T)a.a, a.apply_only, weights_of<T>(o));
}

template <int BO, int M>
void stage_z_t(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  typedef ZTile<BO, M> Z;
  const int hc_bytes = o.n_atoms * BO * (int)sizeof(float2);
  const int hc_in_smem = hc_bytes <= 16384;
  const size_t smem = Z::SMEM_FIXED + (hc_in_smem ? hc_bytes : 0);
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_stage_z<BO, M>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(Z::SMEM_FIXED + 16384));
    attr_done = true;
  }
  const int ntx = (o.n + Z::TX - 1) / Z::TX, nty = (o.n + Z::TY - 1) / Z::TY;
  const int zc = o.zchunk > 0 ? std::min(o.zchunk, o.n)
                             : (o.n <= 64 ? o.n : (o.n + 1) / 2 <= 64 ? (o.n + 1) / 2 : 48);
  dim3 grid(ntx * nty, (o.n + zc - 1) / zc, o.n_blk);
  k_stage_z<BO, M><<<grid, Z::NT, smem, st>>>(
      (const float2 *)a.u_in, (const float2 *)a.psi0, (float2 *)a.u_out,
      (const float *)a.v_eff, a.tab->pt4, a.tab->pt_J, a.tab->pt_pf,
      (const float2 *)a.hc, o.n, ntx, zc, o.n_orb_pad, o.n_atoms, hc_in_smem,
      (float)a.a, a.apply_only, weights_of<float>(o));
}

// ---- tensor maps of the complex64 stage (encoded once per array) ---------
typedef CUresult (*TmEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                               const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                               const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmEncodeFn tm_encode_fn() {
  static TmEncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmEncodeFn>(p);
  });
  return fn;
}

// A 3-D view (inner elements, x, rows) of an array of n x-points per row
// with `inner` 4-byte elements per point, and a box of (inner, bx, by).
bool tm_get(CUtensorMap *out, const void *base, bool is_int, int inner, int n, size_t rows,
            int bx, int by) {
  static std::mutex mu;
  static std::map<std::tuple<const void *, int, int, size_t, int, int>, CUtensorMap> cache;
  const auto key = std::make_tuple(base, inner * (is_int ? -1 : 1), n, rows, bx, by);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return true;
  }
  TmEncodeFn f = tm_encode_fn();
  if (!f) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)n, (cuuint64_t)rows};
  const cuuint64_t strides[2] = {(cuuint64_t)inner * 4, (cuuint64_t)inner * 4 * n};
  const cuuint32_t box[3] = {(cuuint32_t)inner, (cuuint32_t)bx, (cuuint32_t)by};
  const cuuint32_t es[3] = {1, 1, 1};
  CUtensorMap tm;
  if (f(&tm, is_int ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
        const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  cache[key] = tm;
  *out = tm;
  return true;
}

template <int BO, int M, bool HCS, bool TMA>
void stage_c_tt(const OrbLayout &o, const StageArgs &a, size_t smem, cudaStream_t st,
                const CUtensorMap *tm) {
  typedef ZCTile<BO, M> Z;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_stage_c<BO, M, HCS, TMA>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(Z::SMEM_FIXED + 16384 + 256));
    attr_done = true;
  }
  const int ntx = (o.n + Z::TX - 1) / Z::TX, nty = (o.n + Z::TY - 1) / Z::TY;
  // one z-chunk per column unless the columns alone would leave SMs idle:
  // each chunk restages and re-stencils 2M halo planes
  const int zc = stage_zchunk(o, ntx * nty * o.n_blk, 2 * 152);
  dim3 grid(ntx * nty, (o.n + zc - 1) / zc, o.n_blk);
  k_stage_c<BO, M, HCS, TMA><<<grid, Z::NT, smem + 256, st>>>(
      (const float2 *)a.u_in, (const float2 *)a.psi0, (float2 *)a.u_out,
      (const float4 *)a.v_diag, a.tab->pt4, a.tab->pt_J, a.tab->pt_pf,
      (const float2 *)a.hc, o.n, ntx, zc, o.n_orb_pad, o.n_atoms, (float)a.a,
      a.apply_only, wpairs_of(o), tm[0], tm[1], tm[2], a.err);
}

template <int BO, int M>
void stage_c_t(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  typedef ZCTile<BO, M> Z;
  const int hc_bytes = o.n_atoms * BO * (int)sizeof(float2);
  // tensor copies for bo = 4 unless the cp.async form is asked for
  // (variant 2) or a map cannot be encoded
  CUtensorMap tm[3];
  memset(tm, 0, sizeof(tm));
  bool tma = false;
  if (BO == 4 && o.stage_variant != 2) {
    const size_t n2 = (size_t)o.n * o.n;
    tma = tm_get(&tm[0], a.v_diag, false, 4, o.n, n2, Z::TX, Z::TY) &&
          tm_get(&tm[1], a.tab->pt4, true, 8, o.n, n2, Z::TX, Z::TY) &&
          (a.apply_only || tm_get(&tm[2], a.psi0, false, 8, o.n, n2 * o.n * o.n_blk, Z::TX, Z::TY));
  }
  if (tma) {
    if (hc_bytes <= 16384)
      stage_c_tt<BO, M, true, BO == 4>(o, a, Z::SMEM_FIXED + hc_bytes, st, tm);
    else
      stage_c_tt<BO, M, false, BO == 4>(o, a, Z::SMEM_FIXED, st, tm);
  } else {
    if (hc_bytes <= 16384)
      stage_c_tt<BO, M, true, false>(o, a, Z::SMEM_FIXED + hc_bytes, st, tm);
    else
      stage_c_tt<BO, M, false, false>(o, a, Z::SMEM_FIXED, st, tm);
  }
}

template <int BO>
void stage_c_m(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  switch (o.half_order) {
    case 1: stage_c_t<BO, 1>(o, a, st); break;
    case 2: stage_c_t<BO, 2>(o, a, st); break;
    case 3: stage_c_t<BO, 3>(o, a, st); break;
    case 4: stage_c_t<BO, 4>(o, a, st); break;
  }
}

template <int BO, int M, int RY>
void stage_zp_t(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  typedef ZPTile<BO, M, RY> Z;
  const int hc_bytes = o.n_atoms * BO * (int)sizeof(float2);
  const int hc_in_smem = hc_bytes <= 16384;
  const size_t smem = Z::SMEM_FIXED + (hc_in_smem ? hc_bytes : 0);
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_stage_zp<BO, M, RY>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(Z::SMEM_FIXED + 16384));
    attr_done = true;
  }
  const int ntx = (o.n + Z::TX - 1) / Z::TX, nty = (o.n + Z::TY - 1) / Z::TY;
  const int zc = o.zchunk > 0 ? std::min(o.zchunk, o.n)
                             : (o.n <= 64 ? o.n : (o.n + 1) / 2 <= 64 ? (o.n + 1) / 2 : 48);
  dim3 grid(ntx * nty, (o.n + zc - 1) / zc, o.n_blk);
  k_stage_zp<BO, M, RY><<<grid, Z::NT, smem, st>>>(
      (const float2 *)a.u_in, (const float2 *)a.psi0, (float2 *)a.u_out,
      (const float *)a.v_eff, a.tab->pt4, a.tab->pt_J, a.tab->pt_pf,
      (const float2 *)a.hc, o.n, ntx, zc, o.n_orb_pad, o.n_atoms, hc_in_smem,
      (float)a.a, a.apply_only, weights_of<float>(o));
}

template <int BO, int RY>
void stage_zp_m(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  switch (o.half_order) {
    case 1: stage_zp_t<BO, 1, RY>(o, a, st); break;
    case 2: stage_zp_t<BO, 2, RY>(o, a, st); break;
    case 3: stage_zp_t<BO, 3, RY>(o, a, st); break;
    case 4: stage_zp_t<BO, 4, RY>(o, a, st); break;
  }
}

template <int BO>
void stage_z_m(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  switch (o.half_order) {
    case 1: stage_z_t<BO, 1>(o, a, st); break;
    case 2: stage_z_t<BO, 2>(o, a, st); break;
    case 3: stage_z_t<BO, 3>(o, a, st); break;
    case 4: stage_z_t<BO, 4>(o, a, st); break;
  }
}

template <int M, bool HCS, bool MP>
void stage_df_tt(const OrbLayout &o, const StageArgs &a, size_t smem, cudaStream_t st) {
  typedef DFTile<M> Z;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_stage_df<M, HCS, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(Z::SMEM_FIXED + 32768));
    attr_done = true;
  }
  const int ntx = (o.n + Z::TX - 1) / Z::TX, nty = (o.n + Z::TY - 1) / Z::TY;
  const int zc = stage_zchunk(o, ntx * nty * o.n_blk, 2 * 152);
  DFWeights W;
  for (int k = 0; k <= EMD_MAX_HALF_ORDER; ++k) W.num[k] = (float)o.num[k];
  const double sk = -1.0 / (2.0 * o.h * o.h * o.den);
  W.sk_hi = (float)sk;
  W.sk_lo = (float)(sk - (double)W.sk_hi);
  W.dvs = -2.0 * o.h * o.h * o.den;
  W.dv0 = 3.0 * o.num[0];
  dim3 grid(ntx * nty, (o.n + zc - 1) / zc, o.n_blk);
  k_stage_df<M, HCS, MP><<<grid, Z::NT, smem, st>>>(
      (const double2 *)a.u_in, (const double2 *)a.psi0, (double2 *)a.u_out,
      (const double *)a.v_eff, a.tab->pt4d, a.tab->pt_J, a.tab->pt_p, a.tab->pt_rec,
      (const double2 *)a.hc, o.n, ntx, zc, o.n_orb_pad, o.n_proj, a.a, a.apply_only, W);
}

template <int M>
void stage_df_t(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  typedef DFTile<M> Z;
  const int hc_bytes = o.n_proj * Z::BO * (int)sizeof(float4);   // every projector's h c
  const bool mp = a.tab->pt_rec != nullptr;
  if (hc_bytes <= 32768) {
    if (mp) stage_df_tt<M, true, true>(o, a, Z::SMEM_FIXED + hc_bytes, st);
    else stage_df_tt<M, true, false>(o, a, Z::SMEM_FIXED + hc_bytes, st);
  } else {
    if (mp) stage_df_tt<M, false, true>(o, a, Z::SMEM_FIXED, st);
    else stage_df_tt<M, false, false>(o, a, Z::SMEM_FIXED, st);
  }
}

inline void stage_df_m(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  switch (o.half_order) {
    case 1: stage_df_t<1>(o, a, st); break;
    case 2: stage_df_t<2>(o, a, st); break;
    case 3: stage_df_t<3>(o, a, st); break;
    case 4: stage_df_t<4>(o, a, st); break;
  }
}

template <typename T, int BO>
void stage_m(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  switch (o.half_order) {
    case 1: stage_t<T, BO, 1>(o, a, st); break;
    case 2: stage_t<T, BO, 2>(o, a, st); break;
    case 3: stage_t<T, BO, 3>(o, a, st); break;
    case 4: stage_t<T, BO, 4>(o, a, st); break;
  }
}

#define EMD_DISPATCH_BO(T, FN, ...)                  \
  switch (o.bo) {                                    \
    case 1: FN<T, 1>(__VA_ARGS__); break;            \
    case 2: FN<T, 2>(__VA_ARGS__); break;            \
    case 4: FN<T, 4>(__VA_ARGS__); break;            \
  }

template <typename T, int BO>
void project_t(const OrbLayout &o, const TableSet &t, int n_atoms,
               const void *u, double h3, double h_kb, double2 *c, void *hc,
               cudaStream_t st) {
  typedef typename cplx<T>::type V;
  dim3 grid(n_atoms, o.n_blk);
  if (sizeof(T) == 8 && BO == 2 && t.at_rec)   // one CTA per projector
    k_project_df<<<dim3(n_atoms * o.nch, o.n_blk), 256, 0, st>>>(
        (const double2 *)u, (size_t)o.n3, t.at_cnt, t.at_rec, t.cap, o.nch, h3,
        make_double3(h_kb, o.hl[1], o.hl[2]), o.n_orb_pad, c, (double2 *)hc);
  else
    k_project<T, BO><<<grid, 256, 0, st>>>((const V *)u, (size_t)o.n3, t.at_cnt,
                                           t.at_pt, t.at_p, t.cap, h3, h_kb,
                                           o.n_orb_pad, c, (V *)hc);
}

template <typename T, int BO>
void density_t(const OrbLayout &o, const void *u, double occ, double *rho,
               cudaStream_t st) {
  typedef typename cplx<T>::type V;
  if (sizeof(T) == 4)
    k_density_c64<BO><<<(o.n3 + 255) / 256, 256, 0, st>>>(
        (const float2 *)u, (size_t)o.n3, o.n_blk, occ, rho);
  else if (BO == 2)
    k_density_df<BO><<<(o.n3 + 255) / 256, 256, 0, st>>>(
        (const double2 *)u, (size_t)o.n3, o.n_blk, occ, rho);
  else
    k_density<T, BO><<<(o.n3 + 255) / 256, 256, 0, st>>>((const V *)u,
                                                         (size_t)o.n3, o.n_blk,
                                                         occ, rho);
}

template <typename T, int BO, int M>
void kinetic_tm(const OrbLayout &o, const void *u, double *part, int nb,
                cudaStream_t st) {
  typedef typename cplx<T>::type V;
  k_kinetic<T, BO, M><<<nb, 256, 0, st>>>((const V *)u, o.n, o.n_blk, part,
                                          weights_of<double>(o));
}
template <typename T, int BO>
void kinetic_t(const OrbLayout &o, const void *u, double *part, int nb,
               cudaStream_t st) {
  switch (o.half_order) {
    case 1: kinetic_tm<T, BO, 1>(o, u, part, nb, st); break;
    case 2: kinetic_tm<T, BO, 2>(o, u, part, nb, st); break;
    case 3: kinetic_tm<T, BO, 3>(o, u, part, nb, st); break;
    case 4: kinetic_tm<T, BO, 4>(o, u, part, nb, st); break;
  }
}

template <typename T, int BO>
void nlf_t(const OrbLayout &o, const TableSet &t, int n_atoms, const void *u,
           const double2 *c, double h3, double coef, double coef_unit, double inv_rc2,
           double *part, cudaStream_t st) {
  typedef typename cplx<T>::type V;
  dim3 grid(n_atoms, o.n_blk);
  if (sizeof(T) == 8 && BO == 2 && t.at_rec) {
    // the s channel keeps coef = -2 h_kb occ as given
    const double3 coef3 = make_double3(coef, coef_unit * o.hl[1], coef_unit * o.hl[2]);
    k_nl_force_df<<<dim3(n_atoms * o.nch, o.n_blk), 256, 0, st>>>(
        (const double2 *)u, (size_t)o.n3, o.n_blk, t.at_cnt, t.at_rec, t.at_w, t.cap, o.nch, c,
        o.n_orb_pad, o.n_orb, h3, coef3, part);
  } else
    k_nl_force<T, BO><<<grid, 256, 0, st>>>((const V *)u, (size_t)o.n3, o.n_blk,
                                            t.at_cnt, t.at_pt, t.at_p, t.at_d,
                                            t.cap, c, o.n_orb_pad, o.n_orb, h3,
                                            coef, inv_rc2, part);
}

template <typename T, int BO, typename C>
void pack_t(const OrbLayout &o, const C *canon, void *u, int n_vec, cudaStream_t st) {
  typedef typename cplx<T>::type V;
  const int nbv = (n_vec + BO - 1) / BO;
  const size_t tot = (size_t)nbv * o.n3 * BO;
  k_pack<T, BO, C><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      canon, (V *)u, (size_t)o.n3, n_vec, nbv);
}

template <typename T, int BO, typename C>
void unpack_t(const OrbLayout &o, const void *u, C *canon, int n_vec, cudaStream_t st) {
  typedef typename cplx<T>::type V;
  const size_t tot = (size_t)n_vec * o.n3;
  k_unpack<T, BO, C><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      (const V *)u, canon, (size_t)o.n3, n_vec);
}

#define EMD_DISPATCH_BO_C(T, C, FN, ...)             \
  switch (o.bo) {                                    \
    case 1: FN<T, 1, C>(__VA_ARGS__); break;         \
    case 2: FN<T, 2, C>(__VA_ARGS__); break;         \
    case 4: FN<T, 4, C>(__VA_ARGS__); break;         \
  }

}  // namespace

void emd_launch_stage(const OrbLayout &o, const StageArgs &a, cudaStream_t st) {
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    switch (o.bo) {
      case 1: stage_m<double, 1>(o, a, st); break;
      case 2:
        if (o.stage_variant == 1 || !a.tab->pt4d) stage_m<double, 2>(o, a, st);
        else stage_df_m(o, a, st);
        break;
      case 4: stage_m<double, 4>(o, a, st); break;
    }
  } else {
    switch (o.bo) {
      case 1: stage_m<float, 1>(o, a, st); break;
      case 2:
        if (o.stage_variant == 1) stage_z_m<2>(o, a, st);
        else if (o.stage_variant == 2) stage_zp_m<2, 1>(o, a, st);
        else if (o.stage_variant == 3) stage_zp_m<2, 2>(o, a, st);
        else if (a.v_diag) stage_c_m<2>(o, a, st);
        else stage_zp_m<2, 2>(o, a, st);
        break;
      case 4:   // point-per-thread needs > 128 registers
        if (o.stage_variant == 1) stage_z_m<4>(o, a, st);
        else if (a.v_diag) stage_c_m<4>(o, a, st);
        else stage_z_m<4>(o, a, st);
        break;
    }
  }
}

void emd_launch_project(const OrbLayout &o, const TableSet &t, int n_atoms,
                        const void *u, double h3, double h_kb, double2 *c,
                        void *hc, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO(double, project_t, o, t, n_atoms, u, h3, h_kb, c, hc, st)
  } else {
    EMD_DISPATCH_BO(float, project_t, o, t, n_atoms, u, h3, h_kb, c, hc, st)
  }
}

void emd_launch_density(const OrbLayout &o, const void *u, double occ,
                        double *rho, cudaStream_t st) {
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO(double, density_t, o, u, occ, rho, st)
  } else {
    EMD_DISPATCH_BO(float, density_t, o, u, occ, rho, st)
  }
}

void emd_launch_kinetic_partials(const OrbLayout &o, const void *u,
                                 double *partials, int *nparts,
                                 cudaStream_t st) {
  emd_note_launches(1);
  const int nb = (o.n3 + 255) / 256;
  *nparts = nb;
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO(double, kinetic_t, o, u, partials, nb, st)
  } else {
    EMD_DISPATCH_BO(float, kinetic_t, o, u, partials, nb, st)
  }
}

void emd_launch_nl_force(const OrbLayout &o, const TableSet &t, int n_atoms,
                         const void *u, const double2 *c, double h3,
                         double coef, double coef_unit, double inv_rc2, double *part,
                         double *F_nl, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO(double, nlf_t, o, t, n_atoms, u, c, h3, coef, coef_unit, inv_rc2, part, st)
  } else {
    EMD_DISPATCH_BO(float, nlf_t, o, t, n_atoms, u, c, h3, coef, coef_unit, inv_rc2, part, st)
  }
  // an atom's partials: its projectors' (channel-major), each over the blocks
  const int per = (o.prec == EMD_FP64 && o.bo == 2 && t.at_rec) ? o.nch * o.n_blk : o.n_blk;
  const int m = 3 * n_atoms;
  k_nl_force_sum<<<(m + 127) / 128, 128, 0, st>>>(part, n_atoms, per, F_nl);
}

void emd_launch_pack(const OrbLayout &o, const double2 *canon, void *u,
                     int n_vec, cudaStream_t st) {
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO_C(double, double2, pack_t, o, canon, u, n_vec, st)
  } else {
    EMD_DISPATCH_BO_C(float, double2, pack_t, o, canon, u, n_vec, st)
  }
}

void emd_launch_unpack(const OrbLayout &o, const void *u, double2 *canon,
                       int n_vec, cudaStream_t st) {
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO_C(double, double2, unpack_t, o, u, canon, n_vec, st)
  } else {
    EMD_DISPATCH_BO_C(float, double2, unpack_t, o, u, canon, n_vec, st)
  }
}

void emd_launch_pack_c64(const OrbLayout &o, const float2 *canon, void *u, int n_vec,
                         cudaStream_t st) {
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO_C(double, float2, pack_t, o, canon, u, n_vec, st)
  } else {
    EMD_DISPATCH_BO_C(float, float2, pack_t, o, canon, u, n_vec, st)
  }
}

void emd_launch_unpack_c64(const OrbLayout &o, const void *u, float2 *canon, int n_vec,
                           cudaStream_t st) {
  emd_note_launches(1);
  if (o.prec == EMD_FP64) {
    EMD_DISPATCH_BO_C(double, float2, unpack_t, o, u, canon, n_vec, st)
  } else {
    EMD_DISPATCH_BO_C(float, float2, unpack_t, o, u, canon, n_vec, st)
  }
}

void emd_launch_abs2_sum(const double2 *c, int n, int row, int nch, const double *w, double *out,
                         cudaStream_t st) {
  emd_note_launches(1);
  k_abs2_sum<<<1, 256, 0, st>>>(c, n, row, nch, make_double3(w[0], w[1], w[2]), out);
}

void emd_launch_cdot_re_c64(const OrbLayout &o, const void *a, const void *b,
                            double *partials, int *nparts, cudaStream_t st) {
  emd_note_launches(1);
  const int nb = (o.n3 + 255) / 256;
  *nparts = nb;
  switch (o.bo) {
    case 1: k_cdot_re_c64<1><<<nb, 256, 0, st>>>((const float2 *)a, (const float2 *)b, (size_t)o.n3, o.n_blk, partials); break;
    case 2: k_cdot_re_c64<2><<<nb, 256, 0, st>>>((const float2 *)a, (const float2 *)b, (size_t)o.n3, o.n_blk, partials); break;
    case 4: k_cdot_re_c64<4><<<nb, 256, 0, st>>>((const float2 *)a, (const float2 *)b, (size_t)o.n3, o.n_blk, partials); break;
  }
}
