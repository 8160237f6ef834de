// Point-major projections c_JA = h^3 sum_r p_J(r) u_A(r) (the separable term
// of H, paper Sec. 5: norm-conserving pseudopotentials in separable form).
//
// The atom-major gather (one CTA per atom) reads every grid point once per
// atom whose sphere covers it, kappa ~ 2.4 times on the dense workloads.  Here
// a CTA owns one 8^3 tile of points and one orbital block and reads them once:
// for every atom of the tile (distinct atoms of the tile's candidate list),
// each warp reduces its lanes' contributions with a fixed shuffle tree
// (warps without that atom skip it), the CTA adds its warps in order, and a
// second kernel adds the tiles of each atom in tile order.  The result is
// deterministic run to run.
#include "emd_internal.cuh"

namespace {

// distinct atoms of each tile's (atom, image) candidate list, in atom order
__global__ void k_tile_atoms(const int *tile_cnt, const int *tile_ent, int ntiles,
                             int *tile_nat, int *tile_atoms, int *err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  int last = -1, s = 0;
  for (int e = 0; e < tile_cnt[t]; ++e) {
    const int J = tile_ent[t * EMD_TILE_CAND_MAX + e] / 27;
    if (J != last) {
      if (s < EMD_TILE_ATOM_MAX) tile_atoms[t * EMD_TILE_ATOM_MAX + s] = J;
      else atomicOr(err, EMD_ERRBIT_TILE);
      ++s;
      last = J;
    }
  }
  tile_nat[t] = min(s, EMD_TILE_ATOM_MAX);
}

// exclusive prefix sum of tile_nat (one CTA, fixed order) -> tile_off
__global__ void k_tile_offsets(const int *tile_nat, int ntiles, int *tile_off) {
  __shared__ int part[1024];
  const int per = (ntiles + blockDim.x - 1) / blockDim.x;
  const int t0 = threadIdx.x * per, t1 = min(ntiles, t0 + per);
  int s = 0;
  for (int t = t0; t < t1; ++t) s += tile_nat[t];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const int v = part[i];
      part[i] = acc;
      acc += v;
    }
  }
  __syncthreads();
  int acc = part[threadIdx.x];
  for (int t = t0; t < t1; ++t) {
    tile_off[t] = acc;
    acc += tile_nat[t];
  }
}

// For atom J: the (tile, slot) pairs of the tiles listing J, in tile order.
__global__ void __launch_bounds__(256)
k_atom_tiles(const int *tile_nat, const int *tile_atoms, int ntiles, int cap,
             int *at_ntiles, int2 *at_tiles, int *err) {
  __shared__ int warp_tot[8];
  __shared__ int s_base;
  const int J = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
    const int t = b0 + threadIdx.x;
    int slot = -1;
    if (t < ntiles)
      for (int s = 0; s < tile_nat[t]; ++s)
        if (tile_atoms[t * EMD_TILE_ATOM_MAX + s] == J) slot = s;
    const bool hit = slot >= 0;
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
      if (e < cap) at_tiles[(size_t)J * cap + e] = make_int2(t, slot);
      else atomicOr(err, EMD_ERRBIT_AT);
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) at_ntiles[J] = min(s_base, cap);
}

template <typename T> struct Acc;
template <> struct Acc<float> { typedef float type; };
template <> struct Acc<double> { typedef double type; };

// partial[(blk * sum_t S_t + tile_off[t] + s) * BO + j] = sum over the tile's
// points of p_Js(r) u_j(r), FP64 (warp sums in T, CTA sum of warps in FP64).
template <typename T, int BO>
__global__ void __launch_bounds__(512)
k_project_pm(const typename cplx<T>::type *__restrict__ u, int n, int nt,
             const int *__restrict__ pt_cnt, const int *__restrict__ pt_J,
             const double *__restrict__ pt_p, const int *__restrict__ tile_nat,
             const int *__restrict__ tile_atoms, const int *__restrict__ tile_off,
             int n_slots_total, double2 *__restrict__ partial) {
  typedef typename cplx<T>::type V;
  __shared__ int js[EMD_TILE_ATOM_MAX];
  __shared__ T wsum[16][EMD_TILE_ATOM_MAX][2 * BO];
  const int t = blockIdx.x, blk = blockIdx.y;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  const int S = tile_nat[t];
  for (int i = threadIdx.x; i < S; i += blockDim.x)
    js[i] = tile_atoms[t * EMD_TILE_ATOM_MAX + i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = tx * EMD_TILE + (threadIdx.x & 7);
  const int y = ty * EMD_TILE + ((threadIdx.x >> 3) & 7);
  const int z = tz * EMD_TILE + (threadIdx.x >> 6);
  const bool in = x < n && y < n && z < n;
  const size_t n3 = (size_t)n * n * n;
  const size_t p = in ? ((size_t)z * n + y) * n + x : 0;
  V uv[BO];
  int cnt = 0;
  if (in) {
    cnt = pt_cnt[p];
    const V *ub = u + ((size_t)blk * n3 + p) * BO;
#pragma unroll
    for (int j = 0; j < BO; ++j) uv[j] = ub[j];
  }
  __syncthreads();
  int ep = 0;                                   // next own entry (sorted by J)
  int Je = ep < cnt ? pt_J[p] : -1;
  for (int s = 0; s < S; ++s) {
    const int J = js[s];
    T c[2 * BO];
#pragma unroll
    for (int k = 0; k < 2 * BO; ++k) c[k] = 0;
    bool has = false;
    if (Je == J) {
      const T pv = (T)pt_p[(size_t)ep * n3 + p];
#pragma unroll
      for (int j = 0; j < BO; ++j) {
        c[2 * j] = pv * uv[j].x;
        c[2 * j + 1] = pv * uv[j].y;
      }
      has = true;
      ++ep;
      Je = ep < cnt ? pt_J[(size_t)ep * n3 + p] : -1;
    }
    if (__ballot_sync(0xffffffffu, has) == 0u) {
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < 2 * BO; ++k) wsum[warp][s][k] = 0;
      continue;
    }
#pragma unroll
    for (int k = 0; k < 2 * BO; ++k) {
      T v = c[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[warp][s][k] = v;
    }
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int q = threadIdx.x; q < S * BO; q += blockDim.x) {
    const int s = q / BO, j = q % BO;
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nw; ++w) {
      re += (double)wsum[w][s][2 * j];
      im += (double)wsum[w][s][2 * j + 1];
    }
    partial[((size_t)blk * n_slots_total + tile_off[t] + s) * BO + j] = make_double2(re, im);
  }
}

// c[J][A] = h^3 sum over J's (tile, slot) list, in tile order; hc = h_kb c.
template <typename T, int BO>
__global__ void k_project_pm_reduce(const double2 *__restrict__ partial,
                                    const int *__restrict__ at_ntiles,
                                    const int2 *__restrict__ at_tiles, int cap,
                                    const int *__restrict__ tile_off,
                                    int n_slots_total, int n_orb_pad, double h3,
                                    double h_kb, double2 *c,
                                    typename cplx<T>::type *hc) {
  typedef typename cplx<T>::type V;
  const int J = blockIdx.x;
  const int A = blockIdx.y * blockDim.x + threadIdx.x;
  if (A >= n_orb_pad) return;
  const int blk = A / BO, j = A % BO;
  double re = 0.0, im = 0.0;
  const int m = at_ntiles[J];
  for (int i = 0; i < m; ++i) {
    const int2 ts = at_tiles[(size_t)J * cap + i];
    const double2 v = partial[((size_t)blk * n_slots_total + tile_off[ts.x] + ts.y) * BO + j];
    re += v.x;
    im += v.y;
  }
  const size_t o = (size_t)J * n_orb_pad + A;
  c[o] = make_double2(h3 * re, h3 * im);
  V w;
  w.x = (T)(h_kb * h3 * re);
  w.y = (T)(h_kb * h3 * im);
  hc[o] = w;
}

template <typename T, int BO>
void project_pm_t(const OrbLayout &o, const TableSet &t, int n_atoms, const void *u,
                  double h3, double h_kb, double2 *c, void *hc, double2 *partial,
                  cudaStream_t st) {
  typedef typename cplx<T>::type V;
  const int nt = (o.n + EMD_TILE - 1) / EMD_TILE;
  dim3 grid(nt * nt * nt, o.n_blk);
  k_project_pm<T, BO><<<grid, 512, 0, st>>>((const V *)u, o.n, nt, t.pt_cnt, t.pt_J,
                                           t.pt_p, t.tile_nat, t.tile_atoms,
                                           t.tile_off, t.n_slots_cap, partial);
  dim3 g2(n_atoms, (o.n_orb_pad + 127) / 128);
  k_project_pm_reduce<T, BO><<<g2, 128, 0, st>>>(partial, t.at_ntiles, t.at_tiles,
                                                nt * nt * nt, t.tile_off, t.n_slots_cap,
                                                o.n_orb_pad, h3, h_kb, c, (V *)hc);
}

// ---------------------------------------------------------------------------
// complex64 path: projections and nonlocal forces from the per-tile entry
// lists of the point table.  A small CTA (4 warps) owns one 8^3 tile of one
// orbital block: it stages the tile in shared memory (each point read once
// from HBM), then warp w handles the tile's slots w, w + 4, ...: its lanes
// stride over the slot's entries with FP32 per-lane sums, a fixed shuffle
// tree reduces the warp, and lane 0 writes the slot's FP64 partial, orbital
// index fastest.  Many such CTAs share an SM (16 KB of shared memory each),
// so one CTA's latency chains overlap the others' loads.  A second kernel
// adds each atom's partials over its tiles in a fixed order.
// ---------------------------------------------------------------------------
#define EMD_TG_WARPS 4

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <int NV>
__device__ __forceinline__ void warp_sum(float (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    v[k] = a;
  }
}

// FORCE = false: partial[(tile_off[t] + s) * n_orb_pad + A] = sum p u_A
// FORCE = true:  partial[((tile_off[t] + s) * n_orb_pad + A) * 3 + a]
//                = sum (p d_a / r_c^2) u_A
template <int BO, bool FORCE>
__global__ void __launch_bounds__(EMD_TG_WARPS * 32)
k_tile_gather(const float2 *__restrict__ u, int n, int nt, int n_orb_pad,
              const int *__restrict__ tile_nat, const int *__restrict__ tile_off,
              const int *__restrict__ te_off, const uint2 *__restrict__ te_pp,
              const float4 *__restrict__ te_q,
              double2 *__restrict__ partial) {
  constexpr int NT = EMD_TG_WARPS * 32;
  constexpr int NA = FORCE ? 6 * BO : 2 * BO;
  __shared__ __align__(16) float2 us[512 * BO];
  const int t = blockIdx.x, blk = blockIdx.y;
  const int tx = t % nt, ty = (t / nt) % nt, tz = t / (nt * nt);
  const size_t n3 = (size_t)n * n * n;
  const float2 *ub = u + (size_t)blk * n3 * BO;
  // stage: 512 points, BO float2 each, in 16-byte (8-byte for BO = 1) pieces
  constexpr int PER = BO == 1 ? 1 : BO / 2;          // pieces per point
  for (int q = threadIdx.x; q < 512 * PER; q += NT) {
    const int pt = q / PER, h = q % PER;
    const int x = tx * EMD_TILE + (pt & 7), y = ty * EMD_TILE + ((pt >> 3) & 7),
              z = tz * EMD_TILE + (pt >> 6);
    float2 *dst = us + pt * BO + 2 * h;
    if (x < n && y < n && z < n) {
      const float2 *src = ub + (((size_t)z * n + y) * n + x) * BO + 2 * h;
      if (BO == 1) cp8(dst, src);
      else cp16(dst, src);
    } else {
      dst[0] = make_float2(0.f, 0.f);
      if (BO > 1) dst[1] = make_float2(0.f, 0.f);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const int S = tile_nat[t];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int *off = te_off + (size_t)t * (EMD_TILE_ATOM_MAX + 1);
  const size_t tb = (size_t)t * EMD_TE_CAP;
  const size_t row0 = (size_t)tile_off[t];
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  for (int sl = warp; sl < S; sl += EMD_TG_WARPS) {
    float acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0.f;
    const int e1 = off[sl + 1];
    for (int e = off[sl] + lane; e < e1; e += 32) {
      if (FORCE) {
        const float4 w = __ldg(te_q + tb + e);
        const float4 *v4 = reinterpret_cast<const float4 *>(us + __float_as_int(w.w) * BO);
#pragma unroll
        for (int h = 0; h < (BO + 1) / 2; ++h) {
          const float4 v = BO == 1 ? make_float4(us[__float_as_int(w.w)].x,
                                                 us[__float_as_int(w.w)].y, 0.f, 0.f)
                                   : v4[h];
#pragma unroll
          for (int jj = 0; jj < (BO == 1 ? 1 : 2); ++jj) {
            const int j = 2 * h + jj;
            const float vx = jj ? v.z : v.x, vy = jj ? v.w : v.y;
            acc[6 * j + 0] += w.x * vx;
            acc[6 * j + 1] += w.x * vy;
            acc[6 * j + 2] += w.y * vx;
            acc[6 * j + 3] += w.y * vy;
            acc[6 * j + 4] += w.z * vx;
            acc[6 * j + 5] += w.z * vy;
          }
        }
      } else {
        // up to EU entries of this lane in flight: records first, then the
        // tile values, then the multiply-adds (in entry order)
        constexpr int EU = 4;
        uint2 rec[EU];
#pragma unroll
        for (int u = 0; u < EU; ++u)
          rec[u] = e + 32 * u < e1 ? __ldg(te_pp + tb + e + 32 * u) : make_uint2(0u, 0u);
        float4 vv[EU][(BO + 1) / 2];
#pragma unroll
        for (int u = 0; u < EU; ++u)
#pragma unroll
          for (int h = 0; h < (BO + 1) / 2; ++h)
            vv[u][h] = BO == 1 ? make_float4(us[rec[u].x].x, us[rec[u].x].y, 0.f, 0.f)
                               : reinterpret_cast<const float4 *>(us + rec[u].x * BO)[h];
#pragma unroll
        for (int u = 0; u < EU; ++u) {
          const float pv = __uint_as_float(rec[u].y);   // 0 past the slot's end
#pragma unroll
          for (int h = 0; h < (BO + 1) / 2; ++h)
#pragma unroll
            for (int jj = 0; jj < (BO == 1 ? 1 : 2); ++jj) {
              const int j = 2 * h + jj;
              acc[2 * j] += pv * (jj ? vv[u][h].z : vv[u][h].x);
              acc[2 * j + 1] += pv * (jj ? vv[u][h].w : vv[u][h].y);
            }
        }
        e += 32 * (EU - 1);
      }
    }
    warp_sum<NA>(acc);
    if (lane == 0) {
      double2 *dst = partial + ((row0 + sl) * n_orb_pad + (size_t)blk * BO) * (FORCE ? 3 : 1);
#pragma unroll
      for (int k = 0; k < NA / 2; ++k)
        dst[k] = make_double2((double)acc[2 * k], (double)acc[2 * k + 1]);
    }
  }
}

// c[J][A] = h^3 sum over J's (tile, slot) list; hc = h_kb c.  Block
// (atom, 32 orbitals), 8 warps: warp w adds the list entries i = w mod 8 in
// increasing order (lane = orbital), then the 8 warp sums are added in warp
// order (deterministic).
__global__ void __launch_bounds__(256)
k_project_tile_reduce(const double2 *__restrict__ partial, const int *__restrict__ at_ntiles,
                      const int2 *__restrict__ at_tiles, int cap,
                      const int *__restrict__ tile_off, int n_orb_pad, int n_orb_used,
                      double h3, double h_kb, double2 *c, float2 *hc) {
  __shared__ double2 ws[8][32];
  const int J = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int A = blockIdx.y * 32 + lane;
  const int m = at_ntiles[J];
  double re = 0.0, im = 0.0;
  if (A < n_orb_used) {
#pragma unroll 4
    for (int i = warp; i < m; i += 8) {
      const int2 ts = __ldg(at_tiles + (size_t)J * cap + i);
      const double2 v = partial[((size_t)__ldg(tile_off + ts.x) + ts.y) * n_orb_pad + A];
      re += v.x;
      im += v.y;
    }
  }
  ws[warp][lane] = make_double2(re, im);
  __syncthreads();
  if (warp == 0 && A < n_orb_used) {
    re = 0.0;
    im = 0.0;
    for (int w = 0; w < 8; ++w) {
      re += ws[w][lane].x;
      im += ws[w][lane].y;
    }
    const size_t o = (size_t)J * n_orb_pad + A;
    c[o] = make_double2(h3 * re, h3 * im);
    hc[o] = make_float2((float)(h_kb * h3 * re), (float)(h_kb * h3 * im));
  }
}

// F_J = coef sum_A Re(conj(c_JA) h^3 dc_JA), dc summed over J's tiles in
// tile order; one block per atom, orbitals over threads, fixed-tree sum.
__global__ void __launch_bounds__(128)
k_nl_force_tile_reduce(const double2 *__restrict__ partial, const int *__restrict__ at_ntiles,
                       const int2 *__restrict__ at_tiles, int cap,
                       const int *__restrict__ tile_off, const double2 *__restrict__ c,
                       int n_orb, int n_orb_pad, double h3, double coef, double *F) {
  __shared__ double red[4 * 3];
  const int J = blockIdx.x;
  const int m = at_ntiles[J];
  double f[3] = {0.0, 0.0, 0.0};
  for (int A = threadIdx.x; A < n_orb; A += blockDim.x) {
    double dr[3] = {0.0, 0.0, 0.0}, di[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < m; ++i) {
      const int2 ts = at_tiles[(size_t)J * cap + i];
      const double2 *v = partial + (((size_t)tile_off[ts.x] + ts.y) * n_orb_pad + A) * 3;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dr[a] += v[a].x;
        di[a] += v[a].y;
      }
    }
    const double2 cj = c[(size_t)J * n_orb_pad + A];
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] += cj.x * (h3 * dr[a]) + cj.y * (h3 * di[a]);
  }
  emd_block_sum<3>(f, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) F[3 * J + a] = coef * f[a];
}

template <int BO, bool FORCE>
void tile_gather_t(const OrbLayout &o, const TableSet &t, const void *u, double2 *partial,
                   cudaStream_t st) {
  const int nt = (o.n + EMD_TILE - 1) / EMD_TILE;
  dim3 grid(nt * nt * nt, o.n_blk);
  k_tile_gather<BO, FORCE><<<grid, EMD_TG_WARPS * 32, 0, st>>>(
      (const float2 *)u, o.n, nt, o.n_orb_pad, t.tile_nat, t.tile_off, t.te_off, t.te_pp,
      t.te_q, partial);
}

}  // namespace

void emd_launch_tile_atoms(const GridInfo &g, int n_atoms, TableSet &t, int *err,
                           cudaStream_t st) {
  const int nt = (g.n + EMD_TILE - 1) / EMD_TILE;
  const int ntiles = nt * nt * nt;
  emd_note_launches(2 + (n_atoms > 0));
  k_tile_atoms<<<(ntiles + 127) / 128, 128, 0, st>>>(t.tile_cnt, t.tile_ent, ntiles,
                                                     t.tile_nat, t.tile_atoms, err);
  k_tile_offsets<<<1, 1024, 0, st>>>(t.tile_nat, ntiles, t.tile_off);
  if (n_atoms > 0)
    k_atom_tiles<<<n_atoms, 256, 0, st>>>(t.tile_nat, t.tile_atoms, ntiles, ntiles,
                                          t.at_ntiles, t.at_tiles, err);
}

void emd_launch_project_pm(const OrbLayout &o, const TableSet &t, int n_atoms,
                           const void *u, double h3, double h_kb, double2 *c,
                           void *hc, double2 *partial, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  if (o.prec == EMD_FP64) {
    switch (o.bo) {
      case 1: project_pm_t<double, 1>(o, t, n_atoms, u, h3, h_kb, c, hc, partial, st); break;
      case 2: project_pm_t<double, 2>(o, t, n_atoms, u, h3, h_kb, c, hc, partial, st); break;
      case 4: project_pm_t<double, 4>(o, t, n_atoms, u, h3, h_kb, c, hc, partial, st); break;
    }
  } else {
    switch (o.bo) {
      case 1: project_pm_t<float, 1>(o, t, n_atoms, u, h3, h_kb, c, hc, partial, st); break;
      case 2: project_pm_t<float, 2>(o, t, n_atoms, u, h3, h_kb, c, hc, partial, st); break;
      case 4: project_pm_t<float, 4>(o, t, n_atoms, u, h3, h_kb, c, hc, partial, st); break;
    }
  }
}

void emd_launch_project_tile(const OrbLayout &o, const TableSet &t, int n_atoms,
                             const void *u, double h3, double h_kb, double2 *c,
                             void *hc, double2 *partial, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  switch (o.bo) {
    case 1: tile_gather_t<1, false>(o, t, u, partial, st); break;
    case 2: tile_gather_t<2, false>(o, t, u, partial, st); break;
    case 4: tile_gather_t<4, false>(o, t, u, partial, st); break;
  }
  const int nt = (o.n + EMD_TILE - 1) / EMD_TILE;
  const int used = o.n_blk * o.bo;
  dim3 g2(n_atoms, (used + 31) / 32);
  k_project_tile_reduce<<<g2, 256, 0, st>>>(partial, t.at_ntiles, t.at_tiles, nt * nt * nt,
                                           t.tile_off, o.n_orb_pad, used, h3, h_kb, c,
                                           (float2 *)hc);
}

void emd_launch_nl_force_tile(const OrbLayout &o, const TableSet &t, int n_atoms,
                              const void *u, const double2 *c, double h3, double coef,
                              double2 *partial, double *F_nl, cudaStream_t st) {
  if (n_atoms <= 0) return;
  emd_note_launches(2);
  switch (o.bo) {
    case 1: tile_gather_t<1, true>(o, t, u, partial, st); break;
    case 2: tile_gather_t<2, true>(o, t, u, partial, st); break;
    case 4: tile_gather_t<4, true>(o, t, u, partial, st); break;
  }
  const int nt = (o.n + EMD_TILE - 1) / EMD_TILE;
  k_nl_force_tile_reduce<<<n_atoms, 128, 0, st>>>(partial, t.at_ntiles, t.at_tiles,
                                                 nt * nt * nt, t.tile_off, c, o.n_orb,
                                                 o.n_orb_pad, h3, coef, F_nl);
}
