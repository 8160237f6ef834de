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
