// C ABI of libemd: validation, device memory, and the order of operations of
// one molecular-dynamics step of the modified Ehrenfest scheme.
//
// Step (paper Sec. 5.1; eq. aetrs, eq. transf, eq. new_EoM):
//   1. R(t+dt) = R + V dt + F dt^2/(2M)                     (velocity Verlet)
//   2. ionic potential and projector tables at R(t+dt)      (eq. ionicpotential)
//   3. H1 = H[R(t), v_Hxc(t)], H2 = H[R(t+dt), extrapolated v_Hxc]
//   4. psi <- T4(-i tau H2) T4(-i tau H1) psi, tau = dt/(2 mu)   (AETRS)
//   5. rho, v_H, v_xc at t+dt                               (eq. density)
//   6. F(t+dt) = -dE_KS/dR; V += (F(t) + F(t+dt)) dt/(2M)
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>
#include "emd_internal.cuh"

namespace {

thread_local std::string g_err;
std::atomic<long long> g_launches{0};

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                             \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return fail(EMD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

double fd_weight(int order, int k) {
  // central second-derivative weights (Fornberg), k = 0..order/2
  static const double w2[] = {-2.0, 1.0};
  static const double w4[] = {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0};
  static const double w6[] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
  static const double w8[] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                              -1.0 / 560.0};
  switch (order) {
    case 2: return w2[k];
    case 4: return w4[k];
    case 6: return w6[k];
    default: return w8[k];
  }
}

}  // namespace

void emd_note_launches(int k) { g_launches += k; }

struct emd_system {
  emd_config cfg;
  GridInfo g;
  SpeciesDev sp;
  OrbLayout o;
  cudaStream_t st = nullptr;
  int n_atoms = 0;
  size_t orb_bytes = 0;
  void *psi = nullptr, *ua = nullptr, *ub = nullptr;
  double2 *stage_buf = nullptr;   // canonical staging for one orbital block
  double *veff1 = nullptr, *veff2 = nullptr;
  float *veff1f = nullptr, *veff2f = nullptr;
  double *hist[3] = {nullptr, nullptr, nullptr};
  int hist_len = 0;
  double *rho = nullptr, *v_h = nullptr, *v_xc = nullptr, *eps_xc = nullptr;
  double *neg = nullptr;          // scratch grid
  double2 *fft_a = nullptr, *fft_b = nullptr;
  TableSet ts[2];
  int cur = 0;
  double2 *c = nullptr;
  void *hc = nullptr;
  int c_valid = 0;
  double *V = nullptr, *F = nullptr, *F_loc = nullptr, *F_nl = nullptr,
         *F_sr = nullptr, *e_sr = nullptr, *nl_part = nullptr;
  double *partials = nullptr;
  int n_partials = 0;
  double *scal = nullptr;
  int *err = nullptr;
  int ions_set = 0, orbs_set = 0;
  int frozen_ions = 0, profile = 0, check_stable = 1;
  double v_max = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending, prof_free;
  double prof_ms = 0.0;
  long long prof_launches = 0;
  std::vector<void *> allocs;
};

namespace {

int dalloc(emd_system *s, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(EMD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes,
                cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  return EMD_OK;
}

#define DALLOC(ptr, bytes)                                              \
  do {                                                                  \
    int r_ = dalloc(s, (void **)&(ptr), (bytes));                       \
    if (r_) return r_;                                                  \
  } while (0)

int launch_check(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(EMD_ECUDA, "%s: kernel launch failed: %s", what,
                cudaGetErrorString(e));
  return EMD_OK;
}

int read_err_flag(emd_system *s) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (h)
    return fail(EMD_ETABLE,
                "atom list overflow (bits %d: 1 point list > %d atoms, 2 tile "
                "candidates > %d, 4 atom table)",
                h, EMD_PT_KMAX, EMD_TILE_CAND_MAX);
  return EMD_OK;
}

// Build every table of set k from ts[k].R.
int build_set(emd_system *s, int k) {
  TableSet &t = s->ts[k];
  emd_launch_wrap(t.R, t.Rw, s->n_atoms, s->g.L, s->st);
  emd_launch_tables(s->g, s->sp, s->n_atoms, t, s->err, s->st);
  // v_loc = Poisson(-g): solve for g, negate in the final pass
  emd_launch_poisson(s->g, t.g_ion, t.v_loc, s->fft_a, s->fft_b, s->st);
  return launch_check("build_set");
}

void negate_grid(double *v, int n3, cudaStream_t st);

void project(emd_system *s, const void *u, int set) {
  emd_launch_project(s->o, s->ts[set], s->n_atoms, u, s->g.h * s->g.h * s->g.h,
                     s->sp.h_kb, s->c, s->hc, s->st);
}

void stage(emd_system *s, const void *u_in, const void *psi0, void *u_out,
           int set, int which_veff, double a) {
  StageArgs a_;
  a_.u_in = u_in;
  a_.psi0 = psi0;
  a_.u_out = u_out;
  if (s->o.prec == EMD_FP64)
    a_.v_eff = which_veff == 1 ? (const void *)s->veff1 : (const void *)s->veff2;
  else
    a_.v_eff = which_veff == 1 ? (const void *)s->veff1f : (const void *)s->veff2f;
  a_.tab = &s->ts[set];
  a_.hc = s->hc;
  a_.a = a;
  a_.apply_only = 0;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (s->profile) {
    if (!s->prof_free.empty()) {
      ev = s->prof_free.back();
      s->prof_free.pop_back();
    } else {
      cudaEventCreate(&ev.first);
      cudaEventCreate(&ev.second);
    }
    cudaEventRecord(ev.first, s->st);
  }
  emd_launch_stage(s->o, a_, s->st);
  if (s->profile) {
    cudaEventRecord(ev.second, s->st);
    s->prof_pending.push_back(ev);
  }
}

// One exponential T4(-i tau H) psi0 -> out, H given by (set, veff).
// Requires hc to hold the projections of psi0 at `set` on entry.
void exponential(emd_system *s, void *psi0, void *w1, void *out, int set,
                 int which_veff, double tau) {
  stage(s, psi0, psi0, w1, set, which_veff, tau / 4.0);
  project(s, w1, set);
  stage(s, w1, psi0, out, set, which_veff, tau / 3.0);
  project(s, out, set);
  stage(s, out, psi0, w1, set, which_veff, tau / 2.0);
  project(s, w1, set);
  stage(s, w1, psi0, out, set, which_veff, tau);
}

// rho, v_H, v_xc of psi into hist slot `slot`.
void electrons(emd_system *s, int slot) {
  emd_launch_density(s->o, s->psi, s->cfg.occ, s->rho, s->st);
  emd_launch_poisson(s->g, s->rho, s->v_h, s->fft_a, s->fft_b, s->st);
  emd_launch_lda(s->g.n3, s->rho, s->v_h, s->eps_xc, s->v_xc, s->hist[slot],
                 s->st);
}

// Forces at set k (projections of psi at k must be in c).
void forces(emd_system *s, int k, double field, double dt, int update_v) {
  emd_launch_local_force(s->g, s->sp, s->n_atoms, s->ts[k].Rw, s->v_h,
                         s->ts[k].v_loc, s->F_loc, s->st);
  emd_launch_nl_force(s->o, s->ts[k], s->n_atoms, s->psi, s->c,
                      s->g.h * s->g.h * s->g.h,
                      -2.0 * s->sp.h_kb * s->cfg.occ, s->sp.inv_rc2,
                      s->nl_part, s->F_nl, s->st);
  emd_launch_short_range(s->sp, s->n_atoms, s->ts[k].Rw, s->g.L, s->F_sr,
                         s->e_sr, s->st);
  emd_launch_vv_velocities(s->n_atoms, s->F_loc, s->F_nl, s->F_sr, field,
                           s->sp.z, s->F, s->V, dt, s->sp.mass, update_v,
                           s->st);
}

int reduce_max_veff(emd_system *s, double *out);

// After new orbitals or ions: rho(0), v_Hxc(0), F(0); history restarts.
int restart_dynamics(emd_system *s) {
  electrons(s, 0);
  s->hist_len = 1;
  project(s, s->psi, s->cur);
  s->c_valid = 1;
  forces(s, s->cur, 0.0, 0.0, 0);
  int r = launch_check("restart_dynamics");
  if (r) return r;
  return reduce_max_veff(s, &s->v_max);
}

double kinetic_lambda_max(int order) {
  // max over theta of -(c0 + 2 sum c_k cos k theta), attained at theta = pi
  double s = fd_weight(order, 0);
  for (int k = 1; k <= order / 2; ++k) s += 2.0 * fd_weight(order, k) * (k % 2 ? -1.0 : 1.0);
  return -s;
}

}  // namespace

// ---------------------------------------------------------------------------
// small helper kernels local to this file
// ---------------------------------------------------------------------------
namespace {
__global__ void k_negate(double *v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = -v[i];
}
__global__ void k_max_sum(const double *a, const double *b, int n, double *out) {
  __shared__ double sm[256];
  double m = -1e300;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, a[i] + b[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}
void negate_grid(double *v, int n3, cudaStream_t st) {
  emd_note_launches(1);
  k_negate<<<(n3 + 255) / 256, 256, 0, st>>>(v, n3);
}
int reduce_max_veff(emd_system *s, double *out) {
  emd_note_launches(1);
  k_max_sum<<<1, 256, 0, s->st>>>(s->hist[0], s->ts[s->cur].v_loc, s->g.n3,
                                   s->scal + 15);
  CK(cudaMemcpyAsync(out, s->scal + 15, sizeof(double), cudaMemcpyDeviceToHost,
                     s->st));
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}
}  // namespace

extern "C" {

const char *emd_last_error(void) { return g_err.c_str(); }
const char *emd_version(void) { return "libemd 0.1 (sm_103a)"; }

int emd_init_system(const emd_config *cfg, emd_system **out) {
  g_err.clear();
  if (!cfg || !out) return fail(EMD_EINVAL, "NULL argument");
  *out = nullptr;
  const emd_config &c = *cfg;
  if (c.fd_order != 2 && c.fd_order != 4 && c.fd_order != 6 && c.fd_order != 8)
    return fail(EMD_EINVAL, "fd_order must be 2, 4, 6 or 8 (got %d)", c.fd_order);
  if (c.n < 8 || c.n > 1024 || c.n < 2 * c.fd_order)
    return fail(EMD_EINVAL, "n must be in [max(8, 2*fd_order), 1024] (got %d)", c.n);
  if (!(c.h > 0.0) || !std::isfinite(c.h)) return fail(EMD_EINVAL, "h must be > 0");
  if (c.n_orb < 1) return fail(EMD_EINVAL, "n_orb must be >= 1");
  if (!(c.occ > 0.0)) return fail(EMD_EINVAL, "occ must be > 0");
  if (c.precision != EMD_FP64 && c.precision != EMD_FP32_ORBITALS)
    return fail(EMD_EINVAL, "precision must be EMD_FP64 or EMD_FP32_ORBITALS");
  if (c.n_atoms < 0) return fail(EMD_EINVAL, "n_atoms must be >= 0");
  const emd_species &p = c.species;
  const double L = c.n * c.h;
  if (c.n_atoms > 0) {
    if (!(p.a_loc > 0) || !(p.r_c > 0) || !(p.mass > 0) || !(p.r_loc > 0) ||
        !(p.r_proj > 0))
      return fail(EMD_EINVAL, "species widths, radii and mass must be > 0");
    if (p.r_loc > L || p.r_proj > L)
      return fail(EMD_EINVAL, "support radii (%g, %g) exceed the box length %g",
                  p.r_loc, p.r_proj, L);
  }
  int ok = 0;
  emd_fft_plan_check(c.n, &ok);
  if (!ok) return fail(EMD_EINVAL, "n = %d has a prime factor above 13", c.n);
  if (c.block_orbitals != 0 && c.block_orbitals != 1 && c.block_orbitals != 2 &&
      c.block_orbitals != 4)
    return fail(EMD_EINVAL, "block_orbitals must be 0, 1, 2 or 4");

  if (emd_fft_prepare(c.n))
    return fail(EMD_ENOMEM, "FFT twiddle tables for n = %d: %s", c.n,
                cudaGetErrorString(cudaGetLastError()));
  emd_system *s = new emd_system();
  s->cfg = c;
  s->st = (cudaStream_t)c.cuda_stream;
  s->n_atoms = c.n_atoms;
  s->g.n = c.n;
  s->g.n3 = c.n * c.n * c.n;
  s->g.h = c.h;
  s->g.L = L;
  s->sp.z = p.z;
  s->sp.mass = p.mass;
  s->sp.a_loc = p.a_loc;
  s->sp.r_loc = p.r_loc;
  s->sp.r_c = p.r_c;
  s->sp.h_kb = p.h_kb;
  s->sp.r_proj = p.r_proj;
  s->sp.c_g = c.n_atoms ? p.z * pow(M_PI, -1.5) * pow(p.a_loc, -3.0) : 0.0;
  s->sp.c_p = c.n_atoms ? pow(M_PI, -0.75) * pow(p.r_c, -1.5) : 0.0;
  s->sp.inv_a2 = c.n_atoms ? 1.0 / (p.a_loc * p.a_loc) : 0.0;
  s->sp.inv_2rc2 = c.n_atoms ? 1.0 / (2.0 * p.r_c * p.r_c) : 0.0;
  s->sp.inv_rc2 = c.n_atoms ? 1.0 / (p.r_c * p.r_c) : 0.0;

  OrbLayout &o = s->o;
  o.n = c.n;
  o.n3 = s->g.n3;
  o.h = c.h;
  o.prec = c.precision;
  o.bo = c.block_orbitals ? c.block_orbitals : (c.precision == EMD_FP64 ? 2 : 4);
  o.n_orb = c.n_orb;
  o.n_blk = (c.n_orb + o.bo - 1) / o.bo;
  o.n_orb_pad = o.n_blk * o.bo;
  o.half_order = c.fd_order / 2;
  for (int k = 0; k <= EMD_MAX_HALF_ORDER; ++k) o.w[k] = 0.0;
  o.w[0] = -1.5 * fd_weight(c.fd_order, 0) / (c.h * c.h);
  for (int k = 1; k <= o.half_order; ++k)
    o.w[k] = -0.5 * fd_weight(c.fd_order, k) / (c.h * c.h);

  const size_t n3 = s->g.n3;
  const size_t esz = c.precision == EMD_FP64 ? sizeof(double2) : sizeof(float2);
  s->orb_bytes = (size_t)o.n_blk * n3 * o.bo * esz;
  int r = 0;
#define TRY(x) do { r = (x); if (r) { emd_destroy(s); return r; } } while (0)
  auto A = [&](void **ptr, size_t bytes) { return dalloc(s, ptr, bytes); };
  TRY(A(&s->psi, s->orb_bytes));
  TRY(A(&s->ua, s->orb_bytes));
  TRY(A(&s->ub, s->orb_bytes));
  TRY(A((void **)&s->stage_buf, (size_t)o.bo * n3 * sizeof(double2)));
  TRY(A((void **)&s->veff1, n3 * 8));
  TRY(A((void **)&s->veff2, n3 * 8));
  if (c.precision != EMD_FP64) {
    TRY(A((void **)&s->veff1f, n3 * 4));
    TRY(A((void **)&s->veff2f, n3 * 4));
  }
  for (int k = 0; k < 3; ++k) TRY(A((void **)&s->hist[k], n3 * 8));
  TRY(A((void **)&s->rho, n3 * 8));
  TRY(A((void **)&s->v_h, n3 * 8));
  TRY(A((void **)&s->v_xc, n3 * 8));
  TRY(A((void **)&s->eps_xc, n3 * 8));
  TRY(A((void **)&s->neg, n3 * 8));
  TRY(A((void **)&s->fft_a, n3 * 16));
  TRY(A((void **)&s->fft_b, n3 * 16));
  const int nt = (c.n + EMD_TILE - 1) / EMD_TILE;
  const int ntiles = nt * nt * nt;
  const int na = std::max(1, c.n_atoms);
  // atom-table capacity: every (point, image) pair within r_proj
  const int ext = 2 * (int)std::ceil(p.r_proj / c.h) + 3;
  const long cube = (long)ext * ext * ext;
  long cap = (L > 2.0 * p.r_proj) ? std::min<long>((long)n3, cube)
                                  : std::min<long>(8L * (long)n3, 27L * cube);
  if (c.n_atoms == 0) cap = 1;
  for (int k = 0; k < 2; ++k) {
    TableSet &t = s->ts[k];
    t.cap = (int)cap;
    TRY(A((void **)&t.R, na * 3 * 8));
    TRY(A((void **)&t.Rw, na * 3 * 8));
    TRY(A((void **)&t.tile_cnt, ntiles * 4));
    TRY(A((void **)&t.tile_ent, (size_t)ntiles * EMD_TILE_CAND_MAX * 4));
    TRY(A((void **)&t.pt_cnt, n3 * 4));
    TRY(A((void **)&t.pt_J, n3 * EMD_PT_KMAX * 4));
    TRY(A((void **)&t.pt_p, n3 * EMD_PT_KMAX * 8));
    TRY(A((void **)&t.at_cnt, na * 4));
    TRY(A((void **)&t.at_pt, (size_t)na * cap * 4));
    TRY(A((void **)&t.at_p, (size_t)na * cap * 8));
    TRY(A((void **)&t.at_d, (size_t)na * cap * 24));
    TRY(A((void **)&t.g_ion, n3 * 8));
    TRY(A((void **)&t.v_loc, n3 * 8));
  }
  TRY(A((void **)&s->c, (size_t)na * o.n_orb_pad * sizeof(double2)));
  TRY(A(&s->hc, (size_t)na * o.n_orb_pad * esz));
  TRY(A((void **)&s->V, na * 3 * 8));
  TRY(A((void **)&s->F, na * 3 * 8));
  TRY(A((void **)&s->F_loc, na * 3 * 8));
  TRY(A((void **)&s->F_nl, na * 3 * 8));
  TRY(A((void **)&s->F_sr, na * 3 * 8));
  TRY(A((void **)&s->e_sr, na * 8));
  TRY(A((void **)&s->nl_part, (size_t)na * o.n_blk * 3 * 8));
  s->n_partials = std::max(1024, (int)((n3 + 255) / 256));
  TRY(A((void **)&s->partials, (size_t)s->n_partials * 8));
  TRY(A((void **)&s->scal, 16 * 8));
  TRY(A((void **)&s->err, sizeof(int)));
#undef TRY
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->V, 0, na * 3 * 8, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->F, 0, na * 3 * 8, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->c, 0, (size_t)na * o.n_orb_pad * 16, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->hc, 0, (size_t)na * o.n_orb_pad * esz, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) {
    emd_destroy(s);
    return fail(EMD_ECUDA, "initialisation: %s", cudaGetErrorString(e));
  }
  *out = s;
  return EMD_OK;
}

int emd_set_ions(emd_system *s, int n_atoms, const double *R, const double *V) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  if (n_atoms != s->n_atoms)
    return fail(EMD_EINVAL, "n_atoms %d differs from the configured %d", n_atoms,
                s->n_atoms);
  if (n_atoms > 0 && (!R || !V)) return fail(EMD_EINVAL, "NULL R or V");
  for (int i = 0; i < 3 * n_atoms; ++i)
    if (!std::isfinite(R[i]) || !std::isfinite(V[i]))
      return fail(EMD_EINVAL, "non-finite position or velocity");
  TableSet &t = s->ts[s->cur];
  if (n_atoms > 0) {
    CK(cudaMemcpyAsync(t.R, R, 3 * n_atoms * 8, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->V, V, 3 * n_atoms * 8, cudaMemcpyHostToDevice, s->st));
  }
  int r = build_set(s, s->cur);
  if (r) return r;
  negate_grid(t.v_loc, s->g.n3, s->st);
  s->ions_set = 1;
  if (s->orbs_set) return restart_dynamics(s);
  CK(cudaStreamSynchronize(s->st));
  return launch_check("emd_set_ions");
}

static int upload_orbitals(emd_system *s, const double *psi, int n_vec,
                           void *dst) {
  const size_t n3 = s->g.n3;
  for (int b = 0; b * s->o.bo < n_vec; ++b) {
    const int nv = std::min(s->o.bo, n_vec - b * s->o.bo);
    CK(cudaMemcpyAsync(s->stage_buf, psi + 2 * (size_t)b * s->o.bo * n3,
                       (size_t)nv * n3 * 16, cudaMemcpyHostToDevice, s->st));
    OrbLayout one = s->o;
    char *d = (char *)dst + (size_t)b * n3 * s->o.bo *
                                (s->o.prec == EMD_FP64 ? 16 : 8);
    emd_launch_pack(one, s->stage_buf, d, nv, s->st);
  }
  // zero the padding orbitals of the last block and any unused blocks
  return launch_check("upload_orbitals");
}

static int download_orbitals(emd_system *s, const void *src, int n_vec,
                             double *psi) {
  const size_t n3 = s->g.n3;
  for (int b = 0; b * s->o.bo < n_vec; ++b) {
    const int nv = std::min(s->o.bo, n_vec - b * s->o.bo);
    const char *d = (const char *)src + (size_t)b * n3 * s->o.bo *
                                            (s->o.prec == EMD_FP64 ? 16 : 8);
    emd_launch_unpack(s->o, d, s->stage_buf, nv, s->st);
    CK(cudaMemcpyAsync(psi + 2 * (size_t)b * s->o.bo * n3, s->stage_buf,
                       (size_t)nv * n3 * 16, cudaMemcpyDeviceToHost, s->st));
  }
  CK(cudaStreamSynchronize(s->st));
  return launch_check("download_orbitals");
}

int emd_set_orbitals(emd_system *s, const double *psi) {
  g_err.clear();
  if (!s || !psi) return fail(EMD_EINVAL, "NULL argument");
  CK(cudaMemsetAsync(s->psi, 0, s->orb_bytes, s->st));
  int r = upload_orbitals(s, psi, s->o.n_orb, s->psi);
  if (r) return r;
  s->orbs_set = 1;
  if (s->ions_set) return restart_dynamics(s);
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}

int emd_set_option(emd_system *s, int option, double value) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  switch (option) {
    case EMD_OPT_FROZEN_IONS: s->frozen_ions = value != 0.0; return EMD_OK;
    case EMD_OPT_PROFILE: s->profile = value != 0.0; return EMD_OK;
    case EMD_OPT_CHECK_STABLE: s->check_stable = value != 0.0; return EMD_OK;
  }
  return fail(EMD_EINVAL, "unknown option %d", option);
}

int emd_propagate(emd_system *s, int n_steps, double dt, double mu,
                  const double *field) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  if (!s->ions_set || !s->orbs_set)
    return fail(EMD_ESTATE, "set ions and orbitals before propagating");
  if (n_steps < 0) return fail(EMD_EINVAL, "n_steps must be >= 0");
  if (!(dt > 0.0) || !(mu > 0.0) || !std::isfinite(dt) || !std::isfinite(mu))
    return fail(EMD_EINVAL, "dt and mu must be finite and > 0");
  if (field)
    for (int i = 0; i < n_steps; ++i)
      if (!std::isfinite(field[i])) return fail(EMD_EINVAL, "non-finite field");
  const double tau = 0.5 * (dt / mu);
  if (s->check_stable) {
    const double lam = 1.5 * kinetic_lambda_max(s->cfg.fd_order) / (s->g.h * s->g.h) +
                       std::max(0.0, s->v_max) + std::max(0.0, s->sp.h_kb);
    const double x = tau * lam;
    if (x > 2.0 * std::sqrt(2.0))
      return fail(EMD_EUNSTABLE,
                  "tau*lambda_max = %.3f exceeds the Taylor-4 stability bound "
                  "2*sqrt(2) (tau = dt/(2 mu) = %g, lambda_max ~ %.2f)",
                  x, tau, lam);
  }
  for (int step = 0; step < n_steps; ++step) {
    const double e = field ? field[step] : 0.0;
    const int cur = s->cur;
    const int nw = s->frozen_ions ? cur : 1 - cur;
    if (!s->frozen_ions) {
      emd_launch_vv_positions(s->n_atoms, s->ts[cur].R, s->V, s->F, dt,
                              s->sp.mass, s->ts[nw].R, s->st);
      int r = build_set(s, nw);
      if (r) return r;
      negate_grid(s->ts[nw].v_loc, s->g.n3, s->st);
    }
    emd_launch_veff(s->g, s->ts[cur].v_loc, s->hist, 1, e, s->veff1, s->veff1f,
                    s->st);
    emd_launch_veff(s->g, s->ts[nw].v_loc, s->hist, s->hist_len, e, s->veff2,
                    s->veff2f, s->st);
    if (!s->c_valid) project(s, s->psi, cur);
    // exponential 1: psi -> ub with H(t)
    exponential(s, s->psi, s->ua, s->ub, cur, 1, tau);
    project(s, s->ub, nw);
    // exponential 2: ub -> psi with H(t+dt)
    exponential(s, s->ub, s->ua, s->psi, nw, 2, tau);
    // new density and potentials; history slot of the oldest entry
    double *oldest = s->hist[2];
    s->hist[2] = s->hist[1];
    s->hist[1] = s->hist[0];
    s->hist[0] = oldest;
    electrons(s, 0);
    s->hist_len = std::min(3, s->hist_len + 1);
    if (!s->frozen_ions) {
      project(s, s->psi, nw);
      forces(s, nw, e, dt, 1);
      s->cur = nw;
      s->c_valid = 1;
    } else {
      s->c_valid = 0;
    }
    int r = launch_check("emd_propagate");
    if (r) return r;
  }
  return EMD_OK;
}

int emd_get_forces(emd_system *s, double *F) {
  g_err.clear();
  if (!s || (!F && s->n_atoms)) return fail(EMD_EINVAL, "NULL argument");
  int r = read_err_flag(s);
  if (r) return r;
  if (s->n_atoms) {
    CK(cudaMemcpyAsync(F, s->F, 3 * s->n_atoms * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
  }
  return EMD_OK;
}

int emd_get_energy(emd_system *s, emd_energy *out) {
  g_err.clear();
  if (!s || !out) return fail(EMD_EINVAL, "NULL argument");
  if (!s->ions_set || !s->orbs_set)
    return fail(EMD_ESTATE, "set ions and orbitals first");
  const int cur = s->cur;
  const double h3 = s->g.h * s->g.h * s->g.h;
  int np = 0;
  emd_launch_kinetic_partials(s->o, s->psi, s->partials, &np, s->st);
  emd_launch_sum(s->partials, np, s->scal + 0, s->st);
  if (!s->c_valid) {
    project(s, s->psi, cur);
    s->c_valid = 1;
  }
  emd_launch_abs2_sum(s->c, s->n_atoms * s->o.n_orb_pad, s->scal + 1, s->st);
  const int nb = std::min(s->n_partials, 1024);
  emd_launch_dot_partials(s->g.n3, s->rho, s->v_h, s->ts[cur].g_ion,
                          s->ts[cur].v_loc, s->partials, nb, s->st);
  emd_launch_sum(s->partials, nb, s->scal + 2, s->st);
  emd_launch_short_range(s->sp, s->n_atoms, s->ts[cur].Rw, s->g.L, s->F_sr,
                         s->e_sr, s->st);
  emd_launch_sum(s->e_sr, s->n_atoms, s->scal + 3, s->st);
  emd_launch_dot_partials(s->g.n3, s->rho, s->eps_xc, nullptr, nullptr,
                          s->partials, nb, s->st);
  emd_launch_sum(s->partials, nb, s->scal + 4, s->st);
  emd_launch_dot_partials(s->g.n3, s->rho, nullptr, nullptr, nullptr,
                          s->partials, nb, s->st);
  emd_launch_sum(s->partials, nb, s->scal + 5, s->st);
  int r = launch_check("emd_get_energy");
  if (r) return r;
  double hs[6];
  std::vector<double> V(3 * std::max(1, s->n_atoms));
  CK(cudaMemcpyAsync(hs, s->scal, sizeof hs, cudaMemcpyDeviceToHost, s->st));
  if (s->n_atoms)
    CK(cudaMemcpyAsync(V.data(), s->V, 3 * s->n_atoms * 8, cudaMemcpyDeviceToHost,
                       s->st));
  CK(cudaStreamSynchronize(s->st));
  r = read_err_flag(s);
  if (r) return r;
  const double occ = s->cfg.occ;
  out->kin_e = occ * h3 * hs[0];
  out->nl = occ * s->sp.h_kb * hs[1];
  out->sr = s->n_atoms ? hs[3] : 0.0;
  const double self = s->n_atoms * s->sp.z * s->sp.z /
                      (std::sqrt(2.0 * M_PI) * (s->n_atoms ? s->sp.a_loc : 1.0));
  out->es = 0.5 * h3 * hs[2] - (s->n_atoms ? self : 0.0) + out->sr;
  out->xc = h3 * hs[4];
  out->n_elec = h3 * hs[5];
  double t = 0.0;
  for (int i = 0; i < 3 * s->n_atoms; ++i) t += V[i] * V[i];
  out->kin_ion = 0.5 * s->sp.mass * t;
  out->ks = out->kin_e + out->nl + out->es + out->xc;
  out->total = out->ks + out->kin_ion;
  if (!std::isfinite(out->total) ||
      std::fabs(out->n_elec - occ * s->o.n_orb) > 1e-3 * occ * s->o.n_orb)
    return fail(EMD_EUNSTABLE, "density normalisation lost: h^3 sum rho = %g, "
                "expected %g", out->n_elec, occ * s->o.n_orb);
  return EMD_OK;
}

int emd_get_state(emd_system *s, double *R, double *V, double *psi, double *rho) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  int r = read_err_flag(s);
  if (r) return r;
  if (R && s->n_atoms)
    CK(cudaMemcpyAsync(R, s->ts[s->cur].R, 3 * s->n_atoms * 8,
                       cudaMemcpyDeviceToHost, s->st));
  if (V && s->n_atoms)
    CK(cudaMemcpyAsync(V, s->V, 3 * s->n_atoms * 8, cudaMemcpyDeviceToHost, s->st));
  if (rho)
    CK(cudaMemcpyAsync(rho, s->rho, s->g.n3 * 8, cudaMemcpyDeviceToHost, s->st));
  if (psi) {
    r = download_orbitals(s, s->psi, s->o.n_orb, psi);
    if (r) return r;
  }
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}

int emd_get_potentials(emd_system *s, double *v_loc, double *v_h, double *v_xc,
                       double *g_ion) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  const size_t b = (size_t)s->g.n3 * 8;
  if (v_loc) CK(cudaMemcpyAsync(v_loc, s->ts[s->cur].v_loc, b, cudaMemcpyDeviceToHost, s->st));
  if (v_h) CK(cudaMemcpyAsync(v_h, s->v_h, b, cudaMemcpyDeviceToHost, s->st));
  if (v_xc) CK(cudaMemcpyAsync(v_xc, s->v_xc, b, cudaMemcpyDeviceToHost, s->st));
  if (g_ion) CK(cudaMemcpyAsync(g_ion, s->ts[s->cur].g_ion, b, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return read_err_flag(s);
}

int emd_get_projections(emd_system *s, double *c) {
  g_err.clear();
  if (!s || !c) return fail(EMD_EINVAL, "NULL argument");
  if (!s->orbs_set || !s->ions_set) return fail(EMD_ESTATE, "set ions and orbitals first");
  if (!s->c_valid) {
    project(s, s->psi, s->cur);
    s->c_valid = 1;
  }
  for (int J = 0; J < s->n_atoms; ++J)
    CK(cudaMemcpyAsync(c + 2 * (size_t)J * s->o.n_orb, s->c + (size_t)J * s->o.n_orb_pad,
                       (size_t)s->o.n_orb * 16, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return read_err_flag(s);
}

int emd_apply_hamiltonian(emd_system *s, int n_vec, const double *psi,
                          double *hpsi) {
  g_err.clear();
  if (!s || !psi || !hpsi) return fail(EMD_EINVAL, "NULL argument");
  if (n_vec < 1 || n_vec > s->o.n_orb)
    return fail(EMD_EINVAL, "n_vec must be in [1, n_orb]");
  if (!s->ions_set || !s->orbs_set) return fail(EMD_ESTATE, "set ions and orbitals first");
  CK(cudaMemsetAsync(s->ua, 0, s->orb_bytes, s->st));
  int r = upload_orbitals(s, psi, n_vec, s->ua);
  if (r) return r;
  OrbLayout o = s->o;
  o.n_blk = (n_vec + o.bo - 1) / o.bo;
  emd_launch_veff(s->g, s->ts[s->cur].v_loc, s->hist, 1, 0.0, s->veff1,
                  s->veff1f, s->st);
  emd_launch_project(o, s->ts[s->cur], s->n_atoms, s->ua,
                     s->g.h * s->g.h * s->g.h, s->sp.h_kb, s->c, s->hc, s->st);
  s->c_valid = 0;
  StageArgs a;
  a.u_in = s->ua;
  a.psi0 = s->ua;
  a.u_out = s->ub;
  a.v_eff = s->o.prec == EMD_FP64 ? (const void *)s->veff1 : (const void *)s->veff1f;
  a.tab = &s->ts[s->cur];
  a.hc = s->hc;
  a.a = 0.0;
  a.apply_only = 1;
  emd_launch_stage(o, a, s->st);
  r = launch_check("emd_apply_hamiltonian");
  if (r) return r;
  r = download_orbitals(s, s->ub, n_vec, hpsi);
  if (r) return r;
  return read_err_flag(s);
}

int emd_kernel_stats(emd_system *s, int kernel, double *ms_total,
                     long long *launches) {
  g_err.clear();
  if (!s || !ms_total || !launches) return fail(EMD_EINVAL, "NULL argument");
  if (kernel == EMD_KERNEL_ALL) {
    CK(cudaStreamSynchronize(s->st));
    *ms_total = 0.0;
    *launches = g_launches.exchange(0);
    return EMD_OK;
  }
  if (kernel != EMD_KERNEL_HORNER) return fail(EMD_EINVAL, "unknown kernel %d", kernel);
  CK(cudaStreamSynchronize(s->st));
  for (auto &ev : s->prof_pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev.first, ev.second));
    s->prof_ms += ms;
    s->prof_launches += 1;
    s->prof_free.push_back(ev);
  }
  s->prof_pending.clear();
  *ms_total = s->prof_ms;
  *launches = s->prof_launches;
  s->prof_ms = 0.0;
  s->prof_launches = 0;
  return EMD_OK;
}

void emd_destroy(emd_system *s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  for (void *p : s->allocs) cudaFree(p);
  for (auto &ev : s->prof_pending) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  for (auto &ev : s->prof_free) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  delete s;
}

}  // extern "C"
