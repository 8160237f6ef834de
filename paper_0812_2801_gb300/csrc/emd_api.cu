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
//
// Also here: host I/O of orbitals (complex128 and complex64, pipelined),
// the deferred restart after the setters, energies and forces, batches of
// systems replayed as CUDA graphs (also used by emd_propagate for long
// runs), the adjoint propagation (driver; kernels in adjoint.cu), the dipole
// read-out and the ground-state solver (driver; element-wise kernels in
// groundstate.cu).
#include <algorithm>
#include <complex>
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
#include "gs_host.h"

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

// central second-derivative weights (Fornberg), k = 0..order/2, as integer
// numerators over the common denominator fd_den(order): c_k = fd_num / fd_den.
// The numerators are exact in float and sum to zero (num_0 + 2 sum num_k = 0).
double fd_num(int order, int k) {
  static const double n2[] = {-2.0, 1.0};
  static const double n4[] = {-30.0, 16.0, -1.0};
  static const double n6[] = {-490.0, 270.0, -27.0, 2.0};
  static const double n8[] = {-14350.0, 8064.0, -1008.0, 128.0, -9.0};
  switch (order) {
    case 2: return n2[k];
    case 4: return n4[k];
    case 6: return n6[k];
    default: return n8[k];
  }
}
double fd_den(int order) {
  switch (order) {
    case 2: return 1.0;
    case 4: return 12.0;
    case 6: return 180.0;
    default: return 5040.0;
  }
}
double fd_weight(int order, int k) { return fd_num(order, k) / fd_den(order); }

}  // namespace

void emd_note_launches(int k) { g_launches += k; }

// Device workspace of the adjoint propagation, sized on first use.
struct Adjoint {
  int n_ck = 0, K = 0;
  std::vector<double2 *> ck_psi, seg_psi, st_u;      // orbital sets
  std::vector<double *> ck_hist, seg_hist;          // 3 grids each
  std::vector<int> ck_len, seg_len;
  double2 *lam = nullptr, *mu = nullptr, *acc = nullptr, *zero = nullptr;
  double *gv1 = nullptr, *gv2 = nullptr, *gvloc = nullptr, *L0 = nullptr,
         *L1 = nullptr, *L2 = nullptr, *tmp = nullptr, *tmp2 = nullptr,
         *saw = nullptr, *zgrid = nullptr, *gR = nullptr, *dfield = nullptr,
         *scal = nullptr;
  double2 *cm = nullptr, *dcm = nullptr, *cu = nullptr, *dcu = nullptr,
          *hcu = nullptr;
  // moving ions: (R, V, F) per checkpoint and per segment step, the force
  // adjoint lam_F, its products and the extra grids
  double *ck_ion = nullptr, *seg_ion = nullptr, *lamF = nullptr, *fl = nullptr,
         *fr = nullptr, *fs = nullptr, *gR1 = nullptr, *fconv = nullptr,
         *vh = nullptr, *w = nullptr, *tmp3 = nullptr;
  double2 *m2 = nullptr;
  int n_field = 0;
  std::vector<void *> mem;
};

int emd_set_error(int code, const char *msg) {
  g_err = msg;
  return code;
}

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
  // complex64 host I/O: copies on their own stream (created on first use),
  // alternating between the two halves of stage_buf; events: start, half
  // k filled (1 + k), half k free again (3 + k)
  cudaStream_t cst = nullptr;
  cudaEvent_t cev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // an MD step builds the next position set's tables, v_loc and v_eff on
  // their own stream (created on first use) while exponential 1 runs on st
  // with the current set: fork (0) and join (1) events
  cudaStream_t tst = nullptr;
  cudaEvent_t tev[2] = {nullptr, nullptr};
  double *veff1 = nullptr, *veff2 = nullptr;
  float *veff1f = nullptr, *veff2f = nullptr;
  float4 *veff1d = nullptr, *veff2d = nullptr;   // complex64: (w_0 + v_eff) x4
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
         *F_sr = nullptr, *e_sr = nullptr, *nl_part = nullptr, *lf_part = nullptr,
         *sr_part = nullptr;
  double *partials = nullptr;
  int n_partials = 0;
  double *scal = nullptr;
  int *err = nullptr;
  int ions_set = 0, orbs_set = 0;
  // occupations f_A (host).  The device holds the orbitals as
  // u_A = sqrt(f_A / occ) phi_A, so that occ sum_A |u_A|^2 = sum_A f_A
  // |phi_A|^2 and every energy and force term, quadratic in each orbital,
  // carries the weight f_A; the propagation is linear in each orbital and
  // keeps its weight.  occ_w holds those weights, occ_winv their inverses;
  // f_uniform: every f_A = occ (weights 1, nothing scaled).
  std::vector<double> f;
  int f_uniform = 1;
  double *occ_w = nullptr, *occ_winv = nullptr;
  // set by emd_set_ions / emd_set_orbitals*: rho, v_Hxc (history restarted),
  // projections and F(0) are recomputed by the next call that reads them
  int needs_restart = 0;
  int frozen_ions = 0, profile = 0, check_stable = 1, proj_atom_major = 1;
  double2 *proj_part = nullptr;   // point-major projection partials
  void *hc_zero = nullptr;          // complex64: zero projector coefficients
  double v_max = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending, prof_free;
  double prof_ms = 0.0;
  long long prof_launches = 0;
  std::vector<void *> allocs;
  struct Adjoint *adj = nullptr;
  struct GroundStateWork *gsw = nullptr;
  // a batch of this system alone: emd_propagate replays its captured
  // graph of 6 MD steps for long field-free runs
  emd_batch *self_batch = nullptr;
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

// Occupations f (n_orb values in (0, occ]) into the system: values below
// 1e-30 occ are raised to it, so that every weight sqrt(f / occ) is a
// normal FP32 number; the orbitals on the device are not touched.
int set_occupation_state(emd_system *s, const double *f) {
  const double occ = s->cfg.occ;
  const int n = s->o.n_orb;
  std::vector<double> w(n), wi(n);
  bool uniform = true;
  for (int i = 0; i < n; ++i) {
    const double fi = std::max(f[i], 1e-30 * occ);
    s->f[i] = fi;
    uniform = uniform && fi == occ;
    w[i] = std::sqrt(fi / occ);
    wi[i] = 1.0 / w[i];
  }
  s->f_uniform = uniform;
  CK(cudaMemcpyAsync(s->occ_w, w.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->occ_winv, wi.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}

double occupation_sum(const emd_system *s) {
  double t = 0.0;
  for (double fi : s->f) t += fi;
  return t;
}

int read_err_flag(emd_system *s) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (h & EMD_ERRBIT_WAIT) {
    CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->st));
    return fail(EMD_ETIMEOUT, "a bounded wait in a stage kernel gave up (tensor copies "
                              "not completed within ~1 s); results of that call are invalid");
  }
  if (h)
    return fail(EMD_ETABLE,
                "atom list overflow (bits %d: 1 point list > %d projectors, 2 tile "
                "candidates > %d, 4 atom table)",
                h, s->ts[0].kmax, EMD_TILE_CAND_MAX);
  return EMD_OK;
}

// Build every table of set k from ts[k].R, on stream st (uses the FFT
// scratch fft_a / fft_b).
int build_set(emd_system *s, int k, cudaStream_t st) {
  TableSet &t = s->ts[k];
  emd_launch_wrap(t.R, t.Rw, s->n_atoms, s->g.L, st);
  emd_launch_tables(s->g, s->sp, s->n_atoms, t, s->err, st);
  emd_launch_tile_atoms(s->g, s->n_atoms, t, s->err, st);
  // v_loc = Poisson(-g): solve for g, negate in the final pass
  emd_launch_poisson(s->g, t.g_ion, t.v_loc, s->fft_a, s->fft_b, st);
  return launch_check("build_set");
}
int build_set(emd_system *s, int k) { return build_set(s, k, s->st); }

int table_pipe(emd_system *s) {
  if (s->tst) return EMD_OK;
  if (cudaStreamCreateWithFlags(&s->tst, cudaStreamNonBlocking) != cudaSuccess)
    return fail(EMD_ECUDA, "table stream creation failed");
  for (cudaEvent_t &e : s->tev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(EMD_ECUDA, "event creation failed");
  return EMD_OK;
}

void negate_grid(double *v, int n3, cudaStream_t st);

void project(emd_system *s, const void *u, int set, cudaStream_t st) {
  if (s->o.prec == EMD_FP32_ORBITALS)
    emd_launch_project_tile(s->o, s->ts[set], s->n_atoms, u,
                            s->g.h * s->g.h * s->g.h, s->sp.h_kb, s->c, s->hc,
                            s->proj_part, st);
  else if (s->proj_atom_major || s->sp.nch > 1)
    emd_launch_project(s->o, s->ts[set], s->n_atoms, u, s->g.h * s->g.h * s->g.h,
                       s->sp.h_kb, s->c, s->hc, st);
  else
    emd_launch_project_pm(s->o, s->ts[set], s->n_atoms, u,
                          s->g.h * s->g.h * s->g.h, s->sp.h_kb, s->c, s->hc,
                          s->proj_part, st);
}
void project(emd_system *s, const void *u, int set) { project(s, u, set, s->st); }

void stage(emd_system *s, const void *u_in, const void *psi0, void *u_out,
           int set, int which_veff, double a) {
  StageArgs a_;
  a_.u_in = u_in;
  a_.psi0 = psi0;
  a_.u_out = u_out;
  if (s->o.prec == EMD_FP64) {
    a_.v_eff = which_veff == 1 ? (const void *)s->veff1 : (const void *)s->veff2;
  } else {
    a_.v_eff = which_veff == 1 ? (const void *)s->veff1f : (const void *)s->veff2f;
    a_.v_diag = which_veff == 1 ? (const void *)s->veff1d : (const void *)s->veff2d;
  }
  a_.tab = &s->ts[set];
  a_.err = s->err;
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

// The force terms that read neither rho nor the potentials: nonlocal (from
// psi and its projections c at set k) and ion short range.
void forces_nl_sr(emd_system *s, int k, cudaStream_t st) {
  if (s->o.prec == EMD_FP32_ORBITALS)
    emd_launch_nl_force_tile(s->o, s->ts[k], s->n_atoms, s->psi, s->c,
                             s->g.h * s->g.h * s->g.h,
                             -2.0 * s->sp.h_kb * s->cfg.occ, s->proj_part, s->F_nl, st);
  else
    emd_launch_nl_force(s->o, s->ts[k], s->n_atoms, s->psi, s->c,
                        s->g.h * s->g.h * s->g.h,
                        -2.0 * s->sp.h_kb * s->cfg.occ, -2.0 * s->cfg.occ, s->sp.inv_rc2,
                        s->nl_part, s->F_nl, st);
  emd_launch_short_range(s->sp, s->n_atoms, s->ts[k].Rw, s->g.L, s->F_sr,
                         s->e_sr, s->sr_part, st);
}

void local_force(emd_system *s, int k) {
  emd_launch_local_force(s->g, s->sp, s->n_atoms, s->ts[k], s->v_h,
                         s->ts[k].v_loc, s->lf_part, s->F_loc, s->st);
}

// F = the three terms (+ the field's force); V += F dt / (2 M) if update_v
void total_force(emd_system *s, double field, double dt, int update_v) {
  emd_launch_vv_velocities(s->n_atoms, s->F_loc, s->F_nl, s->F_sr, field,
                           s->sp.z, s->F, s->V, dt, s->sp.mass, update_v,
                           s->st);
}

// Forces at set k (projections of psi at k must be in c).
void forces(emd_system *s, int k, double field, double dt, int update_v) {
  local_force(s, k);
  forces_nl_sr(s, k, s->st);
  total_force(s, field, dt, update_v);
}

int reduce_max_veff(emd_system *s, double *out);
double kinetic_fp32(emd_system *s, int *np);

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

// The derived state of a set_ions / set_orbitals, computed once before the
// first call that reads it (two setters in a row pay for one restart).
int ensure_state(emd_system *s) {
  if (!s->needs_restart) return EMD_OK;
  s->needs_restart = 0;
  return restart_dynamics(s);
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
__global__ void k_fill4(float4 *v, int n, float d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = make_float4(d, d, d, d);
}
__global__ void k_max_sum(const double *a, const double *b, int n, double *out) {
  __shared__ double sm[256];
  double m = -1e300;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmax(m, a[i] + b[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}
void negate_grid(double *v, int n3, cudaStream_t st) {
  emd_note_launches(1);
  k_negate<<<(n3 + 255) / 256, 256, 0, st>>>(v, n3);
}
// complex64: partial sums of Re<psi|S psi>, S = sum over axes of the
// stencil with the integer weights fd_num (S psi by the stage kernel with
// diagonal 3 num_0, no potential and zero projector coefficients, into ua).
// T = -S / (2 fd_den h^2); the returned factor turns the sum into <psi|T psi>.
// Integer weights are exact in float, so S annihilates constants exactly;
// float-rounded w_k = -c_k / (2 h^2) would shift T by a constant of order
// 1e-6 Ha and bias the kinetic energy by that times the electron count.
double kinetic_fp32(emd_system *s, int *np) {
  const int order = 2 * s->o.half_order;
  emd_note_launches(1);
  k_fill4<<<(s->g.n3 + 255) / 256, 256, 0, s->st>>>(s->veff1d, s->g.n3,
                                                     (float)(3.0 * fd_num(order, 0)));
  OrbLayout o = s->o;
  o.stage_variant = 0;
  o.zchunk = 0;
  o.w[0] = 3.0 * fd_num(order, 0);
  for (int k = 1; k <= o.half_order; ++k) o.w[k] = fd_num(order, k);
  StageArgs a;
  a.u_in = s->psi;
  a.psi0 = s->psi;
  a.u_out = s->ua;
  a.v_eff = s->veff1f;
  a.v_diag = s->veff1d;
  a.tab = &s->ts[s->cur];
  a.err = s->err;
  a.hc = s->hc_zero;
  a.a = 0.0;
  a.apply_only = 1;
  emd_launch_stage(o, a, s->st);
  emd_launch_cdot_re_c64(s->o, s->psi, s->ua, s->partials, np, s->st);
  return -1.0 / (2.0 * fd_den(order) * s->g.h * s->g.h);
}
int reduce_max_veff(emd_system *s, double *out) {
  emd_note_launches(1);
  const int nb = std::min(s->n_partials, 512);
  k_max_sum<<<nb, 256, 0, s->st>>>(s->hist[0], s->ts[s->cur].v_loc, s->g.n3,
                                    s->partials);
  std::vector<double> hm(nb);
  CK(cudaMemcpyAsync(hm.data(), s->partials, nb * sizeof(double),
                     cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  *out = *std::max_element(hm.begin(), hm.end());
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
  if (c.n_atoms < 0 || c.n_atoms > 32767)
    return fail(EMD_EINVAL, "n_atoms must be in [0, 32767]");
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
  if (p.lmax < 0 || p.lmax > 2) return fail(EMD_EINVAL, "species lmax must be 0, 1 or 2");
  if (p.lmax > 0 && !(c.precision == EMD_FP64 && (c.block_orbitals == 0 || c.block_orbitals == 2)))
    return fail(EMD_EINVAL, "several projectors per atom (lmax > 0) need EMD_FP64 with block "
                            "width 2 (the double-float projection kernels)");
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
  s->sp.lmax = p.lmax;
  s->sp.nch = (p.lmax + 1) * (p.lmax + 1);
  s->sp.hl[0] = p.h_kb;
  s->sp.hl[1] = p.lmax >= 1 ? p.h_l[0] : 0.0;
  s->sp.hl[2] = p.lmax >= 2 ? p.h_l[1] : 0.0;
  // N_l^-2 = 2 pi Gamma(l + 3/2) r_c^(2l+3) / (2l + 1): unit norm in the continuum
  for (int l = 0; l < 3; ++l)
    s->sp.nl[l] = c.n_atoms ? 1.0 / std::sqrt(2.0 * M_PI * std::tgamma(l + 1.5) *
                                              std::pow(p.r_c, 2 * l + 3) / (2 * l + 1))
                            : 0.0;
  s->sp.nl[0] = s->sp.c_p;

  OrbLayout &o = s->o;
  o.n = c.n;
  o.n3 = s->g.n3;
  o.h = c.h;
  o.prec = c.precision;
  // default block width: measured fastest stage kernel on the 96^3 order-8
  // workload (complex64: 4 orbitals, column kernel; complex128: 2)
  o.bo = c.block_orbitals ? c.block_orbitals : (c.precision == EMD_FP64 ? 2 : 4);
  o.n_orb = c.n_orb;
  o.n_blk = (c.n_orb + o.bo - 1) / o.bo;
  o.n_orb_pad = o.n_blk * o.bo;
  o.half_order = c.fd_order / 2;
  o.n_atoms = c.n_atoms;
  o.stage_variant = 0;
  o.zchunk = 0;
  o.nch = s->sp.nch;
  o.n_proj = c.n_atoms * o.nch;
  for (int l = 0; l < 3; ++l) o.hl[l] = s->sp.hl[l];
  for (int k = 0; k <= EMD_MAX_HALF_ORDER; ++k) o.w[k] = o.num[k] = 0.0;
  o.w[0] = -1.5 * fd_weight(c.fd_order, 0) / (c.h * c.h);
  for (int k = 1; k <= o.half_order; ++k)
    o.w[k] = -0.5 * fd_weight(c.fd_order, k) / (c.h * c.h);
  for (int k = 0; k <= o.half_order; ++k) o.num[k] = fd_num(c.fd_order, k);
  o.den = fd_den(c.fd_order);

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
    TRY(A((void **)&s->veff1d, n3 * 16));
    TRY(A((void **)&s->veff2d, n3 * 16));
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
  // the complex64 path reads the per-tile entries instead of the atom table
  if (c.n_atoms == 0 || c.precision == EMD_FP32_ORBITALS) cap = 1;
  const int nproj = na * s->sp.nch;      // projector rows of c and hc
  for (int k = 0; k < 2; ++k) {
    TableSet &t = s->ts[k];
    t.cap = (int)cap;
    t.kmax = EMD_PT_KMAX * s->sp.nch;
    TRY(A((void **)&t.R, na * 3 * 8));
    TRY(A((void **)&t.Rw, na * 3 * 8));
    TRY(A((void **)&t.tile_cnt, ntiles * 4));
    TRY(A((void **)&t.tile_ent, (size_t)ntiles * EMD_TILE_CAND_MAX * 4));
    TRY(A((void **)&t.pt_cnt, n3 * 4));
    TRY(A((void **)&t.pt_J, n3 * t.kmax * 4));
    TRY(A((void **)&t.pt_p, n3 * t.kmax * 8));
    TRY(A((void **)&t.pt_pf, n3 * t.kmax * 4));
    TRY(A((void **)&t.pt4, n3 * 4 * sizeof(int2)));
    TRY(A((void **)&t.at_cnt, na * 4));
    TRY(A((void **)&t.split_cnt, na * EMD_SPLIT * 4));
    TRY(A((void **)&t.at_pt, (size_t)na * cap * 4));
    TRY(A((void **)&t.at_p, (size_t)na * cap * 8));
    TRY(A((void **)&t.at_d, (size_t)na * cap * 24));
    t.at_rec = nullptr;
    t.at_w = nullptr;
    if (c.precision == EMD_FP64 && o.bo == 2 && c.n_atoms > 0) {
      TRY(A((void **)&t.at_rec, (size_t)nproj * cap * sizeof(uint4)));
      TRY(A((void **)&t.at_w, (size_t)nproj * cap * 2 * sizeof(float4)));
    }
    t.te_off = nullptr;
    t.te_pp = nullptr;
    t.te_q = nullptr;
    t.pt4d = nullptr;
    t.pt_rec = nullptr;
    if (c.precision == EMD_FP64 && o.bo == 2 && s->sp.nch > 1)
      TRY(A((void **)&t.pt_rec, n3 * t.kmax * sizeof(int4)));
    if (c.precision == EMD_FP64 && o.bo == 2) TRY(A((void **)&t.pt4d, n3 * 3 * sizeof(int4)));
    if (c.precision == EMD_FP32_ORBITALS) {
      TRY(A((void **)&t.te_off, (size_t)ntiles * (EMD_TILE_ATOM_MAX + 1) * 4));
      TRY(A((void **)&t.te_pp, (size_t)ntiles * EMD_TE_CAP * sizeof(uint2)));
      TRY(A((void **)&t.te_q, (size_t)ntiles * EMD_TE_CAP * 16));
    }
    t.n_slots_cap = ntiles * EMD_TILE_ATOM_MAX;
    TRY(A((void **)&t.tile_nat, ntiles * 4));
    TRY(A((void **)&t.tile_atoms, (size_t)ntiles * EMD_TILE_ATOM_MAX * 4));
    TRY(A((void **)&t.tile_off, ntiles * 4));
    TRY(A((void **)&t.at_ntiles, na * 4));
    TRY(A((void **)&t.at_tiles, (size_t)na * ntiles * sizeof(int2)));
    TRY(A((void **)&t.g_ion, n3 * 8));
    t.gtab = nullptr;
    t.glo = nullptr;
    t.gtabd = nullptr;
    // an image box spans at most 2 r / h + 5 points per axis
    if (c.n_atoms > 0 && 2 * (int)std::ceil(p.r_loc / c.h) + 6 <= EMD_GT_EXT) {
      TRY(A((void **)&t.gtab, (size_t)na * 27 * 3 * EMD_GT_EXT * sizeof(double)));
      TRY(A((void **)&t.glo, (size_t)na * 27 * 3 * sizeof(int)));
      TRY(A((void **)&t.gtabd, (size_t)na * 27 * EMD_GT_EXT * sizeof(double)));
    }
    TRY(A((void **)&t.v_loc, n3 * 8));
  }
  TRY(A((void **)&s->proj_part, (size_t)o.n_blk * ntiles * EMD_TILE_ATOM_MAX *
                                     o.bo * (c.precision == EMD_FP32_ORBITALS ? 3 : 1) *
                                     sizeof(double2)));
  if (c.precision == EMD_FP32_ORBITALS) {
    TRY(A(&s->hc_zero, (size_t)na * o.n_orb_pad * sizeof(float2)));
    TRY(cudaMemset(s->hc_zero, 0, (size_t)na * o.n_orb_pad * sizeof(float2)) == cudaSuccess
            ? EMD_OK
            : fail(EMD_ECUDA, "cudaMemset failed"));
  }
  TRY(A((void **)&s->c, (size_t)nproj * o.n_orb_pad * sizeof(double2)));
  TRY(A(&s->hc, (size_t)nproj * o.n_orb_pad * esz));
  TRY(A((void **)&s->V, na * 3 * 8));
  TRY(A((void **)&s->F, na * 3 * 8));
  TRY(A((void **)&s->F_loc, na * 3 * 8));
  TRY(A((void **)&s->F_nl, na * 3 * 8));
  TRY(A((void **)&s->F_sr, na * 3 * 8));
  TRY(A((void **)&s->e_sr, na * 8));
  TRY(A((void **)&s->sr_part, (size_t)na * EMD_SR_SPLIT * 4 * 8));
  TRY(A((void **)&s->nl_part, (size_t)nproj * o.n_blk * 3 * 8));
  TRY(A((void **)&s->lf_part, (size_t)na * EMD_SPLIT * 3 * 8));
  s->n_partials = std::max(1024, (int)((n3 + 255) / 256));
  TRY(A((void **)&s->partials, (size_t)s->n_partials * 8));
  TRY(A((void **)&s->scal, 16 * 8));
  TRY(A((void **)&s->err, sizeof(int)));
  TRY(A((void **)&s->occ_w, (size_t)o.n_orb_pad * 8));
  TRY(A((void **)&s->occ_winv, (size_t)o.n_orb_pad * 8));
  s->f.assign(o.n_orb, c.occ);
#undef TRY
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->V, 0, na * 3 * 8, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->F, 0, na * 3 * 8, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->c, 0, (size_t)nproj * o.n_orb_pad * 16, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->hc, 0, (size_t)nproj * o.n_orb_pad * esz, s->st);
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
  if (s->orbs_set) {
    s->needs_restart = 1;
    s->c_valid = 0;
  }
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

// winv (device, one factor per orbital, or NULL): each orbital is scaled by
// it on the way out (the system's orbitals have their occupation weights
// removed this way)
static int download_orbitals(emd_system *s, const void *src, int n_vec,
                             double *psi, const double *winv = nullptr) {
  const size_t n3 = s->g.n3;
  for (int b = 0; b * s->o.bo < n_vec; ++b) {
    const int nv = std::min(s->o.bo, n_vec - b * s->o.bo);
    const char *d = (const char *)src + (size_t)b * n3 * s->o.bo *
                                            (s->o.prec == EMD_FP64 ? 16 : 8);
    emd_launch_unpack(s->o, d, s->stage_buf, nv, s->st);
    if (winv)
      emd_launch_scale_canon(false, s->stage_buf, n3, nv, winv + (size_t)b * s->o.bo, s->st);
    CK(cudaMemcpyAsync(psi + 2 * (size_t)b * s->o.bo * n3, s->stage_buf,
                       (size_t)nv * n3 * 16, cudaMemcpyDeviceToHost, s->st));
  }
  CK(cudaStreamSynchronize(s->st));
  return launch_check("download_orbitals");
}

static int copy_pipe(emd_system *s) {
  if (s->cst) return EMD_OK;
  if (cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking) != cudaSuccess)
    return fail(EMD_ECUDA, "copy stream creation failed");
  for (cudaEvent_t &e : s->cev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(EMD_ECUDA, "event creation failed");
  return EMD_OK;
}

// complex64 host arrays: one orbital block per half of stage_buf; the copy
// of block b + 1 (copy stream) overlaps the pack of block b (s->st)
static int upload_orbitals_c64(emd_system *s, const float *psi, void *dst) {
  int r = copy_pipe(s);
  if (r) return r;
  const size_t n3 = s->g.n3;
  const int n_vec = s->o.n_orb;
  float2 *half[2] = {(float2 *)s->stage_buf, (float2 *)s->stage_buf + (size_t)s->o.bo * n3};
  CK(cudaEventRecord(s->cev[0], s->st));
  CK(cudaStreamWaitEvent(s->cst, s->cev[0], 0));
  for (int b = 0; b * s->o.bo < n_vec; ++b) {
    const int k = b & 1;
    const int nv = std::min(s->o.bo, n_vec - b * s->o.bo);
    if (b >= 2) CK(cudaStreamWaitEvent(s->cst, s->cev[3 + k], 0));
    CK(cudaMemcpyAsync(half[k], psi + 2 * (size_t)b * s->o.bo * n3,
                       (size_t)nv * n3 * 8, cudaMemcpyHostToDevice, s->cst));
    CK(cudaEventRecord(s->cev[1 + k], s->cst));
    CK(cudaStreamWaitEvent(s->st, s->cev[1 + k], 0));
    char *d = (char *)dst + (size_t)b * n3 * s->o.bo *
                                (s->o.prec == EMD_FP64 ? 16 : 8);
    emd_launch_pack_c64(s->o, half[k], d, nv, s->st);
    CK(cudaEventRecord(s->cev[3 + k], s->st));
  }
  return launch_check("upload_orbitals_c64");
}

int emd_set_orbitals_c64(emd_system *s, const float *psi) {
  g_err.clear();
  if (!s || !psi) return fail(EMD_EINVAL, "NULL argument");
  CK(cudaMemsetAsync(s->psi, 0, s->orb_bytes, s->st));
  int r = upload_orbitals_c64(s, psi, s->psi);
  if (r) return r;
  if (!s->f_uniform) emd_launch_scale_orbitals(s->o, s->psi, s->o.n_orb, s->occ_w, s->st);
  s->orbs_set = 1;
  s->c_valid = 0;
  if (s->ions_set) s->needs_restart = 1;
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}

int emd_get_orbitals_c64(emd_system *s, float *psi) {
  g_err.clear();
  if (!s || !psi) return fail(EMD_EINVAL, "NULL argument");
  int r = read_err_flag(s);
  if (r) return r;
  r = copy_pipe(s);
  if (r) return r;
  const size_t n3 = s->g.n3;
  float2 *half[2] = {(float2 *)s->stage_buf, (float2 *)s->stage_buf + (size_t)s->o.bo * n3};
  // the unpack of block b + 1 (s->st) overlaps the copy of block b
  for (int b = 0; b * s->o.bo < s->o.n_orb; ++b) {
    const int k = b & 1;
    const int nv = std::min(s->o.bo, s->o.n_orb - b * s->o.bo);
    if (b >= 2) CK(cudaStreamWaitEvent(s->st, s->cev[3 + k], 0));
    const char *d = (const char *)s->psi + (size_t)b * n3 * s->o.bo *
                                               (s->o.prec == EMD_FP64 ? 16 : 8);
    emd_launch_unpack_c64(s->o, d, half[k], nv, s->st);
    if (!s->f_uniform)
      emd_launch_scale_canon(true, half[k], n3, nv, s->occ_winv + (size_t)b * s->o.bo, s->st);
    CK(cudaEventRecord(s->cev[1 + k], s->st));
    CK(cudaStreamWaitEvent(s->cst, s->cev[1 + k], 0));
    CK(cudaMemcpyAsync(psi + 2 * (size_t)b * s->o.bo * n3, half[k],
                       (size_t)nv * n3 * 8, cudaMemcpyDeviceToHost, s->cst));
    CK(cudaEventRecord(s->cev[3 + k], s->cst));
  }
  CK(cudaStreamSynchronize(s->cst));
  CK(cudaStreamSynchronize(s->st));
  return launch_check("emd_get_orbitals_c64");
}

int emd_set_orbitals(emd_system *s, const double *psi) {
  g_err.clear();
  if (!s || !psi) return fail(EMD_EINVAL, "NULL argument");
  CK(cudaMemsetAsync(s->psi, 0, s->orb_bytes, s->st));
  int r = upload_orbitals(s, psi, s->o.n_orb, s->psi);
  if (r) return r;
  if (!s->f_uniform) emd_launch_scale_orbitals(s->o, s->psi, s->o.n_orb, s->occ_w, s->st);
  s->orbs_set = 1;
  s->c_valid = 0;
  if (s->ions_set) s->needs_restart = 1;
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}

int emd_set_occupations(emd_system *s, const double *f) {
  g_err.clear();
  if (!s || !f) return fail(EMD_EINVAL, "NULL argument");
  for (int i = 0; i < s->o.n_orb; ++i)
    if (!(f[i] > 0.0 && f[i] <= s->cfg.occ))
      return fail(EMD_EINVAL, "occupation %d = %g outside (0, occ = %g]", i, f[i], s->cfg.occ);
  // orbitals already on the device: u_A <- sqrt(f_new / f_old) u_A in two
  // scalings (remove the old weight, apply the new one)
  const int had = s->orbs_set && !s->f_uniform;
  if (had) emd_launch_scale_orbitals(s->o, s->psi, s->o.n_orb, s->occ_winv, s->st);
  int r = set_occupation_state(s, f);
  if (r) return r;
  if (s->orbs_set && !s->f_uniform)
    emd_launch_scale_orbitals(s->o, s->psi, s->o.n_orb, s->occ_w, s->st);
  if (s->orbs_set) {
    s->c_valid = 0;
    if (s->ions_set) s->needs_restart = 1;
  }
  CK(cudaStreamSynchronize(s->st));
  return launch_check("emd_set_occupations");
}

int emd_get_occupations(emd_system *s, double *f) {
  g_err.clear();
  if (!s || !f) return fail(EMD_EINVAL, "NULL argument");
  std::copy(s->f.begin(), s->f.end(), f);
  return EMD_OK;
}

int emd_set_option(emd_system *s, int option, double value) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  switch (option) {
    case EMD_OPT_FROZEN_IONS: s->frozen_ions = value != 0.0; return EMD_OK;
    case EMD_OPT_PROFILE: s->profile = value != 0.0; return EMD_OK;
    case EMD_OPT_CHECK_STABLE: s->check_stable = value != 0.0; return EMD_OK;
    case EMD_OPT_PROJECTION:
      if (value != 0.0 && value != 1.0) return fail(EMD_EINVAL, "projection form must be 0 or 1");
      s->proj_atom_major = (int)value;
      return EMD_OK;
    case EMD_OPT_STAGE_VARIANT:
      if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0)
        return fail(EMD_EINVAL, "stage variant must be 0, 1, 2 or 3");
      s->o.stage_variant = (int)value;
      return EMD_OK;
    case EMD_OPT_ZCHUNK:
      if (!(value >= 0.0 && value <= 1024.0) || value != (double)(int)value)
        return fail(EMD_EINVAL, "z-chunk must be an integer in 0 .. 1024");
      s->o.zchunk = (int)value;
      return EMD_OK;
  }
  return fail(EMD_EINVAL, "unknown option %d", option);
}

}  // extern "C"

namespace {

// Argument validation and the Taylor-4 stability refusal shared by the
// single-system and batched propagation.
int check_propagate(emd_system *s, double dt, double mu) {
  if (!s) return fail(EMD_EINVAL, "NULL system");
  if (!s->ions_set || !s->orbs_set)
    return fail(EMD_ESTATE, "set ions and orbitals before propagating");
  if (!(dt > 0.0) || !(mu > 0.0) || !std::isfinite(dt) || !std::isfinite(mu))
    return fail(EMD_EINVAL, "dt and mu must be finite and > 0");
  int r = ensure_state(s);   // v_max for the bound below
  if (r) return r;
  const double tau = 0.5 * (dt / mu);
  if (s->check_stable) {
    const double lam = 1.5 * kinetic_lambda_max(s->cfg.fd_order) / (s->g.h * s->g.h) +
                       std::max(0.0, s->v_max) +
                       std::max({0.0, s->sp.hl[0], s->sp.hl[1], s->sp.hl[2]});
    const double x = tau * lam;
    if (x > 2.0 * std::sqrt(2.0))
      return fail(EMD_EUNSTABLE,
                  "tau*lambda_max = %.3f exceeds the Taylor-4 stability bound "
                  "2*sqrt(2) (tau = dt/(2 mu) = %g, lambda_max ~ %.2f)",
                  x, tau, lam);
  }
  return EMD_OK;
}

// One MD step on s->st (enqueue only; no host synchronisation, so it can be
// captured into a CUDA graph).
int step_once(emd_system *s, double dt, double mu, double e) {
  const double tau = 0.5 * (dt / mu);
  const int cur = s->cur;
  const int nw = s->frozen_ions ? cur : 1 - cur;
  if (!s->frozen_ions) {
    emd_launch_vv_positions(s->n_atoms, s->ts[cur].R, s->V, s->F, dt,
                            s->sp.mass, s->ts[nw].R, s->st);
    // set nw and veff2 on the table stream; exponential 1 reads neither, and
    // the FFT scratch they use is free until electrons() after the join
    int r = table_pipe(s);
    if (r) return r;
    CK(cudaEventRecord(s->tev[0], s->st));
    CK(cudaStreamWaitEvent(s->tst, s->tev[0], 0));
    r = build_set(s, nw, s->tst);
    if (r) return r;
    negate_grid(s->ts[nw].v_loc, s->g.n3, s->tst);
    emd_launch_veff(s->g, s->ts[nw].v_loc, s->hist, s->hist_len, e, s->veff2,
                    s->veff2f, s->tst, s->veff2d, s->o.w[0]);
    CK(cudaEventRecord(s->tev[1], s->tst));
  } else {
    emd_launch_veff(s->g, s->ts[nw].v_loc, s->hist, s->hist_len, e, s->veff2,
                    s->veff2f, s->st, s->veff2d, s->o.w[0]);
  }
  emd_launch_veff(s->g, s->ts[cur].v_loc, s->hist, 1, e, s->veff1, s->veff1f,
                  s->st, s->veff1d, s->o.w[0]);
  if (!s->c_valid) project(s, s->psi, cur);
  // exponential 1: psi -> ub with H(t)
  exponential(s, s->psi, s->ua, s->ub, cur, 1, tau);
  if (!s->frozen_ions) CK(cudaStreamWaitEvent(s->st, s->tev[1], 0));
  project(s, s->ub, nw);
  // exponential 2: ub -> psi with H(t+dt)
  exponential(s, s->ub, s->ua, s->psi, nw, 2, tau);
  if (!s->frozen_ions) {
    // psi's projections at set nw and the nonlocal and short-range forces
    // on the table stream, beside the density and potentials (which they
    // neither read nor write)
    CK(cudaEventRecord(s->tev[0], s->st));
    CK(cudaStreamWaitEvent(s->tst, s->tev[0], 0));
    project(s, s->psi, nw, s->tst);
    forces_nl_sr(s, nw, s->tst);
    CK(cudaEventRecord(s->tev[1], s->tst));
  }
  // new density and potentials; history slot of the oldest entry
  double *oldest = s->hist[2];
  s->hist[2] = s->hist[1];
  s->hist[1] = s->hist[0];
  s->hist[0] = oldest;
  electrons(s, 0);
  s->hist_len = std::min(3, s->hist_len + 1);
  if (!s->frozen_ions) {
    local_force(s, nw);
    CK(cudaStreamWaitEvent(s->st, s->tev[1], 0));
    total_force(s, e, dt, 1);
    s->cur = nw;
    s->c_valid = 1;
  } else {
    s->c_valid = 0;
  }
  return launch_check("emd_propagate");
}

}  // namespace

// ---------------------------------------------------------------------------
// Batched replicas: independent systems advanced together.  After a short
// eager warm-up (until every v_Hxc history is full), chunks of 6 MD steps of
// all systems are captured once into a CUDA graph -- one parallel branch per
// system, so ragged replicas share the GPU -- and replayed.  6 steps is the
// period of the host-side state (position sets alternate with period 2, the
// three v_Hxc history slots rotate with period 3), so a replay leaves it
// unchanged.
// ---------------------------------------------------------------------------
struct emd_batch {
  std::vector<emd_system *> sys;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  double key_dt = 0.0, key_mu = 0.0;
  // host-side state baked into the captured graph: the position-set parity,
  // the v_Hxc history slots (rotated by pointer, period 3) and the options
  // that select kernels
  std::vector<int> key_cur, key_variant, key_proj, key_zchunk;
  std::vector<const double *> key_hist;
  long long graph_launches = 0;
};

namespace {
constexpr int kGraphSteps = 6;

int batch_capture(emd_batch *b, double dt, double mu) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  std::vector<int> prof(b->sys.size());
  for (size_t i = 0; i < b->sys.size(); ++i) {
    prof[i] = b->sys[i]->profile;
    b->sys[i]->profile = 0;
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  int rc = EMD_OK;
  if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) rc = EMD_ECUDA;
  for (size_t i = 0; i < b->sys.size() && rc == EMD_OK; ++i) {
    if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) {
      rc = EMD_ECUDA;
      break;
    }
    for (int k = 0; k < kGraphSteps && rc == EMD_OK; ++k)
      rc = step_once(b->sys[i], dt, mu, 0.0);
    if (rc == EMD_OK && (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess ||
                         cudaStreamWaitEvent(b->origin, b->done[i], 0) != cudaSuccess))
      rc = EMD_ECUDA;
  }
  cudaError_t e = cudaStreamEndCapture(b->origin, &graph);
  for (size_t i = 0; i < b->sys.size(); ++i) b->sys[i]->profile = prof[i];
  if (rc != EMD_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != EMD_OK ? rc : fail(EMD_ECUDA, "graph capture failed: %s",
                                     cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return fail(EMD_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  b->key_dt = dt;
  b->key_mu = mu;
  const size_t m = b->sys.size();
  b->key_cur.resize(m);
  b->key_variant.resize(m);
  b->key_zchunk.resize(m);
  b->key_proj.resize(m);
  b->key_hist.resize(m);
  for (size_t i = 0; i < m; ++i) {
    b->key_cur[i] = b->sys[i]->cur;
    b->key_variant[i] = b->sys[i]->o.stage_variant;
    b->key_zchunk[i] = b->sys[i]->o.zchunk;
    b->key_proj[i] = b->sys[i]->proj_atom_major;
    b->key_hist[i] = b->sys[i]->hist[0];
  }
  return EMD_OK;
}

bool batch_graph_valid(const emd_batch *b, double dt, double mu) {
  if (!b->exec || b->key_dt != dt || b->key_mu != mu) return false;
  for (size_t i = 0; i < b->sys.size(); ++i)
    if (b->key_cur[i] != b->sys[i]->cur || b->key_hist[i] != b->sys[i]->hist[0] ||
        b->key_variant[i] != b->sys[i]->o.stage_variant ||
        b->key_zchunk[i] != b->sys[i]->o.zchunk ||
        b->key_proj[i] != b->sys[i]->proj_atom_major)
      return false;
  return true;
}
}  // namespace

extern "C" {

int emd_propagate(emd_system *s, int n_steps, double dt, double mu,
                  const double *field) {
  g_err.clear();
  int r = check_propagate(s, dt, mu);
  if (r) return r;
  if (n_steps < 0) return fail(EMD_EINVAL, "n_steps must be >= 0");
  if (field)
    for (int i = 0; i < n_steps; ++i)
      if (!std::isfinite(field[i])) return fail(EMD_EINVAL, "non-finite field");
  // long field-free runs replay a captured graph (launch overhead dominates
  // small grids); profiling needs one event pair per launch, so it stays eager
  if (!field && !s->frozen_ions && !s->profile && n_steps >= kGraphSteps) {
    if (!s->self_batch) {
      emd_system *one[1] = {s};
      r = emd_batch_create(1, one, &s->self_batch);
      if (r) return r;
    }
    return emd_batch_propagate(s->self_batch, n_steps, dt, mu);
  }
  for (int step = 0; step < n_steps; ++step) {
    r = step_once(s, dt, mu, field ? field[step] : 0.0);
    if (r) return r;
  }
  return EMD_OK;
}

int emd_batch_create(int n, emd_system *const *systems, emd_batch **out) {
  g_err.clear();
  if (!out || !systems || n < 1) return fail(EMD_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!systems[i]) return fail(EMD_EINVAL, "NULL system %d", i);
    for (int k = 0; k < i; ++k)
      if (systems[k] == systems[i]) return fail(EMD_EINVAL, "system %d repeated", i);
  }
  emd_batch *b = new emd_batch();
  b->sys.assign(systems, systems + n);
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->streams.push_back(st);
    ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->done.push_back(ev);
  }
  if (!ok) {
    emd_batch_destroy(b);
    return fail(EMD_ECUDA, "stream/event creation failed");
  }
  *out = b;
  return EMD_OK;
}

int emd_batch_propagate(emd_batch *b, int n_steps, double dt, double mu) {
  g_err.clear();
  if (!b) return fail(EMD_EINVAL, "NULL batch");
  if (n_steps < 0) return fail(EMD_EINVAL, "n_steps must be >= 0");
  const size_t m = b->sys.size();
  for (size_t i = 0; i < m; ++i) {
    int r = check_propagate(b->sys[i], dt, mu);
    if (r) return r;
  }
  // internal streams follow each system's own stream, and back at the end
  std::vector<cudaStream_t> user(m);
  for (size_t i = 0; i < m; ++i) {
    user[i] = b->sys[i]->st;
    CK(cudaEventRecord(b->done[i], user[i]));
    CK(cudaStreamWaitEvent(b->streams[i], b->done[i], 0));
    b->sys[i]->st = b->streams[i];
  }
  int rc = EMD_OK;
  int done_steps = 0;
  auto eager = [&](int k) {
    for (int s = 0; s < k && rc == EMD_OK; ++s)
      for (size_t i = 0; i < m && rc == EMD_OK; ++i)
        rc = step_once(b->sys[i], dt, mu, 0.0);
  };
  // a captured chunk assumes the full v_Hxc history and valid projections
  // of psi (its first step skips re-projecting): step eagerly until both hold
  auto full_history = [&]() {
    for (size_t i = 0; i < m; ++i)
      if (b->sys[i]->hist_len < 3 || b->sys[i]->frozen_ions || !b->sys[i]->c_valid)
        return false;
    return true;
  };
  while (rc == EMD_OK && done_steps < n_steps &&
         !(full_history() && n_steps - done_steps >= kGraphSteps)) {
    eager(1);
    ++done_steps;
  }
  while (rc == EMD_OK && n_steps - done_steps >= kGraphSteps) {
    if (!batch_graph_valid(b, dt, mu)) rc = batch_capture(b, dt, mu);
    if (rc != EMD_OK) break;
    for (size_t i = 0; i < m && rc == EMD_OK; ++i)
      if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess ||
          cudaStreamWaitEvent(b->origin, b->done[i], 0) != cudaSuccess)
        rc = fail(EMD_ECUDA, "batch ordering failed");
    if (rc != EMD_OK) break;
    cudaError_t e = cudaGraphLaunch(b->exec, b->origin);
    if (e != cudaSuccess) {
      rc = fail(EMD_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
      break;
    }
    ++b->graph_launches;
    emd_note_launches(0);
    CK(cudaEventRecord(b->fork, b->origin));
    for (size_t i = 0; i < m; ++i) CK(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
    done_steps += kGraphSteps;
  }
  if (rc == EMD_OK) eager(n_steps - done_steps);
  for (size_t i = 0; i < m; ++i) {
    b->sys[i]->st = user[i];
    if (cudaEventRecord(b->done[i], b->streams[i]) == cudaSuccess)
      cudaStreamWaitEvent(user[i], b->done[i], 0);
  }
  return rc;
}

void emd_batch_destroy(emd_batch *b) {
  if (!b) return;
  for (cudaStream_t st : b->streams) cudaStreamSynchronize(st);
  if (b->origin) cudaStreamSynchronize(b->origin);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->done) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

}  // extern "C"

namespace {

int adj_alloc(emd_system *s, int n_ck, int K, int n_steps) {
  Adjoint *&A = s->adj;
  if (A && A->n_ck >= n_ck && A->K >= K && A->n_field >= n_steps &&
      (s->frozen_ions || A->ck_ion))
    return EMD_OK;
  if (A) {
    for (void *p : A->mem) cudaFree(p);
    delete A;
    A = nullptr;
  }
  A = new Adjoint();
  const size_t n3 = s->g.n3;
  const size_t ob = s->orb_bytes, gb = n3 * sizeof(double);
  const size_t cb = (size_t)std::max(1, s->n_atoms) * s->o.n_orb_pad * sizeof(double2);
  auto get = [&](void **p, size_t b) -> int {
    if (cudaMalloc(p, b) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail(EMD_ENOMEM, "adjoint workspace: cudaMalloc(%zu) failed", b);
    }
    A->mem.push_back(*p);
    return EMD_OK;
  };
#define AG(ptr, b) do { int r_ = get((void **)&(ptr), (b)); if (r_) return r_; } while (0)
  A->n_ck = n_ck;
  A->K = K;
  A->n_field = n_steps;
  A->ck_psi.resize(n_ck + 1);   // last: the final state, restored at the end
  A->ck_hist.resize(n_ck + 1);
  A->ck_len.resize(n_ck + 1);
  for (int i = 0; i <= n_ck; ++i) {
    AG(A->ck_psi[i], ob);
    AG(A->ck_hist[i], 3 * gb);
  }
  A->seg_psi.resize(K);
  A->seg_hist.resize(K);
  A->seg_len.resize(K);
  for (int i = 0; i < K; ++i) {
    AG(A->seg_psi[i], ob);
    AG(A->seg_hist[i], 3 * gb);
  }
  A->st_u.resize(7);
  for (int i = 0; i < 7; ++i) AG(A->st_u[i], ob);
  AG(A->lam, ob);
  AG(A->mu, 2 * ob);
  AG(A->acc, ob);
  AG(A->zero, ob);
  double **grids[] = {&A->gv1, &A->gv2, &A->gvloc, &A->L0, &A->L1, &A->L2,
                      &A->tmp, &A->tmp2, &A->saw, &A->zgrid};
  for (double **gp : grids) AG(*gp, gb);
  AG(A->gR, 3 * std::max(1, s->n_atoms) * sizeof(double));
  AG(A->dfield, std::max(1, n_steps) * sizeof(double));
  AG(A->scal, 8 * sizeof(double));
  AG(A->cm, cb);
  AG(A->cu, cb);
  AG(A->hcu, cb);
  AG(A->dcm, 3 * cb);
  AG(A->dcu, 3 * cb);
  if (!s->frozen_ions) {
    const size_t ib = 9 * (size_t)std::max(1, s->n_atoms) * sizeof(double);
    const size_t ab = 3 * (size_t)std::max(1, s->n_atoms) * sizeof(double);
    AG(A->ck_ion, (n_ck + 1) * ib);
    AG(A->seg_ion, K * ib);
    AG(A->lamF, ab);
    AG(A->fl, ab);
    AG(A->fr, ab);
    AG(A->fs, ab);
    AG(A->gR1, ab);
    AG(A->fconv, ab);
    AG(A->vh, gb);
    AG(A->w, gb);
    AG(A->tmp3, gb);
    AG(A->m2, 3 * cb);
  }
#undef AG
  CK(cudaMemsetAsync(A->zero, 0, ob, s->st));
  CK(cudaMemsetAsync(A->zgrid, 0, gb, s->st));
  // s(z) = z h - L/2 on the grid (length-gauge field coordinate)
  std::vector<double> saw(n3);
  for (size_t p = 0; p < n3; ++p)
    saw[p] = (double)(p / ((size_t)s->g.n * s->g.n)) * s->g.h - 0.5 * s->g.L;
  CK(cudaMemcpy(A->saw, saw.data(), gb, cudaMemcpyHostToDevice));
  return EMD_OK;
}

void copy_hist_out(emd_system *s, double *dst) {
  const size_t gb = (size_t)s->g.n3 * sizeof(double);
  for (int k = 0; k < 3; ++k)
    cudaMemcpyAsync(dst + (size_t)k * s->g.n3, s->hist[k], gb,
                    cudaMemcpyDeviceToDevice, s->st);
}
void copy_hist_in(emd_system *s, const double *src) {
  const size_t gb = (size_t)s->g.n3 * sizeof(double);
  for (int k = 0; k < 3; ++k)
    cudaMemcpyAsync(s->hist[k], src + (size_t)k * s->g.n3, gb,
                    cudaMemcpyDeviceToDevice, s->st);
}

// grid dot product a . b into *dst (device)
void grid_dot(emd_system *s, const double *a, const double *b, double *dst) {
  const int nb = std::min(s->n_partials, 1024);
  emd_launch_dot_partials(s->g.n3, a, b, nullptr, nullptr, s->partials, nb, s->st);
  emd_launch_sum(s->partials, nb, dst, s->st);
}

// Reverse of one exponential T4(-i tau H) (nested stages k = 1..4 whose
// inputs are u[0..3] = u_2, u_3, u_4, psi0).  mu_in: adjoint of the output;
// on return acc holds the adjoint of psi0; gv += dL/dv_eff; gR += dL/dR.
void reverse_exponential(emd_system *s, const double2 *mu_in, double2 *acc,
                         double2 *const u[4], int which_veff, double tau,
                         double *gv, int set, double *gR) {
  Adjoint *A = s->adj;
  const OrbLayout &o = s->o;
  const size_t nel = (size_t)o.n_blk * o.n3 * o.bo;
  const double h3 = s->g.h * s->g.h * s->g.h;
  double2 *mu = A->mu, *mu2 = A->mu + nel;
  cudaMemcpyAsync(mu, mu_in, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st);
  cudaMemsetAsync(acc, 0, s->orb_bytes, s->st);
  const TableSet &t = s->ts[set];
  for (int k = 1; k <= 4; ++k) {
    const double b = tau / k;
    emd_adj_axpy(acc, mu, nel, s->st);
    emd_adj_gv(o, mu, u[k - 1], b, gv, s->st);
    emd_adj_project_grad(o, t, s->n_atoms, mu, h3, s->sp.h_kb, s->sp.inv_rc2,
                         A->cm, (double2 *)s->hc, A->dcm, s->st);
    emd_adj_project_grad(o, t, s->n_atoms, u[k - 1], h3, s->sp.h_kb,
                         s->sp.inv_rc2, A->cu, A->hcu, A->dcu, s->st);
    emd_adj_proj_sens(A->cm, A->dcm, A->cu, A->dcu, s->n_atoms, o.n_orb,
                      o.n_orb_pad, s->sp.h_kb * b / h3, gR, s->st);
    // mu <- conj(a_k) H mu = (+i b) H mu
    stage(s, mu, A->zero, mu2, set, which_veff, -b);
    std::swap(mu, mu2);
  }
  emd_adj_axpy(acc, mu, nel, s->st);
}

// (R, V, F) of the current state to dst[0..9 na) / back; positions into
// table set k with every table rebuilt.
void save_ions(emd_system *s, double *dst) {
  const size_t b = 3 * (size_t)s->n_atoms * sizeof(double);
  cudaMemcpyAsync(dst, s->ts[s->cur].R, b, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(dst + 3 * s->n_atoms, s->V, b, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(dst + 6 * s->n_atoms, s->F, b, cudaMemcpyDeviceToDevice, s->st);
}
int load_positions(emd_system *s, int k, const double *src) {
  const size_t b = 3 * (size_t)s->n_atoms * sizeof(double);
  cudaMemcpyAsync(s->ts[k].R, src, b, cudaMemcpyDeviceToDevice, s->st);
  int r = build_set(s, k);
  if (r) return r;
  negate_grid(s->ts[k].v_loc, s->g.n3, s->st);
  return EMD_OK;
}
int load_ions(emd_system *s, const double *src) {
  const size_t b = 3 * (size_t)s->n_atoms * sizeof(double);
  cudaMemcpyAsync(s->V, src + 3 * s->n_atoms, b, cudaMemcpyDeviceToDevice, s->st);
  cudaMemcpyAsync(s->F, src + 6 * s->n_atoms, b, cudaMemcpyDeviceToDevice, s->st);
  return load_positions(s, s->cur, src);
}

// Reverse of the forces F(R, psi, v_es) at table set k for the direction
// lam_F (already in A->lamF): fl, fr, fs = position terms (local, nonlocal,
// short range); w = adjoint of v_es; lam += orbital term (if lam != NULL).
// vh must hold Poisson(rho(psi)).
void reverse_forces(emd_system *s, int k, const double2 *psi, double2 *lam) {
  Adjoint *A = s->adj;
  const OrbLayout &o = s->o;
  const TableSet &t = s->ts[k];
  const double h3 = s->g.h * s->g.h * s->g.h;
  const double coef = -2.0 * s->sp.h_kb * s->cfg.occ;
  emd_adj_project_grad(o, t, s->n_atoms, psi, h3, s->sp.h_kb, s->sp.inv_rc2,
                       A->cu, A->hcu, A->dcu, s->st);
  emd_adj_force_splat(s->g, s->sp, t, A->lamF, A->w, s->st);
  if (lam)
    emd_adj_nl_force_orb(o, s->g, s->sp, t, A->lamF, A->dcu, A->cu, coef * h3,
                         lam, s->st);
  emd_adj_nl_second_moment(o, t, s->n_atoms, psi, h3, s->sp.inv_rc2, A->lamF,
                           A->m2, s->st);
  emd_adj_nl_force_r(A->cu, A->dcu, A->m2, A->lamF, s->n_atoms, o.n_orb,
                     o.n_orb_pad, coef, A->fr, s->st);
  emd_launch_local_force_hvp(s->g, s->sp, s->n_atoms, t, A->vh, t.v_loc,
                             A->lamF, s->lf_part, A->fl, s->st);
  emd_adj_sr_hvp(s->sp, s->n_atoms, t.Rw, s->g.L, A->lamF, A->fs, s->st);
}

// The adjoint with moving ions.  Forward map of step n (Sec. 5.1):
//   R' = R + dt V + c2 F;  tables at R';  psi' = T4(H(R', v2)) T4(H(R, v1)) psi;
//   F' = F(R', psi', v_H(rho') + v_loc(R')) + Z e_n z;  V' = V + c1 (F + F'),
// c1 = dt / (2M), c2 = dt^2 / (2M).  The reverse of step n, from the adjoints
// (lam_psi, Lam_0..2, lam_R, lam_V, lam_F) of state n+1, first takes
// mu_F = lam_F + c1 lam_V through the forces at R' (orbital, potential and
// position terms), then the electrons as for fixed ions (the two
// exponentials at their own table sets), converts the adjoint of v_loc(R')
// into positions, and ends with the reverse of the position update:
//   lam_R <- lam_R' (+ exponential-1 terms at R), lam_V = lam_V' + dt lam_R',
//   lam_F = c1 lam_V' + c2 lam_R'.
// The small per-atom vectors live on the host; one synchronisation per step.
int adjoint_moving(emd_system *s, int n_steps, double dt, double mu,
                   const std::vector<double> &fe, int K, int observable,
                   double *L_out, double *dL_dR, double *dL_dfield) {
  const int n_ck = (n_steps + K - 1) / K;
  int r = adj_alloc(s, n_ck, K, n_steps);
  if (r) return r;
  Adjoint *A = s->adj;
  const OrbLayout &o = s->o;
  const int n3 = s->g.n3;
  const size_t gb = (size_t)n3 * sizeof(double);
  const double h3 = s->g.h * s->g.h * s->g.h;
  const double tau = 0.5 * (dt / mu);
  const double occ = s->cfg.occ;
  const int na = s->n_atoms;
  const size_t ionw = 9 * (size_t)na;
  const double M = s->sp.mass;
  const double c1 = dt / (2.0 * M), c2 = (dt * dt) / (2.0 * M);

  // ---- forward sweep: orbitals, history and (R, V, F) every K steps
  for (int n = 0; n < n_steps; ++n) {
    if (n % K == 0) {
      const int ck = n / K;
      CK(cudaMemcpyAsync(A->ck_psi[ck], s->psi, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
      copy_hist_out(s, A->ck_hist[ck]);
      A->ck_len[ck] = s->hist_len;
      save_ions(s, A->ck_ion + ck * ionw);
    }
    r = step_once(s, dt, mu, fe[n]);
    if (r) return r;
  }
  CK(cudaMemcpyAsync(A->ck_psi[n_ck], s->psi, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
  copy_hist_out(s, A->ck_hist[n_ck]);
  A->ck_len[n_ck] = s->hist_len;
  save_ions(s, A->ck_ion + n_ck * ionw);

  // ---- observable and the adjoint of the final state
  std::vector<double> lR(3 * std::max(1, na), 0.0), lV(lR), lF(lR), mF(lR);
  std::vector<double> fl(lR), fr(lR), fs(lR), g2(lR), g1(lR), fc(lR);
  std::vector<double> dfi(n_steps, 0.0);
  CK(cudaMemsetAsync(A->lam, 0, s->orb_bytes, s->st));
  double L = 0.0;
  if (observable == EMD_OBS_DIPOLE_Z) {
    grid_dot(s, s->rho, A->saw, A->scal);
    double dot = 0.0;
    std::vector<double> Rw(3 * std::max(1, na));
    CK(cudaMemcpyAsync(&dot, A->scal, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    if (na) CK(cudaMemcpyAsync(Rw.data(), s->ts[s->cur].Rw, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    L = -h3 * dot;
    for (int J = 0; J < na; ++J) {
      L += s->sp.z * (Rw[3 * J + 2] - 0.5 * s->g.L);
      lR[3 * J + 2] += s->sp.z;
    }
    emd_adj_scale_add(o, A->lam, (const double2 *)s->psi, A->saw, -2.0 * occ * h3, s->st);
  } else {
    // L = E_KS + sum M V^2 / 2: lam_psi = 2 f h^3 H psi, lam_R = -F_KS,
    // lam_V = M V
    emd_energy e;
    r = emd_get_energy(s, &e);
    if (r) return r;
    L = e.ks + e.kin_ion;
    emd_launch_veff(s->g, s->ts[s->cur].v_loc, s->hist, 1, 0.0, s->veff1, s->veff1f, s->st);
    project(s, s->psi, s->cur);
    StageArgs a_;
    a_.u_in = s->psi;
    a_.psi0 = s->psi;
    a_.u_out = A->acc;
    a_.v_eff = s->veff1;
    a_.tab = &s->ts[s->cur];
    a_.err = s->err;
    a_.hc = s->hc;
    a_.a = 0.0;
    a_.apply_only = 1;
    emd_launch_stage(o, a_, s->st);
    std::vector<double> ones(n3, 1.0);
    CK(cudaMemcpyAsync(A->tmp, ones.data(), gb, cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    emd_adj_scale_add(o, A->lam, A->acc, A->tmp, 2.0 * occ * h3, s->st);
    forces(s, s->cur, 0.0, 0.0, 0);
    std::vector<double> F(3 * std::max(1, na)), V(3 * std::max(1, na));
    if (na) {
      CK(cudaMemcpyAsync(F.data(), s->F, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
      CK(cudaMemcpyAsync(V.data(), s->V, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    for (int i = 0; i < 3 * na; ++i) {
      lR[i] -= F[i];
      lV[i] = M * V[i];
    }
  }
  CK(cudaMemsetAsync(A->L0, 0, gb, s->st));
  CK(cudaMemsetAsync(A->L1, 0, gb, s->st));
  CK(cudaMemsetAsync(A->L2, 0, gb, s->st));
  CK(cudaMemsetAsync(A->gvloc, 0, gb, s->st));
  CK(cudaMemsetAsync(A->dfield, 0, n_steps * 8, s->st));
  const size_t ab = 3 * (size_t)na * sizeof(double);

  // ---- reverse sweep, last segment first
  int setA = 0;
  for (int ck = n_ck - 1; ck >= 0; --ck) {
    const int n0 = ck * K, n1 = std::min(n_steps, n0 + K);
    CK(cudaMemcpyAsync(s->psi, A->ck_psi[ck], s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
    copy_hist_in(s, A->ck_hist[ck]);
    s->hist_len = A->ck_len[ck];
    r = load_ions(s, A->ck_ion + ck * ionw);
    if (r) return r;
    s->c_valid = 0;
    for (int n = n0; n < n1; ++n) {
      CK(cudaMemcpyAsync(A->seg_psi[n - n0], s->psi, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
      copy_hist_out(s, A->seg_hist[n - n0]);
      A->seg_len[n - n0] = s->hist_len;
      save_ions(s, A->seg_ion + (n - n0) * ionw);
      r = step_once(s, dt, mu, fe[n]);
      if (r) return r;
    }
    // positions R_{n1} in set cur, R_{n1 - 1} in the other
    int setB = s->cur;
    setA = 1 - s->cur;
    for (int n = n1 - 1; n >= n0; --n) {
      const double2 *psi_next = n == n1 - 1 ? (const double2 *)s->psi : A->seg_psi[n + 1 - n0];
      // adjoint of F_{n+1}
      for (int i = 0; i < 3 * na; ++i) {
        mF[i] = lF[i] + c1 * lV[i];
        lF[i] = c1 * lV[i];
      }
      for (int J = 0; J < na; ++J) dfi[n] += s->sp.z * mF[3 * J + 2];
      if (na) CK(cudaMemcpyAsync(A->lamF, mF.data(), ab, cudaMemcpyHostToDevice, s->st));
      emd_launch_density(o, psi_next, occ, A->tmp2, s->st);
      emd_launch_poisson(s->g, A->tmp2, A->vh, s->fft_a, s->fft_b, s->st);
      reverse_forces(s, setB, psi_next, A->lam);
      emd_adj_lincomb(n3, A->gvloc, 1.0, A->gvloc, 1.0, A->w, 0.0, nullptr, 0.0, nullptr, s->st);
      // adjoint of rho_{n+1}: through v_Hxc (history slot 0) and v_H in v_es
      emd_adj_lincomb(n3, A->tmp3, 1.0, A->L0, 1.0, A->w, 0.0, nullptr, 0.0, nullptr, s->st);
      emd_launch_poisson(s->g, A->tmp3, A->tmp, s->fft_a, s->fft_b, s->st);
      emd_adj_rho(n3, A->tmp2, A->L0, A->tmp, s->st);
      emd_adj_scale_add(o, A->lam, psi_next, A->tmp, 2.0 * occ, s->st);
      // recompute the stage inputs of step n: exponential 1 at R_n (set A),
      // exponential 2 at R_{n+1} (set B)
      const double2 *psi_n = A->seg_psi[n - n0];
      const double *hn = A->seg_hist[n - n0];
      const double *hp[3] = {hn, hn + n3, hn + 2 * (size_t)n3};
      const int len = A->seg_len[n - n0];
      emd_launch_veff(s->g, s->ts[setA].v_loc, hp, 1, fe[n], s->veff1, s->veff1f, s->st);
      emd_launch_veff(s->g, s->ts[setB].v_loc, hp, len, fe[n], s->veff2, s->veff2f, s->st);
      double2 *const *U = A->st_u.data();
      project(s, psi_n, setA);
      stage(s, psi_n, psi_n, U[0], setA, 1, tau / 4.0);
      project(s, U[0], setA);
      stage(s, U[0], psi_n, U[1], setA, 1, tau / 3.0);
      project(s, U[1], setA);
      stage(s, U[1], psi_n, U[2], setA, 1, tau / 2.0);
      project(s, U[2], setA);
      stage(s, U[2], psi_n, U[3], setA, 1, tau);
      project(s, U[3], setB);
      stage(s, U[3], U[3], U[4], setB, 2, tau / 4.0);
      project(s, U[4], setB);
      stage(s, U[4], U[3], U[5], setB, 2, tau / 3.0);
      project(s, U[5], setB);
      stage(s, U[5], U[3], U[6], setB, 2, tau / 2.0);
      CK(cudaMemsetAsync(A->gv2, 0, gb, s->st));
      CK(cudaMemsetAsync(A->gv1, 0, gb, s->st));
      if (na) {
        CK(cudaMemsetAsync(A->gR, 0, ab, s->st));
        CK(cudaMemsetAsync(A->gR1, 0, ab, s->st));
      }
      double2 *const in2[4] = {U[6], U[5], U[4], U[3]};
      reverse_exponential(s, A->lam, A->acc, in2, 2, tau, A->gv2, setB, A->gR);
      double2 *const in1[4] = {U[2], U[1], U[0], (double2 *)psi_n};
      reverse_exponential(s, A->acc, A->lam, in1, 1, tau, A->gv1, setA, A->gR1);
      // v_loc(R_{n+1}) adjoint complete: to positions, then restart with gv1
      emd_adj_lincomb(n3, A->gvloc, 1.0, A->gvloc, 1.0, A->gv2, 0.0, nullptr, 0.0, nullptr, s->st);
      emd_launch_poisson(s->g, A->gvloc, A->tmp, s->fft_a, s->fft_b, s->st);
      emd_launch_local_force(s->g, s->sp, na, s->ts[setB], A->tmp, A->zgrid,
                             s->lf_part, A->fconv, s->st);
      emd_adj_lincomb(n3, A->tmp, 1.0, A->gv1, 1.0, A->gv2, 0.0, nullptr, 0.0, nullptr, s->st);
      grid_dot(s, A->tmp, A->saw, A->dfield + n);
      emd_adj_lincomb(n3, A->gvloc, 1.0, A->gv1, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, s->st);
      const double x0 = len <= 1 ? 1.0 : len == 2 ? 2.0 : 3.0;
      const double x1 = len <= 1 ? 0.0 : len == 2 ? -1.0 : -3.0;
      const double x2 = len <= 2 ? 0.0 : 1.0;
      emd_adj_lincomb(n3, A->tmp, 1.0, A->L1, 1.0, A->gv1, x0, A->gv2, 0.0, nullptr, s->st);
      emd_adj_lincomb(n3, A->L1, 1.0, A->L2, x1, A->gv2, 0.0, nullptr, 0.0, nullptr, s->st);
      emd_adj_lincomb(n3, A->L2, x2, A->gv2, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, s->st);
      std::swap(A->L0, A->tmp);
      r = launch_check("emd_propagate_adjoint");
      if (r) return r;
      if (na) {
        CK(cudaMemcpyAsync(fl.data(), A->fl, ab, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(fr.data(), A->fr, ab, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(fs.data(), A->fs, ab, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(g2.data(), A->gR, ab, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(g1.data(), A->gR1, ab, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(fc.data(), A->fconv, ab, cudaMemcpyDeviceToHost, s->st));
      }
      CK(cudaStreamSynchronize(s->st));
      for (int i = 0; i < 3 * na; ++i) {
        const double lr1 = lR[i] + fl[i] + fr[i] + fs[i] + g2[i] - fc[i] / h3;
        lR[i] = lr1 + g1[i];
        lV[i] += dt * lr1;
        lF[i] += c2 * lr1;
      }
      if (n > n0) {
        // set B now takes R_{n-1}; set A (R_n) becomes the next step's B
        r = load_positions(s, setB, A->seg_ion + (n - 1 - n0) * ionw);
        if (r) return r;
        std::swap(setA, setB);
      }
    }
  }

  // ---- the initial forces F(R_0, psi_0, v_es_0) and v_loc(R_0)
  for (int i = 0; i < 3 * na; ++i) mF[i] = lF[i];
  if (na) CK(cudaMemcpyAsync(A->lamF, mF.data(), ab, cudaMemcpyHostToDevice, s->st));
  emd_launch_density(o, A->seg_psi[0], occ, A->tmp2, s->st);
  emd_launch_poisson(s->g, A->tmp2, A->vh, s->fft_a, s->fft_b, s->st);
  reverse_forces(s, setA, A->seg_psi[0], nullptr);
  emd_adj_lincomb(n3, A->gvloc, 1.0, A->gvloc, 1.0, A->w, 0.0, nullptr, 0.0, nullptr, s->st);
  emd_launch_poisson(s->g, A->gvloc, A->tmp, s->fft_a, s->fft_b, s->st);
  emd_launch_local_force(s->g, s->sp, na, s->ts[setA], A->tmp, A->zgrid,
                         s->lf_part, A->fconv, s->st);
  if (na) {
    CK(cudaMemcpyAsync(fl.data(), A->fl, ab, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(fr.data(), A->fr, ab, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(fs.data(), A->fs, ab, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(fc.data(), A->fconv, ab, cudaMemcpyDeviceToHost, s->st));
  }
  std::vector<double> df(n_steps);
  CK(cudaMemcpyAsync(df.data(), A->dfield, n_steps * 8, cudaMemcpyDeviceToHost, s->st));
  // leave the system at the final state
  CK(cudaMemcpyAsync(s->psi, A->ck_psi[n_ck], s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
  copy_hist_in(s, A->ck_hist[n_ck]);
  s->hist_len = A->ck_len[n_ck];
  r = load_ions(s, A->ck_ion + n_ck * ionw);
  if (r) return r;
  s->c_valid = 0;
  electrons(s, 0);
  CK(cudaStreamSynchronize(s->st));
  for (int i = 0; i < 3 * na; ++i)
    dL_dR[i] = lR[i] + fl[i] + fr[i] + fs[i] - fc[i] / h3;
  if (dL_dfield)
    for (int i = 0; i < n_steps; ++i) dL_dfield[i] = df[i] + dfi[i];
  *L_out = L;
  r = launch_check("emd_propagate_adjoint");
  if (r) return r;
  return read_err_flag(s);
}

}  // namespace

extern "C" {

int emd_propagate_adjoint(emd_system *s, int n_steps, double dt, double mu,
                          const double *field, int ckpt_every, int observable,
                          double *L_out, double *dL_dR, double *dL_dfield) {
  g_err.clear();
  if (s && s->sp.nch > 1)
    return fail(EMD_EINVAL, "the adjoint covers the s-projector only (species lmax = 0)");
  int r = check_propagate(s, dt, mu);
  if (r) return r;
  if (s->o.prec != EMD_FP64)
    return fail(EMD_EINVAL, "adjoint propagation needs FP64 orbitals");
  if (n_steps < 1 || ckpt_every < 1)
    return fail(EMD_EINVAL, "n_steps and ckpt_every must be >= 1");
  if (observable != EMD_OBS_ENERGY && observable != EMD_OBS_DIPOLE_Z)
    return fail(EMD_EINVAL, "unknown observable %d", observable);
  if (!L_out || (!dL_dR && s->n_atoms) || (field && !dL_dfield))
    return fail(EMD_EINVAL, "NULL output");
  std::vector<double> fe(n_steps, 0.0);
  if (field)
    for (int i = 0; i < n_steps; ++i) {
      if (!std::isfinite(field[i])) return fail(EMD_EINVAL, "non-finite field");
      fe[i] = field[i];
    }
  const int K = std::min(ckpt_every, n_steps);
  if (!s->frozen_ions)
    return adjoint_moving(s, n_steps, dt, mu, fe, K, observable, L_out, dL_dR,
                          dL_dfield);
  const int n_ck = (n_steps + K - 1) / K;
  r = adj_alloc(s, n_ck, K, n_steps);
  if (r) return r;
  Adjoint *A = s->adj;
  const OrbLayout &o = s->o;
  const int n3 = s->g.n3;
  const size_t gb = (size_t)n3 * sizeof(double);
  const double h3 = s->g.h * s->g.h * s->g.h;
  const double tau = 0.5 * (dt / mu);
  const double occ = s->cfg.occ;
  const int na = s->n_atoms;

  // ---- forward sweep with orbital + history checkpoints every K steps
  for (int n = 0; n < n_steps; ++n) {
    if (n % K == 0) {
      const int ck = n / K;
      CK(cudaMemcpyAsync(A->ck_psi[ck], s->psi, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
      copy_hist_out(s, A->ck_hist[ck]);
      A->ck_len[ck] = s->hist_len;
    }
    r = step_once(s, dt, mu, fe[n]);
    if (r) return r;
  }
  CK(cudaMemcpyAsync(A->ck_psi[n_ck], s->psi, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
  copy_hist_out(s, A->ck_hist[n_ck]);
  A->ck_len[n_ck] = s->hist_len;

  // ---- observable and the adjoint of the final state
  std::vector<double> gR_host(3 * std::max(1, na), 0.0);
  CK(cudaMemsetAsync(A->lam, 0, s->orb_bytes, s->st));
  double L = 0.0;
  if (observable == EMD_OBS_DIPOLE_Z) {
    grid_dot(s, s->rho, A->saw, A->scal);
    double dot = 0.0;
    std::vector<double> Rw(3 * std::max(1, na));
    CK(cudaMemcpyAsync(&dot, A->scal, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    if (na) CK(cudaMemcpyAsync(Rw.data(), s->ts[s->cur].Rw, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    L = -h3 * dot;
    for (int J = 0; J < na; ++J) {
      L += s->sp.z * (Rw[3 * J + 2] - 0.5 * s->g.L);
      gR_host[3 * J + 2] += s->sp.z;
    }
    emd_adj_scale_add(o, A->lam, (const double2 *)s->psi, A->saw, -2.0 * occ * h3, s->st);
  } else {
    emd_energy e;
    r = emd_get_energy(s, &e);
    if (r) return r;
    L = e.ks;
    // lambda = 2 f h^3 H[rho_N] psi_N ; dL/dR = -F at fixed orbitals
    emd_launch_veff(s->g, s->ts[s->cur].v_loc, s->hist, 1, 0.0, s->veff1, s->veff1f, s->st);
    project(s, s->psi, s->cur);
    StageArgs a_;
    a_.u_in = s->psi;
    a_.psi0 = s->psi;
    a_.u_out = A->acc;
    a_.v_eff = s->veff1;
    a_.tab = &s->ts[s->cur];
    a_.err = s->err;
    a_.hc = s->hc;
    a_.a = 0.0;
    a_.apply_only = 1;
    emd_launch_stage(o, a_, s->st);
    // w = 1 on every point: tmp as a grid of ones
    std::vector<double> ones(n3, 1.0);
    CK(cudaMemcpyAsync(A->tmp, ones.data(), gb, cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    emd_adj_scale_add(o, A->lam, A->acc, A->tmp, 2.0 * occ * h3, s->st);
    s->c_valid = 1;
    forces(s, s->cur, 0.0, 0.0, 0);
    std::vector<double> F(3 * std::max(1, na));
    if (na) CK(cudaMemcpyAsync(F.data(), s->F, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int i = 0; i < 3 * na; ++i) gR_host[i] -= F[i];
  }
  CK(cudaMemsetAsync(A->L0, 0, gb, s->st));
  CK(cudaMemsetAsync(A->L1, 0, gb, s->st));
  CK(cudaMemsetAsync(A->L2, 0, gb, s->st));
  CK(cudaMemsetAsync(A->gvloc, 0, gb, s->st));
  CK(cudaMemsetAsync(A->gR, 0, 3 * std::max(1, na) * 8, s->st));
  CK(cudaMemsetAsync(A->dfield, 0, n_steps * 8, s->st));

  // ---- reverse sweep, last segment first
  for (int ck = n_ck - 1; ck >= 0; --ck) {
    const int n0 = ck * K, n1 = std::min(n_steps, n0 + K);
    CK(cudaMemcpyAsync(s->psi, A->ck_psi[ck], s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
    copy_hist_in(s, A->ck_hist[ck]);
    s->hist_len = A->ck_len[ck];
    s->c_valid = 0;
    for (int n = n0; n < n1; ++n) {
      CK(cudaMemcpyAsync(A->seg_psi[n - n0], s->psi, s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
      copy_hist_out(s, A->seg_hist[n - n0]);
      A->seg_len[n - n0] = s->hist_len;
      r = step_once(s, dt, mu, fe[n]);
      if (r) return r;
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const double2 *psi_next = n == n1 - 1 ? (const double2 *)s->psi : A->seg_psi[n + 1 - n0];
      // adjoint of v_Hxc(rho_{n+1}) (history slot 0 of step n+1) -> psi_{n+1}
      emd_launch_density(o, psi_next, occ, A->tmp2, s->st);
      emd_launch_poisson(s->g, A->L0, A->tmp, s->fft_a, s->fft_b, s->st);
      emd_adj_rho(n3, A->tmp2, A->L0, A->tmp, s->st);
      emd_adj_scale_add(o, A->lam, psi_next, A->tmp, 2.0 * occ, s->st);
      // recompute the stage inputs of step n
      const double2 *psi_n = A->seg_psi[n - n0];
      const double *hn = A->seg_hist[n - n0];
      const double *hp[3] = {hn, hn + n3, hn + 2 * (size_t)n3};
      const int len = A->seg_len[n - n0];
      emd_launch_veff(s->g, s->ts[s->cur].v_loc, hp, 1, fe[n], s->veff1, s->veff1f, s->st);
      emd_launch_veff(s->g, s->ts[s->cur].v_loc, hp, len, fe[n], s->veff2, s->veff2f, s->st);
      double2 *const *U = A->st_u.data();
      // exponential 1 from psi_n: U0 = u4, U1 = u3, U2 = u2, U3 = output psi1
      project(s, psi_n, s->cur);
      stage(s, psi_n, psi_n, U[0], s->cur, 1, tau / 4.0);
      project(s, U[0], s->cur);
      stage(s, U[0], psi_n, U[1], s->cur, 1, tau / 3.0);
      project(s, U[1], s->cur);
      stage(s, U[1], psi_n, U[2], s->cur, 1, tau / 2.0);
      project(s, U[2], s->cur);
      stage(s, U[2], psi_n, U[3], s->cur, 1, tau);
      // exponential 2 from psi1 = U3: U4 = u4', U5 = u3', U6 = u2'
      project(s, U[3], s->cur);
      stage(s, U[3], U[3], U[4], s->cur, 2, tau / 4.0);
      project(s, U[4], s->cur);
      stage(s, U[4], U[3], U[5], s->cur, 2, tau / 3.0);
      project(s, U[5], s->cur);
      stage(s, U[5], U[3], U[6], s->cur, 2, tau / 2.0);
      // reverse exponential 2 then exponential 1
      CK(cudaMemsetAsync(A->gv2, 0, gb, s->st));
      CK(cudaMemsetAsync(A->gv1, 0, gb, s->st));
      double2 *const in2[4] = {U[6], U[5], U[4], U[3]};
      reverse_exponential(s, A->lam, A->acc, in2, 2, tau, A->gv2, s->cur, A->gR);
      double2 *const in1[4] = {U[2], U[1], U[0], (double2 *)psi_n};
      reverse_exponential(s, A->acc, A->lam, in1, 1, tau, A->gv1, s->cur, A->gR);
      // field, ionic potential and history adjoints
      emd_adj_lincomb(n3, A->tmp, 1.0, A->gv1, 1.0, A->gv2, 0.0, nullptr, 0.0, nullptr, s->st);
      grid_dot(s, A->tmp, A->saw, A->dfield + n);
      emd_adj_lincomb(n3, A->gvloc, 1.0, A->gvloc, 1.0, A->tmp, 0.0, nullptr, 0.0, nullptr, s->st);
      const double x0 = len <= 1 ? 1.0 : len == 2 ? 2.0 : 3.0;
      const double x1 = len <= 1 ? 0.0 : len == 2 ? -1.0 : -3.0;
      const double x2 = len <= 2 ? 0.0 : 1.0;
      // new L0 = L1 + gv1 + x0 gv2 ; L1 = L2 + x1 gv2 ; L2 = x2 gv2
      emd_adj_lincomb(n3, A->tmp, 1.0, A->L1, 1.0, A->gv1, x0, A->gv2, 0.0, nullptr, s->st);
      emd_adj_lincomb(n3, A->L1, 1.0, A->L2, x1, A->gv2, 0.0, nullptr, 0.0, nullptr, s->st);
      emd_adj_lincomb(n3, A->L2, x2, A->gv2, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, s->st);
      std::swap(A->L0, A->tmp);
      r = launch_check("emd_propagate_adjoint");
      if (r) return r;
    }
  }

  // ---- ionic potential adjoint: dL/dR_J = -h^-3 F_loc[w], w = Poisson(gvloc)
  emd_launch_poisson(s->g, A->gvloc, A->tmp, s->fft_a, s->fft_b, s->st);
  emd_launch_local_force(s->g, s->sp, na, s->ts[s->cur], A->tmp, A->zgrid,
                         s->lf_part, s->F_loc, s->st);
  std::vector<double> Fw(3 * std::max(1, na)), gRd(3 * std::max(1, na));
  if (na) {
    CK(cudaMemcpyAsync(Fw.data(), s->F_loc, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(gRd.data(), A->gR, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
  }
  if (dL_dfield)
    CK(cudaMemcpyAsync(dL_dfield, A->dfield, n_steps * 8, cudaMemcpyDeviceToHost, s->st));
  // leave the system at the final state
  CK(cudaMemcpyAsync(s->psi, A->ck_psi[n_ck], s->orb_bytes, cudaMemcpyDeviceToDevice, s->st));
  copy_hist_in(s, A->ck_hist[n_ck]);
  s->hist_len = A->ck_len[n_ck];
  s->c_valid = 0;
  electrons(s, 0);
  CK(cudaStreamSynchronize(s->st));
  for (int i = 0; i < 3 * na; ++i)
    dL_dR[i] = gR_host[i] + gRd[i] - Fw[i] / h3;
  *L_out = L;
  r = launch_check("emd_propagate_adjoint");
  if (r) return r;
  return read_err_flag(s);
}

int emd_get_forces(emd_system *s, double *F) {
  g_err.clear();
  if (!s || (!F && s->n_atoms)) return fail(EMD_EINVAL, "NULL argument");
  int r = ensure_state(s);
  if (r) return r;
  r = read_err_flag(s);
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
  int r0 = ensure_state(s);
  if (r0) return r0;
  const int cur = s->cur;
  const double h3 = s->g.h * s->g.h * s->g.h;
  int np = 0;
  double kin_scale = 1.0;
  if (s->o.prec == EMD_FP32_ORBITALS)
    kin_scale = kinetic_fp32(s, &np);
  else
    emd_launch_kinetic_partials(s->o, s->psi, s->partials, &np, s->st);
  emd_launch_sum(s->partials, np, s->scal + 0, s->st);
  if (!s->c_valid) {
    project(s, s->psi, cur);
    s->c_valid = 1;
  }
  {
    // nl = occ sum_P h_P |c_P|^2: weights 1 with one projector (times h_kb below)
    const double w1[3] = {1.0, 1.0, 1.0};
    emd_launch_abs2_sum(s->c, s->o.n_proj * s->o.n_orb_pad, s->o.n_orb_pad, s->sp.nch,
                        s->sp.nch > 1 ? s->sp.hl : w1, s->scal + 1, s->st);
  }
  const int nb = std::min(s->n_partials, 1024);
  emd_launch_dot_partials(s->g.n3, s->rho, s->v_h, s->ts[cur].g_ion,
                          s->ts[cur].v_loc, s->partials, nb, s->st);
  emd_launch_sum(s->partials, nb, s->scal + 2, s->st);
  emd_launch_short_range(s->sp, s->n_atoms, s->ts[cur].Rw, s->g.L, s->F_sr,
                         s->e_sr, s->sr_part, s->st);
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
  out->kin_e = occ * h3 * kin_scale * hs[0];
  out->nl = s->sp.nch > 1 ? occ * hs[1] : occ * s->sp.h_kb * hs[1];
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
  const double n_expect = occupation_sum(s);
  if (!std::isfinite(out->total) || std::fabs(out->n_elec - n_expect) > 1e-3 * n_expect)
    return fail(EMD_EUNSTABLE, "density normalisation lost: h^3 sum rho = %g, "
                "expected %g", out->n_elec, n_expect);
  return EMD_OK;
}

int emd_get_state(emd_system *s, double *R, double *V, double *psi, double *rho) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  int r = ensure_state(s);
  if (r) return r;
  r = read_err_flag(s);
  if (r) return r;
  if (R && s->n_atoms)
    CK(cudaMemcpyAsync(R, s->ts[s->cur].R, 3 * s->n_atoms * 8,
                       cudaMemcpyDeviceToHost, s->st));
  if (V && s->n_atoms)
    CK(cudaMemcpyAsync(V, s->V, 3 * s->n_atoms * 8, cudaMemcpyDeviceToHost, s->st));
  if (rho)
    CK(cudaMemcpyAsync(rho, s->rho, s->g.n3 * 8, cudaMemcpyDeviceToHost, s->st));
  if (psi) {
    r = download_orbitals(s, s->psi, s->o.n_orb, psi, s->f_uniform ? nullptr : s->occ_winv);
    if (r) return r;
  }
  CK(cudaStreamSynchronize(s->st));
  return EMD_OK;
}

int emd_get_potentials(emd_system *s, double *v_loc, double *v_h, double *v_xc,
                       double *g_ion) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  int r = ensure_state(s);
  if (r) return r;
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
  int r = ensure_state(s);
  if (r) return r;
  if (!s->c_valid) {
    project(s, s->psi, s->cur);
    s->c_valid = 1;
  }
  for (int P = 0; P < s->o.n_proj; ++P)
    CK(cudaMemcpyAsync(c + 2 * (size_t)P * s->o.n_orb, s->c + (size_t)P * s->o.n_orb_pad,
                       (size_t)s->o.n_orb * 16, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (!s->f_uniform)                        // projections of phi_A, not of u_A
    for (int P = 0; P < s->o.n_proj; ++P)
      for (int i = 0; i < s->o.n_orb; ++i) {
        const double w = std::sqrt(s->f[i] / s->cfg.occ);
        c[2 * ((size_t)P * s->o.n_orb + i)] /= w;
        c[2 * ((size_t)P * s->o.n_orb + i) + 1] /= w;
      }
  return read_err_flag(s);
}

int emd_apply_hamiltonian(emd_system *s, int n_vec, const double *psi,
                          double *hpsi) {
  g_err.clear();
  if (!s || !psi || !hpsi) return fail(EMD_EINVAL, "NULL argument");
  if (n_vec < 1 || n_vec > s->o.n_orb)
    return fail(EMD_EINVAL, "n_vec must be in [1, n_orb]");
  if (!s->ions_set || !s->orbs_set) return fail(EMD_ESTATE, "set ions and orbitals first");
  int r = ensure_state(s);
  if (r) return r;
  CK(cudaMemsetAsync(s->ua, 0, s->orb_bytes, s->st));
  r = upload_orbitals(s, psi, n_vec, s->ua);
  if (r) return r;
  OrbLayout o = s->o;
  o.n_blk = (n_vec + o.bo - 1) / o.bo;
  emd_launch_veff(s->g, s->ts[s->cur].v_loc, s->hist, 1, 0.0, s->veff1,
                  s->veff1f, s->st, s->veff1d, s->o.w[0]);
  if (o.prec == EMD_FP32_ORBITALS)
    emd_launch_project_tile(o, s->ts[s->cur], s->n_atoms, s->ua,
                            s->g.h * s->g.h * s->g.h, s->sp.h_kb, s->c, s->hc,
                            s->proj_part, s->st);
  else
    emd_launch_project(o, s->ts[s->cur], s->n_atoms, s->ua,
                       s->g.h * s->g.h * s->g.h, s->sp.h_kb, s->c, s->hc, s->st);
  s->c_valid = 0;
  StageArgs a;
  a.u_in = s->ua;
  a.psi0 = s->ua;
  a.u_out = s->ub;
  a.v_eff = s->o.prec == EMD_FP64 ? (const void *)s->veff1 : (const void *)s->veff1f;
  if (s->o.prec != EMD_FP64) a.v_diag = s->veff1d;
  a.tab = &s->ts[s->cur];
  a.err = s->err;
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

}  // extern "C"

// ---------------------------------------------------------------------------
// Ground state at fixed ions (Sec. 4.1, eqs. EoM_BO_a, EoM_BO_b): Chebyshev-
// filtered subspace iteration with Rayleigh-Ritz and Anderson mixing of rho.
// ---------------------------------------------------------------------------

struct GroundStateWork {
  static constexpr int kHist = 6;          // Anderson history
  OrbLayout og;                            // the subspace: n_orb + buffer states
  int n_occ = 0;
  void *A = nullptr, *B = nullptr, *C = nullptr;   // three sets in layout og
  double2 *c = nullptr;                    // projections of the subspace
  void *hc = nullptr;
  double2 *part = nullptr;                 // per-tile projection partials
  double2 *Sz = nullptr, *Hz = nullptr;             // m x m, FP64 (Hz: then V)
  double2 *gpart = nullptr;                         // subspace-product partials
  double *rho_in = nullptr, *rho_out = nullptr;
  double *wd = nullptr;                             // occupation weights sqrt(f / occ)
  double *hr[kHist] = {}, *hf[kHist] = {};          // rho_in and F = rho_out - rho_in
  std::vector<void *> mem;
};

namespace {

void gs_release(GroundStateWork *g) {
  if (!g) return;
  for (void *p : g->mem) cudaFree(p);
  delete g;
}

// Buffer states above the occupied ones: the Chebyshev filter damps the
// spectrum above the largest Ritz value of the whole subspace, so the
// occupied edge needs states above it (otherwise an occupied state missing
// from the start rotates in only slowly).
int gs_buffer_states(int n_orb) { return std::max(4, (n_orb + 9) / 10); }

int gs_setup(emd_system *s) {
  if (s->gsw) return EMD_OK;
  GroundStateWork *g = new GroundStateWork();
  g->n_occ = s->o.n_orb;
  g->og = s->o;
  g->og.n_orb = s->o.n_orb + gs_buffer_states(s->o.n_orb);
  g->og.n_blk = (g->og.n_orb + g->og.bo - 1) / g->og.bo;
  g->og.n_orb_pad = g->og.n_blk * g->og.bo;
  const int m = g->og.n_orb;
  const size_t n3 = s->g.n3;
  const size_t esz = s->o.prec == EMD_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t set_bytes = (size_t)g->og.n_blk * n3 * g->og.bo * esz;
  const int nt = (s->g.n + EMD_TILE - 1) / EMD_TILE;
  const size_t ntiles = (size_t)nt * nt * nt;
  const size_t na = std::max(1, s->n_atoms);
  auto A = [&](void **p, size_t b) {
    if (cudaMalloc(p, b) != cudaSuccess) return false;
    g->mem.push_back(*p);
    return true;
  };
  bool ok = A(&g->A, set_bytes) && A(&g->B, set_bytes) && A(&g->C, set_bytes) &&
       A((void **)&g->c, na * g->og.n_orb_pad * sizeof(double2)) &&
       A(&g->hc, na * g->og.n_orb_pad * esz) &&
       A((void **)&g->part, ntiles * EMD_TILE_ATOM_MAX * g->og.n_orb_pad * sizeof(double2)) &&
       A((void **)&g->Sz, (size_t)m * m * 16) && A((void **)&g->Hz, (size_t)m * m * 16) &&
       A((void **)&g->gpart, emd_gram_scratch((int)n3, m) * sizeof(double2)) &&
       A((void **)&g->rho_in, n3 * 8) &&
       A((void **)&g->rho_out, n3 * 8) && A((void **)&g->wd, (size_t)m * 8);
  for (int k = 0; ok && k < GroundStateWork::kHist; ++k)
    ok = A((void **)&g->hr[k], n3 * 8) && A((void **)&g->hf[k], n3 * 8);
  if (!ok) {
    gs_release(g);
    return fail(EMD_ENOMEM, "ground-state workspace: allocation failed");
  }
  s->gsw = g;
  return EMD_OK;
}

// u_out = H u_in over the subspace (layout og), H with the potential in
// veff1 (and its complex64 forms) and the projectors of the current set
void gs_apply(emd_system *s, const void *u_in, void *u_out) {
  GroundStateWork *g = s->gsw;
  const double h3 = s->g.h * s->g.h * s->g.h;
  if (s->o.prec == EMD_FP32_ORBITALS)
    emd_launch_project_tile(g->og, s->ts[s->cur], s->n_atoms, u_in, h3, s->sp.h_kb, g->c,
                            g->hc, g->part, s->st);
  else
    emd_launch_project(g->og, s->ts[s->cur], s->n_atoms, u_in, h3, s->sp.h_kb, g->c, g->hc,
                       s->st);
  StageArgs a;
  a.u_in = u_in;
  a.psi0 = u_in;
  a.u_out = u_out;
  a.v_eff = s->o.prec == EMD_FP64 ? (const void *)s->veff1 : (const void *)s->veff1f;
  if (s->o.prec != EMD_FP64) a.v_diag = s->veff1d;
  a.tab = &s->ts[s->cur];
  a.err = s->err;
  a.hc = g->hc;
  a.a = 0.0;
  a.apply_only = 1;
  emd_launch_stage(g->og, a, s->st);
}

// veff1 = v_loc + v_H[rho] + v_xc[rho]; hist[0] holds v_H + v_xc
void gs_potential(emd_system *s, const double *rho) {
  emd_launch_poisson(s->g, rho, s->v_h, s->fft_a, s->fft_b, s->st);
  emd_launch_lda(s->g.n3, rho, s->v_h, s->eps_xc, s->v_xc, s->hist[0], s->st);
  emd_launch_veff(s->g, s->ts[s->cur].v_loc, s->hist, 1, 0.0, s->veff1, s->veff1f, s->st,
                  s->o.prec == EMD_FP64 ? nullptr : s->veff1d, s->o.w[0]);
}

void gs_pack(const OrbLayout &o, const void *canon, void *u, int n_vec, cudaStream_t st) {
  if (o.prec == EMD_FP64) emd_launch_pack(o, (const double2 *)canon, u, n_vec, st);
  else emd_launch_pack_c64(o, (const float2 *)canon, u, n_vec, st);
}

void gs_unpack(const OrbLayout &o, const void *u, void *canon, int n_vec, cudaStream_t st) {
  if (o.prec == EMD_FP64) emd_launch_unpack(o, u, (double2 *)canon, n_vec, st);
  else emd_launch_unpack_c64(o, u, (float2 *)canon, n_vec, st);
}

// A <- Chebyshev polynomial of degree m of H applied to A, damping [a, b]
// and scaled to 1 at a0 < a (three-term recurrence in the scaled form of
// Zhou and Saad); B and C are work sets.
int gs_filter(emd_system *s, int m, double a, double b, double a0) {
  GroundStateWork *g = s->gsw;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  double sigma = e / (a0 - c);
  const double gamma = 2.0 / sigma;
  const size_t nel = (size_t)g->og.n_blk * s->g.n3 * g->og.bo;
  const size_t bytes = nel * (s->o.prec == EMD_FP64 ? sizeof(double2) : sizeof(float2));
  void *X = g->A, *Y = g->B, *W = g->C;
  gs_apply(s, X, W);
  emd_launch_cheb(s->o.prec, nel, W, X, Y, sigma / e, c, 0.0, s->st);
  for (int i = 2; i <= m; ++i) {
    const double sigma2 = 1.0 / (gamma - sigma);
    gs_apply(s, Y, W);
    emd_launch_cheb(s->o.prec, nel, W, Y, X, 2.0 * sigma2 / e, c, sigma * sigma2, s->st);
    std::swap(X, Y);
    sigma = sigma2;
  }
  if (Y != g->A) CK(cudaMemcpyAsync(g->A, Y, bytes, cudaMemcpyDeviceToDevice, s->st));
  return launch_check("ground state Chebyshev filter");
}


// A <- Rayleigh-Ritz vectors of span(A) (h^3-orthonormal, ascending Ritz
// values into eps); on return B holds them canonically (column-major
// n3 x m), so the occupied ones are its first n_occ columns.
int gs_rayleigh_ritz(emd_system *s, std::vector<double> &eps) {
  GroundStateWork *g = s->gsw;
  const OrbLayout &og = g->og;
  const int m = og.n_orb;
  const int n3 = s->g.n3;
  const double h3 = s->g.h * s->g.h * s->g.h;
  const bool f64 = s->o.prec == EMD_FP64;
  gs_apply(s, g->A, g->B);
  gs_unpack(og, g->A, g->C, m, s->st);      // X (canonical) in C
  gs_unpack(og, g->B, g->A, m, s->st);      // H X (canonical) in A
  const int prec = f64 ? EMD_FP64 : EMD_FP32_ORBITALS;
  emd_launch_gram(prec, g->C, g->C, n3, m, h3, g->gpart, g->Sz, s->st);
  emd_launch_gram(prec, g->C, g->A, n3, m, h3, g->gpart, g->Hz, s->st);
  std::vector<std::complex<double>> Sh((size_t)m * m), Hh((size_t)m * m), Vh;
  CK(cudaMemcpyAsync(Sh.data(), g->Sz, (size_t)m * m * 16, cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(Hh.data(), g->Hz, (size_t)m * m * 16, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (!emd_host::hermitian_generalized_eig(m, Hh, Sh, eps, Vh))
    return fail(EMD_ECUDA, "subspace eigenproblem: the overlap matrix is not positive "
                           "definite (the filtered set lost rank), or its QR iteration "
                           "did not converge");
  // X V (V = eigenvectors, ascending Ritz values) into B (canonical), packed into A
  CK(cudaMemcpyAsync(g->Hz, Vh.data(), (size_t)m * m * 16, cudaMemcpyHostToDevice, s->st));
  emd_launch_rotate(prec, g->C, g->Hz, n3, m, g->B, s->st);
  gs_pack(og, g->B, g->A, m, s->st);
  return launch_check("ground state Rayleigh-Ritz");
}

// density of the occupied Ritz vectors (the first n_occ columns of the
// canonical set in B), packed into C with the occupied blocks only; with
// weights w (device, sqrt(f_A / occ)) rho = sum_A f_A |phi_A|^2, else
// occ sum_A |phi_A|^2
void gs_density(emd_system *s, double *rho, const double *w) {
  GroundStateWork *g = s->gsw;
  OrbLayout oo = g->og;
  oo.n_orb = g->n_occ;
  oo.n_blk = (g->n_occ + oo.bo - 1) / oo.bo;
  oo.n_orb_pad = oo.n_blk * oo.bo;
  gs_pack(oo, g->B, g->C, g->n_occ, s->st);
  if (w) emd_launch_scale_orbitals(oo, g->C, g->n_occ, w, s->st);
  emd_launch_density(oo, g->C, s->cfg.occ, rho, s->st);
}




}  // namespace

extern "C" {

int emd_ground_state_smeared(emd_system *s, int max_scf, double tol, int degree, double mix,
                             double kT, double n_electrons, double kerker_q0,
                             double *eigenvalues, double *occupations, emd_gs_info *info) {
  g_err.clear();
  if (!s) return fail(EMD_EINVAL, "NULL system");
  if (s->sp.nch > 1)
    return fail(EMD_EINVAL, "the ground-state solver covers the s-projector only (species lmax = 0)");
  if (!s->ions_set || !s->orbs_set) return fail(EMD_ESTATE, "set ions and orbitals first");
  if (max_scf < 1 || !(tol > 0.0) || degree < 1 || degree > 64 || !(mix > 0.0) || mix > 1.0)
    return fail(EMD_EINVAL, "need max_scf >= 1, tol > 0, 1 <= degree <= 64, 0 < mix <= 1");
  const double occ = s->cfg.occ;
  if (!(kT >= 0.0) || !std::isfinite(kT) || !(kerker_q0 >= 0.0) || !std::isfinite(kerker_q0))
    return fail(EMD_EINVAL, "need kT >= 0 and kerker_q0 >= 0 (finite)");
  if (kT > 0.0 && !(n_electrons > 0.0 && n_electrons < occ * s->o.n_orb))
    return fail(EMD_EINVAL, "with kT > 0 need 0 < n_electrons < occ n_orb = %g",
                occ * s->o.n_orb);
  int r = gs_setup(s);
  if (r) return r;
  GroundStateWork *g = s->gsw;
  const int n_occ = g->n_occ, m = g->og.n_orb;
  const int n3 = s->g.n3;
  const double h3 = s->g.h * s->g.h * s->g.h;
  const bool smear = kT > 0.0;
  const double n_e = smear ? n_electrons : occ * n_occ;
  const int nb = std::min(s->n_partials, 1024);
  constexpr int K = GroundStateWork::kHist;
  s->c_valid = 0;
  s->needs_restart = 1;                     // whatever happens, derived state is stale
  // starting subspace: the current orbitals (occupation weights removed) and
  // random buffer states; starting density: theirs, scaled to n_e electrons
  gs_unpack(s->o, s->psi, g->B, n_occ, s->st);
  if (!s->f_uniform)
    emd_launch_scale_canon(s->o.prec != EMD_FP64, g->B, (size_t)n3, n_occ, s->occ_winv, s->st);
  emd_launch_fill_random(s->o.prec, g->B, (size_t)n3, n_occ, m, 0x5eedu, s->st);
  gs_pack(g->og, g->B, g->A, m, s->st);
  emd_launch_density(s->o, s->psi, occ, g->rho_in, s->st);
  const double n_now = occupation_sum(s);
  if (n_now != n_e) {
    EmdComb sc{};
    sc.p[0] = g->rho_in;
    sc.w[0] = n_e / n_now;
    sc.m = 1;
    emd_launch_comb(n3, sc, g->rho_out, s->st);
    std::swap(g->rho_in, g->rho_out);
  }
  gs_potential(s, g->rho_in);
  std::vector<double> eps;
  r = gs_rayleigh_ritz(s, eps);
  if (r) return r;
  double B[K][K] = {};
  std::vector<int> act;
  std::vector<double> f(n_occ, occ), wh(n_occ, 1.0);
  double mu_f = 0.0;
  double res = 0.0;
  int it = 0;
  bool converged = false;
  const double lam_kin = 1.5 * kinetic_lambda_max(s->cfg.fd_order) / (s->g.h * s->g.h);
  for (it = 1; it <= max_scf; ++it) {
    double vmax = 0.0;
    r = reduce_max_veff(s, &vmax);
    if (r) return r;
    const double b = lam_kin + std::max(0.0, vmax) + std::max(0.0, s->sp.h_kb);
    const double a0 = eps.front(), a = eps.back();
    if (!(a < b) || !(a0 < a)) return fail(EMD_ECUDA, "Ritz values outside the filter bounds");
    r = gs_filter(s, degree, a, b, a0);
    if (r) return r;
    r = gs_rayleigh_ritz(s, eps);
    if (r) return r;
    if (smear) {
      mu_f = emd_host::fermi_dirac(eps, n_occ, n_e, occ, kT, f);
      for (int i = 0; i < n_occ; ++i) wh[i] = std::sqrt(f[i] / occ);
      CK(cudaMemcpyAsync(g->wd, wh.data(), (size_t)n_occ * 8, cudaMemcpyHostToDevice, s->st));
    }
    gs_density(s, g->rho_out, smear ? g->wd : nullptr);
    emd_launch_absdiff_partials(n3, g->rho_out, g->rho_in, s->partials, nb, s->st);
    emd_launch_sum(s->partials, nb, s->scal + 8, s->st);
    double l1 = 0.0;
    CK(cudaMemcpyAsync(&l1, s->scal + 8, 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    res = h3 * l1 / n_e;
    if (!std::isfinite(res)) return fail(EMD_ECUDA, "ground state: non-finite density");
    if (res < tol) {
      converged = true;
      break;
    }
    // store (rho_in, F) in the oldest slot
    const int k = (it - 1) % K;
    CK(cudaMemcpyAsync(g->hr[k], g->rho_in, (size_t)n3 * 8, cudaMemcpyDeviceToDevice, s->st));
    EmdComb fd{};
    fd.p[0] = g->rho_out;
    fd.w[0] = 1.0;
    fd.p[1] = g->rho_in;
    fd.w[1] = -1.0;
    fd.m = 2;
    emd_launch_comb(n3, fd, g->hf[k], s->st);
    act.erase(std::remove(act.begin(), act.end(), k), act.end());
    act.push_back(k);
    for (size_t j = 0; j < act.size(); ++j) {
      emd_launch_dot_partials(n3, g->hf[k], g->hf[act[j]], nullptr, nullptr, s->partials, nb,
                              s->st);
      emd_launch_sum(s->partials, nb, s->scal + 8 + j, s->st);
    }
    double dots[K];
    CK(cudaMemcpyAsync(dots, s->scal + 8, act.size() * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (size_t j = 0; j < act.size(); ++j) B[k][act[j]] = B[act[j]][k] = dots[j];
    std::vector<double> c;
    emd_host::anderson_coefficients(K, &B[0][0], act, k, c);
    // rho_in <- sum_j c_j rho_in_j + mix K[sum_j c_j F_j] (K: Kerker's
    // factor, or 1), the combined residual formed in rho_out
    EmdComb cf{};
    for (size_t j = 0; j < act.size(); ++j) {
      cf.p[cf.m] = g->hf[act[j]];
      cf.w[cf.m++] = c[j];
    }
    emd_launch_comb(n3, cf, g->rho_out, s->st);
    if (kerker_q0 > 0.0)
      emd_launch_kerker(s->g, kerker_q0, g->rho_out, g->rho_out, s->fft_a, s->fft_b, s->st);
    EmdComb cb{};
    for (size_t j = 0; j < act.size(); ++j) {
      cb.p[cb.m] = g->hr[act[j]];
      cb.w[cb.m++] = c[j];
    }
    cb.p[cb.m] = g->rho_out;
    cb.w[cb.m++] = mix;
    emd_launch_comb(n3, cb, g->rho_in, s->st);
    gs_potential(s, g->rho_in);
  }
  // the occupied Ritz vectors become the system's orbitals, with their
  // occupations (the last iteration's)
  gs_pack(s->o, g->B, s->psi, n_occ, s->st);
  r = launch_check("emd_ground_state");
  if (r) return r;
  r = set_occupation_state(s, f.data());
  if (r) return r;
  if (!s->f_uniform) emd_launch_scale_orbitals(s->o, s->psi, n_occ, s->occ_w, s->st);
  r = launch_check("emd_ground_state");
  if (r) return r;
  CK(cudaStreamSynchronize(s->st));
  if (eigenvalues) std::copy(eps.begin(), eps.begin() + n_occ, eigenvalues);
  if (occupations) std::copy(s->f.begin(), s->f.end(), occupations);
  if (info) {
    info->iterations = converged ? it : max_scf;
    info->residual = res;
    double sum = 0.0;
    for (int i = 0; i < n_occ; ++i) sum += f[i] * eps[i];
    info->band_energy = sum;
    info->gap = eps[n_occ] - eps[n_occ - 1];
    info->fermi_level = smear ? mu_f : 0.5 * (eps[n_occ - 1] + eps[n_occ]);
    info->entropy = smear ? emd_host::smearing_entropy(eps, n_occ, mu_f, occ, kT) : 0.0;
  }
  if (!converged)
    return fail(EMD_ENOTCONV, "ground state: residual %.3e after %d iterations (tol %.3e)",
                res, max_scf, tol);
  return EMD_OK;
}

int emd_ground_state(emd_system *s, int max_scf, double tol, int degree, double mix,
                     double *eigenvalues, emd_gs_info *info) {
  return emd_ground_state_smeared(s, max_scf, tol, degree, mix, 0.0, 0.0, 0.0, eigenvalues,
                                  nullptr, info);
}

int emd_get_dipole(emd_system *s, double *D) {
  g_err.clear();
  if (!s || !D) return fail(EMD_EINVAL, "NULL argument");
  if (!s->ions_set || !s->orbs_set) return fail(EMD_ESTATE, "set ions and orbitals first");
  int r = ensure_state(s);
  if (r) return r;
  const int nb = std::min(s->n_partials / 3, 512);
  emd_launch_dipole_partials(s->g.n, s->g.h, s->rho, s->partials, nb, s->st);
  for (int a = 0; a < 3; ++a) emd_launch_sum(s->partials + a * nb, nb, s->scal + 8 + a, s->st);
  double sums[3];
  const int na = s->n_atoms;
  std::vector<double> Rw(3 * std::max(1, na));
  CK(cudaMemcpyAsync(sums, s->scal + 8, sizeof sums, cudaMemcpyDeviceToHost, s->st));
  if (na)
    CK(cudaMemcpyAsync(Rw.data(), s->ts[s->cur].Rw, 3 * na * 8, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  r = launch_check("emd_get_dipole");
  if (r) return r;
  const double h3 = s->g.h * s->g.h * s->g.h;
  for (int a = 0; a < 3; ++a) {
    double d = -h3 * sums[a];
    for (int J = 0; J < na; ++J) d += s->sp.z * (Rw[3 * J + a] - 0.5 * s->g.L);
    D[a] = d;
  }
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
  emd_batch_destroy(s->self_batch);
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  if (s->cst) {
    cudaStreamSynchronize(s->cst);
    cudaStreamDestroy(s->cst);
  }
  for (cudaEvent_t e : s->cev)
    if (e) cudaEventDestroy(e);
  if (s->tst) {
    cudaStreamSynchronize(s->tst);
    cudaStreamDestroy(s->tst);
  }
  for (cudaEvent_t e : s->tev)
    if (e) cudaEventDestroy(e);
  for (void *p : s->allocs) cudaFree(p);
  if (s->adj) {
    for (void *p : s->adj->mem) cudaFree(p);
    delete s->adj;
  }
  gs_release(s->gsw);
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
