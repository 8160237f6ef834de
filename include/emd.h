/*
 * emd.h -- C ABI of libemd, a GB300 (sm_103a) implementation of the
 * per-step propagation of the modified Ehrenfest TDDFT molecular dynamics of
 * Alonso, Andrade et al., arXiv:0812.2801.
 *
 * The method (paper, Sec. 4.1 eq. new_L and eq. new_EoM; Sec. 5.1):
 *   i mu dphi_A/dt = H_KS phi_A          (complex Kohn-Sham orbitals)
 *   M_J d^2 R_J/dt^2 = -grad_J E_KS      (classical ions)
 * with E_KS of eq. E_KS on a periodic real-space grid with finite-difference
 * derivatives (Sec. 5).  One step = velocity-Verlet positions, AETRS
 * (eq. aetrs) with each half exponential exp(-i tau H), tau = dt/(2 mu)
 * (eq. transf), replaced by its degree-4 Taylor polynomial (Sec. 5.1), the new
 * density rho = f sum_A |phi_A|^2 (eq. density), Hartree + LDA potentials,
 * Hellmann-Feynman forces and velocity-Verlet velocities.
 *
 * Units: atomic units throughout (bohr, hartree, electron mass, hbar = 1).
 * Grid: N^3 points, spacing h, box [0, N h)^3, periodic.  Point (x, y, z)
 * has coordinates (x h, y h, z h) and canonical flat index (z N + y) N + x.
 *
 * Conventions for every entry point:
 *   - Return value: EMD_OK (0) or a positive EMD_E* status.  Nothing is
 *     thrown across the ABI.  emd_last_error() returns a message for the
 *     last failure on the calling thread (valid until the next call).
 *   - Host pointers are owned by the caller; the library copies what it
 *     needs before returning (inputs) or writes complete results (outputs).
 *   - Device memory is owned by the library (cudaMalloc at emd_init_system,
 *     released by emd_destroy).  Work is issued on the caller's CUDA stream
 *     (emd_config.cuda_stream; NULL = the legacy default stream).
 *   - Calls that return data to the host (emd_get_*) synchronise that stream;
 *     emd_propagate only enqueues work.  Device-side consistency problems
 *     found during propagation (a table overflow) are reported by the next
 *     emd_get_* call.
 *   - A system handle must not be used from two threads at once.
 */
#ifndef EMD_H
#define EMD_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define EMD_OK        0
#define EMD_EINVAL    1   /* bad argument (sizes, order, neutrality, NULL) */
#define EMD_ENOMEM    2   /* device or pinned host allocation failed      */
#define EMD_ECUDA     3   /* a CUDA runtime call failed                   */
#define EMD_EUNSTABLE 4   /* tau * lambda_max above the Taylor-4 bound, or
                             the density lost its normalisation           */
#define EMD_ESTATE    5   /* call out of order (e.g. propagate before
                             orbitals and ions are set)                   */
#define EMD_ETABLE    6   /* a per-point or per-tile atom list overflowed */
#define EMD_ENOTCONV  7   /* emd_ground_state: tolerance not reached        */
#define EMD_ETIMEOUT  8   /* a bounded wait inside a kernel gave up (its
                             tensor copies did not complete in ~1 s); the
                             results of the calls since the last check are
                             invalid; reported by the next emd_get_* call */

/* orbital storage precision */
#define EMD_FP64           0  /* complex128 orbitals, FP64 stencil          */
#define EMD_FP32_ORBITALS  1  /* complex64 orbitals and stencil; density,
                                 energies, forces and ions stay FP64        */

/* options for emd_set_option */
#define EMD_OPT_FROZEN_IONS  1  /* value != 0: ions fixed, no forces/VV      */
#define EMD_OPT_PROFILE      2  /* value != 0: time Horner-stage launches
                                   (one event pair each; emd_propagate then
                                   steps without graph replay)              */
#define EMD_OPT_CHECK_STABLE 3  /* value == 0: skip the stability refusal    */
#define EMD_OPT_STAGE_VARIANT 4 /* Horner-stage kernel.  complex64: 0 one
                                   thread per (orbital column, 2 rows) with
                                   compile-time ring slots (default); 1 the
                                   same tiling, earlier form; bo = 2 only:
                                   2 one thread per point, 3 one thread per
                                   (point column, 2 rows).  bo = 4: 0 with
                                   the per-plane diagonal, projector records
                                   and psi0 fetched by tensor copies (TMA),
                                   2 the same kernel with per-thread
                                   cp.async copies, 1 the earlier form.
                                   complex128 with
                                   bo = 2: 0 double-float arithmetic on the
                                   FP32 pipes (48-bit (hi, lo) float pairs,
                                   default), 1 plain FP64 arithmetic     */
#define EMD_OPT_PROJECTION   5  /* complex128 projections <p_J|u>: 1
                                   atom-major (each atom gathers its sphere,
                                   default), 0 point-major (each 8^3 tile
                                   read once, one warp-tree reduction per
                                   atom and warp).  complex64 orbitals always
                                   use per-tile entry lists grouped by atom
                                   (each tile read once, one warp per atom) */

#define EMD_OPT_ZCHUNK       6  /* planes per z-chunk of the z-marching
                                   stage kernels (each CTA marches through
                                   one chunk and restages 2 * order / 2 halo
                                   planes): 0 automatic (whole columns unless
                                   that leaves SMs idle), else an integer
                                   1 .. 1024 (clamped to the grid)          */

/* kernels that can be timed with EMD_OPT_PROFILE */
#define EMD_KERNEL_HORNER    0  /* one Taylor/Horner stage u' = psi0 + a H u */
#define EMD_KERNEL_ALL       1  /* every kernel the library launched (count
                                   only, process-wide; ms_total = 0)      */

/*
 * Synthetic pseudo-atom (the paper uses Troullier-Martins pseudopotentials,
 * Sec. 5; this stands in with the same structure: a local part plus a
 * separable nonlocal part).
 *   z       valence charge Z
 *   mass    ionic mass M (electron masses)
 *   a_loc   Gaussian ion charge g(d) = Z pi^-3/2 a^-3 exp(-d^2/a^2), so that
 *           the local potential is -Z erf(d/a)/d (eq. ionicpotential)
 *   r_loc   support radius of g on the grid (points with d < r_loc)
 *   r_c     projector p(d) = pi^-3/4 r_c^-3/2 exp(-d^2/(2 r_c^2))
 *   h_kb    strength of the term h_kb |p><p|
 *   r_proj  support radius of p on the grid (d < r_proj)
 *   lmax    angular momenta of the separable term, 0, 1 or 2 (the paper's
 *           norm-conserving pseudopotentials carry one term per l): each
 *           l <= lmax adds 2l + 1 projectors p_lm(d) = N_l S_lm(d)
 *           exp(-d^2/(2 r_c^2)), S_lm the real solid harmonics (x, y, z;
 *           sqrt3 xy, sqrt3 yz, sqrt3 zx, sqrt3/2 (x^2 - y^2),
 *           (3z^2 - d^2)/2), N_l^-2 = 2 pi Gamma(l + 3/2) r_c^(2l+3) /
 *           (2l + 1) (unit norm); lmax > 0 needs EMD_FP64 with block
 *           width 2 and is refused by the adjoint and the ground state
 *   h_l     strengths of the l = 1 and l = 2 terms (h_kb is l = 0)
 * Both radii must not exceed the box length N h.  Projector P of atom J is
 * row J (lmax + 1)^2 + k of the projections, k in the order above (s, then
 * x y z, then the five l = 2 functions).
 */
typedef struct {
  double z, mass, a_loc, r_loc, r_c, h_kb, r_proj;
  int lmax;
  double h_l[2];
} emd_species;

typedef struct {
  int n;                 /* grid points per axis, 2*fd_order <= n <= 1024,
                            and n may have no prime factor above 13     */
  double h;              /* grid spacing (bohr), > 0                     */
  int fd_order;          /* finite-difference order: 2, 4, 6 or 8        */
  int n_orb;             /* number of orbitals, >= 1                     */
  double occ;            /* occupation per orbital (2 = closed shell)    */
  int precision;         /* EMD_FP64 or EMD_FP32_ORBITALS                */
  int n_atoms;           /* number of atoms, >= 0                        */
  emd_species species;   /* one species for all atoms                    */
  void *cuda_stream;     /* cudaStream_t to issue work on, or NULL        */
  int block_orbitals;    /* orbitals interleaved per grid point: 1, 2, 4;
                            0 = 4 for complex64, 2 for complex128      */
} emd_config;

/* Energy components (hartree), eq. E_KS and eq. E_new:
 *   kin_e   sum_A f <phi_A| -1/2 nabla^2_FD |phi_A>
 *   nl      sum_{J,A} f h_kb |<p_J|phi_A>|^2
 *   es      electrostatics: 1/2 h^3 sum n_tot v_es - sum_J Z^2/(sqrt(2 pi) a)
 *           + sr, with n_tot = rho - sum_J g_J and v_es its periodic
 *           potential (the G = 0 component is dropped)
 *   xc      h^3 sum rho eps_xc (Perdew-Zunger LDA)
 *   sr      1/2 sum' Z_J Z_K erfc(d/(sqrt2 a))/d over images, d < 12 bohr
 *           (already included in es)
 *   kin_ion sum_J M |V_J|^2 / 2
 *   ks      kin_e + nl + es + xc
 *   total   ks + kin_ion (the conserved energy of eq. E_new)
 *   n_elec  h^3 sum rho (health check: equals n_orb * occ)            */
typedef struct {
  double kin_e, nl, es, xc, sr, kin_ion, ks, total, n_elec;
} emd_energy;

typedef struct emd_system emd_system;

/* Create a system: validates cfg, allocates all device buffers.  *out is set
 * on success.  Errors: EMD_EINVAL, EMD_ENOMEM, EMD_ECUDA. */
int emd_init_system(const emd_config *cfg, emd_system **out);

/* Set ions: R[n_atoms][3], V[n_atoms][3] (host, float64; x, y, z).
 * n_atoms must equal cfg.n_atoms.  Positions may lie outside the box; they
 * are folded with X - L floor(X/L) wherever a grid support is built.
 * Recomputes the ionic potential.  If orbitals are set, rho, v_Hxc and F(0)
 * are recomputed and the v_Hxc history restarted by the next call that
 * reads them (propagate, get_forces, get_energy, get_state, get_potentials,
 * get_projections, apply_hamiltonian), so set_ions followed by set_orbitals
 * pays for one recomputation; errors of that recomputation are returned by
 * that call. */
int emd_set_ions(emd_system *s, int n_atoms, const double *R, const double *V);

/* Set orbitals: psi is complex128 interleaved (re, im), canonical layout
 * [n_orb][N][N][N] (host).  Orbitals should be orthonormal under
 * <a|b> = h^3 sum conj(a) b; they are not modified.  If ions are set, rho,
 * v_Hxc and F(0) are recomputed and the v_Hxc history restarted (Sec. 2,
 * eq. Ehr_ic: initial condition) by the next call that reads them, as for
 * emd_set_ions.  Returns after the host array has been read. */
int emd_set_orbitals(emd_system *s, const double *psi);

/* The same with complex64 host arrays (float32 interleaved (re, im), same
 * canonical layout), for callers that keep orbitals in single precision:
 * half the bytes over the host link, copied block by block on a second
 * stream so that the link and the repacking overlap (page-locked psi lets
 * the copies run asynchronously).  For EMD_FP32_ORBITALS systems the
 * stored orbitals are identical to those set from the complex128 values
 * rounded to complex64.  No counterpart in the paper (host I/O). */
int emd_set_orbitals_c64(emd_system *s, const float *psi);

/* Orbitals of the current state as complex64 (float32 interleaved (re, im),
 * canonical [n_orb][N][N][N], host).  EMD_FP64 systems round to float32. */
int emd_get_orbitals_c64(emd_system *s, float *psi);

/* Occupations f[n_orb] (host): the density is rho = sum_A f_A |phi_A|^2
 * (eq. density with a weight per orbital; f_A = occ for every orbital
 * after emd_init_system and after emd_ground_state, the closed-shell
 * case).  Each f_A must lie in (0, occ]; values below 1e-30 occ are raised
 * to it.  The weights enter the energies and forces with the density (each
 * term is quadratic in an orbital with its weight f_A) and stay fixed while
 * the orbitals evolve (the propagation is linear in each orbital).
 * Storage: the device holds u_A = sqrt(f_A / occ) phi_A, so the kernels
 * work unchanged with the single weight occ; emd_set_orbitals*,
 * emd_get_state, emd_get_orbitals_c64 and emd_get_projections take and
 * return phi_A (the weights applied on the way in and removed on the way
 * out).  Set before or after the orbitals; if orbitals are set, rho,
 * v_Hxc and F are recomputed by the next call that reads them.  A
 * smeared ground state (emd_ground_state_smeared) sets them.  Not in the
 * paper, whose systems are closed-shell.  Errors: EMD_EINVAL. */
int emd_set_occupations(emd_system *s, const double *f);
int emd_get_occupations(emd_system *s, double *f);

/* Advance n_steps MD steps of length dt with the electronic mass-like
 * parameter mu (mu = 1: plain Ehrenfest).  field: NULL, or n_steps
 * amplitudes e_n (host) of a uniform field along z in the length gauge,
 * v_ext = e_n (z - L/2), held during step n, force Z e_n on each ion.
 * Refuses with EMD_EUNSTABLE if tau*lambda_max > 2 sqrt(2), the Taylor-4
 * stability bound on the imaginary axis (lambda_max estimated as the
 * largest FD kinetic eigenvalue + max v_eff + h_kb).  Enqueues only.
 * With field == NULL, moving ions and EMD_OPT_PROFILE off, runs of 6 or more
 * steps replay a CUDA graph of 6 steps captured on first use (captured
 * again when dt, mu, the stage variant, the projection form, the position
 * set or the v_Hxc history slots no longer match it); the results are
 * bitwise those of step-by-step propagation. */
int emd_propagate(emd_system *s, int n_steps, double dt, double mu,
                  const double *field);

/* F[n_atoms][3] = -dE_KS/dR at the current state (eq. new_EoM_b). */
int emd_get_forces(emd_system *s, double *F);

/* Energy components at the current state (see emd_energy). */
int emd_get_energy(emd_system *s, emd_energy *out);

/* Current state; any pointer may be NULL.  R, V: [n_atoms][3];
 * psi: complex128 canonical [n_orb][N][N][N]; rho: [N][N][N]. */
int emd_get_state(emd_system *s, double *R, double *V, double *psi, double *rho);

/* Grid potentials of the current state, each [N][N][N] or NULL:
 * v_loc (ionic, eq. ionicpotential), v_h (Hartree), v_xc (LDA),
 * g_ion (sum of the Gaussian ion charges). */
int emd_get_potentials(emd_system *s, double *v_loc, double *v_h, double *v_xc,
                       double *g_ion);

/* Projections c[n_atoms (lmax + 1)^2][n_orb] complex128 (re, im) of the
 * current orbitals: c_PA = h^3 sum_r p_P(r) phi_A(r) (the separable term of
 * H), row P = J (lmax + 1)^2 + k for channel k of atom J. */
int emd_get_projections(emd_system *s, double *c);

/* hpsi = H psi for n_vec orbitals (complex128 canonical [n_vec][N][N][N],
 * host), with H = -1/2 nabla^2_FD + v_eff + sum_J h_kb |p_J><p_J| of the
 * current state: v_eff = v_loc + v_H + v_xc, projectors at the current R
 * (eq. new_EoM_a).  1 <= n_vec <= n_orb.  Uses the propagation kernels in
 * the configured precision (FP32 mode rounds psi to complex64). */
int emd_apply_hamiltonian(emd_system *s, int n_vec, const double *psi,
                          double *hpsi);

/* Set an EMD_OPT_* option. */
int emd_set_option(emd_system *s, int option, double value);

/* Accumulated device time (ms) and launch count of a timed kernel since
 * EMD_OPT_PROFILE was enabled or the previous call (EMD_KERNEL_HORNER), or
 * the number of kernels the library launched since the previous call
 * (EMD_KERNEL_ALL).  Both counters reset on reading.  Synchronises. */
int emd_kernel_stats(emd_system *s, int kernel, double *ms_total,
                     long long *launches);

/* Adjoint (backward-in-time) propagation.  The paper gives the forward
 * dynamics only (Sec. 4.1, eq. new_EoM; Sec. 5.1, eq. aetrs); this is the
 * exact discrete adjoint of the implemented step, for gradient-based uses of
 * the trajectory (field optimisation, sensitivities).  FP64 orbitals only.
 * The electrons evolve self-consistently (density -> Hartree + LDA ->
 * extrapolated H(t+dt)) under the field e_n.  With EMD_OPT_FROZEN_IONS set
 * the ions stay at their positions; otherwise they move by velocity Verlet
 * under the forces of eq. new_EoM_b plus Z e_n along z, and the reverse
 * sweep also runs through the forces (their orbital, potential and position
 * dependence) and the Verlet updates.  The gradient is taken with respect to
 * the initial ion positions R(0) (velocities held) and every e_n.
 *   observable EMD_OBS_DIPOLE_Z: L = -h^3 sum rho (z - L/2) + sum_J Z (Z_J - L/2)
 *   observable EMD_OBS_ENERGY:   L = E_KS of the final state (eq. E_KS), plus
 *                                sum_J M V_J^2 / 2 when the ions move
 * Runs n_steps forward from the current state (storing orbitals, the v_Hxc
 * history and the ions' R, V, F every ckpt_every steps), then backward
 * segment by segment, recomputing each segment's steps from its checkpoint.
 * On return the system is at the final state; *L_out = L, dL_dR[n_atoms][3],
 * dL_dfield[n_steps] (may be NULL if field is NULL).  Device workspace
 * (about (n_steps/ckpt_every + ckpt_every + 13) orbital sets) is allocated
 * on first use and kept until emd_destroy.  Synchronises (once per reverse
 * step with moving ions).
 * Errors: EMD_EINVAL, EMD_ESTATE, EMD_ENOMEM, EMD_ECUDA, EMD_ETABLE. */
#define EMD_OBS_ENERGY   0
#define EMD_OBS_DIPOLE_Z 1
int emd_propagate_adjoint(emd_system *s, int n_steps, double dt, double mu,
                          const double *field, int ckpt_every, int observable,
                          double *L_out, double *dL_dR, double *dL_dfield);

/* Batched replicas: independent systems (any sizes, precisions, orders)
 * advanced together.  Each system keeps its own state; a batch only
 * schedules them.  After an eager warm-up (until every system's v_Hxc
 * history holds three entries) the batch captures 6 MD steps of all systems
 * into one CUDA graph, one parallel branch per system, and replays it for
 * every further chunk of 6 steps; the remainder runs eagerly.  The graph is
 * captured again if dt, mu or a system's position-set parity changes.  Work
 * runs on internal streams ordered after, and followed by, each system's own
 * stream.  No external field.  The paper has no batched form; replicas are
 * how independent trajectories (e.g. thermal sampling, Sec. 6.3's 300 K
 * starts) share one GPU.
 *   emd_batch_create: systems[n] (caller keeps ownership; they must outlive
 *     the batch and not be used concurrently with it).  Errors: EMD_EINVAL
 *     (NULL or repeated system), EMD_ECUDA.
 *   emd_batch_propagate: n_steps MD steps of every system (same dt, mu).
 *     Errors as emd_propagate; EMD_ECUDA if graph capture fails (the systems
 *     must then be re-initialised with emd_set_orbitals).  Enqueues only.
 *   emd_batch_destroy: synchronises and releases the batch (not the systems). */
typedef struct emd_batch emd_batch;
int emd_batch_create(int n, emd_system *const *systems, emd_batch **out);
int emd_batch_propagate(emd_batch *b, int n_steps, double dt, double mu);
void emd_batch_destroy(emd_batch *b);

/* Periodic Poisson solve that allocates nothing.  The paper has no
 * counterpart: this is a convenience for callers that cannot call cudaMalloc
 * -- code that runs while a CUDA graph is being captured, applications whose
 * device memory belongs to another allocator or a fixed budget, and
 * latency-critical loops where an allocation would synchronise the device.
 *
 * v = periodic solution of nabla^2 v = -4 pi charge on an n^3 grid of
 * spacing h with the G = 0 component removed (the Hartree step of
 * emd_propagate).  charge and v are DEVICE pointers to n^3 doubles in the
 * canonical layout (x fastest), owned by the caller; they may not alias.
 * Work is issued on cuda_stream (NULL = legacy default stream); the call
 * returns without synchronising.
 *
 * Limits and sharing: the FFT work arrays live in one file-scope device
 * array sized for n <= 64 (8 MB, held on every GPU that loads the library
 * until the process exits); n > 64 or a prime factor of n above 13 returns
 * EMD_EINVAL with a message.  The array keeps the last call's contents and
 * every call uses it, so calls that overlap on the GPU (different streams,
 * or different host threads on one device) race; serialise them.  The first
 * call on each device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process, so the entry
 * point must not be called on a device after cudaDeviceReset on it.
 * Errors: EMD_EINVAL, EMD_ECUDA. */
int emd_poisson_static(int n, double h, const double *charge, double *v,
                       void *cuda_stream);

/* Dipole of the current state, D[3] (host): D_a = -h^3 sum_r rho(r)
 * (r_a - L/2) + sum_J Z (R_Ja - L/2), grid points r_a = i h in [0, L) and
 * positions folded into [0, L): the sawtooth coordinate of the field's
 * length gauge along each axis.  Meaningful for a system well inside the
 * box (a molecule away from the faces).  Used for the infrared spectrum of
 * a trajectory (the time derivative of D).  Errors: EMD_EINVAL,
 * EMD_ESTATE. */
int emd_get_dipole(emd_system *s, double *D);

/* Kohn-Sham ground state at the current ions (Sec. 4.1, eqs. EoM_BO_a and
 * EoM_BO_b): orthonormal orbitals that satisfy H_KS[rho] phi_A =
 * sum_B Lambda_AB phi_B with rho built from them and fill the n_orb lowest
 * eigenstates of that H, i.e. phi_gs(R) of eq. EoM_BO_2, the start on the
 * BO surface of the paper's runs.  The paper gives no algorithm; here each
 * self-consistency iteration
 *   1. filters the orbitals with the Chebyshev polynomial of degree
 *      `degree` (1..64) of H[rho_in] on [largest Ritz value, spectral upper
 *      bound] (the bound of emd_propagate's stability check), scaled to 1
 *      at the lowest Ritz value;
 *   2. replaces them by the Rayleigh-Ritz vectors of the filtered set
 *      (generalized eigenproblem of h^3 X^H H X against h^3 X^H X);
 *   3. forms rho_out and mixes rho_in with it (Anderson over the last six
 *      iterations, step `mix` in (0, 1]);
 * and stops when h^3 sum |rho_out - rho_in| < tol * n_electrons or after
 * max_scf iterations.  The current orbitals are the starting guess (an
 * orthonormal set of atom-centred functions will do).  On return the
 * orbitals are the last Ritz vectors in ascending order, eigenvalues (if not
 * NULL, host, n_orb doubles) their Ritz values, info (if not NULL) the
 * iteration count, final residual, occ * sum of the Ritz values, the gap
 * to the first unoccupied Ritz value (the subspace carries max(4,
 * n_orb/10) buffer states above the occupied ones), the middle of that gap
 * and zero entropy; the occupations are reset to occ; rho,
 * v_Hxc and F are recomputed from the new orbitals by the next call that
 * reads them (as after emd_set_orbitals).  The subspace products X^H X,
 * X^H H X and X V are the library's own kernels (FP64 sums, in a fixed
 * order); the m x m generalized eigenproblem is solved on the host
 * (Cholesky of the overlap, Householder reduction to a real tridiagonal,
 * implicit QR with Wilkinson shifts), m = n_orb + the
 * buffer states; no vendor library is called.
 * Errors: EMD_EINVAL, EMD_ESTATE (ions or orbitals not set),
 * EMD_ENOTCONV (tolerance not reached; the orbitals are the last iterate),
 * EMD_ECUDA (including a subspace that lost rank). */
typedef struct {
  int iterations;
  double residual;       /* h^3 sum |rho_out - rho_in| / n_electrons */
  double band_energy;    /* sum_A f_A eps_A over the n_orb states      */
  double gap;            /* first buffer-state Ritz value minus the
                            n_orb-th one; integer occupations need
                            it > 0                                    */
  double fermi_level;    /* mu_F of the Fermi-Dirac occupations; with
                            kT = 0 the middle of that gap             */
  double entropy;        /* S = -sum_A occ [g ln g + (1-g) ln(1-g)],
                            g = f_A / occ (0 with kT = 0); the Mermin
                            free energy is E_KS - kT S               */
} emd_gs_info;
int emd_ground_state(emd_system *s, int max_scf, double tol, int degree,
                     double mix, double *eigenvalues, emd_gs_info *info);

/* The same with fractional occupations, for cells with a small or no gap
 * (the paper's systems are gapped and it uses none; a reading).  With
 * kT > 0 the n_orb states of the system carry Fermi-Dirac occupations
 *   f_A = occ / (1 + exp((eps_A - mu_F) / kT)),  sum_A f_A = n_electrons,
 * mu_F found by bisection each iteration from the n_orb lowest Ritz values
 * (0 < n_electrons < occ n_orb: give the system more orbitals than
 * n_electrons / occ), rho_out = sum_A f_A |phi_A|^2, and the fixed point is
 * the stationary point of the Mermin free energy E_KS - kT S.  kT = 0 is
 * emd_ground_state (n_electrons ignored).  kerker_q0 > 0 preconditions
 * the mixing step: the Anderson-combined residual R(G) is multiplied by
 * |G|^2 / (|G|^2 + q0^2) (R(0) unchanged; an FFT pass like the Hartree
 * solve), which damps the long-wavelength charge sloshing of metallic
 * cells; 0 mixes unpreconditioned.  Neither kT's search nor the
 * preconditioner moves the fixed point.  On return the occupations are
 * the system's (emd_set_occupations), occupations (if not NULL, host,
 * n_orb doubles) a copy of them, and the starting density is that of the
 * current orbitals and occupations scaled to n_electrons.  Errors as for
 * emd_ground_state. */
int emd_ground_state_smeared(emd_system *s, int max_scf, double tol, int degree,
                             double mix, double kT, double n_electrons,
                             double kerker_q0, double *eigenvalues,
                             double *occupations, emd_gs_info *info);

/* Release all device memory and the handle.  NULL is accepted. */
void emd_destroy(emd_system *s);

/* Message of the last failure on this thread ("" if none). */
const char *emd_last_error(void);

/* Library version string. */
const char *emd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EMD_H */
