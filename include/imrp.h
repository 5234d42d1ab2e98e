/*
 * imrp.h -- C ABI of the GB300-native spectral kinetic simulation of the ideal
 * Multipole Resonance Probe (Gong, Friedrichs, Oberrath, Brinkmann,
 * "Kinetic Simulation of the Ideal Multipole Resonance Probe", arXiv 2111.13072).
 *
 * One context owns one plasma instance on one GPU: N electron super-particles
 * (charge q = -1, mass m = 1 in the units below) around a metal sphere of radius
 * R_E covered by a dielectric shell (permittivity eps_D) out to R, with an
 * immobile ion background filling R <= r <= R_out: uniform, or the radial
 * profile of the floating sheath equilibrium (App. D, imrp_set_ion_profile).
 *
 * Units (Sec. 4 of the paper): lengths in R (= R_D, outer radius of the
 * dielectric), time in 1/omega_pe, velocities in R*omega_pe, charge in e, mass
 * in m_e. Positions and velocities cross this ABI in these units as FP64.
 *
 * Conventions for every entry point:
 *   - returns IMRP_OK (0) on success or a negative IMRP_E_* code; the message
 *     of the last failure on a context is available from imrp_last_error();
 *   - no exception crosses the ABI; no entry point aborts the process;
 *   - host buffers are owned by the caller and only read or written during the
 *     call; all device memory is owned by the context;
 *   - calls on one context must not overlap (one host thread at a time);
 *   - calls return after the GPU work they issued has finished, except
 *     imrp_step_async().
 */
#ifndef IMRP_H
#define IMRP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IMRP_OK 0
#define IMRP_E_INVAL (-1)   /* invalid argument or parameter                     */
#define IMRP_E_NOMEM (-2)   /* device or host allocation failed                  */
#define IMRP_E_CUDA (-3)    /* a CUDA call failed (message has the CUDA error)   */
#define IMRP_E_TIMEOUT (-4) /* reserved: no entry point returns it (no kernel of the
                               path waits on another, so no wait can give up) */
#define IMRP_E_NAN (-5)     /* a non-finite value appeared in the state          */
#define IMRP_E_STATE (-6)   /* call out of order (e.g. step before load)         */

typedef struct imrp_ctx imrp_ctx;

/* Physical problem and numerical choices. Fill with imrp_default_params()
 * and override fields. */
typedef struct imrp_params {
  double R_E_m;      /* electrode radius R_E [m] (Sec. 2: R_E = R - Rd)            */
  double R_D_m;      /* outer radius of the dielectric shell, the length unit R [m] */
  double eps_D;      /* relative permittivity eps_r of the shell (App. A)         */
  double R_out_m;    /* radius of the outer particle wall [m] (Sec. 4)            */
  double n_e_m3;     /* electron density n_inf [m^-3] (Sec. 4 units)              */
  double T_e_eV;     /* electron temperature [eV]: the thermal speed lambda_D omega_pe of the
                        plasma that wall_rule 2 injects (the field does not use it) */
  int64_t N;         /* capacity: maximum number of super-particles               */
  int32_t l_max;     /* truncation degree of the projection P^ (Sec. 2/3); one of 1,2,4,8,12,16,24 */
  int32_t m0_only;   /* 0: all (l, m); 1: only the m = 0 terms of each degree -- with
                        l_max = 1 the truncated kernel of Sec. 3 (cos t cos t' dipole) */
  double dt;         /* time step [1/omega_pe]                                    */
  int32_t drive_kind; /* 0 Gaussian pulse, 1 impulse at the first step (Sec. 4), 2 off */
  int32_t wall_rule;  /* 0 diffuse reflection (Sec. 4), 1 specular reflection,
                         2 absorb and re-inject: an electron that crosses r = R is
                         absorbed and its charge joins the probe's surface charge
                         Q_S (homogeneous on the surface, Sec. 2), which the field of
                         the following steps feels (Sec. 3); one that crosses R_out
                         leaves; either is replaced, under its id, by an electron
                         entering through the outer wall from the bulk plasma (a
                         flux-weighted Maxwellian of thermal speed lambda_D omega_pe,
                         drawn from Philox keyed by (step, id, seed))            */
  double V_volts;    /* drive amplitude u_asy [V]: peak of the pulse or the impulse */
  double width_wpe;  /* Gaussian pulse standard deviation [1/omega_pe]             */
  double t0_wpe;     /* Gaussian pulse centre [1/omega_pe]; <= 0 selects 4*width   */
  int32_t self_image; /* 0: a particle does not feel its own image (the pair sum of Sec. 2 has i != k); 1: it does */
  int32_t precision;  /* 0 FP64 throughout; 1 mixed: FP32 state, harmonics and push, FP64 carries */
  uint64_t seed;     /* key of the counter-based wall random numbers              */
  double q_s;        /* surface charge Q_S in super-particle charges (Sec. 3), usually 0 */
  double nu_coll;    /* electron-neutral collision rate nu [omega_pe] (Sec. 5 names collisions as
                        the next addition; the Drude model of Sec. 4 damps with nu): in each step
                        an electron scatters elastically and isotropically (same speed, direction
                        uniform on the sphere) with probability 1 - exp(-nu dt), decided by Philox
                        keyed by (step, id, seed). 0: collisionless, as in the paper's runs */
} imrp_params;

/* Derived dimensionless quantities of a context (read-only). */
typedef struct imrp_info {
  double d;          /* relative dielectric thickness, R_E = (1 - d) R             */
  double r_out;      /* outer wall radius in units of R                            */
  double n_tilde;    /* super-particles per unit cube at density n_inf (Sec. 4)    */
  double n_ion;      /* ion super-particles of the uniform background (= N loaded) */
  double v_hat;      /* drive amplitude in units of e n_inf R^2 / eps0            */
  double lambda_D;   /* Debye length in units of R                                 */
  double omega_pe;   /* electron plasma frequency [1/s]                            */
  int64_t n;         /* particles currently loaded                                 */
  int64_t step;      /* steps taken since the last load (a restore sets it)        */
  int32_t l_max;
  int32_t precision;
} imrp_info;

/* Fills p with the small FP64 workload: R_E = 4 mm, R_D = 5 mm, eps_D = 4,
 * n_e = 1e15 m^-3, T_e = 2 eV, R_out = R_D + 20 lambda_D, l_max = 8, dt = 0.05,
 * Gaussian pulse 1 V, width 2, diffuse walls, N = 20000, FP64. */
void imrp_default_params(imrp_params* p);

/* Validates p, derives the dimensionless problem (Sec. 4), allocates all
 * device memory for N particles on the current CUDA device and creates the
 * context's stream. *out receives the context; on failure *out is NULL.
 * Errors: IMRP_E_INVAL (bad geometry, l_max not instantiated, N < 1 ...),
 * IMRP_E_NOMEM, IMRP_E_CUDA. */
int imrp_create(const imrp_params* p, imrp_ctx** out);

/* Device memory in bytes that imrp_create(p) allocates, plus the Q_diff history
 * of n_steps steps: what an admission controller needs before creating a
 * context. Errors: IMRP_E_INVAL. */
int imrp_footprint(const imrp_params* p, int64_t n_steps, size_t* bytes);

/* Frees all device memory and the stream. NULL is accepted. */
int imrp_destroy(imrp_ctx* ctx);

/* Message of the last failure on ctx ("" if none). Valid until the next call. */
const char* imrp_last_error(const imrp_ctx* ctx);

/* Makes the context issue its work on a caller-owned cudaStream_t (passed as
 * void*). NULL restores the context's own stream. */
int imrp_set_stream(imrp_ctx* ctx, void* cuda_stream);

/* Loads n <= N particles from host FP64 arrays x[n][3] (positions, units of R,
 * each with 1 < |x| < r_out) and v[n][3] (velocities synchronous with x, units
 * of R omega_pe). Particle ids are 0..n-1 in input order. Resets the step
 * counter and the Q_diff history; the uniform ion background is set to n
 * ions (with a profile from imrp_set_ion_profile, n~ = n / its electron
 * charge instead). Errors: IMRP_E_INVAL (n out of range, a position outside
 * the shell, a non-finite value). */
int imrp_load_particles(imrp_ctx* ctx, const double* x, const double* v, int64_t n);

/* Streamed form of imrp_load_particles, for callers that feed a new particle
 * set every few steps and want the host-to-device copy to overlap the steps
 * still running. The copy of x and v runs on the context's own copy stream
 * into one of two staging buffers (allocated on the first call, 2 x 48 bytes
 * per particle of capacity); the conversion into the particle state is
 * queued on the context's stream after the work already queued there. The
 * call returns without waiting. x and v must stay valid and unchanged until
 * the next synchronising call (imrp_sync, imrp_step, imrp_get_*); pinned host
 * memory is needed for the copy to run asynchronously. A position outside
 * the shell or a non-finite value is reported by the next synchronising call
 * (IMRP_E_INVAL). Errors: IMRP_E_INVAL (n out of range), IMRP_E_CUDA. */
int imrp_load_particles_async(imrp_ctx* ctx, const double* x, const double* v, int64_t n);

/* Advances n_steps leapfrog steps (Sec. 2 canonical equations; kick-drift
 * with merged kicks, the first kick after a load is dt/2). Each step sorts the
 * particles by radius, evaluates the field of the modified, truncated Green's
 * function G~ (Sec. 3) plus ions, Q_S and the drive u_asy(t_n) Psi_anti
 * (Sec. 3-4), pushes, applies the wall rule (Sec. 4) and records
 * Q_diff(t_n) = -(1/n~) sum_i q_i Psi_anti,L(x_i) (Sec. 4) at the positions
 * x_n used by the step. qdiff_out and uasy_out (host, n_steps doubles each,
 * either may be NULL) receive Q_diff(t_n) and u_asy(t_n).
 * Errors: IMRP_E_STATE (nothing loaded), IMRP_E_NAN, IMRP_E_CUDA. */
int imrp_step(imrp_ctx* ctx, int64_t n_steps, double* qdiff_out, double* uasy_out);

/* As imrp_step without host outputs and without waiting for the GPU: the work
 * is queued on the context's stream (replayed CUDA graphs). Device-side errors
 * surface at the next synchronising call. */
int imrp_step_async(imrp_ctx* ctx, int64_t n_steps);

/* Waits for queued work and checks the device error flags. */
int imrp_sync(imrp_ctx* ctx);

/* Without waiting: *ready = 1 when all work queued on the context's stream has
 * finished, 0 while some is still running (for a host loop that serves many
 * contexts). It does not check the device error flags; imrp_sync does.
 * Errors: IMRP_E_INVAL, IMRP_E_CUDA (an earlier asynchronous failure). */
int imrp_ready(imrp_ctx* ctx, int* ready);

/* Copies Q_diff(t_n) and u_asy(t_n) for steps first .. first+count-1 since the
 * last load to host arrays (either may be NULL). */
int imrp_get_qdiff(imrp_ctx* ctx, int64_t first, int64_t count, double* qdiff, double* uasy);

/* Queues the copy of the recorded samples [first, first + count) of Q_diff and
 * u_asy (as imrp_get_qdiff) to caller memory (host, preferably pinned, or
 * device) on the context's stream and returns without waiting; the values are
 * there once the stream has reached the copy. Either pointer may be NULL.
 * Errors: IMRP_E_INVAL (range outside the recorded steps), IMRP_E_CUDA. */
int imrp_copy_qdiff_async(imrp_ctx* ctx, int64_t first, int64_t count, double* qdiff, double* uasy);

/* Field E at the current positions (what the next step would use, with the
 * drive u_asy(t_n) of the next step), written to E[n][3] in particle-id
 * order. Does not advance the state. */
int imrp_get_field(imrp_ctx* ctx, double* E);

/* Current state in particle-id order: x[n][3] and the half-step velocity
 * v_{n-1/2}[n][3] (v synchronous with x right after a load). Either may be NULL. */
int imrp_get_particles(imrp_ctx* ctx, double* x, double* v);

/* Probe surface charge Q_S (super-particle charges, Sec. 3) and the number of
 * electrons absorbed at the probe since the load (wall_rule 2; with the other
 * rules Q_S stays the parameters' value and the count 0). Waits for the queued
 * work. Either pointer may be NULL. Errors: IMRP_E_STATE (nothing loaded),
 * IMRP_E_CUDA. */
int imrp_get_surface_charge(imrp_ctx* ctx, double* q_s, int64_t* n_absorbed);

/* Checkpoint of a run: the state in its storage order (the order of the last
 * push), x[n][3], v[n][3] (the half-step velocity), the particle ids id[n],
 * and *step, the number of steps taken since the load. Host arrays of the
 * loaded n. With imrp_restore it continues the run bit for bit: the wall and
 * collision random numbers are counter based on (seed, id, step), and the
 * storage order keeps the order of equal radius keys. Errors: IMRP_E_INVAL
 * (a NULL output), IMRP_E_STATE (nothing loaded). */
int imrp_checkpoint(imrp_ctx* ctx, double* x, double* v, uint32_t* id, int64_t* step);

/* Restores a checkpoint into a context made with the same parameters (with
 * wall_rule 2, q_s set to the surface charge that imrp_get_surface_charge
 * returned at the checkpoint, since the accrual restarts at the restore): the
 * state in the given order with the given ids (a permutation of 0..n-1), the
 * next step is `step`, and the velocities are taken as a half step behind
 * the positions (as imrp_checkpoint returns them) unless step == 0. Q_diff is
 * recorded from step `step` on: imrp_get_qdiff takes first >= step, and
 * imrp_spectrum, which needs the series from the drive, returns IMRP_E_STATE
 * (transform the joined series with imrp_admittance instead). Errors:
 * IMRP_E_INVAL (n out of range, step < 0, ids not a permutation, a particle
 * outside 1 < r < r_out), IMRP_E_NAN, IMRP_E_CUDA. */
int imrp_restore(imrp_ctx* ctx, const double* x, const double* v, const uint32_t* id, int64_t n, int64_t step);

/* Spectrum of the run since the last load (Sec. 4): admittance
 * Y(w) = i w Q^(w)/U^(w) with Q^ = dt sum_n (Q_n - Q_0) e^{-i w t_n} and
 * U^ = sum_n w_n u_n e^{-i w t_n} (w_n: kick weight of step n), at
 * w_j = (j+1) w_max / n_freq, j < n_freq; the sums run on the GPU in FP64.
 * omega, reY, imY: host arrays of n_freq (any may be NULL). w_res: argmax Re Y
 * (parabolic refinement); dw: full width at half maximum of Re Y around it.
 * fit[4] (may be NULL): a, b, c, phi of the least-squares fit
 * a e^{-b tau} sin(c tau + phi), tau = t - t_fit, over t >= t_fit, with
 * t_fit = t0 + 3 width for the Gaussian pulse and 0 otherwise (Sec. 4, s = 1).
 * Errors: IMRP_E_STATE (fewer than 8 steps recorded), IMRP_E_INVAL. */
int imrp_spectrum(imrp_ctx* ctx, int64_t n_freq, double w_max, double* omega, double* reY,
                  double* imY, double* w_res, double* dw, double* fit);

/* Admittance of a given series (Sec. 4), the transform of imrp_spectrum applied
 * to host arrays q[ns] (Q_diff at t_n = n dt) and u[ns] (u_asy at t_n): for
 * example the difference of two runs from the same state with and without the
 * kick (the spontaneous fluctuations, identical in both, cancel), or an
 * ensemble mean. Y(w) = i w Q^(w)/U^(w), Q^ = dt sum_n (q_n - q_0) e^{-i w t_n},
 * U^ = sum_n k_n u_n e^{-i w t_n} with k_0 = first_kick and k_n = dt after it,
 * at w_j = (j+1) w_max / n_freq; the sums run on the GPU (current device) in
 * FP64. omega, reY, imY: host arrays of n_freq (any may be NULL).
 * Errors: IMRP_E_INVAL (ns < 8, n_freq < 3, w_max <= 0, dt <= 0), IMRP_E_NOMEM,
 * IMRP_E_CUDA. */
int imrp_admittance(const double* q, const double* u, int64_t ns, double dt, double first_kick,
                    int64_t n_freq, double w_max, double* omega, double* reY, double* imY);

/* Damped-sine fit of a given series (Sec. 4, the paper's fit of the charge
 * difference, s = 1): least squares of a e^{-b tau} sin(c tau + phi),
 * tau = t - t_fit, against q_n - q_0 over t_fit <= t_n = n dt <= t_end, from
 * the starting rate b0 and frequency w0 (best of four starting phases), as
 * imrp_spectrum does for a context's own series. After a kick of unit area its
 * transform is the Drude dipole term with nu = 2 b, eta = sqrt(b^2 + c^2),
 * C = a c / eta^2. fit[4] = a, b, c, phi (a >= 0, c >= 0, 0 <= phi < 2 pi).
 * Host computation. Errors: IMRP_E_INVAL (fewer than 8 points in the window,
 * non-positive w0, b0 or dt, no convergence). */
int imrp_fit_damped_sine(const double* q, int64_t ns, double dt, double t_fit, double t_end, double w0,
                         double b0, double* fit);

/* Drude fit of a kinetic admittance (Sec. 4, comparison with the Drude model):
 * the dipole term of the Drude admittance,
 *   Y_D(w) = C (1/(i w) + (i w + nu)/eta^2)^{-1} = C i w eta^2 / (eta^2 - w^2 + i w nu)
 * (w, nu, eta in units of w_pe; eta w_pe is the resonance, nu the collision
 * rate), is fitted to Y(w) = reY + i imY by least squares of the integral of
 * |Y_D - Y|^2 over w_lo <= w <= w_hi (the paper integrates from 0 to w_pe),
 * with the trapezoid rule on the given points. The sheath thickness of the
 * paper enters Y_D only through C and eta, which are fitted directly; the
 * vacuum term i w C_vac is left out, as in Q_diff (Sec. 4). The fitted nu is
 * the effective collision rate nu_eff. Host computation (no GPU), on host
 * arrays of n points with increasing omega.
 * out[4]: C, eta, nu, and the relative residual
 * sqrt(int |Y_D - Y|^2 / int |Y|^2).
 * Errors: IMRP_E_INVAL (fewer than 5 points in the window, non-finite input,
 * no positive peak of reY in the window). */
int imrp_drude_fit(const double* omega, const double* reY, const double* imY, int64_t n,
                   double w_lo, double w_hi, double* out);

/* The paper's temperature diagnostic (Sec. 4): nu_eff = K lambda_D w_pe / R
 * with lambda_D = sqrt(eps0 T_e / (n_e e)). imrp_drude_k gives K from nu_eff
 * (in units of w_pe), T_e (eV), R (m) and n_e (m^-3); imrp_drude_te inverts it
 * for T_e (eV) given K. Errors: IMRP_E_INVAL (non-positive argument). */
int imrp_drude_k(double nu_eff_wpe, double T_e_eV, double R_m, double n_e_m3, double* K);
int imrp_drude_te(double nu_eff_wpe, double K, double R_m, double n_e_m3, double* T_e_eV);

/* Floating probe-plasma equilibrium (App. D), the initial condition of the
 * simulation. Units of Sec. 4: r in R, densities in n_inf, psi = e Phi / T_e,
 * charges in e n_inf R^3. It solves
 *   lambda^2 (1/r^2) (r^2 psi')' = exp(psi) - Rhat^2 / (r^2 sqrt(-2 psi))
 * (Boltzmann electrons; cold ions falling in from infinity with the constant
 * flux 4 pi Rhat^2 n_inf sqrt(T_e/m_i)) with the floating condition
 * Rhat^2 = sqrt(m_i/(2 pi m_e)) exp(psi(1)) (Hertz-Langmuir electron flux equal
 * to the ion flux), by shooting from the quasi-neutral branch
 * (exp(psi) = n_i, -1/2 < psi < 0) at r_out inwards to the probe.
 *   lambda      lambda_D / R (> 0)
 *   mass_ratio  m_i / m_e (> 2 pi)
 *   r_out       outer radius of the domain in R (> 1)
 *   n_grid      nodes of the output grid r_k = 1 + k (r_out - 1)/(n_grid - 1) (>= 2)
 *   psi, dpsi   psi and psi' at the nodes (host arrays of n_grid, or NULL)
 *   q_ion, q_elec  ion and electron charge between 1 and r_k (n_grid, or NULL)
 *   out[5]      Rhat, psi(1), psi'(1), the probe's surface charge
 *               Q_S = -4 pi lambda^2 psi'(1) (Gauss's law), and the residual
 *               of the floating condition.
 * Host computation (no GPU, no context). Errors: IMRP_E_INVAL (argument out
 * of range, or no equilibrium whose Bohm radius lies inside r_out). */
int imrp_sheath_solve(double lambda, double mass_ratio, double r_out, int64_t n_grid, double* psi,
                      double* dpsi, double* q_ion, double* q_elec, double* out);

/* Mobile ions. The paper moves its ions as super-particles, like the
 * electrons (Sec. 4: 1e6 super-particles including ions). After this call the
 * particles whose id (their index in the loaded arrays) is at least n_electrons
 * are ions of charge ion_charge (in e, > 0) and mass ion_mass (in m_e, > 0);
 * the others are electrons (q = -1, m = 1). They enter the moments and the
 * pair sums with their charge, the l = 0 term takes the charge inside each
 * particle's radius from a scan of the charges, the push scales by q/m, the
 * walls treat both alike, and collisions act on electrons only. n~ counts the
 * electrons (n_electrons per shell volume, or per the profile's electron
 * charge), and the immobile uniform background keeps background_ions ion
 * super-particles (0 when every ion moves; a profile of imrp_set_ion_profile
 * still applies as given). ion_charge = 0 restores all electrons and the
 * default background (as many ions as particles). Takes effect for the next
 * steps and loads; allocates a few FP64 arrays of the tile count on the first
 * call. Errors: IMRP_E_INVAL (n_electrons outside [1, N], non-positive or
 * non-finite charge or mass, negative background, wall_rule 2), IMRP_E_CUDA. */
int imrp_set_species(imrp_ctx* ctx, int64_t n_electrons, double ion_charge, double ion_mass,
                     double background_ions);

/* Replaces the context's uniform immobile ion background by a radial ion
 * profile, e.g. the equilibrium of imrp_sheath_solve (App. D: the simulation
 * starts from that equilibrium). q_ion[k] (host array of n_tab >= 2, copied)
 * is the ion charge between 1 and r_k = 1 + k (r_out - 1)/(n_tab - 1) in units
 * of e n_inf R^3; between nodes it is taken linear in r, outside [1, r_out]
 * constant. q_elec_total (> 0, same unit) is the electron charge that the
 * loaded super-particles represent, so n~ = N / q_elec_total at every load;
 * q_s (same unit) replaces the surface charge Q_S. The ions stay immobile: on
 * the electron time scale of the runs they move little (m_i/m_e ~ 7e4). Takes
 * effect for the following steps (before or after a load). n_tab = 0 restores
 * the uniform background and the parameters' Q_S. Errors: IMRP_E_INVAL
 * (n_tab == 1, a non-finite or decreasing table, q_elec_total <= 0),
 * IMRP_E_NOMEM, IMRP_E_CUDA. */
int imrp_set_ion_profile(imrp_ctx* ctx, const double* q_ion, int64_t n_tab, double q_elec_total,
                         double q_s);

/* Derived quantities of the context. */
int imrp_get_info(const imrp_ctx* ctx, imrp_info* info);

/* Stage timing. Runs n_steps steps launched one by one (no CUDA graph) with a
 * CUDA event pair around each stage on the context's stream, and writes the
 * summed device time of each stage in milliseconds to ms[IMRP_N_STAGES]:
 * 0 radix sort, 1 reorder, 2 tile moments with the in-group scans,
 * 3 group scan + finalize,
 * 4 field gather + push. The steps are real steps (they advance the state and
 * are recorded like imrp_step). */
#define IMRP_N_STAGES 5
int imrp_profile_steps(imrp_ctx* ctx, int64_t n_steps, double* ms);

/* Measured FP32 FMA throughput of the current device in TFLOP/s (the roofline
 * denominator of the field kernel, which is FP32 arithmetic rather than a
 * tensor-core contraction; the paper has no counterpart): independent FMA
 * chains on every SM (the SM count is read from the device, *sm_count if not
 * NULL), issued once as scalar FMAs and once as packed pairs (two FMAs per
 * instruction), best of ten timed launches of each after a warm-up, the larger
 * of the two, at whatever clock the device runs. Allocates a few bytes and a
 * stream; takes some tens of ms.
 * Errors: IMRP_E_INVAL (tflops NULL), IMRP_E_NOMEM, IMRP_E_CUDA. */
int imrp_fp32_peak(double* tflops, int* sm_count);

/* ---------------------------------------------------------------------------
 * Autotuning and batched ensembles (no counterpart in the paper: they serve the
 * ensemble and request-serving workloads built on the same hot path).
 *
 * imrp_autotune times, on the loaded particles and with field evaluations only
 * (the state does not advance), the field kernel at 8, 4, 2 and 1 warps per
 * CTA and the group scan (the FP64 scan over the 1024-particle scan groups)
 * at 16, 32 and 64 groups per segment at least, and keeps the fastest of each
 * for the context. wpb_out / gseg_out (may be NULL) receive the choices.
 * Errors: IMRP_E_STATE (nothing loaded), IMRP_E_CUDA. */
int imrp_autotune(imrp_ctx* ctx, int* wpb_out, int* gseg_out);

/* A batch steps several loaded contexts of one device together: every step of
 * every context is captured into one CUDA graph, replayed per pair of steps.
 * Within a step, each context sorts and reorders on its own stream (forked
 * from and joined to the batch's stream); then the moments of all contexts of
 * one degree and precision run as one launch over a work list of (context,
 * block of 1024 particles); then each context's scans and finalize; then the
 * field, push and walls of all contexts of one degree and precision as one
 * launch over a work list of (context, CTA of tiles). Instances of uneven N
 * share those launches and overlap on the GPU. The batch does not
 * own the contexts; they must stay alive and must not be used through their
 * own entry points between imrp_batch_step and imrp_batch_sync. Each context
 * computes exactly what imrp_step would compute for it alone.
 * imrp_batch_create: ctxs[n] distinct, loaded, same device.
 * imrp_batch_step: queues n_steps steps of every context (asynchronous).
 * imrp_batch_sync: waits and checks every context's device error flags. */
typedef struct imrp_batch imrp_batch;
int imrp_batch_create(imrp_ctx* const* ctxs, int n, imrp_batch** out);
int imrp_batch_step(imrp_batch* b, int64_t n_steps);
int imrp_batch_sync(imrp_batch* b);
int imrp_batch_destroy(imrp_batch* b);
/* Autotuner of a batch: times the batched field launch of each degree and
 * precision at 8, 4, 2 and 1 warps per CTA (those that fit), on the contexts'
 * current particles with field-only passes (the state does not advance), and
 * keeps the fastest for the batch's later steps. Shapes never change a
 * particle's arithmetic: results stay bit-identical. Errors: IMRP_E_CUDA,
 * IMRP_E_NOMEM, a context's device error (see imrp_batch_failed). */
int imrp_batch_autotune(imrp_batch* b);
/* Issues the batch's work on a caller-owned cudaStream_t (NULL: its own). */
int imrp_batch_set_stream(imrp_batch* b, void* cuda_stream);
const char* imrp_batch_last_error(const imrp_batch* b);
/* Index (in the ctxs of imrp_batch_create) of the context whose error the
 * last imrp_batch_step or imrp_batch_sync returned, or -1 (no error, or one
 * of the batch itself). imrp_batch_sync reports the first failing context
 * and clears its flags; other contexts keep theirs for imrp_sync. */
int imrp_batch_failed(const imrp_batch* b);

/* ---------------------------------------------------------------------------
 * Field evaluation without any allocation. (The paper has no counterpart: this
 * entry point exists for the software that embeds the library.)
 *
 * Some callers cannot call cudaMalloc: code that runs where a framework owns
 * all device memory through its own pool, code issued while another library
 * holds the device's allocation lock, and allocation-free service loops that
 * must not add to device memory after start-up. imrp_field_noalloc computes
 * exactly what imrp_get_field computes (the field E of the modified, truncated
 * Green's function, the ions, Q_S and the drive at step `step`), for a
 * particle set given in device memory, with no context and no allocation: its
 * intermediate buffers live in one static device array of fixed size (about
 * 10 MB), which every GPU that loads this library holds until the process
 * exits.
 *
 *   p       physical parameters as for imrp_create (p->N is ignored, m0_only = 0);
 *           1 <= p->l_max <= IMRP_NOALLOC_MAX_L and l_max instantiated
 *   x_dev   device pointer, FP64 positions [n][3] in units of R, 1 < |x| < r_out
 *   n       1 <= n <= IMRP_NOALLOC_MAX_N; n~ and the ion background follow n
 *           as after imrp_load_particles
 *   step    step index whose drive u_asy(t_step) enters the field (0 as
 *           right after a load)
 *   E_dev   device pointer, FP64 field [n][3] in input order (written)
 *   stream  cudaStream_t (as void*) on which the work is issued; NULL = the
 *           legacy default stream. The call waits for its own work on that
 *           stream before it returns.
 *
 * The first call on a device performs that device's set-up, with that device
 * current: CUDA loads device code lazily, and loading reserves device memory
 * (the code, its tables and the static array itself), so the set-up loads
 * every kernel this entry point can launch (both precisions, every degree up
 * to IMRP_NOALLOC_MAX_L), fills their constant tables and looks up the device
 * address of the static array with cudaGetSymbolAddress. Make that first call
 * at start-up, where reserving memory is allowed, and before any stream
 * capture; later calls load and reserve nothing. The set-up does not survive
 * a cudaDeviceReset of the device (nor does anything else of this library):
 * do not call it across one. Every call on a device shares the one array, and
 * the array keeps the last call's contents (what must start at zero is
 * cleared by each call): calls that overlap on the GPU, from two streams or
 * two host threads, race on it and must not be made.
 * Errors: IMRP_E_INVAL (n or l_max beyond the limits, bad parameters, a
 * position outside the shell), IMRP_E_NAN, IMRP_E_CUDA. */
#define IMRP_NOALLOC_MAX_N 16384
#define IMRP_NOALLOC_MAX_L 16
int imrp_field_noalloc(const imrp_params* p, const double* x_dev, int64_t n, int64_t step,
                       double* E_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IMRP_H */
