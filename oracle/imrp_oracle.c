/*
 * FP64 CPU oracle for the spectral kinetic model of the ideal Multipole
 * Resonance Probe (Gong, Friedrichs, Oberrath, Brinkmann, arXiv 2111.13072).
 *
 * TEST INFRASTRUCTURE. This file is the independent reference that the CUDA
 * path is checked against. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm may load it. It shares no code, header, table
 * or constant generator with the CUDA library.
 *
 * Units (Sec. 4): lengths in the probe radius R, time in 1/omega_pe, charge in
 * e, mass in m_e. The electrode radius is R_E = 1 - d. Every electron
 * super-particle has q = -1, m = 1.
 *
 * What is computed, and where it comes from:
 *   f_l, g_l ........ radial Green's-function coefficients, App. A (last two
 *                     displayed equations of the appendix).
 *   a^D_l, b^D_l, b^P_l  characteristic-function coefficients, Sec. 3.
 *   c_l' ............ Legendre coefficients of Psi_anti, Sec. 3, with
 *                     l = 2l'-1 (the reading is that the series runs over the
 *                     odd degrees l and c_l' belongs to degree 2l'-1).
 *   G~_L(x,x') ...... modified, truncated Green's function for r, r' > R:
 *                     (1/4pi)[1/r_> + sum_{l=1..L} (r_<^l/r_>^{l+1}
 *                     - f_l/(r r')^{l+1}) P_l(cos gamma)]. It follows from the
 *                     spherical-harmonic expansion of G (Sec. 3, R^(p,p)_l),
 *                     the addition theorem, and the floating-potential term
 *                     Psi_sym(r)/(4 pi r'), which cancels the l = 0 image
 *                     (f_0 equals the Psi_sym coefficient for r >= R).
 *   E_k ............. -(1/n~) sum_{i != k} q_i grad_k G~ - grad(Q_S/(4pi n~ r))
 *                     - u_asy grad Psi_anti,L + ion background (Sec. 4,
 *                     dimensionless equations of motion).
 *   Q_diff .......... -(1/n~) sum_i q_i Psi_anti,L(x_i)   (Sec. 4).
 *   push ............ leapfrog (kick-drift-kick with merged kicks) of the
 *                     canonical equations (Sec. 2).
 *   walls ........... diffuse reflection: same speed, random direction, at the
 *                     probe surface r = 1 and at the outer wall (Sec. 4); or
 *                     absorption (the probe's surface charge Q_S takes the
 *                     charge, Sec. 2) with re-injection at the outer wall from
 *                     a flux-weighted Maxwellian.
 *
 * Two field evaluators:
 *   (a) orc_field_brute: the definition, a direct sum over all pairs with
 *       Legendre polynomials; the gradient is taken by forward-mode dual
 *       numbers, so no derivative formula is written by hand.
 *   (b) orc_field_scan: the same sum regrouped by radius order (particles
 *       sorted by (r, id)); prefix sums (from the innermost particle out) and
 *       suffix sums (from the outermost in) of unnormalised complex solid
 *       harmonics r^l P_l^m e^{im phi}/(l+m)! and
 *       (l-m)! P_l^m e^{im phi}/r^{l+1}; gradients again by dual numbers.
 *       It is pinned against (a).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Parameters                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
  double d;        /* relative dielectric thickness; R_E = 1 - d          */
  double eps;      /* relative permittivity of the dielectric shell       */
  double r_out;    /* outer wall radius                                   */
  double n_tilde;  /* super-particles per unit cube at density n_inf      */
  double n_ion;    /* ion super-particles, uniform and immobile in [1,r_out] */
  double q_s;      /* surface charge Q_S in super-particle charge units   */
  int32_t L;       /* truncation degree l_max of the projection P^       */
  int32_t m0_only; /* 1: keep only the m = 0 terms of every degree        */
  int32_t self_image; /* 1: a particle also feels its own image         */
  int32_t pad;
  /* Immobile ions of a given radial profile (App. D) in place of the uniform
   * background: ion_q[k] is the ion charge inside r_k = 1 + k (r_out - 1) /
   * (ion_n - 1), in super-particle charges; between the nodes it is linear in
   * r, outside [1, r_out] constant. NULL: the uniform background n_ion. */
  const double *ion_q;
  int64_t ion_n;
  /* Mobile ions as particles (the paper moves its ions, Sec. 4): charge[i]
   * in e and mass[i] in m_e of particle i in the order of the arrays passed
   * with these parameters; NULL: every particle is an electron (q = -1,
   * m = 1). Electron-neutral collisions act on negative particles only. */
  const double *charge;
  const double *mass;
} orc_field_params;

static inline double orc_q(const orc_field_params *p, int64_t i) { return p->charge ? p->charge[i] : -1.0; }
static inline double orc_m(const orc_field_params *p, int64_t i) { return p->mass ? p->mass[i] : 1.0; }

typedef struct {
  orc_field_params fp;
  double dt;       /* time step                                          */
  int32_t drive_kind; /* 0 Gaussian pulse, 1 impulse at step 0, 2 off   */
  int32_t wall_rule;  /* 0 diffuse reflection, 1 specular reflection,
                         2 absorb (probe: charge to Q_S) and re-inject at r_out */
  double v_hat;    /* drive amplitude (dimensionless voltage)            */
  double sigma;    /* Gaussian pulse width                               */
  double t0;       /* Gaussian pulse centre                              */
  uint64_t seed;   /* wall random-number key                             */
  double nu_coll;  /* electron-neutral collision rate nu (units of omega_pe), 0: none */
  double sigma_v;  /* thermal speed lambda_D omega_pe (units of R omega_pe) of the plasma
                      that wall_rule 2 injects from                                 */
} orc_run_params;

/* ------------------------------------------------------------------ */
/* Coefficients                                                        */
/* ------------------------------------------------------------------ */

/* f_l and g_l of App. A, with R = 1 and R_E = 1 - d. */
static double orc_f(int l, double d, double eps) {
  double x = pow(1.0 - d, 2 * l + 1); /* (R_E/R)^{2l+1} */
  double num = l * (eps - 1.0) + (l + eps + l * eps) * x;
  double den = (l + 1 + l * eps) + (l + 1) * (eps - 1.0) * x;
  return num / den;
}
static double orc_g(int l, double d, double eps) {
  double x = pow(1.0 - d, 2 * l + 1);
  return 1.0 / ((l + 1 + l * eps) + (l + 1) * (eps - 1.0) * x);
}

/* a^D_l, b^D_l, b^P_l of Sec. 3 (common denominator written once). */
static void orc_psi_coeffs(int l, double d, double eps, double *aD, double *bD, double *bP) {
  double den = (l + 1) * (eps - 1.0) * pow(1.0 - d, 2 * l + 1) + l * eps + l + 1;
  *aD = (l + 1) * (eps - 1.0) * pow(1.0 - d, l + 1) / den;
  *bD = pow(1.0 - d, l + 1) * (l * eps + l + 1) / den;
  *bP = (2 * l + 1) * eps * pow(1.0 - d, l + 1) / den;
}

/* Double factorial n!! for odd n >= -1, with (-1)!! = 1. */
static double orc_dfact(int n) {
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}
static double orc_fact(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= k;
  return r;
}

/* c_l' of Sec. 3: (-1/2)^{l'+1} (4l'-1)(2l'-3)!! / l'!, for degree l = 2l'-1. */
static double orc_c_prime(int lp) {
  return pow(-0.5, lp + 1) * (4.0 * lp - 1.0) * orc_dfact(2 * lp - 3) / orc_fact(lp);
}

/* Fills the coefficient tables for degrees 0..L. canti[l] is the coefficient
 * of r^{-(l+1)} P_l(cos theta) in Psi_anti for r >= R: c_l' b^P_l for odd
 * l = 2l'-1 and zero for even l. Any output pointer may be NULL. */
void orc_coeffs(int L, double d, double eps, double *f, double *g, double *aD, double *bD,
                double *bP, double *canti) {
  for (int l = 0; l <= L; ++l) {
    double a, b, p;
    orc_psi_coeffs(l, d, eps, &a, &b, &p);
    if (f) f[l] = orc_f(l, d, eps);
    if (g) g[l] = orc_g(l, d, eps);
    if (aD) aD[l] = a;
    if (bD) bD[l] = b;
    if (bP) bP[l] = p;
    if (canti) canti[l] = (l % 2 == 1) ? orc_c_prime((l + 1) / 2) * p : 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* Dual numbers: a value and its gradient with respect to the field    */
/* point (three partial derivatives).                                  */
/* ------------------------------------------------------------------ */
typedef struct { double v, d[3]; } dual;

static inline dual dc(double v) { dual r = {v, {0, 0, 0}}; return r; }
static inline dual dadd(dual a, dual b) {
  dual r = {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}}; return r;
}
static inline dual dsub(dual a, dual b) {
  dual r = {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}}; return r;
}
static inline dual dscale(dual a, double s) {
  dual r = {a.v * s, {a.d[0] * s, a.d[1] * s, a.d[2] * s}}; return r;
}
static inline dual dmul(dual a, dual b) {
  dual r;
  r.v = a.v * b.v;
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
static inline dual ddiv(dual a, dual b) {
  dual r;
  r.v = a.v / b.v;
  for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r;
}
static inline dual dsqrt(dual a) {
  dual r;
  r.v = sqrt(a.v);
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] / (2.0 * r.v);
  return r;
}
static inline dual dpowi(dual a, int n) {
  dual r = dc(1.0);
  for (int k = 0; k < n; ++k) r = dmul(r, a);
  return r;
}

/* complex dual */
typedef struct { dual re, im; } cdual;
static inline cdual cdmul(cdual a, cdual b) {
  cdual r;
  r.re = dsub(dmul(a.re, b.re), dmul(a.im, b.im));
  r.im = dadd(dmul(a.re, b.im), dmul(a.im, b.re));
  return r;
}
static inline cdual cdscale_d(cdual a, dual s) {
  cdual r = {dmul(a.re, s), dmul(a.im, s)}; return r;
}
static inline cdual cdscale(cdual a, double s) {
  cdual r = {dscale(a.re, s), dscale(a.im, s)}; return r;
}

/* Field point as dual numbers: x = x0 + e_k. */
static void orc_point(const double *x, dual *X, dual *Y, dual *Z) {
  *X = dc(x[0]); X->d[0] = 1.0;
  *Y = dc(x[1]); Y->d[1] = 1.0;
  *Z = dc(x[2]); Z->d[2] = 1.0;
}

/* Legendre polynomials P_0..P_L at u by the three-term recurrence
 * (l+1) P_{l+1} = (2l+1) u P_l - l P_{l-1}. */
static void orc_legendre(int L, dual u, dual *P) {
  P[0] = dc(1.0);
  if (L >= 1) P[1] = u;
  for (int l = 1; l < L; ++l)
    P[l + 1] = dscale(dsub(dscale(dmul(u, P[l]), 2 * l + 1), dscale(P[l - 1], l)), 1.0 / (l + 1));
}

/* ------------------------------------------------------------------ */
/* Psi_anti, the ion background and the drive                          */
/* ------------------------------------------------------------------ */

/* Psi_anti,L(x) = sum over odd l <= L of canti[l] r^{-(l+1)} P_l(z/r), r >= R. */
static dual orc_psi_anti_dual(int L, const double *canti, dual X, dual Y, dual Z) {
  dual r = dsqrt(dadd(dadd(dmul(X, X), dmul(Y, Y)), dmul(Z, Z)));
  dual u = ddiv(Z, r);
  dual P[L + 2];
  orc_legendre(L, u, P);
  dual s = dc(0.0), rinv = ddiv(dc(1.0), r), rp = rinv;
  for (int l = 1; l <= L; ++l) {
    rp = dmul(rp, rinv); /* r^{-(l+1)} */
    if (canti[l] != 0.0) s = dadd(s, dscale(dmul(rp, P[l]), canti[l]));
  }
  return s;
}

double orc_psi_anti(int L, double d, double eps, const double *x) {
  double canti[L + 1];
  orc_coeffs(L, d, eps, NULL, NULL, NULL, NULL, NULL, canti);
  dual X, Y, Z;
  orc_point(x, &X, &Y, &Z);
  return orc_psi_anti_dual(L, canti, X, Y, Z).v;
}

/* Q_diff = -(1/n~) sum_i q_i Psi_anti,L(x_i) (Sec. 4). */
double orc_qdiff(const orc_field_params *p, int64_t n, const double *x) {
  double canti[p->L + 1];
  orc_coeffs(p->L, p->d, p->eps, NULL, NULL, NULL, NULL, NULL, canti);
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    dual X, Y, Z;
    orc_point(x + 3 * i, &X, &Y, &Z);
    s += orc_q(p, i) * orc_psi_anti_dual(p->L, canti, X, Y, Z).v;
  }
  return -s / p->n_tilde;
}

/* Ion charge inside radius r in super-particle charges: the uniform
 * background (density n_ion / V_shell on 1 <= r <= r_out), or the linear
 * interpolation of the given profile ion_q. */
static double orc_ion_charge(const orc_field_params *p, double r) {
  double rc = r < 1.0 ? 1.0 : (r > p->r_out ? p->r_out : r);
  if (!p->ion_q) return p->n_ion * (rc * rc * rc - 1.0) / (p->r_out * p->r_out * p->r_out - 1.0);
  double h = (p->r_out - 1.0) / (double)(p->ion_n - 1);
  int64_t k = (int64_t)floor((rc - 1.0) / h);
  if (k > p->ion_n - 2) k = p->ion_n - 2;
  if (k < 0) k = 0;
  double r0 = 1.0 + k * h;
  return p->ion_q[k] + (rc - r0) / h * (p->ion_q[k + 1] - p->ion_q[k]);
}

/* Electric field of the immobile ions through the l = 0 part 1/(4 pi r_>) of
 * G~, i.e. Gauss's law: E = (1/n~) Q_enc(r) / (4 pi r^2) r^. */
static void orc_ion_field(const orc_field_params *p, const double *x, double *E) {
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double s = orc_ion_charge(p, r) / (4.0 * ORC_PI * p->n_tilde * r * r * r);
  for (int k = 0; k < 3; ++k) E[k] += s * x[k];
}

/* Potential of the same ions (for the energy diagnostic), zero outside r_out:
 * (1/(4 pi n~)) [Q(r)/r + int_r^r_out Q'(s)/s ds]. Uniform background:
 * (n_ion/V_shell/n~) [ (r^3-1)/(3r) + (r_out^2 - r^2)/2 ]. Profile: Q' is
 * constant on each interval of the table, so the integral is a sum of
 * Q' ln(s_b/s_a). */
static double orc_ion_potential(const orc_field_params *p, double r) {
  if (!p->ion_q) {
    double vsh = 4.0 * ORC_PI / 3.0 * (p->r_out * p->r_out * p->r_out - 1.0);
    double rho = p->n_ion / vsh;
    return rho / p->n_tilde * ((r * r * r - 1.0) / (3.0 * r) + 0.5 * (p->r_out * p->r_out - r * r));
  }
  double rc = r < 1.0 ? 1.0 : (r > p->r_out ? p->r_out : r);
  double h = (p->r_out - 1.0) / (double)(p->ion_n - 1);
  double s = 0.0;
  for (int64_t k = 0; k + 1 < p->ion_n; ++k) {
    double a = 1.0 + k * h, b = 1.0 + (k + 1) * h;
    if (b <= rc) continue;
    if (a < rc) a = rc;
    s += (p->ion_q[k + 1] - p->ion_q[k]) / h * log(b / a);
  }
  return (orc_ion_charge(p, r) / r + s) / (4.0 * ORC_PI * p->n_tilde);
}

/* Field of the surface charge, -grad(Q_S/(4 pi n~ r)), and of the drive,
 * -u grad Psi_anti,L, added to E. */
static void orc_external_field(const orc_field_params *p, const double *canti, double u,
                               const double *x, double *E) {
  double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  double r = sqrt(r2);
  double s = p->q_s / (4.0 * ORC_PI * p->n_tilde * r2 * r);
  for (int k = 0; k < 3; ++k) E[k] += s * x[k];
  if (u != 0.0) {
    dual X, Y, Z;
    orc_point(x, &X, &Y, &Z);
    dual psi = orc_psi_anti_dual(p->L, canti, X, Y, Z);
    for (int k = 0; k < 3; ++k) E[k] -= u * psi.d[k];
  }
}

/* ------------------------------------------------------------------ */
/* (a) Brute force: the definition                                    */
/* ------------------------------------------------------------------ */

/* "i is inside k": smaller radius, ties by smaller id (stable (r, id) order). */
static inline int orc_inner(double ri, int64_t idi, double rk, int64_t idk) {
  return ri < rk || (ri == rk && idi < idk);
}

/* sum over l = 1..L of the pair kernel of G~ at field point (X,Y,Z) with a
 * fixed source point xi, multiplied by 4 pi (the l = 0 term 1/r_> included).
 * inner = 1 when the source is the inner one of the pair. with_direct = 0
 * keeps only the image part (used for the self-image). */
static dual orc_pair_kernel(const orc_field_params *p, const double *f, dual X, dual Y, dual Z,
                            const double *xi, int inner, int with_direct) {
  int L = p->L;
  dual rk = dsqrt(dadd(dadd(dmul(X, X), dmul(Y, Y)), dmul(Z, Z)));
  double ri = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
  dual P[L + 2], Pk[L + 2], Pi[L + 2];
  if (p->m0_only) {
    /* m = 0 term of the addition theorem: P_l(cos theta) P_l(cos theta'). */
    orc_legendre(L, ddiv(Z, rk), Pk);
    orc_legendre(L, dc(xi[2] / ri), Pi);
    for (int l = 0; l <= L; ++l) P[l] = dmul(Pk[l], Pi[l]);
  } else {
    dual u = ddiv(dadd(dadd(dscale(X, xi[0]), dscale(Y, xi[1])), dscale(Z, xi[2])), dscale(rk, ri));
    orc_legendre(L, u, P);
  }
  dual rl = inner ? dc(ri) : rk;  /* r_< */
  dual rg = inner ? rk : dc(ri);  /* r_> */
  dual s = with_direct ? ddiv(dc(1.0), rg) : dc(0.0);
  dual ratio = ddiv(rl, rg);               /* r_< / r_> */
  dual dir = ddiv(dc(1.0), rg);            /* r_<^l / r_>^{l+1}, l = 0 */
  dual prod = ddiv(dc(1.0), dscale(rk, ri)); /* 1/(r r') */
  dual img = dc(1.0);
  for (int l = 1; l <= L; ++l) {
    dir = dmul(dir, ratio);
    img = dmul(img, prod);
    dual imgl = dmul(img, prod); /* (r r')^{-(l+1)} */
    dual term = dscale(imgl, -f[l]);
    if (with_direct) term = dadd(term, dir);
    s = dadd(s, dmul(term, P[l]));
  }
  return s;
}

/* Field at the particles listed in ks[0..nk) (all particles when ks is NULL),
 * evaluated by the direct pair sum. x is [n][3], id[n] are the particle ids
 * used for radius ties. u is the drive u_asy at this instant. E is [nk][3]. */
void orc_field_brute(const orc_field_params *p, int64_t n, const double *x, const int64_t *id,
                     double u, int64_t nk, const int64_t *ks, double *E) {
  int L = p->L;
  double f[L + 1], canti[L + 1];
  orc_coeffs(L, p->d, p->eps, f, NULL, NULL, NULL, NULL, canti);
  int64_t cnt = ks ? nk : n;
  for (int64_t a = 0; a < cnt; ++a) {
    int64_t k = ks ? ks[a] : a;
    const double *xk = x + 3 * k;
    double rk = sqrt(xk[0] * xk[0] + xk[1] * xk[1] + xk[2] * xk[2]);
    dual X, Y, Z;
    orc_point(xk, &X, &Y, &Z);
    double g[3] = {0, 0, 0}; /* grad_k of sum_i q_i * 4pi G~ */
    for (int64_t i = 0; i < n; ++i) {
      if (i == k) continue;
      const double *xi = x + 3 * i;
      double ri = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
      dual s = orc_pair_kernel(p, f, X, Y, Z, xi, orc_inner(ri, id[i], rk, id[k]), 1);
      const double qi = orc_q(p, i);
      for (int c = 0; c < 3; ++c) g[c] += qi * s.d[c];
    }
    if (p->self_image) {
      dual s = orc_pair_kernel(p, f, X, Y, Z, xk, 0, 0);
      const double qk = orc_q(p, k);
      for (int c = 0; c < 3; ++c) g[c] += qk * s.d[c];
    }
    double *Ek = E + 3 * a;
    for (int c = 0; c < 3; ++c) Ek[c] = -g[c] / (4.0 * ORC_PI * p->n_tilde);
    orc_ion_field(p, xk, Ek);
    orc_external_field(p, canti, u, xk, Ek);
  }
}

/* G~_L(x, x') (value) and its gradient with respect to x, for r, r' > R.
 * Used by the closed-form (Kelvin) pin. out = {G, dG/dx, dG/dy, dG/dz}. */
void orc_green(const orc_field_params *p, const double *x, const double *xs, double *out) {
  int L = p->L;
  double f[L + 1];
  orc_coeffs(L, p->d, p->eps, f, NULL, NULL, NULL, NULL, NULL);
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double rs = sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
  dual X, Y, Z;
  orc_point(x, &X, &Y, &Z);
  dual s = orc_pair_kernel(p, f, X, Y, Z, xs, rs < r, 1);
  out[0] = s.v / (4.0 * ORC_PI);
  for (int c = 0; c < 3; ++c) out[1 + c] = s.d[c] / (4.0 * ORC_PI);
}

/* ------------------------------------------------------------------ */
/* (b) Sorted scan                                                     */
/* ------------------------------------------------------------------ */

/* Unnormalised complex solid harmonics at a dual field point, 0 <= m <= l <= L:
 *   Mh[l][m] = r^l P_l^m(cos t) e^{im phi} / (l+m)!
 *   Nh[l][m] = (l-m)! P_l^m(cos t) e^{im phi} / r^{l+1}
 * with P_l^m carrying the Condon-Shortley phase. The angular factor
 * Q_l^m = P_l^m e^{im phi} uses sin(t) e^{i phi} = (x + i y)/r, so no pole
 * singularity appears. Arrays are indexed l*(l+1)/2 + m. */
static void orc_solid(int L, dual X, dual Y, dual Z, cdual *Mh, cdual *Nh) {
  dual r = dsqrt(dadd(dadd(dmul(X, X), dmul(Y, Y)), dmul(Z, Z)));
  dual ct = ddiv(Z, r);
  cdual se = {ddiv(X, r), ddiv(Y, r)}; /* sin(t) e^{i phi} */
  int nt = (L + 1) * (L + 2) / 2;
  cdual Q[nt];
  cdual diag = {dc(1.0), dc(0.0)};
  for (int m = 0; m <= L; ++m) {
    if (m > 0) diag = cdscale(cdmul(se, diag), -(2.0 * m - 1.0)); /* P_m^m e^{im phi} */
    Q[m * (m + 1) / 2 + m] = diag;
    if (m + 1 <= L) Q[(m + 1) * (m + 2) / 2 + m] = cdscale(cdscale_d(diag, ct), 2.0 * m + 1.0);
    for (int l = m + 2; l <= L; ++l) {
      cdual a = cdscale(cdscale_d(Q[(l - 1) * l / 2 + m], ct), 2.0 * l - 1.0);
      cdual b = cdscale(Q[(l - 2) * (l - 1) / 2 + m], -(double)(l + m - 1));
      cdual s = {dadd(a.re, b.re), dadd(a.im, b.im)};
      Q[l * (l + 1) / 2 + m] = cdscale(s, 1.0 / (l - m));
    }
  }
  dual rinv = ddiv(dc(1.0), r);
  dual rl = dc(1.0), rm = rinv; /* r^l and r^{-(l+1)} */
  for (int l = 0; l <= L; ++l) {
    for (int m = 0; m <= l; ++m) {
      int j = l * (l + 1) / 2 + m;
      Mh[j] = cdscale(cdscale_d(Q[j], rl), 1.0 / orc_fact(l + m));
      Nh[j] = cdscale(cdscale_d(Q[j], rm), orc_fact(l - m));
    }
    rl = dmul(rl, r);
    rm = dmul(rm, rinv);
  }
}

typedef struct { double re, im; } cplx;

/* sum over m = -l..l of conj(c_l^m) H_l^m for coefficient and harmonic sets
 * with the symmetry X^{-m} = (-1)^m conj(X^m): the m = 0 term plus twice the
 * real part of the m > 0 terms. */
static dual orc_contract(int L, int m0_only, const cplx *c, const cdual *H, int lmin,
                         const double *wl) {
  dual s = dc(0.0);
  for (int l = lmin; l <= L; ++l) {
    dual sl = dc(0.0);
    for (int m = 0; m <= (m0_only ? 0 : l); ++m) {
      int j = l * (l + 1) / 2 + m;
      dual t = dadd(dscale(H[j].re, c[j].re), dscale(H[j].im, c[j].im));
      sl = dadd(sl, m == 0 ? t : dscale(t, 2.0));
    }
    s = dadd(s, wl ? dscale(sl, wl[l]) : sl);
  }
  return s;
}

typedef struct { double r; int64_t id; int64_t idx; } orc_key;
static int orc_key_cmp(const void *a, const void *b) {
  const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
  if (x->r < y->r) return -1;
  if (x->r > y->r) return 1;
  return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Field at every particle by the sorted scan (E is [n][3] in input order). */
void orc_field_scan(const orc_field_params *p, int64_t n, const double *x, const int64_t *id,
                    double u, double *E) {
  int L = p->L;
  int nt = (L + 1) * (L + 2) / 2;
  double f[L + 1], canti[L + 1], negf[L + 1];
  orc_coeffs(L, p->d, p->eps, f, NULL, NULL, NULL, NULL, canti);
  for (int l = 0; l <= L; ++l) negf[l] = -f[l];
  orc_key *ord = (orc_key *)malloc(sizeof(orc_key) * (n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    const double *xi = x + 3 * i;
    ord[i].r = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    ord[i].id = id[i];
    ord[i].idx = i;
  }
  qsort(ord, n, sizeof(orc_key), orc_key_cmp);

  cplx *A = calloc(nt, sizeof(cplx));    /* prefix of q M over inner particles   */
  cplx *B = calloc(nt, sizeof(cplx));    /* suffix of q N over outer particles   */
  cplx *Wim = calloc(nt, sizeof(cplx));  /* total of q M(x_i)/r_i^{2l+1} (image)  */
  cplx *Wk = calloc(nt, sizeof(cplx));
  cdual *Mh = malloc(sizeof(cdual) * nt), *Nh = malloc(sizeof(cdual) * nt);

  /* totals of the image moments */
  for (int64_t j = 0; j < n; ++j) {
    const double *xi = x + 3 * ord[j].idx;
    dual X, Y, Z;
    orc_point(xi, &X, &Y, &Z);
    orc_solid(L, X, Y, Z, Mh, Nh);
    double ri = ord[j].r;
    const double qj = orc_q(p, ord[j].idx);
    for (int l = 0; l <= L; ++l) {
      double sc = pow(ri, -(2 * l + 1));
      for (int m = 0; m <= l; ++m) {
        int q = l * (l + 1) / 2 + m;
        Wim[q].re += qj * Mh[q].re.v * sc; Wim[q].im += qj * Mh[q].im.v * sc;
      }
    }
  }
  /* inner particles, the image and l = 0, in (r, id) order; the prefix A is
   * summed from the innermost outwards */
  for (int64_t j = 0; j < n; ++j) {
    int64_t k = ord[j].idx;
    const double *xk = x + 3 * k;
    double rk = ord[j].r;
    dual X, Y, Z;
    orc_point(xk, &X, &Y, &Z);
    orc_solid(L, X, Y, Z, Mh, Nh);
    const double qk = orc_q(p, k);
    /* image moments without particle k unless it feels its own image */
    for (int l = 0; l <= L; ++l) {
      double sc = pow(rk, -(2 * l + 1));
      for (int m = 0; m <= l; ++m) {
        int q = l * (l + 1) / 2 + m;
        Wk[q] = Wim[q];
        if (!p->self_image) { Wk[q].re -= qk * Mh[q].re.v * sc; Wk[q].im -= qk * Mh[q].im.v * sc; }
      }
    }
    /* 4 pi * potential (without the 1/n~) as a function of the field point */
    dual phi = orc_contract(L, p->m0_only, A, Nh, 1, NULL);
    phi = dadd(phi, orc_contract(L, p->m0_only, Wk, Nh, 1, negf));
    /* l = 0: inner charge A_00 times 1/r; outer charges give a constant */
    phi = dadd(phi, dscale(Nh[0].re, A[0].re));
    double *Ek = E + 3 * k;
    for (int c = 0; c < 3; ++c) Ek[c] = -phi.d[c] / (4.0 * ORC_PI * p->n_tilde);
    orc_ion_field(p, xk, Ek);
    orc_external_field(p, canti, u, xk, Ek);
    for (int q = 0; q < nt; ++q) {
      A[q].re += qk * Mh[q].re.v; A[q].im += qk * Mh[q].im.v;
    }
  }
  /* outer particles, in reverse order: the suffix B is summed from the
   * outermost inwards (as total minus prefix it would cancel: at high l the
   * inner particles' r^-(l+1) outweigh the outer ones' by orders of magnitude) */
  for (int64_t j = n - 1; j >= 0; --j) {
    int64_t k = ord[j].idx;
    dual X, Y, Z;
    orc_point(x + 3 * k, &X, &Y, &Z);
    orc_solid(L, X, Y, Z, Mh, Nh);
    const double qk = orc_q(p, k);
    dual phi = orc_contract(L, p->m0_only, B, Mh, 1, NULL);
    double *Ek = E + 3 * k;
    for (int c = 0; c < 3; ++c) Ek[c] -= phi.d[c] / (4.0 * ORC_PI * p->n_tilde);
    for (int q = 0; q < nt; ++q) {
      B[q].re += qk * Nh[q].re.v; B[q].im += qk * Nh[q].im.v;
    }
  }
  free(A); free(B); free(Wim); free(Wk); free(Mh); free(Nh); free(ord);
}

/* ------------------------------------------------------------------ */
/* Energy                                                              */
/* ------------------------------------------------------------------ */

/* H = sum v^2/2 + (1/2n~) sum_{k != i} q_k q_i G~(x_k,x_i)
 *     + sum_k q_k (Phi_ion + Q_S/(4 pi n~ r_k) + u Psi_anti,L)     (Sec. 2).
 * With self_image = 1 each particle adds (1/2n~) q_k^2 G~_image(x_k, x_k). */
double orc_energy(const orc_field_params *p, int64_t n, const double *x, const double *v,
                  const int64_t *id, double u) {
  int L = p->L;
  double f[L + 1], canti[L + 1];
  orc_coeffs(L, p->d, p->eps, f, NULL, NULL, NULL, NULL, canti);
  double kin = 0.0, pot = 0.0, ext = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    const double *xk = x + 3 * k, *vk = v + 3 * k;
    const double qk = orc_q(p, k);
    kin += 0.5 * orc_m(p, k) * (vk[0] * vk[0] + vk[1] * vk[1] + vk[2] * vk[2]);
    double rk = sqrt(xk[0] * xk[0] + xk[1] * xk[1] + xk[2] * xk[2]);
    dual X, Y, Z;
    orc_point(xk, &X, &Y, &Z);
    for (int64_t i = k + 1; i < n; ++i) {
      const double *xi = x + 3 * i;
      double ri = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
      dual s = orc_pair_kernel(p, f, X, Y, Z, xi, orc_inner(ri, id[i], rk, id[k]), 1);
      pot += qk * orc_q(p, i) * s.v / (4.0 * ORC_PI * p->n_tilde);
    }
    if (p->self_image) {
      dual s = orc_pair_kernel(p, f, X, Y, Z, xk, 0, 0);
      pot += 0.5 * qk * qk * s.v / (4.0 * ORC_PI * p->n_tilde);
    }
    ext += qk * (orc_ion_potential(p, rk) + p->q_s / (4.0 * ORC_PI * p->n_tilde * rk));
    if (u != 0.0) ext += qk * u * orc_psi_anti_dual(L, canti, X, Y, Z).v;
  }
  return kin + pot + ext;
}

/* ------------------------------------------------------------------ */
/* Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel */
/* random numbers: as easy as 1, 2, 3", SC 2011).                       */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Walls (Sec. 4): a particle that left [1, r_out] is mirrored back    */
/* radially and leaves with the same speed. Diffuse: the direction is  */
/* uniform in solid angle over the inward hemisphere, drawn from       */
/* Philox with counter (step, step>>32, id, 0x494D5250) and key (seed).*/
/* The tangent frame is the branchless orthonormal basis of Duff et    */
/* al., "Building an orthonormal basis, revisited", JCGT 2017.         */
/* Specular: the radial velocity component changes sign.               */
/* ------------------------------------------------------------------ */

/* Tangent frame (t1, t2) of the unit vector n (Duff et al. 2017). */
static void orc_onb(const double *n, double *t1, double *t2) {
  double s = n[2] >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (s + n[2]);
  double b = n[0] * n[1] * a;
  t1[0] = 1.0 + s * n[0] * n[0] * a; t1[1] = s * b; t1[2] = -s * n[0];
  t2[0] = b; t2[1] = s + n[1] * n[1] * a; t2[2] = -n[1];
}

/* Uniform in (0, 1) from the top 24 bits of a Philox word (never 0 or 1). */
static double orc_u24(uint32_t w) { return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Absorb and re-inject (wall_rule 2; north_star names "absorbs or re-injects",
 * and the paper's floating probe collects the electrons that reach it: its
 * surface charge Q_S is homogeneous on S, Sec. 2). The particle that left is
 * replaced, under the same id, by one entering through the outer wall from
 * the bulk plasma: a flux-weighted Maxwellian of thermal speed sigma_v. Six
 * uniforms from two Philox blocks, counter (step, step>>32, id, 0x494E4A30 and
 * 0x494E4A31), key (seed):
 *   u1, u2: the entry point r_out n, n isotropic (cos = 1 - 2 u1, phi = 2 pi u2);
 *   u3: inward normal speed v_n = sigma_v sqrt(-2 ln u3) (the density of the
 *       normal speeds that cross a surface, v_n exp(-v_n^2 / (2 sigma_v^2)));
 *   u4, u5: the two tangential components, normal with deviation sigma_v
 *       (Box-Muller: rho = sigma_v sqrt(-2 ln u4), angle 2 pi u5);
 *   u6: the fraction of the step since it crossed, so it sits at radius
 *       r_out - u6 dt v_n (at least 1), on the ray of n.
 * The velocity is -v_n n + vt1 t1 + vt2 t2 with (t1, t2) the frame of n. */
static void orc_inject(const orc_run_params *rp, double *x, double *v, int64_t pid, int64_t step) {
  uint32_t ctr[4] = {(uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)pid,
                     0x494E4A30u};
  uint32_t key[2] = {(uint32_t)rp->seed, (uint32_t)(rp->seed >> 32)};
  uint32_t a[4], b[4];
  orc_philox4x32_10(ctr, key, a);
  ctr[3] = 0x494E4A31u;
  orc_philox4x32_10(ctr, key, b);
  double u1 = orc_u24(a[0]), u2 = orc_u24(a[1]), u3 = orc_u24(a[2]), u4 = orc_u24(a[3]);
  double u5 = orc_u24(b[0]), u6 = orc_u24(b[1]);
  double ct = 1.0 - 2.0 * u1, st = sqrt(1.0 - ct * ct), ph = 2.0 * ORC_PI * u2;
  double n[3] = {st * cos(ph), st * sin(ph), ct};
  double vn = rp->sigma_v * sqrt(-2.0 * log(u3));
  double rho = rp->sigma_v * sqrt(-2.0 * log(u4)), ps = 2.0 * ORC_PI * u5;
  double vt1 = rho * cos(ps), vt2 = rho * sin(ps);
  double t1[3], t2[3];
  orc_onb(n, t1, t2);
  double r = rp->fp.r_out - u6 * rp->dt * vn;
  if (r < 1.0) r = 1.0;
  for (int c = 0; c < 3; ++c) {
    x[c] = r * n[c];
    v[c] = -vn * n[c] + vt1 * t1[c] + vt2 * t2[c];
  }
}

/* The wall rule on one particle after its drift. Returns 0 (inside),
 * 1 (reflected), 2 (absorbed at the probe and re-injected), 3 (left through
 * the outer wall and re-injected). */
static int orc_wall(const orc_run_params *rp, double *x, double *v, int64_t pid, int64_t step) {
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double r_out = rp->fp.r_out;
  double sgn; /* +1: inward normal points outward (probe wall), -1: outer wall */
  double rn;
  if (r < 1.0) { sgn = 1.0; rn = 2.0 - r; }
  else if (r > r_out) { sgn = -1.0; rn = 2.0 * r_out - r; }
  else return 0;
  if (rp->wall_rule == 2) {
    orc_inject(rp, x, v, pid, step);
    return sgn > 0.0 ? 2 : 3;
  }
  if (rn < 1.0) rn = 1.0;
  if (rn > r_out) rn = r_out;
  double e[3] = {x[0] / r, x[1] / r, x[2] / r};
  for (int c = 0; c < 3; ++c) x[c] = e[c] * rn;
  double nrm[3] = {sgn * e[0], sgn * e[1], sgn * e[2]}; /* inward unit normal */
  if (rp->wall_rule == 1) {
    double vr = v[0] * e[0] + v[1] * e[1] + v[2] * e[2];
    for (int c = 0; c < 3; ++c) v[c] -= 2.0 * vr * e[c];
    return 1;
  }
  double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  uint32_t ctr[4] = {(uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)pid,
                     0x494D5250u};
  uint32_t key[2] = {(uint32_t)rp->seed, (uint32_t)(rp->seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  double u1 = (double)(o[0] >> 8) * (1.0 / 16777216.0);
  double u2 = (double)(o[1] >> 8) * (1.0 / 16777216.0);
  double ca = 1.0 - u1;                 /* cos of the angle to the normal, (0,1] */
  double sa = sqrt(1.0 - ca * ca);
  double ph = 2.0 * ORC_PI * u2;
  double t1[3], t2[3];
  orc_onb(nrm, t1, t2);
  double cp = cos(ph), sp = sin(ph);
  for (int c = 0; c < 3; ++c) v[c] = speed * (ca * nrm[c] + sa * (cp * t1[c] + sp * t2[c]));
  return 1;
}

/* The injection alone for n particle ids at a step (for pins): x, v [n][3]. */
void orc_inject_many(const orc_run_params *rp, int64_t n, double *x, double *v, const int64_t *id,
                     int64_t step) {
  for (int64_t i = 0; i < n; ++i) orc_inject(rp, x + 3 * i, v + 3 * i, id[i], step);
}

/* Electron-neutral collisions (Sec. 5 names them as the next addition; the  */
/* Drude model of Sec. 4 damps with the collision rate nu). Reading: a      */
/* constant rate nu; in each step an electron collides with probability     */
/* P = 1 - exp(-nu dt) and scatters elastically and isotropically: same      */
/* speed, direction uniform on the sphere (the neutral's recoil neglected).  */
/* The decision and the direction come from Philox with counter             */
/* (step, step>>32, id, 0x434F4C4C) and key (seed): collide when the top 24 */
/* bits of the first word are below floor(P 2^24); cos(theta) = 1 - 2 u1,   */
/* phi = 2 pi u2 from the next two words. Returns 1 on a collision.         */
/* ------------------------------------------------------------------ */
uint32_t orc_coll_threshold(double nu, double dt) {
  if (!(nu > 0.0)) return 0u;
  double p = 1.0 - exp(-nu * dt);
  return (uint32_t)floor(p * 16777216.0);
}

static int orc_collide(const orc_run_params *rp, uint32_t thr, double *v, int64_t pid, int64_t step) {
  if (thr == 0u) return 0;
  uint32_t ctr[4] = {(uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)pid,
                     0x434F4C4Cu};
  uint32_t key[2] = {(uint32_t)rp->seed, (uint32_t)(rp->seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  if ((o[0] >> 8) >= thr) return 0;
  double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double u1 = (double)(o[1] >> 8) * (1.0 / 16777216.0);
  double u2 = (double)(o[2] >> 8) * (1.0 / 16777216.0);
  double ct = 1.0 - 2.0 * u1;
  double st = sqrt(1.0 - ct * ct);
  double ph = 2.0 * ORC_PI * u2;
  v[0] = speed * st * cos(ph);
  v[1] = speed * st * sin(ph);
  v[2] = speed * ct;
  return 1;
}

/* The collision operator alone on n velocities (for pins): returns the */
/* number of collisions of this step.                                   */
int64_t orc_collisions(const orc_run_params *rp, int64_t n, double *v, const int64_t *id, int64_t step) {
  const uint32_t thr = orc_coll_threshold(rp->nu_coll, rp->dt);
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i) c += orc_collide(rp, thr, v + 3 * i, id[i], step);
  return c;
}

/* Drive u_asy(t_n) (Sec. 4 and the Gaussian-pulse reading). */
double orc_drive(const orc_run_params *rp, int64_t step) {
  double t = step * rp->dt;
  if (rp->drive_kind == 0) {
    double z = (t - rp->t0) / rp->sigma;
    return rp->v_hat * exp(-0.5 * z * z);
  }
  if (rp->drive_kind == 1) return step == 0 ? rp->v_hat : 0.0;
  return 0.0;
}

/* Advances n particles by nsteps leapfrog steps, starting at absolute step
 * index step0. x and v are [n][3]; v holds the half-step velocity except when
 * first_half_kick = 1 (velocities synchronous with x, so the first kick is
 * dt/2). evaluator: 0 brute force, 1 sorted scan. qdiff[s] and uasy[s]
 * receive Q_diff and u_asy at the positions used by step s (either may be
 * NULL). With wall_rule 2 the charge of every particle absorbed at the probe
 * joins the surface charge Q_S (starting from rp->fp.q_s), which the field of
 * the following steps feels; q_s_out (may be NULL) receives Q_S after the last
 * step and absorbed (may be NULL) the number of probe absorptions. Returns the
 * number of wall hits (reflections, or absorptions at either wall). */
int64_t orc_run(const orc_run_params *rp, int64_t n, double *x, double *v, const int64_t *id,
                int64_t step0, int64_t nsteps, int first_half_kick, int evaluator, double *qdiff,
                double *uasy, double *q_s_out, int64_t *absorbed) {
  double *E = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  int64_t hits = 0, nabs = 0;
  orc_field_params fp = rp->fp; /* its q_s accrues the absorbed charge */
  const uint32_t thr = orc_coll_threshold(rp->nu_coll, rp->dt);
  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t step = step0 + s;
    double u = orc_drive(rp, step);
    if (evaluator == 0) orc_field_brute(&fp, n, x, id, u, n, NULL, E);
    else orc_field_scan(&fp, n, x, id, u, E);
    if (qdiff) qdiff[s] = orc_qdiff(&fp, n, x);
    if (uasy) uasy[s] = u;
    double kick = (s == 0 && first_half_kick) ? 0.5 * rp->dt : rp->dt;
    double dq = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double qm = orc_q(&fp, i) / orc_m(&fp, i);  /* -1 for electrons */
      for (int c = 0; c < 3; ++c) v[3 * i + c] += kick * qm * E[3 * i + c];
      for (int c = 0; c < 3; ++c) x[3 * i + c] += rp->dt * v[3 * i + c];
      int w = orc_wall(rp, x + 3 * i, v + 3 * i, id[i], step);
      hits += w != 0;
      if (w == 2) { dq += orc_q(&fp, i); ++nabs; }
      if (orc_q(&fp, i) < 0.0) orc_collide(rp, thr, v + 3 * i, id[i], step);
    }
    fp.q_s += dq;
  }
  if (q_s_out) *q_s_out = fp.q_s;
  if (absorbed) *absorbed = nabs;
  free(E);
  return hits;
}
