// Floating probe-plasma equilibrium of App. D, the initial condition of the
// simulation: host code of the C ABI, no GPU work.
//
// In the units of Sec. 4 (r in R, densities in n_inf, psi = e Phi / T_e,
// lambda = lambda_D / R) the appendix's system is
//   lambda^2 (psi'' + 2 psi' / r) = exp(psi) - Rhat^2 / (r^2 sqrt(-2 psi)),
// Boltzmann electrons against cold ions that fall in from infinity with a
// constant radial flux 4 pi Rhat^2 n_inf c_s, and the floating condition (the
// Hertz-Langmuir electron flux equals the ion flux at the probe)
//   Rhat^2 = sqrt(m_i / (2 pi m_e)) exp(psi(1)).
// Shooting: for a trial Rhat the solution starts on the quasi-neutral branch
// (exp(psi) = n_i, -1/2 < psi < 0) at r_out and is integrated inwards to r = 1
// with an embedded Runge-Kutta 5(4) pair (Dormand and Prince, 1980) under
// local error control; Rhat is the root of the floating condition, found by
// regula falsi with the Illinois modification inside a bracket. The charges
// inside r come from integrating 4 pi r^2 n along with psi.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "../../include/imrp.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Quasi-neutral branch at radius r: with x = ln(-2 psi) the condition
// psi + ln(-2 psi)/2 = 2 ln(Rhat/r) =: t becomes x - e^x = 2 t, whose left side
// rises and is concave on x < 0; Newton from x = 2 t (where it is -e^{2t} < 0)
// approaches the root monotonically from below.
bool quasi_neutral(double r, double rhat, double* psi, double* dpsi) {
  const double t = 2.0 * log(rhat / r);
  if (!(t < -0.5)) return false;
  double x = 2.0 * t;
  for (int it = 0; it < 200; ++it) {
    const double ex = exp(x);
    const double f = x - ex - 2.0 * t;
    const double dx = -f / (1.0 - ex);
    x += dx;
    if (fabs(dx) <= 1e-15 * fmax(1.0, fabs(x))) break;
  }
  const double p = -0.5 * exp(x);
  *psi = p;
  *dpsi = -2.0 / (r * (1.0 + 1.0 / (2.0 * p)));  // d/dr of the branch condition
  return true;
}

struct System {
  double rhat2, inv_lam2;
  // y = (psi, psi', charge of ions outside r, of electrons outside r)
  bool rhs(double r, const double* y, double* f) const {
    if (!(y[0] < 0.0)) return false;
    const double ni = rhat2 / (r * r * sqrt(-2.0 * y[0]));
    const double ne = exp(y[0]);
    f[0] = y[1];
    f[1] = (ne - ni) * inv_lam2 - 2.0 * y[1] / r;
    f[2] = -4.0 * kPi * r * r * ni;
    f[3] = -4.0 * kPi * r * r * ne;
    return true;
  }
};

// Dormand-Prince 5(4) tableau.
constexpr double c2 = 1.0 / 5, c3 = 3.0 / 10, c4 = 4.0 / 5, c5 = 8.0 / 9;
constexpr double a21 = 1.0 / 5;
constexpr double a31 = 3.0 / 40, a32 = 9.0 / 40;
constexpr double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
constexpr double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561, a54 = -212.0 / 729;
constexpr double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247, a64 = 49.0 / 176,
                 a65 = -5103.0 / 18656;
constexpr double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192, b5 = -2187.0 / 6784,
                 b6 = 11.0 / 84;
// fifth- minus fourth-order weights
constexpr double e1 = 71.0 / 57600, e3 = -71.0 / 16695, e4 = 71.0 / 1920, e5 = -17253.0 / 339200,
                 e6 = 22.0 / 525, e7 = -1.0 / 40;

constexpr int kDim = 4;
constexpr double kRtol = 1e-11;
constexpr double kAtol[kDim] = {1e-16, 1e-13, 1e-12, 1e-12};
constexpr int64_t kMaxSteps = 20000000;

// Integrates from r_out down to 1; when grid is non-null, y is recorded at
// the nodes r_k = 1 + k h (k = n-1 ... 0) by landing on each of them.
// Returns false on a non-finite state or too many steps.
bool integrate(const System& s, double r_out, double* y, int64_t n, double* grid_y) {
  double r = r_out;
  const double hg = n > 1 ? (r_out - 1.0) / double(n - 1) : (r_out - 1.0);
  int64_t node = n - 1;  // next node to record (recorded when r reaches it)
  if (grid_y) {
    for (int i = 0; i < kDim; ++i) grid_y[node * kDim + i] = y[i];
    --node;
  }
  double k1[kDim], k2[kDim], k3[kDim], k4[kDim], k5[kDim], k6[kDim], k7[kDim], yt[kDim], yn[kDim];
  if (!s.rhs(r, y, k1)) return false;
  double h = -1e-4 * (r_out - 1.0);
  for (int64_t step = 0; step < kMaxSteps; ++step) {
    if (r <= 1.0) return true;
    double target = grid_y ? 1.0 + double(node) * hg : 1.0;
    if (grid_y && node == 0) target = 1.0;
    bool land = false;
    if (r + h <= target) {
      h = target - r;
      land = true;
    }
#define DP_STAGE(K, R, EXPR)                                   \
  for (int i = 0; i < kDim; ++i) yt[i] = y[i] + h * (EXPR);    \
  if (!s.rhs(R, yt, K)) { h *= 0.25; continue; }
    DP_STAGE(k2, r + c2 * h, a21 * k1[i])
    DP_STAGE(k3, r + c3 * h, a31 * k1[i] + a32 * k2[i])
    DP_STAGE(k4, r + c4 * h, a41 * k1[i] + a42 * k2[i] + a43 * k3[i])
    DP_STAGE(k5, r + c5 * h, a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i])
    DP_STAGE(k6, r + h, a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i])
#undef DP_STAGE
    for (int i = 0; i < kDim; ++i)
      yn[i] = y[i] + h * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
    if (!s.rhs(r + h, yn, k7)) {
      h *= 0.25;
      continue;
    }
    double err = 0.0;
    for (int i = 0; i < kDim; ++i) {
      const double ei =
          h * (e1 * k1[i] + e3 * k3[i] + e4 * k4[i] + e5 * k5[i] + e6 * k6[i] + e7 * k7[i]);
      const double sc = kAtol[i] + kRtol * fmax(fabs(y[i]), fabs(yn[i]));
      err += (ei / sc) * (ei / sc);
    }
    err = sqrt(err / kDim);
    if (!isfinite(err)) return false;
    if (err <= 1.0) {
      r = land ? target : r + h;
      for (int i = 0; i < kDim; ++i) {
        y[i] = yn[i];
        k1[i] = k7[i];  // first-same-as-last
      }
      if (land && grid_y) {
        for (int i = 0; i < kDim; ++i) grid_y[node * kDim + i] = y[i];
        --node;
      }
      if (land && r <= 1.0) return true;
      const double fac = err > 0.0 ? 0.9 * pow(err, -0.2) : 5.0;
      h *= fmin(5.0, fmax(0.2, fac));
    } else {
      h *= fmax(0.2, 0.9 * pow(err, -0.2));
    }
  }
  return false;
}

// psi(1; Rhat) minus the floating condition's value 2 ln Rhat - C.
bool residual(double rhat, double lam, double C, double r_out, double* res, double* y_out,
              int64_t n, double* grid_y) {
  double y[kDim] = {0, 0, 0, 0};
  if (!quasi_neutral(r_out, rhat, &y[0], &y[1])) return false;
  const System s{rhat * rhat, 1.0 / (lam * lam)};
  if (!integrate(s, r_out, y, n, grid_y)) return false;
  *res = y[0] - 2.0 * log(rhat) + C;
  if (y_out)
    for (int i = 0; i < kDim; ++i) y_out[i] = y[i];
  return true;
}

}  // namespace

extern "C" int imrp_sheath_solve(double lambda, double mass_ratio, double r_out, int64_t n_grid,
                                 double* psi, double* dpsi, double* q_ion, double* q_elec,
                                 double* out) {
  if (!(lambda > 0.0) || !isfinite(lambda) || !(mass_ratio > 2.0 * kPi) || !isfinite(mass_ratio) ||
      !(r_out > 1.0) || !isfinite(r_out) || n_grid < 2 || !out)
    return IMRP_E_INVAL;
  const double C = 0.5 * log(mass_ratio / (2.0 * kPi));
  // Bracket: small Rhat leaves the probe in the quasi-neutral plasma (psi(1) >
  // -1/2 > 2 ln Rhat - C), large Rhat puts it deep in a sheath.
  double lo = 0.5 * exp(-0.25), hi = 2.0, flo, fhi;
  if (!residual(lo, lambda, C, r_out, &flo, nullptr, 0, nullptr) || !(flo > 0.0)) return IMRP_E_INVAL;
  for (;;) {
    if (hi * exp(0.25) >= r_out) return IMRP_E_INVAL;  // the Bohm point must lie inside r_out
    if (!residual(hi, lambda, C, r_out, &fhi, nullptr, 0, nullptr)) return IMRP_E_INVAL;
    if (fhi < 0.0) break;
    lo = hi;
    flo = fhi;
    hi *= 1.5;
  }
  // Illinois regula falsi
  int side = 0;
  double rhat = lo;
  for (int it = 0; it < 200; ++it) {
    rhat = (lo * fhi - hi * flo) / (fhi - flo);
    double f;
    if (!residual(rhat, lambda, C, r_out, &f, nullptr, 0, nullptr)) return IMRP_E_INVAL;
    if (f > 0.0) {
      lo = rhat;
      flo = f;
      if (side == 1) fhi *= 0.5;
      side = 1;
    } else if (f < 0.0) {
      hi = rhat;
      fhi = f;
      if (side == -1) flo *= 0.5;
      side = -1;
    } else {
      lo = hi = rhat;
    }
    if (hi - lo <= 1e-15 * rhat) break;
  }
  std::vector<double> gy(size_t(n_grid) * kDim);
  double y1[kDim], f;
  if (!residual(rhat, lambda, C, r_out, &f, y1, n_grid, gy.data())) return IMRP_E_INVAL;
  const double a_ion = gy[2], a_elec = gy[3];  // charges outside r = 1: everything
  for (int64_t k = 0; k < n_grid; ++k) {
    if (psi) psi[k] = gy[k * kDim + 0];
    if (dpsi) dpsi[k] = gy[k * kDim + 1];
    if (q_ion) q_ion[k] = a_ion - gy[k * kDim + 2];
    if (q_elec) q_elec[k] = a_elec - gy[k * kDim + 3];
  }
  out[0] = rhat;
  out[1] = y1[0];
  out[2] = y1[1];
  out[3] = -4.0 * kPi * lambda * lambda * y1[1];
  out[4] = f;
  return IMRP_OK;
}
