// Drude fit of the kinetic admittance and the temperature diagnostic (Sec. 4,
// comparison with the Drude model): host code of the C ABI, no GPU work.
#include <math.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/imrp.h"

namespace {

constexpr double kE = 1.602176634e-19;     // C
constexpr double kEps0 = 8.8541878128e-12; // F/m

struct Cplx {
  double re, im;
};
inline Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline Cplx cdiv(Cplx a, Cplx b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// g(w) = i w eta^2 / D, D = eta^2 - w^2 + i w nu, and its derivatives with
// respect to log eta and log nu:
//   dg/deta = 2 i w eta (i w nu - w^2) / D^2,  dg/dnu = w^2 eta^2 / D^2.
struct Model {
  Cplx g, g_la, g_ln;
};
inline Model model(double w, double eta, double nu) {
  const Cplx D = {eta * eta - w * w, w * nu};
  const Cplx D2 = cmul(D, D);
  Model m;
  m.g = cdiv({0.0, w * eta * eta}, D);
  const Cplx dge = cdiv(cmul({0.0, 2.0 * w * eta}, {-w * w, w * nu}), D2);
  const Cplx dgn = cdiv({w * w * eta * eta, 0.0}, D2);
  m.g_la = {eta * dge.re, eta * dge.im};
  m.g_ln = {nu * dgn.re, nu * dgn.im};
  return m;
}

// sum of weights * |C g - Y|^2
double objective(const std::vector<double>& w, const std::vector<double>& wt, const std::vector<Cplx>& y,
                 double C, double eta, double nu) {
  double s = 0.0;
  for (size_t j = 0; j < w.size(); ++j) {
    const Cplx g = model(w[j], eta, nu).g;
    const double dr = C * g.re - y[j].re, di = C * g.im - y[j].im;
    s += wt[j] * (dr * dr + di * di);
  }
  return s;
}

// 3 x 3 linear solve by Gaussian elimination with partial pivoting; false if singular.
bool solve3(double A[3][3], double b[3], double x[3]) {
  int p[3] = {0, 1, 2};
  for (int c = 0; c < 3; ++c) {
    int best = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(A[p[r]][c]) > fabs(A[p[best]][c])) best = r;
    std::swap(p[c], p[best]);
    if (!(fabs(A[p[c]][c]) > 0.0)) return false;
    for (int r = c + 1; r < 3; ++r) {
      const double f = A[p[r]][c] / A[p[c]][c];
      for (int k = c; k < 3; ++k) A[p[r]][k] -= f * A[p[c]][k];
      b[p[r]] -= f * b[p[c]];
    }
  }
  for (int c = 2; c >= 0; --c) {
    double s = b[p[c]];
    for (int k = c + 1; k < 3; ++k) s -= A[p[c]][k] * x[k];
    x[c] = s / A[p[c]][c];
  }
  return true;
}

}  // namespace

extern "C" int imrp_drude_fit(const double* omega, const double* reY, const double* imY, int64_t n,
                              double w_lo, double w_hi, double* out) {
  if (!omega || !reY || !imY || !out || n < 1 || !(w_hi > w_lo)) return IMRP_E_INVAL;
  std::vector<double> w;
  std::vector<Cplx> y;
  for (int64_t j = 0; j < n; ++j) {
    if (!(isfinite(omega[j]) && isfinite(reY[j]) && isfinite(imY[j]))) return IMRP_E_INVAL;
    if (j > 0 && !(omega[j] > omega[j - 1])) return IMRP_E_INVAL;
    if (omega[j] >= w_lo && omega[j] <= w_hi) {
      w.push_back(omega[j]);
      y.push_back({reY[j], imY[j]});
    }
  }
  const size_t m = w.size();
  if (m < 5) return IMRP_E_INVAL;
  // trapezoid weights of the integral over the window's points
  std::vector<double> wt(m, 0.0);
  for (size_t j = 0; j + 1 < m; ++j) {
    const double h = 0.5 * (w[j + 1] - w[j]);
    wt[j] += h;
    wt[j + 1] += h;
  }
  // starting point: eta at the peak of Re Y, nu its full width at half
  // maximum (both exact for the model: Re Y_D peaks at eta with FWHM nu)
  size_t jp = 0;
  for (size_t j = 1; j < m; ++j)
    if (y[j].re > y[jp].re) jp = j;
  if (!(y[jp].re > 0.0)) return IMRP_E_INVAL;
  const double half = 0.5 * y[jp].re;
  double wl = w.front(), wr = w.back();
  for (size_t j = jp; j > 0; --j)
    if (y[j - 1].re < half) {
      wl = w[j - 1] + (half - y[j - 1].re) * (w[j] - w[j - 1]) / (y[j].re - y[j - 1].re);
      break;
    }
  for (size_t j = jp; j + 1 < m; ++j)
    if (y[j + 1].re < half) {
      wr = w[j] + (y[j].re - half) * (w[j + 1] - w[j]) / (y[j].re - y[j + 1].re);
      break;
    }
  double eta = w[jp];
  double nu = wr - wl > 0.0 ? wr - wl : 0.1 * eta;
  // C by linear least squares at the starting (eta, nu)
  double C;
  {
    double num = 0.0, den = 0.0;
    for (size_t j = 0; j < m; ++j) {
      const Cplx g = model(w[j], eta, nu).g;
      num += wt[j] * (g.re * y[j].re + g.im * y[j].im);
      den += wt[j] * (g.re * g.re + g.im * g.im);
    }
    C = den > 0.0 ? num / den : 1.0;
  }
  // Levenberg-Marquardt on (C, log eta, log nu)
  double f = objective(w, wt, y, C, eta, nu);
  double lam = 1e-3;
  for (int it = 0; it < 500; ++it) {
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
    for (size_t j = 0; j < m; ++j) {
      const Model md = model(w[j], eta, nu);
      const double rr = C * md.g.re - y[j].re, ri = C * md.g.im - y[j].im;
      const double Jr[3] = {md.g.re, C * md.g_la.re, C * md.g_ln.re};
      const double Ji[3] = {md.g.im, C * md.g_la.im, C * md.g_ln.im};
      for (int a = 0; a < 3; ++a) {
        b[a] -= wt[j] * (Jr[a] * rr + Ji[a] * ri);
        for (int c = 0; c < 3; ++c) A[a][c] += wt[j] * (Jr[a] * Jr[c] + Ji[a] * Ji[c]);
      }
    }
    bool improved = false;
    for (int tries = 0; tries < 40 && !improved; ++tries) {
      double M[3][3], rhs[3] = {b[0], b[1], b[2]}, dx[3];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) M[a][c] = A[a][c] + (a == c ? lam * A[a][a] : 0.0);
      if (!solve3(M, rhs, dx)) {
        lam *= 10.0;
        continue;
      }
      const double C2 = C + dx[0], eta2 = eta * exp(dx[1]), nu2 = nu * exp(dx[2]);
      const double f2 = objective(w, wt, y, C2, eta2, nu2);
      if (isfinite(f2) && f2 <= f) {
        const double rel = (f - f2) / (f > 0.0 ? f : 1.0);
        C = C2;
        eta = eta2;
        nu = nu2;
        f = f2;
        lam = lam > 1e-12 ? lam * 0.3 : lam;
        improved = true;
        if (rel < 1e-15 && fabs(dx[1]) < 1e-13 && fabs(dx[2]) < 1e-13) it = 500;
      } else {
        lam *= 10.0;
      }
    }
    if (!improved) break;
  }
  double ny = 0.0;
  for (size_t j = 0; j < m; ++j) ny += wt[j] * (y[j].re * y[j].re + y[j].im * y[j].im);
  out[0] = C;
  out[1] = eta;
  out[2] = nu;
  out[3] = ny > 0.0 ? sqrt(f / ny) : 0.0;
  return IMRP_OK;
}

extern "C" int imrp_drude_k(double nu_eff_wpe, double T_e_eV, double R_m, double n_e_m3, double* K) {
  if (!K || !(nu_eff_wpe > 0) || !(T_e_eV > 0) || !(R_m > 0) || !(n_e_m3 > 0)) return IMRP_E_INVAL;
  const double lambda_D = sqrt(kEps0 * T_e_eV / (n_e_m3 * kE));
  *K = nu_eff_wpe * R_m / lambda_D;
  return IMRP_OK;
}

extern "C" int imrp_drude_te(double nu_eff_wpe, double K, double R_m, double n_e_m3, double* T_e_eV) {
  if (!T_e_eV || !(nu_eff_wpe > 0) || !(K > 0) || !(R_m > 0) || !(n_e_m3 > 0)) return IMRP_E_INVAL;
  const double lambda_D = nu_eff_wpe * R_m / K;
  *T_e_eV = lambda_D * lambda_D * n_e_m3 * kE / kEps0;
  return IMRP_OK;
}
