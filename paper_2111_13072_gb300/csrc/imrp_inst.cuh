// Instantiation of the per-degree kernels for one precision and a list of
// degrees. Each unit that includes this file owns its constant-memory
// recurrence tables and fills them once per device.
#pragma once

#include <math.h>

#include <mutex>

#include "imrp_internal.h"
#include "imrp_kernels.cuh"

namespace imrp {
namespace {

// a_lm, b_lm of the solid-harmonic recurrences and the rescaling nu_lm.
inline double rec_a(int l, int m) { return m < l ? (2.0 * l - 1.0) / sqrt(double(l + m) * double(l - m)) : 0.0; }
inline double rec_b(int l, int m) {
  return m < l ? sqrt(double(l + m - 1) * double(l - m - 1) / (double(l + m) * double(l - m))) : 0.0;
}
inline double rec_nu(int l, int m) {
  double v = 1.0;
  for (int k = l; k >= m + 2; k -= 2) v *= rec_b(k, m);
  return v;
}

template <class T> void fill_tables(Tables<T>& t) {
  for (int l = 0; l < kTabL; ++l)
    for (int m = 0; m < kTabL; ++m) {
      t.an[l * kTabL + m] = T(m < l ? rec_a(l, m) * rec_nu(l - 1, m) / rec_nu(l, m) : 0.0);
      t.nu[l * kTabL + m] = T(m <= l ? rec_nu(l, m) : 0.0);
    }
  for (int m = 0; m < kTabL; ++m) t.dg[m] = m == 0 ? T(1) : T(-sqrt((2.0 * m - 1.0) / (2.0 * m)));
}

// Host copies of the prologue tables, computed when the library is loaded
// (fixed-size arrays: no allocation), uploaded once per device by unit_init.
EntryRec h_ent[kEntTotal];
uint16_t h_comp[kCompTotal];

void fill_prologue_tables() {
  for (int di = 0; di < kNumDegrees; ++di) {
    const int L = degree_at(di);
    const int eo = ent_off(L), co = comp_tab_off(L);
    for (int m = 0; m <= L; ++m)
      for (int l = (m > 1 ? m : 1); l <= L; ++l)
        for (int part = 0; part < (m > 0 ? 2 : 1); ++part)
          h_comp[co + comp_idx(L, l, m, part)] =
              uint16_t(l | ((m == 0 && (l & 1)) ? (1 << 8) : 0) | (m > 0 ? (1 << 9) : 0));
    auto record = [&](bool isI, int Lp, int M) {
      EntryRec r{};
      const int s = isI ? 0 : 1;
      const int lq = isI ? Lp - 1 : Lp + 1;
      const int ms[3] = {M - 1, M + 1, M};
      const int16_t zero = int16_t(2 * ncomp(L));  // the scratch's zero slot
      double sgn_r = 1.0, sgn_i = 1.0;             // sign of source 1 (m = M - 1 < 0 only at M = 0)
      for (int q = 0; q < 3; ++q) {
        const int mq = ms[q], am = mq < 0 ? -mq : mq;
        if (lq < 1 || lq > L || am > lq) {
          r.src[2 * q] = zero;
          r.src[2 * q + 1] = zero;
          continue;
        }
        r.src[2 * q] = int16_t(2 * comp_idx(L, lq, am, 0) + s);
        r.src[2 * q + 1] = am > 0 ? int16_t(2 * comp_idx(L, lq, am, 1) + s) : zero;
        if (mq < 0) {  // X^{-m} = (-1)^m conj(X^m); only source 1 can have m < 0
          if (am & 1) sgn_r = -1.0;
          else sgn_i = -1.0;
        }
      }
      // ladder factors, times nu of the evaluated (rescaled) harmonic (Lp, M)
      const double nu = rec_nu(Lp, M);
      double s1, s2, sz;
      if (isI) {
        s1 = nu * sqrt(double((Lp + M) * (Lp + M - 1)));
        s2 = -nu * sqrt(double((Lp - M) * (Lp - M - 1)));
        sz = -nu * sqrt(double((Lp + M) * (Lp - M)));
      } else {
        s1 = nu * sqrt(double((Lp - M + 2) * (Lp - M + 1)));
        s2 = -nu * sqrt(double((Lp + M + 2) * (Lp + M + 1)));
        sz = nu * sqrt(double((Lp + 1 + M) * (Lp + 1 - M)));
      }
      // d/dx = (s1 c1 + s2 c2) / 2, d/dy = (i / 2)(s1 c1 - s2 c2), d/dz = sz c0;
      // entries of m > 0 count twice (the -m terms)
      const double fac = M > 0 ? 2.0 : 1.0;
      r.s1r = float(0.5 * fac * sgn_r * s1);
      r.s1i = float(0.5 * fac * sgn_i * s1);
      r.s2 = float(0.5 * fac * s2);
      r.sz = float(fac * sz);
      return r;
    };
    for (int M = 0; M <= L + 1; ++M)
      for (int Lp = (M > 1 ? M : 1); Lp <= L + 1; ++Lp) h_ent[eo + idxI(L, Lp, M)] = record(true, Lp, M);
    for (int M = 0; M <= L - 1; ++M)
      for (int Lp = M; Lp <= L - 1; ++Lp) h_ent[eo + nI(L) + idxR(L, Lp, M)] = record(false, Lp, M);
  }
}
struct PrologueInit {
  PrologueInit() { fill_prologue_tables(); }
};
const PrologueInit g_prologue_init;

// CTAs of 64 threads, mom_ppt particles per thread, covering whole scan groups
// of 1024 particles (every tile the scans read is written; past the particles
// the sums are zero)
template <class T, int L> void mom_launch(const MomArgs<T>& a, cudaStream_t s) {
  if (a.n <= 0) return;
  const int ppt = mom_ppt(sizeof(T), a.n);
  const unsigned blocks = unsigned(mom_blocks(a.n, ppt));
  if (ppt == kMomPPT)
    k_moments<T, L, kMomPPT><<<blocks, kMomThreads, moments_smem<T, L, kMomPPT>(), s>>>(a);
  else
    k_moments<T, L, kMomPPTSmall><<<blocks, kMomThreads, moments_smem<T, L, kMomPPTSmall>(), s>>>(a);
}

template <class T, int L> void field_launch(const FieldArgs<T>& a, int wpb, cudaStream_t s) {
  const int64_t ntiles = (a.n + 31) / 32;
  const int64_t blocks = (ntiles + wpb - 1) / wpb;
  const size_t smem = size_t(wpb) * field_smem_per_warp<T>(L);
  if (blocks > 0) k_field<T, L><<<unsigned(blocks), wpb * 32, smem, s>>>(a);
}

template <class T, int L>
void mom_batch_launch(const MomArgs<T>* args, const int2* items, int nitems, int ppt, cudaStream_t s) {
  if (nitems <= 0) return;
  if (ppt == kMomPPT)
    k_moments_batch<T, L, kMomPPT><<<unsigned(nitems), kMomThreads, moments_smem<T, L, kMomPPT>(), s>>>(args, items);
  else
    k_moments_batch<T, L, kMomPPTSmall>
        <<<unsigned(nitems), kMomThreads, moments_smem<T, L, kMomPPTSmall>(), s>>>(args, items);
}

template <class T, int L>
void field_batch_launch(const FieldArgs<T>* args, const int2* items, int nitems, int wpb, cudaStream_t s) {
  const size_t smem = size_t(wpb) * field_smem_per_warp<T>(L);
  if (nitems > 0) k_field_batch<T, L><<<unsigned(nitems), wpb * 32, smem, s>>>(args, items);
}

template <class T, int L> int field_occ(int wpb) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_field<T, L>, wpb * 32,
                                                    size_t(wpb) * field_smem_per_warp<T>(L)) != cudaSuccess)
    return 0;
  return nb;
}

template <class T, int L> cudaError_t set_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_moments<T, L, kMomPPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(moments_smem<T, L, kMomPPT>()));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_moments<T, L, kMomPPTSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(moments_smem<T, L, kMomPPTSmall>()));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_moments_batch<T, L, kMomPPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(moments_smem<T, L, kMomPPT>()));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_moments_batch<T, L, kMomPPTSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(moments_smem<T, L, kMomPPTSmall>()));
  if (e != cudaSuccess) return e;
  const int fmax = int(8 * field_smem_per_warp<T>(L) > 227 * 1024 ? 227 * 1024 : 8 * field_smem_per_warp<T>(L));
  e = cudaFuncSetAttribute(k_field<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, fmax);
  if (e != cudaSuccess) return e;
  // the batched kernel also holds one instance's arguments in static shared memory
  const int bmax = int(227 * 1024 - sizeof(FieldArgs<T>));
  return cudaFuncSetAttribute(k_field_batch<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              fmax < bmax ? fmax : bmax);
}

}  // namespace
}  // namespace imrp

// IMRP_UNIT(name, T, L...) defines register function `name` for the degrees L...
#define IMRP_UNIT(NAME, T, ...)                                                              \
  namespace imrp {                                                                           \
  namespace {                                                                                \
  template <int... Ls> int unit_init(int dev) {                                              \
    static std::mutex mu;                                                                    \
    static bool done[64] = {false};                                                          \
    std::lock_guard<std::mutex> g(mu);                                                       \
    if (dev < 0 || dev >= 64) return -1;                                                     \
    if (done[dev]) return 0;                                                                 \
    Tables<T> t;                                                                             \
    fill_tables(t);                                                                          \
    cudaError_t e = sizeof(T) == 4 ? cudaMemcpyToSymbol(c_tab_f, &t, sizeof(t))              \
                                   : cudaMemcpyToSymbol(c_tab_d, &t, sizeof(t));             \
    if (e != cudaSuccess) return int(e);                                                     \
    e = cudaMemcpyToSymbol(g_ent, h_ent, sizeof(h_ent));                                     \
    if (e != cudaSuccess) return int(e);                                                     \
    e = cudaMemcpyToSymbol(g_comp, h_comp, sizeof(h_comp));                                  \
    if (e != cudaSuccess) return int(e);                                                     \
    cudaError_t es[] = {set_attr<T, Ls>()...};                                               \
    for (cudaError_t x : es)                                                                 \
      if (x != cudaSuccess) return int(x);                                                   \
    done[dev] = true;                                                                        \
    return 0;                                                                                \
  }                                                                                          \
  template <int... Ls> void unit_register(std::vector<KernelSet<T>>& v) {                   \
    KernelSet<T> ks[] = {KernelSet<T>{Ls, &mom_launch<T, Ls>, &field_launch<T, Ls>,         \
                                      &unit_init<Ls...>, field_smem_per_warp<T>(Ls),        \
                                      &field_occ<T, Ls>, &mom_batch_launch<T, Ls>,          \
                                      &field_batch_launch<T, Ls>}...};                      \
    for (auto& k : ks) v.push_back(k);                                                       \
  }                                                                                          \
  }                                                                                          \
  void NAME(std::vector<KernelSet<T>>& v) { unit_register<__VA_ARGS__>(v); }                 \
  }
