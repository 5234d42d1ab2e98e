// Internal interfaces between the host API (imrp_api.cu), the generic kernels
// (imrp_core.cu) and the per-degree instantiation units (imrp_inst_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "imrp_device.cuh"

namespace imrp {

// ---- coefficients (host; written from App. A and Sec. 3 with R = 1) ---------
// f_l of the radial Green's function R^(p,p)_l (App. A).
inline double coef_f(int l, double d, double eps) {
  const double x = pow(1.0 - d, 2 * l + 1);
  return (l * (eps - 1.0) + (l + eps + l * eps) * x) / ((l + 1 + l * eps) + (l + 1) * (eps - 1.0) * x);
}
// b^P_l of the characteristic function outside the dielectric (Sec. 3).
inline double coef_bP(int l, double d, double eps) {
  const double den = (l + 1) * (eps - 1.0) * pow(1.0 - d, 2 * l + 1) + l * eps + l + 1;
  return (2 * l + 1) * eps * pow(1.0 - d, l + 1) / den;
}
// c_l' of Sec. 3 for odd degree l = 2l'-1: (-1/2)^{l'+1} (4l'-1) (2l'-3)!! / l'!
inline double coef_cprime(int lp) {
  double df = 1.0;
  for (int k = 2 * lp - 3; k > 1; k -= 2) df *= k;
  double fact = 1.0;
  for (int k = 2; k <= lp; ++k) fact *= k;
  const double sgn = ((lp + 1) % 2 == 0) ? 1.0 : -1.0;
  return sgn * pow(0.5, lp + 1) * (4.0 * lp - 1.0) * df / fact;
}
// Coefficient of r^{-(l+1)} P_l(cos t) in Psi_anti for r >= R (Sec. 3): c_l' b^P_l
// for odd l = 2l'-1, zero for even l.
inline double coef_canti(int l, double d, double eps) {
  return (l % 2 == 1) ? coef_cprime((l + 1) / 2) * coef_bP(l, d, eps) : 0.0;
}

// ---- radix sort (imrp_core.cu) ---------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per CTA
constexpr int64_t sort_blocks(int64_t n) { return (n + kSortTile - 1) / kSortTile; }
// Words of the sort's histogram buffer for n keys: block counts of up to 512
// digits per block, and the digit totals.
constexpr int64_t sort_hist_words(int64_t n) { return 512 * sort_blocks(n) + 512; }
// Sorts (key, val) pairs by the key bytes first_byte..3 (stable radix sort;
// keys equal in those bytes keep their order). k0/v0 hold the input; k1/v1 are
// scratch of n; hist: sort_hist_words(n) words. Returns the buffer that holds
// the sorted values (v0 after an even number of passes, v1 after an odd one).
// Key bytes sorted: all four, in both precisions. The radius key is
// floor((r^2 - 1) / (r_out^2 - 1) * 2^32) of the exact FP64 r^2 of the stored
// position, and the sorted index j of a particle is its count of electrons
// inside (the l = 0 term), which jumps by one electron per misordered pair;
// so even radii that FP32 arithmetic cannot tell apart are ordered exactly.
inline int sort_first_byte(int) { return 0; }
const uint32_t* launch_radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist,
                                  int64_t n, int first_byte, cudaStream_t s,
                                  bool shared_gpu = false);

// ---- state movement and keys (imrp_core.cu) ---------------------------------
// The state is an array of Part<T> records in the order of the last push (or
// load); each step gathers it into radius order as component arrays.
template <class T>
void launch_reorder(const Part<T>* src, T* const* dst, uint32_t* id_dst, const uint32_t* perm, int64_t n,
                    cudaStream_t s);
template <class T>
void launch_keys(const Part<T>* st, uint32_t* key, uint32_t* kidx, int64_t n, double r_out, cudaStream_t s);
template <class T>
void launch_load(const double* x /* [n][3] */, const double* v /* [n][3] */, const uint32_t* ids /* or null */,
                 Part<T>* st, uint32_t* key, uint32_t* kidx, int64_t n, double r_out, int* err, cudaStream_t s);
// The state in its storage order: x[j][3], v[j][3], id[j] (checkpoint).
template <class T>
void launch_state_dump(const Part<T>* st, double* x, double* v, uint32_t* id, int64_t n, cudaStream_t s);
// out[id[j]][c] = comp_c[j] for c < ncomp
template <class T>
void launch_scatter_by_id(const T* const* comps, int ncomp, const uint32_t* id, double* out,
                          int64_t n, cudaStream_t s);
// the state in id order: x[n][3], v[n][3] (FP64)
template <class T>
void launch_state_out(const Part<T>* st, double* x, double* v, int64_t n, cudaStream_t s);

// ---- scans (imrp_core.cu) ---------------------------------------------------
// in-group scans of agg[u][tile] (row stride tile_stride(ntiles)) into
// pfx[tile][u] (tile-major: one tile's nc carries contiguous), group totals
// into gagg[g][u] (FP64)
template <class T>
void launch_tile_scan(const T* agg, T* pfx, double* gagg, int64_t ntiles, int nc, cudaStream_t s);
// group scan over gagg:
// gseg: least number of groups per segment (16, 32 or 64; chosen by the
// autotuner). work: gs_work_doubles(nc) doubles; ticket: gs_col_blocks(nc)
// counters, zero before the first call (each call leaves them zero).
template <class T>
void launch_group_scan(const double* gagg, double* work, unsigned* ticket, T* gbase, T* tot, double* totd,
                       int64_t ngroups, int nc, int gseg, cudaStream_t s);

struct FinalizeArgs {
  StepState* st;
  const double* totd;
  double* qhist;     // qhist[n - first] holds Q_diff of step n (first: step of the load or restore)
  double* uhist;
  int64_t cap;
  int64_t first;
  int record;
  int L;
  int drive_kind;
  double inv_ntilde;
  double v_hat, sigma, t0, dt;
  double canti[kTabL];
};
void launch_finalize(const FinalizeArgs& a, cudaStream_t s);
// Loads the device code of every degree-independent kernel of both precisions
// (CUDA loads modules lazily, at a kernel's first launch or query, and the
// load reserves device memory): the allocation-free entry point calls it at
// its set-up so that later calls load nothing.
cudaError_t preload_core_kernels();
// opt-in shared memory of the sort's bucket kernel (once per device, before
// the first sort)
cudaError_t set_sort_attributes();
void launch_init_step(StepState* st, cudaStream_t s);

// Spectrum sums: Qh[j] = dt sum_n (q_n - q_0) e^{-i w_j t_n},
// Uh[j] = sum_n kw_n u_n e^{-i w_j t_n}, w_j = (j+1) w_max / nf; out [nf][4].
void launch_dft(const double* q, const double* u, int64_t ns, double dt, double first_kick,
                int64_t nf, double w_max, double* out, cudaStream_t s);

// ---- per-degree kernels (imrp_inst_*.cu) ------------------------------------
// SMs of the current device (cached per device; contexts may be created from
// several host threads, hence the atomics)
inline int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int c = cache[dev].load(std::memory_order_relaxed);
  if (c == 0) {
    int v = 0;
    c = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0 ? v : 152;
    cache[dev].store(c, std::memory_order_relaxed);
  }
  return c;
}
// Particles per thread of the moments kernel for an instance of n particles:
// 16 (1024 per CTA of 64 threads), or 4 (256 per CTA) for an FP64 instance
// that would give fewer than two CTAs per SM. FP64 runs at a small fraction
// of the FP32 rate here, so a small FP64 instance gains from four times the
// SMs (N = 2e4, l_max = 8: 0.292 -> 0.103 ms); in FP32 the wider reduction
// over each tile's threads costs more than the SMs bring (N = 1e5, l_max =
// 16: 0.045 -> 0.068 ms), so FP32 keeps 16.
inline int mom_ppt(int elem_size, int64_t n) {
  return (elem_size == 8 && (n + 1023) / 1024 < 2 * sm_count()) ? 4 : 16;
}
// CTAs of the moments kernel (64 threads of ppt particles): whole scan groups
// of 1024 particles, so that every tile the scans read is written
inline int64_t mom_blocks(int64_t n, int ppt) { return (n + 1023) / 1024 * (16 / ppt); }

template <class T> struct KernelSet {
  int L;
  void (*moments)(const MomArgs<T>&, cudaStream_t);
  void (*field)(const FieldArgs<T>&, int wpb, cudaStream_t);
  int (*init)(int device);  // tables + attributes, once per device
  size_t smem_per_warp;
  int (*field_blocks_per_sm)(int wpb);  // occupancy of the field kernel at wpb warps per CTA
  // Batched launches over several instances of this degree and precision:
  // args[i] in device memory, items[b] = (instance, block) for the moments
  // (blocks of 64 ppt particles, ppt = mom_ppt of every listed instance) and
  // (instance, first tile) for the field (CTAs of wpb tiles).
  void (*moments_batch)(const MomArgs<T>* args, const int2* items, int nitems, int ppt, cudaStream_t);
  void (*field_batch)(const FieldArgs<T>* args, const int2* items, int nitems, int wpb, cudaStream_t);
};
void register_all(std::vector<KernelSet<float>>& f, std::vector<KernelSet<double>>& d);

}  // namespace imrp
