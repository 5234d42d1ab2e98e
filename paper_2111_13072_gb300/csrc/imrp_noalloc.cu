// imrp_field_noalloc: the field evaluation of imrp_get_field for callers that
// cannot allocate device memory (see include/imrp.h). All intermediate
// buffers live in one file-scope device array of fixed size; nothing here
// calls cudaMalloc, cudaFree or any other allocating routine.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/imrp.h"
#include "imrp_internal.h"

using namespace imrp;

namespace {

constexpr int64_t kMaxN = IMRP_NOALLOC_MAX_N;
constexpr int kMaxL = IMRP_NOALLOC_MAX_L;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Byte layout of the scratch for n particles, degree L, element size es.
struct Layout {
  size_t part, st[6], id, key0, idx0, key1, idx1, hist, agg, pfx, gagg, gbase, tot, totd, gswork, gsticket, eout,
      step, err, total;
};
constexpr Layout layout(int64_t n, int L, size_t es) {
  Layout o{};
  const int64_t ntiles = (n + 31) / 32;
  const int64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  const int64_t nc = 2 * int64_t(ncomp(L));
  size_t at = 0;
  o.part = at; at += align256(size_t(n) * 8 * es);  // Part<T> records: 8 elements each
  for (int k = 0; k < 6; ++k) { o.st[k] = at; at += align256(size_t(n) * es); }
  o.id = at; at += align256(size_t(n) * 4);
  o.key0 = at; at += align256(size_t(n) * 4);
  o.idx0 = at; at += align256(size_t(n) * 4);
  o.key1 = at; at += align256(size_t(n) * 4);
  o.idx1 = at; at += align256(size_t(n) * 4);
  o.hist = at; at += align256(size_t(sort_hist_words(n)) * 4);
  o.agg = at; at += align256(size_t(nc * tile_stride(ntiles)) * es);
  o.pfx = at; at += align256(size_t(nc * tile_stride(ntiles)) * es);
  o.gagg = at; at += align256(size_t(nc * ngroups) * 8);
  o.gbase = at; at += align256(size_t(nc * ngroups) * es);
  o.tot = at; at += align256(size_t(nc) * es);
  o.totd = at; at += align256(size_t(nc) * 8);
  o.gswork = at; at += align256(size_t(gs_work_doubles(int(nc))) * 8);
  o.gsticket = at; at += align256(size_t(gs_col_blocks(int(nc))) * 4);
  o.eout = at; at += align256(size_t(3 * n) * es);
  o.step = at; at += align256(sizeof(StepState));
  o.err = at; at += align256(sizeof(int));
  o.total = at;
  return o;
}

constexpr size_t kScratchBytes = layout(kMaxN, kMaxL, sizeof(double)).total;

// The scratch: held by every device that loads this library, until exit.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};  // device address of g_scratch, per device
// The table of per-degree kernels is built when the library is loaded, so
// that the entry point itself never allocates (not even host memory).
std::vector<KernelSet<float>> g_f;
std::vector<KernelSet<double>> g_d;
struct Registry {
  Registry() { register_all(g_f, g_d); }
};
const Registry g_registry;

template <class T> const std::vector<KernelSet<T>>& sets();
template <> const std::vector<KernelSet<float>>& sets<float>() { return g_f; }
template <> const std::vector<KernelSet<double>>& sets<double>() { return g_d; }

constexpr double kPi = 3.14159265358979323846;
constexpr double kE = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;

// FP64 [n][3] positions -> particle records, ids 0..n-1, zero velocities; flags positions
// outside 1 < r < r_out or non-finite.
template <class T>
__global__ void k_na_load(const double* __restrict__ x, Part<T>* st, int64_t n, double r_out, int* err) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double a = x[3 * j], b = x[3 * j + 1], c = x[3 * j + 2];
  Part<T> p;
  p.x = T(a); p.y = T(b); p.z = T(c);
  p.vx = T(0); p.vy = T(0); p.vz = T(0);
  p.id = uint32_t(j);
  const double r2 = double(p.x) * double(p.x) + double(p.y) * double(p.y) + double(p.z) * double(p.z);
  if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(err, kErrNaN);
  else if (!(r2 > 1.0 && r2 < r_out * r_out)) atomicOr(err, kErrRange);
  st[j] = p;
}

// Per-call set-up of what must start at zero or at the given step: the step
// state, the error flag and the group scan's tickets (the scratch keeps the
// previous call's contents, and another n or degree lays it out differently).
__global__ void k_na_init(StepState* st, int64_t step, int* err, unsigned* ticket, int nticket) {
  st->step = step;
  st->next = step;
  st->u = 0.0;
  st->kick = 0.0;
  st->sync = 0;
  st->nabs_step = 0;
  st->qs_acc = 0.0;
  st->nabs_total = 0;
  *err = 0;
  for (int k = 0; k < nticket; ++k) ticket[k] = 0u;
}

cudaError_t preload_noalloc_kernels() {
  cudaFuncAttributes fa;
  const void* fns[] = {reinterpret_cast<const void*>(&k_na_load<float>),
                       reinterpret_cast<const void*>(&k_na_load<double>), reinterpret_cast<const void*>(&k_na_init)};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
int run(const imrp_params* p, const double* x, int64_t n, int64_t step, double* E, cudaStream_t s,
        unsigned char* base) {
  const int L = p->l_max;
  const KernelSet<T>* ks = nullptr;
  for (const auto& k : sets<T>())
    if (k.L == L) ks = &k;
  if (!ks) return IMRP_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IMRP_E_CUDA;
  if (ks->init(dev) != 0) return IMRP_E_CUDA;
  const Layout o = layout(n, L, sizeof(T));
  const double R = p->R_D_m;
  const double d = 1.0 - p->R_E_m / R;
  const double r_out = p->R_out_m / R;
  const double n_tilde = double(n) / (4.0 * kPi / 3.0 * (r_out * r_out * r_out - 1.0));
  const int64_t ntiles = (n + 31) / 32;
  const int64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  const int nc = 2 * ncomp(L);
  auto P = [&](size_t off) { return static_cast<void*>(base + off); };
  Part<T>* st0 = static_cast<Part<T>*>(P(o.part));
  T* st1[6];
  for (int k = 0; k < 6; ++k) st1[k] = static_cast<T*>(P(o.st[k]));
  uint32_t* id1 = static_cast<uint32_t*>(P(o.id));
  uint32_t* key0 = static_cast<uint32_t*>(P(o.key0));
  uint32_t* idx0 = static_cast<uint32_t*>(P(o.idx0));
  StepState* st = static_cast<StepState*>(P(o.step));
  int* err = static_cast<int*>(P(o.err));
  k_na_init<<<1, 1, 0, s>>>(st, step, err, static_cast<unsigned*>(P(o.gsticket)), gs_col_blocks(nc));
  k_na_load<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(x, st0, n, r_out, err);
  launch_keys<T>(st0, key0, idx0, n, r_out, s);
  const uint32_t* perm = launch_radix_sort(key0, idx0, static_cast<uint32_t*>(P(o.key1)), static_cast<uint32_t*>(P(o.idx1)),
                    static_cast<uint32_t*>(P(o.hist)), n, sort_first_byte(sizeof(T) == 4 ? 1 : 0), s);
  launch_reorder<T>(st0, st1, id1, perm, n, s);
  MomArgs<T> ma;
  memset(&ma, 0, sizeof(ma));  // all electrons (species = 0)
  ma.x = st1[0]; ma.y = st1[1]; ma.z = st1[2];
  ma.n = n;
  ma.rho = T(r_out);
  ma.rho_inv = T(1.0 / r_out);
  ma.agg = static_cast<T*>(P(o.agg));
  ks->moments(ma, s);
  launch_tile_scan<T>(static_cast<T*>(P(o.agg)), static_cast<T*>(P(o.pfx)), static_cast<double*>(P(o.gagg)),
                      ntiles, nc, s);
  launch_group_scan<T>(static_cast<double*>(P(o.gagg)), static_cast<double*>(P(o.gswork)),
                       static_cast<unsigned*>(P(o.gsticket)), static_cast<T*>(P(o.gbase)),
                       static_cast<T*>(P(o.tot)), static_cast<double*>(P(o.totd)), ngroups, nc, 32, s);
  double canti[kTabL] = {0}, f[kTabL] = {0};
  for (int l = 1; l <= L; ++l) {
    f[l] = coef_f(l, d, p->eps_D);
    canti[l] = coef_canti(l, d, p->eps_D);
  }
  FinalizeArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.st = st;
  fa.totd = static_cast<const double*>(P(o.totd));
  fa.record = 0;
  fa.L = L;
  fa.drive_kind = p->drive_kind;
  fa.inv_ntilde = 1.0 / n_tilde;
  fa.v_hat = p->V_volts * kEps0 / (p->n_e_m3 * kE * R * R);
  fa.sigma = p->width_wpe;
  fa.t0 = p->t0_wpe > 0 ? p->t0_wpe : 4.0 * p->width_wpe;
  fa.dt = p->dt;
  for (int l = 0; l < kTabL; ++l) fa.canti[l] = canti[l];
  launch_finalize(fa, s);
  FieldArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.x = st1[0]; a.y = st1[1]; a.z = st1[2]; a.vx = st1[3]; a.vy = st1[4]; a.vz = st1[5];
  a.id = id1;
  a.key = key0;
  a.kidx = idx0;
  a.n = n;
  a.pfx = static_cast<const T*>(P(o.pfx));
  a.gbase = static_cast<const T*>(P(o.gbase));
  a.tot = static_cast<const T*>(P(o.tot));
  a.agg = static_cast<const T*>(P(o.agg));
  a.img_in_tile = img_in_tile_for<T>(n);
  a.st = st;
  a.Eout = static_cast<T*>(P(o.eout));
  a.err = err;
  a.mode = 1;
  a.L = L;
  a.rho = T(r_out);
  a.rho_inv = T(1.0 / r_out);
  a.pf = 1.0 / (4.0 * kPi * n_tilde);
  a.ion_coef = double(n) / (r_out * r_out * r_out - 1.0);
  a.q_s = p->q_s;
  a.r_out2 = r_out * r_out;
  a.rk = make_radius_key(r_out);
  a.dt = T(p->dt);
  a.r_out = T(r_out);
  a.wall_rule = p->wall_rule;
  a.nabs = nullptr;  // field only: nothing is pushed or absorbed
  a.sigma_v = 0.0;
  a.self_image = p->self_image;
  a.seed = p->seed;
  double rl = 1.0;
  for (int l = 0; l < kTabL; ++l) {
    a.f[l] = T(f[l]);
    a.rhol[l] = T(rl);
    rl *= r_out;
    a.cdrive[l] = canti[l] * 4.0 * kPi * n_tilde;
  }
  const size_t spw = ks->smem_per_warp;
  const int wpb = int(spw * 8 <= 227 * 1024 ? 8 : (227 * 1024) / spw);
  ks->field(a, wpb, s);
  const T* eo = static_cast<const T*>(P(o.eout));
  const T* cs[3] = {eo, eo + n, eo + 2 * n};
  launch_scatter_by_id<T>(cs, 3, id1, E, n, s);
  if (cudaGetLastError() != cudaSuccess) return IMRP_E_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return IMRP_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return IMRP_E_CUDA;
  if (h & kErrNaN) return IMRP_E_NAN;
  if (h & kErrRange) return IMRP_E_INVAL;
  return IMRP_OK;
}

}  // namespace

extern "C" int imrp_field_noalloc(const imrp_params* p, const double* x_dev, int64_t n, int64_t step,
                                  double* E_dev, void* stream) {
  if (!p || !x_dev || !E_dev) return IMRP_E_INVAL;
  if (n < 1 || n > kMaxN) return IMRP_E_INVAL;
  if (p->l_max < 1 || p->l_max > kMaxL || p->m0_only != 0) return IMRP_E_INVAL;
  if (p->precision != 0 && p->precision != 1) return IMRP_E_INVAL;
  if (!(p->R_D_m > 0 && p->R_E_m > 0 && p->R_E_m < p->R_D_m && p->R_out_m > p->R_D_m)) return IMRP_E_INVAL;
  if (!(p->eps_D >= 1.0) || !(p->n_e_m3 > 0) || !(p->dt > 0)) return IMRP_E_INVAL;
  if (p->drive_kind < 0 || p->drive_kind > 2 || (p->drive_kind == 0 && !(p->width_wpe > 0))) return IMRP_E_INVAL;
  if (step < 0) return IMRP_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return IMRP_E_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
      // Set-up, once per device: CUDA loads device code lazily, and loading a
      // module reserves device memory (its code and its static arrays, this
      // file's scratch included). So every kernel that a call may launch, in
      // both precisions and at every degree up to the limit, is loaded here,
      // with its tables filled, and later calls load nothing.
      if (preload_core_kernels() != cudaSuccess || preload_noalloc_kernels() != cudaSuccess)
        return IMRP_E_CUDA;
      for (const auto& k : g_f)
        if (k.L <= kMaxL && k.init(dev) != 0) return IMRP_E_CUDA;
      for (const auto& k : g_d)
        if (k.L <= kMaxL && k.init(dev) != 0) return IMRP_E_CUDA;
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return IMRP_E_CUDA;
      g_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return p->precision == 1 ? run<float>(p, x_dev, n, step, E_dev, s, base)
                           : run<double>(p, x_dev, n, step, E_dev, s, base);
}
