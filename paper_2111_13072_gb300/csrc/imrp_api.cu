// Host side of the C ABI declared in include/imrp.h: parameter derivation
// (Sec. 4 units), device memory, the per-step launch sequence, CUDA graphs of
// step pairs, and the spectrum post-processing (Sec. 4).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/imrp.h"
#include "imrp_internal.h"

using namespace imrp;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kE = 1.602176634e-19;     // C
constexpr double kEps0 = 8.8541878128e-12; // F/m
constexpr double kMe = 9.1093837015e-31;   // kg

std::once_flag g_reg_once;
std::vector<KernelSet<float>> g_ks_f;
std::vector<KernelSet<double>> g_ks_d;

void ensure_registry() {
  std::call_once(g_reg_once, [] { register_all(g_ks_f, g_ks_d); });
}

template <class T> const KernelSet<T>* find_set(int L);
template <> const KernelSet<float>* find_set<float>(int L) {
  for (auto& k : g_ks_f) if (k.L == L) return &k;
  return nullptr;
}
template <> const KernelSet<double>* find_set<double>(int L) {
  for (auto& k : g_ks_d) if (k.L == L) return &k;
  return nullptr;
}

// Collision threshold: a step's collision probability 1 - exp(-nu dt) in
// units of 2^-24 (compared with the top 24 bits of a Philox word).
uint32_t coll_threshold(double nu, double dt) {
  if (!(nu > 0.0)) return 0u;
  return uint32_t(floor((1.0 - exp(-nu * dt)) * 16777216.0));
}

}  // namespace

struct imrp_ctx {
  imrp_params p{};
  std::string err;
  int device = 0;
  int L = 8;
  int prec = 0;  // 0 fp64, 1 mixed (fp32)
  // derived
  double d = 0, r_out = 0, v_hat = 0, lambda_D = 0, omega_pe = 0, t0 = 0;
  double n_tilde = 0, n_ion = 0;
  double f[kTabL] = {0}, canti[kTabL] = {0};
  int64_t cap = 0, n = 0;
  int64_t host_step = 0;
  int64_t hist_first = 0;     // step of the last load (0) or restore: qhist[k] is Q_diff of step hist_first + k
  uint64_t gen = 0;           // configuration generation: bumped whenever the captured graphs are dropped
  bool loaded = false, keys_valid = false;
  int nc = 0;
  int64_t ntiles = 0, ngroups = 0;
  int wpb = 8;
  int gseg = 32;  // least groups per segment of the group scan
  // streams / graphs
  cudaStream_t own_stream = nullptr, stream = nullptr;
  cudaGraphExec_t graph2 = nullptr;  // two steps
  cudaGraphExec_t graph1 = nullptr;  // one step
  int graph_cur = -1;
  // device memory
  void* state = nullptr;      // Part<T>[N]: the particles in the order of the last push (or load)
  void* srt[6] = {nullptr};   // x, y, z, vx, vy, vz in radius order (rebuilt every step)
  uint32_t* srt_id = nullptr; // their ids
  int cur = 0;                // stays 0: one state buffer (checked by the captured graphs)
  uint32_t *key0 = nullptr, *idx0 = nullptr, *key1 = nullptr, *idx1 = nullptr, *hist = nullptr;
  void *agg = nullptr, *pfx = nullptr, *gbase = nullptr, *tot = nullptr, *eout = nullptr;
  double *gagg = nullptr, *totd = nullptr, *gswork = nullptr;
  unsigned* gsticket = nullptr;
  double *qhist = nullptr, *uhist = nullptr;
  int64_t hcap = 0;
  double* stage = nullptr;  // [cap][6] FP64 staging for load / readback
  // streamed loads: two staging buffers filled on the copy stream (allocated on first use)
  double* astage[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  int next_stage = 0;
  StepState* st = nullptr;
  int* derr = nullptr;
  double* dft = nullptr;
  int64_t dft_cap = 0;
  // radial ion profile (App. D) in place of the uniform background
  double* ion_q = nullptr;    // device copy, units e n_inf R^3
  int64_t ion_n = 0;
  int64_t ion_cap = 0;
  double ion_qe = 0.0;        // electron charge the loaded particles represent
  double ion_qs = 0.0;        // surface charge, units e n_inf R^3
  // mobile ions (imrp_set_species): ids >= sp_ne are ions of charge sp_q (e) and mass sp_m (m_e)
  int species = 0;
  int64_t sp_ne = 0;
  double sp_q = 0.0, sp_m = 0.0, sp_bg = 0.0;  // sp_bg: ions of the immobile uniform background
  double *qtile = nullptr, *qpfx = nullptr, *qgagg = nullptr, *qgbase = nullptr, *qtot = nullptr,
         *qtotd = nullptr, *qwork = nullptr;
  unsigned* qticket = nullptr;

  int fail(int code, const char* fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof(b), fmt, ap);
    va_end(ap);
    err = b;
    return code;
  }
};

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ctx->fail(IMRP_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                       __FILE__, __LINE__);                                             \
  } while (0)

namespace {

template <class T> T** sorted_ptrs(imrp_ctx* c) { return reinterpret_cast<T**>(c->srt); }
template <class T> Part<T>* state_of(imrp_ctx* c) { return static_cast<Part<T>*>(c->state); }

// The captured step graphs hold the field arguments, buffer pointers and
// launch shapes; any change of those drops them.
void drop_graphs(imrp_ctx* c) {
  if (c->graph2) cudaGraphExecDestroy(c->graph2);
  if (c->graph1) cudaGraphExecDestroy(c->graph1);
  c->graph2 = c->graph1 = nullptr;
  ++c->gen;  // batches that captured this context recapture too
}

// Super-particles per unit cube at density n_inf: N over the shell volume
// for the uniform start, N over the electron charge of the given profile.
double n_tilde_of(const imrp_ctx* c, int64_t n) {
  const int64_t ne = c->species ? std::min<int64_t>(c->sp_ne, n) : n;  // electron super-particles
  if (c->ion_n) return double(ne) / c->ion_qe;
  return double(ne) / (4.0 * kPi / 3.0 * (c->r_out * c->r_out * c->r_out - 1.0));
}
// Ion super-particles of the immobile uniform background after a load of n.
double n_ion_of(const imrp_ctx* c, int64_t n) { return c->species ? c->sp_bg : double(n); }

void free_all(imrp_ctx* c) {
  drop_graphs(c);
  cudaFree(c->state);
  c->state = nullptr;
  for (int k = 0; k < 6; ++k) { cudaFree(c->srt[k]); c->srt[k] = nullptr; }
  cudaFree(c->srt_id);
  c->srt_id = nullptr;
  void* ps[] = {c->key0, c->idx0, c->key1, c->idx1, c->hist, c->agg, c->pfx, c->gbase, c->tot,
                c->eout, c->gagg, c->totd, c->gswork, c->gsticket, c->qhist, c->uhist, c->stage, c->st,
                c->derr, c->dft};
  for (void* p : ps) cudaFree(p);
  cudaFree(c->ion_q);
  c->ion_q = nullptr;
  {
    void* qs[] = {c->qtile, c->qpfx, c->qgagg, c->qgbase, c->qtot, c->qtotd, c->qwork, c->qticket};
    for (void* q : qs) cudaFree(q);
    c->qtile = c->qpfx = c->qgagg = c->qgbase = c->qtot = c->qtotd = c->qwork = nullptr;
    c->qticket = nullptr;
  }
  c->ion_n = c->ion_cap = 0;
  c->key0 = c->idx0 = c->key1 = c->idx1 = c->hist = nullptr;
  c->agg = c->pfx = c->gbase = c->tot = c->eout = nullptr;
  c->gagg = c->totd = c->gswork = c->qhist = c->uhist = c->stage = c->dft = nullptr;
  c->gsticket = nullptr;
  c->st = nullptr;
  c->derr = nullptr;
  for (int k = 0; k < 2; ++k) {
    cudaFree(c->astage[k]);
    c->astage[k] = nullptr;
    if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
    if (c->ev_free[k]) cudaEventDestroy(c->ev_free[k]);
    c->ev_copied[k] = c->ev_free[k] = nullptr;
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_stream = nullptr;
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  c->own_stream = nullptr;
}

int check_err(imrp_ctx* ctx) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) {
    CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->stream));
    if (h & kErrNaN) return ctx->fail(IMRP_E_NAN, "non-finite value in the particle state");
    if (h & kErrRange) return ctx->fail(IMRP_E_INVAL, "a particle lies outside 1 < r < r_out");
  }
  return IMRP_OK;
}

int grow_history(imrp_ctx* ctx, int64_t need) {
  if (need <= ctx->hcap) return IMRP_OK;
  int64_t ncap = std::max<int64_t>(need, std::max<int64_t>(2 * ctx->hcap, 4096));
  double *q = nullptr, *u = nullptr;
  CK(cudaMalloc(&q, ncap * sizeof(double)));
  CK(cudaMalloc(&u, ncap * sizeof(double)));
  if (ctx->hcap) {
    CK(cudaMemcpyAsync(q, ctx->qhist, ctx->hcap * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(u, ctx->uhist, ctx->hcap * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  cudaFree(ctx->qhist);
  cudaFree(ctx->uhist);
  ctx->qhist = q;
  ctx->uhist = u;
  ctx->hcap = ncap;
  drop_graphs(ctx);
  return IMRP_OK;
}

// Arguments of the moments kernel of a context (its sorted arrays).
template <class T> MomArgs<T> make_mom_args(imrp_ctx* ctx) {
  T** S = sorted_ptrs<T>(ctx);
  MomArgs<T> ma;
  memset(&ma, 0, sizeof(ma));
  ma.x = S[0]; ma.y = S[1]; ma.z = S[2];
  ma.n = ctx->n;
  ma.rho = T(ctx->r_out);
  ma.rho_inv = T(1.0 / ctx->r_out);
  ma.agg = static_cast<T*>(ctx->agg);
  ma.species = ctx->species;
  ma.n_e = uint32_t(std::min<int64_t>(ctx->sp_ne, int64_t(UINT32_MAX)));
  ma.q_ion = T(ctx->sp_q);
  ma.id = ctx->srt_id;
  ma.qtile = ctx->qtile;
  return ma;
}

// Arguments of the field kernel of a context: push (record) or field only.
template <class T> FieldArgs<T> make_field_args(imrp_ctx* ctx, bool record) {
  T** S = sorted_ptrs<T>(ctx);
  const int64_t n = ctx->n;
  FieldArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.x = S[0]; a.y = S[1]; a.z = S[2]; a.vx = S[3]; a.vy = S[4]; a.vz = S[5];
  a.id = ctx->srt_id;
  a.out = state_of<T>(ctx);
  a.key = ctx->key0;
  a.kidx = ctx->idx0;
  a.n = n;
  a.pfx = static_cast<const T*>(ctx->pfx);
  a.gbase = static_cast<const T*>(ctx->gbase);
  a.tot = static_cast<const T*>(ctx->tot);
  a.agg = static_cast<const T*>(ctx->agg);
  a.img_in_tile = img_in_tile_for<T>(n);
  a.st = ctx->st;
  a.Eout = static_cast<T*>(ctx->eout);
  a.err = ctx->derr;
  a.mode = record ? 0 : 1;
  a.L = ctx->L;
  a.rho = T(ctx->r_out);
  a.rho_inv = T(1.0 / ctx->r_out);
  a.pf = 1.0 / (4.0 * kPi * ctx->n_tilde);
  a.ion_coef = ctx->n_ion / (ctx->r_out * ctx->r_out * ctx->r_out - 1.0);
  a.ion_q = ctx->ion_n ? ctx->ion_q : nullptr;
  a.ion_n = int(ctx->ion_n);
  a.ion_inv_h = ctx->ion_n ? double(ctx->ion_n - 1) / (ctx->r_out - 1.0) : 0.0;
  a.ion_scale = ctx->n_tilde;
  a.q_s = ctx->ion_n ? ctx->ion_qs * ctx->n_tilde : ctx->p.q_s;
  a.r_out2 = ctx->r_out * ctx->r_out;
  a.rk = make_radius_key(ctx->r_out);
  a.dt = T(ctx->p.dt);
  a.r_out = T(ctx->r_out);
  a.wall_rule = ctx->p.wall_rule;
  a.nabs = &ctx->st->nabs_step;
  a.sigma_v = ctx->lambda_D;
  a.self_image = ctx->p.self_image;
  a.m0_only = ctx->p.m0_only;
  a.species = ctx->species;
  a.n_e = uint32_t(std::min<int64_t>(ctx->sp_ne, int64_t(UINT32_MAX)));
  a.q_ion = T(ctx->sp_q);
  a.qm_ion = T(ctx->species ? ctx->sp_q / ctx->sp_m : 0.0);
  a.qpfx = ctx->qpfx;
  a.qgbase = ctx->qgbase;
  a.coll_thr = coll_threshold(ctx->p.nu_coll, ctx->p.dt);
  a.seed = ctx->p.seed;
  double rl = 1.0;
  for (int l = 0; l < kTabL; ++l) {
    a.f[l] = T(ctx->f[l]);
    a.rhol[l] = T(rl);
    rl *= ctx->r_out;
    a.cdrive[l] = ctx->canti[l] * 4.0 * kPi * ctx->n_tilde;
  }
  return a;
}

// The stages of one step (or field evaluation) of a context: radius keys (if
// stale), sort and reorder; then the moments; then the scans and finalize;
// then the field. The batch runs the moments and the field of many contexts
// as one launch each (per degree and precision) between the others.
template <class T> void enqueue_pre(imrp_ctx* ctx, cudaEvent_t* ev = nullptr, bool shared_gpu = false) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  Part<T>* st = state_of<T>(ctx);
  if (!ctx->keys_valid) {
    launch_keys<T>(st, ctx->key0, ctx->idx0, n, ctx->r_out, s);
  }
  if (ev) cudaEventRecord(ev[0], s);
  const uint32_t* perm = launch_radix_sort(ctx->key0, ctx->idx0, ctx->key1, ctx->idx1, ctx->hist, n,
                                           sort_first_byte(ctx->prec), s, shared_gpu);
  if (ev) cudaEventRecord(ev[1], s);
  launch_reorder<T>(st, sorted_ptrs<T>(ctx), ctx->srt_id, perm, n, s);
}

template <class T> void enqueue_mid(imrp_ctx* ctx, bool record) {
  cudaStream_t s = ctx->stream;
  if (ctx->species) {
    // the charge inside each particle's radius: a scan of the tiles' charges (FP64)
    launch_tile_scan<double>(ctx->qtile, ctx->qpfx, ctx->qgagg, ctx->ntiles, 1, s);
    launch_group_scan<double>(ctx->qgagg, ctx->qwork, ctx->qticket, ctx->qgbase, ctx->qtot, ctx->qtotd,
                              ctx->ngroups, 1, ctx->gseg, s);
  }
  launch_tile_scan<T>(static_cast<T*>(ctx->agg), static_cast<T*>(ctx->pfx), ctx->gagg, ctx->ntiles, ctx->nc, s);
  launch_group_scan<T>(ctx->gagg, ctx->gswork, ctx->gsticket, static_cast<T*>(ctx->gbase),
                       static_cast<T*>(ctx->tot), ctx->totd, ctx->ngroups, ctx->nc, ctx->gseg, s);
  FinalizeArgs fa;
  fa.st = ctx->st;
  fa.totd = ctx->totd;
  fa.qhist = ctx->qhist;
  fa.uhist = ctx->uhist;
  fa.cap = ctx->hcap;
  fa.first = ctx->hist_first;
  fa.record = record ? 1 : 0;
  fa.L = ctx->L;
  fa.drive_kind = ctx->p.drive_kind;
  fa.inv_ntilde = 1.0 / ctx->n_tilde;
  fa.v_hat = ctx->v_hat;
  fa.sigma = ctx->p.width_wpe;
  fa.t0 = ctx->t0;
  fa.dt = ctx->p.dt;
  for (int l = 0; l < kTabL; ++l) fa.canti[l] = ctx->canti[l];
  launch_finalize(fa, s);
}

// Launches one step (record = 1) or the field evaluation without push (record = 0).
// ev (optional): IMRP_N_STAGES + 1 events recorded at the stage boundaries.
template <class T> int enqueue(imrp_ctx* ctx, bool record, cudaEvent_t* ev = nullptr) {
  const KernelSet<T>* ks = find_set<T>(ctx->L);
  cudaStream_t s = ctx->stream;
  enqueue_pre<T>(ctx, ev);
  if (ev) cudaEventRecord(ev[2], s);
  ks->moments(make_mom_args<T>(ctx), s);
  if (ev) cudaEventRecord(ev[3], s);
  enqueue_mid<T>(ctx, record);
  if (ev) cudaEventRecord(ev[4], s);
  ks->field(make_field_args<T>(ctx, record), ctx->wpb, s);
  if (ev) cudaEventRecord(ev[5], s);
  // the field kernel wrote fresh keys for the (now sorted) state in push mode
  ctx->keys_valid = record;
  return IMRP_OK;
}

int enqueue_any(imrp_ctx* ctx, bool record, cudaEvent_t* ev = nullptr) {
  return ctx->prec == 1 ? enqueue<float>(ctx, record, ev) : enqueue<double>(ctx, record, ev);
}

// Captures `count` steps (1 or 2) of the current configuration into *out.
int capture_steps(imrp_ctx* ctx, int count, cudaGraphExec_t* out) {
  const int cur0 = ctx->cur;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  int r = 0;
  for (int k = 0; k < count && !r; ++k) r = enqueue_any(ctx, true);
  cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
  if (r) { if (g) cudaGraphDestroy(g); return r; }
  if (ec != cudaSuccess) return ctx->fail(IMRP_E_CUDA, "graph capture: %s", cudaGetErrorString(ec));
  ec = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ec != cudaSuccess) return ctx->fail(IMRP_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
  ctx->cur = cur0;  // capture did not execute anything
  return IMRP_OK;
}

int launch_steps(imrp_ctx* ctx, int64_t nsteps) {
  int rc = grow_history(ctx, ctx->host_step - ctx->hist_first + nsteps + 1);
  if (rc) return rc;
  int64_t done = 0;
  // keys must be valid before a captured step (it assumes that the push or
  // the load wrote them)
  while (done < nsteps && !ctx->keys_valid) {
    rc = enqueue_any(ctx, true);
    if (rc) return rc;
    CK(cudaGetLastError());
    ++done;
  }
  if (done < nsteps && ctx->graph_cur != ctx->cur) drop_graphs(ctx);
  // pairs, then a single step for an odd remainder (one captured graph each)
  while (done < nsteps) {
    const int k = nsteps - done >= 2 ? 2 : 1;
    cudaGraphExec_t& ge = k == 2 ? ctx->graph2 : ctx->graph1;
    if (!ge) {
      rc = capture_steps(ctx, k, &ge);
      if (rc) return rc;
      ctx->graph_cur = ctx->cur;
    }
    CK(cudaGraphLaunch(ge, ctx->stream));
    done += k;
  }
  CK(cudaGetLastError());
  ctx->host_step += nsteps;
  return IMRP_OK;
}

// Device bytes that alloc_ctx requests for N particles at degree L (before
// the Q_diff history, which grows with the steps taken).
size_t footprint_bytes(int64_t N, int L, int prec) {
  const size_t es = prec == 1 ? sizeof(float) : sizeof(double);
  const int64_t ntiles = (N + 31) / 32;
  const int64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  const int64_t nc = 2 * int64_t(ncomp(L));
  size_t b = 0;
  b += N * (es == 4 ? sizeof(Part<float>) : sizeof(Part<double>));  // state records
  b += 6 * N * es + N * 4;                          // radius-ordered copy + ids
  b += 4 * size_t(N) * 4;                           // keys and slots
  b += size_t(sort_hist_words(N)) * 4;              // histogram
  b += 2 * size_t(tile_stride(ntiles) * nc) * es;   // tile sums and in-group scans
  b += size_t(ngroups * nc) * (es + 8) + size_t(nc) * (es + 8);
  b += size_t(gs_work_doubles(int(nc))) * 8 + size_t(gs_col_blocks(int(nc))) * 4;
  b += 3 * size_t(N) * es + 6 * size_t(N) * 8;      // field output, staging
  b += sizeof(StepState) + sizeof(int);
  return b;
}

int alloc_ctx(imrp_ctx* ctx) {
  const int64_t N = ctx->p.N;
  const size_t es = ctx->prec == 1 ? sizeof(float) : sizeof(double);
  const int64_t ntiles = (N + 31) / 32;
  const int64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  const int nc = 2 * ncomp(ctx->L);
  CK(cudaMalloc(&ctx->state, N * (ctx->prec == 1 ? sizeof(Part<float>) : sizeof(Part<double>))));
  for (int k = 0; k < 6; ++k) CK(cudaMalloc(&ctx->srt[k], N * es));
  CK(cudaMalloc(&ctx->srt_id, N * sizeof(uint32_t)));
  CK(cudaMalloc(&ctx->key0, N * sizeof(uint32_t)));
  CK(cudaMalloc(&ctx->idx0, N * sizeof(uint32_t)));
  CK(cudaMalloc(&ctx->key1, N * sizeof(uint32_t)));
  CK(cudaMalloc(&ctx->idx1, N * sizeof(uint32_t)));
  CK(cudaMalloc(&ctx->hist, size_t(sort_hist_words(N)) * sizeof(uint32_t)));
  CK(cudaMalloc(&ctx->agg, tile_stride(ntiles) * nc * es));
  CK(cudaMalloc(&ctx->pfx, tile_stride(ntiles) * nc * es));
  CK(cudaMalloc(&ctx->gbase, ngroups * nc * es));
  CK(cudaMalloc(&ctx->tot, nc * es));
  CK(cudaMalloc(&ctx->gagg, ngroups * nc * sizeof(double)));
  CK(cudaMalloc(&ctx->totd, nc * sizeof(double)));
  CK(cudaMalloc(&ctx->gswork, gs_work_doubles(nc) * sizeof(double)));
  CK(cudaMalloc(&ctx->gsticket, gs_col_blocks(nc) * sizeof(unsigned)));
  CK(cudaMemset(ctx->gsticket, 0, gs_col_blocks(nc) * sizeof(unsigned)));
  CK(cudaMalloc(&ctx->eout, 3 * N * es));
  CK(cudaMalloc(&ctx->stage, 6 * N * sizeof(double)));
  CK(cudaMalloc(&ctx->st, sizeof(StepState)));
  CK(cudaMalloc(&ctx->derr, sizeof(int)));
  CK(cudaMemset(ctx->derr, 0, sizeof(int)));
  return IMRP_OK;
}

}  // namespace

extern "C" {

int imrp_footprint(const imrp_params* p, int64_t n_steps, size_t* bytes) {
  if (!p || !bytes || p->N < 1 || n_steps < 0) return IMRP_E_INVAL;
  if (p->precision != 0 && p->precision != 1) return IMRP_E_INVAL;
  if (p->l_max < 1 || p->l_max >= kTabL - 2) return IMRP_E_INVAL;
  *bytes = footprint_bytes(p->N, p->l_max, p->precision) + size_t(2 * std::max<int64_t>(n_steps + 1, 4096)) * 8;
  return IMRP_OK;
}

void imrp_default_params(imrp_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->R_E_m = 4e-3;
  p->R_D_m = 5e-3;
  p->eps_D = 4.0;
  p->n_e_m3 = 1e15;
  p->T_e_eV = 2.0;
  const double lam = sqrt(kEps0 * p->T_e_eV / (p->n_e_m3 * kE));
  p->R_out_m = p->R_D_m + 20.0 * lam;
  p->N = 20000;
  p->l_max = 8;
  p->m0_only = 0;
  p->dt = 0.05;
  p->drive_kind = 0;
  p->wall_rule = 0;
  p->V_volts = 1.0;
  p->width_wpe = 2.0;
  p->t0_wpe = 0.0;
  p->self_image = 0;
  p->precision = 0;
  p->seed = 0;
  p->q_s = 0.0;
  p->nu_coll = 0.0;
}

int imrp_create(const imrp_params* p, imrp_ctx** out) {
  if (!out) return IMRP_E_INVAL;
  *out = nullptr;
  if (!p) return IMRP_E_INVAL;
  ensure_registry();
  imrp_ctx* ctx = new (std::nothrow) imrp_ctx();
  if (!ctx) return IMRP_E_NOMEM;
  ctx->p = *p;
  auto bad = [&](const char* m) {
    delete ctx;
    (void)m;
    return IMRP_E_INVAL;
  };
  if (!(p->R_D_m > 0 && p->R_E_m > 0 && p->R_E_m < p->R_D_m)) return bad("geometry");
  if (!(p->R_out_m > p->R_D_m)) return bad("outer wall");
  if (!(p->eps_D >= 1.0) || !(p->n_e_m3 > 0) || !(p->dt > 0) || !(p->T_e_eV > 0)) return bad("plasma");
  if (p->N < 1 || p->N > (int64_t(1) << 31)) return bad("N");
  if (p->m0_only != 0 && p->m0_only != 1) return bad("m0_only");
  if (p->precision != 0 && p->precision != 1) return bad("precision");
  if (p->drive_kind < 0 || p->drive_kind > 2 || p->wall_rule < 0 || p->wall_rule > 2) return bad("rules");
  if (!(p->nu_coll >= 0.0) || !std::isfinite(p->nu_coll)) return bad("nu_coll");
  if (p->drive_kind == 0 && !(p->width_wpe > 0)) return bad("width");
  ctx->L = p->l_max;
  ctx->prec = p->precision;
  const bool have = ctx->prec == 1 ? find_set<float>(ctx->L) != nullptr : find_set<double>(ctx->L) != nullptr;
  if (!have) return bad("l_max not instantiated");
  const double R = p->R_D_m;
  ctx->d = 1.0 - p->R_E_m / R;
  ctx->r_out = p->R_out_m / R;
  ctx->v_hat = p->V_volts * kEps0 / (p->n_e_m3 * kE * R * R);
  ctx->lambda_D = sqrt(kEps0 * p->T_e_eV / (p->n_e_m3 * kE)) / R;
  ctx->omega_pe = sqrt(p->n_e_m3 * kE * kE / (kEps0 * kMe));
  ctx->t0 = p->t0_wpe > 0 ? p->t0_wpe : 4.0 * p->width_wpe;
  for (int l = 0; l < kTabL; ++l) {
    ctx->f[l] = coef_f(l, ctx->d, p->eps_D);
    ctx->canti[l] = l <= ctx->L ? coef_canti(l, ctx->d, p->eps_D) : 0.0;
    if (l > ctx->L) ctx->f[l] = 0.0;
  }
  ctx->nc = 2 * ncomp(ctx->L);
  cudaGetDevice(&ctx->device);
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete ctx; return IMRP_E_CUDA; }
  ctx->stream = ctx->own_stream;
  int rc = ctx->prec == 1 ? find_set<float>(ctx->L)->init(ctx->device)
                          : find_set<double>(ctx->L)->init(ctx->device);
  if (rc == 0 && set_sort_attributes() != cudaSuccess) rc = 1;
  if (rc != 0) { free_all(ctx); delete ctx; return IMRP_E_CUDA; }
  // warps per CTA of the field kernel: the largest of 8, 4, 2, 1 whose
  // resident warps per SM reach 85% of the best. Larger CTAs keep their warps
  // at nearby points of the long unrolled body (fewer instruction-cache
  // misses); more resident warps hide latency. Measured on GB300 at
  // l_max = 16: 4 warps (20 resident) beat 2 warps (22 resident) by 27%;
  // at l_max = 24: 2 warps (10 resident) beat 4 warps (8 resident) by 9%.
  {
    int nbw[4] = {0, 0, 0, 0}, best = 0;
    const int ws[4] = {8, 4, 2, 1};
    for (int q = 0; q < 4; ++q) {
      const int nb = ctx->prec == 1 ? find_set<float>(ctx->L)->field_blocks_per_sm(ws[q])
                                    : find_set<double>(ctx->L)->field_blocks_per_sm(ws[q]);
      nbw[q] = nb * ws[q];
      best = std::max(best, nbw[q]);
    }
    ctx->wpb = 0;
    for (int q = 0; q < 4 && !ctx->wpb; ++q)
      if (nbw[q] > 0 && 100 * nbw[q] >= 85 * best) ctx->wpb = ws[q];
  }
  if (ctx->wpb < 1) { free_all(ctx); delete ctx; return IMRP_E_INVAL; }
  rc = alloc_ctx(ctx);
  if (rc) {
    free_all(ctx);
    delete ctx;
    return rc == IMRP_E_CUDA ? IMRP_E_NOMEM : rc;
  }
  ctx->cap = p->N;
  *out = ctx;
  return IMRP_OK;
}

int imrp_destroy(imrp_ctx* ctx) {
  if (!ctx) return IMRP_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return IMRP_OK;
}

const char* imrp_last_error(const imrp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int imrp_set_stream(imrp_ctx* ctx, void* stream) {
  if (!ctx) return IMRP_E_INVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own_stream;
  return IMRP_OK;
}

int imrp_set_species(imrp_ctx* ctx, int64_t n_electrons, double ion_charge, double ion_mass,
                     double background_ions) {
  if (!ctx) return IMRP_E_INVAL;
  if (ion_charge == 0.0) {  // all electrons again
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->species = 0;
  } else {
    if (!(ion_charge > 0.0) || !std::isfinite(ion_charge) || !(ion_mass > 0.0) || !std::isfinite(ion_mass) ||
        !(background_ions >= 0.0) || !std::isfinite(background_ions) || n_electrons < 1 || n_electrons > ctx->cap)
      return ctx->fail(IMRP_E_INVAL, "set_species: n_electrons %lld, ion charge %g, mass %g, background %g",
                       (long long)n_electrons, ion_charge, ion_mass, background_ions);
    if (ctx->p.wall_rule == 2)
      return ctx->fail(IMRP_E_INVAL, "set_species: mobile ions with the absorbing wall are not supported");
    CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->qtile) {
      const int64_t nt = (ctx->cap + 31) / 32, ng = (nt + kTilesPerGroup - 1) / kTilesPerGroup;
      CK(cudaMalloc(&ctx->qtile, tile_stride(nt) * sizeof(double)));
      CK(cudaMalloc(&ctx->qpfx, tile_stride(nt) * sizeof(double)));
      CK(cudaMalloc(&ctx->qgagg, ng * sizeof(double)));
      CK(cudaMalloc(&ctx->qgbase, ng * sizeof(double)));
      CK(cudaMalloc(&ctx->qtot, sizeof(double)));
      CK(cudaMalloc(&ctx->qtotd, sizeof(double)));
      CK(cudaMalloc(&ctx->qwork, gs_work_doubles(1) * sizeof(double)));
      CK(cudaMalloc(&ctx->qticket, gs_col_blocks(1) * sizeof(unsigned)));
      CK(cudaMemset(ctx->qticket, 0, gs_col_blocks(1) * sizeof(unsigned)));
    }
    ctx->species = 1;
    ctx->sp_ne = n_electrons;
    ctx->sp_q = ion_charge;
    ctx->sp_m = ion_mass;
    ctx->sp_bg = background_ions;
  }
  if (ctx->loaded) {
    ctx->n_tilde = n_tilde_of(ctx, ctx->n);
    ctx->n_ion = n_ion_of(ctx, ctx->n);
  }
  drop_graphs(ctx);  // the captured steps hold the old arguments
  return IMRP_OK;
}

int imrp_set_ion_profile(imrp_ctx* ctx, const double* q_ion, int64_t n_tab, double q_elec_total,
                         double q_s) {
  if (!ctx) return IMRP_E_INVAL;
  if (n_tab == 0) {
    ctx->ion_n = 0;
  } else {
    if (n_tab < 2 || n_tab > (int64_t(1) << 30) || !q_ion)
      return ctx->fail(IMRP_E_INVAL, "set_ion_profile: table of %lld nodes", (long long)n_tab);
    if (!(q_elec_total > 0.0) || !std::isfinite(q_elec_total) || !std::isfinite(q_s))
      return ctx->fail(IMRP_E_INVAL, "set_ion_profile: electron charge %g, surface charge %g",
                       q_elec_total, q_s);
    for (int64_t k = 0; k < n_tab; ++k)
      if (!std::isfinite(q_ion[k]) || (k > 0 && q_ion[k] < q_ion[k - 1]))
        return ctx->fail(IMRP_E_INVAL, "set_ion_profile: node %lld not finite or decreasing",
                         (long long)k);
    // the previous table may still be read by queued steps
    CK(cudaStreamSynchronize(ctx->stream));
    if (n_tab > ctx->ion_cap) {
      cudaFree(ctx->ion_q);
      ctx->ion_q = nullptr;
      ctx->ion_cap = 0;
      if (cudaMalloc(&ctx->ion_q, n_tab * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        ctx->ion_n = 0;
        return ctx->fail(IMRP_E_NOMEM, "set_ion_profile: %lld nodes", (long long)n_tab);
      }
      ctx->ion_cap = n_tab;
    }
    CK(cudaMemcpy(ctx->ion_q, q_ion, n_tab * sizeof(double), cudaMemcpyHostToDevice));
    ctx->ion_n = n_tab;
    ctx->ion_qe = q_elec_total;
    ctx->ion_qs = q_s;
  }
  if (ctx->loaded) ctx->n_tilde = n_tilde_of(ctx, ctx->n);
  // the captured step pair holds the old field arguments
  drop_graphs(ctx);
  return IMRP_OK;
}

int imrp_load_particles(imrp_ctx* ctx, const double* x, const double* v, int64_t n) {
  if (!ctx) return IMRP_E_INVAL;
  if (!x || !v || n < 1 || n > ctx->cap) return ctx->fail(IMRP_E_INVAL, "load: n = %lld out of range [1, %lld]", (long long)n, (long long)ctx->cap);
  // two contiguous copies into the staging buffer: x [n][3], then v [n][3]
  CK(cudaMemcpyAsync(ctx->stage, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->stage + 3 * n, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  ctx->cur = 0;
  if (ctx->prec == 1)
    launch_load<float>(ctx->stage, ctx->stage + 3 * n, nullptr, state_of<float>(ctx), ctx->key0, ctx->idx0,
                       n, ctx->r_out, ctx->derr, ctx->stream);
  else
    launch_load<double>(ctx->stage, ctx->stage + 3 * n, nullptr, state_of<double>(ctx), ctx->key0, ctx->idx0,
                        n, ctx->r_out, ctx->derr, ctx->stream);
  StepState s0{};
  s0.step = 0;
  s0.next = 0;
  s0.u = 0;
  s0.kick = 0;
  s0.sync = 1;
  CK(cudaMemcpyAsync(ctx->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, ctx->stream));
  const bool same_n = ctx->loaded && ctx->n == n && ctx->hist_first == 0;
  int rc = check_err(ctx);
  if (rc) { ctx->loaded = false; return rc; }
  ctx->n = n;
  ctx->n_tilde = n_tilde_of(ctx, n);
  ctx->n_ion = n_ion_of(ctx, n);
  ctx->ntiles = (n + 31) / 32;
  ctx->ngroups = (ctx->ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  ctx->host_step = 0;
  ctx->hist_first = 0;
  ctx->loaded = true;
  ctx->keys_valid = true;  // the load kernel wrote the keys of its order
  // the captured steps depend on n only through their launch shapes and scalars
  if (!same_n) drop_graphs(ctx);
  return IMRP_OK;
}

int imrp_step_async(imrp_ctx* ctx, int64_t n_steps) {
  if (!ctx) return IMRP_E_INVAL;
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "step before load");
  if (n_steps < 0) return ctx->fail(IMRP_E_INVAL, "n_steps < 0");
  if (n_steps == 0) return IMRP_OK;
  return launch_steps(ctx, n_steps);
}

int imrp_ready(imrp_ctx* ctx, int* ready) {
  if (!ctx || !ready) return IMRP_E_INVAL;
  const cudaError_t e = cudaStreamQuery(ctx->stream);
  if (e == cudaErrorNotReady) {
    *ready = 0;
    return IMRP_OK;
  }
  CK(e);
  *ready = 1;
  return IMRP_OK;
}

int imrp_sync(imrp_ctx* ctx) {
  if (!ctx) return IMRP_E_INVAL;
  CK(cudaGetLastError());
  return check_err(ctx);
}

int imrp_get_qdiff(imrp_ctx* ctx, int64_t first, int64_t count, double* qd, double* ua) {
  if (!ctx) return IMRP_E_INVAL;
  if (first < ctx->hist_first || count < 0 || first + count > ctx->host_step)
    return ctx->fail(IMRP_E_INVAL, "get_qdiff: range [%lld, %lld) outside the recorded steps [%lld, %lld)",
                     (long long)first, (long long)(first + count), (long long)ctx->hist_first,
                     (long long)ctx->host_step);
  if (count == 0) return IMRP_OK;
  const int64_t h = first - ctx->hist_first;
  if (qd) CK(cudaMemcpyAsync(qd, ctx->qhist + h, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (ua) CK(cudaMemcpyAsync(ua, ctx->uhist + h, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return check_err(ctx);
}

int imrp_load_particles_async(imrp_ctx* ctx, const double* x, const double* v, int64_t n) {
  if (!ctx) return IMRP_E_INVAL;
  if (!x || !v || n < 1 || n > ctx->cap)
    return ctx->fail(IMRP_E_INVAL, "load_async: n = %lld out of range [1, %lld]", (long long)n, (long long)ctx->cap);
  if (!ctx->copy_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CK(cudaMalloc(&ctx->astage[k], 6 * ctx->cap * sizeof(double)));
      CK(cudaEventCreateWithFlags(&ctx->ev_copied[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_free[k], cudaEventDisableTiming));
    }
  }
  const int s = ctx->next_stage;
  ctx->next_stage ^= 1;
  double* S = ctx->astage[s];
  // the buffer is free once the conversion of the load before the last is done
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[s], 0));
  CK(cudaMemcpyAsync(S, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->copy_stream));
  CK(cudaMemcpyAsync(S + 3 * n, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->copy_stream));
  CK(cudaEventRecord(ctx->ev_copied[s], ctx->copy_stream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[s], 0));
  if (ctx->prec == 1)
    launch_load<float>(S, S + 3 * n, nullptr, state_of<float>(ctx), ctx->key0, ctx->idx0, n, ctx->r_out,
                       ctx->derr, ctx->stream);
  else
    launch_load<double>(S, S + 3 * n, nullptr, state_of<double>(ctx), ctx->key0, ctx->idx0, n, ctx->r_out,
                        ctx->derr, ctx->stream);
  CK(cudaEventRecord(ctx->ev_free[s], ctx->stream));
  launch_init_step(ctx->st, ctx->stream);
  CK(cudaGetLastError());
  const bool same_n = ctx->loaded && ctx->n == n && ctx->hist_first == 0;
  ctx->cur = 0;
  ctx->n = n;
  ctx->n_tilde = n_tilde_of(ctx, n);
  ctx->n_ion = n_ion_of(ctx, n);
  ctx->ntiles = (n + 31) / 32;
  ctx->ngroups = (ctx->ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  ctx->host_step = 0;
  ctx->hist_first = 0;
  ctx->loaded = true;
  ctx->keys_valid = true;  // the load kernel wrote the keys of its order
  // a captured step pair depends on n only through its launch shapes and scalars
  if (!same_n) drop_graphs(ctx);
  return IMRP_OK;
}

int imrp_copy_qdiff_async(imrp_ctx* ctx, int64_t first, int64_t count, double* qd, double* ua) {
  if (!ctx) return IMRP_E_INVAL;
  if (first < ctx->hist_first || count < 0 || first + count > ctx->host_step)
    return ctx->fail(IMRP_E_INVAL, "copy_qdiff_async: range [%lld, %lld) outside the recorded steps [%lld, %lld)",
                     (long long)first, (long long)(first + count), (long long)ctx->hist_first,
                     (long long)ctx->host_step);
  if (count == 0) return IMRP_OK;
  const int64_t h = first - ctx->hist_first;
  if (qd) CK(cudaMemcpyAsync(qd, ctx->qhist + h, count * sizeof(double), cudaMemcpyDefault, ctx->stream));
  if (ua) CK(cudaMemcpyAsync(ua, ctx->uhist + h, count * sizeof(double), cudaMemcpyDefault, ctx->stream));
  return IMRP_OK;
}

int imrp_step(imrp_ctx* ctx, int64_t n_steps, double* qdiff_out, double* uasy_out) {
  int rc = imrp_step_async(ctx, n_steps);
  if (rc) return rc;
  const int64_t first = ctx->host_step - n_steps;
  if ((qdiff_out || uasy_out) && n_steps > 0) return imrp_get_qdiff(ctx, first, n_steps, qdiff_out, uasy_out);
  return imrp_sync(ctx);
}

int imrp_get_field(imrp_ctx* ctx, double* E) {
  if (!ctx || !E) return IMRP_E_INVAL;
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "get_field before load");
  int rc = enqueue_any(ctx, false);
  if (rc) return rc;
  CK(cudaGetLastError());
  const int64_t n = ctx->n;
  if (ctx->prec == 1) {
    const float* e = static_cast<const float*>(ctx->eout);
    const float* cs[3] = {e, e + n, e + 2 * n};
    launch_scatter_by_id<float>(cs, 3, ctx->srt_id, ctx->stage, n, ctx->stream);
  } else {
    const double* e = static_cast<const double*>(ctx->eout);
    const double* cs[3] = {e, e + n, e + 2 * n};
    launch_scatter_by_id<double>(cs, 3, ctx->srt_id, ctx->stage, n, ctx->stream);
  }
  CK(cudaMemcpyAsync(E, ctx->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return check_err(ctx);
}

int imrp_get_particles(imrp_ctx* ctx, double* x, double* v) {
  if (!ctx) return IMRP_E_INVAL;
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "get_particles before load");
  const int64_t n = ctx->n;
  // positions to stage[0, 3n) and velocities to stage[3n, 6n), each [n][3] in id order
  if (ctx->prec == 1) launch_state_out<float>(state_of<float>(ctx), ctx->stage, ctx->stage + 3 * n, n, ctx->stream);
  else launch_state_out<double>(state_of<double>(ctx), ctx->stage, ctx->stage + 3 * n, n, ctx->stream);
  if (x) CK(cudaMemcpyAsync(x, ctx->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (v) CK(cudaMemcpyAsync(v, ctx->stage + 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return check_err(ctx);
}

int imrp_get_surface_charge(imrp_ctx* ctx, double* q_s, int64_t* n_absorbed) {
  if (!ctx) return IMRP_E_INVAL;
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "get_surface_charge before load");
  StepState h{};
  CK(cudaMemcpyAsync(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = check_err(ctx);
  if (rc) return rc;
  // absorptions of the last step are folded in by the next step's finalize
  const double base = ctx->ion_n ? ctx->ion_qs * ctx->n_tilde : ctx->p.q_s;
  if (q_s) *q_s = base + h.qs_acc - double(h.nabs_step);
  if (n_absorbed) *n_absorbed = h.nabs_total + h.nabs_step;
  return IMRP_OK;
}

int imrp_checkpoint(imrp_ctx* ctx, double* x, double* v, uint32_t* id, int64_t* step) {
  if (!ctx) return IMRP_E_INVAL;
  if (!x || !v || !id || !step) return ctx->fail(IMRP_E_INVAL, "checkpoint: null output");
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "checkpoint before load");
  const int64_t n = ctx->n;
  uint32_t* ids = ctx->key1;  // free between steps
  if (ctx->prec == 1)
    launch_state_dump<float>(state_of<float>(ctx), ctx->stage, ctx->stage + 3 * n, ids, n, ctx->stream);
  else
    launch_state_dump<double>(state_of<double>(ctx), ctx->stage, ctx->stage + 3 * n, ids, n, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(x, ctx->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(v, ctx->stage + 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(id, ids, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  *step = ctx->host_step;
  return check_err(ctx);
}

int imrp_restore(imrp_ctx* ctx, const double* x, const double* v, const uint32_t* id, int64_t n, int64_t step) {
  if (!ctx) return IMRP_E_INVAL;
  if (!x || !v || !id || n < 1 || n > ctx->cap)
    return ctx->fail(IMRP_E_INVAL, "restore: n = %lld out of range [1, %lld]", (long long)n, (long long)ctx->cap);
  if (step < 0) return ctx->fail(IMRP_E_INVAL, "restore: step %lld < 0", (long long)step);
  {
    // the ids must be a permutation of 0..n-1 (they index the output and the random numbers)
    std::vector<uint8_t> seen(size_t(n), 0);
    for (int64_t j = 0; j < n; ++j) {
      if (int64_t(id[j]) >= n || seen[id[j]])
        return ctx->fail(IMRP_E_INVAL, "restore: ids are not a permutation of 0..n-1 (entry %lld)", (long long)j);
      seen[id[j]] = 1;
    }
  }
  CK(cudaMemcpyAsync(ctx->stage, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->stage + 3 * n, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->key1, id, n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  ctx->cur = 0;
  if (ctx->prec == 1)
    launch_load<float>(ctx->stage, ctx->stage + 3 * n, ctx->key1, state_of<float>(ctx), ctx->key0, ctx->idx0, n,
                       ctx->r_out, ctx->derr, ctx->stream);
  else
    launch_load<double>(ctx->stage, ctx->stage + 3 * n, ctx->key1, state_of<double>(ctx), ctx->key0, ctx->idx0,
                        n, ctx->r_out, ctx->derr, ctx->stream);
  // the step state as the run left it: the next step is `step`, velocities a
  // half step behind the positions unless nothing was stepped yet
  StepState s0{};
  s0.step = step;
  s0.next = step;
  s0.u = 0;
  s0.kick = 0;
  s0.sync = step == 0 ? 1 : 0;
  CK(cudaMemcpyAsync(ctx->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, ctx->stream));
  int rc = check_err(ctx);
  if (rc) { ctx->loaded = false; return rc; }
  ctx->n = n;
  ctx->n_tilde = n_tilde_of(ctx, n);
  ctx->n_ion = n_ion_of(ctx, n);
  ctx->ntiles = (n + 31) / 32;
  ctx->ngroups = (ctx->ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
  ctx->host_step = step;
  ctx->hist_first = step;
  ctx->loaded = true;
  ctx->keys_valid = true;
  drop_graphs(ctx);  // the history offset is part of the captured arguments
  return IMRP_OK;
}

int imrp_profile_steps(imrp_ctx* ctx, int64_t n_steps, double* ms) {
  if (!ctx || !ms || n_steps < 1) return IMRP_E_INVAL;
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "profile before load");
  int rc = grow_history(ctx, ctx->host_step - ctx->hist_first + n_steps + 1);
  if (rc) return rc;
  for (int k = 0; k < IMRP_N_STAGES; ++k) ms[k] = 0.0;
  std::vector<cudaEvent_t> ev(size_t(n_steps) * (IMRP_N_STAGES + 1));
  for (auto& e : ev) CK(cudaEventCreate(&e));
  int err = IMRP_OK;
  for (int64_t s = 0; s < n_steps && !err; ++s) {
    cudaEvent_t* e = ev.data() + s * (IMRP_N_STAGES + 1);
    err = enqueue_any(ctx, true, e);
  }
  if (!err) {
    ctx->host_step += n_steps;
    cudaError_t ce = cudaStreamSynchronize(ctx->stream);
    if (ce != cudaSuccess) err = ctx->fail(IMRP_E_CUDA, "profile: %s", cudaGetErrorString(ce));
    for (int64_t s = 0; s < n_steps && !err; ++s) {
      cudaEvent_t* e = ev.data() + s * (IMRP_N_STAGES + 1);
      for (int k = 0; k < IMRP_N_STAGES; ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e[k], e[k + 1]);
        ms[k] += t;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err) return err;
  return check_err(ctx);
}

int imrp_get_info(const imrp_ctx* ctx, imrp_info* info) {
  if (!ctx || !info) return IMRP_E_INVAL;
  info->d = ctx->d;
  info->r_out = ctx->r_out;
  info->n_tilde = ctx->n_tilde;
  info->n_ion = ctx->n_ion;
  info->v_hat = ctx->v_hat;
  info->lambda_D = ctx->lambda_D;
  info->omega_pe = ctx->omega_pe;
  info->n = ctx->n;
  info->step = ctx->host_step;
  info->l_max = ctx->L;
  info->precision = ctx->prec;
  return IMRP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner and batched stepping of many contexts.
// ---------------------------------------------------------------------------
namespace {

// Radius keys for the current storage order (no step is taken).
int ensure_keys(imrp_ctx* ctx) {
  if (ctx->keys_valid) return IMRP_OK;
  if (ctx->prec == 1) launch_keys<float>(state_of<float>(ctx), ctx->key0, ctx->idx0, ctx->n, ctx->r_out, ctx->stream);
  else launch_keys<double>(state_of<double>(ctx), ctx->key0, ctx->idx0, ctx->n, ctx->r_out, ctx->stream);
  CK(cudaGetLastError());
  ctx->keys_valid = true;
  return IMRP_OK;
}

// Device time of stage k (events ev[k] .. ev[k+1]) of a field-only pass, summed over reps.
int time_stage(imrp_ctx* ctx, int stage, int reps, float* ms) {
  cudaEvent_t ev[IMRP_N_STAGES + 1];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  float tot = 0.f;
  int rc = IMRP_OK;
  for (int r = 0; r < reps && !rc; ++r) {
    rc = enqueue_any(ctx, false, ev);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(ev[IMRP_N_STAGES]);
    if (e != cudaSuccess) { rc = ctx->fail(IMRP_E_CUDA, "autotune: %s", cudaGetErrorString(e)); break; }
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[stage], ev[stage + 1]);
    tot += t;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  *ms = tot;
  return rc;
}

}  // namespace

extern "C" int imrp_autotune(imrp_ctx* ctx, int* wpb_out, int* gseg_out) {
  if (!ctx) return IMRP_E_INVAL;
  if (!ctx->loaded) return ctx->fail(IMRP_E_STATE, "autotune before load");
  const int reps = 3;
  // field kernel: warps per CTA
  {
    int best_w = ctx->wpb;
    float best = 1e30f;
    for (int w : {8, 4, 2, 1}) {
      const int nb = ctx->prec == 1 ? find_set<float>(ctx->L)->field_blocks_per_sm(w)
                                    : find_set<double>(ctx->L)->field_blocks_per_sm(w);
      if (nb < 1) continue;
      ctx->wpb = w;
      float ms = 0.f;
      int rc = time_stage(ctx, 4, reps, &ms);
      if (rc) return rc;
      if (ms < best) { best = ms; best_w = w; }
    }
    ctx->wpb = best_w;
  }
  // group scan: least groups per segment
  {
    int best_c = ctx->gseg;
    float best = 1e30f;
    for (int c : {16, 32, 64}) {
      ctx->gseg = c;
      float ms = 0.f;
      int rc = time_stage(ctx, 3, reps, &ms);
      if (rc) return rc;
      if (ms < best) { best = ms; best_c = c; }
    }
    ctx->gseg = best_c;
  }
  drop_graphs(ctx);
  if (wpb_out) *wpb_out = ctx->wpb;
  if (gseg_out) *gseg_out = ctx->gseg;
  return check_err(ctx);
}

// A degree and precision of a batch: its contexts' moments and field run as
// one launch each over a work list of (context, block) items.
struct BatchGroup {
  int prec = 0, L = 0, wpb = 0;
  std::vector<int> members;     // indices into the batch's contexts
  void* dmom = nullptr;         // MomArgs<T>[members]
  void* dfield = nullptr;       // FieldArgs<T>[members] (push mode)
  int2* dmom_items = nullptr;   // (member, block): first the members of mom_ppt 16, then of 4
  int2* dfield_items = nullptr; // (member, first tile of a CTA)
  int nmom = 0, nmom_small = 0, nfield = 0;
};

struct imrp_batch {
  std::vector<imrp_ctx*> c;
  std::vector<BatchGroup> groups;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t g = nullptr;
  std::vector<int> cur_at_capture;
  std::vector<const double*> hist_at_capture;
  std::vector<uint64_t> gen_at_capture;
  std::string err;
  int failed = -1;  // index of the context whose error the last call returned
  std::vector<int3> tuned;  // (precision, degree, warps per CTA) chosen by imrp_batch_autotune
};

extern "C" int imrp_batch_create(imrp_ctx* const* ctxs, int n, imrp_batch** out) {
  if (!out || !ctxs || n < 1) return IMRP_E_INVAL;
  *out = nullptr;
  int dev0 = -1;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->loaded) return IMRP_E_STATE;
    if (dev0 < 0) dev0 = ctxs[i]->device;
    if (ctxs[i]->device != dev0) return IMRP_E_INVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return IMRP_E_INVAL;
  }
  imrp_batch* b = new (std::nothrow) imrp_batch();
  if (!b) return IMRP_E_NOMEM;
  b->c.assign(ctxs, ctxs + n);
  bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  b->join.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i) ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto e : b->join) if (e) cudaEventDestroy(e);
    delete b;
    return IMRP_E_CUDA;
  }
  *out = b;
  return IMRP_OK;
}

namespace {
void free_groups(imrp_batch* b) {
  if (!b->groups.empty()) cudaStreamSynchronize(b->stream);  // a replay may still read them
  for (auto& g : b->groups) {
    cudaFree(g.dmom);
    cudaFree(g.dfield);
    cudaFree(g.dmom_items);
    cudaFree(g.dfield_items);
  }
  b->groups.clear();
}

// The contexts' arguments and work lists per degree and precision, in device
// memory, for the batched launches (built before a capture: they hold buffer
// pointers and scalars that the captured graph keeps using).
template <class T> int fill_group(imrp_batch* b, BatchGroup& g) {
  std::vector<MomArgs<T>> ma;
  std::vector<FieldArgs<T>> fa;
  std::vector<int2> mi, ms, fi;
  for (size_t k = 0; k < g.members.size(); ++k) {
    imrp_ctx* ctx = b->c[g.members[k]];
    ma.push_back(make_mom_args<T>(ctx));
    fa.push_back(make_field_args<T>(ctx, true));
    // the moments' blocks as the context's own launch takes them (bit-identical sums)
    const int ppt = mom_ppt(sizeof(T), ctx->n);
    const int64_t mblocks = mom_blocks(ctx->n, ppt);
    for (int64_t q = 0; q < mblocks; ++q) (ppt == 16 ? mi : ms).push_back(make_int2(int(k), int(q)));
    for (int64_t t = 0; t < ctx->ntiles; t += g.wpb) fi.push_back(make_int2(int(k), int(t)));
  }
  g.nmom_small = int(ms.size());
  mi.insert(mi.end(), ms.begin(), ms.end());
  g.nmom = int(mi.size());
  g.nfield = int(fi.size());
  if (cudaMalloc(&g.dmom, ma.size() * sizeof(MomArgs<T>)) != cudaSuccess ||
      cudaMalloc(&g.dfield, fa.size() * sizeof(FieldArgs<T>)) != cudaSuccess ||
      cudaMalloc(&g.dmom_items, mi.size() * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&g.dfield_items, fi.size() * sizeof(int2)) != cudaSuccess)
    return IMRP_E_NOMEM;
  if (cudaMemcpy(g.dmom, ma.data(), ma.size() * sizeof(MomArgs<T>), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g.dfield, fa.data(), fa.size() * sizeof(FieldArgs<T>), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g.dmom_items, mi.data(), mi.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g.dfield_items, fi.data(), fi.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
    return IMRP_E_CUDA;
  return IMRP_OK;
}

int build_groups(imrp_batch* b) {
  free_groups(b);
  for (size_t i = 0; i < b->c.size(); ++i) {
    imrp_ctx* ctx = b->c[i];
    BatchGroup* g = nullptr;
    for (auto& h : b->groups)
      if (h.prec == ctx->prec && h.L == ctx->L) g = &h;
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
      g->prec = ctx->prec;
      g->L = ctx->L;
      g->wpb = ctx->wpb;  // the launch shape of the group's first context, unless tuned
      for (const int3& t : b->tuned)
        if (t.x == g->prec && t.y == g->L) g->wpb = t.z;
    }
    g->members.push_back(int(i));
  }
  for (auto& g : b->groups) {
    const int rc = g.prec == 1 ? fill_group<float>(b, g) : fill_group<double>(b, g);
    if (rc) return rc;
  }
  return IMRP_OK;
}

// One step of every context of the batch: sort and reorder on each context's
// stream; the moments of all contexts of a degree in one launch; the scans and
// finalize per context; the field of all contexts of a degree in one launch.
int enqueue_batch_step(imrp_batch* b) {
  const int n = int(b->c.size());
  cudaEventRecord(b->fork, b->stream);
  for (int i = 0; i < n; ++i) {
    imrp_ctx* ctx = b->c[i];
    cudaStreamWaitEvent(ctx->stream, b->fork, 0);
    if (ctx->prec == 1) enqueue_pre<float>(ctx, nullptr, true);
    else enqueue_pre<double>(ctx, nullptr, true);
    cudaEventRecord(b->join[i], ctx->stream);
    cudaStreamWaitEvent(b->stream, b->join[i], 0);
  }
  for (auto& g : b->groups) {
    const int nbig = g.nmom - g.nmom_small;
    if (g.prec == 1) {
      const KernelSet<float>* ks = find_set<float>(g.L);
      const MomArgs<float>* ma = static_cast<const MomArgs<float>*>(g.dmom);
      ks->moments_batch(ma, g.dmom_items, nbig, 16, b->stream);
      ks->moments_batch(ma, g.dmom_items + nbig, g.nmom_small, 4, b->stream);
    } else {
      const KernelSet<double>* ks = find_set<double>(g.L);
      const MomArgs<double>* ma = static_cast<const MomArgs<double>*>(g.dmom);
      ks->moments_batch(ma, g.dmom_items, nbig, 16, b->stream);
      ks->moments_batch(ma, g.dmom_items + nbig, g.nmom_small, 4, b->stream);
    }
  }
  cudaEventRecord(b->fork, b->stream);
  for (int i = 0; i < n; ++i) {
    imrp_ctx* ctx = b->c[i];
    cudaStreamWaitEvent(ctx->stream, b->fork, 0);
    if (ctx->prec == 1) enqueue_mid<float>(ctx, true);
    else enqueue_mid<double>(ctx, true);
    cudaEventRecord(b->join[i], ctx->stream);
    cudaStreamWaitEvent(b->stream, b->join[i], 0);
  }
  for (auto& g : b->groups) {
    if (g.prec == 1)
      find_set<float>(g.L)->field_batch(static_cast<const FieldArgs<float>*>(g.dfield), g.dfield_items, g.nfield,
                                        g.wpb, b->stream);
    else
      find_set<double>(g.L)->field_batch(static_cast<const FieldArgs<double>*>(g.dfield), g.dfield_items,
                                         g.nfield, g.wpb, b->stream);
  }
  for (imrp_ctx* ctx : b->c) ctx->keys_valid = true;  // the field kernels wrote the next keys
  return IMRP_OK;
}
}  // namespace

extern "C" int imrp_batch_destroy(imrp_batch* b) {
  if (!b) return IMRP_OK;
  cudaStreamSynchronize(b->stream);
  if (b->g) cudaGraphExecDestroy(b->g);
  free_groups(b);
  cudaStreamDestroy(b->own_stream ? b->own_stream : b->stream);
  cudaEventDestroy(b->fork);
  for (auto e : b->join) cudaEventDestroy(e);
  delete b;
  return IMRP_OK;
}

extern "C" const char* imrp_batch_last_error(const imrp_batch* b) { return b ? b->err.c_str() : "null batch"; }

namespace {
int batch_fail(imrp_batch* b, imrp_ctx* ctx, int rc) {
  b->err = ctx ? ctx->err : std::string("batch error");
  b->failed = -1;
  for (size_t i = 0; ctx && i < b->c.size(); ++i)
    if (b->c[i] == ctx) b->failed = int(i);
  return rc;
}
}  // namespace

extern "C" int imrp_batch_failed(const imrp_batch* b) { return b ? b->failed : -1; }

extern "C" int imrp_batch_set_stream(imrp_batch* b, void* stream) {
  if (!b) return IMRP_E_INVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return IMRP_E_CUDA;
  if (b->own_stream == nullptr) b->own_stream = b->stream;
  b->stream = stream ? static_cast<cudaStream_t>(stream) : b->own_stream;
  return IMRP_OK;
}

extern "C" int imrp_batch_step(imrp_batch* b, int64_t n_steps) {
  if (!b) return IMRP_E_INVAL;
  b->failed = -1;
  if (n_steps < 0) return IMRP_E_INVAL;
  if (n_steps == 0) return IMRP_OK;
  const int n = int(b->c.size());
  // prior work of each context happens before the batch; histories large enough
  for (imrp_ctx* ctx : b->c) {
    int rc = grow_history(ctx, ctx->host_step - ctx->hist_first + n_steps + 1);
    if (rc) return batch_fail(b, ctx, rc);
    rc = ensure_keys(ctx);
    if (rc) return batch_fail(b, ctx, rc);
    cudaEventRecord(b->join[0], ctx->stream);
    cudaStreamWaitEvent(b->stream, b->join[0], 0);
  }
  int64_t pairs = n_steps / 2;
  if (pairs > 0) {
    bool valid = b->g != nullptr;
    for (int i = 0; i < n && valid; ++i)
      valid = b->cur_at_capture[i] == b->c[i]->cur && b->hist_at_capture[i] == b->c[i]->qhist &&
              b->gen_at_capture[i] == b->c[i]->gen;
    if (!valid) {
      if (b->g) { cudaGraphExecDestroy(b->g); b->g = nullptr; }
      // work lists and arguments of the batched launches (outside the capture)
      int rc = build_groups(b);
      if (rc) { b->err = "batch work lists"; return rc; }
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return batch_fail(b, nullptr, IMRP_E_CUDA);
      rc = enqueue_batch_step(b);
      if (!rc) rc = enqueue_batch_step(b);
      cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
      if (rc) { if (g) cudaGraphDestroy(g); return rc; }
      if (ec != cudaSuccess) { b->err = cudaGetErrorString(ec); return IMRP_E_CUDA; }
      ec = cudaGraphInstantiate(&b->g, g, 0);
      cudaGraphDestroy(g);
      if (ec != cudaSuccess) { b->err = cudaGetErrorString(ec); return IMRP_E_CUDA; }
      b->cur_at_capture.resize(n);
      b->hist_at_capture.resize(n);
      b->gen_at_capture.resize(n);
      for (int i = 0; i < n; ++i) {
        b->cur_at_capture[i] = b->c[i]->cur;
        b->hist_at_capture[i] = b->c[i]->qhist;
        b->gen_at_capture[i] = b->c[i]->gen;
      }
    }
    for (int64_t k = 0; k < pairs; ++k)
      if (cudaGraphLaunch(b->g, b->stream) != cudaSuccess) { b->err = "graph launch"; return IMRP_E_CUDA; }
  }
  if (n_steps & 1) {
    cudaEventRecord(b->fork, b->stream);
    for (int i = 0; i < n; ++i) {
      imrp_ctx* ctx = b->c[i];
      cudaStreamWaitEvent(ctx->stream, b->fork, 0);
      int rc = enqueue_any(ctx, true);
      if (rc) return batch_fail(b, ctx, rc);
      cudaEventRecord(b->join[i], ctx->stream);
      cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
  }
  for (imrp_ctx* ctx : b->c) {
    ctx->host_step += n_steps;
    // later work on the context's own stream waits for the batch
    cudaEventRecord(b->fork, b->stream);
    cudaStreamWaitEvent(ctx->stream, b->fork, 0);
  }
  if (cudaGetLastError() != cudaSuccess) { b->err = "launch"; return IMRP_E_CUDA; }
  return IMRP_OK;
}

namespace {
// Times the batched field launch of group g in field-only mode (the contexts'
// sorted arrays and scans must be current) at `wpb` warps per CTA: the best
// of `reps` launches after one warm-up, in ms.
template <class T> int time_group_field(imrp_batch* b, const BatchGroup& g, int wpb, int reps, float* ms) {
  std::vector<FieldArgs<T>> fa;
  std::vector<int2> fi;
  for (size_t k = 0; k < g.members.size(); ++k) {
    imrp_ctx* ctx = b->c[g.members[k]];
    fa.push_back(make_field_args<T>(ctx, false));
    for (int64_t t = 0; t < ctx->ntiles; t += wpb) fi.push_back(make_int2(int(k), int(t)));
  }
  void* dfa = nullptr;
  int2* dfi = nullptr;
  int rc = IMRP_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&dfa, fa.size() * sizeof(FieldArgs<T>)) != cudaSuccess ||
      cudaMalloc(&dfi, fi.size() * sizeof(int2)) != cudaSuccess ||
      cudaMemcpy(dfa, fa.data(), fa.size() * sizeof(FieldArgs<T>), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dfi, fi.data(), fi.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = IMRP_E_CUDA;
  } else {
    const KernelSet<T>* ks = find_set<T>(g.L);
    float best = 1e30f;
    for (int r = 0; r <= reps && rc == IMRP_OK; ++r) {
      cudaEventRecord(e0, b->stream);
      ks->field_batch(static_cast<const FieldArgs<T>*>(dfa), dfi, int(fi.size()), wpb, b->stream);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = IMRP_E_CUDA; break; }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0 && t < best) best = t;
    }
    *ms = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dfa);
  cudaFree(dfi);
  return rc;
}
}  // namespace

extern "C" int imrp_batch_autotune(imrp_batch* b) {
  if (!b) return IMRP_E_INVAL;
  b->failed = -1;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) { b->err = "sync"; return IMRP_E_CUDA; }
  // the contexts' sorted arrays and scans at their current state (field-only
  // stages: the state does not advance; the radius keys are recomputed later)
  for (imrp_ctx* ctx : b->c) {
    int rc = ensure_keys(ctx);
    if (rc) return batch_fail(b, ctx, rc);
    if (ctx->prec == 1) {
      enqueue_pre<float>(ctx);
      find_set<float>(ctx->L)->moments(make_mom_args<float>(ctx), ctx->stream);
      enqueue_mid<float>(ctx, false);
    } else {
      enqueue_pre<double>(ctx);
      find_set<double>(ctx->L)->moments(make_mom_args<double>(ctx), ctx->stream);
      enqueue_mid<double>(ctx, false);
    }
    ctx->keys_valid = false;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return batch_fail(b, ctx, IMRP_E_CUDA);
  }
  int rc = build_groups(b);
  if (rc) { b->err = "batch work lists"; return rc; }
  b->tuned.clear();
  for (auto& g : b->groups) {
    int best_w = g.wpb;
    float best = 1e30f;
    for (int w : {8, 4, 2, 1}) {
      const int nb = g.prec == 1 ? find_set<float>(g.L)->field_blocks_per_sm(w)
                                 : find_set<double>(g.L)->field_blocks_per_sm(w);
      if (nb < 1) continue;
      float ms = 0.f;
      rc = g.prec == 1 ? time_group_field<float>(b, g, w, 3, &ms) : time_group_field<double>(b, g, w, 3, &ms);
      if (rc) { b->err = "batch autotune"; return rc; }
      if (ms < best) { best = ms; best_w = w; }
    }
    b->tuned.push_back(make_int3(g.prec, g.L, best_w));
  }
  if (b->g) { cudaGraphExecDestroy(b->g); b->g = nullptr; }  // the next step recaptures with these shapes
  free_groups(b);
  for (imrp_ctx* ctx : b->c) {
    rc = check_err(ctx);
    if (rc) return batch_fail(b, ctx, rc);
  }
  return IMRP_OK;
}

extern "C" int imrp_batch_sync(imrp_batch* b) {
  if (!b) return IMRP_E_INVAL;
  b->failed = -1;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) { b->err = "sync"; return IMRP_E_CUDA; }
  for (imrp_ctx* ctx : b->c) {
    int rc = check_err(ctx);
    if (rc) return batch_fail(b, ctx, rc);
  }
  return IMRP_OK;
}

// ---------------------------------------------------------------------------
// Spectrum post-processing on the host (peak, width, damped-sine fit).
// ---------------------------------------------------------------------------
namespace {

void peak_fwhm(const std::vector<double>& w, const std::vector<double>& re, double* wr, double* dw) {
  const size_t nf = re.size();
  size_t j = 0;
  for (size_t k = 1; k < nf; ++k) if (re[k] > re[j]) j = k;
  double res = w[j];
  if (j > 0 && j + 1 < nf) {
    const double y0 = re[j - 1], y1 = re[j], y2 = re[j + 1];
    const double den = y0 - 2 * y1 + y2;
    if (den != 0) res = w[j] + 0.5 * (y0 - y2) / den * (w[1] - w[0]);
  }
  const double half = 0.5 * re[j];
  size_t lo = j, hi = j;
  while (lo > 0 && re[lo] > half) --lo;
  while (hi + 1 < nf && re[hi] > half) ++hi;
  auto cross = [&](size_t a, size_t b) {
    if (re[a] == re[b]) return w[a];
    return w[a] + (half - re[a]) * (w[b] - w[a]) / (re[b] - re[a]);
  };
  const double wl = re[lo] <= half ? cross(lo, lo + 1) : w[lo];
  const double wh = re[hi] <= half ? cross(hi - 1, hi) : w[hi];
  *wr = res;
  *dw = wh - wl;
}

// Levenberg-Marquardt for y(tau) = a e^{-b tau} sin(c tau + phi).
double fit_model(const std::vector<double>& tau, const std::vector<double>& y, double p[4]) {
  auto resid = [&](const double* q, double* jac, double* r2) {
    double s = 0;
    double JtJ[16] = {0}, Jtr[4] = {0};
    for (size_t i = 0; i < tau.size(); ++i) {
      const double t = tau[i], e = exp(-q[1] * t), sn = sin(q[2] * t + q[3]), cs = cos(q[2] * t + q[3]);
      const double f = q[0] * e * sn, r = y[i] - f;
      const double g[4] = {e * sn, -t * q[0] * e * sn, t * q[0] * e * cs, q[0] * e * cs};
      s += r * r;
      if (jac) {
        for (int a = 0; a < 4; ++a) {
          Jtr[a] += g[a] * r;
          for (int b = 0; b < 4; ++b) JtJ[4 * a + b] += g[a] * g[b];
        }
      }
    }
    if (jac) { memcpy(jac, JtJ, sizeof(JtJ)); memcpy(jac + 16, Jtr, sizeof(Jtr)); }
    *r2 = s;
  };
  double lam = 1e-3, cur;
  double buf[20];
  resid(p, buf, &cur);
  for (int it = 0; it < 200; ++it) {
    double A[16], g[4];
    memcpy(A, buf, sizeof(A));
    memcpy(g, buf + 16, sizeof(g));
    for (int a = 0; a < 4; ++a) A[5 * a] *= (1.0 + lam);
    // solve A dp = g (4x4 Gaussian elimination with partial pivoting)
    double M[4][5];
    for (int a = 0; a < 4; ++a) { for (int b = 0; b < 4; ++b) M[a][b] = A[4 * a + b]; M[a][4] = g[a]; }
    bool ok = true;
    for (int c = 0; c < 4 && ok; ++c) {
      int pv = c;
      for (int r = c + 1; r < 4; ++r) if (fabs(M[r][c]) > fabs(M[pv][c])) pv = r;
      if (M[pv][c] == 0) { ok = false; break; }
      for (int k = 0; k < 5; ++k) std::swap(M[c][k], M[pv][k]);
      for (int r = 0; r < 4; ++r) if (r != c) {
        const double fct = M[r][c] / M[c][c];
        for (int k = c; k < 5; ++k) M[r][k] -= fct * M[c][k];
      }
    }
    if (!ok) break;
    double q[4];
    for (int a = 0; a < 4; ++a) q[a] = p[a] + M[a][4] / M[a][a];
    double nb[20], nr;
    resid(q, nb, &nr);
    if (nr < cur) {
      const double rel = (cur - nr) / (cur + 1e-300);
      memcpy(p, q, sizeof(q));
      memcpy(buf, nb, sizeof(nb));
      cur = nr;
      lam = std::max(lam * 0.3, 1e-12);
      if (rel < 1e-14) break;
    } else {
      lam *= 10.0;
      if (lam > 1e12) break;
    }
  }
  return cur;
}

// Best of four starting phases; reports a >= 0, c >= 0, phi in [0, 2 pi).
void fit_damped(const std::vector<double>& tau, const std::vector<double>& y, double b0, double w0,
                double best[4]) {
  for (int k = 0; k < 4; ++k) best[k] = NAN;
  if (tau.size() < 8) return;
  double amax = 0;
  for (double v : y) amax = std::max(amax, fabs(v));
  double bres = INFINITY;
  const double phs[4] = {0.0, kPi / 2, kPi, -kPi / 2};
  for (double ph : phs) {
    double pp[4] = {amax > 0 ? amax : 1.0, b0, w0, ph};
    const double r = fit_model(tau, y, pp);
    if (r < bres && std::isfinite(r)) { bres = r; memcpy(best, pp, 4 * sizeof(double)); }
  }
  if (best[2] < 0) { best[2] = -best[2]; best[3] = kPi - best[3]; }
  if (best[0] < 0) { best[0] = -best[0]; best[3] += kPi; }
  best[3] = fmod(best[3], 2.0 * kPi);
  if (best[3] < 0) best[3] += 2.0 * kPi;
}

}  // namespace

extern "C" int imrp_spectrum(imrp_ctx* ctx, int64_t n_freq, double w_max, double* omega, double* reY,
                             double* imY, double* w_res, double* dw, double* fit) {
  if (!ctx) return IMRP_E_INVAL;
  if (ctx->hist_first != 0)
    return ctx->fail(IMRP_E_STATE, "spectrum after a restore: the history starts at step %lld, not at the drive; "
                     "transform the whole series with imrp_admittance", (long long)ctx->hist_first);
  const int64_t ns = ctx->host_step;
  if (ns < 8) return ctx->fail(IMRP_E_STATE, "spectrum needs at least 8 recorded steps (have %lld)", (long long)ns);
  if (n_freq < 3 || !(w_max > 0)) return ctx->fail(IMRP_E_INVAL, "spectrum: n_freq >= 3 and w_max > 0 required");
  if (n_freq > ctx->dft_cap) {
    cudaFree(ctx->dft);
    ctx->dft = nullptr;
    CK(cudaMalloc(&ctx->dft, 4 * n_freq * sizeof(double)));
    ctx->dft_cap = n_freq;
  }
  const double dt = ctx->p.dt;
  launch_dft(ctx->qhist, ctx->uhist, ns, dt, 0.5 * dt, n_freq, w_max, ctx->dft, ctx->stream);
  CK(cudaGetLastError());
  std::vector<double> h(4 * n_freq), q(ns);
  CK(cudaMemcpyAsync(h.data(), ctx->dft, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(q.data(), ctx->qhist, ns * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<double> w(n_freq), re(n_freq), im(n_freq);
  for (int64_t j = 0; j < n_freq; ++j) {
    w[j] = double(j + 1) * (w_max / double(n_freq));
    // Y = i w Q / U
    const double Qr = h[4 * j], Qi = h[4 * j + 1], Ur = h[4 * j + 2], Ui = h[4 * j + 3];
    const double den = Ur * Ur + Ui * Ui;
    const double Rr = (Qr * Ur + Qi * Ui) / den, Ri = (Qi * Ur - Qr * Ui) / den;  // Q/U
    re[j] = -w[j] * Ri;
    im[j] = w[j] * Rr;
  }
  double wr = 0, width = 0;
  peak_fwhm(w, re, &wr, &width);
  if (omega) memcpy(omega, w.data(), n_freq * sizeof(double));
  if (reY) memcpy(reY, re.data(), n_freq * sizeof(double));
  if (imY) memcpy(imY, im.data(), n_freq * sizeof(double));
  if (w_res) *w_res = wr;
  if (dw) *dw = width;
  if (fit) {
    const double tfit = ctx->p.drive_kind == 0 ? ctx->t0 + 3.0 * ctx->p.width_wpe : 0.0;
    std::vector<double> tau, y;
    for (int64_t k = 0; k < ns; ++k) {
      const double t = k * dt;
      if (t >= tfit) {
        tau.push_back(t - tfit);
        y.push_back(q[k] - q[0]);
      }
    }
    fit_damped(tau, y, std::max(0.5 * width, 1e-3), wr, fit);
  }
  return IMRP_OK;
}

extern "C" int imrp_fit_damped_sine(const double* q, int64_t ns, double dt, double t_fit, double t_end,
                                    double w0, double b0, double* fit) {
  if (!q || !fit || ns < 1 || !(dt > 0) || !(t_end > t_fit) || !(w0 > 0) || !(b0 > 0)) return IMRP_E_INVAL;
  std::vector<double> tau, y;
  for (int64_t k = 0; k < ns; ++k) {
    const double t = k * dt;
    if (t >= t_fit && t <= t_end) {
      tau.push_back(t - t_fit);
      y.push_back(q[k] - q[0]);
    }
  }
  if (tau.size() < 8) return IMRP_E_INVAL;
  fit_damped(tau, y, b0, w0, fit);
  return std::isfinite(fit[0]) ? IMRP_OK : IMRP_E_INVAL;
}

extern "C" int imrp_admittance(const double* q, const double* u, int64_t ns, double dt, double first_kick,
                               int64_t n_freq, double w_max, double* omega, double* reY, double* imY) {
  if (!q || !u || ns < 8 || n_freq < 3 || !(w_max > 0) || !(dt > 0)) return IMRP_E_INVAL;
  double *dq = nullptr, *du = nullptr, *dout = nullptr;
  const size_t bs = size_t(ns) * sizeof(double), bo = size_t(4 * n_freq) * sizeof(double);
  if (cudaMalloc(&dq, bs) != cudaSuccess || cudaMalloc(&du, bs) != cudaSuccess ||
      cudaMalloc(&dout, bo) != cudaSuccess) {
    cudaFree(dq);
    cudaFree(du);
    cudaFree(dout);
    return IMRP_E_NOMEM;
  }
  std::vector<double> h(4 * n_freq);
  cudaError_t e = cudaMemcpy(dq, q, bs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(du, u, bs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_dft(dq, du, ns, dt, first_kick, n_freq, w_max, dout, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), dout, bo, cudaMemcpyDeviceToHost);
  cudaFree(dq);
  cudaFree(du);
  cudaFree(dout);
  if (e != cudaSuccess) return IMRP_E_CUDA;
  for (int64_t j = 0; j < n_freq; ++j) {
    const double w = double(j + 1) * (w_max / double(n_freq));
    const double Qr = h[4 * j], Qi = h[4 * j + 1], Ur = h[4 * j + 2], Ui = h[4 * j + 3];
    const double den = Ur * Ur + Ui * Ui;
    const double Rr = (Qr * Ur + Qi * Ui) / den, Ri = (Qi * Ur - Qr * Ui) / den;  // Q/U
    if (omega) omega[j] = w;
    if (reY) reY[j] = -w * Ri;
    if (imY) imY[j] = w * Rr;
  }
  return IMRP_OK;
}

// ---- registry of the instantiation units ------------------------------------
namespace imrp {
void register_f32_small(std::vector<KernelSet<float>>&);
void register_f32_mid(std::vector<KernelSet<float>>&);
void register_f32_24(std::vector<KernelSet<float>>&);
void register_f64_small(std::vector<KernelSet<double>>&);
void register_f64_mid(std::vector<KernelSet<double>>&);
void register_f64_24(std::vector<KernelSet<double>>&);
void register_all(std::vector<KernelSet<float>>& f, std::vector<KernelSet<double>>& d) {
  register_f32_small(f);
  register_f32_mid(f);
  register_f32_24(f);
  register_f64_small(d);
  register_f64_mid(d);
  register_f64_24(d);
}
}  // namespace imrp
