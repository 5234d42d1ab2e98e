// Device-side building blocks shared by the IMRP kernels (sm_103a).
//
// Notation: Rs_l^m(x) and Is_l^m(x) are complex solid harmonics, m >= 0, with
// the symmetric scaling
//   Rs_l^m = r^l sqrt((l-m)!/(l+m)!) P_l^m(cos t) e^{i m phi}
//   Is_l^m = sqrt((l-m)!/(l+m)!) P_l^m(cos t) e^{i m phi} / r^{l+1}
// (Condon-Shortley phase), so that |Rs| <= r^l, |Is| <= r^{-(l+1)} and the
// addition theorem reads, for |y| < |x|,
//   r_<^l / r_>^{l+1} P_l(cos g) = Rs_l^0(y) Is_l^0(x) + 2 sum_{m>0} Re(conj(Rs_l^m(y)) Is_l^m(x))
// and P_l(cos g)/(|x||y|)^{l+1} is the same sum with Is(y) in place of Rs(y).
// This is how the series of G~ (Sec. 3: sum_l sum_m R_l(r,r') Y*_lm Y_lm with
// R^(p,p)_l) separates into prefix sums over inner and suffix sums over outer
// particles once they are ordered by radius.
//
// Both families follow the Cartesian recurrences (a_lm = (2l-1)/sqrt((l+m)(l-m)),
// b_lm = sqrt((l+m-1)(l-m-1)/((l+m)(l-m)))):
//   Rs_m^m = -sqrt((2m-1)/(2m)) (x+iy) Rs_{m-1}^{m-1},   Rs_0^0 = 1
//   Rs_l^m = a_lm z Rs_{l-1}^m - b_lm r^2 Rs_{l-2}^m
//   Is_m^m = -sqrt((2m-1)/(2m)) (x+iy)/r^2 Is_{m-1}^{m-1}, Is_0^0 = 1/r
//   Is_l^m = (a_lm z Is_{l-1}^m - b_lm Is_{l-2}^m) / r^2
// Derivatives (the ladder identities of these functions):
//   d_z Rs_l^m = sqrt((l+m)(l-m)) Rs_{l-1}^m
//   (d_x + i d_y) Rs_l^m = sqrt((l-m)(l-m-1)) Rs_{l-1}^{m+1}
//   (d_x - i d_y) Rs_l^m = -sqrt((l+m)(l+m-1)) Rs_{l-1}^{m-1}
//   d_z Is_l^m = -sqrt((l+1+m)(l+1-m)) Is_{l+1}^m
//   (d_x + i d_y) Is_l^m = sqrt((l+m+2)(l+m+1)) Is_{l+1}^{m+1}
//   (d_x - i d_y) Is_l^m = -sqrt((l-m+2)(l-m+1)) Is_{l+1}^{m-1}
// with X^{-m} = (-1)^m conj(X^m).
#pragma once

#include <math.h>

#include <cuda_runtime.h>
#include <stdint.h>

namespace imrp {

constexpr int kTabL = 27;  // recurrence tables cover degrees 0..26

// Number of packed real components of one moment set for degrees 1..L:
// column m = 0 holds Re for l = 1..L; columns m >= 1 hold (Re, Im) for l = m..L.
__host__ __device__ constexpr int ncomp(int L) { return L * (L + 2); }
// Index of the first component of column m (degrees 1..L).
__host__ __device__ constexpr int col_off(int L, int m) {
  return m == 0 ? 0 : L + 2 * ((m - 1) * (L + 1) - (m - 1) * m / 2);
}
// Index of (l, m, part) in a set, part 0 = Re, 1 = Im (m >= 1 only).
__host__ __device__ constexpr int comp_idx(int L, int l, int m, int part) {
  return m == 0 ? (l - 1) : col_off(L, m) + 2 * (l - m) + part;
}

// Per-step scalars written by the finalize kernel and read by the field kernel.
struct StepState {
  int64_t step;     // absolute index of the step being taken (since the last load)
  int64_t next;     // index of the next step to record
  double u;         // u_asy(t_step)
  double kick;      // kick weight of this step (dt, or dt/2 right after a load)
  int32_t sync;     // 1: velocities synchronous with x (next kick is dt/2)
  int32_t nabs_step;  // electrons absorbed at the probe in the step in progress (wall_rule 2)
  double qs_acc;      // surface charge they brought since the load (super-particle charges),
                      // folded in by the finalize kernel before each field evaluation
  int64_t nabs_total; // electrons absorbed at the probe since the load, as folded
};

// ---- radius key -------------------------------------------------------------
// The sort key of a particle: r^2 quantised to 32 bits,
// floor((r^2 - 1) 2^32 / (r_out^2 - 1)) clamped to [0, 2^32 - 1]. FP32
// positions take a fixed-point form in 64-bit integer arithmetic (FP64 runs at
// a small fraction of the FP32 rate on this part): r^2 with 56 fraction bits,
// each square S^2 2^(2e - 244) of the 24-bit significand S truncated (an error
// below 3 2^-56), times ks = round(2^40 / (r_out^2 - 1)), of which the high
// 64 bits of the 128-bit product are the key. It is monotone in r^2 and within
// one unit of the FP64 formula, which FP64 positions keep (and FP32 positions
// with a coordinate of 8 or more, or r_out^2 of 48 or more, where the
// fixed-point sum could overflow). Every kernel that writes keys for one
// context uses radius_key, so keys compare alike across them.
struct RadiusKey {
  double kscale;      // 2^32 / (r_out^2 - 1)
  uint64_t rout2_fx;  // r_out^2 2^56
  uint64_t ks_fx;     // round(2^40 / (r_out^2 - 1))
  int use_fx;         // the fixed-point form applies to FP32 positions
};
inline RadiusKey make_radius_key(double r_out) {
  RadiusKey rk{};
  const double r2 = r_out * r_out;
  rk.kscale = 4294967296.0 / (r2 - 1.0);
  const double ks = ldexp(1.0, 40) / (r2 - 1.0);
  if (r2 < 48.0 && ks < ldexp(1.0, 62)) {
    rk.use_fx = 1;
    rk.rout2_fx = uint64_t(ldexp(r2, 56));
    rk.ks_fx = uint64_t(llround(ks));
  }
  return rk;
}
constexpr uint64_t kFxOne = 1ull << 56;
// floor(v^2 2^56) for |v| < 8
__device__ __forceinline__ uint64_t sq_fx56(float v) {
  const uint32_t u = __float_as_uint(v);
  const int e8 = int((u >> 23) & 0xffu);
  if (e8 == 0) return 0;  // zero or subnormal: v^2 < 2^-252
  const uint64_t S = uint64_t((u & 0x7fffffu) | 0x800000u);
  const uint64_t S2 = S * S;  // < 2^48
  const int t = 2 * e8 - 244;  // <= 14 for |v| < 8
  if (t >= 0) return S2 << t;
  return t <= -64 ? 0 : (S2 >> (-t));
}
__device__ __forceinline__ bool key_fx_applies(float x, float y, float z, const RadiusKey& rk) {
  return rk.use_fx && fabsf(x) < 8.f && fabsf(y) < 8.f && fabsf(z) < 8.f;
}
__device__ __forceinline__ uint64_t r2_fx(float x, float y, float z) { return sq_fx56(x) + sq_fx56(y) + sq_fx56(z); }
__device__ __forceinline__ uint32_t key_of_fx(uint64_t R2, const RadiusKey& rk) {
  if (R2 <= kFxOne) return 0u;
  if (R2 >= rk.rout2_fx) return 4294967295u;
  const uint64_t hi = __umul64hi(R2 - kFxOne, rk.ks_fx);
  return hi < 4294967295ull ? uint32_t(hi) : 4294967295u;
}
__device__ __forceinline__ uint32_t key_of_r2(double r2, const RadiusKey& rk) {
  double kf = (r2 - 1.0) * rk.kscale;
  kf = kf < 0.0 ? 0.0 : (kf > 4294967295.0 ? 4294967295.0 : kf);
  return uint32_t(kf);
}
template <class T> __device__ __forceinline__ uint32_t radius_key(T x, T y, T z, const RadiusKey& rk) {
  if constexpr (sizeof(T) == 4) {
    if (key_fx_applies(x, y, z, rk)) return key_of_fx(r2_fx(x, y, z), rk);
  }
  const double xd = x, yd = y, zd = z;
  return key_of_r2(xd * xd + yd * yd + zd * zd, rk);
}

// Device error flags (bitwise or).
enum : int { kErrNaN = 1, kErrRange = 4 };

template <class T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };
template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Recurrence tables in constant memory, one copy per translation unit. The
// kernels run the recurrences on rescaled harmonics Rs_l^m / nu_lm and
// Is_l^m / nu_lm, with nu_lm = b_lm nu_{l-2,m} (nu = 1 for l <= m + 1), for which
//   R_l = an_lm z R_{l-1} - r^2 R_{l-2},   I_l = (an_lm z I_{l-1} - I_{l-2}) / r^2,
//   an_lm = a_lm nu_{l-1,m} / nu_lm:
// one product per step less. nu lies in [0.15, 1] for l <= 26; the factor is
// put back in the tile sums and in the gradient entries.
template <class T> struct Tables {
  T an[kTabL * kTabL];
  T nu[kTabL * kTabL];
  T dg[kTabL];
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Transpose reduction of 32 registers over the warp: on return lane i holds
// sum over all lanes of v[i]. 31 shuffles instead of 32 x 5.
template <class T>
__device__ __forceinline__ T warp_transpose_reduce(T (&v)[32]) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < off; ++k) {
      T send = up ? v[k] : v[k + off];
      T keep = up ? v[k + off] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) and the branchless
// orthonormal basis of Duff et al., JCGT 2017, used by the diffuse wall.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Re-injection of the absorbing wall rule (wall_rule 2): the particle that
// left is replaced, under the same id, by one entering through the outer wall
// from the bulk plasma, whose crossing flux is a flux-weighted Maxwellian of
// thermal speed sigma_v. Six 24-bit uniforms u = (k + 1/2) 2^-24 from two
// Philox blocks, counter (step, step >> 32, id, 0x494E4A30 / 0x494E4A31), key
// seed: u1, u2 the isotropic entry direction n (cos = 1 - 2 u1, phi = 2 pi u2);
// u3 the inward normal speed v_n = sigma_v sqrt(-2 ln u3) (density of the
// crossing normal speeds v exp(-v^2 / 2 sigma_v^2)); u4, u5 the tangential
// components by Box-Muller (rho = sigma_v sqrt(-2 ln u4), angle 2 pi u5) in the
// frame of n of Duff et al.; u6 the fraction of the step since the crossing,
// so the particle sits at radius r_out - u6 dt v_n (at least 1) on the ray of
// n. Evaluated in FP64 in both precisions (a few particles per step), so that
// the FP32 state is the FP64 value rounded once.
__device__ __forceinline__ double inj_u24(uint32_t w) { return (double(w >> 8) + 0.5) * (1.0 / 16777216.0); }
__device__ __forceinline__ void inject_particle(uint32_t id, uint64_t step, uint64_t seed, double r_out, double dt,
                                                double sigma_v, double* x, double* v) {
  const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
  const uint4 a = philox4x32_10(make_uint4(uint32_t(step), uint32_t(step >> 32), id, 0x494E4A30u), key);
  const uint4 b = philox4x32_10(make_uint4(uint32_t(step), uint32_t(step >> 32), id, 0x494E4A31u), key);
  const double u1 = inj_u24(a.x), u2 = inj_u24(a.y), u3 = inj_u24(a.z), u4 = inj_u24(a.w);
  const double u5 = inj_u24(b.x), u6 = inj_u24(b.y);
  const double ct = 1.0 - 2.0 * u1, st = sqrt(1.0 - ct * ct);
  double sp, cp;
  sincospi(2.0 * u2, &sp, &cp);
  const double n0 = st * cp, n1 = st * sp, n2 = ct;
  const double vn = sigma_v * sqrt(-2.0 * log(u3));
  const double rho = sigma_v * sqrt(-2.0 * log(u4));
  double s5, c5;
  sincospi(2.0 * u5, &s5, &c5);
  const double vt1 = rho * c5, vt2 = rho * s5;
  const double sg = n2 >= 0.0 ? 1.0 : -1.0;
  const double aa = -1.0 / (sg + n2);
  const double bb = n0 * n1 * aa;
  const double t10 = 1.0 + sg * n0 * n0 * aa, t11 = sg * bb, t12 = -sg * n0;
  const double t20 = bb, t21 = sg + n1 * n1 * aa, t22 = -n1;
  double r = r_out - u6 * dt * vn;
  r = r < 1.0 ? 1.0 : r;
  x[0] = r * n0; x[1] = r * n1; x[2] = r * n2;
  v[0] = -vn * n0 + vt1 * t10 + vt2 * t20;
  v[1] = -vn * n1 + vt1 * t11 + vt2 * t21;
  v[2] = -vn * n2 + vt1 * t12 + vt2 * t22;
}

// Scan groups: one group = 32 tiles (1024 particles), scanned by one warp
// with lane = tile. Sums inside a group are formed in the working precision
// T; sums across groups in FP64 (the group scan below).
constexpr int kTilesPerGroup = 32;
// Tiles in whole groups, and the row stride (in tiles) of the [component]
// [tile] arrays: whole groups plus kTilePad tiles, so that rows start at
// staggered offsets (a stride that is a multiple of 256 bytes sends the rows
// read for one tile to the same memory channels) while every row stays
// aligned for 4-wide vector access.
constexpr int kTilePad = 4;
__host__ __device__ constexpr int64_t tiles_whole(int64_t ntiles) { return (ntiles + 31) / 32 * 32; }
__host__ __device__ constexpr int64_t tile_stride(int64_t ntiles) { return tiles_whole(ntiles) + kTilePad; }

// Group scan over the FP64 group totals: the groups are cut into at most
// kGsMaxSeg segments of gs_seg_len groups, each segment summed by one CTA of
// kGsWarps warps (32 components per CTA, one per lane).
constexpr int kGsWarps = 8;
constexpr int kGsMaxSeg = 64;
__host__ __device__ inline int64_t gs_seg_len(int64_t ngroups, int gseg) {
  int64_t G = (ngroups + kGsMaxSeg - 1) / kGsMaxSeg;
  if (G < gseg) G = gseg;
  return (G + kGsWarps - 1) / kGsWarps * kGsWarps;
}
__host__ __device__ inline int64_t gs_nseg(int64_t ngroups, int gseg) {
  const int64_t G = gs_seg_len(ngroups, gseg);
  return ngroups > 0 ? (ngroups + G - 1) / G : 0;
}
// FP64 work space of the group scan for nc components: per segment the
// kGsWarps warp sums, the segment sum and the segment's base.
__host__ __device__ constexpr int64_t gs_work_doubles(int nc) { return int64_t(kGsMaxSeg) * (kGsWarps + 2) * nc; }
__host__ __device__ constexpr int gs_col_blocks(int nc) { return (nc + 31) / 32; }

// One particle of the persistent state: position, velocity and id in one
// record (32 bytes in FP32, 64 in FP64). The state is kept in the order of
// the last push and gathered into radius order by index each step; whole
// records make that gather read whole sectors instead of one sector per
// component.
template <class T> struct alignas(16) Part {
  T x, y, z, vx, vy, vz;
  uint32_t id;
  uint32_t pad[sizeof(T) == 4 ? 1 : 3];
};
static_assert(sizeof(Part<float>) == 32 && sizeof(Part<double>) == 64, "particle record sizes");

template <class T> struct MomArgs {
  const T* x;
  const T* y;
  const T* z;
  int64_t n;
  T rho;       // r_out
  T rho_inv;   // 1 / r_out: regular harmonics use x / r_out so |Rs| <= 1
  T* agg;      // [2 ncomp(L)][ntiles] tile sums, u = 2 e + s (s = 0 Rs, s = 1 Is)
  // mobile ions (species = 1): particles with id >= n_e have charge q_ion,
  // the others -1; qtile[tile] receives each tile's charge (FP64)
  int species;
  uint32_t n_e;
  T q_ion;
  const uint32_t* id;
  double* qtile;
};

// Entry tables of the gradient coefficients held in shared memory per warp.
// I part: degrees 1..L+1 (gradient of the multipole expansion in Is);
// R part: degrees 0..L-1 (gradient of the local expansion in Rs).
__host__ __device__ constexpr int nI(int L) { return (L + 1) * (L + 4) / 2; }
__host__ __device__ constexpr int nR(int L) { return L * (L + 1) / 2; }
__host__ __device__ constexpr int offI(int L, int m) {
  return m == 0 ? 0 : (L + 1) + (m - 1) * (L + 2) - (m - 1) * m / 2;
}
__host__ __device__ constexpr int offR(int L, int m) { return m * L - m * (m - 1) / 2; }
__host__ __device__ constexpr int idxI(int L, int l, int m) { return offI(L, m) + l - (m > 1 ? m : 1); }
__host__ __device__ constexpr int idxR(int L, int l, int m) { return offR(L, m) + l - m; }

template <class T> struct FieldArgs {
  const T *x, *y, *z, *vx, *vy, *vz;  // the particles in radius order
  const uint32_t* id;
  Part<T>* out;       // push mode: the pushed particle j is written to out[j]
  uint32_t* key;      // next radius key (push mode)
  uint32_t* kidx;     // identity payload for the next sort (push mode)
  int64_t n;
  const T* pfx;       // [tile][NC] in-group: Rs exclusive prefix, Is exclusive suffix
  const T* gbase;     // [ngroups][NC] Rs: sum over earlier groups; Is: sum over later groups
  const T* tot;       // [NC] totals (Is components used)
  const T* agg;       // [NC][ntiles] tile sums (read only with img_in_tile)
  int img_in_tile;    // 1: image pairs inside a tile summed directly (img_in_tile_for)
  const StepState* st;
  T* Eout;            // field mode: E in sorted order [3][n]
  int* err;
  int mode;           // 0 push, 1 field only
  int L;              // degree (equals the template L)
  T rho, rho_inv;     // r_out and 1 / r_out
  double pf;          // 1 / (4 pi n~)
  double ion_coef;    // n_ion / (r_out^3 - 1) (uniform ions, used when ion_q is null)
  const double* ion_q;  // radial ion profile (App. D): ion charge inside r_k = 1 + k h, units e n_inf R^3
  double ion_inv_h;   // 1 / h
  double ion_scale;   // n~: super-particle charges per e n_inf R^3
  int ion_n;          // nodes of ion_q (>= 2 when ion_q is set)
  double q_s;         // surface charge of the parameters (the absorbed charge st->qs_acc adds to it)
  double r_out2;      // r_out^2
  RadiusKey rk;       // the radius key of the next step's sort
  T dt;
  T r_out;
  int wall_rule;      // 0 diffuse, 1 specular, 2 absorb (probe charge to Q_S) and re-inject
  int* nabs;          // wall_rule 2: counter of the step's probe absorptions (&st->nabs_step)
  double sigma_v;     // thermal speed of the injected plasma (lambda_D / R)
  int self_image;
  int m0_only;        // 1: keep only the m = 0 terms of every degree (the paper's truncation)
  // mobile ions (species = 1): ids >= n_e are ions of charge q_ion and charge
  // to mass ratio qm_ion; the inner charge of the l = 0 term is then the
  // scanned charge of the particles inside: qgbase[group] + qpfx[tile] + the
  // charges of the lower lanes of the tile (FP64)
  int species;
  uint32_t n_e;
  T q_ion, qm_ion;
  const double* qpfx;
  const double* qgbase;
  uint32_t coll_thr;  // collision when the top 24 bits of a Philox word are below this (0: none)
  uint64_t seed;
  T f[kTabL];         // f_l of App. A
  T rhol[kTabL];      // r_out^l
  double cdrive[kTabL];  // 4 pi n~ * c_l' b^P_l for odd l (drive in units of pf)
};

// The image moments of the far field include every particle, its own tile and
// itself too; the particle's own image is then taken off analytically. When
// the self image far outweighs the field (a lone electron next to the probe:
// 1500 times in one case), that difference cancels in FP32 beyond 1e-4. So in
// FP32 contexts of at most kImgInTileMaxN particles the own tile is left out of
// the image moments and its image pairs are summed directly (a slower loop that
// only such small contexts run). From a few tiles up the ratio is of order one.
constexpr int64_t kImgInTileMaxN = 1024;
template <class T>
__host__ __device__ constexpr int img_in_tile_for(int64_t n) {
  return sizeof(T) == 4 && n <= kImgInTileMaxN ? 1 : 0;
}

// Column chunks of the far field: chunk q of the multipole (Is) part covers
// columns [chunkI(L, q), chunkI(L, q + 1)), greedily filled to at most kChunk
// gradient entries; likewise for the local (Rs) part.
constexpr int kChunk = 192;
__host__ __device__ constexpr int entI(int L, int m) { return m == 0 ? L + 1 : L + 2 - m; }
__host__ __device__ constexpr int entR(int L, int m) { return L - m; }
__host__ __device__ constexpr int chunkI(int L, int q) {
  int m = 0;
  for (int c = 0; c < q && m <= L + 1; ++c) {
    int acc = 0;
    while (m <= L + 1 && acc + entI(L, m) <= kChunk) acc += entI(L, m++);
  }
  return m;
}
__host__ __device__ constexpr int nchunkI(int L) {
  int q = 0;
  while (chunkI(L, q) <= L + 1) ++q;
  return q;
}
__host__ __device__ constexpr int chunkR(int L, int q) {
  int m = 0;
  for (int c = 0; c < q && m <= L - 1; ++c) {
    int acc = 0;
    while (m <= L - 1 && acc + entR(L, m) <= kChunk) acc += entR(L, m++);
  }
  return m;
}
__host__ __device__ constexpr int nchunkR(int L) {
  int q = 0;
  while (chunkR(L, q) <= L - 1) ++q;
  return q;
}
// Degrees at or above kChunkFrom build the far field chunk by chunk (their
// full coefficient set would limit residency to a few warps per SM); lower
// degrees build all gradient entries of both parts at once (measured faster:
// 0.80 against 0.92-0.96 ms at l_max = 16, N = 2e6, while at l_max = 24,
// N = 4e6, chunks of 192 give 3.93 against 6.02 ms).
constexpr int kChunkFrom = 20;
__host__ __device__ constexpr bool chunked(int L) { return L >= kChunkFrom; }
// Far-field loop form per degree (field kernel at N = 2e6, ms per launch,
// unrolled / rolled): l_max = 8: 0.32 / 0.35; 12: 0.64 / 0.53; 16: 0.80 /
// 0.96; 24 (N = 4e6): 3.87 / 3.79.
__host__ __device__ constexpr bool rolled_far(int L) { return L == 12 || L >= 20; }
__host__ __device__ constexpr int chunk_cap(int L) {
  return chunked(L) ? (kChunk < nI(L) ? kChunk : (nI(L) > nR(L) ? nI(L) : nR(L))) : nI(L) + nR(L);
}

// Shared memory of one warp of the field kernel: per gradient entry six
// values (d/dx, d/dy, d/dz of the Re and Im coefficient) split as
// (re.x, re.y, re.z, im.x) + (im.y, im.z), for one chunk of at most kChunk
// entries, then the 2 ncomp(L) expansion coefficients of the tile.
template <class T>
__host__ __device__ constexpr size_t field_smem_per_warp(int L) {
  return (sizeof(typename Vec4<T>::type) + sizeof(typename Vec2<T>::type)) * chunk_cap(L) +
         sizeof(T) * (2 * ncomp(L) + 2);
}

}  // namespace imrp
