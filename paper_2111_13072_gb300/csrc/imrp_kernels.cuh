// Per-degree kernel templates of the IMRP hot path: tile moments and the fused
// field gather + leapfrog push + wall + next radius key. Included by the
// instantiation units imrp_inst_*.cu, each of which owns its copy of the
// recurrence tables in constant memory.
#pragma once

#include "imrp_device.cuh"

namespace imrp {

// Recurrence tables of this translation unit (filled by init_tables<T>()).
static __constant__ Tables<float> c_tab_f;
static __constant__ Tables<double> c_tab_d;
template <class T> __device__ __forceinline__ const Tables<T>& tab();
template <> __device__ __forceinline__ const Tables<float>& tab<float>() { return c_tab_f; }
template <> __device__ __forceinline__ const Tables<double>& tab<double>() { return c_tab_d; }

// Per-degree prologue tables of the field kernel, in global memory of this
// translation unit (filled by fill_prologue_tables at initialisation), for
// every instantiated degree.
// EntryRec: one gradient entry k of the shared-memory coefficient arrays.
// Its six sources are scratch entries (the zero slot 2 ncomp(L) where a ladder
// step leaves the table); the factors are the ladder factors times nu of the
// evaluated harmonic, with the 1/2 of d/dx and d/dy, the 2 of the m > 0
// entries and the sign of a negative-m source (X^{-m} = (-1)^m conj(X^m))
// folded in, so the entry is
//   d/dx = s1r c1.re + s2 c2.re + i (s1i c1.im + s2 c2.im)
//   d/dy = (s2 c2.im - s1i c1.im) + i (s1r c1.re - s2 c2.re),  d/dz = sz c0.
struct __align__(16) EntryRec {
  int16_t src[6];   // scratch index of c1.re, c1.im, c2.re, c2.im, c0.re, c0.im
  uint16_t pad[2];
  float s1r, s1i, s2, sz;
};
constexpr int kNumDegrees = 7;  // the instantiated degrees: 1, 2, 4, 8, 12, 16, 24
__host__ __device__ constexpr int degree_at(int i) {
  return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 4 : i == 3 ? 8 : i == 4 ? 12 : i == 5 ? 16 : 24;
}
__host__ __device__ constexpr int ent_off(int L) {
  int o = 0;
  for (int i = 0; i < kNumDegrees; ++i) {
    const int d = degree_at(i);
    if (d == L) return o;
    o += nI(d) + nR(d);
  }
  return -1;
}
__host__ __device__ constexpr int comp_tab_off(int L) {
  int o = 0;
  for (int i = 0; i < kNumDegrees; ++i) {
    const int d = degree_at(i);
    if (d == L) return o;
    o += ncomp(d);
  }
  return -1;
}
constexpr int kEntTotal = ent_off(24) + nI(24) + nR(24);
constexpr int kCompTotal = comp_tab_off(24) + ncomp(24);
static __device__ EntryRec g_ent[kEntTotal];
static __device__ uint16_t g_comp[kCompTotal];  // per component: l | (drive << 8) | (m > 0) << 9

template <class T> __device__ __forceinline__ T rsqrt_t(T v);
template <> __device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double v) { return rsqrt(v); }
template <class T> __device__ __forceinline__ T fma_t(T x, T y, T z);
template <> __device__ __forceinline__ float fma_t<float>(float x, float y, float z) { return fmaf(x, y, z); }
template <> __device__ __forceinline__ double fma_t<double>(double x, double y, double z) { return fma(x, y, z); }

// Tile moments: the sums over each tile of 32 radius-sorted particles of
// q Rs_l^m(x/r_out) and q Is_l^m(x), 1 <= l <= L (q = -1 per electron).
// Two threads per tile, 16 particles each. The recurrences run column by
// column (fixed m, rising l = m + j) in a rolled loop over m, so the code
// stays small at any degree; the column sums stay in registers while the
// thread walks its particles (kMomChains at a time: independent recurrence
// chains), whose scaled positions, r_out / r^2 and diagonal terms live in
// shared memory in a [particle][thread] layout (conflict-free). The multipole
// harmonics follow from the regular ones by the Kelvin relation
//   Is_l^m(x) = Rs_l^m(x / r_out) * r_out^l / r^(2l+1),
// the scale advancing by one factor r_out / r^2 per degree. A CTA of 64
// threads takes 64 PPT particles (2 PPT tiles), PPT particles per thread,
// 32 / PPT threads per tile.
// At the end of a column the threads of each tile are combined: with two
// (PPT = 16), one shuffle per Rs/Is pair (the even lane keeps the Rs sum, the
// odd lane the Is sum); with more, a butterfly over the tile's threads, each
// then writing its share. Written: agg[u][tile], u = 2 e + s (s = 0 Rs, s = 1 Is).
constexpr int kMomThreads = 64;
constexpr int kMomPPT = 16;       // particles per thread (1024 per CTA) when that fills the GPU
constexpr int kMomPPTSmall = 4;   // particles per thread (256 per CTA) when it would leave SMs idle
constexpr int kMomBreak = 2;      // steps between the column-end tests
// particles advanced together (independent recurrence chains): four in FP32
// (N = 2e6, l_max = 16: 0.174 -> 0.168 ms against two; l_max = 24, N = 4e6:
// 0.676 -> 0.652 ms, though 150 registers lower the occupancy there), two in
// FP64, where four would spill at l_max = 24
template <class T, int L>
__host__ __device__ constexpr int mom_chains() { return sizeof(T) == 4 ? 4 : 2; }

template <class T, int L, int PPT = kMomPPT>
__host__ __device__ constexpr size_t moments_smem() {
  return sizeof(T) * 7 * PPT * (kMomThreads + 1);
}

// Body of the moments kernel for CTA `blk` of the instance whose arguments are
// `a` (a kernel parameter, or a copy in shared memory for the batched launch).
template <class T, int L, int PPT>
__device__ __forceinline__ void moments_block(const MomArgs<T>& a, int64_t blk, unsigned char* smem_raw) {
  constexpr int NT = kMomThreads;  // threads of the CTA
  constexpr int TPT = 32 / PPT;    // threads per tile
  constexpr int S = NT + 1;       // padded row
  T* sx = reinterpret_cast<T*>(smem_raw);  // x / r_out
  T* sy = sx + PPT * S;                    // y / r_out
  T* sz = sy + PPT * S;                    // z / r_out
  T* sq = sz + PPT * S;                    // r_out / r^2
  T* sRr = sq + PPT * S;                   // q Rs_m^m(x / r_out), real and imaginary
  T* sRi = sRr + PPT * S;
  T* ssc = sRi + PPT * S;                  // r_out^m / r^(2m+1)
  const Tables<T>& tb = tab<T>();
  const int th = threadIdx.x;
  const int64_t ntiles = (a.n + 31) >> 5;
  const int64_t pbase = blk * (NT * PPT);
  const T ri = a.rho_inv;
  constexpr int kMomChains = mom_chains<T, L>() < PPT ? mom_chains<T, L>() : PPT;
  // stage 1024 particles: particle k of the CTA goes to row k % PPT, column k / PPT
#pragma unroll 4
  for (int i = 0; i < PPT; ++i) {
    const int k = i * NT + th;
    const int64_t j = pbase + k;
    const bool valid = j < a.n;
    const T X = valid ? a.x[j] : T(1), Y = valid ? a.y[j] : T(0), Z = valid ? a.z[j] : T(0);
    const int o = (k % PPT) * S + k / PPT;
    const T r2 = X * X + Y * Y + Z * Z;
    sx[o] = X * ri; sy[o] = Y * ri; sz[o] = Z * ri;
    sq[o] = a.rho / r2;
    // the particle's charge seeds its harmonics: -1 for an electron, q_ion
    // for a mobile ion
    sRr[o] = valid ? ((a.species && a.id[j] >= a.n_e) ? a.q_ion : T(-1)) : T(0);
    sRi[o] = T(0);
    ssc[o] = rsqrt_t(r2);
  }
  __syncthreads();
  const int sub = th % TPT;  // this thread's part of its tile
  const bool odd = (th & 1) != 0;
  const int64_t tile = blk * (NT * PPT / 32) + th / TPT;
  if (a.species) {
    // the tile's charge (FP64): this thread's particles, then the tile's threads
    double qs = 0.0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) qs += double(sRr[p * S + th]);
#pragma unroll
    for (int d = 1; d < TPT; d <<= 1) qs += __shfl_xor_sync(0xffffffffu, qs, d);
    if (sub == 0) a.qtile[tile] = qs;
  }
  // every tile of the whole groups is written (tiles past the particles hold
  // zeros: their particles carry no charge)
  const int64_t ts = tile_stride(ntiles);
  T* const agg_t = a.agg + tile + (odd ? ts : 0);  // row u = 2 e + odd

#pragma unroll 1
  for (int m = 0; m <= L; ++m) {
    T acc[4 * (L + 1)];  // [j][R re, I re, R im, I im], l = m + j
#pragma unroll
    for (int k = 0; k < 4 * (L + 1); ++k) acc[k] = T(0);
    T cA[L + 1];  // recurrence coefficients of this column (rescaled harmonics)
#pragma unroll
    for (int j = 1; j <= L; ++j) cA[j] = m + j <= L ? tb.an[(m + j) * kTabL + m] : T(0);
    const T dg = tb.dg[m];
#pragma unroll 1
    for (int p = 0; p < PPT; p += kMomChains) {
      // a column's harmonics are the diagonal Rs_m^m = (Dr + i Di) times a real
      // p_l that obeys the column's three-term recurrence from p_m = 1
      T Zs[kMomChains], rs2[kMomChains], q[kMomChains], Dr[kMomChains], Di[kMomChains], P1[kMomChains],
          P0[kMomChains], sc[kMomChains];
#pragma unroll
      for (int u = 0; u < kMomChains; ++u) {
        const int o = (p + u) * S + th;
        const T Xs = sx[o], Ys = sy[o];
        Zs[u] = sz[o]; q[u] = sq[o];
        Dr[u] = sRr[o]; Di[u] = sRi[o]; sc[u] = ssc[o];
        if (m > 0) {  // diagonal step: Rs_m^m = dg_m (x + i y) / r_out * Rs_{m-1}^{m-1}
          const T cx = dg * Xs, cy = dg * Ys;
          const T nr = cx * Dr[u] - cy * Di[u], ni = cx * Di[u] + cy * Dr[u];
          Dr[u] = nr; Di[u] = ni; sc[u] *= q[u];
          sRr[o] = nr; sRi[o] = ni; ssc[o] = sc[u];
        }
        rs2[u] = Xs * Xs + Ys * Ys + Zs[u] * Zs[u];
        P1[u] = T(1); P0[u] = T(0);
      }
      if (m > 0) {
#pragma unroll
        for (int u = 0; u < kMomChains; ++u) {
          acc[0] += Dr[u]; acc[1] = fma_t(Dr[u], sc[u], acc[1]);
          acc[2] += Di[u]; acc[3] = fma_t(Di[u], sc[u], acc[3]);
        }
      }
#pragma unroll
      for (int j = 1; j <= L; ++j) {
        // the column ends at j = L - m; the test runs every kMomBreak steps (the
        // coefficients past the end are zero, so the extra steps add zeros to
        // sums that are not written)
        if ((j - 1) % kMomBreak == 0 && m + j > L) break;
#pragma unroll
        for (int u = 0; u < kMomChains; ++u) {
          const T az = cA[j] * Zs[u];
          const T pn = az * P1[u] - rs2[u] * P0[u];
          P0[u] = P1[u]; P1[u] = pn;
          sc[u] *= q[u];
          const T ps = pn * sc[u];
          acc[4 * j + 0] = fma_t(Dr[u], pn, acc[4 * j + 0]); acc[4 * j + 1] = fma_t(Dr[u], ps, acc[4 * j + 1]);
          acc[4 * j + 2] = fma_t(Di[u], pn, acc[4 * j + 2]); acc[4 * j + 3] = fma_t(Di[u], ps, acc[4 * j + 3]);
        }
      }
    }
    // ---- tile sums of the column, pair p = packed component e0 + p
    // (m = 0: p = l - 1, acc[4 l + s]; m > 0: p = 2 j + part, acc[2 p + s])
    const int64_t e0 = col_off(L, m);
    if constexpr (TPT == 2) {
      if (m == 0) {
#pragma unroll
        for (int p = 0; p < L; ++p) {
          const T send = odd ? acc[4 * (p + 1)] : acc[4 * (p + 1) + 1];
          const T recv = __shfl_xor_sync(0xffffffffu, send, 1);
          const T v = (odd ? acc[4 * (p + 1) + 1] : acc[4 * (p + 1)]) + recv;
          agg_t[(2 * (e0 + p)) * ts] = v * tb.nu[(p + 1) * kTabL];
        }
      } else {
        const int np = 2 * (L - m + 1);
#pragma unroll
        for (int p = 0; p < 2 * L; ++p) {
          if (p >= np) break;
          const T send = odd ? acc[2 * p] : acc[2 * p + 1];
          const T recv = __shfl_xor_sync(0xffffffffu, send, 1);
          const T v = (odd ? acc[2 * p + 1] : acc[2 * p]) + recv;
          agg_t[(2 * (e0 + p)) * ts] = v * tb.nu[(m + (p >> 1)) * kTabL + m];
        }
      }
    } else {
      // sums over the tile's threads (butterfly), then value 2 p + s of the
      // column goes out from the thread with sub = (2 p + s) % TPT
      T* const agg_c = a.agg + tile;
      if (m == 0) {
#pragma unroll
        for (int p = 0; p < L; ++p) {
#pragma unroll
          for (int sp = 0; sp < 2; ++sp) {
            T v = acc[4 * (p + 1) + sp];
#pragma unroll
            for (int d = 1; d < TPT; d <<= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if ((2 * p + sp) % TPT == sub) agg_c[(2 * (e0 + p) + sp) * ts] = v * tb.nu[(p + 1) * kTabL];
          }
        }
      } else {
        const int np = 2 * (L - m + 1);
#pragma unroll
        for (int p = 0; p < 2 * L; ++p) {
          if (p >= np) break;
#pragma unroll
          for (int sp = 0; sp < 2; ++sp) {
            T v = acc[2 * p + sp];
#pragma unroll
            for (int d = 1; d < TPT; d <<= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if ((2 * p + sp) % TPT == sub)
              agg_c[(2 * (e0 + p) + sp) * ts] = v * tb.nu[(m + (p >> 1)) * kTabL + m];
          }
        }
      }
    }
  }
}

template <class T, int L, int PPT>
__global__ void __launch_bounds__(kMomThreads) k_moments(MomArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  moments_block<T, L, PPT>(a, blockIdx.x, smem_raw);
}

// Batched moments: CTA b takes block items[b].y (of 64 PPT particles) of
// instance items[b].x, whose arguments args[items[b].x] are first copied to
// shared memory.
template <class T> __device__ __forceinline__ void copy_args(const T* src, T* dst) {
  static_assert(sizeof(T) % 4 == 0, "argument blocks are copied in words");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int k = threadIdx.x; k < int(sizeof(T) / 4); k += blockDim.x) d[k] = s[k];
}
template <class T, int L, int PPT>
__global__ void __launch_bounds__(kMomThreads) k_moments_batch(const MomArgs<T>* __restrict__ args,
                                                               const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MomArgs<T> sa;
  const int2 it = items[blockIdx.x];
  copy_args(args + it.x, &sa);
  __syncthreads();
  moments_block<T, L, PPT>(sa, it.y, smem_raw);
}

// Constants of the scaled Legendre recurrences of the near field. With
// c_l = (2l-1)!!/l! (the leading coefficient of P_l), q_l = s^l P_l(u) / c_l
// follows q_{l+1} = (s u) q_l - g_l s^2 q_{l-1}, g_l = l^2 / (4 l^2 - 1)
// (Bonnet's recurrence divided by c_{l+1}); and with eps_{l+1} = (2l+1) c_l,
// e_l = s^{l-1} P'_l(u) / eps_l follows e_{l+1} = r_l s^2 e_{l-1} + q_l,
// r_l = eps_{l-1} / eps_{l+1} (from P'_{l+1} = P'_{l-1} + (2l+1) P_l).
__host__ __device__ constexpr double leg_c(int l) {
  double c = 1.0;
  for (int k = 1; k <= l; ++k) c *= double(2 * k - 1) / double(k);
  return c;
}
__host__ __device__ constexpr double leg_g(int l) { return double(l) * l / (4.0 * l * l - 1.0); }
__host__ __device__ constexpr double leg_eps(int l) { return l == 0 ? 1.0 : double(2 * l - 1) * leg_c(l - 1); }
__host__ __device__ constexpr double leg_r(int l) { return leg_eps(l - 1) / leg_eps(l + 1); }

// One warp per tile. Phase 1 forms the tile's expansion coefficients, phase 2
// their gradients (ladder identities) in shared memory, phase 3 evaluates the
// far field of all other tiles, the near field of the pairs inside the tile,
// the l = 0 terms, and then pushes the particle.
// Body of the field kernel for warp `warp` of a CTA of `wpb` warps, tile
// `tile` of the instance whose arguments are `a`.
template <class T, int L>
__device__ __forceinline__ void field_tile(const FieldArgs<T>& a, unsigned char* smem_raw, int warp, int wpb,
                                           int64_t tile) {
  using V4 = typename Vec4<T>::type;
  using V2 = typename Vec2<T>::type;
  constexpr int NC = 2 * ncomp(L);
  constexpr int NI = nI(L), NR = nR(L);
  constexpr int NE = NI + NR;
  const Tables<T>& tb = tab<T>();
  const unsigned lane = lane_id();
  const int64_t ntiles = (a.n + 31) >> 5;
  if (tile >= ntiles) return;  // warp-uniform; no block-wide barrier below
  const int64_t ts = tile_stride(ntiles);
  constexpr int CH = chunk_cap(L);
  V4* coefA = reinterpret_cast<V4*>(smem_raw) + size_t(warp) * CH;
  V2* coefB = reinterpret_cast<V2*>(reinterpret_cast<V4*>(smem_raw) + size_t(wpb) * CH) + size_t(warp) * CH;
  T* sc = reinterpret_cast<T*>(reinterpret_cast<V2*>(reinterpret_cast<V4*>(smem_raw) + size_t(wpb) * CH) +
                               size_t(wpb) * CH) + size_t(warp) * (NC + 2);
  const int64_t g = tile / kTilesPerGroup;
  const double u_drive = a.st->u;
  const T kick = T(a.st->kick);
  const double q_s = a.q_s + a.st->qs_acc;  // with the charge absorbed at the probe so far
  const bool img_in_tile = img_in_tile_for<T>(0) && a.img_in_tile;  // FP32 contexts only

  // the particle of this lane, loaded first so that its latency overlaps the
  // prologue
  const int64_t j = tile * 32 + lane;
  const bool valid = j < a.n;
  T X = valid ? a.x[j] : T(1), Y = valid ? a.y[j] : T(0), Z = valid ? a.z[j] : T(0);
  T VX = T(0), VY = T(0), VZ = T(0);
  if (a.mode == 0 && valid) { VX = a.vx[j]; VY = a.vy[j]; VZ = a.vz[j]; }
  // mobile ions: ids from n_e on are ions; qneg = -q (1 for an electron), 0 on an empty lane
  const bool is_ion = a.species && valid && a.id[j] >= a.n_e;
  const T qneg = valid ? (is_ion ? -a.q_ion : T(1)) : T(0);

  // ---- phase 1: cI (coefficients of Is, s = 0) and cR (of Rs(x/r_out), s = 1),
  // with the gradient's scale -pf (and 1/r_out for Rs) applied, and the zero slot.
  // The loop has a fixed trip count and is unrolled, so that all loads of the
  // scan carries are in flight at once.
  const T mpf = T(-a.pf), mpfr = T(-a.pf) * a.rho_inv;
  if (lane == 0) { sc[NC] = T(0); sc[NC + 1] = T(0); }
  {
    const V2* pt = reinterpret_cast<const V2*>(a.pfx + tile * NC);  // [tile][u]: (A, B) pairs
    const T* gb = a.gbase + g * NC;
    const T* at = a.agg + tile;   // [u][tile]
    const uint16_t* ctab = g_comp + comp_tab_off(L);
    constexpr int NIT = (NC / 2 + 31) / 32;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int e = int(lane) + 32 * it;
      if (e < NC / 2) {
        const uint16_t cr = ctab[e];
        const int l = cr & 0xff;
        const T rl = a.rhol[l];  // r_out^l
        const V2 ab = pt[e];
        const T A = gb[2 * e] + ab.x;      // sum over inner tiles of q Rs(x_i / r_out)
        const T B = gb[2 * e + 1] + ab.y;  // sum over outer tiles of q Is(x_i)
        // sum of q Is(x_i) of the image term: over all particles, or over the
        // other tiles when the own tile's image pairs are summed directly
        const T W = img_in_tile ? a.tot[2 * e + 1] - at[(2 * e + 1) * ts] : a.tot[2 * e + 1];
        T cI = rl * A - a.f[l] * W;
        if ((cr >> 8) & 1) cI += T(u_drive * a.cdrive[l]);
        T cR = rl * B;
        if (a.m0_only && ((cr >> 9) & 1)) { cI = T(0); cR = T(0); }
        sc[2 * e] = cI * mpf;
        sc[2 * e + 1] = cR * mpfr;
      }
    }
  }
  __syncwarp();
  // ---- phase 3: the particle of this lane
  const T r2 = X * X + Y * Y + Z * Z;
  const T ir2 = T(1) / r2;
  const T ir = rsqrt_t(r2);
  T Ex = T(0), Ey = T(0), Ez = T(0);
  T Fx = T(0), Fy = T(0), Fz = T(0);  // second accumulator chain (Im parts)

  // ---- far field, in column chunks of at most kChunk gradient entries: the
  // entries of a chunk are formed in shared memory (phase 2) and evaluated at
  // once; the recurrence's diagonal term is carried from chunk to chunk in
  // registers.
  const EntryRec* etab = g_ent + ent_off(L);
  auto build = [&](int k0, int k1) {
    __syncwarp();
    constexpr int NB = (CH + 31) / 32;  // at most CH entries per build
#pragma unroll 1
    for (int it = 0; it < NB; ++it) {
      const int k = k0 + int(lane) + 32 * it;
      if (k < k1) {
        const EntryRec er = etab[k];
        const T c1r = sc[er.src[0]], c1i = sc[er.src[1]], c2r = sc[er.src[2]], c2i = sc[er.src[3]],
                c0r = sc[er.src[4]], c0i = sc[er.src[5]];
        const T s1r = T(er.s1r), s1i = T(er.s1i), s2 = T(er.s2), sz = T(er.sz);
        V4 ca;
        V2 cb;
        ca.x = s1r * c1r + s2 * c2r;  // d/dx, d/dy, d/dz (Re), d/dx (Im)
        ca.y = s2 * c2i - s1i * c1i;
        ca.z = sz * c0r;
        ca.w = s1i * c1i + s2 * c2i;
        cb.x = s1r * c1r - s2 * c2r;  // d/dy, d/dz (Im)
        cb.y = sz * c0i;
        coefA[k - k0] = ca;
        coefB[k - k0] = cb;
      }
    }
    __syncwarp();
  };

  if constexpr (!chunked(L)) build(0, NE);  // all entries of both parts at once
  // Two forms of the far-field loops, chosen per degree by measurement
  // (rolled_far): fully unrolled (compile-time coefficients and entry
  // addresses), or with the columns m >= 1 in a rolled loop (the recurrence
  // over l = m + j unrolled, with a uniform exit at the column end; the real
  // column m = 0 peeled), which keeps the code and the register count small.
  if constexpr (!rolled_far(L)) {
    // multipole part: sum over Is_l^m(x), 1 <= l <= L+1
    {
      const T Zir2 = Z * ir2;
      T dr = ir, di = T(0);
      constexpr int QI = chunked(L) ? nchunkI(L) : 1;
#pragma unroll
      for (int q = 0; q < QI; ++q) {
        const int m0 = chunked(L) ? chunkI(L, q) : 0, m1 = chunked(L) ? chunkI(L, q + 1) : L + 2;
        const int k0 = chunked(L) ? offI(L, m0) : 0;
        if constexpr (chunked(L)) build(k0, offI(L, m1));
#pragma unroll
        for (int m = m0; m < m1; ++m) {
          if (m > 0) {
            const T c = tb.dg[m];
            const T ex = c * X * ir2, ey = c * Y * ir2;
            const T nr = ex * dr - ey * di, ni = ex * di + ey * dr;
            dr = nr;
            di = ni;
          }
          // the column is (dr + i di) times the real p_l, which obeys the
          // same recurrence from p_m = 1: sum the contractions with p_l, then
          // multiply by the diagonal once per column
          T p1 = T(1), p0 = T(0);
          T Sx = T(0), Sy = T(0), Sz = T(0), Tx = T(0), Ty = T(0), Tz = T(0);
#pragma unroll
          for (int l = m; l <= L + 1; ++l) {
            if (l > m) {
              const T A = tb.an[l * kTabL + m] * Zir2;
              const T pn = A * p1 - ir2 * p0;
              p0 = p1; p1 = pn;
            }
            if (l >= 1) {
              const V4 ca = coefA[idxI(L, l, m) - k0];
              if (l == m) {
                Sx = ca.x; Sy = ca.y; Sz = ca.z;
              } else {
                Sx += ca.x * p1; Sy += ca.y * p1; Sz += ca.z * p1;
              }
              if (m > 0) {
                const V2 cb = coefB[idxI(L, l, m) - k0];
                if (l == m) {
                  Tx = ca.w; Ty = cb.x; Tz = cb.y;
                } else {
                  Tx += ca.w * p1; Ty += cb.x * p1; Tz += cb.y * p1;
                }
              }
            }
          }
          Ex += dr * Sx; Ey += dr * Sy; Ez += dr * Sz;
          if (m > 0) { Fx += di * Tx; Fy += di * Ty; Fz += di * Tz; }
        }
      }
    }
    // local part: sum over Rs_l^m(x / r_out), 0 <= l <= L-1
    {
      const T Xs = X * a.rho_inv, Ys = Y * a.rho_inv, Zs = Z * a.rho_inv;
      const T rs2 = r2 * a.rho_inv * a.rho_inv;
      T dr = T(1), di = T(0);
      constexpr int QR = chunked(L) ? nchunkR(L) : 1;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int m0 = chunked(L) ? chunkR(L, q) : 0, m1 = chunked(L) ? chunkR(L, q + 1) : L;
        const int k0 = chunked(L) ? NI + offR(L, m0) : 0;
        if constexpr (chunked(L)) build(k0, NI + offR(L, m1));
#pragma unroll
        for (int m = m0; m < m1; ++m) {
          if (m > 0) {
            const T c = tb.dg[m];
            const T ex = c * Xs, ey = c * Ys;
            const T nr = ex * dr - ey * di, ni = ex * di + ey * dr;
            dr = nr;
            di = ni;
          }
          T p1 = T(1), p0 = T(0);
          T Sx = T(0), Sy = T(0), Sz = T(0), Tx = T(0), Ty = T(0), Tz = T(0);
#pragma unroll
          for (int l = m; l <= L - 1; ++l) {
            if (l > m) {
              const T A = tb.an[l * kTabL + m] * Zs;
              const T pn = A * p1 - rs2 * p0;
              p0 = p1; p1 = pn;
            }
            const V4 ca = coefA[NI + idxR(L, l, m) - k0];
            if (l == m) {
              Sx = ca.x; Sy = ca.y; Sz = ca.z;
            } else {
              Sx += ca.x * p1; Sy += ca.y * p1; Sz += ca.z * p1;
            }
            if (m > 0) {
              const V2 cb = coefB[NI + idxR(L, l, m) - k0];
              if (l == m) {
                Tx = ca.w; Ty = cb.x; Tz = cb.y;
              } else {
                Tx += ca.w * p1; Ty += cb.x * p1; Tz += cb.y * p1;
              }
            }
          }
          Ex += dr * Sx; Ey += dr * Sy; Ez += dr * Sz;
          if (m > 0) { Fx += di * Tx; Fy += di * Ty; Fz += di * Tz; }
        }
      }
    }

  } else {
    // multipole part: sum over Is_l^m(x), 1 <= l <= L+1
    {
      const T Zir2 = Z * ir2;
      T dr = ir, di = T(0);
      constexpr int QI = chunked(L) ? nchunkI(L) : 1;
#pragma unroll
      for (int q = 0; q < QI; ++q) {
        const int m0 = chunked(L) ? chunkI(L, q) : 0, m1 = chunked(L) ? chunkI(L, q + 1) : L + 2;
        const int k0 = chunked(L) ? offI(L, m0) : 0;
        if constexpr (chunked(L)) build(k0, offI(L, m1));
        if (m0 == 0) {
          T c1 = dr, c0 = T(0);
#pragma unroll
          for (int l = 1; l <= L + 1; ++l) {
            const T A = tb.an[l * kTabL] * Zir2, B = ir2;
            const T n1 = A * c1 - B * c0;
            c0 = c1; c1 = n1;
            const V4 ca = coefA[idxI(L, l, 0) - k0];
            Ex += ca.x * c1; Ey += ca.y * c1; Ez += ca.z * c1;
          }
        }
  #pragma unroll 1
        for (int m = m0 > 1 ? m0 : 1; m < m1; ++m) {
          const T c = tb.dg[m];
          {
            const T ex = c * X * ir2, ey = c * Y * ir2;
            const T nr = ex * dr - ey * di, ni = ex * di + ey * dr;
            dr = nr;
            di = ni;
          }
          const int eb = offI(L, m) - k0 - (m > 1 ? m : 1);  // entry of degree l: eb + l
          T cA[L + 1];  // the column's recurrence coefficients, loaded before its steps
#pragma unroll
          for (int j = 1; j <= L; ++j) cA[j] = m + j <= L + 1 ? tb.an[(m + j) * kTabL + m] : T(0);
          T p1 = T(1), p0 = T(0);  // the column is (dr + i di) p_l
          T Sx, Sy, Sz, Tx, Ty, Tz;
          {
            const V4 ca = coefA[eb + m];
            const V2 cb = coefB[eb + m];
            Sx = ca.x; Sy = ca.y; Sz = ca.z;
            Tx = ca.w; Ty = cb.x; Tz = cb.y;
          }
#pragma unroll
          for (int j = 1; j <= L; ++j) {
            const int l = m + j;
            if (l > L + 1) break;
            const T A = cA[j] * Zir2;
            const T pn = A * p1 - ir2 * p0;
            p0 = p1; p1 = pn;
            const V4 ca = coefA[eb + l];
            const V2 cb = coefB[eb + l];
            Sx += ca.x * p1; Sy += ca.y * p1; Sz += ca.z * p1;
            Tx += ca.w * p1; Ty += cb.x * p1; Tz += cb.y * p1;
          }
          Ex += dr * Sx; Ey += dr * Sy; Ez += dr * Sz;
          Fx += di * Tx; Fy += di * Ty; Fz += di * Tz;
        }
      }
    }
    // local part: sum over Rs_l^m(x / r_out), 0 <= l <= L-1
    {
      const T Xs = X * a.rho_inv, Ys = Y * a.rho_inv, Zs = Z * a.rho_inv;
      const T rs2 = r2 * a.rho_inv * a.rho_inv;
      T dr = T(1), di = T(0);
      constexpr int QR = chunked(L) ? nchunkR(L) : 1;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int m0 = chunked(L) ? chunkR(L, q) : 0, m1 = chunked(L) ? chunkR(L, q + 1) : L;
        const int k0 = chunked(L) ? NI + offR(L, m0) : 0;
        if constexpr (chunked(L)) build(k0, NI + offR(L, m1));
        if (m0 == 0) {
          T c1 = dr, c0 = T(0);
#pragma unroll
          for (int l = 0; l <= L - 1; ++l) {
            if (l > 0) {
              const T A = tb.an[l * kTabL] * Zs, B = rs2;
              const T n1 = A * c1 - B * c0;
              c0 = c1; c1 = n1;
            }
            const V4 ca = coefA[NI + idxR(L, l, 0) - k0];
            Ex += ca.x * c1; Ey += ca.y * c1; Ez += ca.z * c1;
          }
        }
  #pragma unroll 1
        for (int m = m0 > 1 ? m0 : 1; m < m1; ++m) {
          const T c = tb.dg[m];
          {
            const T ex = c * Xs, ey = c * Ys;
            const T nr = ex * dr - ey * di, ni = ex * di + ey * dr;
            dr = nr;
            di = ni;
          }
          const int eb = NI + offR(L, m) - k0 - m;  // entry of degree l: eb + l
          T cA[L];  // the column's recurrence coefficients, loaded before its steps
#pragma unroll
          for (int j = 1; j <= L - 1; ++j) cA[j] = m + j <= L - 1 ? tb.an[(m + j) * kTabL + m] : T(0);
          T p1 = T(1), p0 = T(0);
          T Sx, Sy, Sz, Tx, Ty, Tz;
          {
            const V4 ca = coefA[eb + m];
            const V2 cb = coefB[eb + m];
            Sx = ca.x; Sy = ca.y; Sz = ca.z;
            Tx = ca.w; Ty = cb.x; Tz = cb.y;
          }
#pragma unroll
          for (int j = 1; j <= L - 1; ++j) {
            const int l = m + j;
            if (l > L - 1) break;
            const T A = cA[j] * Zs;
            const T pn = A * p1 - rs2 * p0;
            p0 = p1; p1 = pn;
            const V4 ca = coefA[eb + l];
            const V2 cb = coefB[eb + l];
            Sx += ca.x * p1; Sy += ca.y * p1; Sz += ca.z * p1;
            Tx += ca.w * p1; Ty += cb.x * p1; Tz += cb.y * p1;
          }
          Ex += dr * Sx; Ey += dr * Sy; Ez += dr * Sz;
          Fx += di * Tx; Fy += di * Ty; Fz += di * Tz;
        }
      }
    }

  }
  Ex += Fx; Ey += Fy; Ez += Fz;

  // near field: the direct pair terms r_<^l / r_>^{l+1} P_l (l >= 1) of the
  // particles of this tile (their image terms are separable and are part of
  // the far field). Lower lane = smaller sorted radius = inner.
  {
    const T rk = r2 * ir;
    const T ex = X * ir, ey = Y * ir, ez = Z * ir;
    T Nx = T(0), Ny = T(0), Nz = T(0);  // sum of grad phi (phi = sum_l r_<^l/r_>^{l+1} P_l), weighted by -q
    // -q of this particle (1 for an electron), 0 for the empty lanes of a
    // ragged tile: a partner's contribution to my field is weighted by its
    // -q (pm), mine to the partner's by vmask
    const T vmask = qneg;
#pragma unroll 1
    for (int s = 1; s <= 16 && !a.m0_only; ++s) {
      const int src = (lane + s) & 31;
      const T pex = __shfl_sync(0xffffffffu, ex, src);
      const T pey = __shfl_sync(0xffffffffu, ey, src);
      const T pez = __shfl_sync(0xffffffffu, ez, src);
      const T prk = __shfl_sync(0xffffffffu, rk, src);
      const T pir = __shfl_sync(0xffffffffu, ir, src);
      const T pm = __shfl_sync(0xffffffffu, vmask, src);
      const bool me_inner = int(lane) < src;
      const T sr = me_inner ? rk * pir : prk * ir;  // r_inner / r_outer
      const T uu = ex * pex + ey * pey + ez * pez;
      // Q_l = s^l P_l(u) and E_l = s^(l-1) P'_l(u), scaled (leg_c, leg_eps) so
      // that each step is one product with a per-degree constant less:
      // S0 = sum Q_l, S1 = sum l Q_l, S2 = sum s E_l = sum s^l P'_l(u).
      const T x1 = sr * uu, y2 = sr * sr;
      T qm = T(1), q = x1, em = T(0), e = T(1);
      T S0 = x1, S1 = x1, S2 = T(1);
#pragma unroll
      for (int l = 1; l < L; ++l) {
        const T qn = fma_t(x1, q, -(T(leg_g(l)) * y2) * qm);
        const T en = l == 1 ? q : fma_t(T(leg_r(l)) * y2, em, q);
        qm = q; q = qn; em = e; e = en;
        S0 = fma_t(T(leg_c(l + 1)), q, S0);
        S1 = fma_t(T((l + 1) * leg_c(l + 1)), q, S1);
        S2 = fma_t(T(leg_eps(l + 1)), e, S2);
      }
      S2 *= sr;
      // grad of phi = sum_l r_i^l/r_o^{l+1} P_l(u): at the inner end
      // (S1 r^_i + S2 (r^_o - u r^_i)) / (r_i r_o), at the outer end
      // (-(S0 + S1) r^_o + S2 (r^_i - u r^_o)) / r_o^2; radial (r) and angular
      // (a) factors of my end and of the partner's, with the validity mask
      const T gab = ir * pir;                          // 1 / (r_i r_o)
      const T go2 = me_inner ? pir * pir : ir * ir;    // 1 / r_o^2
      const T in_r = S1 * gab, in_a = S2 * gab;
      const T out_r = -(S0 + S1) * go2, out_a = S2 * go2;
      const T mr = (me_inner ? in_r : out_r) * pm, ma = (me_inner ? in_a : out_a) * pm;
      Nx += mr * ex + ma * (pex - uu * ex);
      Ny += mr * ey + ma * (pey - uu * ey);
      Nz += mr * ez + ma * (pez - uu * ez);
      if (s < 16) {
        const T pr = (me_inner ? out_r : in_r) * vmask, pa = (me_inner ? out_a : in_a) * vmask;
        const T tx = pr * pex + pa * (ex - uu * pex), ty = pr * pey + pa * (ey - uu * pey),
                tz = pr * pez + pa * (ez - uu * pez);
        const int dst = (lane - s) & 31;
        Nx += __shfl_sync(0xffffffffu, tx, dst);
        Ny += __shfl_sync(0xffffffffu, ty, dst);
        Nz += __shfl_sync(0xffffffffu, tz, dst);
      }
    }
#pragma unroll 1
    for (int s = 1; s <= 16 && a.m0_only; ++s) {
      // m = 0 truncation: sum_l r_i^l / r_o^{l+1} P_l(cos t_i) P_l(cos t_o)
      const int src = (lane + s) & 31;
      const T pex = __shfl_sync(0xffffffffu, ex, src);
      const T pey = __shfl_sync(0xffffffffu, ey, src);
      const T pez = __shfl_sync(0xffffffffu, ez, src);
      const T prk = __shfl_sync(0xffffffffu, rk, src);
      const T pir = __shfl_sync(0xffffffffu, ir, src);
      const T pm = __shfl_sync(0xffffffffu, vmask, src);
      const bool me_inner = int(lane) < src;
      const T ri = me_inner ? rk : prk;
      const T iri = me_inner ? ir : pir, iro = me_inner ? pir : ir;
      const T xix = me_inner ? ex : pex, xiy = me_inner ? ey : pey, xiz = me_inner ? ez : pez;
      const T xox = me_inner ? pex : ex, xoy = me_inner ? pey : ey, xoz = me_inner ? pez : ez;
      const T sr = ri * iro;
      const T ui = xiz, uo = xoz;  // cos of the polar angles
      T Pim = T(1), Pi = ui, Dim = T(0), Di = T(1);
      T Pom = T(1), Po = uo, Dom = T(0), Do = T(1);
      T sp = sr;  // s^l at l = 1
      T A1 = T(0), A3 = T(0), C1 = T(0), C2 = T(0);
#pragma unroll
      for (int l = 1; l <= L; ++l) {
        if (l > 1) {
          const T cl = T(2 * l - 1) / T(l), dl = T(l - 1) / T(l);
          const T Pin = cl * ui * Pi - dl * Pim, Pon = cl * uo * Po - dl * Pom;
          const T Din = Dim + T(2 * l - 1) * Pi, Don = Dom + T(2 * l - 1) * Po;
          Pim = Pi; Pi = Pin; Dim = Di; Di = Din;
          Pom = Po; Po = Pon; Dom = Do; Do = Don;
          sp *= sr;
        }
        const T pp = Pi * Po;
        A1 += T(l + 1) * sp * pp;
        A3 += T(l) * sp * pp;
        const T wgt = sp * iro;
        C1 += wgt * Pi * Do;
        C2 += wgt * Di * Po;
      }
      // grad at the outer point and at the inner point
      const T go = -A1 * iro * iro, gi = A3 * iro * iri;
      const T ogx = go * xox - C1 * iro * uo * xox, ogy = go * xoy - C1 * iro * uo * xoy,
              ogz = go * xoz + C1 * iro * (T(1) - uo * xoz);
      const T igx = gi * xix - C2 * iri * ui * xix, igy = gi * xiy - C2 * iri * ui * xiy,
              igz = gi * xiz + C2 * iri * (T(1) - ui * xiz);
      Nx += pm * (me_inner ? igx : ogx); Ny += pm * (me_inner ? igy : ogy); Nz += pm * (me_inner ? igz : ogz);
      if (s < 16) {
        const T tx = vmask * (me_inner ? ogx : igx), ty = vmask * (me_inner ? ogy : igy),
                tz = vmask * (me_inner ? ogz : igz);
        const int dst = (lane - s) & 31;
        Nx += __shfl_sync(0xffffffffu, tx, dst);
        Ny += __shfl_sync(0xffffffffu, ty, dst);
        Nz += __shfl_sync(0xffffffffu, tz, dst);
      }
    }
    if (img_in_tile) {
      // image terms of the other particles of the tile: grad at x_k of
      // -sum_l f_l P_l(u) / (r_k r_i)^{l+1}, u = x^_k . x^_i (m0_only:
      // P_l(cos t_k) P_l(cos t_i) in place of P_l(u)); d is the direction
      // along which u varies (x^_i, or z^ for m0_only)
      T Gx = T(0), Gy = T(0), Gz = T(0);
#pragma unroll 1
      for (int s = 1; s < 32; ++s) {
        const int src = (lane + s) & 31;
        const T pex = __shfl_sync(0xffffffffu, ex, src);
        const T pey = __shfl_sync(0xffffffffu, ey, src);
        const T pez = __shfl_sync(0xffffffffu, ez, src);
        const T pir = __shfl_sync(0xffffffffu, ir, src);
        const T pm = __shfl_sync(0xffffffffu, vmask, src);
        const T uu = a.m0_only ? ez : ex * pex + ey * pey + ez * pez;
        const T dx = a.m0_only ? T(0) : pex, dy = a.m0_only ? T(0) : pey, dz = a.m0_only ? T(1) : pez;
        const T tau = ir * pir;
        T Pm = T(1), P = uu, Dm = T(0), D = T(1);  // P_l(uu), P'_l(uu)
        T Qm = T(1), Q = a.m0_only ? pez : T(1);  // P_l(cos t_i) (m0_only), else 1
        T tp = tau * tau;                         // tau^{l+1}
        T hr = T(0), ha = T(0);
#pragma unroll 1
        for (int l = 1; l <= L; ++l) {
          if (l > 1) {
            const T Pn = (T(2 * l - 1) * uu * P - T(l - 1) * Pm) / T(l);
            const T Dn = Dm + T(2 * l - 1) * P;
            Pm = P; P = Pn; Dm = D; D = Dn;
            if (a.m0_only) {
              const T Qn = (T(2 * l - 1) * pez * Q - T(l - 1) * Qm) / T(l);
              Qm = Q; Q = Qn;
            }
            tp *= tau;
          }
          const T wgt = a.f[l] * tp * Q;
          hr += T(l + 1) * wgt * P;
          ha += wgt * D;
        }
        Gx += pm * (hr * ex - ha * (dx - uu * ex));
        Gy += pm * (hr * ey - ha * (dy - uu * ey));
        Gz += pm * (hr * ez - ha * (dz - uu * ez));
      }
      Nx += ir * Gx; Ny += ir * Gy; Nz += ir * Gz;
    }
    // E = -pf sum_i q_i grad phi (N holds the sum weighted by -q_i)
    const T pfT = T(a.pf);
    Ex += pfT * Nx; Ey += pfT * Ny; Ez += pfT * Nz;
  }

  // l = 0: electrons inside (sorted index j), ions inside, surface charge;
  // then the self-image correction. The image moments of the far field sum
  // over all particles, the particle itself included, so without the self
  // image (self_image = 0) its own image field is taken off again; with
  // img_in_tile the own tile is left out of them, so with the self image
  // (self_image = 1) it is added. The count difference is formed in FP64 from
  // the exact FP64 radius of the (FP32 or FP64) position.
  {
    const double xd = double(X), yd = double(Y), zd = double(Z);
    const double r2d = xd * xd + yd * yd + zd * zd;  // exact for FP32 positions
    double rd;
    if constexpr (sizeof(T) == 4) {
      // FP32 root refined by one Newton step in FP64 (no FP64 sqrt or division)
      const float rf = r2 * ir;
      rd = double(rf) + (r2d - double(rf) * double(rf)) * double(0.5f * ir);
    } else {
      rd = sqrt(r2d);
    }
    // inner charge in units of e: ions inside minus electrons inside (+ Q_S); the
    // difference is small, so it is formed in FP64 and then scaled in T
    double qion;
    if (a.ion_q) {
      // radial profile, linear between the nodes, constant outside [1, r_out]
      const double t = fmin(fmax((rd - 1.0) * a.ion_inv_h, 0.0), double(a.ion_n - 1));
      const int k = min(int(t), a.ion_n - 2);
      const double q0 = __ldg(a.ion_q + k), q1 = __ldg(a.ion_q + k + 1);
      qion = a.ion_scale * fma(t - double(k), q1 - q0, q0);
    } else {
      qion = a.ion_coef * (r2d * rd - 1.0);
    }
    double qmob;  // charge of the mobile particles inside (sorted before this one)
    if (a.species) {
      double qc = valid ? -double(qneg) : 0.0, incl = qc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, incl, d);
        if (int(lane) >= d) incl += t;
      }
      qmob = a.qgbase[g] + a.qpfx[tile] + (incl - qc);
    } else {
      qmob = -double(j);  // j electrons inside
    }
    const double qin = qion + (q_s + qmob);
    const T er = T(qin) * (T(a.pf) * ir2 * ir);  // multiplies x (gives r^ / r^2)
    Ex += er * X; Ey += er * Y; Ez += er * Z;
    const int self_sign = img_in_tile ? (a.self_image ? 1 : 0) : (a.self_image ? 0 : -1);
    if (self_sign != 0 && a.m0_only) {
      // own image with the m = 0 kernel: pf sum_l f_l r^{-(2l+3)} [(l+1) P_l^2 r^ - P_l P_l' (z^ - u r^)]
      const T u = Z * ir;
      T Pm = T(1), P = u, Dm = T(0), D = T(1), rp = ir2 * ir2 * ir;  // r^{-5} at l = 1
      T hr = T(0), ha = T(0);
#pragma unroll
      for (int l = 1; l <= L; ++l) {
        if (l > 1) {
          const T Pn = (T(2 * l - 1) * u * P - T(l - 1) * Pm) / T(l);
          const T Dn = Dm + T(2 * l - 1) * P;
          Pm = P; P = Pn; Dm = D; D = Dn;
          rp *= ir2;
        }
        hr += a.f[l] * T(l + 1) * P * P * rp;
        ha += a.f[l] * P * D * rp;
      }
      const T pfT = T(self_sign * a.pf) * qneg;
      // r^ = x / r, z^ - u r^ = (0, 0, 1) - u x / r
      Ex += pfT * (hr * X * ir + ha * u * X * ir);
      Ey += pfT * (hr * Y * ir + ha * u * Y * ir);
      Ez += pfT * (hr * Z * ir - ha * (T(1) - u * Z * ir));
    } else if (self_sign != 0) {
      // the particle's own image: pf sum_l f_l (l+1) r^{-(2l+3)} r^
      T h = T(0);
#pragma unroll
      for (int l = L; l >= 1; --l) h = h * ir2 + a.f[l] * T(l + 1);
      const T es = T(self_sign * a.pf) * qneg * h * ir2 * ir2 * ir2;  // r^{-(2l+3)} r^ = ir2^{l-1} ir2^3 x
      Ex += es * X; Ey += es * Y; Ez += es * Z;
    }
  }

  if (a.mode == 1) {
    if (valid) {
      a.Eout[j] = Ex;
      a.Eout[a.n + j] = Ey;
      a.Eout[2 * a.n + j] = Ez;
    }
    return;
  }
  if (!valid) return;

  // ---- leapfrog: v += kick (q/m) E (q/m = -1 for an electron); x += dt v
  if (is_ion) {
    const T kq = kick * a.qm_ion;
    VX += kq * Ex; VY += kq * Ey; VZ += kq * Ez;
  } else {
    VX -= kick * Ex; VY -= kick * Ey; VZ -= kick * Ez;
  }
  X += a.dt * VX; Y += a.dt * VY; Z += a.dt * VZ;

  // ---- walls (Sec. 4): mirror the radius back, keep the speed
  {
    double rr = 0.0;
    bool hit = false;
    {
      const T rt = X * X + Y * Y + Z * Z;
      const bool near_wall = rt < T(1.0 + 1e-5) || rt > T(a.r_out2 * (1.0 - 1e-5));
      if (near_wall) {  // the exact test in FP64 only near a wall
        const double xd = double(X), yd = double(Y), zd = double(Z);
        rr = xd * xd + yd * yd + zd * zd;  // exact for FP32 positions
        hit = rr < 1.0 || rr > a.r_out2;
      }
    }
    if (hit && a.wall_rule == 2) {
      // absorbed (at the probe its charge joins Q_S) and replaced from the outer wall
      if (rr < 1.0) atomicAdd(a.nabs, 1);
      double xn[3], vn[3];
      inject_particle(a.id[j], uint64_t(a.st->step), a.seed, double(a.r_out), double(a.dt), a.sigma_v, xn, vn);
      X = T(xn[0]); Y = T(xn[1]); Z = T(xn[2]);
      VX = T(vn[0]); VY = T(vn[1]); VZ = T(vn[2]);
    } else if (hit) {
      const double xd = double(X), yd = double(Y), zd = double(Z);
      const double rd = sqrt(rr);
      const bool inner = rr < 1.0;
      double rn = inner ? 2.0 - rd : 2.0 * double(a.r_out) - rd;
      rn = rn < 1.0 ? 1.0 : (rn > double(a.r_out) ? double(a.r_out) : rn);
      const double e0 = xd / rd, e1 = yd / rd, e2 = zd / rd;
      X = T(e0 * rn); Y = T(e1 * rn); Z = T(e2 * rn);
      if (a.wall_rule == 1) {
        const T vr = VX * T(e0) + VY * T(e1) + VZ * T(e2);
        VX -= T(2) * vr * T(e0); VY -= T(2) * vr * T(e1); VZ -= T(2) * vr * T(e2);
      } else {
        const T sgn = inner ? T(1) : T(-1);
        const T n0 = sgn * T(e0), n1 = sgn * T(e1), n2 = sgn * T(e2);
        const T speed = sqrt(VX * VX + VY * VY + VZ * VZ);
        const uint64_t stp = uint64_t(a.st->step);
        const uint4 o = philox4x32_10(
            make_uint4(uint32_t(stp), uint32_t(stp >> 32), a.id[j], 0x494D5250u),
            make_uint2(uint32_t(a.seed), uint32_t(a.seed >> 32)));
        const T u1 = T(o.x >> 8) * T(1.0 / 16777216.0);
        const T u2 = T(o.y >> 8) * T(1.0 / 16777216.0);
        const T ca = T(1) - u1;
        const T sa = sqrt(T(1) - ca * ca);
        T sp, cp;
        if constexpr (sizeof(T) == 4) sincospif(T(2) * u2, &sp, &cp);
        else sincospi(T(2) * u2, &sp, &cp);
        const T sg = n2 >= T(0) ? T(1) : T(-1);
        const T aa = T(-1) / (sg + n2);
        const T bb = n0 * n1 * aa;
        const T t10 = T(1) + sg * n0 * n0 * aa, t11 = sg * bb, t12 = -sg * n0;
        const T t20 = bb, t21 = sg + n1 * n1 * aa, t22 = -n1;
        VX = speed * (ca * n0 + sa * (cp * t10 + sp * t20));
        VY = speed * (ca * n1 + sa * (cp * t11 + sp * t21));
        VZ = speed * (ca * n2 + sa * (cp * t12 + sp * t22));
      }
    }
    if (a.coll_thr != 0u && !is_ion) {
      // electron-neutral collision: isotropic elastic scattering with
      // probability 1 - exp(-nu dt) (Philox counter (step, step >> 32, id,
      // 0x434F4C4C), key = seed; top 24 bits below the threshold)
      const uint64_t stp = uint64_t(a.st->step);
      const uint4 o = philox4x32_10(make_uint4(uint32_t(stp), uint32_t(stp >> 32), a.id[j], 0x434F4C4Cu),
                                    make_uint2(uint32_t(a.seed), uint32_t(a.seed >> 32)));
      if ((o.x >> 8) < a.coll_thr) {
        const T speed = sqrt(VX * VX + VY * VY + VZ * VZ);
        const T u1 = T(o.y >> 8) * T(1.0 / 16777216.0);
        const T u2 = T(o.z >> 8) * T(1.0 / 16777216.0);
        const T ct = T(1) - T(2) * u1;
        const T st = sqrt(T(1) - ct * ct);
        T sp, cp;
        if constexpr (sizeof(T) == 4) sincospif(T(2) * u2, &sp, &cp);
        else sincospi(T(2) * u2, &sp, &cp);
        VX = speed * st * cp;
        VY = speed * st * sp;
        VZ = speed * ct;
      }
    }
    const bool fin = isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(VX) && isfinite(VY) && isfinite(VZ);
    if (!fin) atomicOr(a.err, kErrNaN);
    a.key[j] = fin ? radius_key<T>(X, Y, Z, a.rk) : 0u;
    a.kidx[j] = uint32_t(j);
  }
  Part<T> rec;
  rec.x = X; rec.y = Y; rec.z = Z;
  rec.vx = VX; rec.vy = VY; rec.vz = VZ;
  rec.id = a.id[j];
  a.out[j] = rec;
}

// Register budget: in FP32, at least 3 CTAs of 256 threads per SM (80
// registers): ptxas otherwise settles at 64 with spills in the far-field
// loops; FP64 keeps its ~124.
template <class T>
__host__ __device__ constexpr int field_min_blocks() { return sizeof(T) == 4 ? 3 : 1; }

template <class T, int L>
__global__ void __launch_bounds__(256, field_min_blocks<T>()) k_field(FieldArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  // tiles in decreasing order: the particle rows written last (still in L2) first
  field_tile<T, L>(a, smem_raw, warp, wpb, int64_t(gridDim.x - 1 - blockIdx.x) * wpb + warp);
}

// Batched field: the instances of one degree and precision in one launch. CTA
// b takes the tiles items[b].y .. items[b].y + wpb - 1 of instance items[b].x,
// whose arguments args[items[b].x] are first copied to shared memory (a warp
// past its instance's last tile returns at once, as in the single launch).
template <class T, int L>
__global__ void __launch_bounds__(256, field_min_blocks<T>()) k_field_batch(const FieldArgs<T>* __restrict__ args,
                                                     const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FieldArgs<T> sa;
  const int2 it = items[blockIdx.x];
  copy_args(args + it.x, &sa);
  __syncthreads();
  const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  field_tile<T, L>(sa, smem_raw, warp, wpb, int64_t(it.y) + warp);
}

}  // namespace imrp
