// Degree-independent kernels of the IMRP hot path: the radius radix sort, state
// reorder, key generation, loading, the FP64 scans of the tile moments, the
// per-step finalize (drive u_asy and the Q_diff tally), and the spectrum sums.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "imrp_internal.h"

namespace imrp {

// ============================================================================
// Radix sort: stable LSD passes of 8-bit digits, and a wide first pass of
// 9-bit digits for the bucket sort of large arrays. Each CTA owns
// kSortTile = 2048 consecutive keys in a striped layout (item i of thread t is
// key base + i*256 + t), which keeps the slot order (item, warp, lane) equal
// to the key order, so the local ranks below are stable. ND: digits of the
// pass (256 or 512); hist holds ND rows of nblk block counts.
// ============================================================================
template <int ND>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys,
                                                           int64_t n, int shift, int64_t nblk,
                                                           uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[ND];
  for (int d = threadIdx.x; d < ND; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  const int nvalid = n - base < kSortTile ? int(n - base) : kSortTile;
  const unsigned lane = threadIdx.x & 31;
  uint32_t k[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int o = i * kSortThreads + int(threadIdx.x);
    k[i] = o < nvalid ? keys[base + o] : 0u;
  }
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    // a warp holds 32 consecutive keys: when they share the digit (nearly
    // sorted input), one atomic adds all 32
    const bool ok = i * kSortThreads + int(threadIdx.x) < nvalid;
    const unsigned d = (k[i] >> shift) & unsigned(ND - 1);
    const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
    if (__all_sync(0xffffffffu, ok && d == d0)) {
      if (lane == 0) atomicAdd(&h[d0], 32u);
    } else if (ok) {
      atomicAdd(&h[d], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < ND; d += kSortThreads) hist[int64_t(d) * nblk + blockIdx.x] = h[d];
}

// Exclusive prefix over the kSortThreads threads of a CTA of the per-thread
// values v (warp shuffles, then the warp sums through wsum); *total gets the
// sum over the CTA. All threads call it; the caller separates two uses of wsum
// by a barrier.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* wsum, uint32_t* total = nullptr) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= unsigned(o)) s += x;
  }
  if (lane == 31) wsum[warp] = s;
  __syncthreads();
  uint32_t woff = 0, tot = 0;
#pragma unroll
  for (unsigned w = 0; w < kSortThreads / 32; ++w) {
    const uint32_t x = wsum[w];
    woff += w < warp ? x : 0u;
    tot += x;
  }
  if (total) *total = tot;
  return woff + s - v;
}

// Exclusive scan of one digit's row hist[d][0..nblk) in place; the row total
// goes to rowtot[d]. One CTA per digit.
__global__ void __launch_bounds__(kSortThreads) k_sort_rowscan(uint32_t* __restrict__ hist, int64_t nblk,
                                                              uint32_t* __restrict__ rowtot) {
  constexpr int R = 8;  // consecutive entries per thread, loaded together
  __shared__ uint32_t wsum[kSortThreads / 32];
  uint32_t* row = hist + int64_t(blockIdx.x) * nblk;
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nblk; b0 += int64_t(kSortThreads) * R) {
    const int64_t i0 = b0 + int64_t(R) * threadIdx.x;
    uint32_t v[R], sum = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = i0 + r < nblk ? row[i0 + r] : 0u;
      sum += v[r];
    }
    uint32_t tot;
    uint32_t run = carry + block_excl_scan(sum, wsum, &tot);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (i0 + r < nblk) row[i0 + r] = run;
      run += v[r];
    }
    carry += tot;
    __syncthreads();  // wsum reuse
  }
  if (threadIdx.x == 0) rowtot[blockIdx.x] = carry;
}

// Lanes of the warp whose digit equals this lane's (bits BITS of d), among
// the lanes with ok set: one ballot per digit bit.
template <int BITS>
__device__ __forceinline__ unsigned digit_peers(unsigned d, bool ok) {
  unsigned p = __ballot_sync(0xffffffffu, ok);
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const unsigned m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    p &= ((d >> b) & 1u) ? m : ~m;
  }
  return p;
}

// Scatter of one pass. Warp w of the block owns the keys base + 256 w ..
// base + 256 w + 255 (item i of lane l is key base + 256 w + 32 i + l), so the
// order (warp, item, lane) is the key order. The items of a warp are ranked
// one after the other against the warp's running digit counts whist[w][d];
// a key's block-local position is then (start of its digit in the block) +
// (keys of that digit in earlier warps) + (its rank in its warp): stable.
// The block's keys and slots are staged in shared memory in that order, so
// that consecutive threads write consecutive positions of each digit's run
// in the output (coalesced even when the digits are uniformly spread). Thread
// t owns the digits DPT t .. DPT t + DPT - 1 in the per-digit steps. With 256
// digits about 22 KB of shared memory and at most 36 registers per thread (7
// blocks per SM, so all blocks of N = 2e6 keys are resident at once); with
// 512 digits about 29 KB. Ranking by __match_any_sync: the keys of a warp
// arrive nearly sorted, so few distinct top digits (faster here than ballots).
template <int ND>
__global__ void __launch_bounds__(kSortThreads, ND == 256 ? 7 : 6) k_sort_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, int64_t nblk,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ rowtot) {
  constexpr int kWarps = kSortThreads / 32;
  constexpr int DPT = ND / kSortThreads;
  static_assert(kSortItems * 32 <= 256 && kSortTile <= 65535, "per-warp counts fit 16 bits");
  __shared__ __align__(16) uint16_t whist[kWarps][ND];
  __shared__ __align__(16) uint32_t sk[kSortTile];
  __shared__ __align__(16) uint32_t sv[kSortTile];
  __shared__ uint32_t dbase[ND];   // global start of digit d for this block
  __shared__ uint32_t lstart[ND];  // block-local start of digit d
  __shared__ uint32_t wsum[kWarps];
  const unsigned t = threadIdx.x, lane = t & 31, warp = t >> 5;
  {
    uint4* z = reinterpret_cast<uint4*>(&whist[0][0]);
    for (int k = t; k < kWarps * ND * 2 / 16; k += kSortThreads) z[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  // exclusive scan of the digit totals -> global start of each digit
  {
    uint32_t c[DPT], sum = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      c[k] = rowtot[DPT * t + k];
      sum += c[k];
    }
    uint32_t off = block_excl_scan(sum, wsum);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      const unsigned d = DPT * t + k;
      dbase[d] = off + hist[int64_t(d) * nblk + blockIdx.x];
      off += c[k];
    }
  }
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  const int64_t wbase = base + int64_t(warp) * (32 * kSortItems);
  const unsigned lt = (1u << lane) - 1u;
  uint32_t key[kSortItems];
  uint32_t wrank[(kSortItems + 3) / 4] = {};  // rank in the warp (< 256), one byte per item
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t idx = wbase + 32 * i + lane;
    key[i] = idx < n ? kin[idx] : 0u;
  }
  __syncthreads();  // whist zeroed, wsum consumed
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const bool ok = wbase + 32 * i + lane < n;
    const unsigned d = ok ? ((key[i] >> shift) & unsigned(ND - 1)) : unsigned(ND);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned before = ok ? unsigned(whist[warp][d]) : 0u;
    wrank[i / 4] |= (before + __popc(peers & lt)) << (8 * (i % 4));
    __syncwarp();
    if (ok && lane == unsigned(__ffs(peers) - 1)) whist[warp][d] = uint16_t(before + __popc(peers));
    __syncwarp();
  }
  __syncthreads();
  // block count of each digit of this thread; whist[w][d] becomes the count in warps before w
  uint32_t total[DPT], tsum = 0;
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    const unsigned d = DPT * t + k;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = whist[w][d];
      whist[w][d] = uint16_t(run);
      run += c;
    }
    total[k] = run;
    tsum += run;
  }
  // block-local digit starts: exclusive scan of the block counts over d
  {
    __syncthreads();  // wsum reuse
    uint32_t off = block_excl_scan(tsum, wsum);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      lstart[DPT * t + k] = off;
      off += total[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t idx = wbase + 32 * i + lane;
    if (idx < n) {
      const unsigned d = (key[i] >> shift) & unsigned(ND - 1);
      const uint32_t lpos = lstart[d] + whist[warp][d] + ((wrank[i / 4] >> (8 * (i % 4))) & 255u);
      sk[lpos] = key[i];
      sv[lpos] = vin[idx];
    }
  }
  __syncthreads();
  const int64_t nvalid = n - base < kSortTile ? n - base : kSortTile;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int p = i * kSortThreads + int(t);
    if (p < nvalid) {
      const uint32_t k = sk[p];
      const unsigned d = (k >> shift) & unsigned(ND - 1);
      const uint32_t g = dbase[d] + (uint32_t(p) - lstart[d]);
      kout[g] = k;
      vout[g] = sv[p];
    }
  }
}

// Sort of one top-digit bucket by the key bits below the digit, in one CTA.
// The first pass of the sort (on the top byte, or on the top 9 bits, over the
// whole array) leaves the keys of bucket b contiguous and in their input
// order; this CTA then runs three stable LSD passes over its bucket, bytes 0,
// 1, 2 (with a 9-bit top digit the top bit of byte 2 is the same for the
// whole bucket), which need no global synchronisation: in shared memory when
// the bucket fits (the first pass reads the bucket from global memory, the
// last writes it back), else between the two global key/value buffers (in L2;
// the CTA alone touches that range). A pass: the scan of the byte's digit
// counts, then the bucket in chunks of NT * kBsItems keys in order; each warp
// ranks its 256 keys (item i of lane l is chunk slot 256 w + 32 i + l) against
// its running digit counts, the warps' counts are scanned per digit, and each
// key goes to (digit start) + (keys of that digit in earlier chunks and warps)
// + (its rank in its warp): stable. A warp whose part of the chunk holds no
// keys, and items past the end, skip the ranking. The peers of a key in its
// warp come from one ballot per digit bit (the low bytes are spread evenly
// over the digits, where that is faster than __match_any_sync). The next
// byte's counts are gathered as keys are placed. The result is the
// permutation of a stable LSD sort on all four bytes.
constexpr int kBsItems = 8;

template <int NT> struct BsShared {
  uint32_t cnt[2][256];              // digit counts of this pass's byte and of the next
  uint32_t dst[256];                 // output place of the next key of digit d
  uint16_t whist[NT / 32][256];      // per-warp counts, then the counts of earlier warps
  uint32_t wsum[8];
};

// One pass over len (< 2^31) keys (slots 0 .. len-1 of ki/vi into ko/vo), digit =
// byte at `shift`; cnt: this byte's counts; cnx (or null): zeroed here, then
// the counts of the byte at shift + 8.
template <int NT, class K>
__device__ __forceinline__ void bucket_pass(const K* ki, const K* vi, K* ko, K* vo, int len, int shift,
                                            const uint32_t* cnt, uint32_t* cnx, BsShared<NT>& sh) {
  constexpr int kWarps = NT / 32, kChunk = NT * kBsItems;
  const unsigned t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t c = 0, s1 = 0;
  if (t < 256) {
    c = cnt[t];
    s1 = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, s1, o);
      if (lane >= unsigned(o)) s1 += x;
    }
    if (lane == 31) sh.wsum[warp] = s1;
    if (cnx) cnx[t] = 0u;
  }
  __syncthreads();
  if (t < 256) {
    uint32_t off = 0;
    for (unsigned w = 0; w < warp; ++w) off += sh.wsum[w];
    sh.dst[t] = off + s1 - c;
  }
  for (int c0 = 0; c0 < len; c0 += kChunk) {
    for (int k = t; k < kWarps * 256; k += NT) (&sh.whist[0][0])[k] = 0;
    __syncthreads();
    const int wb = c0 + int(warp) * (32 * kBsItems);
    const int nv = len - wb;  // keys of this warp's range that exist (warp-uniform)
    uint32_t key[kBsItems], val[kBsItems];
    uint32_t wrank[(kBsItems + 1) / 2] = {};
    if (nv > 0) {
#pragma unroll
      for (int i = 0; i < kBsItems; ++i) {
        const int o = 32 * i + int(lane);
        key[i] = o < nv ? ki[wb + o] : 0u;
        val[i] = o < nv ? vi[wb + o] : 0u;
      }
#pragma unroll
      for (int i = 0; i < kBsItems; ++i) {
        if (32 * i >= nv) break;
        const bool ok = 32 * i + int(lane) < nv;
        const unsigned d = ok ? ((key[i] >> shift) & 255u) : 256u;
        const unsigned peers = digit_peers<8>(d, ok);
        const unsigned before = ok ? unsigned(sh.whist[warp][d]) : 0u;
        wrank[i / 2] |= (before + __popc(peers & lt)) << (16 * (i % 2));
        __syncwarp();
        if (ok && lane == unsigned(__ffs(peers) - 1)) sh.whist[warp][d] = uint16_t(before + __popc(peers));
        __syncwarp();
      }
    }
    __syncthreads();
    uint32_t total = 0;
    if (t < 256) {
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t x = sh.whist[w][t];
        sh.whist[w][t] = uint16_t(total);
        total += x;
      }
    }
    __syncthreads();
    if (nv > 0) {
#pragma unroll
      for (int i = 0; i < kBsItems; ++i) {
        if (32 * i >= nv) break;
        if (32 * i + int(lane) < nv) {
          const unsigned d = (key[i] >> shift) & 255u;
          const uint32_t g = sh.dst[d] + sh.whist[warp][d] + ((wrank[i / 2] >> (16 * (i % 2))) & 0xffffu);
          ko[g] = key[i];
          vo[g] = val[i];
          if (cnx) atomicAdd(&cnx[(key[i] >> (shift + 8)) & 255u], 1u);
        }
      }
    }
    __syncthreads();
    if (t < 256) sh.dst[t] += total;
  }
  __syncthreads();  // this pass's writes are visible to the CTA's next pass
}

// Counts of the low byte of keys[0 .. len) into cnt (loads in flight together).
template <int NT>
__device__ __forceinline__ void count_low_byte(const uint32_t* keys, int64_t len, uint32_t* cnt) {
  for (int64_t i0 = 0; i0 < len; i0 += int64_t(NT) * kBsItems) {
    uint32_t k[kBsItems];
#pragma unroll
    for (int i = 0; i < kBsItems; ++i) {
      const int64_t idx = i0 + int64_t(i) * NT + threadIdx.x;
      k[i] = idx < len ? keys[idx] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kBsItems; ++i)
      if (i0 + int64_t(i) * NT + threadIdx.x < len) atomicAdd(&cnt[k[i] & 255u], 1u);
  }
}

// cap: the largest segment sorted in shared memory (dynamic shared memory of
// 16 cap bytes: two key and two value buffers). With rowtot (nd digit totals
// of the first pass), CTA c sorts the top-digit buckets g c .. g c + g - 1 of
// k1/v1 into k0/v0: by bytes 0..2 when g = 1, by all four bytes when a CTA
// takes several buckets (small instances: fewer, fuller CTAs). Without rowtot
// (one CTA, n_single <= cap), the whole array k0/v0 by all four bytes, in
// place. MINB: resident CTAs per SM asked of the register allocation.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_bucket_sort(uint32_t* k1, uint32_t* v1, uint32_t* k0, uint32_t* v0,
                                                          const uint32_t* __restrict__ rowtot, int64_t n_single,
                                                          int cap, int g, int nd) {
  extern __shared__ __align__(16) uint32_t sbuf[];
  __shared__ BsShared<NT> sh;
  __shared__ uint32_t s_len[8];
  __shared__ int64_t s_start, s_n;
  const unsigned t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned b0 = blockIdx.x * unsigned(g), b1 = b0 + unsigned(g);
  // segment start and length: the sizes of the buckets before it and in it
  // (thread t < 256 adds the digits nd / 256 t .. nd / 256 (t + 1) - 1)
  if (t < 256) {
    uint32_t v = 0u, w = 0u;
    if (rowtot) {
      const unsigned per = unsigned(nd) / 256u;
      for (unsigned k = 0; k < per; ++k) {
        const unsigned d = per * t + k;
        const uint32_t c = rowtot[d];
        if (d < b0) v += c;
        else if (d < b1) w += c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_down_sync(0xffffffffu, v, o);
      w += __shfl_down_sync(0xffffffffu, w, o);
    }
    if (lane == 0) {
      sh.wsum[warp] = v;
      s_len[warp] = w;
    }
    sh.cnt[0][t] = 0u;
  }
  __syncthreads();
  if (t == 0) {
    int64_t a = 0, m = 0;
    for (int k = 0; k < 8; ++k) {
      a += sh.wsum[k];
      m += s_len[k];
    }
    s_start = a;
    s_n = m;
  }
  __syncthreads();
  const bool single = rowtot == nullptr;
  const int64_t start = s_start;
  const int64_t len = single ? n_single : s_n;
  if (len == 0) return;  // uniform over the CTA
  const bool all4 = single || g > 1;  // the segment spans several top digits
  uint32_t *sk = single ? k0 : k1 + start, *sv = single ? v0 : v1 + start;
  uint32_t *gk0 = k0 + start, *gv0 = v0 + start, *gk1 = k1 + start, *gv1 = v1 + start;
  count_low_byte<NT>(sk, len, sh.cnt[0]);
  __syncthreads();
  if (len <= cap) {
    // first pass from global memory, the middle ones in shared memory, the
    // last into global memory
    uint32_t *ka = sbuf, *va = sbuf + cap, *kb = sbuf + 2 * cap, *vb = sbuf + 3 * cap;
    bucket_pass<NT>(sk, sv, ka, va, int(len), 0, sh.cnt[0], sh.cnt[1], sh);
    bucket_pass<NT>(ka, va, kb, vb, int(len), 8, sh.cnt[1], sh.cnt[0], sh);
    if (all4) {
      bucket_pass<NT>(kb, vb, ka, va, int(len), 16, sh.cnt[0], sh.cnt[1], sh);
      bucket_pass<NT>(ka, va, gk0, gv0, int(len), 24, sh.cnt[1], nullptr, sh);
    } else {
      bucket_pass<NT>(kb, vb, gk0, gv0, int(len), 16, sh.cnt[0], nullptr, sh);
    }
  } else {  // a segment (never the single array) larger than cap: through L2
    bucket_pass<NT>(gk1, gv1, gk0, gv0, int(len), 0, sh.cnt[0], sh.cnt[1], sh);
    bucket_pass<NT>(gk0, gv0, gk1, gv1, int(len), 8, sh.cnt[1], sh.cnt[0], sh);
    if (all4) {
      bucket_pass<NT>(gk1, gv1, gk0, gv0, int(len), 16, sh.cnt[0], sh.cnt[1], sh);
      bucket_pass<NT>(gk0, gv0, gk1, gv1, int(len), 24, sh.cnt[1], nullptr, sh);
      for (int64_t i = t; i < len; i += NT) {
        gk0[i] = gk1[i];
        gv0[i] = gv1[i];
      }
    } else {
      bucket_pass<NT>(gk1, gv1, gk0, gv0, int(len), 16, sh.cnt[0], nullptr, sh);
    }
  }
}

// Largest N for the bucket sort: the buckets of a uniform shell (density in
// r^2 up to 1.45 times its mean) must fit the shared-memory capacity; beyond
// it they take the global path, and one CTA's share of the work outweighs the
// saved passes (N = 4e6: 0.256 ms against 0.222 for the four global passes;
// N = 1.6e7: 0.91 against 0.74 ms, both with the 8-bit first pass).
constexpr int64_t kBucketSortMaxN = 2250000;
constexpr int kBsCapMax = 13312;  // 208 KB of buckets beside the static shared memory
constexpr int64_t kBsSmallN = 1 << 19;  // up to here an 8-bit first pass (256 buckets), beyond a 9-bit one (512)
constexpr int64_t kBsSingleN = 3072;     // up to here, one CTA sorts everything (N = 1000: 13 us)
// shared-memory capacity for segments of g of nd buckets: three times the mean
// segment with 256 buckets; 1.5 times with 512 (at N = 2e6 two CTAs per SM of
// 101 KB, 94 KB of them buckets; a larger bucket goes through L2)
inline int bucket_cap(int64_t n, int g, int nd) {
  const int64_t mean = int64_t(g) * n / nd;
  int64_t c = ((nd == 256 ? 3 * mean : mean + mean / 2) + 255) / 256 * 256;
  if (c < 2048) c = 2048;
  return int(c < kBsCapMax ? c : kBsCapMax);
}

cudaError_t set_sort_attributes() {
  const cudaError_t e = cudaFuncSetAttribute(k_bucket_sort<256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             16 * kBsCapMax);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_bucket_sort<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 * kBsCapMax);
}

const uint32_t* launch_radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist,
                                  int64_t n, int first_byte, cudaStream_t s, bool shared_gpu) {
  if (n <= 1) return v0;
  const int64_t nblk = sort_blocks(n);
  if (first_byte == 0 && n <= kBsSingleN) {
    // one CTA sorts the whole array in shared memory, all four bytes
    const int cap = int((n + 255) / 256 * 256);
    k_bucket_sort<256, 3><<<1, 256, size_t(16) * cap, s>>>(k1, v1, k0, v0, nullptr, n, cap, 256, 256);
    return v0;
  }
  if (first_byte == 0 && n <= kBucketSortMaxN) {
    // the top digit over the whole array into nd contiguous buckets (k0 -> k1),
    // then the bits below it per bucket (into k0): 256 buckets (the top byte)
    // up to kBsSmallN keys, 512 (the top 9 bits, buckets of ~3900 keys at
    // N = 2e6, two CTAs per SM) beyond. Alone on the GPU, one CTA per bucket
    // (the most parallel); sharing it (a batch), a small instance takes
    // segments of several buckets, about 2048 keys per CTA (fewer CTAs, all
    // four bytes each): the same permutation either way
    const bool wide = n > kBsSmallN;
    const int nd = wide ? 512 : 256, shift = wide ? 23 : 24;
    uint32_t* rowtot = hist + int64_t(nd) * nblk;
    int g = 1;
    while (shared_gpu && g < nd && int64_t(g) * 2 * n <= int64_t(2048) * nd) g *= 2;
    const int cap = bucket_cap(n, g, nd);
    if (wide) {
      k_sort_hist<512><<<unsigned(nblk), kSortThreads, 0, s>>>(k0, n, shift, nblk, hist);
      k_sort_rowscan<<<512, kSortThreads, 0, s>>>(hist, nblk, rowtot);
      k_sort_scatter<512><<<unsigned(nblk), kSortThreads, 0, s>>>(k0, v0, k1, v1, n, shift, nblk, hist, rowtot);
      k_bucket_sort<256, 2><<<unsigned(512 / g), 256, size_t(16) * cap, s>>>(k1, v1, k0, v0, rowtot, 0, cap, g,
                                                                             512);
    } else {
      k_sort_hist<256><<<unsigned(nblk), kSortThreads, 0, s>>>(k0, n, shift, nblk, hist);
      k_sort_rowscan<<<256, kSortThreads, 0, s>>>(hist, nblk, rowtot);
      k_sort_scatter<256><<<unsigned(nblk), kSortThreads, 0, s>>>(k0, v0, k1, v1, n, shift, nblk, hist, rowtot);
      k_bucket_sort<256, 3><<<unsigned(256 / g), 256, size_t(16) * cap, s>>>(k1, v1, k0, v0, rowtot, 0, cap, g,
                                                                             256);
    }
    return v0;
  }
  uint32_t* rowtot = hist + 256 * nblk;
  uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int pass = first_byte; pass < 4; ++pass) {
    const int shift = 8 * pass;
    k_sort_hist<256><<<unsigned(nblk), kSortThreads, 0, s>>>(ki, n, shift, nblk, hist);
    k_sort_rowscan<<<256, kSortThreads, 0, s>>>(hist, nblk, rowtot);
    k_sort_scatter<256><<<unsigned(nblk), kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, nblk, hist, rowtot);
    uint32_t* tk = ki; ki = ko; ko = tk;
    uint32_t* tv = vi; vi = vo; vo = tv;
  }
  return vi;
}

// ============================================================================
// State movement
// ============================================================================
template <class T> struct SoA { T* d[6]; uint32_t* id; };

// Gather of the state into radius order: sorted position j takes the record
// perm[j] (one particle: whole sectors) and splits it into the component
// arrays the moments and field kernels read.
template <class T>
__global__ void k_reorder(const Part<T>* __restrict__ src, SoA<T> dst, const uint32_t* __restrict__ perm,
                          int64_t n) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Part<T> p = src[perm[j]];
  dst.d[0][j] = p.x; dst.d[1][j] = p.y; dst.d[2][j] = p.z;
  dst.d[3][j] = p.vx; dst.d[4][j] = p.vy; dst.d[5][j] = p.vz;
  dst.id[j] = p.id;
}

template <class T>
void launch_reorder(const Part<T>* src, T* const* dst, uint32_t* id_dst, const uint32_t* perm, int64_t n,
                    cudaStream_t s) {
  SoA<T> d;
  for (int c = 0; c < 6; ++c) d.d[c] = dst[c];
  d.id = id_dst;
  k_reorder<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, d, perm, n);
}

// Radius keys of the state in its storage order (after a load or a field
// evaluation; a step's field kernel writes the next keys itself).
template <class T>
__global__ void k_keys(const Part<T>* __restrict__ st, uint32_t* __restrict__ key, uint32_t* __restrict__ kidx,
                       int64_t n, RadiusKey rk) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Part<T> p = st[j];
  key[j] = radius_key<T>(p.x, p.y, p.z, rk);
  kidx[j] = uint32_t(j);
}

template <class T>
void launch_keys(const Part<T>* st, uint32_t* key, uint32_t* kidx, int64_t n, double r_out, cudaStream_t s) {
  k_keys<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(st, key, kidx, n, make_radius_key(r_out));
}

// FP64 -> FP32 rounding to nearest, ties to even (IEEE 754 binary64 ->
// binary32), in integer operations: FP64 arithmetic, conversions included,
// runs at a small fraction of the FP32 rate on this part and bound the load
// kernel. Normal results keep the top 23 of the 52 mantissa bits and round on
// the other 29 (a carry steps the exponent, up to infinity at the top of the
// range); subnormal results shift the full 53-bit significand into the
// subnormal units and round on the shifted-out bits; overflow gives infinity,
// NaN stays a (quiet) NaN.
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const uint64_t b = uint64_t(__double_as_longlong(d));
  const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
  const int e = int(b >> 52) & 0x7ff;
  const uint64_t m = b & 0xfffffffffffffull;
  uint32_t bits;
  if (e >= 897 && e <= 1150) {  // normal FP32 result
    const uint32_t top = uint32_t(m >> 29), rest = uint32_t(m) & 0x1fffffffu;
    bits = (uint32_t(e - 896) << 23) | top;
    if (rest > 0x10000000u || (rest == 0x10000000u && (top & 1u))) bits += 1u;
  } else if (e == 0x7ff) {  // infinity, NaN
    bits = 0x7f800000u | (m ? (0x400000u | uint32_t(m >> 29)) : 0u);
  } else if (e > 1150) {    // overflow
    bits = 0x7f800000u;
  } else if (e >= 873) {    // subnormal result: M 2^(e - 926) units of 2^-149
    const uint64_t M = m | (1ull << 52);
    const int sh = 926 - e;  // 30 .. 53
    const uint64_t q = M >> sh, r = M & ((1ull << sh) - 1), h = 1ull << (sh - 1);
    bits = uint32_t(q) + ((r > h || (r == h && (q & 1u))) ? 1u : 0u);
  } else {                  // below half the smallest subnormal
    bits = 0u;
  }
  return __uint_as_float(sign | bits);
}
// FP32 -> FP64, exact, in integer operations: the exponent rebiased and the
// mantissa widened; a subnormal is normalised from its leading bit.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = uint64_t(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint64_t bits;
  if (e == 255u) {
    bits = 0x7ff0000000000000ull | (uint64_t(m) << 29);
  } else if (e != 0u) {
    bits = (uint64_t(e + 896u) << 52) | (uint64_t(m) << 29);
  } else if (m == 0u) {
    bits = 0;
  } else {  // m 2^-149, leading bit at p
    const int p = 31 - __clz(m);
    bits = (uint64_t(p - 149 + 1023) << 52) | ((uint64_t(m) << (52 - p)) & 0xfffffffffffffull);
  }
  return __longlong_as_double(int64_t(sign | bits));
}
template <class T> __device__ __forceinline__ T narrow(double d);
template <> __device__ __forceinline__ float narrow<float>(double d) { return f64_to_f32_rn(d); }
template <> __device__ __forceinline__ double narrow<double>(double d) { return d; }
template <class T> __device__ __forceinline__ double widen(T v);
template <> __device__ __forceinline__ double widen<float>(float v) { return f32_to_f64(v); }
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }

// Host FP64 [n][3] positions and velocities into the state, ids 0..n-1, with
// the radius keys of that order, so that the first step after a load needs no
// separate key pass.
template <class T>
__global__ void k_load(const double* __restrict__ xs, const double* __restrict__ vs,
                       const uint32_t* __restrict__ ids, Part<T>* __restrict__ st, uint32_t* __restrict__ key,
                       uint32_t* __restrict__ kidx, int64_t n, double r_out2, RadiusKey rk, int* err) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double v[6];
  bool fin = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = xs[3 * j + c];
    v[3 + c] = vs[3 * j + c];
  }
  // finiteness from the exponent bits (integer work: FP64 operations run at a
  // small fraction of the FP32 rate on this part and bound this kernel)
#pragma unroll
  for (int c = 0; c < 6; ++c)
    fin = fin && ((uint32_t(__double_as_longlong(v[c]) >> 32) & 0x7ff00000u) != 0x7ff00000u);
  Part<T> p;
  p.x = narrow<T>(v[0]); p.y = narrow<T>(v[1]); p.z = narrow<T>(v[2]);
  p.vx = narrow<T>(v[3]); p.vy = narrow<T>(v[4]); p.vz = narrow<T>(v[5]);
  p.id = ids ? ids[j] : uint32_t(j);
  st[j] = p;
  // range test and radius key (radius_key's two forms, with r^2 shared)
  bool inside;
  uint32_t k;
  bool fx = false;
  if constexpr (sizeof(T) == 4) fx = key_fx_applies(p.x, p.y, p.z, rk);
  if (fx) {
    const uint64_t R2 = r2_fx(float(p.x), float(p.y), float(p.z));
    inside = R2 > kFxOne && R2 < rk.rout2_fx;
    k = key_of_fx(R2, rk);
  } else {
    const double xd = widen<T>(p.x), yd = widen<T>(p.y), zd = widen<T>(p.z);
    const double r2 = xd * xd + yd * yd + zd * zd;
    inside = r2 > 1.0 && r2 < r_out2;
    k = key_of_r2(r2, rk);
  }
  if (!fin) atomicOr(err, kErrNaN);
  else if (!inside) atomicOr(err, kErrRange);
  key[j] = k;
  kidx[j] = uint32_t(j);
}

template <class T>
void launch_load(const double* x, const double* v, const uint32_t* ids, Part<T>* st, uint32_t* key,
                 uint32_t* kidx, int64_t n, double r_out, int* err, cudaStream_t s) {
  k_load<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(x, v, ids, st, key, kidx, n, r_out * r_out,
                                                      make_radius_key(r_out), err);
}

template <class T>
__global__ void k_state_dump(const Part<T>* __restrict__ st, double* __restrict__ x, double* __restrict__ v,
                             uint32_t* __restrict__ id, int64_t n) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Part<T> p = st[j];
  x[3 * j] = p.x; x[3 * j + 1] = p.y; x[3 * j + 2] = p.z;
  v[3 * j] = p.vx; v[3 * j + 1] = p.vy; v[3 * j + 2] = p.vz;
  id[j] = p.id;
}

template <class T>
void launch_state_dump(const Part<T>* st, double* x, double* v, uint32_t* id, int64_t n, cudaStream_t s) {
  k_state_dump<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(st, x, v, id, n);
}

// out[id[j]][c] = comp_c[j] for c < nc (field values in radius order to id order)
template <class T> struct Ptr6 { const T* d[6]; };
template <class T>
__global__ void k_scatter_by_id(Ptr6<T> p, int nc, const uint32_t* __restrict__ id,
                                double* __restrict__ out, int64_t n) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t k = id[j];
  for (int c = 0; c < nc; ++c) out[k * nc + c] = double(p.d[c][j]);
}

template <class T>
void launch_scatter_by_id(const T* const* comps, int ncomp, const uint32_t* id, double* out, int64_t n,
                          cudaStream_t s) {
  Ptr6<T> p;
  for (int c = 0; c < ncomp; ++c) p.d[c] = comps[c];
  k_scatter_by_id<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(p, ncomp, id, out, n);
}

// The state in id order: x[id][3] and v[id][3], FP64.
template <class T>
__global__ void k_state_out(const Part<T>* __restrict__ st, double* __restrict__ x, double* __restrict__ v,
                            int64_t n) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Part<T> p = st[j];
  const int64_t k = p.id;
  x[3 * k] = p.x; x[3 * k + 1] = p.y; x[3 * k + 2] = p.z;
  v[3 * k] = p.vx; v[3 * k + 1] = p.vy; v[3 * k + 2] = p.vz;
}

template <class T>
void launch_state_out(const Part<T>* st, double* x, double* v, int64_t n, cudaStream_t s) {
  k_state_out<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(st, x, v, n);
}

// ============================================================================
// Scans of the tile moments (FP64 accumulation)
// ============================================================================
// Tile scan: the in-group scans of the tile sums agg[u][tile] over the tw
// tiles of whole groups (row stride ts). One warp task = 128 consecutive tiles of
// one row = 4 groups; lane l holds tiles 4l..4l+3 (one vector load), so a
// group is 8 lanes. Each lane sums its 4 tiles in order, an 8-lane shuffle
// scan gives the lane's offset, and the lane writes its 4 results with one
// vector store. Rs rows (u even): exclusive prefix towards higher tiles; Is
// rows (u odd): exclusive suffix towards lower tiles; each summed in its own
// direction (no total minus a partial sum, which would cancel). The group
// total (the inclusive sum at the far end) goes to gagg[g][u] in FP64. Each
// warp takes kTsTasks consecutive tasks and issues their loads first.
// ============================================================================

// Compensated partial sums of the in-group scans. In FP32 every partial sum is
// the unevaluated pair hi + lo: hi is the plain running sum and lo collects the
// rounding error of every addition, which Knuth's TwoSum gives exactly, so a
// sum over the 1024 particles of a scan group keeps about twice the working
// precision (the radius-ordered scans are where cancellation sets the
// accuracy). The results are rounded to FP32 once (hi + lo), the group totals
// to FP64. In FP64 the sums are plain.
template <class T> struct CSum { T hi, lo; };
template <class T> __device__ __forceinline__ CSum<T> cs_add(CSum<T> a, CSum<T> b) {
  if constexpr (sizeof(T) == 4) {
    const T s = a.hi + b.hi;
    const T bb = s - a.hi;
    const T e = (a.hi - (s - bb)) + (b.hi - bb);  // a.hi + b.hi = s + e exactly
    return {s, (a.lo + b.lo) + e};
  } else {
    return {a.hi + b.hi, T(0)};
  }
}
template <class T> __device__ __forceinline__ T cs_round(CSum<T> v) { return v.hi + v.lo; }
template <class T> __device__ __forceinline__ CSum<T> cs_of(T v) { return {v, T(0)}; }
template <class T> __device__ __forceinline__ CSum<T> cs_shfl_down(CSum<T> v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.hi, d, 8), __shfl_down_sync(0xffffffffu, v.lo, d, 8)};
}
template <class T> __device__ __forceinline__ CSum<T> cs_shfl_up(CSum<T> v, int d) {
  return {__shfl_up_sync(0xffffffffu, v.hi, d, 8), __shfl_up_sync(0xffffffffu, v.lo, d, 8)};
}
template <class T> __device__ __forceinline__ double cs_double(CSum<T> v) { return double(v.hi) + double(v.lo); }

// In-group scans of the tile sums. A CTA takes 32 rows (components u) x 128
// tiles (4 scan groups) of agg[u][tile]: each warp scans 4 rows, one V4 of 4
// tiles per lane (a 4-element in-lane scan plus an 8-lane shuffle scan per
// group), and the CTA writes the results transposed, pfx[tile][u], through
// shared memory, so that the field kernel reads the carries of one tile as
// contiguous lines. Is rows (u odd) get exclusive suffixes, Rs rows (u even)
// exclusive prefixes; the group totals go to gagg[g][u] in FP64.
constexpr int kTsRows = 32;    // components per CTA
constexpr int kTsTiles = 128;  // tiles per CTA

template <class T>
__global__ void __launch_bounds__(256) k_tile_scan(const T* __restrict__ agg, T* __restrict__ pfx,
                                                   double* __restrict__ gagg, int64_t tw, int64_t ts, int nc) {
  using V4 = typename Vec4<T>::type;
  using C = CSum<T>;
  __shared__ T buf[kTsRows][kTsTiles + 1];  // [row][tile], padded: the transposed reads hit distinct banks
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, r = lane & 7;
  const int64_t tile0 = int64_t(blockIdx.x) * kTsTiles;
  const int u0 = int(blockIdx.y) * kTsRows;
  const int64_t tile = tile0 + 4 * lane;
  V4 v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int u = u0 + 4 * warp + k;
    if (u < nc && tile < tw) {
      v[k] = *reinterpret_cast<const V4*>(agg + int64_t(u) * ts + tile);
    } else {
      v[k].x = v[k].y = v[k].z = v[k].w = T(0);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int row = 4 * warp + k, u = u0 + row;
    if (u >= nc) break;  // warp-uniform
    const int64_t g = tile / 32;
    V4 o;
    if (u & 1) {  // Is: exclusive suffix
      const C f2 = cs_of(v[k].w), f1 = cs_add(f2, cs_of(v[k].z)), f0 = cs_add(f1, cs_of(v[k].y)),
              sum = cs_add(f0, cs_of(v[k].x));
      C x = cs_shfl_down(sum, 1);
      if (r == 7) x = cs_of(T(0));
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const C y = cs_shfl_down(x, d);
        if (r + d < 8) x = cs_add(x, y);
      }
      o.x = cs_round(cs_add(x, f0)); o.y = cs_round(cs_add(x, f1)); o.z = cs_round(cs_add(x, f2));
      o.w = cs_round(x);
      if (r == 0 && tile < tw) gagg[g * nc + u] = cs_double(cs_add(x, sum));
    } else {      // Rs: exclusive prefix
      const C e1 = cs_of(v[k].x), e2 = cs_add(e1, cs_of(v[k].y)), e3 = cs_add(e2, cs_of(v[k].z)),
              sum = cs_add(e3, cs_of(v[k].w));
      C x = cs_shfl_up(sum, 1);
      if (r == 0) x = cs_of(T(0));
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const C y = cs_shfl_up(x, d);
        if (r >= d) x = cs_add(x, y);
      }
      o.x = cs_round(x); o.y = cs_round(cs_add(x, e1)); o.z = cs_round(cs_add(x, e2));
      o.w = cs_round(cs_add(x, e3));
      if (r == 7 && tile < tw) gagg[g * nc + u] = cs_double(cs_add(x, sum));
    }
    buf[row][4 * lane] = o.x; buf[row][4 * lane + 1] = o.y;
    buf[row][4 * lane + 2] = o.z; buf[row][4 * lane + 3] = o.w;
  }
  __syncthreads();
  // transposed write: warp w writes tiles w, w + 8, ..., lane = row
  const int u = u0 + lane;
  if (u < nc) {
    const int tend = tw - tile0 < kTsTiles ? int(tw - tile0) : kTsTiles;
    T* dst = pfx + (tile0 + warp) * nc + u;
    const int64_t step = 8 * int64_t(nc);
#pragma unroll 4
    for (int t = warp; t < tend; t += 8, dst += step) *dst = buf[lane][t];
  }
}

template <class T>
void launch_tile_scan(const T* agg, T* pfx, double* gagg, int64_t ntiles, int nc, cudaStream_t s) {
  const int64_t tw = tiles_whole(ntiles), ts = tile_stride(ntiles);
  const dim3 grid(unsigned((tw + kTsTiles - 1) / kTsTiles), unsigned((nc + kTsRows - 1) / kTsRows));
  if (tw > 0) k_tile_scan<T><<<grid, 256, 0, s>>>(agg, pfx, gagg, tw, ts, nc);
}

// ============================================================================
// Group scan. Input: the FP64 totals gagg[g][u] of the scan groups (written
// by the moments kernel). Output: gbase[g][u] = the sum over the earlier
// groups (Rs components, u even) or over the later groups (Is components, u
// odd), each summed in its own direction, and the totals tot / totd.
// The groups are cut into nseg segments of G groups (G a multiple of 8);
// CTA (column block b, segment s) handles components 32 b + lane with its 8
// warps splitting the segment. k_group_sums forms the warp and segment sums;
// the last CTA of a column block to finish (an atomic ticket, no waiting)
// scans the segment sums of that block in a fixed order, so the result is
// the same whichever CTA finishes last. k_group_bases then walks each warp's
// groups once more and writes the bases.
// Work space w (FP64): [nseg][8][nc] warp sums, then [nseg][nc] segment sums,
// then [nseg][nc] segment bases.
// ============================================================================
template <class T>
__global__ void __launch_bounds__(kGsWarps * 32) k_group_sums(const double* __restrict__ gagg,
                                                              double* __restrict__ w, unsigned* __restrict__ ticket,
                                                              T* __restrict__ tot, double* __restrict__ totd,
                                                              int64_t ngroups, int nc, int64_t G, int nseg) {
  __shared__ double ws[kGsWarps][32];
  __shared__ double sst[kGsMaxSeg][32];  // the segment sums of this column block (last CTA)
  __shared__ bool last;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const bool okc = c < nc;
  const int seg = blockIdx.y;
  double* wsum = w;
  double* ssum = w + int64_t(kGsMaxSeg) * kGsWarps * nc;
  double* sbase = ssum + int64_t(kGsMaxSeg) * nc;
  const int64_t per = G / kGsWarps;
  const int64_t g0 = int64_t(seg) * G + warp * per;
  const int64_t g1 = g0 + per < ngroups ? g0 + per : ngroups;
  double run = 0.0;
  if (okc) {
#pragma unroll 4
    for (int64_t g = g0; g < g1; ++g) run += gagg[g * nc + c];
    wsum[(int64_t(seg) * kGsWarps + warp) * nc + c] = run;
  }
  ws[warp][lane] = run;
  __syncthreads();
  if (warp == 0 && okc) {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < kGsWarps; ++k) sum += ws[k][lane];
    ssum[int64_t(seg) * nc + c] = sum;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ticket[blockIdx.x], 1u) == unsigned(nseg - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // all warps stage the segment sums (independent loads in flight together),
  // then warp 0 scans them from shared memory in a fixed order
  for (int k = int(warp); k < nseg; k += kGsWarps) sst[k][lane] = okc ? __ldcg(ssum + int64_t(k) * nc + c) : 0.0;
  __syncthreads();
  if (warp == 0 && okc) {
    double all = 0.0;
    const bool suffix = (c & 1) != 0;
    for (int k = 0; k < nseg; ++k) {
      const int s2 = suffix ? nseg - 1 - k : k;
      sbase[int64_t(s2) * nc + c] = all;
      all += sst[s2][lane];
    }
    tot[c] = T(all);
    totd[c] = all;
  }
  if (threadIdx.x == 0) ticket[blockIdx.x] = 0u;  // ready for the next step
}

template <class T>
__global__ void __launch_bounds__(kGsWarps * 32) k_group_bases(const double* __restrict__ gagg,
                                                               const double* __restrict__ w, T* __restrict__ gbase,
                                                               int64_t ngroups, int nc, int64_t G) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  if (c >= nc) return;  // no barrier below
  const int seg = blockIdx.y;
  const bool suffix = (c & 1) != 0;
  const double* wsum = w;
  const double* sbase = w + int64_t(kGsMaxSeg) * (kGsWarps + 1) * nc;
  double run = sbase[int64_t(seg) * nc + c];
#pragma unroll
  for (int k = 0; k < kGsWarps; ++k)
    if (suffix ? unsigned(k) > warp : unsigned(k) < warp) run += wsum[(int64_t(seg) * kGsWarps + k) * nc + c];
  const int64_t per = G / kGsWarps;
  const int64_t g0 = int64_t(seg) * G + warp * per;
  const int64_t g1 = g0 + per < ngroups ? g0 + per : ngroups;
#pragma unroll 4
  for (int64_t k = 0; k < g1 - g0; ++k) {
    const int64_t g = suffix ? g1 - 1 - k : g0 + k;
    gbase[g * nc + c] = T(run);
    run += gagg[g * nc + c];
  }
}

template <class T>
void launch_group_scan(const double* gagg, double* work, unsigned* ticket, T* gbase, T* tot, double* totd,
                       int64_t ngroups, int nc, int gseg, cudaStream_t s) {
  if (ngroups <= 0) return;
  const int64_t G = gs_seg_len(ngroups, gseg);
  const int nseg = int(gs_nseg(ngroups, gseg));
  dim3 grid(unsigned(gs_col_blocks(nc)), unsigned(nseg));
  k_group_sums<T><<<grid, kGsWarps * 32, 0, s>>>(gagg, work, ticket, tot, totd, ngroups, nc, G, nseg);
  k_group_bases<T><<<grid, kGsWarps * 32, 0, s>>>(gagg, work, gbase, ngroups, nc, G);
}

// ============================================================================
// Finalize: u_asy(t_n), the kick weight, and Q_diff(t_n) = -(1/n~) sum over odd
// l of c_l' b^P_l * (sum_i q_i Is_l^0(x_i)) (Sec. 4; Is_l^0 = P_l(cos t)/r^{l+1}).
// ============================================================================
__global__ void k_finalize(FinalizeArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  StepState* st = a.st;
  const int64_t n = st->next;
  const double t = double(n) * a.dt;
  double u = 0.0;
  if (a.drive_kind == 0) {
    const double z = (t - a.t0) / a.sigma;
    u = a.v_hat * exp(-0.5 * z * z);
  } else if (a.drive_kind == 1) {
    u = n == 0 ? a.v_hat : 0.0;
  }
  st->step = n;
  st->u = u;
  st->kick = st->sync ? 0.5 * a.dt : a.dt;
  // electrons absorbed at the probe since the last fold (wall_rule 2) join Q_S
  // (charge -1 each) before the field of this step is evaluated
  st->qs_acc -= double(st->nabs_step);
  st->nabs_total += st->nabs_step;
  st->nabs_step = 0;
  if (a.record) {
    double q = 0.0;
    for (int l = 1; l <= a.L; l += 2) q += a.canti[l] * a.totd[2 * (l - 1) + 1];
    q *= -a.inv_ntilde;
    const int64_t h = n - a.first;
    if (h >= 0 && h < a.cap) {
      a.qhist[h] = q;
      a.uhist[h] = u;
    }
    st->next = n + 1;
    st->sync = 0;
  }
}

void launch_finalize(const FinalizeArgs& a, cudaStream_t s) { k_finalize<<<1, 32, 0, s>>>(a); }

// Step state after a load: step 0, nothing recorded, the first kick is a half kick.
__global__ void k_init_step(StepState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->step = 0;
  st->next = 0;
  st->u = 0.0;
  st->kick = 0.0;
  st->sync = 1;
  st->nabs_step = 0;
  st->qs_acc = 0.0;
  st->nabs_total = 0;
}

void launch_init_step(StepState* st, cudaStream_t s) { k_init_step<<<1, 32, 0, s>>>(st); }

// ============================================================================
// Spectrum sums (FP64). One thread per frequency; the phase factor advances
// by a rotation and is recomputed exactly every 256 steps.
// ============================================================================
__global__ void k_dft(const double* __restrict__ q, const double* __restrict__ u, int64_t ns, double dt,
                      double first_kick, int64_t nf, double w_max, double* __restrict__ out) {
  const int64_t jf = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (jf >= nf) return;
  const double w = double(jf + 1) * (w_max / double(nf));
  double sr, cr;
  sincos(w * dt, &sr, &cr);  // rotation by e^{-i w dt}
  const double q0 = q[0];
  double Qr = 0, Qi = 0, Ur = 0, Ui = 0, pr = 1.0, pi = 0.0;
  for (int64_t k = 0; k < ns; ++k) {
    if ((k & 255) == 0) {
      double s, c;
      sincos(w * dt * double(k), &s, &c);
      pr = c;
      pi = -s;
    }
    const double dq = q[k] - q0;
    const double kw = k == 0 ? first_kick : dt;
    const double uu = kw * u[k];
    Qr += dq * pr; Qi += dq * pi;
    Ur += uu * pr; Ui += uu * pi;
    const double npr = pr * cr + pi * sr, npi = pi * cr - pr * sr;
    pr = npr;
    pi = npi;
  }
  out[4 * jf + 0] = dt * Qr;
  out[4 * jf + 1] = dt * Qi;
  out[4 * jf + 2] = Ur;
  out[4 * jf + 3] = Ui;
}

void launch_dft(const double* q, const double* u, int64_t ns, double dt, double first_kick, int64_t nf,
                double w_max, double* out, cudaStream_t s) {
  k_dft<<<unsigned((nf + 127) / 128), 128, 0, s>>>(q, u, ns, dt, first_kick, nf, w_max, out);
}

template <class T> cudaError_t preload_core_kernels_t() {
  cudaFuncAttributes fa;
  const void* fns[] = {
      reinterpret_cast<const void*>(&k_reorder<T>),     reinterpret_cast<const void*>(&k_keys<T>),
      reinterpret_cast<const void*>(&k_load<T>),        reinterpret_cast<const void*>(&k_state_dump<T>),
      reinterpret_cast<const void*>(&k_scatter_by_id<T>), reinterpret_cast<const void*>(&k_state_out<T>),
      reinterpret_cast<const void*>(&k_tile_scan<T>),   reinterpret_cast<const void*>(&k_group_sums<T>),
      reinterpret_cast<const void*>(&k_group_bases<T>)};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t preload_core_kernels() {
  if (set_sort_attributes() != cudaSuccess) return cudaErrorInvalidValue;
  cudaFuncAttributes fa;
  const void* fns[] = {reinterpret_cast<const void*>(&k_sort_hist<256>),
                       reinterpret_cast<const void*>(&k_sort_hist<512>),
                       reinterpret_cast<const void*>(&k_sort_rowscan),
                       reinterpret_cast<const void*>(&k_sort_scatter<256>),
                       reinterpret_cast<const void*>(&k_sort_scatter<512>),
                       reinterpret_cast<const void*>(&k_bucket_sort<256, 3>),
                       reinterpret_cast<const void*>(&k_bucket_sort<256, 2>),
                       reinterpret_cast<const void*>(&k_finalize),
                       reinterpret_cast<const void*>(&k_init_step), reinterpret_cast<const void*>(&k_dft)};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = preload_core_kernels_t<float>();
  return e != cudaSuccess ? e : preload_core_kernels_t<double>();
}

// explicit instantiations
#define IMRP_INST_CORE(T)                                                                          \
  template void launch_reorder<T>(const Part<T>*, T* const*, uint32_t*, const uint32_t*, int64_t,  \
                                  cudaStream_t);                                                   \
  template void launch_keys<T>(const Part<T>*, uint32_t*, uint32_t*, int64_t, double, cudaStream_t); \
  template void launch_load<T>(const double*, const double*, const uint32_t*, Part<T>*, uint32_t*, \
                               uint32_t*, int64_t, double, int*, cudaStream_t);                    \
  template void launch_state_dump<T>(const Part<T>*, double*, double*, uint32_t*, int64_t,         \
                                     cudaStream_t);                                                \
  template void launch_scatter_by_id<T>(const T* const*, int, const uint32_t*, double*, int64_t,   \
                                        cudaStream_t);                                             \
  template void launch_state_out<T>(const Part<T>*, double*, double*, int64_t, cudaStream_t);     \
  template void launch_tile_scan<T>(const T*, T*, double*, int64_t, int, cudaStream_t);                \
  template void launch_group_scan<T>(const double*, double*, unsigned*, T*, T*, double*, int64_t, int, \
                                     int, cudaStream_t);
IMRP_INST_CORE(float)
IMRP_INST_CORE(double)

}  // namespace imrp
