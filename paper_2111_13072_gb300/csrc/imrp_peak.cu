// Measured FP32 FMA throughput of the current device: the denominator of the
// field kernel's roofline (the field evaluation is FP32 arithmetic, not a
// tensor-core contraction). No counterpart in the paper.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/imrp.h"

namespace {

// Each thread advances kChains independent FMA chains kIters times: enough
// independent work per warp (8 chains) and enough warps per SM (the grid is
// blocks_per_sm CTAs of 256 threads on every SM) to keep the FP32 pipes busy
// whatever the FMA latency. The operands come from the arguments, so nothing
// folds at compile time; the result is written only if it equals an
// impossible value, which keeps the chains alive without memory traffic.
constexpr int kChains = 8;
constexpr int kIters = 16384;

__global__ void __launch_bounds__(256) k_ffma(float a, float b, float* out) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = a + float(threadIdx.x + c);
#pragma unroll 16
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == -1.2345f) out[blockIdx.x] = s;
}

// The same with the packed FP32 instruction (two FMAs on a register pair per
// issued instruction): the FP32 pipes' rate does not depend on how the work
// is issued, so the two kernels should agree; the larger is the peak.
__global__ void __launch_bounds__(256) k_ffma2(float a, float b, float* out) {
  float2 v[kChains / 2];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) v[c] = make_float2(a + float(threadIdx.x + 2 * c), a + float(threadIdx.x + 2 * c + 1));
#pragma unroll 16
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) s += v[c].x + v[c].y;
  if (s == -1.2345f) out[blockIdx.x] = s;
}

template <class K>
int time_kernel(K kern, int blocks, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* out, float* best_ms) {
  *best_ms = 0.f;
  for (int w = 0; w < 20; ++w) {
    kern<<<blocks, 256, 0, s>>>(1.0000001f, 1e-7f, out);
    if (cudaGetLastError() != cudaSuccess) return IMRP_E_CUDA;
  }
  for (int r = 0; r < 10; ++r) {
    cudaEventRecord(e0, s);
    kern<<<blocks, 256, 0, s>>>(1.0000001f, 1e-7f, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return IMRP_E_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (*best_ms == 0.f || ms < *best_ms) *best_ms = ms;
  }
  return *best_ms > 0.f ? IMRP_OK : IMRP_E_CUDA;
}

}  // namespace

extern "C" int imrp_fp32_peak(double* tflops, int* sm_count) {
  if (!tflops) return IMRP_E_INVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IMRP_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IMRP_E_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma, 256, 0) != cudaSuccess) return IMRP_E_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) return IMRP_E_NOMEM;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = IMRP_OK;
  float ms1 = 0.f, ms2 = 0.f;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = IMRP_E_CUDA;
  } else {
    rc = time_kernel(k_ffma, blocks, s, e0, e1, out, &ms1);
    if (rc == IMRP_OK) rc = time_kernel(k_ffma2, blocks, s, e0, e1, out, &ms2);
  }
  if (rc == IMRP_OK) {
    const double flops = 2.0 * double(blocks) * 256.0 * double(kIters) * double(kChains);
    const double t1 = flops / (double(ms1) * 1e-3) / 1e12, t2 = flops / (double(ms2) * 1e-3) / 1e12;
    *tflops = t1 > t2 ? t1 : t2;
    if (sm_count) *sm_count = sms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  return rc;
}
