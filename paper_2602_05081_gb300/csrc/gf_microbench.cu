// gf_microbench.cu -- measured peaks for the roofline of the Gabor evaluation.
//
// A Gabor evaluation A exp(-q/2) cos(theta) costs one MUFU ex2 and one MUFU
// cos (ex2.approx / cos.approx, the instructions the render kernels issue)
// plus a few FMA-pipe operations.  These kernels time the two pipes alone:
// every thread runs independent chains of the instruction, so the pipe, not
// latency, sets the rate.  Results are per second over the whole GPU.
#include <cuda_runtime.h>

#include "gf_host.h"

namespace gf {

constexpr int kMbChains = 8;
constexpr int kMbIters = 2048;

__device__ __forceinline__ float mb_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mb_cos(float x) {
  float y;
  asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// kMbChains independent chains of (ex2, cos) pairs per thread
__global__ void k_mb_sfu(float* out, float seed) {
  float x[kMbChains];
#pragma unroll
  for (int c = 0; c < kMbChains; ++c) x[c] = seed + 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < kMbIters; ++i) {
#pragma unroll
    for (int c = 0; c < kMbChains; ++c) x[c] = mb_cos(mb_ex2(x[c]));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kMbChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;  // keeps the chains live; never true for these inputs
}

// kMbChains independent FMA chains per thread, 4 FMAs per chain step
__global__ void k_mb_fma(float* out, float seed) {
  float x[kMbChains];
#pragma unroll
  for (int c = 0; c < kMbChains; ++c) x[c] = seed + 1e-3f * (float)(threadIdx.x + c);
  const float a = 0.999f, b = 1e-4f;
  for (int i = 0; i < kMbIters; ++i) {
#pragma unroll
    for (int c = 0; c < kMbChains; ++c) {
      float y = x[c];
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y) : "f"(a), "f"(b));
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y) : "f"(a), "f"(b));
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y) : "f"(a), "f"(b));
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y) : "f"(a), "f"(b));
      x[c] = y;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kMbChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;
}

}  // namespace gf

namespace {

template <class K>
gf_status time_kernel(K kernel, int device, int reps, double ops_per_thread, double* per_s) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return gf::report(GF_ECUDA, cudaGetErrorString(e));
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
    return gf::report(GF_ECUDA, cudaGetErrorString(e));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int blocks = prop.multiProcessorCount * per_sm * 4;  // four waves of full residency
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  // the kernels write out only if their chains reach a value they cannot reach
  // (cos(ex2(x)) stays in [-1, 1] and the FMA chains converge to 0.1), so no
  // buffer is needed
  float* out = nullptr;
  gf_status st = GF_OK;
  double best = 0.0;
  do {
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) break;
    kernel<<<blocks, 256, 0, s>>>(out, 0.5f);  // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      cudaEventRecord(a, s);
      kernel<<<blocks, 256, 0, s>>>(out, 0.25f + 0.01f * (float)r);
      cudaEventRecord(b, s);
      if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      const double rate = (double)blocks * 256.0 * ops_per_thread / ((double)ms * 1e-3);
      if (rate > best) best = rate;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  } while (0);
  if (s) cudaStreamSynchronize(s);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) st = gf::report(GF_ECUDA, cudaGetErrorString(e));
  *per_s = best;
  return st;
}

}  // namespace

extern "C" gf_status gf_measure_peaks(int device, double* sfu_pairs_per_s, double* fma_per_s) {
  if (!sfu_pairs_per_s || !fma_per_s) return gf::report(GF_EINVAL, "null argument");
  gf_status st = time_kernel(gf::k_mb_sfu, device, 5, (double)gf::kMbChains * gf::kMbIters,
                             sfu_pairs_per_s);
  if (st) return st;
  return time_kernel(gf::k_mb_fma, device, 5, 4.0 * gf::kMbChains * gf::kMbIters, fma_per_s);
}
