// Measured peak rates of the arithmetic pipes the plain FP64 path and the evaluation run on
// (no paper counterpart): the denominators of the FP64- and FP32-bound rooflines, taken on
// the device itself rather than from a datasheet.  Each rate comes from launches of
// independent dependent-FMA chains (8 per thread, 4 CTAs of 256 threads per SM, every SM):
// the fastest of three launches timed by CUDA events after a warm-up launch.  The chains stay
// bounded (x <- x m + c with |m| < 1) and the result reaches a device sink only under a
// condition that never holds, so nothing is stored and nothing is optimised away.
#include <cuda_runtime.h>

#include "psq.h"
#include "psq_internal.h"

namespace psq {
namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;

__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(int iters, T m, T c) {
  T x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = (T)(threadIdx.x + 1 + k) * (T)1e-3;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = fma(x[k], m, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if ((double)s == -1.0) g_peak_sink = (double)s;  // the chains converge to c / (1 - m) > 0
}

// SFU: 2^x by the special-function unit's approximation, x kept in [-1, 0) (2^x - 1 is in
// [-0.5, 0)); one FP32 add per SFU operation, which the FMA pipe issues alongside.
__global__ void __launch_bounds__(kPeakThreads) ex2_chain_kernel(int iters) {
  float x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = -0.5f - 0.01f * (float)k - 1e-5f * (float)threadIdx.x;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
      x[k] = y - 1.0f;
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if (s == 1.0f) g_peak_sink = (double)s;  // every x stays negative
}

// Milliseconds of the fastest of three timed launches of `launch` on stream s, after one
// untimed launch (-1 on a CUDA error).
template <typename F>
float time_launch(F launch, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = -1.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  launch();
  for (int r = 0; r < 3; ++r) {
    float ms = -1.0f;
    if (cudaEventRecord(e0, s) != cudaSuccess) goto done;
    launch();
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
    if (cudaGetLastError() != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      best = -1.0f;
      goto done;
    }
    if (best < 0.0f || ms < best) best = ms;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return best;
}

}  // namespace
}  // namespace psq

extern "C" psq_status psq_measure_peaks(void* stream, double* fp64_tflops, double* fp32_tflops, double* sfu_gops) {
  using namespace psq;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    return set_error(PSQ_ERR_CUDA, "psq_measure_peaks: no CUDA device");
  cudaStream_t s = (cudaStream_t)stream;
  const int ctas = sms * kPeakCtasPerSm;
  const double lanes = (double)ctas * kPeakThreads * kPeakChains;  // independent chains
  // iteration counts for ~30 ms at GB300's rates (multiples of the unroll factor)
  const int it64 = 16 * 1000, it32 = 16 * 60000, itsfu = 16 * 8000;
  const float t64 = time_launch([&] { fma_chain_kernel<double><<<ctas, kPeakThreads, 0, s>>>(it64, 0.999999, 1e-7); }, s);
  const float t32 = time_launch([&] { fma_chain_kernel<float><<<ctas, kPeakThreads, 0, s>>>(it32, 0.999f, 1e-4f); }, s);
  const float tsf = time_launch([&] { ex2_chain_kernel<<<ctas, kPeakThreads, 0, s>>>(itsfu); }, s);
  if (t64 <= 0.0f || t32 <= 0.0f || tsf <= 0.0f) return set_error(PSQ_ERR_CUDA, "psq_measure_peaks: a timed launch failed");
  if (fp64_tflops) *fp64_tflops = 2.0 * lanes * it64 / (t64 * 1e-3) / 1e12;
  if (fp32_tflops) *fp32_tflops = 2.0 * lanes * it32 / (t32 * 1e-3) / 1e12;
  if (sfu_gops) *sfu_gops = lanes * itsfu / (tsf * 1e-3) / 1e9;
  return PSQ_OK;
}
