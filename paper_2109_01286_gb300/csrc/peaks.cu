// hfd_measure_fma_peaks: the device's fused multiply-add throughput in FP64 and FP32, measured
// with hand-written loops, so that a kernel's fraction of the arithmetic peak rests on a
// measurement of this device at its current clocks rather than on a data-sheet figure.
//
// Each thread runs eight independent FMA chains x <- x*a + b (a just below 1, so the values stay
// bounded), 16 steps per chain per loop trip.  Eight chains per thread and 8 blocks of 256
// threads per SM keep enough independent instructions in flight to cover the FMA latency, so
// the loop is bound by the FMA pipe alone: no memory traffic, no other instructions in the
// inner loop (the trip count and the loop branch are amortised over 128 FMAs).  The chains'
// sum is stored only if it equals an impossible sentinel, which keeps the compiler from
// removing the work without adding stores.
#include <cuda_runtime.h>

#include <algorithm>

#include "hfd.h"
#include "prep.hpp"

namespace {

template <typename T>
__global__ void k_fma_peak(T* out, int trips, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int s = 0; s < 16; ++s) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
  }
  T sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += x[k];
  if (sum == (T)-1234.5) out[blockIdx.x] = sum;
}

template <typename T>
cudaError_t time_peak(int sms, T* out, int trips, cudaStream_t s, double* flops) {
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {     // launch 0 warms up
    cudaEventRecord(e0, s);
    k_fma_peak<T><<<blocks, threads, 0, s>>>(out, trips, (T)0.999999, (T)1e-6);
    e = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms > 0.f) {
      const double fmas = (double)blocks * threads * trips * 16.0 * 8.0;
      best = std::max(best, 2.0 * fmas / (ms * 1e-3));
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *flops = best;
  return e;
}

}  // namespace

extern "C" hfd_status hfd_measure_fma_peaks(double* fp64_flops, double* fp32_flops,
                                             int32_t* sm_count, void* stream) {
  if (!fp64_flops || !fp32_flops || !sm_count) {
    hfd::set_error("hfd_measure_fma_peaks: null output pointer");
    return HFD_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) {
    hfd::set_error("hfd_measure_fma_peaks: device query: %s", cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  void* out = nullptr;
  e = cudaMalloc(&out, (size_t)sms * 8 * sizeof(double));
  cudaStream_t s = (cudaStream_t)stream;
  // about 20-40 ms per timed launch at the expected rates (FP64 ~0.6e12, FP32 ~40e12 FMA/s)
  if (e == cudaSuccess) e = time_peak<double>(sms, (double*)out, 400, s, fp64_flops);
  if (e == cudaSuccess) e = time_peak<float>(sms, (float*)out, 24000, s, fp32_flops);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    hfd::set_error("hfd_measure_fma_peaks: %s", cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  *sm_count = sms;
  return HFD_OK;
}
