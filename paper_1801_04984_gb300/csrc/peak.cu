// Measured arithmetic peak of the CUDA cores, the denominator of the operator
// kernels' ALU roofline.  The paper has no counterpart: the sum-factorised operator
// applies are bound by plain FP32 / FP64 fused multiply-adds (no tensor-core form
// pays for a 5-tap banded stencil), so their efficiency is reported against what
// this kernel reaches on the same GPU at the same clocks.
//
// Every thread runs NCH independent FMA chains (enough instruction-level parallelism
// to cover the FMA latency at full occupancy); the grid covers every SM several times.
// Operands are kernel arguments, so nothing folds at compile time; one conditional
// store into a file-scope sink keeps the chains live without any allocation.
#include <cuda_runtime.h>

#include "../../include/biot.h"
#include "internal.h"

namespace {

constexpr int NCH = 8;
constexpr int PEAK_THREADS = 256;
__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_chains(int iters, T a, T b) {
  T v[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) v[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += v[c];
  if (s == T(-12345.0)) g_peak_sink = (double)s;
}

template <typename T>
int run(int iters, int blocks, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BIOT_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BIOT_ECUDA;
  }
  cudaEventRecord(e0, st);
  k_fma_chains<T><<<blocks, PEAK_THREADS, 0, st>>>(iters, T(0.9999999), T(1e-7));
  biot::note_launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? BIOT_OK : BIOT_ECUDA;
}

template <typename T>
int measure(cudaStream_t st, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BIOT_ECUDA;
  const int blocks = sms * 8;  // 2048 threads per SM, every SM eight blocks deep
  // calibrate on a short run, then time one run of about 60 ms (and warm the clocks)
  int iters = 1 << 12;
  float ms = 0;
  int rc = run<T>(iters, blocks, st, &ms);
  if (rc != BIOT_OK) return rc;
  for (int rep = 0; rep < 4 && ms < 20.f; ++rep) {
    const double scale = ms > 0.05f ? 60.0 / ms : 16.0;
    const double it = iters * (scale < 16.0 ? scale : 16.0);
    iters = it > (double)(1 << 28) ? (1 << 28) : (int)it;
    rc = run<T>(iters, blocks, st, &ms);
    if (rc != BIOT_OK) return rc;
  }
  rc = run<T>(iters, blocks, st, &ms);  // the timed run
  if (rc != BIOT_OK) return rc;
  const double flop = 2.0 * NCH * (double)iters * blocks * PEAK_THREADS;
  if (tflops) *tflops = flop / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return BIOT_OK;
}

}  // namespace

extern "C" int biot_fma_peak(int prec, double* tflops, double* ms, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == BIOT_FP64) return measure<double>(st, tflops, ms);
  if (prec == BIOT_FP32) return measure<float>(st, tflops, ms);
  return BIOT_EINVAL;
}
