// Arithmetic peak probe: the FP64 and FP32 fused multiply-add rates of this GPU.
//
// The element kernels of the FP64 path are bound by the FP64 pipe, the
// double-float and FP32 contractions by the FP32 pipe (Sec. VI.A contractions on
// GB300), so their roofline denominators are these two rates.  Every thread runs
// kChains independent FMA chains a <- a * b + c (no dependence between chains,
// so the pipe, not the FMA latency, bounds the rate) over a grid of several
// resident CTAs per SM; the result of every chain is stored, so no chain can be
// removed.  Timed with CUDA events on the caller's stream.
#include "tdks_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(T* __restrict__ out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
tdks_status probe_t(int ctas_per_sm, int iters, int reps, cudaStream_t st, double* tflops, double* ms) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TDKS_ERR_CUDA;
  const int grid = sms * ctas_per_sm;
  T* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * kThreads * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return TDKS_ERR_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tdks_status rc = TDKS_OK;
  float t = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = TDKS_ERR_CUDA;
  } else {
    const T b = (T)0.9999999, c = (T)1e-7;
    k_fma_probe<T><<<grid, kThreads, 0, st>>>(out, iters, b, c);   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) k_fma_probe<T><<<grid, kThreads, 0, st>>>(out, iters, b, c);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      rc = TDKS_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != TDKS_OK) return rc;
  const double flops = 2.0 * kChains * (double)iters * grid * kThreads * reps;
  if (ms) *ms = t / reps;
  if (tflops) *tflops = flops / (t * 1e-3) / 1e12;
  return TDKS_OK;
}

}  // namespace

extern "C" tdks_status tdks_fma_probe(int prec, int ctas_per_sm, int iters, int reps, void* stream,
                                      double* tflops_host, double* ms_host) {
  if (ctas_per_sm < 1 || ctas_per_sm > 32 || iters < 1 || reps < 1) return TDKS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == TDKS_FP64) return probe_t<double>(ctas_per_sm, iters, reps, st, tflops_host, ms_host);
  if (prec == TDKS_FP32) return probe_t<float>(ctas_per_sm, iters, reps, st, tflops_host, ms_host);
  return TDKS_ERR_ARG;
}
