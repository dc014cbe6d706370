// peak.cu -- FMA-throughput microbenchmarks behind qcl_measure_peak: the
// roofline denominators of the FP32-bulk kernels (FFMA) and of the FP64 path
// (DFMA), measured on the device the library runs on.  Each thread runs
// kChains independent multiply-add chains (enough to cover the pipe latency);
// the grid fills every SM several times over; results go to a static device
// sink so that nothing is allocated and the compiler keeps every operation.
#include <cstdio>

#include "kernels.h"
#include "model.h"

namespace qcl {

namespace {
constexpr int kChains = 8;
__device__ double g_peak_sink[1024];

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)1.2345e-30) g_peak_sink[threadIdx.x & 1023] = (double)s;  // never true in practice
}

template <typename T>
qcl_status time_peak(int blocks, int iters, double* flops, cudaStream_t st) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error(QCL_ERR_CUDA, "cudaEventCreate failed");
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_peak<T><<<blocks, 256, 0, st>>>(iters / 8, a, b);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<blocks, 256, 0, st>>>(iters, a, b);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.0f)) return set_error(QCL_ERR_CUDA, "peak kernel failed");
  launches_add(2);
  *flops = 2.0 * kChains * 16.0 * (double)iters * 256.0 * (double)blocks / (ms * 1e-3);
  return QCL_OK;
}
}  // namespace

}  // namespace qcl

extern "C" qcl_status qcl_measure_peak(int32_t which, double* flops_per_s, void* stream) {
  using namespace qcl;
  if (!flops_per_s) return set_error(QCL_ERR_INVALID_ARG, "flops_per_s is NULL");
  if (which != 0 && which != 1) return set_error(QCL_ERR_INVALID_ARG, "which must be 0 (FP32) or 1 (FP64)");
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (n_sm < 1) return set_error(QCL_ERR_CUDA, "no device");
  const int blocks = 8 * n_sm;  // 2048 threads per SM, several waves of issue
  cudaStream_t st = (cudaStream_t)stream;
  qcl_status s = which == 0 ? time_peak<float>(blocks, 4096, flops_per_s, st)
                            : time_peak<double>(blocks, 64, flops_per_s, st);
  return s ? s : set_error(QCL_OK, "");
}
