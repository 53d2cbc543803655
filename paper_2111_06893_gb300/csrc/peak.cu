// Measured arithmetic peak of the CUDA cores (FP32 and FP64 fused
// multiply-add), the denominator of the roofline of the ALU-bound operator
// apply.  Every thread runs kChains independent FMA chains on registers for
// `iters` steps; operands come from kernel arguments so nothing folds, and
// the chains are combined and stored only when a never-true runtime flag is
// set, so nothing is dead either.  Timed with CUDA events on a stream of its
// own after a warm-up launch; clocks are left as they are.
#include <cuda_runtime.h>

#include "tn_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(T b, T c, int iters, int flag, T *out) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = a[j] * b + c;
  }
  if (flag) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  }
}

template <typename T>
cudaError_t time_fma(int iters, double *flops_per_s) {
  const int blocks = 4 * tn_sm_count();
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  const T b = T(0.999999), c = T(1e-7);
  if (err == cudaSuccess) {
    fma_chains_kernel<T><<<blocks, kThreads, 0, st>>>(b, c, iters, 0, nullptr);  // warm-up
    err = cudaGetLastError();
  }
  const int reps = 5;
  if (err == cudaSuccess) err = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    fma_chains_kernel<T><<<blocks, kThreads, 0, st>>>(b, c, iters, 0, nullptr);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaEventRecord(e1, st);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess)
    *flops_per_s = 2.0 * kChains * (double)iters * blocks * kThreads * reps / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return err;
}

}  // namespace

extern "C" tn_status tn_fma_peak(int device, int precision, double *flops_per_s) {
  if (!flops_per_s || (precision != TN_F32 && precision != TN_F64)) return TN_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return TN_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return TN_ECUDA;
  // ~10-20 ms per launch at the nominal rates (FP32 ~80, FP64 ~1.3 TFLOP/s)
  const cudaError_t e = precision == TN_F32 ? time_fma<float>(160000, flops_per_s)
                                            : time_fma<double>(4000, flops_per_s);
  return e == cudaSuccess ? TN_OK : TN_ECUDA;
}
