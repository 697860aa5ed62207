// Measured FP64 arithmetic peaks of the device (roofline denominators).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the FP64 pipe, not
// HBM, bounds most complex128 kernels here.  Two kernels of independent
// operations on every SM, each timed with CUDA events after a warm-up launch:
// * k_probe_dfma: eight independent FMA chains per thread;
// * k_probe_dmma: four independent FP64 matrix multiply-accumulates per warp
//   (mma.sync m8n8k4 with FP64 operands: 8 x 8 x 4 multiply-adds each).
#include <cuda_runtime.h>

#include <string>

#include "qf_internal.h"

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(double* out, int iters) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-9 * (threadIdx.x + 37 * k);
  const double b = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 0.125) out[blockIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_dmma(double* out, int iters) {
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 0.5;
  double c[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = 1e-3 * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  if (s == 0.125) out[blockIdx.x] = s;
}

qf_status pfail(const char* what, cudaError_t e) {
  qf::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return QF_ECUDA;
}

// Seconds of one launch of k (after a warm-up launch), timed with events on s.
template <typename K>
cudaError_t time_kernel(K k, int grid, double* out, int iters, cudaStream_t s, double* sec) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k<<<grid, kProbeThreads, 0, s>>>(out, iters / 8);  // warm-up
    qf::count_launch();
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    k<<<grid, kProbeThreads, 0, s>>>(out, iters);
    qf::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *sec = ms * 1e-3;
  return e;
}

}  // namespace

extern "C" qf_status qf_probe_fp64_peaks(void* stream, double* fma_flops, double* dmma_flops) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return pfail("device query failed", e);
  const int grid = 8 * sms;  // eight CTAs (64 warps) per SM
  double* scratch = nullptr;  // written only if a chain reaches an impossible value
  if ((e = cudaMalloc(&scratch, grid * sizeof(double))) != cudaSuccess) return pfail("cudaMalloc(probe)", e);
  qf_status st = QF_OK;
  if (fma_flops) {
    const int iters = 4096;
    double sec = 0.0;
    e = time_kernel(k_probe_dfma, grid, scratch, iters, s, &sec);
    if (e != cudaSuccess || sec <= 0.0)
      st = pfail("FP64 FMA probe failed", e);
    else
      *fma_flops = 2.0 * 8.0 * iters * (double)grid * kProbeThreads / sec;
  }
  if (st == QF_OK && dmma_flops) {
    const int iters = 1024;
    double sec = 0.0;
    e = time_kernel(k_probe_dmma, grid, scratch, iters, s, &sec);
    if (e != cudaSuccess || sec <= 0.0)
      st = pfail("FP64 MMA probe failed", e);
    else  // per warp and instruction: 8 x 8 x 4 multiply-adds
      *dmma_flops = 2.0 * 256.0 * 4.0 * iters * (double)grid * (kProbeThreads / 32) / sec;
  }
  cudaFree(scratch);
  return st;
}
