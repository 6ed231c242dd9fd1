// Throughput probe of the FP64 FMA pipe (the roofline denominator of the
// FP64-bound kernels): every thread runs 8 independent chains of dependent
// DFMAs; FLOPs = 2 x FMAs.  Bounded loop, no waits.
#include <cuda_runtime.h>

__global__ void k_dfma(double *out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
  double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

extern "C" int sacra_probe_fp64(int blocks, int threads, int iters, int reps, double *tflops, double *ms_best) {
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return -2;
  const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
  *ms_best = best;
  *tflops = flops / (best * 1e-3) / 1e12;
  return 0;
}

// Check of the integer-only FP64 <-> FP32 conversions the mixed-precision
// kernels use (split_f64, f32_of, f64_of of common.cuh) against the hardware
// conversions: for each input u, hi, lo, f32_of(u), the hardware
// __double2float_rn(u), and f64_of(f32_of(u)) - (double)f32_of(u).
#include "common.cuh"

__global__ void k_split(const double *in, int n, float *hi, float *lo, float *f, float *hw, double *dback) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const sacra::F2 s = sacra::split_f64(in[i]);
  hi[i] = s.hi;
  lo[i] = s.lo;
  const float v = sacra::f32_of(in[i]);
  f[i] = v;
  hw[i] = __double2float_rn(in[i]);
  dback[i] = sacra::f64_of(v) - (double)v;
}

extern "C" int sacra_probe_split(const double *host_in, int n, float *host_hi, float *host_lo, float *host_f32,
                                 float *host_hw, double *host_back_err) {
  if (n <= 0) return -1;
  double *din = nullptr, *dback = nullptr;
  float *dbuf = nullptr;
  if (cudaMalloc(&din, sizeof(double) * n) != cudaSuccess) return -1;
  if (cudaMalloc(&dback, sizeof(double) * n) != cudaSuccess) { cudaFree(din); return -1; }
  if (cudaMalloc(&dbuf, sizeof(float) * 4 * (size_t)n) != cudaSuccess) { cudaFree(din); cudaFree(dback); return -1; }
  cudaMemcpy(din, host_in, sizeof(double) * n, cudaMemcpyHostToDevice);
  k_split<<<(n + 127) / 128, 128>>>(din, n, dbuf, dbuf + n, dbuf + 2 * (size_t)n, dbuf + 3 * (size_t)n, dback);
  cudaMemcpy(host_hi, dbuf, sizeof(float) * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(host_lo, dbuf + n, sizeof(float) * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(host_f32, dbuf + 2 * (size_t)n, sizeof(float) * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(host_hw, dbuf + 3 * (size_t)n, sizeof(float) * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(host_back_err, dback, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(din);
  cudaFree(dback);
  cudaFree(dbuf);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
