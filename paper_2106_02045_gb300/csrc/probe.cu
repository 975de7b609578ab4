// probe.cu -- throughput probes for the roofline denominators of the fit kernels.
//
// The fits are bound by plain FP32 arithmetic (the pipe that executes FFMA/FADD/FMUL), with
// the exponentials of the profile on the MUFU unit and a few FP64 operations in the LM step.
// None of these peaks is in the driver's peak file (a copy bandwidth and a bf16 GEMM rate), so
// the benchmark measures them here, on the GPU and at the clock it runs on: independent
// dependency chains per thread, enough resident warps to fill every SM, CUDA events around
// a few launches. Not part of the paper; measurement support only.
#include <cuda_runtime.h>

#include "fitspots.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) ffma_chains(float *out, float a, float b, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// exp2 on the MUFU unit (what __expf issues after its scaling multiply); the chain stays in
// (0, 1] because each step takes 2^-x of a value in (0, 1]
__global__ void __launch_bounds__(kThreads) ex2_chains(float *out, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-4f + 0.01f * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[k]));
      x[k] = y;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_chains(double *out, double a, double b, int iters) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" size_t fit_spots_probe_scratch_bytes(int sms) {
  if (sms < 1 || sms > 4096) return 0;
  return (size_t)sms * kBlocksPerSm * kThreads * sizeof(double);
}

extern "C" int fit_spots_probe_rates(int sms, void *scratch, size_t scratch_bytes, double *ffma,
                                     double *ex2, double *dfma, void *stream) {
  if (!scratch || !ffma || !ex2 || !dfma) return FS_ERR_NULL;
  if (sms < 1 || sms > 4096) return FS_ERR_ARG;
  if (scratch_bytes < fit_spots_probe_scratch_bytes(sms)) return FS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = sms * kBlocksPerSm;
  const double lanes = (double)blocks * kThreads;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // each kernel: one warm-up launch, then `reps` timed launches
  auto time_it = [&](auto launch, int reps, double ops_per_launch, double *rate) {
    if (e != cudaSuccess) return;
    launch();
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return;
    for (int r = 0; r < reps; ++r) launch();
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return;
    *rate = ops_per_launch * reps / (ms * 1e-3);
  };
  float *fo = static_cast<float *>(scratch);
  double *dout = static_cast<double *>(scratch);
  const int fi = 4096, xi = 1024, di = 256;
  time_it([&] { ffma_chains<<<blocks, kThreads, 0, st>>>(fo, 0.999f, 1e-3f, fi); }, 20,
          lanes * fi * kChains, ffma);
  time_it([&] { ex2_chains<<<blocks, kThreads, 0, st>>>(fo, xi); }, 20, lanes * xi * kChains, ex2);
  time_it([&] { dfma_chains<<<blocks, kThreads, 0, st>>>(dout, 0.999, 1e-3, di); }, 5,
          lanes * di * kChains, dfma);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
