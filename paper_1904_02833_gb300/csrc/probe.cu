// FP32 fused multiply-add throughput probe: the measured arithmetic roof of the solver
// kernels (which are bound by FP32 and integer ALU work, not by memory or tensor cores).
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace {

constexpr int kProbeThreads = 256;

// Eight independent dependency chains per thread, 16 rounds unrolled per iteration:
// enough independent work to keep every FMA pipe busy at full occupancy.
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float* out, int iters) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
  const float b = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" SimStatus sim_fp32_fma_probe(float* out_dev, int n_blocks, int iters, void* stream) {
  if (!out_dev || n_blocks < 1 || iters < 1) {
    snakesim::set_last_error("sim_fp32_fma_probe: null output, n_blocks < 1 or iters < 1");
    return SIM_EINVAL;
  }
  fma_probe_kernel<<<n_blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(out_dev, iters);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snakesim::set_last_error((std::string("sim_fp32_fma_probe: ") + cudaGetErrorString(e)).c_str());
    return SIM_ECUDA;
  }
  return SIM_OK;
}
