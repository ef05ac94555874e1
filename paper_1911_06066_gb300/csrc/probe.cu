// Measurement aid (the paper has no counterpart): the FP64 and FP32 fused
// multiply-add rate of the device, the ALU bound against which the FP64 /
// FP32 work of the per-sample sweep is set.  Each thread runs 8 independent
// FMA chains of `iters` steps (enough independent work to cover the pipes'
// latency), on a grid of 16 blocks of 256 threads per SM; the result is stored
// so that the chains are not optimised away.
#include <stdio.h>

#include "internal.cuh"

namespace mlmc {
void set_create_error(const std::string& msg);   // abi.cu: text for mlmc_last_error(NULL)
}
using namespace mlmc;

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T a, T b, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t time_chains(int blocks, int iters, T* out, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  fma_chain_kernel<T><<<blocks, 256, 0, st>>>(iters / 8, (T)0.999, (T)1e-4, out);   // warm-up
  cudaEventRecord(e0, st);
  fma_chain_kernel<T><<<blocks, 256, 0, st>>>(iters, (T)0.999, (T)1e-4, out);
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

// out: device scratch of at least 16 * 256 * (SM count) elements of the type
// (8 bytes each suffice for both); synchronises the stream.
extern "C" mlmc_status mlmc_probe_fma_rate(int fp64, void* out, size_t out_bytes, double* tflops,
                                           void* stream) {
  if (!out || !tflops) {
    set_create_error("mlmc_probe_fma_rate: NULL argument");
    return MLMC_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { set_create_error(cudaGetErrorString(e)); return MLMC_ERR_CUDA; }
  const int blocks = 16 * sms;
  if (out_bytes < (size_t)blocks * 256 * 8) {
    set_create_error("mlmc_probe_fma_rate: output scratch too small");
    return MLMC_ERR_WORKSPACE;
  }
  const int iters = fp64 ? 4096 : 65536;
  float ms = 0.f;
  e = fp64 ? time_chains<double>(blocks, iters, (double*)out, (cudaStream_t)stream, &ms)
           : time_chains<float>(blocks, iters, (float*)out, (cudaStream_t)stream, &ms);
  if (e != cudaSuccess) { set_create_error(cudaGetErrorString(e)); return MLMC_ERR_CUDA; }
  *tflops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0 / ((double)ms * 1e-3) * 1e-12;
  return MLMC_OK;
}
