// Throughput probes of the CUDA-core FMA pipes (diagnostic, not part of the
// method): the FP32 and FP64 peaks against which the pair stage (FP32
// transforms), the FP64 contraction and the Gauss-Jordan updates are rated.
// Every thread runs eight independent fused multiply-add chains, so the
// pipes, not the latency of one chain, set the rate.
#include <string>

#include "internal.h"

namespace chi0 {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(int iters, T b, T c, T* sink) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == (T)-1.25) *sink = s;     // never true; keeps the chains alive
}

__device__ float g_sink_f;
__device__ double g_sink_d;

}  // namespace
}  // namespace chi0

extern "C" chi0_status chi0_peak_fma(int kind, int iters, double* ms, double* flops, void* stream) {
  using namespace chi0;
  if ((kind != 0 && kind != 1) || iters < 1 || iters > (1 << 20) || !ms || !flops) {
    set_global_error("chi0_peak_fma: kind must be 0 (FP32) or 1 (FP64), iters in [1, 2^20], outputs non-NULL");
    return CHI0_ERR_INVALID;
  }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    set_global_error("chi0_peak_fma: no CUDA device");
    return CHI0_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float* sf = nullptr;
  double* sd = nullptr;
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&sf, g_sink_f);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&sd, g_sink_d);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    if (kind == 0) k_peak_fma<float><<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, sf);
    else k_peak_fma<double><<<blocks, threads, 0, s>>>(iters, 0.999, 1e-3, sd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_global_error(std::string("chi0_peak_fma: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return CHI0_ERR_CUDA;
  }
  *ms = t;
  *flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
  return CHI0_OK;
}
