// Frequency factors of Eq. 1 (FP64) and the plain FP64 contraction
//   chi0[w][G][G'] += sum_p f_p(w) M_p(G) conj(M_p(G'))
// on the CUDA cores (DFMA), used by CHI0_FP64 plans.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "cplx.cuh"
#include "internal.h"

namespace chi0 {
namespace {

// 1/(a + i b) = (a - i b)/(a^2 + b^2)
__device__ __forceinline__ double2 cinv(double a, double b) {
  const double d = a * a + b * b;
  return make_double2(a / d, -b / d);
}

// f[w][k] = (w_p/2) [1/(dE_p - omega_w + i delta) + 1/(dE_p + omega_w + i delta)],
// dE_p = E_v[p / n_c] - E_col[p % n_c], w_p = w_col[p % n_c] (or 1), p = p0 + k.
__global__ void k_weights(int64_t p0, int64_t K, int n_c, const double* __restrict__ E_v,
                          const double* __restrict__ E_col, const double* __restrict__ w_col,
                          const double2* __restrict__ omega, int n_freq, double delta, double2* __restrict__ f) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int64_t p = p0 + k;
  const int64_t iv = p / n_c, ic = p - iv * n_c;
  const double dE = E_v[iv] - E_col[ic];
  const double w = w_col ? w_col[ic] : 1.0;
  for (int iw = 0; iw < n_freq; ++iw) {
    const double2 om = omega[iw];
    const double2 a = cinv(dE - om.x, delta - om.y);
    const double2 b = cinv(dE + om.x, delta + om.y);
    f[(int64_t)iw * K + k] = make_double2(0.5 * w * (a.x + b.x), 0.5 * w * (a.y + b.y));
  }
}

constexpr int kT = 64;   // output tile
constexpr int kK = 16;   // pairs per shared-memory step

// one CTA per (64x64 tile of G', 64x64 tile of G, frequency); 16x16 threads, 4x4 outputs each
__global__ void __launch_bounds__(256)
k_contract_f64(int nG, const double2* __restrict__ M, int64_t K, const double2* __restrict__ f,
               double2* __restrict__ chi) {
  __shared__ double2 As[kK][kT];
  __shared__ double2 Bs[kK][kT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int H0 = blockIdx.x * kT, G0 = blockIdx.y * kT, iw = blockIdx.z;
  const double2* fw = f + (int64_t)iw * K;
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);
  for (int64_t k0 = 0; k0 < K; k0 += kK) {
    for (int e = threadIdx.x; e < kK * kT; e += blockDim.x) {
      const int kk = e / kT, g = e - kk * kT;
      const int64_t p = k0 + kk;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (p < K) {
        if (G0 + g < nG) a = cmul(fw[p], M[p * nG + G0 + g]);
        if (H0 + g < nG) {
          b = M[p * nG + H0 + g];
          b.y = -b.y;
        }
      }
      As[kk][g] = a;
      Bs[kk][g] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cfma(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int G = G0 + ty + 16 * r;
    if (G >= nG) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int H = H0 + tx + 16 * c;
      if (H >= nG) continue;
      double2* o = chi + ((int64_t)iw * nG + G) * nG + H;
      double2 v = *o;
      v.x += acc[r][c].x;
      v.y += acc[r][c].y;
      *o = v;
    }
  }
}

}  // namespace

cudaError_t launch_weights(const chi0_plan_s* p, int64_t p0, int64_t K, int n_c, const double* E_v,
                           const double* E_col, const double* w_col, double2* f, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  const int bs = 256;
  k_weights<<<(unsigned)((K + bs - 1) / bs), bs, 0, s>>>(p0, K, n_c, E_v, E_col, w_col, p->d_omega, p->n_freq,
                                                         p->delta, f);
  return cudaGetLastError();
}

cudaError_t launch_contract_f64(const chi0_plan_s* p, int nG, const double2* M, int64_t K, const double2* f,
                                double2* chi, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  const int t = (nG + kT - 1) / kT;
  dim3 grid(t, t, p->n_freq);
  k_contract_f64<<<grid, 256, 0, s>>>(nG, M, K, f, chi);
  return cudaGetLastError();
}

}  // namespace chi0

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP64 accumulate (no counterpart in the paper).
//
// Some callers cannot allocate device memory at the point where they need
// chi0: for example code running inside another framework that has reserved
// all device memory for its own pool, or a latency-critical loop in which a
// cudaMalloc (which may synchronise the device and can fail under memory
// pressure) is not acceptable.  A plan allocates its workspace, so those
// callers cannot use chi0_accumulate.  This variant needs no plan: the only
// scratch it uses (the FP64 frequency factors of one block of pairs) lives in
// the fixed array below, which every device that loads the library holds
// until the process exits.
// ---------------------------------------------------------------------------
namespace chi0 {
namespace {

constexpr int kNoAllocMaxFreq = 64;                       // frequencies per call
constexpr int64_t kNoAllocFactors = (int64_t)1 << 18;     // double2 entries: 4 MiB
static __device__ __align__(256) double2 g_noalloc_factors[kNoAllocFactors];

struct FreqList {
  double2 om[kNoAllocMaxFreq];
};

// f[w][k] as k_weights, with the frequencies passed by value
__global__ void k_weights_noalloc(int64_t p0, int64_t K, int n_c, const double* __restrict__ E_v,
                                  const double* __restrict__ E_col, const double* __restrict__ w_col, FreqList fl,
                                  int n_freq, double delta, double2* __restrict__ f) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int64_t p = p0 + k;
  const int64_t iv = p / n_c, ic = p - iv * n_c;
  const double dE = E_v[iv] - E_col[ic];
  const double w = w_col ? w_col[ic] : 1.0;
  for (int iw = 0; iw < n_freq; ++iw) {
    const double2 om = fl.om[iw];
    const double2 a = cinv(dE - om.x, delta - om.y);
    const double2 b = cinv(dE + om.x, delta + om.y);
    f[(int64_t)iw * K + k] = make_double2(0.5 * w * (a.x + b.x), 0.5 * w * (a.y + b.y));
  }
}

std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
// device address of the array per device, and the id of the CUDA context it was looked up in:
// a new context on the device (after cudaDeviceReset, or a context the caller made current
// through the driver API) holds its own copy of the array at its own address
struct NoAllocSlot {
  unsigned long long ctx_id;
  double2* ptr;
};
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices] = {};
PFN_cuCtxGetId_v12000 g_ctx_get_id = nullptr;
bool g_ctx_get_id_tried = false;

// unique id of the current context (ids are never reused within a process), 0 if unavailable
unsigned long long current_context_id() {
  if (!g_ctx_get_id_tried) {
    g_ctx_get_id_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    cudaGetLastError();
  }
  unsigned long long id = 0;
  if (!g_ctx_get_id || g_ctx_get_id(nullptr, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace
}  // namespace chi0

extern "C" chi0_status chi0_accumulate_fp64_noalloc(int n_G, const void* M, int n_v, int n_c, const double* E_v,
                                                    const double* E_col, const double* w_col, int n_freq,
                                                    const double* freq_re, const double* freq_im, double delta,
                                                    void* chi0, void* stream) {
  using namespace chi0;
  auto bad = [](const std::string& m) {
    set_global_error("chi0_accumulate_fp64_noalloc: " + m);
    return CHI0_ERR_INVALID;
  };
  if (n_G < 1 || n_G > 65536) return bad("n_G must be in [1, 65536]");
  if (n_freq < 1 || n_freq > kNoAllocMaxFreq)
    return bad("n_freq = " + std::to_string(n_freq) + " is outside [1, " + std::to_string(kNoAllocMaxFreq) +
               "], the fixed limit of this allocation-free path");
  if (n_v < 0 || n_c < 0) return bad("negative band count");
  if (!freq_re || !freq_im) return bad("NULL frequency array");
  if ((int64_t)n_v * n_c == 0) return CHI0_OK;
  if (!M || !E_v || !E_col || !chi0) return bad("NULL buffer");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    set_global_error("chi0_accumulate_fp64_noalloc: no usable current device");
    return CHI0_ERR_CUDA;
  }
  double2* scratch = nullptr;
  {
    // set-up, once per device and context, with that device current: the host-side name of
    // the array is only a stand-in, so look up its device address.  Without context ids
    // (an old driver) the address is looked up on every call.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();   // 0 before the runtime's first use of the device
    NoAllocSlot& slot = g_noalloc_slot[dev];
    if (!slot.ptr || ctx == 0 || slot.ctx_id != ctx) {
      double2* ptr = nullptr;
      e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_factors);
      if (e != cudaSuccess) {
        slot.ptr = nullptr;
        set_global_error(std::string("chi0_accumulate_fp64_noalloc: cudaGetSymbolAddress: ") +
                         cudaGetErrorString(e));
        cudaGetLastError();
        return CHI0_ERR_CUDA;
      }
      slot.ptr = ptr;
      slot.ctx_id = current_context_id();                   // the lookup made the context current
    }
    scratch = slot.ptr;
  }
  FreqList fl;
  for (int i = 0; i < kNoAllocMaxFreq; ++i) fl.om[i] = make_double2(i < n_freq ? freq_re[i] : 0.0, i < n_freq ? freq_im[i] : 0.0);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t np = (int64_t)n_v * n_c;
  const int64_t chunk = kNoAllocFactors / n_freq;   // pairs whose factors fit the array
  const int t = (n_G + kT - 1) / kT;
  for (int64_t p0 = 0; p0 < np; p0 += chunk) {
    const int64_t K = std::min<int64_t>(chunk, np - p0);
    // every factor the contraction reads is written first: nothing needs clearing
    k_weights_noalloc<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(p0, K, n_c, E_v, E_col, w_col, fl, n_freq, delta,
                                                                 scratch);
    k_contract_f64<<<dim3(t, t, n_freq), 256, 0, s>>>(n_G, (const double2*)M + p0 * n_G, K, scratch,
                                                     (double2*)chi0);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_global_error(std::string("chi0_accumulate_fp64_noalloc: launch: ") + cudaGetErrorString(e));
      return CHI0_ERR_CUDA;
    }
  }
  return CHI0_OK;
}
