// Frequency factors of Eq. 1 (FP64) and the plain FP64 contraction
//   chi0[w][G][G'] += sum_p f_p(w) M_p(G) conj(M_p(G'))
// on the CUDA cores (DFMA), used by CHI0_FP64 plans.
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
