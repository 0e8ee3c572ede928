// Adjoint of the contraction of Eq. 1.  With upstream Gamma_w = dL/dRe chi0_w
// + i dL/dIm chi0_w and chi0_w = sum_p f_p(w) M_p M_p^H:
//   grad M_p  = sum_w conj(f_p(w)) Gamma_w M_p + f_p(w) Gamma_w^H M_p
//   grad dE_p = sum_w Re( f'_p(w) conj(M_p^H Gamma_w M_p) ),
//   f'_p(w)   = -(w_p/2) [ (dE_p - w + i d)^-2 + (dE_p + w + i d)^-2 ],
// and dE_p = E_v[iv] - E_col[ic] gives grad E_v = sum_ic grad dE, grad E_col = -sum_iv grad dE.
//
// Diagonal upstream (Gamma_w = diag(g_w), g real): one fused bandwidth-bound pass
//   grad M_p(G) = sum_w 2 Re f_p(w) g_w(G) M_p(G),  grad dE_p = sum_w Re f'_p(w) sum_G g_w(G) |M_p(G)|^2.
// Dense upstream: two FP64 complex products per frequency, Y = M Gamma^T and
// Z = M conj(Gamma), combined in the epilogue.
#include "cplx.cuh"
#include "internal.h"

namespace chi0 {
namespace {

__device__ __forceinline__ double2 cinv_d(double a, double b) {
  const double d = a * a + b * b;
  return make_double2(a / d, -b / d);
}

// f and f' of pair p at frequency om
__device__ __forceinline__ void factors(double dE, double w, double2 om, double delta, double2* f, double2* fp) {
  const double2 a = cinv_d(dE - om.x, delta - om.y);
  const double2 b = cinv_d(dE + om.x, delta + om.y);
  *f = make_double2(0.5 * w * (a.x + b.x), 0.5 * w * (a.y + b.y));
  const double2 a2 = cmul(a, a), b2 = cmul(b, b);
  *fp = make_double2(-0.5 * w * (a2.x + b2.x), -0.5 * w * (a2.y + b2.y));
}

__device__ __forceinline__ double2 ld_d(const float2* p, int64_t i) {
  const float2 v = p[i];
  return make_double2(v.x, v.y);
}
__device__ __forceinline__ double2 ld_d(const double2* p, int64_t i) { return p[i]; }
__device__ __forceinline__ void st_c(float2* p, int64_t i, double2 v) { p[i] = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void st_c(double2* p, int64_t i, double2 v) { p[i] = v; }

constexpr int kMaxFreqBwd = 64;

// one CTA per pair of the block p0..p0+K; g is [n_freq][nG] real
template <typename C>
__global__ void __launch_bounds__(256)
k_bwd_diag(const C* __restrict__ M, int nG, int64_t p0, int64_t K, int n_c, const double* __restrict__ E_v,
           const double* __restrict__ E_col, const double* __restrict__ w_col, const double2* __restrict__ omega,
           int n_freq, double delta, const double* __restrict__ g, C* __restrict__ gM, double* __restrict__ gdE) {
  __shared__ double s_fr2[kMaxFreqBwd];   // 2 Re f
  __shared__ double s_fpr[kMaxFreqBwd];   // Re f'
  __shared__ double s_red[1][8];
  const int64_t k = blockIdx.x;
  const int64_t p = p0 + k;
  const int64_t iv = p / n_c, ic = p - iv * n_c;
  if (threadIdx.x < n_freq) {
    double2 f, fp;
    factors(E_v[iv] - E_col[ic], w_col ? w_col[ic] : 1.0, omega[threadIdx.x], delta, &f, &fp);
    s_fr2[threadIdx.x] = 2.0 * f.x;
    s_fpr[threadIdx.x] = fp.x;
  }
  __syncthreads();
  const C* Mp = M + k * nG;
  C* gp = gM + k * nG;
  // t = sum_G |M(G)|^2 sum_w Re f'(w) g_w(G)
  double t = 0.0;
  for (int G = threadIdx.x; G < nG; G += blockDim.x) {
    const double2 m = ld_d(Mp, G);
    const double m2 = m.x * m.x + m.y * m.y;
    double s = 0.0, s2 = 0.0;
    for (int iw = 0; iw < n_freq; ++iw) {
      const double gw = g[(int64_t)iw * nG + G];
      s = fma(s_fr2[iw], gw, s);
      s2 = fma(s_fpr[iw], gw, s2);
    }
    t = fma(s2, m2, t);
    st_c(gp, G, make_double2(s * m.x, s * m.y));
  }
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_red[0][warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_red[0][w];
    gdE[k] = sum;
  }
}

// dense upstream, one frequency: tile of 32 pairs x 64 sphere points, K loop over H
//   Y[p][G] = sum_H M[p][H] Gam[G][H],  Z[p][G] = sum_H M[p][H] conj(Gam[H][G])
//   gM[p][G] += conj(f_p) Y + f_p Z;  part[p][gt] += Re( f'_p conj(sum_{G in tile} conj(M[p][G]) Y[p][G]) )
template <typename C>
__global__ void __launch_bounds__(256)
k_bwd_dense(const C* __restrict__ M, int nG, int64_t p0, int64_t K, int n_c, const double* __restrict__ E_v,
            const double* __restrict__ E_col, const double* __restrict__ w_col, double2 om, double delta,
            const double2* __restrict__ Gam, C* __restrict__ gM, double* __restrict__ part, int ntile) {
  constexpr int TP = 32, TG = 64, TH = 16;
  __shared__ double2 Ms[TP][TH + 1];
  __shared__ double2 Gs[TG][TH + 1];     // Gam[G][H]
  __shared__ double2 Gt[TH][TG + 1];     // conj(Gam[H][G])
  __shared__ double2 sf[TP], sfp[TP];
  __shared__ double sq[TP][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads: 2 pairs x 4 points each
  const int64_t kp0 = (int64_t)blockIdx.y * TP;
  const int G0 = blockIdx.x * TG;
  if (threadIdx.x < TP) {
    const int64_t k = kp0 + threadIdx.x;
    double2 f = make_double2(0, 0), fp = make_double2(0, 0);
    if (k < K) {
      const int64_t p = p0 + k, iv = p / n_c, ic = p - iv * n_c;
      factors(E_v[iv] - E_col[ic], w_col ? w_col[ic] : 1.0, om, delta, &f, &fp);
    }
    sf[threadIdx.x] = f;
    sfp[threadIdx.x] = fp;
  }
  double2 y[2][4], z[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) y[r][c] = z[r][c] = make_double2(0, 0);
  for (int H0 = 0; H0 < nG; H0 += TH) {
    for (int e = threadIdx.x; e < TP * TH; e += blockDim.x) {
      const int r = e / TH, h = e - r * TH;
      const int64_t k = kp0 + r;
      Ms[r][h] = (k < K && H0 + h < nG) ? ld_d(M, k * nG + H0 + h) : make_double2(0, 0);
    }
    for (int e = threadIdx.x; e < TG * TH; e += blockDim.x) {
      const int gg = e / TH, h = e - gg * TH;
      const int G = G0 + gg, H = H0 + h;
      Gs[gg][h] = (G < nG && H < nG) ? Gam[(int64_t)G * nG + H] : make_double2(0, 0);
      const int hh = e / TG, g2 = e - hh * TG;
      const int Gb = G0 + g2, Hb = H0 + hh;
      double2 v = (Gb < nG && Hb < nG) ? Gam[(int64_t)Hb * nG + Gb] : make_double2(0, 0);
      v.y = -v.y;
      Gt[hh][g2] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int h = 0; h < TH; ++h) {
      double2 m[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) m[r] = Ms[ty + 16 * r][h];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double2 a = Gs[tx + 16 * c][h], b = Gt[h][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          cfma(y[r][c], m[r], a);
          cfma(z[r][c], m[r], b);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int rr = ty + 16 * r;
    const int64_t k = kp0 + rr;
    double2 qs = make_double2(0, 0);
    if (k < K) {
      const double2 f = sf[rr];
      const double2 fc = make_double2(f.x, -f.y);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int G = G0 + tx + 16 * c;
        if (G >= nG) continue;
        double2 gv = ld_d(gM, k * nG + G);
        const double2 t1 = cmul(fc, y[r][c]), t2 = cmul(f, z[r][c]);
        gv.x += t1.x + t2.x;
        gv.y += t1.y + t2.y;
        st_c(gM, k * nG + G, gv);
        const double2 m = ld_d(M, k * nG + G);
        cfma(qs, make_double2(m.x, -m.y), y[r][c]);
      }
    }
    sq[rr][tx] = 0.0;
    if (k < K) {
      const double2 fp = sfp[rr];
      sq[rr][tx] = fp.x * qs.x + fp.y * qs.y;     // Re(f' conj(q))
    }
  }
  __syncthreads();
  if (threadIdx.x < TP) {
    const int64_t k = kp0 + threadIdx.x;
    if (k < K) {
      double sum = 0.0;
      for (int t = 0; t < 16; ++t) sum += sq[threadIdx.x][t];
      part[k * ntile + blockIdx.x] += sum;
    }
  }
}

// gdE[k] = sum_t part[k][t]
__global__ void k_rowsum(const double* __restrict__ part, int64_t K, int ntile, double* __restrict__ gdE) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int t = 0; t < ntile; ++t) s += part[k * ntile + t];
  gdE[k] = s;
}

// grad E_v[iv] += sum of gdE over the block's pairs in row iv; grad E_col[ic] -= column sums
__global__ void k_reduce_rows(const double* __restrict__ gdE, int64_t p0, int64_t K, int n_c, double* __restrict__ gEv) {
  const int64_t iv = p0 / n_c + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t last = (p0 + K - 1) / n_c;
  if (iv > last) return;
  const int64_t a = max(p0, iv * n_c), b = min(p0 + K, (iv + 1) * n_c);
  double s = 0.0;
  for (int64_t p = a; p < b; ++p) s += gdE[p - p0];
  gEv[iv] += s;
}
__global__ void k_reduce_cols(const double* __restrict__ gdE, int64_t p0, int64_t K, int n_c, double* __restrict__ gEc) {
  const int64_t ic = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ic >= n_c) return;
  double s = 0.0;
  for (int64_t iv = p0 / n_c; iv * n_c + ic < p0 + K; ++iv) {
    const int64_t p = iv * n_c + ic;
    if (p >= p0) s += gdE[p - p0];
  }
  gEc[ic] -= s;
}

// Eq. 4 step edge e_k = min(E_0 + k dE, E_max), rounded as written (no fused multiply-add, so the
// value is the same as the host selection's)
__device__ __forceinline__ double step_edge(double E0, double dE, int k, double E_max) {
  return fmin(__dadd_rn(E0, __dmul_rn(dE, (double)k)), E_max);
}

// First-order estimate of the energy substitution of Eq. 3/4: every band c >= N0 takes the
// midpoint E_i of the Eq. 4 step [e_k, e_k+1) holding E_c (the last step closed, energies outside
// [E_0, E_max] to the end steps), and the estimate is sum_c sens_c (E_i(c) - E_c).  One block:
// each thread sums a fixed stride of bands, then a fixed tree in shared memory (deterministic).
constexpr int kEstThreads = 1024;
__global__ void __launch_bounds__(kEstThreads)
k_energy_substitution(const double* __restrict__ E_c, const double* __restrict__ sens, int n_c, int N0, double dE,
                      double E_max, double* __restrict__ E_sub, double* __restrict__ out) {
  __shared__ double red[kEstThreads];
  // E_0 = E_c of band N0 and N_E = ceil((E_max - E_0) / dE) steps, as the host selection has them
  const bool grid = N0 > 0 && N0 < n_c;
  const double E0 = grid ? E_c[N0 - 1] : 0.0;
  const int NE = grid ? (int)fmax(ceil((E_max - E0) / dE - 1e-12), 0.0) : 0;
  double acc = 0.0;
  for (int c = threadIdx.x; c < n_c; c += kEstThreads) {
    const double E = E_c[c];
    double Ei = E;
    if (c >= N0 && NE > 0) {
      // last k in [0, NE-1] with e_k <= E: start from the quotient, then step to the exact edge
      int k = (int)fmin(fmax(floor((E - E0) / dE), 0.0), (double)(NE - 1));
      while (k + 1 <= NE - 1 && step_edge(E0, dE, k + 1, E_max) <= E) ++k;
      while (k > 0 && step_edge(E0, dE, k, E_max) > E) --k;
      const double lo = step_edge(E0, dE, k, E_max), hi = step_edge(E0, dE, k + 1, E_max);
      Ei = __dmul_rn(0.5, __dadd_rn(lo, hi));
      acc = __dadd_rn(acc, __dmul_rn(sens[c], __dadd_rn(Ei, -E)));
    }
    if (E_sub) E_sub[c] = Ei;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kEstThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

cudaError_t launch_energy_substitution(const double* E_c, const double* sens, int n_c, int N0, double dE, double E_max,
                                       double* E_sub, double* out, cudaStream_t s) {
  k_energy_substitution<<<1, kEstThreads, 0, s>>>(E_c, sens, n_c, N0, dE, E_max, E_sub, out);
  return cudaGetLastError();
}

int bwd_max_freq() { return kMaxFreqBwd; }

template <typename C>
static cudaError_t bwd_impl(chi0_plan_s* p, int nG, const C* M, int64_t p0, int64_t K, int n_c, const double* E_v,
                            const double* E_col, const double* w_col, const double2* gamma, const double* diag,
                            C* gM, double* gEv, double* gEc, double* work, cudaStream_t s) {
  double* gdE = work;
  if (diag) {
    k_bwd_diag<C><<<(unsigned)K, 256, 0, s>>>(M, nG, p0, K, n_c, E_v, E_col, w_col, p->d_omega, p->n_freq, p->delta,
                                              diag, gM, gdE);
  } else {
    const int ntile = (nG + 63) / 64;
    double* part = work + K;
    cudaError_t e = cudaMemsetAsync(part, 0, sizeof(double) * (size_t)K * ntile, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(gM, 0, sizeof(C) * (size_t)K * nG, s);
    if (e != cudaSuccess) return e;
    dim3 grid(ntile, (unsigned)((K + 31) / 32));
    for (int iw = 0; iw < p->n_freq; ++iw) {
      const double2 om = make_double2(p->om_re[iw], p->om_im[iw]);
      k_bwd_dense<C><<<grid, 256, 0, s>>>(M, nG, p0, K, n_c, E_v, E_col, w_col, om, p->delta,
                                          gamma + (size_t)iw * nG * nG, gM, part, ntile);
    }
    k_rowsum<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(part, K, ntile, gdE);
  }
  const int64_t rows = (p0 + K - 1) / n_c - p0 / n_c + 1;
  k_reduce_rows<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(gdE, p0, K, n_c, gEv);
  k_reduce_cols<<<(unsigned)((n_c + 127) / 128), 128, 0, s>>>(gdE, p0, K, n_c, gEc);
  return cudaGetLastError();
}

cudaError_t launch_backward(chi0_plan_s* p, int nG, const void* M, int64_t p0, int64_t K, int n_c, const double* E_v,
                            const double* E_col, const double* w_col, const double2* gamma, const double* diag,
                            void* gM, double* gEv, double* gEc, double* work, cudaStream_t s) {
  if (is_split(p))
    return bwd_impl<float2>(p, nG, (const float2*)M + p0 * nG, p0, K, n_c, E_v, E_col, w_col, gamma, diag,
                            (float2*)gM + p0 * nG, gEv, gEc, work, s);
  return bwd_impl<double2>(p, nG, (const double2*)M + p0 * nG, p0, K, n_c, E_v, E_col, w_col, gamma, diag,
                           (double2*)gM + p0 * nG, gEv, gEc, work, s);
}

}  // namespace chi0
