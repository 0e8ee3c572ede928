// Coulomb-hole self-energy of Eq. 2 with the Hybertsen-Louie plasmon-pole
// model (the paper's extension of the static dielectric matrix to finite
// frequencies), for the full and the accelerated band sum:
//
//   Omega2_{GG'} = w_p^2 [(q+G).(q+G') / |q+G|^2] rho(G - G') / rho(0)
//   wt_{GG'}     = sqrt(Omega2_{GG'} / (delta_{GG'} - eps^-1_{GG'}(q, 0)))   (principal branch)
//   Sigma_t      = sum_b w_b sum_{GG'} m_tb(G) K_{GG'}(x_tb) conj(m_tb(G')),
//   K_{GG'}(x)   = Omega2_{GG'} v(q+G') / (2 wt_{GG'} (x - wt_{GG'} + i delta)),
//
// with m_tb(G) = <t| e^{iG.r} |b> (pair elements, target band first) and
// x_tb = E_t - E_b.  rho(d) is the Fourier coefficient of the density
// 2 sum_v |u_v(r)|^2 at the distinct differences d = G - G' of the sphere,
// computed by a transform pruned to the offsets those differences span.
#include <cuda_runtime.h>

#include "cplx.cuh"
#include "internal.h"

namespace chi0 {
namespace {

constexpr int CT = 32;          // COH tile: 32 x 32 (G, G') elements, 256 threads x 4
// bands per shared-memory chunk (FP64 tables keep the block under 48 KB of static shared memory)
template <typename R> struct CohBands { static constexpr int V = sizeof(R) == 4 ? 32 : 8; };

template <typename R>
__global__ void k_density(const typename Cx<R>::T* __restrict__ psi, int n_v, int64_t nr, double* __restrict__ dens) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < n_v; ++v) {
      const auto u = psi[(int64_t)v * nr + r];
      s += (double)u.x * (double)u.x + (double)u.y * (double)u.y;
    }
    dens[r] = 2.0 * s;
  }
}

// exp(-2 pi i (k j mod n) / n) with the phase reduced exactly in integers
__device__ __forceinline__ double2 twid(long long k, long long j, int n) {
  const long long m = ((k * j) % n + n) % n;
  double sn, cs;
  sincospi(-2.0 * (double)m / (double)n, &sn, &cs);
  return make_double2(cs, sn);
}

// rho(d) = (1/N_r) sum_r dens(r) exp(-2 pi i (d1 i1/n1 + d2 i2/n2 + d3 i3/n3)) for the
// distinct differences d, as three pruned passes over the offsets d_a in [-s_a, s_a]:
//   A1[i1][i2][k3] = sum_i3 dens * e3,  A2[i1][k2][k3] = sum_i2 A1 * e2,  rho(d) = sum_i1 A2 * e1 / N_r.
__global__ void k_dft_axis3(const double* __restrict__ dens, int n1, int n2, int n3, int s3,
                            double2* __restrict__ A1) {
  const int K3 = 2 * s3 + 1;
  const int64_t total = (int64_t)n1 * n2 * K3;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k3 = (int)(e % K3);
    const int64_t line = e / K3;                    // i1 * n2 + i2
    const double* row = dens + line * n3;
    double2 acc = make_double2(0.0, 0.0);
    for (int i3 = 0; i3 < n3; ++i3) {
      const double2 t = twid(k3 - s3, i3, n3);
      acc.x += row[i3] * t.x;
      acc.y += row[i3] * t.y;
    }
    A1[e] = acc;
  }
}

__global__ void k_dft_axis2(const double2* __restrict__ A1, int n1, int n2, int s2, int s3,
                            double2* __restrict__ A2) {
  const int K2 = 2 * s2 + 1, K3 = 2 * s3 + 1;
  const int64_t total = (int64_t)n1 * K2 * K3;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k3 = (int)(e % K3);
    const int k2 = (int)((e / K3) % K2);
    const int i1 = (int)(e / ((int64_t)K3 * K2));
    double2 acc = make_double2(0.0, 0.0);
    for (int i2 = 0; i2 < n2; ++i2)
      cfma(acc, A1[((int64_t)i1 * n2 + i2) * K3 + k3], twid(k2 - s2, i2, n2));
    A2[e] = acc;
  }
}

__global__ void k_dft_axis1(const double2* __restrict__ A2, int n1, int n2, int n3, int s2, int s3,
                            const int* __restrict__ dvec, int nd, double2* __restrict__ rho) {
  const int K2 = 2 * s2 + 1, K3 = 2 * s3 + 1;
  const double inv = 1.0 / ((double)n1 * n2 * n3);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x) {
    const int d1 = dvec[3 * j], k2 = dvec[3 * j + 1] + s2, k3 = dvec[3 * j + 2] + s3;
    double2 acc = make_double2(0.0, 0.0);
    for (int i1 = 0; i1 < n1; ++i1) cfma(acc, A2[((int64_t)i1 * K2 + k2) * K3 + k3], twid(d1, i1, n1));
    rho[j] = make_double2(acc.x * inv, acc.y * inv);
  }
}

// principal square root of z = x + i y.  Only the non-cancelling one of
// sqrt((|z| + x)/2) and sqrt((|z| - x)/2) is evaluated directly; the other part
// follows from 2 Re Im = y (for nearly real z the direct form of the small part
// would lose all its digits).
__device__ __forceinline__ double2 csqrt_principal(double2 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, z.y);
  if (z.x >= 0.0) {
    const double a = sqrt(0.5 * (r + z.x));
    return make_double2(a, z.y / (2.0 * a));
  }
  const double b = copysign(sqrt(0.5 * (r - z.x)), z.y);
  return make_double2(z.y / (2.0 * b), b);
}

// Omega2 and wt for every (G, G'); rho(G - G') / rho(0) via the difference index
// table (entry 0 of the difference list is the zero vector)
__global__ void k_gpp(const double2* __restrict__ eps_inv, const double2* __restrict__ rho, const int* __restrict__ idx,
                      const double* __restrict__ kvec, double wp2, int nG, double2* __restrict__ Om2,
                      double2* __restrict__ wt) {
  const int64_t n2 = (int64_t)nG * nG;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nG), j = (int)(e - (int64_t)i * nG);
    const double* ki = kvec + 3 * i;
    const double* kj = kvec + 3 * j;
    const double kk = ki[0] * kj[0] + ki[1] * kj[1] + ki[2] * kj[2];
    const double k2 = ki[0] * ki[0] + ki[1] * ki[1] + ki[2] * ki[2];
    const double2 rd = rho[idx[e]], z = rho[0];
    const double zz = z.x * z.x + z.y * z.y;
    const double2 r0 = make_double2((rd.x * z.x + rd.y * z.y) / zz, (rd.y * z.x - rd.x * z.y) / zz);
    const double s = wp2 * kk / k2;
    const double2 om = make_double2(s * r0.x, s * r0.y);
    const double2 ei = eps_inv[e];
    const double2 den = make_double2((i == j ? 1.0 : 0.0) - ei.x, -ei.y);
    double2 w = make_double2(0.0, 0.0);
    if (den.x != 0.0 || den.y != 0.0) {
      const double dd = den.x * den.x + den.y * den.y;
      const double2 q = make_double2((om.x * den.x + om.y * den.y) / dd, (om.y * den.x - om.x * den.y) / dd);
      w = csqrt_principal(q);
    }
    Om2[e] = om;
    wt[e] = w;
  }
}

// c = Omega2 v(G') / (2 wt) (zero without a pole), and wt, in the arithmetic type R
template <typename R>
__global__ void k_coh_coef(const double2* __restrict__ Om2, const double2* __restrict__ wt, const double* __restrict__ v,
                           int nG, typename Cx<R>::T* __restrict__ c, typename Cx<R>::T* __restrict__ wr) {
  const int64_t n2 = (int64_t)nG * nG;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % nG);
    const double2 om = Om2[e], w = wt[e];
    double2 q = make_double2(0.0, 0.0);
    const double ww = w.x * w.x + w.y * w.y;
    if (ww > 0.0 && (om.x != 0.0 || om.y != 0.0)) {
      const double s = 0.5 * v[j] / ww;     // om v / (2 w) = om conj(w) v / (2 |w|^2)
      q = make_double2(s * (om.x * w.x + om.y * w.y), s * (om.y * w.x - om.x * w.y));
    }
    c[e] = to_c(q, typename Cx<R>::T{});
    wr[e] = to_c(w, typename Cx<R>::T{});
  }
}

// partial[t][tile] = sum over the tile's (G, G') and every band b of
// w_b m(G) c (x - wt + i delta)^-1 conj(m(G')); chunks of CB bands in shared
// memory, FP64 sums of R-typed chunk sums.
template <typename R>
__global__ void __launch_bounds__(256)
k_sigma_coh(const typename Cx<R>::T* __restrict__ m, int n_b, int nG, const double* __restrict__ x,
            const double* __restrict__ wb, const typename Cx<R>::T* __restrict__ c,
            const typename Cx<R>::T* __restrict__ wt, double delta, double2* __restrict__ partial) {
  using C = typename Cx<R>::T;
  constexpr int CB = CohBands<R>::V;
  const int t = blockIdx.z;
  const int i0 = blockIdx.y * CT, j0 = blockIdx.x * CT;
  __shared__ C cs[CT][CT + 1], ws[CT][CT + 1];
  __shared__ C mi[CB][CT + 1], mj[CB][CT + 1];
  __shared__ R xs[CB];
  __shared__ double2 red[8];
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
    const int a = e / CT, b = e - a * CT;
    const int i = i0 + a, j = j0 + b;
    const bool in = i < nG && j < nG;
    cs[a][b] = in ? c[(size_t)i * nG + j] : cz(C{});
    ws[a][b] = in ? wt[(size_t)i * nG + j] : cz(C{});
  }
  double2 acc = make_double2(0.0, 0.0);
  const C* mt = m + (size_t)t * n_b * nG;
  for (int b0 = 0; b0 < n_b; b0 += CB) {
    __syncthreads();
    for (int e = threadIdx.x; e < CB * CT; e += blockDim.x) {
      const int bb = e / CT, g = e - bb * CT;
      const int b = b0 + bb;
      const bool okb = b < n_b;
      // the band weight rides on the G side: w_b m(G)
      const R wgt = okb ? (R)(wb ? wb[b] : 1.0) : (R)0;
      C u = (okb && i0 + g < nG) ? mt[(size_t)b * nG + i0 + g] : cz(C{});
      u.x *= wgt;
      u.y *= wgt;
      mi[bb][g] = u;
      mj[bb][g] = (okb && j0 + g < nG) ? mt[(size_t)b * nG + j0 + g] : cz(C{});
    }
    if (threadIdx.x < CB) {
      const int b = b0 + threadIdx.x;
      xs[threadIdx.x] = b < n_b ? (R)x[(size_t)t * n_b + b] : (R)0;
    }
    __syncthreads();
    // the thread's four elements share the column G' (rows a = tid/32 + 8q): m(G') and x are
    // read once per band
    C part = cz(C{});
    const int bcol = threadIdx.x & (CT - 1), a0 = threadIdx.x >> 5;
    C cc[4], wv[4];
    R dy[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cc[q] = cs[a0 + 8 * q][bcol];
      wv[q] = ws[a0 + 8 * q][bcol];
      dy[q] = (R)delta - wv[q].y;
    }
#pragma unroll 2
    for (int bb = 0; bb < CB; ++bb) {
      const C mjv = mj[bb][bcol];
      const R xb = xs[bb];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // c / (x - wt + i delta) = c conj(d) / |d|^2,  d = dx + i dy (c = 0: no pole, adds 0)
        const R dx = xb - wv[q].x;
        R inv;
        if constexpr (sizeof(R) == 4)
          inv = __fdividef(1.0f, dx * dx + dy[q] * dy[q]);   // 2-ulp reciprocal: terms carry FP32 errors anyway
        else
          inv = (R)1 / (dx * dx + dy[q] * dy[q]);
        C cr;                                                 // c conj(d)
        cr.x = fma(cc[q].x, dx, cc[q].y * dy[q]);
        cr.y = fma(cc[q].y, dx, -(cc[q].x * dy[q]));
        const C mm = cconjmul(mjv, mi[bb][a0 + 8 * q]);       // w_b m(G) conj(m(G'))
        const C t2 = cmul(mm, cr);
        part.x = fma(t2.x, inv, part.x);
        part.y = fma(t2.y, inv, part.y);
      }
    }
    acc.x += (double)part.x;
    acc.y += (double)part.y;
  }
  for (int o = 16; o; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < 8; ++w) {
      s.x += red[w].x;
      s.y += red[w].y;
    }
    partial[((size_t)t * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
  }
}

}  // namespace

cudaError_t launch_density(const chi0_plan_s* p, const void* psi_v, int n_v, double* dens, cudaStream_t s) {
  if (is_split(p))
    k_density<float><<<4 * 152, 256, 0, s>>>((const float2*)psi_v, n_v, p->nr, dens);
  else
    k_density<double><<<4 * 152, 256, 0, s>>>((const double2*)psi_v, n_v, p->nr, dens);
  return cudaGetLastError();
}

size_t density_ft_ws_bytes(const chi0_plan_s* p, int s2, int s3) {
  const size_t K2 = 2 * (size_t)s2 + 1, K3 = 2 * (size_t)s3 + 1;
  return ((size_t)p->n1 * p->n2 * K3 + (size_t)p->n1 * K2 * K3) * sizeof(double2);
}

cudaError_t launch_density_ft(const chi0_plan_s* p, const double* dens, const int* dvec, int nd, int s2, int s3,
                              void* ws, double2* rho, cudaStream_t s) {
  if (nd <= 0) return cudaSuccess;
  double2* A1 = reinterpret_cast<double2*>(ws);
  double2* A2 = A1 + (size_t)p->n1 * p->n2 * (2 * s3 + 1);
  k_dft_axis3<<<4 * 152, 256, 0, s>>>(dens, p->n1, p->n2, p->n3, s3, A1);
  k_dft_axis2<<<4 * 152, 256, 0, s>>>(A1, p->n1, p->n2, s2, s3, A2);
  k_dft_axis1<<<(nd + 255) / 256, 256, 0, s>>>(A2, p->n1, p->n2, p->n3, s2, s3, dvec, nd, rho);
  return cudaGetLastError();
}

cudaError_t launch_gpp(int nG, const double2* eps_inv, const double2* rho, const int* idx, const double* kvec,
                       double wp2, double2* Om2, double2* wt, cudaStream_t s) {
  k_gpp<<<4 * 152, 256, 0, s>>>(eps_inv, rho, idx, kvec, wp2, nG, Om2, wt);
  return cudaGetLastError();
}

size_t sigma_coh_ws_bytes(const chi0_plan_s* p, int nG, int n_t) {
  const size_t c = is_split(p) ? sizeof(float2) : sizeof(double2);
  const size_t tiles = (size_t)((nG + CT - 1) / CT) * ((nG + CT - 1) / CT);
  return 2 * (size_t)nG * nG * c + (size_t)n_t * tiles * sizeof(double2) + 256;
}

cudaError_t launch_sigma_coh(const chi0_plan_s* p, int nG, const void* m, int n_t, int n_b, const double* x,
                             const double* w, const double2* Om2, const double2* wt, const double* v, double delta,
                             void* ws, double2* partial_host_order, int* n_tiles, cudaStream_t s) {
  const int T = (nG + CT - 1) / CT;
  *n_tiles = T * T;
  const size_t cb = is_split(p) ? sizeof(float2) : sizeof(double2);
  unsigned char* b = reinterpret_cast<unsigned char*>(ws);
  void* cbuf = b;
  void* wbuf = b + (size_t)nG * nG * cb;
  dim3 grid(T, T, n_t);
  if (is_split(p)) {
    k_coh_coef<float><<<4 * 152, 256, 0, s>>>(Om2, wt, v, nG, (float2*)cbuf, (float2*)wbuf);
    k_sigma_coh<float><<<grid, 256, 0, s>>>((const float2*)m, n_b, nG, x, w, (const float2*)cbuf,
                                            (const float2*)wbuf, delta, partial_host_order);
  } else {
    k_coh_coef<double><<<4 * 152, 256, 0, s>>>(Om2, wt, v, nG, (double2*)cbuf, (double2*)wbuf);
    k_sigma_coh<double><<<grid, 256, 0, s>>>((const double2*)m, n_b, nG, x, w, (const double2*)cbuf,
                                             (const double2*)wbuf, delta, partial_host_order);
  }
  return cudaGetLastError();
}

}  // namespace chi0
