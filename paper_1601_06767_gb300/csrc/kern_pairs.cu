// Wavefunctions on the grid and pair matrix elements M_vc(q,G) (definition
// following Eq. 1): pointwise products conj(psi_v) psi_c on each grid plane,
// pruned forward transforms along i3 and i2 inside the plane (stages 1-2),
// then the transform along i1 evaluated only on the G sphere (stage 3).
//
// FP32 plans on cubic grids of 24, 36, 48 or 96 points transform with
// register FFTs (length-Q FFTs of P interleaved sub-sequences); FP64 plans and
// other grids use direct sums with exact twiddle tables.  Both are restricted
// to the frequencies the sphere needs, and the three stages together equal
// M(G) = (1/N_r) sum_r conj(psi_v(r)) psi_c(r) exp(2 pi i G.r).
#include <algorithm>
#include <type_traits>

#include "cplx.cuh"
#include "internal.h"

namespace chi0 {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// psi[b][i1][i2][i3] = sum_g c_b(g) exp(2 pi i g.r): one CTA per (plane i1, band b)
// stage A: along g1 for every (g2,g3) column of the sphere (sparse)
// stage B: along g2 for every (i2, g3); stage C: along g3 for every (i2, i3)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_wfn_to_grid(const double2* __restrict__ coeff, int npw, int n1, int n2, int n3, int nw1, int nw2,
              int nw3, const int* __restrict__ col_start, const int* __restrict__ col_pw,
              const int* __restrict__ col_g1, const typename Cx<R>::T* __restrict__ T1,
              const typename Cx<R>::T* __restrict__ T2, const typename Cx<R>::T* __restrict__ T3t,
              typename Cx<R>::T* __restrict__ psi) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);   // [nw2][nw3]
  C* B = A + nw2 * nw3;                    // [n2][nw3]
  const int i1 = blockIdx.x;
  const int64_t b = blockIdx.y;
  const double2* cb = coeff + b * npw;
  const C* T1r = T1 + (size_t)i1 * nw1;
  for (int e = threadIdx.x; e < nw2 * nw3; e += blockDim.x) {
    C acc = cz(C());
    const int k1 = col_start[e + 1];
    for (int k = col_start[e]; k < k1; ++k) cfma(acc, to_c(cb[col_pw[k]], C()), T1r[col_g1[k]]);
    A[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n2 * nw3; e += blockDim.x) {
    const int i2 = e / nw3, g3 = e - i2 * nw3;
    const C* t = T2 + (size_t)i2 * nw2;
    C acc = cz(C());
    for (int g2 = 0; g2 < nw2; ++g2) cfma(acc, A[g2 * nw3 + g3], t[g2]);
    B[e] = acc;
  }
  __syncthreads();
  C* out = psi + ((size_t)b * n1 + i1) * (size_t)n2 * n3;
  for (int e = threadIdx.x; e < n2 * n3; e += blockDim.x) {
    const int i2 = e / n3, i3 = e - i2 * n3;
    const C* brow = B + i2 * nw3;
    C acc = cz(C());
    for (int g3 = 0; g3 < nw3; ++g3) cfma(acc, brow[g3], T3t[(size_t)g3 * n3 + i3]);
    out[e] = acc;
  }
}

// ---------------------------------------------------------------------------
// The same three stages in FP32 for WPL planes per CTA, with the tables in
// shared memory and every load reused: stage A applies each coefficient to the
// WPL planes, stages B and C give each thread 4 consecutive outputs (i2 or i3)
// that share the input value and read their 4 twiddles as two 16-byte loads;
// stage C writes 4 consecutive i3 (32 bytes) per thread.
// Shared memory: A[WPL][nw2][nw3], B[WPL][n2][nw3], T2s[nw2][n2] (transposed),
// T3s[nw3][n3], T1s[WPL][nw1].
// ---------------------------------------------------------------------------
constexpr int WPL = 4;

size_t wfn_blk_smem(const chi0_plan_s* p) {
  const WfnSphere& w = p->w;
  return ((size_t)WPL * w.nw2 * w.nw3 + (size_t)WPL * p->n2 * w.nw3 + (size_t)w.nw2 * p->n2 +
          (size_t)w.nw3 * p->n3 + (size_t)WPL * w.nw1) * sizeof(float2);
}

__global__ void __launch_bounds__(kThreads, 2)
k_wfn_to_grid_blk(const double2* __restrict__ coeff, int npw, int n1, int n2, int n3, int nw1, int nw2, int nw3,
                  const int* __restrict__ col_start, const int* __restrict__ col_pw, const int* __restrict__ col_g1,
                  const float2* __restrict__ T1, const float2* __restrict__ T2, const float2* __restrict__ T3t,
                  float2* __restrict__ psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cw = nw2 * nw3;
  float2* A = reinterpret_cast<float2*>(smem_raw);   // [WPL][cw]
  float2* B = A + WPL * cw;                          // [WPL][n2][nw3]
  float2* T2s = B + WPL * n2 * nw3;                  // [nw2][n2]
  float2* T3s = T2s + nw2 * n2;                      // [nw3][n3]
  float2* T1s = T3s + nw3 * n3;                      // [WPL][nw1]
  const int i1_0 = blockIdx.x * WPL;
  const int npl = min(WPL, n1 - i1_0);
  const int64_t b = blockIdx.y;
  const double2* cb = coeff + b * npw;
  for (int e = threadIdx.x; e < nw2 * n2; e += blockDim.x) {
    const int g2 = e / n2, i2 = e - g2 * n2;
    T2s[e] = T2[(size_t)i2 * nw2 + g2];
  }
  for (int e = threadIdx.x; e < nw3 * n3; e += blockDim.x) T3s[e] = T3t[e];
  for (int e = threadIdx.x; e < WPL * nw1; e += blockDim.x) {
    const int pl = e / nw1, g1 = e - pl * nw1;
    T1s[e] = pl < npl ? T1[(size_t)(i1_0 + pl) * nw1 + g1] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // stage A: along g1 for every (g2, g3) column of the sphere, all planes at once
  for (int c = threadIdx.x; c < cw; c += blockDim.x) {
    float2 acc[WPL];
#pragma unroll
    for (int pl = 0; pl < WPL; ++pl) acc[pl] = make_float2(0.f, 0.f);
    const int k1 = col_start[c + 1];
    for (int k = col_start[c]; k < k1; ++k) {
      const double2 d = cb[col_pw[k]];
      const float2 v = make_float2((float)d.x, (float)d.y);
      const int g1 = col_g1[k];
#pragma unroll
      for (int pl = 0; pl < WPL; ++pl) cfma(acc[pl], v, T1s[pl * nw1 + g1]);
    }
#pragma unroll
    for (int pl = 0; pl < WPL; ++pl) A[pl * cw + c] = acc[pl];
  }
  __syncthreads();
  // stage B: B[pl][i2][g3] = sum_g2 A[pl][g2][g3] T2(i2, g2), four i2 per thread
  const int n2q = n2 >> 2;
  for (int it = threadIdx.x; it < npl * n2q * nw3; it += blockDim.x) {
    const int g3 = it % nw3, r = it / nw3, q = r % n2q, pl = r / n2q;
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.f, 0.f);
    const float2* a = A + pl * cw + g3;
    for (int g2 = 0; g2 < nw2; ++g2) {
      const float2 x = a[g2 * nw3];
      const float4 t01 = *reinterpret_cast<const float4*>(T2s + g2 * n2 + 4 * q);
      const float4 t23 = *reinterpret_cast<const float4*>(T2s + g2 * n2 + 4 * q + 2);
      cfma(acc[0], x, make_float2(t01.x, t01.y));
      cfma(acc[1], x, make_float2(t01.z, t01.w));
      cfma(acc[2], x, make_float2(t23.x, t23.y));
      cfma(acc[3], x, make_float2(t23.z, t23.w));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) B[(pl * n2 + 4 * q + j) * nw3 + g3] = acc[j];
  }
  __syncthreads();
  // stage C: psi[i1][i2][i3] = sum_g3 B[pl][i2][g3] T3(g3, i3), four i3 per thread
  const int n3q = n3 >> 2;
  for (int it = threadIdx.x; it < npl * n2 * n3q; it += blockDim.x) {
    const int q = it % n3q, r = it / n3q, i2 = r % n2, pl = r / n2;
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.f, 0.f);
    const float2* brow = B + (pl * n2 + i2) * nw3;
    for (int g3 = 0; g3 < nw3; ++g3) {
      const float2 x = brow[g3];
      const float4 t01 = *reinterpret_cast<const float4*>(T3s + g3 * n3 + 4 * q);
      const float4 t23 = *reinterpret_cast<const float4*>(T3s + g3 * n3 + 4 * q + 2);
      cfma(acc[0], x, make_float2(t01.x, t01.y));
      cfma(acc[1], x, make_float2(t01.z, t01.w));
      cfma(acc[2], x, make_float2(t23.x, t23.y));
      cfma(acc[3], x, make_float2(t23.z, t23.w));
    }
    float4* out = reinterpret_cast<float4*>(psi + (((size_t)b * n1 + i1_0 + pl) * n2 + i2) * n3 + 4 * q);
    out[0] = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
    out[1] = make_float4(acc[2].x, acc[2].y, acc[3].x, acc[3].y);
  }
}

// ---------------------------------------------------------------------------
// Stages 1+2 for one plane i1, a tile of TV valence bands and a run of
// conduction bands.  Shared memory: Uv[TV][n2][ld3], Uc[n2][ld3], X[TV][n2][nk3p].
//   stage 1: X_j(i2,k3) = sum_i3 conj(u_vj(i1,i2,i3)) u_c(i1,i2,i3) e^{2 pi i k3 i3/n3}
//   stage 2: D_p(i1,k2,k3) = sum_i2 X_j(i2,k3) e^{2 pi i k2 i2/n2}
// D is [pair][i1][nk2][nk3], pair = jv*nc + jc local to the chunk.
// ---------------------------------------------------------------------------
template <typename R, int TV>
__global__ void __launch_bounds__(kThreads)
k_pair_planes(const typename Cx<R>::T* __restrict__ psi_v, const int32_t* __restrict__ v_idx, int v0,
              int nv, const typename Cx<R>::T* __restrict__ psi_c, const int32_t* __restrict__ c_idx,
              int c0, int nc, int c_per_cta, int n1, int n2, int n3, int ld3, int nk2, int nk3, int nk2p,
              int nk3p, const typename Cx<R>::T* __restrict__ T2, const typename Cx<R>::T* __restrict__ T3,
              typename Cx<R>::T* __restrict__ D) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Uv = reinterpret_cast<C*>(smem_raw);
  C* Uc = Uv + (size_t)TV * n2 * ld3;
  C* X = Uc + (size_t)n2 * ld3;
  const int i1 = blockIdx.x;
  const int jv0 = blockIdx.y * TV;
  const int jc_begin = blockIdx.z * c_per_cta;
  const int jc_end = min(nc, jc_begin + c_per_cta);
  const int64_t nr = (int64_t)n1 * n2 * n3;
  const int plane = n2 * n3;
  const int64_t box = (int64_t)nk2 * nk3;

  for (int j = 0; j < TV; ++j) {
    const int jv = jv0 + j;
    const bool ok = jv < nv;
    const int64_t band = ok ? (v_idx ? v_idx[v0 + jv] : v0 + jv) : 0;
    const C* src = psi_v + band * nr + (int64_t)i1 * plane;
    for (int e = threadIdx.x; e < plane; e += blockDim.x) {
      const int i2 = e / n3, i3 = e - i2 * n3;
      Uv[((size_t)j * n2 + i2) * ld3 + i3] = ok ? src[e] : cz(C());
    }
  }
  const int items1 = n2 * (nk3p >> 2);
  const int items2 = nk3 * (nk2p >> 2);
  for (int jc = jc_begin; jc < jc_end; ++jc) {
    const int64_t band = c_idx ? c_idx[c0 + jc] : c0 + jc;
    const C* src = psi_c + band * nr + (int64_t)i1 * plane;
    for (int e = threadIdx.x; e < plane; e += blockDim.x) {
      const int i2 = e / n3, i3 = e - i2 * n3;
      Uc[(size_t)i2 * ld3 + i3] = src[e];
    }
    __syncthreads();
    // stage 1 (along i3)
    for (int it = threadIdx.x; it < items1; it += blockDim.x) {
      const int i2 = it % n2, kb = (it / n2) << 2;
      C acc[TV][4];
#pragma unroll
      for (int j = 0; j < TV; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = cz(C());
      const C* uc = Uc + (size_t)i2 * ld3;
      for (int i3 = 0; i3 < n3; ++i3) {
        const C c = uc[i3];
        const C* t = T3 + (size_t)i3 * nk3p + kb;
        C tw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) tw[q] = __ldg(t + q);
#pragma unroll
        for (int j = 0; j < TV; ++j) {
          const C rho = cconjmul(Uv[((size_t)j * n2 + i2) * ld3 + i3], c);
#pragma unroll
          for (int q = 0; q < 4; ++q) cfma(acc[j][q], rho, tw[q]);
        }
      }
#pragma unroll
      for (int j = 0; j < TV; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) X[((size_t)j * n2 + i2) * nk3p + kb + q] = acc[j][q];
    }
    __syncthreads();
    // stage 2 (along i2)
    for (int it = threadIdx.x; it < items2; it += blockDim.x) {
      const int k3 = it % nk3, kb = (it / nk3) << 2;
      C acc[TV][4];
#pragma unroll
      for (int j = 0; j < TV; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = cz(C());
      for (int i2 = 0; i2 < n2; ++i2) {
        const C* t = T2 + (size_t)i2 * nk2p + kb;
        C tw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) tw[q] = __ldg(t + q);
#pragma unroll
        for (int j = 0; j < TV; ++j) {
          const C x = X[((size_t)j * n2 + i2) * nk3p + k3];
#pragma unroll
          for (int q = 0; q < 4; ++q) cfma(acc[j][q], x, tw[q]);
        }
      }
#pragma unroll
      for (int j = 0; j < TV; ++j) {
        const int jv = jv0 + j;
        if (jv >= nv) continue;
        C* dst = D + ((int64_t)(jv * nc + jc) * n1 + i1) * box + k3;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (kb + q < nk2) dst[(int64_t)(kb + q) * nk3] = acc[j][q];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Stage 3: M[row][j] = (1/N_r) sum_i1 D_p(i1, k2_j, k3_j) e^{2 pi i k1_j i1/n1}
// one CTA per local pair; sphere points visited in column order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pair_gather(const typename Cx<R>::T* __restrict__ D, int nc, int64_t row0, int64_t ldv, int n1,
              int64_t box, int nG, int nk1, const int* __restrict__ ent_box, const int* __restrict__ ent_k1,
              const int* __restrict__ ent_j, const typename Cx<R>::T* __restrict__ T1, R scale,
              typename Cx<R>::T* __restrict__ M) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* T1s = reinterpret_cast<C*>(smem_raw);
  for (int e = threadIdx.x; e < n1 * nk1; e += blockDim.x) T1s[e] = T1[e];
  __syncthreads();
  const int pl = blockIdx.x;
  const int jv = pl / nc, jc = pl - jv * nc;
  const int64_t row = row0 + (int64_t)jv * ldv + jc;
  const C* Dp = D + (int64_t)pl * n1 * box;
  C* out = M + row * nG;
  for (int t = threadIdx.x; t < nG; t += blockDim.x) {
    const int off = ent_box[t], k1 = ent_k1[t];
    C acc = cz(C());
    for (int i1 = 0; i1 < n1; ++i1) cfma(acc, Dp[(int64_t)i1 * box + off], T1s[i1 * nk1 + k1]);
    acc.x *= scale;
    acc.y *= scale;
    out[ent_j[t]] = acc;
  }
}

// ---------------------------------------------------------------------------
// Stages 1+2 with register FFTs, for cubic grids n = P*Q with Q a power of two.
// The frequency shift to the lowest kept k (k2min, k3min) is folded into the
// valence planes when they are loaded:  u_v'(i2,i3) = u_v(i2,i3) e^{-2 pi i (k3min i3 + k2min i2)/n},
// so each line transform only needs its first nk outputs:
//   sum_i x(i) e^{2 pi i kk i/n} = sum_{a<P} e^{2 pi i a kk/n} F_a(kk mod Q),
//   F_a(m) = sum_{b<Q} x(a + P b) e^{2 pi i b m/Q}   (Q-point FFT in registers).
// Shared memory: Uv'[TV][n][ld], Uc[NCB][n][ld], X[NCB][TV][n][ldx].
// ---------------------------------------------------------------------------
constexpr int NKMAX = 28;

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int Q>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < Q; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// n-th roots of unity as compile-time constants in constant memory, so that the
// register FFTs multiply by constant-bank operands (no shared-memory twiddle
// loads, no registers held for them).  Values: cos and sin of 2 pi m / n from
// their Taylor series in double, evaluated by the compiler on |x| <= pi/4 after
// an exact reduction of m / n to the first octant, then rounded to float.
constexpr double kTwoPi = 6.283185307179586476925;
constexpr double cx_sin_series(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / (double)((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
constexpr double cx_cos_series(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / (double)((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
template <int N> struct Roots {
  float re[N];
  float im[N];
};
template <int N>
constexpr Roots<N> make_roots() {
  Roots<N> r{};
  for (int m = 0; m < N; ++m) {
    const int q = (4 * m) / N;                 // quadrant
    const int num = 4 * m - q * N;             // angle within the quadrant = 2 pi num / (4 N), num in [0, N)
    double c = 0.0, sn = 0.0;
    if (2 * num <= N) {                        // <= pi/4
      const double x = kTwoPi * num / (4.0 * N);
      c = cx_cos_series(x);
      sn = cx_sin_series(x);
    } else {                                   // complement, pi/2 - angle < pi/4
      const double x = kTwoPi * (N - num) / (4.0 * N);
      c = cx_sin_series(x);
      sn = cx_cos_series(x);
    }
    double re = c, im = sn;
    if (q == 1) { re = -sn; im = c; }
    if (q == 2) { re = -c; im = -sn; }
    if (q == 3) { re = sn; im = -c; }
    r.re[m] = (float)re;
    r.im[m] = (float)im;
  }
  return r;
}
constexpr Roots<24> k_roots24 = make_roots<24>();
constexpr Roots<36> k_roots36 = make_roots<36>();
constexpr Roots<48> k_roots48 = make_roots<48>();
constexpr Roots<96> k_roots96 = make_roots<96>();
__constant__ Roots<24> c_roots24 = k_roots24;
__constant__ Roots<36> c_roots36 = k_roots36;
__constant__ Roots<48> c_roots48 = k_roots48;
__constant__ Roots<96> c_roots96 = k_roots96;

// combination factors e^{2 pi i a kk / N} of the P sub-transforms, [a][kk] for kk < NKMAX,
// so that a runtime sub-transform index a costs one address computation
template <int P, int N> struct CombTable {
  float re[P][NKMAX];
  float im[P][NKMAX];
};
template <int P, int N>
constexpr CombTable<P, N> make_comb(const Roots<N>& r) {
  CombTable<P, N> t{};
  for (int a = 0; a < P; ++a)
    for (int kk = 0; kk < NKMAX; ++kk) {
      t.re[a][kk] = r.re[(a * kk) % N];
      t.im[a][kk] = r.im[(a * kk) % N];
    }
  return t;
}
constexpr CombTable<3, 24> k_comb24 = make_comb<3, 24>(k_roots24);
constexpr CombTable<9, 36> k_comb36 = make_comb<9, 36>(k_roots36);
constexpr CombTable<3, 48> k_comb48 = make_comb<3, 48>(k_roots48);
constexpr CombTable<3, 96> k_comb96 = make_comb<3, 96>(k_roots96);
__constant__ CombTable<3, 24> c_comb24 = k_comb24;
__constant__ CombTable<9, 36> c_comb36 = k_comb36;
__constant__ CombTable<3, 48> c_comb48 = k_comb48;
__constant__ CombTable<3, 96> c_comb96 = k_comb96;

template <int N>
__device__ __forceinline__ float2 comb(int a, int kk) {
  static_assert(N == 24 || N == 36 || N == 48 || N == 96, "no combination table for this length");
  if constexpr (N == 24) return make_float2(c_comb24.re[a][kk], c_comb24.im[a][kk]);
  if constexpr (N == 36) return make_float2(c_comb36.re[a][kk], c_comb36.im[a][kk]);
  if constexpr (N == 48) return make_float2(c_comb48.re[a][kk], c_comb48.im[a][kk]);
  if constexpr (N == 96) return make_float2(c_comb96.re[a][kk], c_comb96.im[a][kk]);
}

// e^{2 pi i m / N}, 0 <= m < N
template <int N>
__device__ __forceinline__ float2 root(int m) {
  static_assert(N == 24 || N == 36 || N == 48 || N == 96, "no root table for this length");
  if constexpr (N == 24) return make_float2(c_roots24.re[m], c_roots24.im[m]);
  if constexpr (N == 36) return make_float2(c_roots36.re[m], c_roots36.im[m]);
  if constexpr (N == 48) return make_float2(c_roots48.re[m], c_roots48.im[m]);
  if constexpr (N == 96) return make_float2(c_roots96.re[m], c_roots96.im[m]);
}

// in-place Q-point transform with e^{+2 pi i/Q}, twiddles from the N-th roots (Q | N)
template <int Q, int N>
__device__ __forceinline__ void fft_reg(float2 (&x)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int j = bitrev<Q>(i);
    if (j > i) {
      const float2 t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  constexpr int LOG2Q = (Q >= 32) ? 5 : (Q >= 16) ? 4 : (Q >= 8) ? 3 : (Q >= 4) ? 2 : 1;
  static_assert((1 << LOG2Q) == Q, "Q must be a power of two <= 32");
  static_assert(N % Q == 0, "Q must divide N");
  // stage loop with an additive counter so that it unrolls completely and x stays in registers
#pragma unroll
  for (int stage = 0; stage < LOG2Q; ++stage) {
    const int len = 2 << stage;
#pragma unroll
    for (int i = 0; i < Q; i += len) {
#pragma unroll
      for (int k = 0; k < len / 2; ++k) {
        const float2 u = x[i + k];
        float2 v = x[i + k + len / 2];
        const int e = k * (Q / len);
        if (e == 0) {
        } else if (4 * e == Q) {           // multiply by i
          v = make_float2(-v.y, v.x);
        } else {
          v = cmul(v, root<N>(e * (N / Q)));
        }
        x[i + k] = make_float2(u.x + v.x, u.y + v.y);
        x[i + k + len / 2] = make_float2(u.x - v.x, u.y - v.y);
      }
    }
  }
}

// acc[kk] = sum over the P sub-sequences of one length-n line, for every kk < NK
// (the caller uses the first nk; computing all NK avoids a predicate per output)
template <int P, int Q, int NK, typename Load>
__device__ __forceinline__ void line_transform(Load load, float2 (&acc)[NK]) {
  constexpr int n = P * Q;
  {
    float2 x[Q];
#pragma unroll
    for (int b = 0; b < Q; ++b) x[b] = load(P * b);
    fft_reg<Q, n>(x);
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) acc[kk] = x[kk % Q];
  }
  if constexpr (P <= 3 && Q <= 16) {
    // unrolled: every twiddle index is a compile-time constant
#pragma unroll
    for (int a = 1; a < P; ++a) {
      float2 x[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) x[b] = load(a + P * b);
      fft_reg<Q, n>(x);
#pragma unroll
      for (int kk = 0; kk < NK; ++kk) cfma(acc[kk], x[kk % Q], root<n>((a * kk) % n));
    }
  } else {
    // long or many sub-transforms: one at a time (registers), factors by row a of the table
#pragma unroll 1
    for (int a = 1; a < P; ++a) {
      float2 x[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) x[b] = load(a + P * b);
      fft_reg<Q, n>(x);
#pragma unroll
      for (int kk = 0; kk < NK; ++kk) cfma(acc[kk], x[kk % Q], comb<n>(a, kk));
    }
  }
}

template <int P, int Q, int NK, int TV, int NCB>
__global__ void __launch_bounds__(192, (TV * NCB >= 4) ? 2 : 1)
k_pair_planes_fft(const float2* __restrict__ psi_v, const int32_t* __restrict__ v_idx, int v0, int nv,
                  const float2* __restrict__ psi_c, const int32_t* __restrict__ c_idx, int c0, int nc, int c_per_cta,
                  int nk2, int nk3, int nk2p, int nk3p, const float2* __restrict__ T2, const float2* __restrict__ T3,
                  float2* __restrict__ D) {
  constexpr int n = P * Q;
  constexpr int ld = n | 1;
  constexpr int NP = NCB * TV;                               // pairs per iteration
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldx = nk3 | 1;
  float2* Uv = reinterpret_cast<float2*>(smem_raw);          // [TV][n][ld]
  float2* Uc = Uv + TV * n * ld;                             // [NCB][n][ld]
  float2* X = Uc + NCB * n * ld;                             // [NP][n][ldx]
  const int i1 = blockIdx.x;
  const int jv0 = blockIdx.y * TV;
  const int jc_begin = blockIdx.z * c_per_cta;
  const int jc_end = min(nc, jc_begin + c_per_cta);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  constexpr int64_t nr = (int64_t)n * n * n;
  constexpr int plane = n * n;
  const int64_t box = (int64_t)nk2 * nk3;

  for (int j = 0; j < TV; ++j) {
    const int jv = jv0 + j;
    const bool ok = jv < nv;
    const int64_t band = ok ? (v_idx ? v_idx[v0 + jv] : v0 + jv) : 0;
    const float2* src = psi_v + band * nr + (int64_t)i1 * plane;
#pragma unroll 4
    for (int e = threadIdx.x; e < plane; e += blockDim.x) {
      const int i2 = e / n, i3 = e - i2 * n;
      float2 v = make_float2(0.f, 0.f);
      if (ok) {
        // shift to the lowest kept frequencies: u_v * conj(e^{2 pi i (k3min i3 + k2min i2)/n})
        const float2 s = cmul(T3[(size_t)i3 * nk3p], T2[(size_t)i2 * nk2p]);
        v = cmul(src[e], make_float2(s.x, -s.y));
      }
      Uv[(j * n + i2) * ld + i3] = v;
    }
  }
  const int items1 = NP * n;
  const int items2 = NP * nk3;
  // asynchronous copies of the NCB conduction planes starting at jc0, one row per
  // warp: the whole plane is in flight at once
  auto load_conduction = [&](int jc0) {
#pragma unroll
    for (int cb = 0; cb < NCB; ++cb) {
      const int jc = jc0 + cb;
      const int64_t band = jc < jc_end ? (c_idx ? c_idx[c0 + jc] : c0 + jc) : -1;
      const float2* src = psi_c + (band < 0 ? 0 : band) * nr + (int64_t)i1 * plane;
      for (int i2 = warp; i2 < n; i2 += nwarp) {
        float2* dst = Uc + (cb * n + i2) * ld;
        const float2* sr = src + i2 * n;
#pragma unroll
        for (int i3 = lane; i3 < n; i3 += 32) {
          if (band < 0)
            dst[i3] = make_float2(0.f, 0.f);
          else
            cp_async8(dst + i3, sr + i3);
        }
      }
    }
  };
  if (jc_begin < jc_end) load_conduction(jc_begin);
  for (int jc0 = jc_begin; jc0 < jc_end; jc0 += NCB) {
    cp_async_wait_all();
    __syncthreads();
    // stage 1: one line (i2) of one (valence, conduction) pair per thread
    for (int it = threadIdx.x; it < items1; it += blockDim.x) {
      const int i2 = it % n, jj = it / n, j = jj % TV, cb = jj / TV;
      const float2* uv = Uv + (j * n + i2) * ld;
      const float2* uc = Uc + (cb * n + i2) * ld;
      float2 acc[NK];
      line_transform<P, Q, NK>([&](int i3) { return cconjmul(uv[i3], uc[i3]); }, acc);
      float2* xo = X + ((cb * TV + j) * n + i2) * ldx;
#pragma unroll
      for (int kk = 0; kk < NK; ++kk)
        if (kk < nk3) xo[kk] = acc[kk];
    }
    __syncthreads();
    // the conduction planes are free again: the next ones load while stage 2 runs
    if (jc0 + NCB < jc_end) load_conduction(jc0 + NCB);
    // stage 2: one kept k3 column of one pair per thread
    for (int it = threadIdx.x; it < items2; it += blockDim.x) {
      const int kk3 = it % nk3, jj = it / nk3, j = jj % TV, cb = jj / TV;
      const int jv = jv0 + j, jc = jc0 + cb;
      const float2* xi = X + ((cb * TV + j) * n) * ldx + kk3;
      float2 acc[NK];
      line_transform<P, Q, NK>([&](int i2) { return xi[i2 * ldx]; }, acc);
      if (jv < nv && jc < jc_end) {
        float2* dst = D + ((int64_t)(jv * nc + jc) * n + i1) * box + kk3;
#pragma unroll
        for (int kk = 0; kk < NK; ++kk)
          if (kk < nk2) dst[(int64_t)kk * nk3] = acc[kk];
      }
    }
    // no barrier here: the wait and barrier at the top of the next iteration order
    // these reads of X before the next stage 1 writes it
  }
}

template <int P, int Q, int NK, int TV, int NCB>
size_t fft_planes_smem(int nk3) {
  constexpr int n = P * Q, ld = n | 1;
  const size_t ldx = nk3 | 1;
  return ((size_t)TV * n * ld + (size_t)NCB * n * ld + (size_t)NCB * TV * n * ldx) * sizeof(float2);
}

template <int P, int Q, int NK, int TV, int NCB>
cudaError_t launch_fft_planes(const chi0_plan_s* p, const SphereQ& s, const void* psi_v, const int32_t* v_idx,
                              int v0, int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc, void* D,
                              cudaStream_t st) {
  const size_t sm = fft_planes_smem<P, Q, NK, TV, NCB>(s.nk3);
  auto kern = k_pair_planes_fft<P, Q, NK, TV, NCB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int vt = (nv + TV - 1) / TV;
  int cpc = 16 * NCB;
  while (cpc > NCB && (int64_t)p->n1 * vt * ((nc + cpc - 1) / cpc) < 4 * 152) cpc >>= 1;
  dim3 grid(p->n1, vt, (nc + cpc - 1) / cpc);
  kern<<<grid, 192, sm, st>>>((const float2*)psi_v, v_idx, v0, nv, (const float2*)psi_c, c_idx, c0, nc, cpc, s.nk2,
                              s.nk3, s.nk2p, s.nk3p, s.T2f, s.T3f, (float2*)D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Warp-cooperative length-96 transforms (n = 3Q, Q = 32) of the 96^3
// wavefunction passes: a warp transforms one line.  A line is split as i = a + 3b
// (a < 3, b < Q): lane b holds x(3b), x(3b+1), x(3b+2) (24 contiguous bytes,
// so the warp reads its row at once), the three Q-point transforms
// F_a(m) = sum_b x(a+3b) e^{2 pi i m b/Q} run across the lanes by radix-2
// decimation in frequency (one shuffle per value and stage; lane b ends with
// F_a(bitrev(b))), and lane b forms, for kk = bitrev(b) + Q t (t < 3),
//   y(kk) = F_0(kk mod Q) + e^{2 pi i kk/n} F_1(kk mod Q) + e^{4 pi i kk/n} F_2(kk mod Q).
// (On 48^3, Q = 16 with two lines per warp measured slower than the
// per-thread register FFTs above, so 48^3 keeps those.)  WL_NKMAX: the largest
// kept extent along i2 and i3 that the 96^3 pair kernel below takes.
constexpr int WL_NKMAX = 32;

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// per-lane constants of the group transform: stage twiddles e^{2 pi i (b mod h)/(2h)} for
// h = Q/2, ..., 1 and the combination factors e^{2 pi i kk/n}, e^{4 pi i kk/n} of both output sets
// NS output sets: lane b forms y(bitrev(b) + Q t) for t < NS.  Per stage of span h
// the lane keeps its sign (+1 for the lower lane of a pair, -1 for the upper one)
// and its twiddle (1 for the lower lane), so that a butterfly is
// x <- (x sign + partner) twiddle: two fused multiply-adds and a complex product.
template <int Q, int NS = 2> struct WLConsts {
  static constexpr int LOGQ = Q == 32 ? 5 : 4;
  float2 tw[LOGQ];
  float sg[LOGQ];
  float2 c1[NS], c2[NS];
  int kk;
};
template <int Q, int NS = 2>
__device__ __forceinline__ WLConsts<Q, NS> wl_consts(int b) {
  constexpr int n = 3 * Q;
  WLConsts<Q, NS> c;
#pragma unroll
  for (int s = 0; s < WLConsts<Q, NS>::LOGQ; ++s) {
    const int h = (Q / 2) >> s;
    const bool upper = (b & h) != 0;
    c.sg[s] = upper ? -1.f : 1.f;
    // the upper lane's twiddle: (b mod h)/(2h) of a turn
    c.tw[s] = upper ? root<n>((b % h) * (n / (2 * h))) : make_float2(1.f, 0.f);
  }
  c.kk = bitrev<Q>(b);
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int k = c.kk + Q * t;
    c.c1[t] = root<n>(k % n);
    c.c2[t] = root<n>((2 * k) % n);
  }
  return c;
}

// the Q-point transforms of the three sub-sequences across the group (in place, outputs in
// bit-reversed lane order), then y[t] = y(bitrev(b) + Q t) of the length-3Q line whose values
// x(a + 3b) lane b holds in x[a]
template <int Q, int NS>
__device__ __forceinline__ void wl_line(float2 (&x)[3], const WLConsts<Q, NS>& c, int b, float2 (&y)[NS]) {
  // lower lane of a pair: x + partner; upper lane: (partner - x) twiddle
#pragma unroll
  for (int s = 0; s < WLConsts<Q, NS>::LOGQ; ++s) {
    const int h = (Q / 2) >> s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 p = shfl_xor2(x[a], h);
      const float2 u = make_float2(fmaf(c.sg[s], x[a].x, p.x), fmaf(c.sg[s], x[a].y, p.y));
      x[a] = (h == 1) ? u : cmul(u, c.tw[s]);     // the last stage's twiddle is 1
    }
  }
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    y[t] = x[0];
    cfma(y[t], x[1], c.c1[t]);
    cfma(y[t], x[2], c.c2[t]);
  }
}

// ---------------------------------------------------------------------------
// (a, b, c) <- Y_k = sum_j x_j e^{2 pi i jk/3}
__device__ __forceinline__ void dft3p(float2& a, float2& b, float2& c) {
  constexpr float h = k_roots24.im[4];           // sin(pi/3)
  const float2 s = make_float2(b.x + c.x, b.y + c.y), d = make_float2(b.x - c.x, b.y - c.y);
  const float2 m = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
  a = make_float2(a.x + s.x, a.y + s.y);
  b = make_float2(fmaf(-h, d.y, m.x), fmaf(h, d.x, m.y));
  c = make_float2(fmaf(h, d.y, m.x), fmaf(-h, d.x, m.y));
}

// ---------------------------------------------------------------------------
// Stages 1+2 on the 96^3 grid with 8 lanes per line (four lines per warp).  A
// line is split as i = c + 2 b + 16 j (c < 2, b < 8, j < 6): lane b of a group
// of eight holds x(2 b + 16 j) and x(2 b + 16 j + 1) (one 16-byte load per j,
// so a group's load of a row is 128 contiguous bytes).  With the output
// k = kj + 6 kb + 48 kc (kj < 6, kb < 8, kc < 2) the exponent of e^{2 pi i/96}
// reduces to c kj + 6 c kb + 48 c kc + 2 b kj + 12 b kb + 16 j kj, so per lane:
// the 6-point transforms A_c(kj) = sum_j x(c + 2b + 16j) e^{2 pi i j kj/6}
// times e^{2 pi i 2 b kj/96}; the 8-point transforms over b across the group (3
// shuffle stages, against 4 for 16 lanes); then, lane b holding kb =
// bitrev3(b), C_1 times e^{2 pi i (kj + 6 kb)/96} and the 2-point transform
// over c: y(kj + 6 kb + 48 kc) = C_0 + (-1)^kc C_1.  A line moves 18 values
// per lane pair through shuffles (24 with 16 lanes, 30 with a warp per line)
// while its row loads still cover whole 128-byte lines.  128 registers, two
// CTAs per SM: bounding the registers for three made it spill and run 1.7x
// slower.
struct W8Consts {
  float2 t2b[6];     // e^{2 pi i 2 b kj/96}
  float2 tkb[6];     // e^{2 pi i (kj + 6 kb)/96}
  float2 tw4, tw2;   // stage twiddles of the upper lane (1 for the lower), spans 4 and 2
  float sg4, sg2, sg1;
  int kb;            // bitrev3(b)
};
__device__ __forceinline__ W8Consts w8_consts(int b) {
  W8Consts c;
  c.kb = bitrev<8>(b);
#pragma unroll
  for (int kj = 0; kj < 6; ++kj) {
    c.t2b[kj] = root<96>((2 * b * kj) % 96);
    c.tkb[kj] = root<96>((kj + 6 * c.kb) % 96);
  }
  c.sg4 = (b & 4) ? -1.f : 1.f;
  c.sg2 = (b & 2) ? -1.f : 1.f;
  c.sg1 = (b & 1) ? -1.f : 1.f;
  c.tw4 = (b & 4) ? root<96>(12 * (b % 4)) : make_float2(1.f, 0.f);
  c.tw2 = (b & 2) ? root<96>(24 * (b % 2)) : make_float2(1.f, 0.f);
  return c;
}

// 6-point transform with e^{+2 pi i/6}: even outputs from u_j = x_j + x_{j+3}, odd
// ones from v_j = (x_j - x_{j+3}) e^{2 pi i j/6}
__device__ __forceinline__ void dft6p(float2 (&x)[6]) {
  float2 u0 = make_float2(x[0].x + x[3].x, x[0].y + x[3].y), v0 = make_float2(x[0].x - x[3].x, x[0].y - x[3].y);
  float2 u1 = make_float2(x[1].x + x[4].x, x[1].y + x[4].y), v1 = make_float2(x[1].x - x[4].x, x[1].y - x[4].y);
  float2 u2 = make_float2(x[2].x + x[5].x, x[2].y + x[5].y), v2 = make_float2(x[2].x - x[5].x, x[2].y - x[5].y);
  v1 = cmul(v1, root<96>(16));
  v2 = cmul(v2, root<96>(32));
  dft3p(u0, u1, u2);
  dft3p(v0, v1, v2);
  x[0] = u0;
  x[1] = v0;
  x[2] = u1;
  x[3] = v1;
  x[4] = u2;
  x[5] = v2;
}

// x[c][j] = x(c + 2 b + 16 j) -> x[kc][kj] = y(kj + 6 bitrev3(b) + 48 kc)
__device__ __forceinline__ void w8_line(float2 (&x)[2][6], const W8Consts& w) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    dft6p(x[c]);
#pragma unroll
    for (int kj = 1; kj < 6; ++kj) x[c][kj] = cmul(x[c][kj], w.t2b[kj]);
  }
  // 8-point transforms across the group: lower lane x + partner, upper lane (partner - x) twiddle
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int kj = 0; kj < 6; ++kj) {
      float2 p = shfl_xor2(x[c][kj], 4);
      float2 u = make_float2(fmaf(w.sg4, x[c][kj].x, p.x), fmaf(w.sg4, x[c][kj].y, p.y));
      u = cmul(u, w.tw4);
      p = shfl_xor2(u, 2);
      u = make_float2(fmaf(w.sg2, u.x, p.x), fmaf(w.sg2, u.y, p.y));
      u = cmul(u, w.tw2);
      p = shfl_xor2(u, 1);
      x[c][kj] = make_float2(fmaf(w.sg1, u.x, p.x), fmaf(w.sg1, u.y, p.y));
    }
  // 2-point transforms over c
#pragma unroll
  for (int kj = 0; kj < 6; ++kj) {
    const float2 t = cmul(x[1][kj], w.tkb[kj]);
    const float2 a = x[0][kj];
    x[0][kj] = make_float2(a.x + t.x, a.y + t.y);
    x[1][kj] = make_float2(a.x - t.x, a.y - t.y);
  }
}

constexpr int W8_WARPS = 8;

// One CTA per (valence band, plane i1) and a run of conduction bands:
//   stage 1: line slot l = 4 w + (lane / 8) transforms rows i2 = l + 32 r of
//            conj(u_v) u_c along i3 into X[i2][k3];
//   stage 2: the kept columns k3 of X along i2 into Y[k2][k3];
//   Y is copied to D[pair][i1] (contiguous nk2 x nk3 values).
// No frequency shift is applied to the inputs: a line keeps the outputs y(k) for
// k in [kmin, kmin + nk) mod 96.
__global__ void __launch_bounds__(W8_WARPS * 32, 2)
k_pair_planes_w8(const float2* __restrict__ psi_v, const int32_t* __restrict__ v_idx, int v0, int nv,
                 const float2* __restrict__ psi_c, const int32_t* __restrict__ c_idx, int c0, int nc, int c_per_cta,
                 int k2min, int k3min, int nk2, int nk3, float2* __restrict__ D) {
  constexpr int n = 96;
  constexpr int64_t nr = (int64_t)n * n * n;
  constexpr int plane = n * n;
  constexpr int LINES = W8_WARPS * 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldx = nk3 | 1;
  float2* X = reinterpret_cast<float2*>(smem_raw);   // [n][ldx]
  float2* Y = X + n * ldx;                            // [nk2][nk3]
  const int jv = blockIdx.x;
  const int i1 = blockIdx.y;
  const int jc_begin = blockIdx.z * c_per_cta;
  const int jc_end = min(nc, jc_begin + c_per_cta);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = lane & 7, slot = warp * 4 + (lane >> 3);
  const int box = nk2 * nk3;
  if (jv >= nv || jc_begin >= jc_end) return;
  const W8Consts cst = w8_consts(b);
  // kept-range slot of y(kj + 6 kb + 48 kc) is (base + kj + 48 kc) mod 96
  const int base3 = ((6 * cst.kb - k3min) % n + n) % n, base2 = ((6 * cst.kb - k2min) % n + n) % n;
  const int64_t vband = v_idx ? v_idx[v0 + jv] : v0 + jv;
  const float2* vsrc = psi_v + vband * nr + (int64_t)i1 * plane;
  for (int jc = jc_begin; jc < jc_end; ++jc) {
    const int64_t band = c_idx ? c_idx[c0 + jc] : c0 + jc;
    const float2* csrc = psi_c + band * nr + (int64_t)i1 * plane;
    // stage 1: rows (96 = 3 x 32 lines, the same count for every slot)
    for (int i2 = slot; i2 < n; i2 += LINES) {
      const float4* uc = reinterpret_cast<const float4*>(csrc + i2 * n) + b;
      const float4* uv = reinterpret_cast<const float4*>(vsrc + i2 * n) + b;
      float2 x[2][6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float4 a = __ldg(uv + 8 * j), c = __ldg(uc + 8 * j);
        x[0][j] = cconjmul(make_float2(a.x, a.y), make_float2(c.x, c.y));
        x[1][j] = cconjmul(make_float2(a.z, a.w), make_float2(c.z, c.w));
      }
      w8_line(x, cst);
#pragma unroll
      for (int kc = 0; kc < 2; ++kc)
#pragma unroll
        for (int kj = 0; kj < 6; ++kj) {
          int s = base3 + kj + 48 * kc;
          s = s >= n ? s - n : s;
          if (s < nk3) X[i2 * ldx + s] = x[kc][kj];
        }
    }
    __syncthreads();
    // stage 2: kept columns, a warp-uniform loop (groups past nk3 transform zeros)
    for (int kb0 = warp * 4; kb0 < nk3; kb0 += LINES) {
      const int k3 = kb0 + (lane >> 3);
      const bool valid = k3 < nk3;
      const float2* col = X + 2 * b * ldx + (valid ? k3 : 0);
      float2 x[2][6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        x[0][j] = col[16 * j * ldx];
        x[1][j] = col[(16 * j + 1) * ldx];
      }
      w8_line(x, cst);
      if (valid) {
#pragma unroll
        for (int kc = 0; kc < 2; ++kc)
#pragma unroll
          for (int kj = 0; kj < 6; ++kj) {
            int s = base2 + kj + 48 * kc;
            s = s >= n ? s - n : s;
            if (s < nk2) Y[s * nk3 + k3] = x[kc][kj];
          }
      }
    }
    __syncthreads();
    float2* dst = D + ((int64_t)(jv * nc + jc) * n + i1) * box;
    for (int e = threadIdx.x; e < box; e += blockDim.x) dst[e] = Y[e];
  }
}

cudaError_t launch_planes_w8(const chi0_plan_s* p, const SphereQ& s, const void* psi_v, const int32_t* v_idx,
                             int v0, int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc, void* D,
                             cudaStream_t st) {
  constexpr int n = 96;
  const size_t sm = ((size_t)n * (s.nk3 | 1) + (size_t)s.nk2 * s.nk3) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_pair_planes_w8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int cpc = 16;
  while (cpc > 1 && (int64_t)p->n1 * nv * ((nc + cpc - 1) / cpc) < 8 * 152) cpc >>= 1;
  // valence bands fastest: the CTAs running at a time share one plane's conduction rows in L2
  dim3 grid(nv, p->n1, (nc + cpc - 1) / cpc);
  k_pair_planes_w8<<<grid, W8_WARPS * 32, sm, st>>>((const float2*)psi_v, v_idx, v0, nv, (const float2*)psi_c, c_idx,
                                                    c0, nc, cpc, s.k2min, s.k3min, s.nk2, s.nk3, (float2*)D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Wavefunctions on the 96^3 grid (FP32 plans) by three passes of the same
// warp transform, each over whole length-96 lines (all 96 outputs):
//   pass 1 (k_wfn96_cols): for every (g2, g3) column of the sphere, the line
//     along g1 (coefficients at g1 mod 96, zeros elsewhere) -> A[b][i1][col];
//   pass 2 (k_wfn96_planes, one CTA per plane i1 and band): the lines along g2
//     for every g3 (from A[b][i1] in shared memory) -> B[i2][g3], then the
//     lines along g3 for every i2 -> psi[b][i1][i2][:].
// psi_b(r) = sum_g c_b(g) e^{2 pi i g.r} as the direct kernels; the scratch
// A holds 96 x nw2 x nw3 values per band of a chunk.
// ---------------------------------------------------------------------------
constexpr int WF_WARPS = 8;

// the g in [gmin, gmin + 95] with g = i (mod 96); valid when g <= gmax
__device__ __forceinline__ int wf_g(int i, int gmin) { return gmin + (((i - gmin) % 96) + 96) % 96; }

__global__ void __launch_bounds__(WF_WARPS * 32)
k_wfn96_cols(const double2* __restrict__ coeff, int npw, int ncols, const int* __restrict__ col_start,
             const int* __restrict__ col_pw, const int* __restrict__ col_g1, int w1min, float2* __restrict__ A) {
  __shared__ float2 line[WF_WARPS][96];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * WF_WARPS + warp;
  if (c >= ncols) return;                             // whole warps only: no barrier below
  const int64_t b = blockIdx.y;
  float2* L = line[warp];
#pragma unroll
  for (int t = 0; t < 3; ++t) L[lane + 32 * t] = make_float2(0.f, 0.f);
  __syncwarp();
  const double2* cb = coeff + b * npw;
  for (int k = col_start[c] + lane; k < col_start[c + 1]; k += 32) {
    const int g1 = col_g1[k] + w1min;
    const double2 d = cb[col_pw[k]];
    L[((g1 % 96) + 96) % 96] = make_float2((float)d.x, (float)d.y);
  }
  __syncwarp();
  const WLConsts<32, 3> cst = wl_consts<32, 3>(lane);
  float2 x[3], y[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = L[3 * lane + a];
  wl_line<32, 3>(x, cst, lane, y);
  float2* out = A + b * 96 * (int64_t)ncols + c;
#pragma unroll
  for (int t = 0; t < 3; ++t) out[(int64_t)(cst.kk + 32 * t) * ncols] = y[t];
}

__global__ void __launch_bounds__(WF_WARPS * 32, 3)
k_wfn96_planes(const float2* __restrict__ A, int nw2, int nw3, int w2min, int w3min, float2* __restrict__ psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lda = nw3 | 1, ncols = nw2 * nw3;
  float2* As = reinterpret_cast<float2*>(smem_raw);  // [nw2][lda]
  float2* Bs = As + nw2 * lda;                       // [96][lda]
  const int i1 = blockIdx.x;
  const int64_t b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float2* Ap = A + (b * 96 + i1) * (int64_t)ncols;
  for (int e = threadIdx.x; e < ncols; e += blockDim.x) {
    const int r = e / nw3;
    As[r * lda + (e - r * nw3)] = Ap[e];
  }
  __syncthreads();
  const WLConsts<32, 3> cst = wl_consts<32, 3>(lane);
  int g2i[3], g3i[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g2i[a] = wf_g(3 * lane + a, w2min) - w2min;       // row of As at line position 3 lane + a, if < nw2
    g3i[a] = wf_g(3 * lane + a, w3min) - w3min;
  }
  // along g2 for every g3
  for (int j3 = warp; j3 < nw3; j3 += WF_WARPS) {
    float2 x[3], y[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = g2i[a] < nw2 ? As[g2i[a] * lda + j3] : make_float2(0.f, 0.f);
    wl_line<32, 3>(x, cst, lane, y);
#pragma unroll
    for (int t = 0; t < 3; ++t) Bs[(cst.kk + 32 * t) * lda + j3] = y[t];
  }
  __syncthreads();
  // along g3 for every i2
  float2* out = psi + (b * 96 + i1) * (int64_t)(96 * 96);
  for (int i2 = warp; i2 < 96; i2 += WF_WARPS) {
    float2 x[3], y[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = g3i[a] < nw3 ? Bs[i2 * lda + g3i[a]] : make_float2(0.f, 0.f);
    wl_line<32, 3>(x, cst, lane, y);
#pragma unroll
    for (int t = 0; t < 3; ++t) out[i2 * 96 + cst.kk + 32 * t] = y[t];
  }
}

// FP32 planes with register FFTs when the grid is cubic, n = P*Q is supported and
// the kept extents fit NKMAX; returns cudaErrorNotSupported otherwise.
cudaError_t try_fft_planes(const chi0_plan_s* p, const SphereQ& s, const void* psi_v, const int32_t* v_idx, int v0,
                           int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc, void* D,
                           cudaStream_t st) {
  const int nk = std::max(s.nk2, s.nk3);
  if (!(p->n1 == p->n2 && p->n2 == p->n3)) return cudaErrorNotSupported;
  if (p->n3 == 96 && nk <= WL_NKMAX)
    return launch_planes_w8(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st);
  if (nk > NKMAX) return cudaErrorNotSupported;
#define CHI0_FFT_CASE(P, Q, TV, NCB)                                                                    \
  if (nk <= 12) return launch_fft_planes<P, Q, 12, TV, NCB>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st); \
  if (nk <= 16) return launch_fft_planes<P, Q, 16, TV, NCB>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st); \
  if (nk <= 20) return launch_fft_planes<P, Q, 20, TV, NCB>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st); \
  return launch_fft_planes<P, Q, 28, TV, NCB>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st);
  switch (p->n3) {
    case 24: { CHI0_FFT_CASE(3, 8, 2, 2) }
    case 36: { CHI0_FFT_CASE(9, 4, 2, 2) }
    case 48: { CHI0_FFT_CASE(3, 16, 2, 2) }
    case 96: { CHI0_FFT_CASE(3, 32, 1, 1) }
    default: return cudaErrorNotSupported;
  }
#undef CHI0_FFT_CASE
}

// ---------------------------------------------------------------------------
// Stage 3 with register FFTs (FP32, cubic grids n = P*Q): one thread per
// (pair, column (k2, k3) of the sphere).  The thread reads the column's n
// values D_p(i1, k2, k3) (consecutive threads: neighbouring columns, so the
// loads of a warp are contiguous), shifts them by e^{2 pi i k1min i1/n},
// transforms along i1 keeping the first nk1 outputs and writes the column's
// sphere points to M.
// ---------------------------------------------------------------------------
template <int P, int Q, int NK>
__global__ void __launch_bounds__(kThreads)
k_pair_gather_fft(const float2* __restrict__ D, int nc, int64_t row0, int64_t ldv, int64_t box, int nG,
                  int ncol, int64_t n_items, const int* __restrict__ col_off, const int* __restrict__ col_start,
                  const int* __restrict__ ent_k1, const int* __restrict__ ent_j, const float2* __restrict__ T1,
                  int nk1, float scale, float2* __restrict__ M) {
  constexpr int n = P * Q;
  __shared__ float2 sh[n];           // e^{2 pi i k1min i1/n}
  for (int e = threadIdx.x; e < n; e += blockDim.x) sh[e] = T1[(size_t)e * nk1];
  __syncthreads();
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= n_items) return;
  const int pl = (int)(item / ncol), c = (int)(item - (int64_t)pl * ncol);
  const int jv = pl / nc, jc = pl - jv * nc;
  const float2* Dp = D + (int64_t)pl * n * box + col_off[c];
  float2 acc[NK];
  line_transform<P, Q, NK>([&](int i1) { return cmul(Dp[(int64_t)i1 * box], sh[i1]); }, acc);
  float2* out = M + (row0 + (int64_t)jv * ldv + jc) * nG;
  int t = col_start[c];
  const int t_end = col_start[c + 1];
  int k = t < t_end ? ent_k1[t] : NK;
  // entries of a column are sorted by k1; the loop over kk is unrolled so acc stays in registers
#pragma unroll
  for (int kk = 0; kk < NK; ++kk) {
    while (k == kk) {
      out[ent_j[t]] = make_float2(acc[kk].x * scale, acc[kk].y * scale);
      ++t;
      k = t < t_end ? ent_k1[t] : NK;
    }
  }
}

template <int P, int Q, int NK>
cudaError_t launch_gather_fft(const chi0_plan_s* p, const SphereQ& s, const void* D, int nv, int nc, int64_t row0,
                              int64_t ldv, void* M, cudaStream_t st) {
  const int64_t items = (int64_t)nv * nc * s.ncol;
  const int64_t blocks = (items + kThreads - 1) / kThreads;
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  k_pair_gather_fft<P, Q, NK><<<(unsigned)blocks, kThreads, 0, st>>>(
      (const float2*)D, nc, row0, ldv, (int64_t)s.nk2 * s.nk3, s.nG, s.ncol, items, s.col_off, s.col_start,
      s.ent_k1, s.ent_j, s.T1f, s.nk1, (float)(1.0 / (double)p->nr), (float2*)M);
  return cudaGetLastError();
}

// FP32 stage 3 with register FFTs when the grid is cubic, n = P*Q is supported
// and nk1 fits NKMAX; returns cudaErrorNotSupported otherwise.
cudaError_t try_gather_fft(const chi0_plan_s* p, const SphereQ& s, const void* D, int nv, int nc, int64_t row0,
                           int64_t ldv, void* M, cudaStream_t st) {
  if (!(p->n1 == p->n2 && p->n2 == p->n3) || s.nk1 > NKMAX || s.ncol <= 0) return cudaErrorNotSupported;
#define CHI0_GATHER_CASE(P, Q)                                                                         \
  if (s.nk1 <= 12) return launch_gather_fft<P, Q, 12>(p, s, D, nv, nc, row0, ldv, M, st);               \
  if (s.nk1 <= 16) return launch_gather_fft<P, Q, 16>(p, s, D, nv, nc, row0, ldv, M, st);               \
  if (s.nk1 <= 20) return launch_gather_fft<P, Q, 20>(p, s, D, nv, nc, row0, ldv, M, st);               \
  return launch_gather_fft<P, Q, 28>(p, s, D, nv, nc, row0, ldv, M, st);
  switch (p->n1) {
    case 24: { CHI0_GATHER_CASE(3, 8) }
    case 36: { CHI0_GATHER_CASE(9, 4) }
    case 48: { CHI0_GATHER_CASE(3, 16) }
    case 96: { CHI0_GATHER_CASE(3, 32) }
    default: return cudaErrorNotSupported;
  }
#undef CHI0_GATHER_CASE
}

// ---------------------------------------------------------------------------
// Stages 1+2 for planes too large for shared memory (FP64 on large grids):
// stage 1 runs over chunks of ROWS rows (i2) of the plane, reading the valence
// and conduction rows of each chunk; stage 2 follows once X holds every row.
// Shared memory: Uv[ROWS][ld3], Uc[ROWS][ld3], X[n2][nk3p].  One valence band
// per CTA, a run of conduction bands.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pair_planes_rows(const typename Cx<R>::T* __restrict__ psi_v, const int32_t* __restrict__ v_idx, int v0,
                   int nv, const typename Cx<R>::T* __restrict__ psi_c, const int32_t* __restrict__ c_idx, int c0,
                   int nc, int c_per_cta, int n1, int n2, int n3, int ld3, int rows, int nk2, int nk3, int nk2p,
                   int nk3p, const typename Cx<R>::T* __restrict__ T2, const typename Cx<R>::T* __restrict__ T3,
                   typename Cx<R>::T* __restrict__ D) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Uv = reinterpret_cast<C*>(smem_raw);
  C* Uc = Uv + (size_t)rows * ld3;
  C* X = Uc + (size_t)rows * ld3;
  const int i1 = blockIdx.x;
  const int jv = blockIdx.y;
  const int jc_begin = blockIdx.z * c_per_cta;
  const int jc_end = min(nc, jc_begin + c_per_cta);
  const int64_t nr = (int64_t)n1 * n2 * n3;
  const int plane = n2 * n3;
  const int64_t box = (int64_t)nk2 * nk3;
  const int64_t vband = v_idx ? v_idx[v0 + jv] : v0 + jv;
  const C* vsrc = psi_v + vband * nr + (int64_t)i1 * plane;
  for (int jc = jc_begin; jc < jc_end; ++jc) {
    const int64_t band = c_idx ? c_idx[c0 + jc] : c0 + jc;
    const C* csrc = psi_c + band * nr + (int64_t)i1 * plane;
    for (int r0 = 0; r0 < n2; r0 += rows) {
      const int nrow = min(rows, n2 - r0);
      __syncthreads();
      for (int e = threadIdx.x; e < nrow * n3; e += blockDim.x) {
        const int r = e / n3, i3 = e - r * n3;
        Uv[(size_t)r * ld3 + i3] = vsrc[(int64_t)(r0 + r) * n3 + i3];
        Uc[(size_t)r * ld3 + i3] = csrc[(int64_t)(r0 + r) * n3 + i3];
      }
      __syncthreads();
      // stage 1 for rows r0..r0+nrow
      const int items1 = nrow * (nk3p >> 2);
      for (int it = threadIdx.x; it < items1; it += blockDim.x) {
        const int r = it % nrow, kb = (it / nrow) << 2;
        C acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = cz(C());
        const C* uv = Uv + (size_t)r * ld3;
        const C* uc = Uc + (size_t)r * ld3;
        for (int i3 = 0; i3 < n3; ++i3) {
          const C rho = cconjmul(uv[i3], uc[i3]);
          const C* t = T3 + (size_t)i3 * nk3p + kb;
#pragma unroll
          for (int q = 0; q < 4; ++q) cfma(acc[q], rho, __ldg(t + q));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) X[(size_t)(r0 + r) * nk3p + kb + q] = acc[q];
      }
    }
    __syncthreads();
    // stage 2 (along i2)
    const int items2 = nk3 * (nk2p >> 2);
    for (int it = threadIdx.x; it < items2; it += blockDim.x) {
      const int k3 = it % nk3, kb = (it / nk3) << 2;
      C acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = cz(C());
      for (int i2 = 0; i2 < n2; ++i2) {
        const C x = X[(size_t)i2 * nk3p + k3];
        const C* t = T2 + (size_t)i2 * nk2p + kb;
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[q], x, __ldg(t + q));
      }
      C* dst = D + ((int64_t)(jv * nc + jc) * n1 + i1) * box + k3;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (kb + q < nk2) dst[(int64_t)(kb + q) * nk3] = acc[q];
    }
  }
}

template <typename R>
cudaError_t launch_planes_rows(const chi0_plan_s* p, const SphereQ& s, const void* psi_v, const int32_t* v_idx,
                               int v0, int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc, void* D,
                               cudaStream_t st) {
  using C = typename Cx<R>::T;
  const int ld3 = p->n3 | 1;
  const size_t xbytes = (size_t)p->n2 * s.nk3p * sizeof(C);
  const size_t cap = (size_t)200 * 1024;
  if (xbytes + 2 * (size_t)ld3 * sizeof(C) > cap) return cudaErrorInvalidConfiguration;
  int rows = (int)std::min<size_t>((size_t)p->n2, (cap - xbytes) / (2 * (size_t)ld3 * sizeof(C)));
  const size_t sm = 2 * (size_t)rows * ld3 * sizeof(C) + xbytes;
  auto kern = k_pair_planes_rows<R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int cpc = 16;
  while (cpc > 1 && (int64_t)p->n1 * nv * ((nc + cpc - 1) / cpc) < 4 * 152) cpc >>= 1;
  dim3 grid(p->n1, nv, (nc + cpc - 1) / cpc);
  const C* T2 = std::is_same<R, float>::value ? (const C*)s.T2f : (const C*)s.T2d;
  const C* T3 = std::is_same<R, float>::value ? (const C*)s.T3f : (const C*)s.T3d;
  kern<<<grid, kThreads, sm, st>>>((const C*)psi_v, v_idx, v0, nv, (const C*)psi_c, c_idx, c0, nc, cpc, p->n1, p->n2,
                                   p->n3, ld3, rows, s.nk2, s.nk3, s.nk2p, s.nk3p, T2, T3, (C*)D);
  return cudaGetLastError();
}

size_t planes_smem(int tv, int n2, int ld3, int nk3p, size_t cb) {
  return ((size_t)tv * n2 * ld3 + (size_t)n2 * ld3 + (size_t)tv * n2 * nk3p) * cb;
}

template <typename R, int TV>
cudaError_t launch_planes_tv(const chi0_plan_s* p, const SphereQ& s, const void* psi_v, const int32_t* v_idx,
                             int v0, int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc,
                             void* D, cudaStream_t st) {
  using C = typename Cx<R>::T;
  const int ld3 = p->n3 | 1;
  const size_t sm = planes_smem(TV, p->n2, ld3, s.nk3p, sizeof(C));
  auto kern = k_pair_planes<R, TV>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int vt = (nv + TV - 1) / TV;
  // enough CTAs to fill the machine several times over, but long c runs per CTA
  int cpc = 16;
  while (cpc > 1 && (int64_t)p->n1 * vt * ((nc + cpc - 1) / cpc) < 4 * 152) cpc >>= 1;
  dim3 grid(p->n1, vt, (nc + cpc - 1) / cpc);
  const C* T2 = std::is_same<R, float>::value ? (const C*)s.T2f : (const C*)s.T2d;
  const C* T3 = std::is_same<R, float>::value ? (const C*)s.T3f : (const C*)s.T3d;
  kern<<<grid, kThreads, sm, st>>>((const C*)psi_v, v_idx, v0, nv, (const C*)psi_c, c_idx, c0, nc, cpc,
                                   p->n1, p->n2, p->n3, ld3, s.nk2, s.nk3, s.nk2p, s.nk3p, T2, T3, (C*)D);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_planes_r(const chi0_plan_s* p, const SphereQ& s, const void* psi_v, const int32_t* v_idx,
                            int v0, int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc, void* D,
                            cudaStream_t st) {
  const int ld3 = p->n3 | 1;
  const size_t cb = sizeof(typename Cx<R>::T);
  // prefer two resident CTAs per SM; fall back to one
  for (size_t cap : {(size_t)110 * 1024, (size_t)220 * 1024}) {
    if (planes_smem(4, p->n2, ld3, s.nk3p, cb) <= cap)
      return launch_planes_tv<R, 4>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st);
    if (planes_smem(2, p->n2, ld3, s.nk3p, cb) <= cap)
      return launch_planes_tv<R, 2>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st);
    if (planes_smem(1, p->n2, ld3, s.nk3p, cb) <= cap)
      return launch_planes_tv<R, 1>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st);
  }
  // whole planes do not fit: stage 1 over chunks of rows
  return launch_planes_rows<R>(p, s, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, st);
}

}  // namespace

cudaError_t launch_wfn_to_grid(const chi0_plan_s* p, const double2* coeff, int nb, void* psi, cudaStream_t s) {
  // grid.y is limited to 65535 bands per launch
  constexpr int kMaxY = 65535;
  if (nb > kMaxY) {
    const size_t cbw = is_split(p) ? sizeof(float2) : sizeof(double2);
    for (int b0 = 0; b0 < nb; b0 += kMaxY) {
      const int n = std::min(kMaxY, nb - b0);
      cudaError_t e = launch_wfn_to_grid(p, coeff + (size_t)b0 * p->w.npw, n,
                                         (char*)psi + (size_t)b0 * p->nr * cbw, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const WfnSphere& w = p->w;
  dim3 grid(p->n1, nb);
  if (is_split(p) && p->wfn_ws && p->n1 == 96 && p->n2 == 96 && p->n3 == 96) {
    // three passes of warp transforms, bands in chunks that fit the plan's scratch
    const int ncols = w.nw2 * w.nw3;
    const int chunk = (int)std::max<int64_t>(1, p->wfn_ws_bytes / ((size_t)96 * ncols * sizeof(float2)));
    const size_t sm = ((size_t)w.nw2 * (w.nw3 | 1) + (size_t)96 * (w.nw3 | 1)) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_wfn96_planes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    for (int b0 = 0; b0 < nb; b0 += chunk) {
      const int nbc = std::min(chunk, nb - b0);
      dim3 g1((ncols + WF_WARPS - 1) / WF_WARPS, nbc);
      k_wfn96_cols<<<g1, WF_WARPS * 32, 0, s>>>(coeff + (size_t)b0 * w.npw, w.npw, ncols, w.col_start, w.col_pw,
                                                w.col_g1, w.w1min, (float2*)p->wfn_ws);
      dim3 g2(96, nbc);
      k_wfn96_planes<<<g2, WF_WARPS * 32, sm, s>>>((const float2*)p->wfn_ws, w.nw2, w.nw3, w.w2min, w.w3min,
                                                   (float2*)psi + (size_t)b0 * p->nr);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (is_split(p)) {
    const size_t smb = wfn_blk_smem(p);
    // 16-byte stores: psi must be 16-byte aligned (every band plane then is, n3 % 4 == 0)
    if (p->n2 % 4 == 0 && p->n3 % 4 == 0 && smb <= (size_t)110 * 1024 && (reinterpret_cast<uintptr_t>(psi) & 15) == 0) {
      cudaError_t e = cudaFuncSetAttribute(k_wfn_to_grid_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
      if (e != cudaSuccess) return e;
      dim3 gridb((p->n1 + WPL - 1) / WPL, nb);
      k_wfn_to_grid_blk<<<gridb, kThreads, smb, s>>>(coeff, w.npw, p->n1, p->n2, p->n3, w.nw1, w.nw2, w.nw3,
                                                     w.col_start, w.col_pw, w.col_g1, w.T1f, w.T2f, w.T3f,
                                                     (float2*)psi);
      return cudaGetLastError();
    }
    size_t sm = ((size_t)w.nw2 * w.nw3 + (size_t)p->n2 * w.nw3) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_wfn_to_grid<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_wfn_to_grid<float><<<grid, kThreads, sm, s>>>(coeff, w.npw, p->n1, p->n2, p->n3, w.nw1, w.nw2, w.nw3,
                                                    w.col_start, w.col_pw, w.col_g1, w.T1f, w.T2f, w.T3f,
                                                    (float2*)psi);
  } else {
    size_t sm = ((size_t)w.nw2 * w.nw3 + (size_t)p->n2 * w.nw3) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_wfn_to_grid<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_wfn_to_grid<double><<<grid, kThreads, sm, s>>>(coeff, w.npw, p->n1, p->n2, p->n3, w.nw1, w.nw2, w.nw3,
                                                     w.col_start, w.col_pw, w.col_g1, w.T1d, w.T2d, w.T3d,
                                                     (double2*)psi);
  }
  return cudaGetLastError();
}

cudaError_t launch_pair_planes(const chi0_plan_s* p, int iq, const void* psi_v, const int32_t* v_idx, int v0,
                               int nv, const void* psi_c, const int32_t* c_idx, int c0, int nc, void* D,
                               cudaStream_t s) {
  const SphereQ& sq = p->q[iq];
  if (is_split(p)) {
    cudaError_t e = try_fft_planes(p, sq, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, s);
    if (e != cudaErrorNotSupported) return e;
    return launch_planes_r<float>(p, sq, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, s);
  }
  return launch_planes_r<double>(p, sq, psi_v, v_idx, v0, nv, psi_c, c_idx, c0, nc, D, s);
}

cudaError_t launch_pair_gather(const chi0_plan_s* p, int iq, const void* D, int nv, int nc, int64_t row0,
                               int64_t ldv, void* M, cudaStream_t s) {
  const SphereQ& sq = p->q[iq];
  const int64_t box = (int64_t)sq.nk2 * sq.nk3;
  const int npl = nv * nc;
  if (npl == 0) return cudaSuccess;
  if (is_split(p)) {
    cudaError_t e = try_gather_fft(p, sq, D, nv, nc, row0, ldv, M, s);
    if (e != cudaErrorNotSupported) return e;
    size_t sm = (size_t)p->n1 * sq.nk1 * sizeof(float2);
    k_pair_gather<float><<<npl, kThreads, sm, s>>>((const float2*)D, nc, row0, ldv, p->n1, box, sq.nG, sq.nk1,
                                                   sq.ent_box, sq.ent_k1, sq.ent_j, sq.T1f,
                                                   (float)(1.0 / (double)p->nr), (float2*)M);
  } else {
    size_t sm = (size_t)p->n1 * sq.nk1 * sizeof(double2);
    k_pair_gather<double><<<npl, kThreads, sm, s>>>((const double2*)D, nc, row0, ldv, p->n1, box, sq.nG,
                                                    sq.nk1, sq.ent_box, sq.ent_k1, sq.ent_j, sq.T1d,
                                                    1.0 / (double)p->nr, (double2*)M);
  }
  return cudaGetLastError();
}

}  // namespace chi0
