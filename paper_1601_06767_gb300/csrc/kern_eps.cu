// RPA dielectric matrix from chi0 and its inverse (section II: eps = 1 - v chi0,
// W = eps^-1 v; Table III: eps_inf = 1 / [eps^-1]_00).
//
// eps[w] = I - diag(v) chi0[w]  or the symmetrised  I - diag(v^1/2) chi0[w] diag(v^1/2).
//
// Inverse: blocked Gauss-Jordan elimination with partial pivoting, in place, on
// all n_freq matrices at once (grid dimension z / x = frequency).  For each
// panel of NB columns C1 = [k0, k0 + kb):
//   1. k_gj_panel: copy the panel columns of every row to Z, LU-factor rows
//      >= k0 of the panel with partial pivoting (row swaps inside the panel
//      and in Z), then T = A11^-1 = U11^-1 L11^-1 of the pivot block;
//   2. k_gj_rows: apply the row swaps to the other columns and replace the
//      pivot rows R1 = [k0, k0 + kb) there by T A10;
//   3. k_gj_update: every other row i: A[i][j] = A[i][j] - Z[i] . R[:, j] for
//      j outside C1 and -Z[i] . T[:, j] inside C1 (R = the new pivot rows),
//      the block sweep  A00 -= A01 T A10,  A01 = -A01 T,  A10 = T A10,  A11 = T.
// After the last panel the in-place result is (P A)^-1; k_gj_colperm applies
// the column swaps in reverse order to give A^-1.
#include <cuda_runtime.h>

#include "cplx.cuh"
#include "internal.h"

namespace chi0 {
namespace {

constexpr int NB = 32;          // panel width
constexpr int PANEL_THREADS = 1024;
constexpr int SINGULAR_BIT = 0x100;

template <typename C> __device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename C> __device__ __forceinline__ C crecip(C a) {
  const auto d = a.x * a.x + a.y * a.y;
  C r;
  r.x = a.x / d;
  r.y = -a.y / d;
  return r;
}
template <typename C> __device__ __forceinline__ auto cabs1(C a) -> decltype(a.x) { return fabs(a.x) + fabs(a.y); }

__global__ void k_epsilon(const double2* __restrict__ chi, const double* __restrict__ v, int symmetric, int nG,
                          int64_t total, double2* __restrict__ eps) {
  const int64_t n2 = (int64_t)nG * nG;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % n2;
    const int i = (int)(r / nG), j = (int)(r - (int64_t)i * nG);
    const double s = symmetric ? sqrt(v[i]) * sqrt(v[j]) : v[i];
    const double2 c = chi[e];
    eps[e] = make_double2((i == j ? 1.0 : 0.0) - s * c.x, -s * c.y);
  }
}

__global__ void k_to_c64(const double2* __restrict__ a, int64_t n, float2* __restrict__ b) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = make_float2((float)a[e].x, (float)a[e].y);
}
__global__ void k_from_c64(const float2* __restrict__ b, int64_t n, double2* __restrict__ a) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    a[e] = make_double2((double)b[e].x, (double)b[e].y);
}

// ---------------------------------------------------------------------------
// 1. panel: Z copy, LU with partial pivoting of rows >= k0, T = A11^-1
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(PANEL_THREADS)
k_gj_panel(typename Cx<R>::T* __restrict__ A, int N, int k0, int kb, typename Cx<R>::T* __restrict__ Z,
           typename Cx<R>::T* __restrict__ Tb, int* __restrict__ piv, int* __restrict__ status) {
  using C = typename Cx<R>::T;
  const int w = blockIdx.x;
  C* a = A + (size_t)w * N * N;
  C* z = Z + (size_t)w * N * NB;
  C* tb = Tb + (size_t)w * NB * NB;
  int* pv = piv + (size_t)w * N;
  __shared__ C urow[NB];
  __shared__ C lu[NB][NB + 1];
  __shared__ R red_v[PANEL_THREADS / 32];
  __shared__ int red_i[PANEL_THREADS / 32];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (int64_t e = tid; e < (int64_t)N * kb; e += blockDim.x) {
    const int i = (int)(e / kb), t = (int)(e - (int64_t)i * kb);
    z[(size_t)i * NB + t] = a[(size_t)i * N + k0 + t];
  }
  __syncthreads();

  for (int j = 0; j < kb; ++j) {
    const int col = k0 + j, r0 = k0 + j;
    // pivot: largest |re| + |im| in column col over rows >= r0 (ties: lowest row)
    R best = (R)-1;
    int bi = N;
    for (int i = r0 + tid; i < N; i += blockDim.x) {
      const R m = cabs1(a[(size_t)i * N + col]);
      if (m > best) { best = m; bi = i; }
    }
    for (int o = 16; o; o >>= 1) {
      const R ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x >> 5;
      best = lane < nw ? red_v[lane] : (R)-1;
      bi = lane < nw ? red_i[lane] : N;
      for (int o = 16; o; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (!(best > (R)0) || bi >= N) {
          atomicOr(status, SINGULAR_BIT);
          bi = r0;
        }
        s_piv = bi;
        pv[r0] = bi;
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != r0 && tid < kb) {
      C t0 = a[(size_t)r0 * N + k0 + tid];
      a[(size_t)r0 * N + k0 + tid] = a[(size_t)p * N + k0 + tid];
      a[(size_t)p * N + k0 + tid] = t0;
      C t1 = z[(size_t)r0 * NB + tid];
      z[(size_t)r0 * NB + tid] = z[(size_t)p * NB + tid];
      z[(size_t)p * NB + tid] = t1;
    }
    __syncthreads();
    if (tid < kb) urow[tid] = a[(size_t)r0 * N + k0 + tid];
    __syncthreads();
    const C inv = crecip(urow[j]);
    for (int i = r0 + 1 + tid; i < N; i += blockDim.x) {
      C* row = a + (size_t)i * N + k0;
      const C l = cmul(row[j], inv);
      row[j] = l;
      for (int c = j + 1; c < kb; ++c) row[c] = csub(row[c], cmul(l, urow[c]));
    }
    __syncthreads();
  }

  // T = U11^-1 L11^-1 of the kb x kb pivot block (thread t: column t)
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e - i * kb;
    lu[i][c] = a[(size_t)(k0 + i) * N + k0 + c];
  }
  __syncthreads();
  if (tid < kb) {
    const int t = tid;
    C x[NB];
    // x = L^-1 e_t (L unit lower triangular): x_i = 0 (i < t), 1 (i = t), -sum_{t<=q<i} L_iq x_q
    for (int i = 0; i < kb; ++i) {
      C s = cz(C{});
      if (i == t) s.x = (R)1;
      for (int q = t; q < i; ++q) s = csub(s, cmul(lu[i][q], x[q]));
      x[i] = s;
    }
    // x = U^-1 x (back substitution)
    for (int i = kb - 1; i >= 0; --i) {
      C s = x[i];
      for (int q = i + 1; q < kb; ++q) s = csub(s, cmul(lu[i][q], x[q]));
      x[i] = cmul(s, crecip(lu[i][i]));
    }
    for (int i = 0; i < kb; ++i) tb[i * NB + t] = x[i];
  }
  __syncthreads();
  // the pivot block becomes T
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e - i * kb;
    a[(size_t)(k0 + i) * N + k0 + c] = tb[i * NB + c];
  }
}

// ---------------------------------------------------------------------------
// 2. row swaps outside the panel, pivot rows := T A10
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128)
k_gj_rows(typename Cx<R>::T* __restrict__ A, int N, int k0, int kb, const typename Cx<R>::T* __restrict__ Tb,
          const int* __restrict__ piv) {
  using C = typename Cx<R>::T;
  const int w = blockIdx.y;
  C* a = A + (size_t)w * N * N;
  const int* pv = piv + (size_t)w * N;
  __shared__ C ts[NB][NB];
  // entries outside the kb x kb block are never written by the panel kernel: use zeros
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e - r * NB;
    ts[r][c] = (r < kb && c < kb) ? Tb[(size_t)w * NB * NB + e] : cz(C{});
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N || (j >= k0 && j < k0 + kb)) return;
  for (int t = 0; t < kb; ++t) {
    const int p = pv[k0 + t];
    if (p != k0 + t) {
      const C u = a[(size_t)(k0 + t) * N + j];
      a[(size_t)(k0 + t) * N + j] = a[(size_t)p * N + j];
      a[(size_t)p * N + j] = u;
    }
  }
  C x[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) x[t] = t < kb ? a[(size_t)(k0 + t) * N + j] : cz(C{});
#pragma unroll 4
  for (int i = 0; i < kb; ++i) {
    C s = cz(C{});
#pragma unroll
    for (int t = 0; t < NB; ++t) cfma(s, ts[i][t], x[t]);
    a[(size_t)(k0 + i) * N + j] = s;
  }
}

// ---------------------------------------------------------------------------
// 3. trailing update of all rows outside R1 (64 x 64 output tiles, K = kb)
// ---------------------------------------------------------------------------
// output tile: 64 x 64 (FP32) or 32 x 32 (FP64, static shared memory limit); 256 threads
template <typename R> struct UpdTile { static constexpr int T = sizeof(R) == 4 ? 64 : 32; };

template <typename R>
__global__ void __launch_bounds__(256)
k_gj_update(typename Cx<R>::T* __restrict__ A, int N, int k0, int kb, const typename Cx<R>::T* __restrict__ Z) {
  using C = typename Cx<R>::T;
  constexpr int TILE = UpdTile<R>::T, RT = TILE / 16;
  const int w = blockIdx.z;
  C* a = A + (size_t)w * N * N;
  const C* z = Z + (size_t)w * N * NB;
  __shared__ C zs[NB][TILE + 1];     // zs[t][row]
  __shared__ C rs[NB][TILE + 1];     // rs[t][col]
  const int i0 = blockIdx.y * TILE, j0 = blockIdx.x * TILE;
  for (int e = threadIdx.x; e < TILE * NB; e += blockDim.x) {
    const int r = e / NB, t = e - r * NB;
    const int i = i0 + r;
    zs[t][r] = (i < N && t < kb) ? z[(size_t)i * NB + t] : cz(C{});
  }
  for (int e = threadIdx.x; e < NB * TILE; e += blockDim.x) {
    const int t = e / TILE, c = e - t * TILE;
    const int j = j0 + c;
    rs[t][c] = (j < N && t < kb) ? a[(size_t)(k0 + t) * N + j] : cz(C{});
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  C acc[RT][RT];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) acc[r][c] = cz(C{});
  for (int t = 0; t < kb; ++t) {
    C zr[RT], rc[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) zr[r] = zs[t][ty + 16 * r];
#pragma unroll
    for (int c = 0; c < RT; ++c) rc[c] = rs[t][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int c = 0; c < RT; ++c) cfma(acc[r][c], zr[r], rc[c]);
  }
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= N || (i >= k0 && i < k0 + kb)) continue;
#pragma unroll
    for (int c = 0; c < RT; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= N) continue;
      C* o = a + (size_t)i * N + j;
      const C base = (j >= k0 && j < k0 + kb) ? cz(C{}) : *o;
      *o = csub(base, acc[r][c]);
    }
  }
}

// ---------------------------------------------------------------------------
// 4. column swaps in reverse order: (P A)^-1 P = A^-1
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_gj_colperm(typename Cx<R>::T* __restrict__ A, int N, const int* __restrict__ piv) {
  using C = typename Cx<R>::T;
  const int w = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  C* row = A + (size_t)w * N * N + (size_t)i * N;
  const int* pv = piv + (size_t)w * N;
  for (int k = N - 1; k >= 0; --k) {
    const int p = pv[k];
    if (p != k) {
      const C u = row[k];
      row[k] = row[p];
      row[p] = u;
    }
  }
}

template <typename R>
cudaError_t gj_invert(chi0_plan_s* p, typename Cx<R>::T* A, int N, int nf, void* Z, void* Tb, int* piv,
                      cudaStream_t s) {
  using C = typename Cx<R>::T;
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int kb = min(NB, N - k0);
    {
      ProfScope ps(p, CHI0_K_INV_PANEL, s, 2);
      k_gj_panel<R><<<nf, PANEL_THREADS, 0, s>>>(A, N, k0, kb, (C*)Z, (C*)Tb, piv, p->d_status);
      k_gj_rows<R><<<dim3((N + 127) / 128, nf), 128, 0, s>>>(A, N, k0, kb, (const C*)Tb, piv);
    }
    {
      ProfScope ps(p, CHI0_K_INV_UPDATE, s, 1);
      const int t = (N + UpdTile<R>::T - 1) / UpdTile<R>::T;
      k_gj_update<R><<<dim3(t, t, nf), 256, 0, s>>>(A, N, k0, kb, (const C*)Z);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ProfScope ps(p, CHI0_K_INV_PANEL, s, 1);
  k_gj_colperm<R><<<dim3((N + 127) / 128, nf), 128, 0, s>>>(A, N, piv);
  return cudaGetLastError();
}

}  // namespace

int eps_panel_width() { return NB; }

cudaError_t launch_epsilon(chi0_plan_s* p, int nG, const double2* chi, const double* v, int symmetric,
                           double2* eps, cudaStream_t s) {
  ProfScope ps(p, CHI0_K_EPS, s, 1);
  const int64_t total = (int64_t)p->n_freq * nG * nG;
  k_epsilon<<<4 * 152, 256, 0, s>>>(chi, v, symmetric, nG, total, eps);
  return cudaGetLastError();
}

// Workspace (bytes): complex64 copy of the matrices (split plans), Z [nf][N][NB], T [nf][NB][NB], piv [nf][N].
size_t eps_inverse_ws_bytes(const chi0_plan_s* p, int nG) {
  const size_t nf = (size_t)p->n_freq, c = is_split(p) ? sizeof(float2) : sizeof(double2);
  const size_t copy = is_split(p) ? nf * nG * nG * sizeof(float2) : 0;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  return al(copy) + al(nf * nG * NB * c) + al(nf * NB * NB * c) + al(nf * nG * sizeof(int));
}

cudaError_t launch_epsilon_inverse(chi0_plan_s* p, int nG, double2* eps, void* ws, cudaStream_t s) {
  const size_t nf = (size_t)p->n_freq;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  unsigned char* b = reinterpret_cast<unsigned char*>(ws);
  if (is_split(p)) {
    float2* a32 = reinterpret_cast<float2*>(b);
    b += al(nf * nG * nG * sizeof(float2));
    void* Z = b;
    b += al(nf * nG * NB * sizeof(float2));
    void* Tb = b;
    b += al(nf * NB * NB * sizeof(float2));
    int* piv = reinterpret_cast<int*>(b);
    const int64_t n = (int64_t)nf * nG * nG;
    {
      ProfScope ps(p, CHI0_K_EPS, s, 1);
      k_to_c64<<<4 * 152, 256, 0, s>>>(eps, n, a32);
    }
    cudaError_t e = gj_invert<float>(p, a32, nG, (int)nf, Z, Tb, piv, s);
    if (e != cudaSuccess) return e;
    ProfScope ps(p, CHI0_K_EPS, s, 1);
    k_from_c64<<<4 * 152, 256, 0, s>>>(a32, n, eps);
    return cudaGetLastError();
  }
  void* Z = b;
  b += al(nf * nG * NB * sizeof(double2));
  void* Tb = b;
  b += al(nf * NB * NB * sizeof(double2));
  int* piv = reinterpret_cast<int*>(b);
  return gj_invert<double>(p, eps, nG, (int)nf, Z, Tb, piv, s);
}

}  // namespace chi0
