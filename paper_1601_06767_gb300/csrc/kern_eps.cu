// RPA dielectric matrix from chi0 and its inverse (section II: eps = 1 - v chi0,
// W = eps^-1 v; Table III: eps_inf = 1 / [eps^-1]_00).
//
// eps[w] = I - diag(v) chi0[w]  or the symmetrised  I - diag(v^1/2) chi0[w] diag(v^1/2).
//
// Inverse: blocked Gauss-Jordan elimination with partial pivoting, in place, on
// all n_freq matrices at once (grid dimension z / x = frequency).  For each
// panel of NB columns C1 = [k0, k0 + kb):
//   1. pivot rows among rows >= k0 by tournament pivoting (k_tp_select: GEPP
//      on blocks of candidate rows in shared memory, winners merged level by
//      level); k_tp_final moves the winners to R1 = [k0, k0 + kb) (recorded as
//      a swap sequence), copies the panel columns of every row to Z and forms
//      T = A11^-1 by Gauss-Jordan with partial pivoting on the pivot block;
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
// 1. panel: pivot rows by tournament (communication-avoiding) pivoting, then
//    the swaps, the Z copy and T = A11^-1
// ---------------------------------------------------------------------------
// rows of one selection block: 128 (FP32) or 64 (FP64) candidate rows in shared memory
template <typename R> struct SelRows { static constexpr int V = sizeof(R) == 4 ? 128 : 64; };

// Gaussian elimination with partial pivoting on up to ROWS candidate rows of
// the panel (their current values); the first kb pivot rows are the block's
// winners.  Leaf level (cand_in == NULL): block c holds rows k0 + c*ROWS ...;
// merge levels: block c holds entries c*ROWS ... of the previous level's list
// (NB slots per set, -1 = empty).  Writes NB slots per block to cand_out.
template <typename R>
__global__ void __launch_bounds__(SelRows<R>::V)
k_tp_select(const typename Cx<R>::T* __restrict__ A, int N, int k0, int kb, const int* __restrict__ cand_in,
            int n_in, int* __restrict__ cand_out, int ld) {
  using C = typename Cx<R>::T;
  constexpr int ROWS = SelRows<R>::V;
  const int w = blockIdx.y, c = blockIdx.x, r = threadIdx.x;
  const C* a = A + (size_t)w * N * N;
  __shared__ C S[ROWS][NB + 1];
  __shared__ int idx[ROWS];
  __shared__ R red_v[ROWS / 32];
  __shared__ int red_i[ROWS / 32];
  __shared__ int s_n, s_p, wcnt[ROWS / 32];
  int g = -1;
  if (cand_in == nullptr) {
    const int row = k0 + c * ROWS + r;
    g = row < N ? row : -1;
  } else {
    const int e = c * ROWS + r;
    g = e < n_in ? cand_in[(size_t)w * ld + e] : -1;
  }
  // compact the valid rows to the front, keeping their order (deterministic ties)
  const unsigned bal = __ballot_sync(0xffffffffu, g >= 0);
  if ((r & 31) == 0) wcnt[r >> 5] = __popc(bal);
  __syncthreads();
  if (r == 0) {
    int acc = 0;
    for (int q = 0; q < ROWS / 32; ++q) {
      const int n = wcnt[q];
      wcnt[q] = acc;
      acc += n;
    }
    s_n = acc;
  }
  __syncthreads();
  if (g >= 0) idx[wcnt[r >> 5] + __popc(bal & ((1u << (r & 31)) - 1u))] = g;
  __syncthreads();
  const int nr = s_n;
  if (r < nr) {
    const C* src = a + (size_t)idx[r] * N + k0;
    for (int t = 0; t < kb; ++t) S[r][t] = src[t];
  }
  __syncthreads();
  const int steps = min(kb, nr);
  for (int j = 0; j < steps; ++j) {
    R best = (r >= j && r < nr) ? cabs1(S[r][j]) : (R)-1;
    int bi = (r >= j && r < nr) ? r : ROWS;
    for (int o = 16; o; o >>= 1) {
      const R ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((r & 31) == 0) { red_v[r >> 5] = best; red_i[r >> 5] = bi; }
    __syncthreads();
    if (r == 0) {
      for (int q = 1; q < ROWS / 32; ++q)
        if (red_v[q] > best || (red_v[q] == best && red_i[q] < bi)) { best = red_v[q]; bi = red_i[q]; }
      s_p = (bi < nr) ? bi : j;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      if (r < kb) {
        const C u = S[j][r];
        S[j][r] = S[p][r];
        S[p][r] = u;
      }
      if (r == 0) {
        const int u = idx[j];
        idx[j] = idx[p];
        idx[p] = u;
      }
    }
    __syncthreads();
    if (r > j && r < nr) {
      const C piv = S[j][j];
      if (piv.x != (R)0 || piv.y != (R)0) {
        const C l = cmul(S[r][j], crecip(piv));
        for (int t = j + 1; t < kb; ++t) S[r][t] = csub(S[r][t], cmul(l, S[j][t]));
      }
    }
    __syncthreads();
  }
  if (r < NB) cand_out[(size_t)w * ld + (size_t)c * NB + r] = (r < steps) ? idx[r] : -1;
}

// Move the winners to rows k0..k0+kb-1 (recorded as a swap sequence in piv),
// copy the panel columns of every row to Z, invert the pivot block by
// Gauss-Jordan with partial pivoting in shared memory: T = A11^-1 (also
// written over the pivot block).
template <typename R>
__global__ void __launch_bounds__(1024)
k_tp_final(typename Cx<R>::T* __restrict__ A, int N, int k0, int kb, const int* __restrict__ win, int ld,
           typename Cx<R>::T* __restrict__ Z, typename Cx<R>::T* __restrict__ Tb, int* __restrict__ piv,
           int* __restrict__ status) {
  using C = typename Cx<R>::T;
  const int w = blockIdx.x, tid = threadIdx.x;
  C* a = A + (size_t)w * N * N;
  C* z = Z + (size_t)w * N * NB;
  int* pv = piv + (size_t)w * N;
  __shared__ int sp[NB];
  __shared__ C B[NB][2 * NB + 1];
  __shared__ int s_p;
  if (tid == 0) {
    // swap sequence: step t exchanges row k0+t with the current row of winner t
    int orig[2 * NB], cur[2 * NB], n = 0;
    for (int t = 0; t < kb; ++t) {
      const int x = win[(size_t)w * ld + t];
      int px = x;
      for (int q = 0; q < n; ++q)
        if (orig[q] == x) px = cur[q];
      const int y = k0 + t;
      int oy = y;
      for (int q = 0; q < n; ++q)
        if (cur[q] == y) oy = orig[q];
      if (x < 0) px = y;     // fewer candidates than columns (cannot happen for kb <= N - k0)
      sp[t] = px;
      pv[y] = px;
      if (px != y) {
        // the row now at y (original oy) moves to px, winner x moves to y
        bool fo = false, fx = false;
        for (int q = 0; q < n; ++q) {
          if (orig[q] == oy) { cur[q] = px; fo = true; }
          else if (orig[q] == x) { cur[q] = y; fx = true; }
        }
        if (!fo) { orig[n] = oy; cur[n] = px; ++n; }
        if (!fx) { orig[n] = x; cur[n] = y; ++n; }
      }
    }
  }
  __syncthreads();
  for (int t = 0; t < kb; ++t) {
    const int y = k0 + t, p = sp[t];
    if (p != y && tid < kb) {
      const C u = a[(size_t)y * N + k0 + tid];
      a[(size_t)y * N + k0 + tid] = a[(size_t)p * N + k0 + tid];
      a[(size_t)p * N + k0 + tid] = u;
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)N * kb; e += blockDim.x) {
    const int i = (int)(e / kb), t = (int)(e - (int64_t)i * kb);
    z[(size_t)i * NB + t] = a[(size_t)i * N + k0 + t];
  }
  // [A11 | I] -> [I | A11^-1]
  for (int e = tid; e < NB * 2 * NB; e += blockDim.x) {
    const int i = e / (2 * NB), c = e - i * 2 * NB;
    C v = cz(C{});
    if (i < kb && c < kb) v = a[(size_t)(k0 + i) * N + k0 + c];
    else if (i < kb && c >= NB && c - NB == i) v.x = (R)1;
    B[i][c] = v;
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid < 32) {
      R best = (tid >= j && tid < kb) ? cabs1(B[tid][j]) : (R)-1;
      int bi = (tid >= j && tid < kb) ? tid : NB;
      for (int o = 16; o; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        if (!(best > (R)0) || bi >= kb) {
          atomicOr(status, SINGULAR_BIT);
          bi = j;
        }
        s_p = bi;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != j && tid < 2 * NB) {
      const C u = B[j][tid];
      B[j][tid] = B[p][tid];
      B[p][tid] = u;
    }
    __syncthreads();
    const C inv = crecip(B[j][j]);
    __syncthreads();
    if (tid < 2 * NB) B[j][tid] = cmul(B[j][tid], inv);
    __syncthreads();
    // eliminate column j from every other row: thread (i, c)
    for (int e = tid; e < NB * 2 * NB; e += blockDim.x) {
      const int i = e / (2 * NB), c = e - i * 2 * NB;
      if (i != j && i < kb && c != j) B[i][c] = csub(B[i][c], cmul(B[i][j], B[j][c]));
    }
    __syncthreads();
    if (tid < NB && tid != j) B[tid][j] = cz(C{});
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, c = e - i * kb;
    const C t = B[i][NB + c];
    Tb[(size_t)w * NB * NB + i * NB + c] = t;
    a[(size_t)(k0 + i) * N + k0 + c] = t;
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

// candidate-list slots per matrix for an N-row panel (ping-pong pair)
template <typename R> int64_t tp_ld(int N) { return (int64_t)((N + SelRows<R>::V - 1) / SelRows<R>::V) * NB; }

template <typename R>
cudaError_t gj_invert(chi0_plan_s* p, typename Cx<R>::T* A, int N, int nf, void* Z, void* Tb, int* piv,
                      int* cand, cudaStream_t s) {
  using C = typename Cx<R>::T;
  constexpr int ROWS = SelRows<R>::V;
  const int ld = (int)tp_ld<R>(N);
  int* cbuf[2] = {cand, cand + (size_t)nf * ld};
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int kb = min(NB, N - k0);
    {
      // tournament: leaf blocks of ROWS rows, then merges of ROWS / NB sets until one is left
      int nblk = (N - k0 + ROWS - 1) / ROWS, levels = 1, cur = 0;
      for (int b = nblk; b > 1; b = (b * NB + ROWS - 1) / ROWS) ++levels;
      ProfScope ps(p, CHI0_K_INV_PANEL, s, levels + 2);
      k_tp_select<R><<<dim3(nblk, nf), ROWS, 0, s>>>(A, N, k0, kb, nullptr, 0, cbuf[0], ld);
      while (nblk > 1) {
        const int n_in = nblk * NB;
        nblk = (n_in + ROWS - 1) / ROWS;
        k_tp_select<R><<<dim3(nblk, nf), ROWS, 0, s>>>(A, N, k0, kb, cbuf[cur], n_in, cbuf[cur ^ 1], ld);
        cur ^= 1;
      }
      k_tp_final<R><<<nf, 1024, 0, s>>>(A, N, k0, kb, cbuf[cur], ld, (C*)Z, (C*)Tb, piv, p->d_status);
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

// Workspace (bytes): complex64 copy of the matrices (split plans), Z [nf][N][NB], T [nf][NB][NB],
// piv [nf][N], two candidate lists [nf][tp_ld].
size_t eps_inverse_ws_bytes(const chi0_plan_s* p, int nG) {
  const size_t nf = (size_t)p->n_freq, c = is_split(p) ? sizeof(float2) : sizeof(double2);
  const size_t copy = is_split(p) ? nf * nG * nG * sizeof(float2) : 0;
  const size_t ld = (size_t)(is_split(p) ? tp_ld<float>(nG) : tp_ld<double>(nG));
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  return al(copy) + al(nf * nG * NB * c) + al(nf * NB * NB * c) + al(nf * nG * sizeof(int)) +
         al(2 * nf * ld * sizeof(int));
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
    b += al(nf * nG * sizeof(int));
    int* cand = reinterpret_cast<int*>(b);
    const int64_t n = (int64_t)nf * nG * nG;
    {
      ProfScope ps(p, CHI0_K_EPS, s, 1);
      k_to_c64<<<4 * 152, 256, 0, s>>>(eps, n, a32);
    }
    cudaError_t e = gj_invert<float>(p, a32, nG, (int)nf, Z, Tb, piv, cand, s);
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
  b += al(nf * nG * sizeof(int));
  int* cand = reinterpret_cast<int*>(b);
  return gj_invert<double>(p, eps, nG, (int)nf, Z, Tb, piv, cand, s);
}

}  // namespace chi0
