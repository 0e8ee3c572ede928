// Split-precision tensor-core contraction of Eq. 1 on sm_103a:
//   chi0[w][G][H] += sum_p f_p(w) M_p(G) conj(M_p(H))
//
// Real form:   Re chi = sum_p Wr Mr + Wi Mi,   Im chi = sum_p Wi Mr - Wr Mi,
// with W = f_p(w) M_p (FP32).  Every real operand x is split into NT 16-bit
// terms x = t0 + t1 (+ t2), t0 = rn(x), t1 = rn(x - t0), t2 = rn(x - t0 - t1);
// a real product keeps the term products t_i t_j with i + j < NT (plus t1 t1
// for the four-product two-term variant).  Operands are first scaled by exact
// powers of two so that the largest magnitude of the block sits near 2^14
// (keeps FP16 terms normal; harmless for BF16) and the scale is undone exactly
// when the sums are widened to FP64.
//
// pack:     M block [K][nG] (FP32 complex) and f -> K-major 16-bit planes
//           B = {Mr_t..., Mi_t...}[nGp][Kp], A_w = {Wr_t..., Wi_t...}[nGp][Kp].
// contract: one CTA per (128 x 128 output tile, frequency).  Warp 0 issues TMA
//           loads into a 3-stage ring, warp 1 issues tcgen05.mma into two
//           double-buffered TMEM accumulator pairs (Re, Im) (warps 0-3 on few
//           registers, given to the epilogue by setmaxnreg), warps 4..11 drain
//           finished accumulation chains into FP32 registers and finally add
//           the tile into chi0 by FP64 reductions (the additions run in L2).
//
// Hermitian mode: with a real ratio t per frequency and block of pairs,
//   f_p = Re f_p (1 + i t) + i g_p,   g_p = Im f_p - t Re f_p,
//   chi0 = (1 + i t) H1 + i H2,  H1 = sum Re(f) M M^H,  H2 = sum g M M^H,
// H1 and H2 both Hermitian.  An item contracts W1 = Re(f) M and W2 = g M (two
// parts, each with its own power-of-two scale) for one tile on or above the
// diagonal, adds the elements with G < G' and writes their conjugate transpose
// into the lower triangle (in both modes the diagonal G = G' is the pack's
// sum, not the tensor cores').  t is the midrange of
// Im f_p / Re f_p over the block (0 where that does not shrink the weights),
// so max|g| <= rho max|Re f| with rho = half the range of the ratio: about
// delta / |E_v - E_c| spread over the block's energies, 1e-4 for a block of
// neighbouring conduction bands.  H2 takes one product (t0 t0, FP16 operands in
// both precisions: BF16 plans keep an FP16 term 0 of M for it) when rho <=
// 2^-11, three products (two terms) when rho <= 2^-6, else the full count; the
// first two with long chains.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <string.h>

#include <algorithm>
#include <string>

#include "internal.h"
#include "tc_ptx.cuh"

namespace chi0 {
namespace {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int TILE_BYTES = BM * BK * 2;           // 8 KB per plane tile
constexpr int RING_BYTES = 6 * 32768;              // operand ring in shared memory
constexpr int EPI_WARPS = 8;
constexpr int EPI_WARP0 = 4;                       // warpgroup 0: TMA producer, MMA issuer, two idle warps
constexpr int THREADS = EPI_WARP0 * 32 + EPI_WARPS * 32;
// Register split between warpgroups (setmaxnreg): the launch gives every thread
// REG_LAUNCH registers (the most 384 threads can have); warpgroup 0 gives back
// down to REG_LOW and the two epilogue warpgroups take REG_HIGH, so that the
// epilogue's FP32 sums (128 per thread) and a TMEM load buffer fit without
// spilling.  The increase waits until the pool holds the registers, so the
// shares must add up to no more than the launch's total; the host checks that
// the compiled kernel uses exactly REG_LAUNCH before launching it.
constexpr int REG_LAUNCH = 168, REG_LOW = 72, REG_HIGH = 216;
static_assert(EPI_WARP0 * 32 * REG_LOW + EPI_WARPS * 32 * REG_HIGH <= THREADS * REG_LAUNCH,
              "register split exceeds the launch's registers");
static_assert(THREADS * REG_LAUNCH <= 65536 && REG_LAUNCH * THREADS / 4 <= 16384 * 4, "launch registers");
constexpr int TMEM_COLS = 512;                     // 2 buffers x (Re, Im) x 128 columns
constexpr uint64_t WAIT_BUDGET_NS = 2000000000ull; // 2 s per wait
constexpr int BAR_BYTES = 256;                     // barriers and the tensor-memory base
constexpr int XBUF_FLOATS = 32 * 8;                // per epilogue warp: the transpose of red_block
constexpr size_t SMEM_BYTES = (size_t)RING_BYTES + 1024 /*align*/ + BAR_BYTES + EPI_WARPS * XBUF_FLOATS * 4;
constexpr int MAX_STAGES = 3;

template <int NT> struct Ring {
  static constexpr int PLANES = 2 * NT;                       // per operand: Re terms, Im terms
  static constexpr int STAGE_BYTES = 2 * PLANES * TILE_BYTES; // A and B
  static constexpr int STAGES = RING_BYTES / STAGE_BYTES;     // 3 for NT = 2, 2 for NT = 3
};

int round_up_i(int x, int m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// pack: tile of 64 pairs x 32 sphere points, transposed through shared memory
// ---------------------------------------------------------------------------
template <bool BF16>
__device__ __forceinline__ float rn16(float x, uint16_t* bits) {
  if constexpr (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    *bits = __bfloat16_as_ushort(h);
    return __bfloat162float(h);
  } else {
    const __half h = __float2half_rn(x);
    *bits = __half_as_ushort(h);
    return __half2float(h);
  }
}

// split a and b (two consecutive K elements) into NT terms; word t packs term t of (a, b)
template <bool BF16, int NT>
__device__ __forceinline__ void splitn(float a, float b, uint32_t (&w)[NT]) {
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    uint16_t ua, ub;
    const float ta = rn16<BF16>(a, &ua), tb = rn16<BF16>(b, &ub);
    a -= ta;   // exact: the remainder of a rounding to 8 or 11 bits fits FP32
    b -= tb;
    w[t] = (uint32_t)ua | ((uint32_t)ub << 16);
  }
}

// order-preserving map of a float onto an unsigned int (for atomicMin / atomicMax)
__device__ __forceinline__ unsigned int ord_of(float x) {
  const unsigned int u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of_ord(unsigned int o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// largest |component| of the M block -> amax[0]; largest |Re f(w)| -> amax[1 + 2w],
// largest |Im f(w)| -> amax[2 + 2w]; Hermitian mode: the smallest and largest
// Im f / Re f over the block (order-mapped) -> tr[2w], tr[2w + 1]
__global__ void k_absmax(const float2* __restrict__ M, int64_t n, const double2* __restrict__ f, int64_t K,
                         int n_freq, unsigned int* __restrict__ amax, unsigned int* __restrict__ tr) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = M[i];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
  for (int iw = 0; iw < n_freq; ++iw) {
    float gr = 0.f, gi = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
      const double2 v = f[(int64_t)iw * K + i];
      gr = fmaxf(gr, (float)fabs(v.x));
      gi = fmaxf(gi, (float)fabs(v.y));
    }
    for (int o = 16; o; o >>= 1) {
      gr = fmaxf(gr, __shfl_xor_sync(0xffffffffu, gr, o));
      gi = fmaxf(gi, __shfl_xor_sync(0xffffffffu, gi, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(amax + 1 + 2 * iw, __float_as_uint(gr));
      atomicMax(amax + 2 + 2 * iw, __float_as_uint(gi));
    }
    if (tr) {
      float tlo = INFINITY, thi = -INFINITY;
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = f[(int64_t)iw * K + i];
        const float t = (float)(v.y / v.x);   // +-inf or NaN where Re f vanishes: the range is then unusable
        tlo = fminf(tlo, t);
        thi = fmaxf(thi, t);
        if (t != t) thi = INFINITY;
      }
      for (int o = 16; o; o >>= 1) {
        tlo = fminf(tlo, __shfl_xor_sync(0xffffffffu, tlo, o));
        thi = fmaxf(thi, __shfl_xor_sync(0xffffffffu, thi, o));
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMin(tr + 2 * iw, ord_of(tlo));
        atomicMax(tr + 2 * iw + 1, ord_of(thi));
      }
    }
  }
}

// tr[2w] = the largest order value (the running minimum's start), tr[2w + 1] stays 0
__global__ void k_ratio_init(unsigned int* __restrict__ tr, int n_freq) {
  for (int iw = threadIdx.x; iw < n_freq; iw += blockDim.x) tr[2 * iw] = 0xffffffffu;
}

// power of two 2^(14 - e) with x < 2^e (1 when x is zero or not finite)
__device__ __forceinline__ float pow2_scale(float x) {
  if (!(x > 0.f) || !isfinite(x)) return 1.f;
  int e;
  frexpf(x, &e);
  return ldexpf(1.f, 14 - e);
}

// scale[0] = sM; scale[1 + w] = sW(w); inv[w] = 1 / (sM sW(w)).  Hermitian mode:
// scale[1 + w], inv[w] belong to W1 = Re(f) M, scale[1 + n_freq + w],
// inv[n_freq + w] to W2 = g M with g = Im f - t Re f, tbar[w] is t and h2np[w]
// the product count of the W2 part (+16: long chains).
__global__ void k_scales(const unsigned int* __restrict__ amax, const unsigned int* __restrict__ tr, int n_freq,
                         int herm, int n_products, int bf16, float* __restrict__ scale, double* __restrict__ inv,
                         int* __restrict__ h2np, double* __restrict__ tbar) {
  const float mM = __uint_as_float(amax[0]);
  const float sM = pow2_scale(mM);
  if (threadIdx.x == 0) scale[0] = sM;
  for (int iw = threadIdx.x; iw < n_freq; iw += blockDim.x) {
    const float fr = __uint_as_float(amax[1 + 2 * iw]), fi = __uint_as_float(amax[2 + 2 * iw]);
    if (herm) {
      // shift by the midrange t of Im f / Re f when that shrinks the W2 weights:
      // |g_p| = |Re f_p| |t_p - t| <= max|Re f| (t_max - t_min) / 2
      const float tlo = float_of_ord(tr[2 * iw]), thi = float_of_ord(tr[2 * iw + 1]);
      const float half = 0.5f * (thi - tlo);
      const bool shift = isfinite(tlo) && isfinite(thi) && isfinite(half) && half * fr < fi;
      // t is rounded to FP32: the merge forms (1 + i t) H1 in FP32 with this same t
      const float t = shift ? (float)(0.5 * ((double)tlo + (double)thi)) : 0.f;
      // the bound on |g| (margins for the FP32 ratio range and the rounding of t), else max|Im f|
      const float gmax = shift ? half * fr * 1.0001f + fr * 1e-7f * (1.f + fabsf(t)) : fi;
      const float rho = fr > 0.f ? gmax / fr : 0.f;
      // |components of W1| <= max|Re f| max|M|, of W2 <= gmax max|M|
      const float s1 = pow2_scale(fr * mM), s2 = pow2_scale(gmax * mM);
      scale[1 + iw] = s1;
      scale[1 + n_freq + iw] = s2;
      inv[iw] = 1.0 / ((double)sM * (double)s1);
      inv[n_freq + iw] = 1.0 / ((double)sM * (double)s2);
      tbar[iw] = (double)t;
      // a small W2 part needs fewer products (errors scale with rho) and takes long chains (flag 16)
      // one product (FP16 operands in both precisions) where rho <= 2^-11
      (void)bf16;
      h2np[iw] = rho <= ldexpf(1.f, -11) ? 1 + 16 : (rho <= ldexpf(1.f, -6) ? 3 + 16 : n_products);
    } else {
      // |Re W|, |Im W| <= 2 max|f| max|M|
      const float sW = pow2_scale(2.f * fmaxf(fr, fi) * mM);
      scale[1 + iw] = sW;
      inv[iw] = 1.0 / ((double)sM * (double)sW);
    }
  }
}

// tile of 64 pairs x 32 sphere points, transposed through shared memory.
// Also the diagonal of the block's sum, diag[w][G] += sum_p f_p(w) |M_p(G)|^2 over
// the tile's pairs (FP32 over 64 pairs, added to FP64): all its terms have the
// phase of f, so the tensor cores' round-toward-zero would add up along the
// whole block there, while the CUDA cores round to nearest.
template <bool BF16, int NT>
__global__ void __launch_bounds__(256)
k_pack(const float2* __restrict__ M, int nG, int64_t K, int nGp, int Kp, const double2* __restrict__ f,
       int n_freq, int herm, const float* __restrict__ scale, const int* __restrict__ h2np,
       const double* __restrict__ tbar, uint32_t* __restrict__ Bp, uint32_t* __restrict__ Ap,
       double2* __restrict__ diag) {
  extern __shared__ __align__(16) unsigned char smem_pack[];
  float2* tile = reinterpret_cast<float2*>(smem_pack);          // [64][33]
  float2* fs = tile + 64 * 33;                                 // [n_freq][64]
  float2* fo = fs + 64 * n_freq;                               // [n_freq][64] f itself (FP32)
  const int G0 = blockIdx.x * 32;
  const int64_t p0 = (int64_t)blockIdx.y * 64;
  const float sM = scale[0];
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    const int pp = e >> 5, g = e & 31;
    const int64_t p = p0 + pp;
    float2 v = make_float2(0.f, 0.f);
    if (p < K && G0 + g < nG) v = M[p * nG + G0 + g];
    tile[pp * 33 + g] = v;
  }
  for (int e = threadIdx.x; e < n_freq * 64; e += blockDim.x) {
    const int iw = e >> 6, pp = e & 63;
    const int64_t p = p0 + pp;
    float2 v = make_float2(0.f, 0.f), v0 = v;
    if (p < K) {
      const double2 d = f[(int64_t)iw * K + p];
      const float sW = scale[1 + iw], sW2 = herm ? scale[1 + n_freq + iw] : sW;
      // Hermitian mode: the W2 weight is g = Im f - t Re f (in FP64, the t of the merge)
      const double im = herm ? d.y - tbar[iw] * d.x : d.y;
      v = make_float2((float)d.x * sW, (float)im * sW2);
      v0 = make_float2((float)d.x, (float)d.y);
    }
    fs[e] = v;
    fo[e] = v0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (G0 + lane < nG) {
    for (int iw = warp; iw < n_freq; iw += 8) {
      float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int pp = 0; pp < 64; ++pp) {
        const float2 m = tile[pp * 33 + lane];
        const float a = fmaf(m.x, m.x, m.y * m.y);
        const float2 fw = fo[iw * 64 + pp];
        sr[pp & 3] = fmaf(fw.x, a, sr[pp & 3]);
        si[pp & 3] = fmaf(fw.y, a, si[pp & 3]);
      }
      double2* d = diag + (size_t)iw * nGp + G0 + lane;
      atomicAdd(&d->x, (double)((sr[0] + sr[1]) + (sr[2] + sr[3])));
      atomicAdd(&d->y, (double)((si[0] + si[1]) + (si[2] + si[3])));
    }
  }
  const size_t plane = (size_t)nGp * (Kp / 2);                 // uint32 words per plane
  const int64_t kw = p0 / 2 + lane;                            // word index along K
  for (int g = warp; g < 32; g += 8) {
    const int G = G0 + g;
    const float2 m0 = tile[(2 * lane) * 33 + g], m1 = tile[(2 * lane + 1) * 33 + g];
    const size_t row = (size_t)G * (Kp / 2) + kw;
    uint32_t w[NT];
    splitn<BF16, NT>(m0.x * sM, m1.x * sM, w);
#pragma unroll
    for (int t = 0; t < NT; ++t) Bp[t * plane + row] = w[t];
    splitn<BF16, NT>(m0.y * sM, m1.y * sM, w);
#pragma unroll
    for (int t = 0; t < NT; ++t) Bp[(NT + t) * plane + row] = w[t];
    if (BF16 && herm) {
      // FP16 term 0 of M for one-product W2 parts: planes 2 NT (Re) and 2 NT + 1 (Im)
      uint32_t w1[1];
      splitn<false, 1>(m0.x * sM, m1.x * sM, w1);
      Bp[(2 * NT) * plane + row] = w1[0];
      splitn<false, 1>(m0.y * sM, m1.y * sM, w1);
      Bp[(2 * NT + 1) * plane + row] = w1[0];
    }
    for (int iw = 0; iw < n_freq; ++iw) {
      const float2 f0 = fs[iw * 64 + 2 * lane], f1 = fs[iw * 64 + 2 * lane + 1];
      uint32_t* a = Ap + (size_t)iw * 2 * NT * plane + row;
      if (herm) {
        // W1 = Re(f) M into the frequency's planes, W2 = Im(f) M into the second half
        splitn<BF16, NT>(f0.x * m0.x, f1.x * m1.x, w);
#pragma unroll
        for (int t = 0; t < NT; ++t) a[t * plane] = w[t];
        splitn<BF16, NT>(f0.x * m0.y, f1.x * m1.y, w);
#pragma unroll
        for (int t = 0; t < NT; ++t) a[(NT + t) * plane] = w[t];
        uint32_t* a2 = a + (size_t)n_freq * 2 * NT * plane;
        const int np2 = h2np[iw] & 15;
        const int nt2 = np2 == 1 ? 1 : ((NT == 3 && np2 != 6) ? 2 : NT);   // terms the W2 part reads
        if (np2 == 1) {
          // one product: an FP16 term (also in BF16 plans, 11 bits; the scaling keeps it in range)
          uint32_t w1[1];
          splitn<false, 1>(f0.y * m0.x, f1.y * m1.x, w1);
          a2[0] = w1[0];
          splitn<false, 1>(f0.y * m0.y, f1.y * m1.y, w1);
          a2[(size_t)NT * plane] = w1[0];
        } else {
          splitn<BF16, NT>(f0.y * m0.x, f1.y * m1.x, w);
#pragma unroll
          for (int t = 0; t < NT; ++t)
            if (t < nt2) a2[t * plane] = w[t];
          splitn<BF16, NT>(f0.y * m0.y, f1.y * m1.y, w);
#pragma unroll
          for (int t = 0; t < NT; ++t)
            if (t < nt2) a2[(NT + t) * plane] = w[t];
        }
      } else {
        const float wr0 = f0.x * m0.x - f0.y * m0.y, wi0 = f0.x * m0.y + f0.y * m0.x;
        const float wr1 = f1.x * m1.x - f1.y * m1.y, wi1 = f1.x * m1.y + f1.y * m1.x;
        splitn<BF16, NT>(wr0, wr1, w);
#pragma unroll
        for (int t = 0; t < NT; ++t) a[t * plane] = w[t];
        splitn<BF16, NT>(wi0, wi1, w);
#pragma unroll
        for (int t = 0; t < NT; ++t) a[(NT + t) * plane] = w[t];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// contraction
// ---------------------------------------------------------------------------
struct Barriers {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t done;
  uint32_t tmem_base;
};
static_assert(sizeof(Barriers) <= BAR_BYTES, "barriers overlap the transpose buffers");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory above the per-block limit");

// Issue the MMAs of one stage (BK pairs) into the (Re, Im) accumulator pair.
// The tensor cores round the FP32 accumulator toward zero after every MMA, so
// each MMA loses about one ulp of the running sum.  Chains are therefore kept
// to one stage and ordered smallest-first: every term product t_i t_j with
// i + j > 0 goes in while the accumulator is still small, and the t0 t0
// products (the only large ones) come last.
template <bool BF16, int NT, bool PAIR, int NPROD>
__device__ __forceinline__ void issue_stage_np(const unsigned char* st, uint32_t d_re, uint32_t d_im, bool first) {
  constexpr int P = 2 * NT;
  // in a CTA pair each CTA holds 128 rows of A and 64 rows of B; the MMA spans 256 rows
  constexpr int B_BYTES = PAIR ? TILE_BYTES / 2 : TILE_BYTES;
  const uint32_t id_pos = tc::idesc_f16(BF16, false, PAIR ? 2 * BM : BM, BN);
  const uint32_t id_neg = tc::idesc_f16(BF16, true, PAIR ? 2 * BM : BM, BN);
  // one descriptor for the stage; tiles and K steps are constant offsets of its address field
  const uint64_t d0 = tc::sdesc_kmajor_sw64(st);
  constexpr uint64_t kTile = TILE_BYTES >> 4, kBTile = B_BYTES >> 4, kB0 = (uint64_t)(P * TILE_BYTES) >> 4;
  uint32_t acc_re = first ? 0u : 1u, acc_im = acc_re;
#pragma unroll
  for (int order = 2 * NT - 2; order >= 0; --order) {
#pragma unroll
    for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
      for (int i = 0; i < NT; ++i) {
        const int j = order - i;
        if (j < 0 || j >= NT) continue;
        // 1: t0t0; 3: t0t0, t0t1, t1t0; 4: adds t1t1; 6: all t_i t_j with i + j <= 2
        const bool keep = NPROD == 1 ? (i + j == 0)
                                     : (i + j < 2) || (i + j == 2 && (NPROD == 6 || (NPROD == 4 && i == 1)));
        if (!keep) continue;
        // planes: Re terms 0..NT-1, Im terms NT..2NT-1; K step ks is +32 bytes
        const uint64_t ar = d0 + (uint64_t)i * kTile + (uint64_t)(ks * 2);
        const uint64_t ai = d0 + (uint64_t)(NT + i) * kTile + (uint64_t)(ks * 2);
        const uint64_t br = d0 + kB0 + (uint64_t)j * kBTile + (uint64_t)(ks * 2);
        const uint64_t bi = d0 + kB0 + (uint64_t)(NT + j) * kBTile + (uint64_t)(ks * 2);
        if constexpr (PAIR) {
          tc::mma_f16_pair(d_re, ar, br, id_pos, acc_re);
          acc_re = 1u;
          tc::mma_f16_pair(d_re, ai, bi, id_pos, 1u);
          tc::mma_f16_pair(d_im, ai, br, id_pos, acc_im);
          acc_im = 1u;
          tc::mma_f16_pair(d_im, ar, bi, id_neg, 1u);
        } else {
          // Re += Wr Mr + Wi Mi
          tc::mma_f16(d_re, ar, br, id_pos, acc_re);
          acc_re = 1u;
          tc::mma_f16(d_re, ai, bi, id_pos, 1u);
          // Im += Wi Mr - Wr Mi
          tc::mma_f16(d_im, ai, br, id_pos, acc_im);
          acc_im = 1u;
          tc::mma_f16(d_im, ar, bi, id_neg, 1u);
        }
      }
    }
  }
}

// One-product stage holding ns <= NT k-slices of term 0 (slice t in the slots of
// term t): t0 t0 for each slice, into the (Re, Im) accumulator pair.
template <bool BF16, int NT, bool PAIR>
__device__ __forceinline__ void issue_stage_1p(const unsigned char* st, uint32_t d_re, uint32_t d_im, bool first,
                                               int ns) {
  constexpr int B_BYTES = PAIR ? TILE_BYTES / 2 : TILE_BYTES;
  const uint32_t id_pos = tc::idesc_f16(BF16, false, PAIR ? 2 * BM : BM, BN);
  const uint32_t id_neg = tc::idesc_f16(BF16, true, PAIR ? 2 * BM : BM, BN);
  const uint64_t d0 = tc::sdesc_kmajor_sw64(st);
  constexpr uint64_t kTile = TILE_BYTES >> 4, kBTile = B_BYTES >> 4, kB0 = (uint64_t)(2 * NT * TILE_BYTES) >> 4;
  uint32_t acc_re = first ? 0u : 1u, acc_im = acc_re;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (t >= ns) break;
#pragma unroll
    for (int ks = 0; ks < BK / 16; ++ks) {
      const uint64_t ar = d0 + (uint64_t)t * kTile + (uint64_t)(ks * 2);
      const uint64_t ai = d0 + (uint64_t)(NT + t) * kTile + (uint64_t)(ks * 2);
      const uint64_t br = d0 + kB0 + (uint64_t)t * kBTile + (uint64_t)(ks * 2);
      const uint64_t bi = d0 + kB0 + (uint64_t)(NT + t) * kBTile + (uint64_t)(ks * 2);
      if constexpr (PAIR) {
        tc::mma_f16_pair(d_re, ar, br, id_pos, acc_re);
        acc_re = 1u;
        tc::mma_f16_pair(d_re, ai, bi, id_pos, 1u);
        tc::mma_f16_pair(d_im, ai, br, id_pos, acc_im);
        acc_im = 1u;
        tc::mma_f16_pair(d_im, ar, bi, id_neg, 1u);
      } else {
        tc::mma_f16(d_re, ar, br, id_pos, acc_re);
        acc_re = 1u;
        tc::mma_f16(d_re, ai, bi, id_pos, 1u);
        tc::mma_f16(d_im, ai, br, id_pos, acc_im);
        acc_im = 1u;
        tc::mma_f16(d_im, ar, bi, id_neg, 1u);
      }
    }
  }
}

// the product count as a compile-time constant: no per-MMA test in the issue loop
template <bool BF16, int NT, bool PAIR = false>
__device__ __forceinline__ void issue_stage(const unsigned char* st, uint32_t d_re, uint32_t d_im, bool first,
                                            int n_products) {
  if (n_products == 6) issue_stage_np<BF16, NT, PAIR, 6>(st, d_re, d_im, first);
  else if (n_products == 4) issue_stage_np<BF16, NT, PAIR, 4>(st, d_re, d_im, first);
  else if (n_products == 1) issue_stage_np<BF16, NT, PAIR, 1>(st, d_re, d_im, first);
  else issue_stage_np<BF16, NT, PAIR, 3>(st, d_re, d_im, first);
}

// One persistent launch over a list of work items (q-point, frequency, 128x128
// output tile), q-points with different sphere sizes in one batch.  Every
// item contracts the same number of pairs (nK stages), so items are assigned
// round-robin; the stage and chain counters run on across items, so the TMA
// ring and the TMEM double buffers never drain between items.
constexpr int MAXQ = 16;

struct TcBatch {
  CUtensorMap tmA[MAXQ];
  CUtensorMap tmB[MAXQ];
  double2* chi[MAXQ];
  const double* inv[MAXQ];   // [n_parts * n_freq] inverse operand scales
  const int* h2np[MAXQ];     // Hermitian mode: [n_freq] product count of the W2 part (+16 if small)
  const double* tbar[MAXQ];  // Hermitian mode: [n_freq] ratio t of chi0 = (1 + i t) H1 + i H2
  const double2* diag[MAXQ]; // [n_freq][tiles_n * BN] diagonal of chi0's block sum, from the pack
  int nG[MAXQ];
  int tiles_m[MAXQ];         // tiles along G (rows of chi0)
  int tiles_n[MAXQ];         // tiles along G' (columns)
  int64_t tpf[MAXQ];         // tiles per frequency
  int64_t item0[MAXQ + 1];   // first item of each q-point
  int n_q, n_freq, nK, chain_k, n_products, group;
  int n_parts;               // 1, or 2 in Hermitian mode (W1 then W2)
  int rr;                    // tile height / tile width (1, or 2 for CTA-pair tiles)
  int64_t total_items;
};

// products of part `part` of an item, its stages and its chain length in stages.
// A one-product part reads only term 0, so its stage holds NT consecutive
// k-slices of term 0 in the slots of the NT terms (NT times fewer stages, the
// same bytes per MMA).  The W2 part of Hermitian mode with one or three
// products is below 2^-6 of chi0, so its round-toward-zero bias allows chains
// eight times longer.
__device__ __forceinline__ int part_products(const TcBatch& P, int q, int iw, int part) {
  return part ? (P.h2np[q][iw] & 15) : P.n_products;
}
template <int NT>
__device__ __forceinline__ int part_stages(const TcBatch& P, int q, int iw, int part) {
  return part_products(P, q, iw, part) == 1 ? (P.nK + NT - 1) / NT : P.nK;
}
// A one-product W2 part (rho <= 2^-11 FP16, 2^-15 BF16) of up to 512 stages (16384
// pairs) is one chain over the whole K range and is added together with the W1 part
// (h2_fused): the round-toward-zero bias of n accumulator additions is about
// n 2^-25.5 of the part, the part is within a few rho of chi0, and a 16384-pair
// FP16 part makes 2048 additions per accumulator: below 1e-7 of chi0.
__device__ __forceinline__ bool h2_fused(const TcBatch& P, int q, int iw) {
  return P.n_parts == 2 && P.h2np[q][iw] == 1 + 16 && P.nK <= 512;
}
__device__ __forceinline__ int part_chain(const TcBatch& P, int q, int iw, int part, int n_stages) {
  if (part && h2_fused(P, q, iw)) return n_stages;
  return (part && P.h2np[q][iw] >= 16) ? min(n_stages, 8 * P.chain_k) : P.chain_k;
}

// item -> (q, frequency, tile row, tile column); tiles are visited in groups of
// `group` tile rows, column by column inside a group (keeps A and B tiles of
// concurrently running CTAs close together in L2).  Hermitian mode visits only
// the tiles on or above the diagonal (row tm from column rr * tm on), in the
// same order: inside a group of rows, column by column, each column holding
// the group's rows tm with rr * tm <= tn (a staircase over the first columns).
__device__ __forceinline__ void decode_item(const TcBatch& P, int64_t item, int& q, int& iw, int& tm, int& tn) {
  q = 0;
  while (q + 1 < P.n_q && item >= P.item0[q + 1]) ++q;
  const int64_t r = item - P.item0[q];
  const int TM = P.tiles_m[q], TN = P.tiles_n[q];
  const int64_t tt = P.tpf[q];
  iw = (int)(r / tt);
  int t = (int)(r - (int64_t)iw * tt);
  if (P.n_parts == 2) {
    const int rr = P.rr, g = max(1, min(P.group, TM));
    int r0 = 0, r1 = min(g, TM);
    for (;;) {                                     // the group of rows holding item t
      int cnt = 0;
      for (int m = r0; m < r1; ++m) cnt += TN - rr * m;
      if (t < cnt || r1 >= TM) break;
      t -= cnt;
      r0 = r1;
      r1 = min(r1 + g, TM);
    }
    int col = rr * r0;
    for (;;) {                                     // staircase columns: rows r0 .. min(r1, col/rr + 1) - 1
      const int nrow = min(r1, col / rr + 1) - r0;
      if (nrow >= r1 - r0 || t < nrow) {
        if (t < nrow) {
          tm = r0 + t;
          tn = col;
          return;
        }
        break;
      }
      t -= nrow;
      ++col;
    }
    const int nrow = r1 - r0;                      // full columns from here on
    tn = col + t / nrow;
    tm = r0 + t % nrow;
    return;
  }
  const int g = min(P.group, TM);
  const int grp = t / (g * TN);
  const int first = grp * g;
  const int rows = min(g, TM - first);
  const int within = t - grp * g * TN;
  tm = first + within % rows;
  tn = within / rows;
}

// x 2^k as a double, exactly, by integer operations on the bits (the SM's FP64 pipe
// is narrow): zero and subnormal x give a signed zero, a result below the
// smallest normal double gives zero, Inf and NaN stay Inf and NaN.
__device__ __forceinline__ double f64_of_f32_pow2(float x, int k) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t sign = u & 0x80000000u;
  const int e = (int)((u >> 23) & 0xffu);
  const int ed = e + (1023 - 127) + k;
  uint32_t hi = sign | ((uint32_t)ed << 20) | ((u >> 3) & 0xfffffu);
  uint32_t lo = u << 29;
  if (e == 0 || ed <= 0) {
    hi = sign;
    lo = 0u;
  } else if (e == 255 || ed >= 2047) {
    hi = sign | 0x7ff00000u | (e == 255 ? (u >> 3) & 0xfffffu : 0u);
    lo = e == 255 ? lo : 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// chi0 element += v 2^k: the FP64 addition runs in L2 (a reduction, no value returned)
__device__ __forceinline__ void red_add_pow2(double* a, float v, int k) {
  atomicAdd(a, f64_of_f32_pow2(v, k));
}

// chi0[G][G] += the pack's diagonal sum when the row piece Hb..Hb+63 holds column G
__device__ __forceinline__ void add_diag(double2* __restrict__ chi_w, int nG, int G, int Hb,
                                         const double2* __restrict__ dg) {
  if ((unsigned)(G - Hb) < 64u) {
    const double2 d = dg[G];
    atomicAdd(&chi_w[(size_t)G * nG + G].x, d.x);
    atomicAdd(&chi_w[(size_t)G * nG + G].y, d.y);
  }
}

// Add a 32-row x 4-column block of complex values into chi0 by coalesced
// reductions.  The calling lane holds row G0 + lane: v = {re, im} of columns
// H0..H0+3.  The block passes through the warp's 32 x 8 shared-memory buffer xb
// (each row's floats XOR-swizzled by (row / 4) mod 8, so that neither the row
// writes nor the column reads meet a bank conflict), after which one
// reduction instruction covers 4 rows x 64 contiguous bytes instead of 32 rows
// of 8 bytes each.  An element (G, H) is added when G, H < nG and G < H
// (upper) or G != H (the diagonal takes the pack's sum).  Warp-collective.
__device__ __forceinline__ void red_block(double2* __restrict__ chi_w, int nG, int G0, int H0, const float (&v)[8],
                                          float* __restrict__ xb, int lane, int k, bool upper) {
  const int sw = (lane >> 2) & 7;
#pragma unroll
  for (int e = 0; e < 8; ++e) xb[lane * 8 + (e ^ sw)] = v[e];
  __syncwarp();
  const int e = lane & 7;                        // column e / 2, real (e even) or imaginary part
  const int H = H0 + (e >> 1);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int r = 4 * j + (lane >> 3);           // row r was written by lane r, swizzled by j
    const float x = xb[r * 8 + (e ^ j)];
    const int G = G0 + r;
    if (H < nG && G < nG && (upper ? G < H : G != H))
      red_add_pow2(reinterpret_cast<double*>(chi_w + (size_t)G * nG + H) + (e & 1), x, k);
  }
  __syncwarp();
}

// Add one drained part of a tile row (row G, columns Hb..Hb+63; FP32 sums whose
// scale is 2^-k) into chi0 of one frequency.  Plain mode: chi[G][H] += 2^k (re +
// i im).  Hermitian mode: part 0 holds H1(G, H), part 1 holds H2(G, H); chi[G][H]
// += (1 + i t) H1 + i H2 and chi[H][G] += (1 + i t) conj(H1) + i conj(H2) for G
// < H.  Each (1 + i t) product is one FP32 fused multiply-add (one rounding; t
// is an FP32 number), the power of two and the widening to FP64 are exact, and
// the FP64 sums are reductions: the epilogue issues no FP64 arithmetic.  The
// diagonal element is left out: it takes the pack's sum (add_diag).  The
// lanes' reductions into chi[G][H] fall on 32 rows each; this merge runs while
// the next chains accumulate (the part's buffers are released), and going
// through red_block lengthened it past that overlap (a 64-atom BF16 launch took
// 11.66 ms with it, 10.8 ms without).
__device__ __forceinline__ void merge_row(double2* __restrict__ chi_w, int nG, int G, int Hb, const float (&sre)[64],
                                          const float (&sim)[64], int k, bool herm, int part, float t) {
  double2* row = chi_w + (size_t)G * nG;
  if (!herm) {
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      if (Hb + i < nG && Hb + i != G) {
        red_add_pow2(&row[Hb + i].x, sre[i], k);
        red_add_pow2(&row[Hb + i].y, sim[i], k);
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    const int H = Hb + i;
    if (H < nG && G < H) {
      const float a = sre[i], b = sim[i];
      double2* m = chi_w + (size_t)H * nG + G;
      if (part == 0) {
        red_add_pow2(&row[H].x, fmaf(-t, b, a), k);
        red_add_pow2(&row[H].y, fmaf(t, a, b), k);
        red_add_pow2(&m->x, fmaf(t, b, a), k);
        red_add_pow2(&m->y, fmaf(t, a, -b), k);
      } else {
        red_add_pow2(&row[H].x, -b, k);
        red_add_pow2(&row[H].y, a, k);
        red_add_pow2(&m->x, b, k);
        red_add_pow2(&m->y, a, k);
      }
    }
  }
}

// exponent k of a power of two 2^k held as a double
__device__ __forceinline__ int exponent_of_pow2(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}

// Hermitian mode with a one-product W2 part: add both parts of a tile row at once,
// chi[G][H] += (1 + i t) H1 + i H2 and chi[H][G] += (1 + i t) conj(H1) + i
// conj(H2) for G < H (the diagonal takes the pack's sum), both read from
// tensor memory 16 columns at a time: the W1 sums (scale 2^-k1) at column
// address ta1 (Re) and ta1 + 128 (Im), the W2 accumulator at ta2, scaled to the
// W1 units by 2^(k2 - k1) (exact; a ratio outside the FP32 exponent range drops
// H2: below 2^-126 it is negligible, above 2^127 the W2 weights were zero).
// Both tensor-memory buffers stay held while this runs, so the MMAs wait for it:
// the elements (G, H) go through red_block (coalesced), the mirrored ones (H, G)
// directly (consecutive lanes, consecutive addresses).  Warp-collective (the
// loads and red_block): every lane calls it, rows G >= nG add nothing.
__device__ __forceinline__ void merge_row_fused(double2* __restrict__ chi_w, int nG, int G, int Hb, uint32_t ta1,
                                                uint32_t ta2, int k1, int k2, float t, float* __restrict__ xb,
                                                int lane) {
  const int d = k2 - k1;
  const float r21 = d >= -126 && d <= 127 ? __int_as_float((d + 127) << 23) : 0.f;
  const bool in = G < nG;
#pragma unroll 1
  for (int j = 0; j < 64; j += 16) {
    float re1[16], im1[16], re2[16], im2[16];
    tc::tmem_ld16(ta1 + j, re1);
    tc::tmem_ld16(ta1 + 128 + j, im1);
    tc::tmem_ld16(ta2 + j, re2);
    tc::tmem_ld16(ta2 + 128 + j, im2);
    tc::tmem_ld_wait();
    tc::reg_after_wait(re1);
    tc::reg_after_wait(im1);
    tc::reg_after_wait(re2);
    tc::reg_after_wait(im2);
#pragma unroll
    for (int c = 0; c < 16; c += 4) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float a1 = re1[c + i], b1 = im1[c + i], a2 = re2[c + i] * r21, b2 = im2[c + i] * r21;
        v[2 * i] = fmaf(-t, b1, a1) - b2;
        v[2 * i + 1] = fmaf(t, a1, b1) + a2;
      }
      red_block(chi_w, nG, G - lane, Hb + j + c, v, xb, lane, k1, true);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int H = Hb + j + i;
      if (in && H < nG && G < H) {
        const float a1 = re1[i], b1 = im1[i], a2 = re2[i] * r21, b2 = im2[i] * r21;
        double2* m = chi_w + (size_t)H * nG + G;
        red_add_pow2(&m->x, fmaf(t, b1, a1) + b2, k1);
        red_add_pow2(&m->y, fmaf(t, a1, -b1) + a2, k1);
      }
    }
  }
}

// Drain the nch accumulation chains of one part into the FP32 sums (zeroed first),
// two 32-column loads at a time; each buffer is released as soon as its last
// values are in registers, before they are added.
// keep_last: the last chain's buffer is not released and receives the part's
// total sums (held for a later merge).  Returns false when a bounded wait ran out.
template <bool PAIR, class BarT>
__device__ __forceinline__ bool drain_part(BarT* bar, uint32_t tbase, int quad, int half, int lane, int nch,
                                           bool keep_last, int64_t& gc, int* status, float (&sre)[64],
                                           float (&sim)[64]) {
#pragma unroll
  for (int i = 0; i < 64; ++i) { sre[i] = 0.f; sim[i] = 0.f; }
  for (int c = 0; c < nch; ++c, ++gc) {
    const int buf = (int)(gc & 1);
    if (!tc::mbar_wait(&bar->tfull[buf], (uint32_t)((gc >> 1) & 1), status, 1, WAIT_BUDGET_NS)) return false;
    tc::fence_after();
    const uint32_t ta = tbase + ((uint32_t)(quad * 32) << 16) + buf * 256 + half * 64;
    // two loads in flight (the epilogue warps hold REG_HIGH registers); the buffer is
    // released as soon as its last values are in registers, before they are added
    float v[32], w[32];
    tc::tmem_ld32(ta, v);
    tc::tmem_ld32(ta + 32, w);
    tc::tmem_ld_wait();
    tc::reg_after_wait(v);
    tc::reg_after_wait(w);
#pragma unroll
    for (int i = 0; i < 32; ++i) sre[i] += v[i];
#pragma unroll
    for (int i = 0; i < 32; ++i) sre[32 + i] += w[i];
    tc::tmem_ld32(ta + 128, v);
    tc::tmem_ld32(ta + 160, w);
    tc::tmem_ld_wait();
    tc::reg_after_wait(v);
    tc::reg_after_wait(w);
    if (!(keep_last && c == nch - 1)) {
      tc::fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (PAIR) tc::mbar_arrive_cluster(tc::mapa(&bar->tempty[buf], 0));
        else tc::mbar_arrive(&bar->tempty[buf]);
      }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) sim[i] += v[i];
#pragma unroll
    for (int i = 0; i < 32; ++i) sim[32 + i] += w[i];
  }
  if (keep_last) {
    const uint32_t ta = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)((gc - 1) & 1) * 256 + half * 64;
    tc::tmem_st32_part<0>(ta, sre);
    tc::tmem_st32_part<1>(ta + 32, sre);
    tc::tmem_st32_part<0>(ta + 128, sim);
    tc::tmem_st32_part<1>(ta + 160, sim);
    tc::tmem_st_wait();
  }
  return true;
}

// The epilogue of one item (q, frequency, tile): per part, its chains into FP32 sums
// and their reductions into chi0.  In Hermitian mode with a one-product W2 part,
// the W1 total stays in its last chain's buffer, the W2 part is a single chain in
// the other buffer, and both are added in one pass (half the reductions).
// Returns false when a bounded wait ran out.
template <int NT, bool PAIR, class BarT>
__device__ __forceinline__ bool epilogue_item(const TcBatch& P, BarT* bar, uint32_t tbase, int quad, int half,
                                              int lane, int q, int iw, int G, int tn, int64_t& gc, int* status,
                                              float* xb) {
  // (everything else is read from the launch parameters after the drain, where the
  // sums no longer fill the registers)
  const bool fused = h2_fused(P, q, iw);
  for (int part = 0; part < P.n_parts; ++part) {
    const int nks = part_stages<NT>(P, q, iw, part);
    const int ck = part_chain(P, q, iw, part, nks);
    float sre[64], sim[64];
    if (!drain_part<PAIR>(bar, tbase, quad, half, lane, (nks + ck - 1) / ck, fused, gc, status, sre, sim))
      return false;
    const int nG = P.nG[q];
    double2* chi_w = P.chi[q] + (size_t)iw * nG * nG;
    const bool herm = P.n_parts == 2;
    const float t = herm ? (float)P.tbar[q][iw] : 0.f;
    const int k = exponent_of_pow2(P.inv[q][part * P.n_freq + iw]);
    if (fused) {
      const int b1 = (int)((gc - 1) & 1), b2 = (int)(gc & 1);
      if (!tc::mbar_wait(&bar->tfull[b2], (uint32_t)((gc >> 1) & 1), status, 1, WAIT_BUDGET_NS)) return false;
      tc::fence_after();
      const uint32_t tq = tbase + ((uint32_t)(quad * 32) << 16) + half * 64;
      merge_row_fused(chi_w, nG, G, tn * BN + half * 64, tq + b1 * 256, tq + b2 * 256, k,
                      exponent_of_pow2(P.inv[q][P.n_freq + iw]), t, xb, lane);
      if (G < nG) add_diag(chi_w, nG, G, tn * BN + half * 64, P.diag[q] + (size_t)iw * P.tiles_n[q] * BN);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (PAIR) {
          tc::mbar_arrive_cluster(tc::mapa(&bar->tempty[b1], 0));
          tc::mbar_arrive_cluster(tc::mapa(&bar->tempty[b2], 0));
        } else {
          tc::mbar_arrive(&bar->tempty[b1]);
          tc::mbar_arrive(&bar->tempty[b2]);
        }
      }
      ++gc;
      return true;
    }
    if (G < nG) {
      merge_row(chi_w, nG, G, tn * BN + half * 64, sre, sim, k, herm, part, t);
      if (part == 0) add_diag(chi_w, nG, G, tn * BN + half * 64, P.diag[q] + (size_t)iw * P.tiles_n[q] * BN);
    }
  }
  return true;
}

template <bool BF16, int NT>
__global__ void __launch_bounds__(THREADS, 1)
k_contract_tc(const __grid_constant__ TcBatch P, int* __restrict__ status) {
  using RG = Ring<NT>;
  constexpr int STAGES = RG::STAGES, STAGE_BYTES = RG::STAGE_BYTES, PL = RG::PLANES;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* tiles = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_tc) + 1023) & ~uintptr_t(1023));
  Barriers* bar = reinterpret_cast<Barriers*>(tiles + RING_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nK = P.nK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&bar->full[s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->tfull[b], 1);
      tc::mbar_init(&bar->tempty[b], EPI_WARPS);
    }
    tc::mbar_init(&bar->done, 1);
    tc::fence_mbar_init();
    for (int q = 0; q < P.n_q; ++q) {
      tc::prefetch_tmap(&P.tmA[q]);
      tc::prefetch_tmap(&P.tmB[q]);
    }
  }
  if (warp == 1) {
    tc::tmem_alloc(&bar->tmem_base, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = bar->tmem_base;

  // warpgroup 0 (producer, issuer, two idle warps) runs on REG_LOW registers,
  // the epilogue warpgroups on REG_HIGH
  if (warp < EPI_WARP0) {
  tc::setmaxnreg_dec<REG_LOW>();
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int64_t gs = 0;
      int slot = 0;        // ring slot of stage gs and its phase parity (counters, not divisions)
      uint32_t ph = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < P.total_items && ok; item += gridDim.x) {
        int q, iw, tm, tn;
        decode_item(P, item, q, iw, tm, tn);
        for (int part = 0; part < P.n_parts && ok; ++part) {
          // planes of the terms the part's products read (t2 only with six products)
          const int npp = part_products(P, q, iw, part);
          const bool one = npp == 1;                  // k-slices of term 0 in the term slots
          const int nt = one ? 1 : ((NT == 3 && npp != 6) ? 2 : NT);
          const int nks = part_stages<NT>(P, q, iw, part);
          const int plane0 = (part * P.n_freq + iw) * PL;
          const int row_a = tm * BM, row_b = tn * BN;
          for (int kc = 0; kc < nks; ++kc, ++gs) {
            const int s = slot;
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, status, 1, WAIT_BUDGET_NS)) { ok = false; break; }
            if (++slot == STAGES) {
              slot = 0;
              ph ^= 1u;
            }
            const int ns = one ? min(NT, nK - kc * NT) : nt;   // slices (one product) or terms loaded
            tc::mbar_arrive_expect_tx(&bar->full[s], 4 * ns * TILE_BYTES);
            unsigned char* st = tiles + (size_t)s * STAGE_BYTES;
#pragma unroll
            for (int j = 0; j < PL; ++j) {
              const int t = j % NT;
              if (t >= ns) continue;
              // one product: slot j takes term 0 of its re/im half at k-slice kc NT + t
              const int pa = one ? (j / NT) * NT : j;
              // B of a one-product part: the FP16 term-0 planes of BF16 plans (2 NT, 2 NT + 1)
              const int pb = (BF16 && one) ? 2 * NT + j / NT : pa;
              const int kx = one ? (kc * NT + t) * BK : kc * BK;
              tc::tma_load_3d(st + j * TILE_BYTES, &P.tmA[q], &bar->full[s], kx, row_a, plane0 + pa);
              tc::tma_load_3d(st + (PL + j) * TILE_BYTES, &P.tmB[q], &bar->full[s], kx, row_b, pb);
            }
          }
        }
      }
      // copies still in flight must land before the CTA may exit
      for (int64_t g = max((int64_t)0, gs - STAGES); g < gs; ++g)
        tc::mbar_wait(&bar->full[g % STAGES], (uint32_t)((g / STAGES) & 1), status, 1, WAIT_BUDGET_NS);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int64_t gs = 0, gc = 0;
      int slot = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < P.total_items && ok; item += gridDim.x) {
        int q, iw, tm, tn;
        decode_item(P, item, q, iw, tm, tn);
        for (int part = 0; part < P.n_parts && ok; ++part) {
          const int np = part_products(P, q, iw, part), nks = part_stages<NT>(P, q, iw, part);
          const int ck = part_chain(P, q, iw, part, nks);
          // pos: stage within the accumulation chain; s, ph: ring slot and its phase (counters,
          // not divisions, on this single issuing thread)
          for (int kc = 0, pos = 0; kc < nks; ++kc, ++gs) {
            const int buf = (int)(gc & 1);
            const bool first = pos == 0;
            if (first) {
              if (!tc::mbar_wait(&bar->tempty[buf], (uint32_t)(((gc >> 1) & 1) ^ 1), status, 1, WAIT_BUDGET_NS)) {
                ok = false;
                break;
              }
              tc::fence_after();
            }
            const int s = slot;
            if (!tc::mbar_wait(&bar->full[s], ph, status, 1, WAIT_BUDGET_NS)) {
              ok = false;
              break;
            }
            if (++slot == STAGES) {
              slot = 0;
              ph ^= 1u;
            }
            tc::fence_after();
            const unsigned char* st = tiles + (size_t)s * STAGE_BYTES;
            const uint32_t d_re = tbase + buf * 256, d_im = d_re + 128;
            if (np == 1) issue_stage_1p<false, NT, false>(st, d_re, d_im, first, min(NT, nK - kc * NT));
            else issue_stage<BF16, NT>(st, d_re, d_im, first, np);
            tc::mma_commit(&bar->empty[s]);
            if (++pos == ck || kc == nks - 1) {
              tc::mma_commit(&bar->tfull[buf]);
              ++gc;
              pos = 0;
            }
          }
        }
      }
      tc::mma_commit(&bar->done);
      tc::mbar_wait(&bar->done, 0, status, 1, WAIT_BUDGET_NS);
    }
  }
  } else {
    tc::setmaxnreg_inc<REG_HIGH>();
    // ---------------- epilogue: drain chains, then FP64 reductions per item ----------------
    const int ew = warp - EPI_WARP0, quad = warp & 3, half = ew >> 2;
    const int row = quad * 32 + lane;
    float* xb = reinterpret_cast<float*>(tiles + RING_BYTES + BAR_BYTES) + ew * XBUF_FLOATS;
    int64_t gc = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < P.total_items && ok; item += gridDim.x) {
      int q, iw, tm, tn;
      decode_item(P, item, q, iw, tm, tn);
      ok = epilogue_item<NT, false>(P, bar, tbase, quad, half, lane, q, iw, tm * BM + row, tn, gc, status, xb);
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// CTA-pair variant: a cluster of two CTAs computes a 256 x 128 output tile with
// tcgen05.mma.cta_group::2 (each CTA holds 128 rows of A and 64 rows of B, the
// MMA issued by the first CTA reads both).  Shared-memory operand traffic per
// MMA drops from 8 KB to 6 KB per CTA, which is what limits the single-CTA
// kernel.  The first CTA's "full" barriers count the loads of both CTAs; its
// MMA commits release both CTAs' stages and accumulators; both CTAs' epilogues
// release the accumulators on the first CTA's "tempty" barriers.
// ---------------------------------------------------------------------------
constexpr int RING2_BYTES = 216 * 1024;
constexpr size_t SMEM2_BYTES = (size_t)RING2_BYTES + 1024 + BAR_BYTES + EPI_WARPS * XBUF_FLOATS * 4;
static_assert(SMEM2_BYTES <= 227 * 1024, "CTA-pair shared memory above the per-block limit");

template <int NT> struct Ring2 {
  static constexpr int PLANES = 2 * NT;
  static constexpr int A_BYTES = TILE_BYTES;          // 128 rows x 32 pairs
  static constexpr int B_BYTES = TILE_BYTES / 2;      // 64 rows x 32 pairs
  static constexpr int STAGE_BYTES = PLANES * (A_BYTES + B_BYTES);
  static constexpr int STAGES = RING2_BYTES / STAGE_BYTES;   // 4 for NT = 2, 3 for NT = 3
};

template <bool BF16, int NT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
k_contract_tc2(const __grid_constant__ TcBatch P, int* __restrict__ status) {
  using RG = Ring2<NT>;
  constexpr int STAGES = RG::STAGES, STAGE_BYTES = RG::STAGE_BYTES, PL = RG::PLANES;
  static_assert(STAGES <= MAX_STAGES + 1, "barrier array too small");
  extern __shared__ __align__(1024) unsigned char smem_tc2[];
  unsigned char* tiles = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_tc2) + 1023) & ~uintptr_t(1023));
  struct Bars {
    uint64_t full[4], empty[4], tfull[2], tempty[2], done;
    uint32_t tmem_base;
  };
  static_assert(sizeof(Bars) <= BAR_BYTES, "barriers overlap the transpose buffers");
  Bars* bar = reinterpret_cast<Bars*>(tiles + RING2_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = tc::cluster_rank();
  const bool leader = rank == 0;
  const int64_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int nK = P.nK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&bar->full[s], 1);
      tc::mbar_init(&bar->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&bar->tfull[b], 1);
      tc::mbar_init(&bar->tempty[b], 2 * EPI_WARPS);
    }
    tc::mbar_init(&bar->done, 1);
    tc::fence_mbar_init();
    for (int q = 0; q < P.n_q; ++q) {
      tc::prefetch_tmap(&P.tmA[q]);
      tc::prefetch_tmap(&P.tmB[q]);
    }
  }
  if (warp == 1) {
    tc::tmem_alloc_pair(&bar->tmem_base, TMEM_COLS);
    tc::tmem_relinquish_pair();
  }
  tc::fence_before();
  __syncthreads();
  tc::cluster_sync();      // barriers of both CTAs initialised before any remote use
  tc::fence_after();
  const uint32_t tbase = bar->tmem_base;

  // warpgroup 0 (producer, issuer, two idle warps) runs on REG_LOW registers,
  // the epilogue warpgroups on REG_HIGH
  if (warp < EPI_WARP0) {
  tc::setmaxnreg_dec<REG_LOW>();
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs) ----------------
      int64_t gs = 0;
      int slot = 0;        // ring slot of stage gs and its phase parity
      uint32_t ph = 0;
      bool ok = true;
      for (int64_t item = pair; item < P.total_items && ok; item += npairs) {
        int q, iw, tm, tn;
        decode_item(P, item, q, iw, tm, tn);
        const int arow = tm * 2 * BM + (int)rank * BM;     // this CTA's 128 rows of A
        const int brow = tn * BN + (int)rank * (BN / 2);   // this CTA's 64 rows of B
        for (int part = 0; part < P.n_parts && ok; ++part) {
          const int npp = part_products(P, q, iw, part);
          const bool one = npp == 1;                  // k-slices of term 0 in the term slots
          const int nt = one ? 1 : ((NT == 3 && npp != 6) ? 2 : NT);
          const int nks = part_stages<NT>(P, q, iw, part);
          const int plane0 = (part * P.n_freq + iw) * PL;
          for (int kc = 0; kc < nks; ++kc, ++gs) {
            const int s = slot;
            if (!tc::mbar_wait(&bar->empty[s], ph ^ 1u, status, 1, WAIT_BUDGET_NS)) { ok = false; break; }
            if (++slot == STAGES) {
              slot = 0;
              ph ^= 1u;
            }
            const int ns = one ? min(NT, nK - kc * NT) : nt;
            // the first CTA's barrier counts the loads of both CTAs
            if (leader) tc::mbar_arrive_expect_tx(&bar->full[s], 4 * ns * (RG::A_BYTES + RG::B_BYTES));
            const uint32_t fb = tc::mapa(&bar->full[s], 0);
            unsigned char* st = tiles + (size_t)s * STAGE_BYTES;
#pragma unroll
            for (int j = 0; j < PL; ++j) {
              const int t = j % NT;
              if (t >= ns) continue;
              const int pa = one ? (j / NT) * NT : j;
              const int pb = (BF16 && one) ? 2 * NT + j / NT : pa;
              const int kx = one ? (kc * NT + t) * BK : kc * BK;
              tc::tma_load_3d_pair(st + j * RG::A_BYTES, &P.tmA[q], fb, kx, arow, plane0 + pa);
              tc::tma_load_3d_pair(st + PL * RG::A_BYTES + j * RG::B_BYTES, &P.tmB[q], fb, kx, brow, pb);
            }
          }
        }
      }
      // copies of this CTA still in flight land before it may exit: wait until the
      // pair's MMA has released the stages it issued last
      for (int64_t g = max((int64_t)0, gs - STAGES); g < gs; ++g)
        tc::mbar_wait(&bar->empty[g % STAGES], (uint32_t)((g / STAGES) & 1), status, 1, WAIT_BUDGET_NS);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (first CTA of the pair) ----------------
      int64_t gs = 0, gc = 0;
      int slot = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int64_t item = pair; item < P.total_items && ok; item += npairs) {
        int q, iw, tm, tn;
        decode_item(P, item, q, iw, tm, tn);
        for (int part = 0; part < P.n_parts && ok; ++part) {
          const int np = part_products(P, q, iw, part), nks = part_stages<NT>(P, q, iw, part);
          const int ck = part_chain(P, q, iw, part, nks);
          // pos: stage within the accumulation chain; s, ph: ring slot and its phase (counters,
          // not divisions, on this single issuing thread)
          for (int kc = 0, pos = 0; kc < nks; ++kc, ++gs) {
            const int buf = (int)(gc & 1);
            const bool first = pos == 0;
            if (first) {
              if (!tc::mbar_wait(&bar->tempty[buf], (uint32_t)(((gc >> 1) & 1) ^ 1), status, 1, WAIT_BUDGET_NS)) {
                ok = false;
                break;
              }
              tc::fence_after();
            }
            const int s = slot;
            if (!tc::mbar_wait(&bar->full[s], ph, status, 1, WAIT_BUDGET_NS)) {
              ok = false;
              break;
            }
            if (++slot == STAGES) {
              slot = 0;
              ph ^= 1u;
            }
            tc::fence_after();
            const unsigned char* st = tiles + (size_t)s * STAGE_BYTES;
            const uint32_t d_re = tbase + buf * 256, d_im = d_re + 128;
            if (np == 1) issue_stage_1p<false, NT, true>(st, d_re, d_im, first, min(NT, nK - kc * NT));
            else issue_stage<BF16, NT, true>(st, d_re, d_im, first, np);
            tc::mma_commit_pair(&bar->empty[s], 0x3);
            if (++pos == ck || kc == nks - 1) {
              tc::mma_commit_pair(&bar->tfull[buf], 0x3);
              ++gc;
              pos = 0;
            }
          }
        }
      }
      tc::mma_commit_pair(&bar->done, 0x1);
      tc::mbar_wait(&bar->done, 0, status, 1, WAIT_BUDGET_NS);
    }
  }
  } else {
    tc::setmaxnreg_inc<REG_HIGH>();
    // ---------------- epilogue (both CTAs, own 128 rows) ----------------
    const int ew = warp - EPI_WARP0, quad = warp & 3, half = ew >> 2;
    const int row = quad * 32 + lane;
    float* xb = reinterpret_cast<float*>(tiles + RING2_BYTES + BAR_BYTES) + ew * XBUF_FLOATS;
    int64_t gc = 0;
    bool ok = true;
    for (int64_t item = pair; item < P.total_items && ok; item += npairs) {
      int q, iw, tm, tn;
      decode_item(P, item, q, iw, tm, tn);
      ok = epilogue_item<NT, true>(P, bar, tbase, quad, half, lane, q, iw, tm * 2 * BM + (int)rank * BM + row, tn, gc,
                                   status, xb);
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::cluster_sync();      // neither CTA leaves while the pair's MMAs may still read its operands
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc_pair(tbase, TMEM_COLS);
}

// Diagnostic: wait on an mbarrier that nothing arrives on, with the same
// bounded wait as the contraction, so the time-out path can be exercised.
__global__ void k_wait_selftest(uint64_t budget_ns, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) tc::mbar_wait(&bar, 0, status, 1, budget_ns);
  __syncthreads();
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool resolve_encoder(std::string* why) {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    if (why) *why = "cuTensorMapEncodeTiled is not available from the driver";
    cudaGetLastError();
    return false;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

bool encode_planes(CUtensorMap* tm, void* base, bool bf16, int Kp, int nGp, int planes, std::string* why,
                   int box_rows = BM) {
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)nGp, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * nGp};
  cuuint32_t box[3] = {BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (why) *why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

}  // namespace

cudaError_t launch_wait_selftest(chi0_plan_s* p, double budget_ms, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>((uint64_t)(budget_ms * 1e6), p->d_status);
  return cudaGetLastError();
}

bool tc_supported(std::string* why) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    if (why) *why = "no CUDA device";
    return false;
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    if (why) *why = "device is sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + ", kernels are built for sm_103a";
    return false;
  }
  return resolve_encoder(why);
}

int n_terms(const chi0_plan_s* p) { return p->n_products == 6 ? 3 : 2; }

// B planes: the terms of Re M and Im M, and in BF16 Hermitian plans the FP16 term 0
// of both (operands of the one-product W2 parts)
int b_planes(const chi0_plan_s* p) {
  return 2 * n_terms(p) + (p->prec == CHI0_SPLIT_BF16 && p->tc_herm ? 2 : 0);
}

// A planes per frequency and part: W (plain) or W1 and W2 (Hermitian mode)
int n_parts(const chi0_plan_s* p) { return p->tc_herm ? 2 : 1; }

size_t planes_bytes(const chi0_plan_s* p) {
  const size_t nGp = (size_t)round_up_i(p->max_nG, 2 * BM);
  const size_t Kp = (size_t)((p->max_pairs + 63) / 64 * 64);
  return ((size_t)b_planes(p) + 2 * (size_t)n_terms(p) * n_parts(p) * p->n_freq) * nGp * Kp * 2;
}

// amax, ratio range, scales, inverse scales, W2 products, ratios t
static size_t scal_bytes(const chi0_plan_s* p) { return (256 + 64 * (size_t)(p->n_freq + 1) + 255) / 256 * 256; }

size_t tc_pack_bytes(const chi0_plan_s* p, int64_t max_pairs, int max_nG) {
  const size_t nGp = (size_t)round_up_i(max_nG, 2 * BM);
  const size_t Kp = (size_t)((max_pairs + 63) / 64 * 64);
  const size_t planes = (size_t)b_planes(p) + 2 * (size_t)n_terms(p) * n_parts(p) * p->n_freq;
  // then the diagonal sums [n_freq][nGp]
  return planes * nGp * Kp * 2 + scal_bytes(p) + (size_t)p->n_freq * nGp * sizeof(double2);
}

// workspace of one q-point's split planes: B, A, then amax / ratio range /
// scales / inverse scales / W2 product counts / ratios t (each part sized for
// two values per frequency), then the diagonal sums [n_freq][nGp]
struct PackWs {
  uint16_t* Bp;
  uint16_t* Ap;
  unsigned int* amax;
  unsigned int* tr;
  float* scale;
  double* inv;
  int* h2np;
  double* tbar;
  double2* diag;
};

static cudaError_t fill_ratio_min(unsigned int* tr, int n_freq, cudaStream_t s) {
  k_ratio_init<<<1, 128, 0, s>>>(tr, n_freq);
  return cudaGetLastError();
}

static PackWs pack_ws(const chi0_plan_s* p, void* base, int nGp, int Kp) {
  const size_t nf1 = (size_t)(p->n_freq + 1);
  PackWs w;
  w.Bp = reinterpret_cast<uint16_t*>(base);
  w.Ap = w.Bp + (size_t)b_planes(p) * nGp * Kp;
  unsigned char* tail = reinterpret_cast<unsigned char*>(base) + planes_bytes(p);
  w.amax = reinterpret_cast<unsigned int*>(tail);            // 1 + 2 n_freq words
  w.tr = reinterpret_cast<unsigned int*>(tail + 8 * nf1);     // 2 n_freq words
  w.scale = reinterpret_cast<float*>(tail + 16 * nf1);        // 1 + 2 n_freq floats
  w.inv = reinterpret_cast<double*>(tail + 24 * nf1);         // 2 n_freq doubles
  w.h2np = reinterpret_cast<int*>(tail + 40 * nf1);           // n_freq ints
  w.tbar = reinterpret_cast<double*>(tail + 48 * nf1);        // n_freq doubles
  w.diag = reinterpret_cast<double2*>(tail + scal_bytes(p));  // n_freq x nGp
  return w;
}

template <bool BF16, int NT>
static cudaError_t pack_one(chi0_plan_s* p, int nG, const float2* M, int64_t K, const double2* f, const PackWs& w,
                            int nGp, int Kp, cudaStream_t s) {
  ProfScope ps(p, CHI0_K_PACK, s, p->tc_herm ? 4 : 3);
  cudaError_t e = cudaMemsetAsync(w.amax, 0, sizeof(unsigned int) * (2 * p->n_freq + 1), s);
  if (e != cudaSuccess) return e;
  if (p->tc_herm) {
    // ratio range: minimum starts at the largest order value, maximum at the smallest
    e = cudaMemsetAsync(w.tr, 0, sizeof(unsigned int) * 2 * p->n_freq, s);
    if (e == cudaSuccess) e = fill_ratio_min(w.tr, p->n_freq, s);
    if (e != cudaSuccess) return e;
  }
  k_absmax<<<2 * 152, 256, 0, s>>>(M, K * nG, f, K, p->n_freq, w.amax, p->tc_herm ? w.tr : nullptr);
  k_scales<<<1, 128, 0, s>>>(w.amax, w.tr, p->n_freq, p->tc_herm ? 1 : 0, p->n_products, BF16 ? 1 : 0, w.scale,
                             w.inv, w.h2np, w.tbar);
  e = cudaMemsetAsync(w.diag, 0, sizeof(double2) * p->n_freq * nGp, s);
  if (e != cudaSuccess) return e;
  dim3 gpk(nGp / 32, Kp / 64);
  const size_t smp = (size_t)(64 * 33 + 2 * 64 * p->n_freq) * sizeof(float2);
  e = cudaFuncSetAttribute(k_pack<BF16, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
  if (e != cudaSuccess) return e;
  k_pack<BF16, NT><<<gpk, 256, smp, s>>>(M, nG, K, nGp, Kp, f, p->n_freq, p->tc_herm ? 1 : 0, w.scale, w.h2np,
                                         w.tbar, (uint32_t*)w.Bp, (uint32_t*)w.Ap, w.diag);
  return cudaGetLastError();
}

// The warpgroups' register split inside the contraction kernels (REG_LOW, REG_HIGH)
// adds up to the registers of a launch with REG_LAUNCH per thread; a build that
// compiled the kernel with another count would make the increase wait forever,
// so such a kernel is never launched.
template <class Kern>
static bool regs_match(Kern kern, std::string* why) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, kern) != cudaSuccess) {
    cudaGetLastError();
    if (why) *why = "cannot read the contraction kernel's attributes";
    return false;
  }
  if (a.numRegs != REG_LAUNCH) {
    if (why)
      *why = "contraction kernel compiled with " + std::to_string(a.numRegs) + " registers per thread; its "
             "warpgroup register split needs " + std::to_string(REG_LAUNCH);
    return false;
  }
  return true;
}

template <bool BF16, int NT>
static cudaError_t run_tc(chi0_plan_s* p, const TcJob* jobs, int n_jobs, int64_t K, cudaStream_t s,
                          std::string* why, int mode) {
  const int Kp = (int)((K + 63) / 64 * 64);
  TcBatch* P = new TcBatch();
  memset(P, 0, sizeof(TcBatch));
  int64_t items = 0;
  const bool pair = p->tc_pair != 0;
  for (int j = 0; j < n_jobs; ++j) {
    const TcJob& jb = jobs[j];
    const int nGp = round_up_i(jb.nG, pair ? 2 * BM : BM);
    PackWs w = pack_ws(p, jb.pack, nGp, Kp);
    if (mode != 2) {
      cudaError_t e = pack_one<BF16, NT>(p, jb.nG, jb.M, K, jb.f, w, nGp, Kp, s);
      if (e != cudaSuccess) { delete P; return e; }
      if (mode == 1) continue;
    }
    if (!encode_planes(&P->tmB[j], w.Bp, BF16, Kp, nGp, b_planes(p), why, pair ? BN / 2 : BN) ||
        !encode_planes(&P->tmA[j], w.Ap, BF16, Kp, nGp, 2 * NT * n_parts(p) * p->n_freq, why, BM)) {
      delete P;
      return cudaErrorInvalidValue;
    }
    P->chi[j] = jb.chi;
    P->inv[j] = w.inv;
    P->h2np[j] = w.h2np;
    P->tbar[j] = w.tbar;
    P->diag[j] = w.diag;
    P->nG[j] = jb.nG;
    const int TM = nGp / (pair ? 2 * BM : BM), TN = nGp / BN;
    P->tiles_m[j] = TM;
    P->tiles_n[j] = TN;
    // Hermitian mode: row tm holds the TN - rr tm tiles from column rr tm on
    P->tpf[j] = p->tc_herm ? (int64_t)(TN / TM) * TM * (TM + 1) / 2 : (int64_t)TM * TN;
    P->item0[j] = items;
    items += P->tpf[j] * p->n_freq;
  }
  if (mode == 1) {
    delete P;
    return cudaSuccess;
  }
  P->n_parts = n_parts(p);
  P->rr = pair ? 2 : 1;
  P->item0[n_jobs] = items;
  P->n_q = n_jobs;
  P->n_freq = p->n_freq;
  P->nK = Kp / BK;
  P->chain_k = std::max(1, p->chain_pairs / BK);
  P->n_products = p->n_products;
  P->group = p->tc_group > 0 ? p->tc_group : 8;
  P->total_items = items;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (pair) {
    if (!regs_match(k_contract_tc2<BF16, NT>, why)) { delete P; return cudaErrorNotSupported; }
    e = cudaFuncSetAttribute(k_contract_tc2<BF16, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM2_BYTES);
    if (e != cudaSuccess) { delete P; return e; }
    const int pairs = (int)std::min<int64_t>(items, (int64_t)(nsm / 2));
    ProfScope ps(p, CHI0_K_CONTRACT_TC, s, 1);
    k_contract_tc2<BF16, NT><<<2 * pairs, THREADS, SMEM2_BYTES, s>>>(*P, p->d_status);
  } else {
    if (!regs_match(k_contract_tc<BF16, NT>, why)) { delete P; return cudaErrorNotSupported; }
    e = cudaFuncSetAttribute(k_contract_tc<BF16, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
    if (e != cudaSuccess) { delete P; return e; }
    const int grid = (int)std::min<int64_t>(items, (int64_t)nsm * std::max(1, p->tc_ctas_per_sm));
    ProfScope ps(p, CHI0_K_CONTRACT_TC, s, 1);
    k_contract_tc<BF16, NT><<<grid, THREADS, SMEM_BYTES, s>>>(*P, p->d_status);
  }
  delete P;
  return cudaGetLastError();
}

cudaError_t launch_contract_tc_batch(chi0_plan_s* p, const TcJob* jobs, int n_jobs, int64_t K, cudaStream_t s,
                                     std::string* why, int mode) {
  if (K <= 0 || n_jobs <= 0) return cudaSuccess;
  if (n_jobs > MAXQ) {
    if (why) *why = "at most 16 q-points per batch";
    return cudaErrorInvalidValue;
  }
  if (!resolve_encoder(why)) return cudaErrorNotSupported;
  const bool bf16 = p->prec == CHI0_SPLIT_BF16;
  if (n_terms(p) == 3) {
    if (bf16) return run_tc<true, 3>(p, jobs, n_jobs, K, s, why, mode);
    return run_tc<false, 3>(p, jobs, n_jobs, K, s, why, mode);
  }
  if (bf16) return run_tc<true, 2>(p, jobs, n_jobs, K, s, why, mode);
  return run_tc<false, 2>(p, jobs, n_jobs, K, s, why, mode);
}

cudaError_t launch_contract_tc(chi0_plan_s* p, int nG, const float2* M, int64_t K, const double2* f, double2* chi,
                               cudaStream_t s, std::string* why) {
  TcJob jb{nG, M, f, chi, p->d_pack};
  return launch_contract_tc_batch(p, &jb, 1, K, s, why);
}

}  // namespace chi0
