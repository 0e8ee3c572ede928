// Autotuner of the tensor-core contraction's launch parameters (raster group
// of the persistent work list, pairs per launch).  Candidates are timed with
// CUDA events on synthetic operands held in the plan's own workspace; the
// fastest is kept in the plan and appended to a small text cache.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <sys/types.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace chi0 {
namespace {

// deterministic operands: |M| ~ 1e-2 with pseudo-random phases, energies of a gap system
__global__ void k_fill_synthetic(float2* M, int64_t n, double* Ev, int nv, double* Ec, int nc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)(i >> 32);
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float a = (float)(h & 0xFFFF) / 65536.f - 0.5f, b = (float)(h >> 16) / 65536.f - 0.5f;
    M[i] = make_float2(0.02f * a, 0.02f * b);
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nv) Ev[t] = -0.25 + 0.25 * (t + 0.5) / nv;
  if (t < nc) Ec[t] = 0.17 + 2.0 * (t + 0.5) / nc;
}

void mkdir_one(const std::string& dir) { mkdir(dir.c_str(), 0755); }

std::string cache_path() {
  const char* e = getenv("CHI0_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/chi0_tune.txt";
}

std::string key_of(const chi0_plan_s* p, int iq) {
  int dev = 0;
  cudaDeviceProp prop;
  cudaGetDevice(&dev);
  char name[64] = "unknown";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) snprintf(name, sizeof(name), "sm%d%d", prop.major, prop.minor);
  cudaGetLastError();
  char buf[256];
  snprintf(buf, sizeof(buf), "%s nG=%d nf=%d prec=%d np=%d herm=%d maxpairs=%lld", name, p->q[iq].nG, p->n_freq,
           (int)p->prec, p->n_products, p->tc_herm ? 1 : 0, (long long)p->max_pairs);
  return buf;
}

}  // namespace

bool tune_apply_cached(chi0_plan_s* p, int iq) {
  FILE* fh = fopen(cache_path().c_str(), "r");
  if (!fh) return false;
  const std::string key = key_of(p, iq);
  char line[512];
  bool hit = false;
  while (fgets(line, sizeof(line), fh)) {
    if (strncmp(line, key.c_str(), key.size()) != 0 || line[key.size()] != ' ') continue;
    int g = 0, pr = 0;
    long long b = 0;
    if (sscanf(line + key.size(), " group=%d block=%lld pair=%d", &g, &b, &pr) == 3 && g > 0 && b > 0 &&
        b <= p->max_pairs) {
      p->tc_group = g;
      p->block_pairs = b;
      p->tc_pair = pr != 0;
      hit = true;   // the last matching line wins
    }
  }
  fclose(fh);
  return hit;
}

}  // namespace chi0

extern "C" chi0_status chi0_autotune(chi0_plan p, int iq, int flags, double* best_us_per_pair, void* stream) {
  using namespace chi0;
  if (!p) return CHI0_ERR_INVALID;
  if (iq < 0 || iq >= (int)p->q.size()) {
    p->err = "iq out of range";
    return CHI0_ERR_INVALID;
  }
  if (!is_split(p)) {
    p->err = "the autotuner covers the tensor-core contraction of split-precision plans";
    return CHI0_ERR_UNSUPPORTED;
  }
  if (!(flags & 1) && tune_apply_cached(p, iq)) {
    if (best_us_per_pair) *best_us_per_pair = -1.0;
    return CHI0_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nG = p->q[iq].nG;
  const int T = (nG + 127) / 128;
  // synthetic operands: M block in the plan's M workspace, energies in the adjoint workspace
  const int nv = 128;
  const int64_t Kmax = p->max_pairs / nv * nv;
  if (Kmax <= 0) {
    p->err = "max_pairs too small to tune";
    return CHI0_ERR_INVALID;
  }
  const int ncmax = (int)(Kmax / nv);
  double* Ev = p->d_bwd;
  double* Ec = p->d_bwd + nv;
  k_fill_synthetic<<<304, 256, 0, s>>>((float2*)p->d_M, Kmax * nG, Ev, nv, Ec, ncmax);
  double2* chi = nullptr;
  cudaError_t e = cudaMalloc((void**)&chi, sizeof(double2) * (size_t)p->n_freq * nG * nG);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->err = "autotune: cannot allocate a scratch chi0";
    return CHI0_ERR_OOM;
  }
  const bool timing = p->prof_timing;
  p->prof_timing = false;
  std::vector<int> groups = {1, 2, 4, 8, 16};
  if (T > 16) groups.push_back(T);
  std::vector<int64_t> blocks;
  for (int64_t b = 2048; b <= Kmax; b *= 2) blocks.push_back(b / nv * nv);
  if (blocks.empty() || blocks.back() != Kmax) blocks.push_back(Kmax);
  const int saved_group = p->tc_group;
  const int64_t saved_block = p->block_pairs;
  const int saved_pair = p->tc_pair;
  double best = 1e30;
  int best_g = saved_group, best_pair = saved_pair;
  int64_t best_b = saved_block;
  std::string why;
  // time one candidate: one untimed launch, then `reps` launches with an event pair each; the median
  // launch in microseconds per pair, or < 0 on failure
  constexpr int kMaxReps = 9;
  cudaEvent_t ev[kMaxReps + 1];
  for (cudaEvent_t& x : ev) cudaEventCreate(&x);
  auto time_candidate = [&](int pair, int64_t b, int g, int reps) -> double {
    reps = std::min(reps, kMaxReps);
    p->tc_pair = pair;
    p->tc_group = g;
    p->block_pairs = b;
    const int nc = (int)(b / nv);
    cudaError_t le = cudaSuccess;
    for (int rep = 0; rep <= reps && le == cudaSuccess; ++rep) {
      if (rep >= 1) cudaEventRecord(ev[rep - 1], s);
      le = launch_weights(p, 0, b, nc, Ev, Ec, nullptr, p->d_f, s);
      if (le == cudaSuccess) le = launch_contract_tc(p, nG, (const float2*)p->d_M, b, p->d_f, chi, s, &why);
    }
    cudaEventRecord(ev[reps], s);
    if (le != cudaSuccess || cudaEventSynchronize(ev[reps]) != cudaSuccess) {
      cudaGetLastError();
      return -1.0;
    }
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]);
    std::sort(t.begin(), t.end());
    const double med = reps % 2 ? t[reps / 2] : 0.5 * (t[reps / 2 - 1] + t[reps / 2]);
    return 1e3 * med / (double)b;
  };
  // pass 1: every candidate over two launches; pass 2: the three fastest again, the median of
  // nine launches each (so that repeated tuning runs pick the same candidate)
  struct Cand { double us; int pair; int64_t b; int g; };
  std::vector<Cand> cands;
  for (int pair = 0; pair < 2; ++pair)
    for (int64_t b : blocks)
      for (int g : groups) {
        const double us = time_candidate(pair, b, g, 2);
        if (us > 0.0) cands.push_back({us, pair, b, g});
      }
  std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.us < y.us; });
  for (size_t k = 0; k < cands.size() && k < 3; ++k) {
    const double us = time_candidate(cands[k].pair, cands[k].b, cands[k].g, kMaxReps);
    if (us > 0.0 && us < best) {
      best = us;
      best_g = cands[k].g;
      best_b = cands[k].b;
      best_pair = cands[k].pair;
    }
  }
  p->prof_timing = timing;
  for (cudaEvent_t& x : ev) cudaEventDestroy(x);
  cudaFree(chi);
  p->tc_group = best_g;
  p->block_pairs = best_b;
  p->tc_pair = best_pair;
  if (best_us_per_pair) *best_us_per_pair = best;
  if (best < 1e30) {
    const std::string path = cache_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) mkdir_one(path.substr(0, slash));   // one level
    FILE* fh = fopen(path.c_str(), "a");
    if (fh) {
      fprintf(fh, "%s group=%d block=%lld pair=%d us_per_pair=%.6f\n", key_of(p, iq).c_str(), best_g,
              (long long)best_b, best_pair, best);
      fclose(fh);
    }
  }
  return CHI0_OK;
}

extern "C" chi0_status chi0_plan_hermitian(chi0_plan p, int* on) {
  if (!p || !on) return CHI0_ERR_INVALID;
  *on = p->tc_herm ? 1 : 0;
  return CHI0_OK;
}

extern "C" chi0_status chi0_get_tuning(chi0_plan p, int* group, int64_t* block_pairs, int* cta_pair) {
  if (!p) return CHI0_ERR_INVALID;
  if (group) *group = p->tc_group;
  if (block_pairs) *block_pairs = p->block_pairs;
  if (cta_pair) *cta_pair = p->tc_pair;
  return CHI0_OK;
}
