// Plan object, argument validation, workspace and the public entry points of
// libchi0 (host side).  The arithmetic of the hot path lives in the kernels of
// the other translation units.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using chi0::SphereQ;

namespace {

thread_local std::string g_create_err;

chi0_status fail(chi0_plan_s* p, chi0_status st, const std::string& msg) {
  if (p) p->err = msg; else g_create_err = msg;
  return st;
}

#define CK(p, call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail((p), e_ == cudaErrorMemoryAllocation ? CHI0_ERR_OOM : CHI0_ERR_CUDA,  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    }                                                                                   \
  } while (0)

// exp(+2 pi i k j / n) with the phase reduced exactly in integers first.
void twiddle(int k, int j, int n, double* re, double* im) {
  long long m = ((long long)k * (long long)j) % n;
  if (m < 0) m += n;
  double ang = 2.0 * M_PI * (double)m / (double)n;
  *re = cos(ang);
  *im = sin(ang);
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// table[j][k - kmin] = exp(2 pi i k j / n), padded columns are zero
cudaError_t make_table(int n, int kmin, int nk, int nkp, double2** dd, float2** df) {
  std::vector<double2> td((size_t)n * nkp);
  std::vector<float2> tf((size_t)n * nkp);
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < nkp; ++c) {
      double re = 0.0, im = 0.0;
      if (c < nk) twiddle(kmin + c, j, n, &re, &im);
      td[(size_t)j * nkp + c] = make_double2(re, im);
      tf[(size_t)j * nkp + c] = make_float2((float)re, (float)im);
    }
  cudaError_t e = upload(dd, td);
  if (e != cudaSuccess) return e;
  return upload(df, tf);
}

// transposed table[k - kmin][j] = exp(2 pi i k j / n)
cudaError_t make_table_t(int n, int kmin, int nk, double2** dd, float2** df) {
  std::vector<double2> td((size_t)n * nk);
  std::vector<float2> tf((size_t)n * nk);
  for (int c = 0; c < nk; ++c)
    for (int j = 0; j < n; ++j) {
      double re, im;
      twiddle(kmin + c, j, n, &re, &im);
      td[(size_t)c * n + j] = make_double2(re, im);
      tf[(size_t)c * n + j] = make_float2((float)re, (float)im);
    }
  cudaError_t e = upload(dd, td);
  if (e != cudaSuccess) return e;
  return upload(df, tf);
}

void free_sphere(SphereQ& s) {
  cudaFree(s.ent_box); cudaFree(s.ent_k1); cudaFree(s.ent_j); cudaFree(s.col_off); cudaFree(s.col_start);
  cudaFree(s.T1d); cudaFree(s.T1f); cudaFree(s.T2d); cudaFree(s.T2f);
  cudaFree(s.T3d); cudaFree(s.T3f);
  s = SphereQ();
}

void free_plan(chi0_plan_s* p) {
  for (auto& v : p->prof_events)
    for (auto& e : v) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (auto e : p->prof_pool) cudaEventDestroy(e);
  for (auto& s : p->q) free_sphere(s);
  chi0::WfnSphere& w = p->w;
  cudaFree(w.col_start); cudaFree(w.col_pw); cudaFree(w.col_g1);
  cudaFree(w.T1d); cudaFree(w.T1f); cudaFree(w.T2d); cudaFree(w.T2f);
  cudaFree(w.T3d); cudaFree(w.T3f);
  cudaFree(p->d_omega); cudaFree(p->d_D); cudaFree(p->d_M); cudaFree(p->d_f);
  cudaFree(p->d_pack); cudaFree(p->d_status); cudaFree(p->d_bwd); cudaFree(p->d_inv); cudaFree(p->wfn_ws);
  for (size_t i = 1; i < p->bq_M.size(); ++i) {
    cudaFree(p->bq_M[i]);
    cudaFree(p->bq_f[i]);
    cudaFree(p->bq_pack[i]);
  }
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->pipe_M); cudaFree(p->pipe_f); cudaFree(p->pipe_pack);
  for (cudaEvent_t e : p->pipe_ev)
    if (e) cudaEventDestroy(e);
  if (p->pipe_lo) cudaStreamDestroy(p->pipe_lo);
  if (p->pipe_hi) cudaStreamDestroy(p->pipe_hi);
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

chi0_status analyse_sphere(chi0_plan_s* p, const int32_t* g, int nG, SphereQ* s) {
  int lo[3] = {g[0], g[1], g[2]}, hi[3] = {g[0], g[1], g[2]};
  for (int j = 0; j < nG; ++j)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], g[3 * j + a]);
      hi[a] = std::max(hi[a], g[3 * j + a]);
    }
  const int n[3] = {p->n1, p->n2, p->n3};
  for (int a = 0; a < 3; ++a)
    if (hi[a] - lo[a] + 1 > n[a])
      return fail(p, CHI0_ERR_INVALID, "a G sphere spans more grid points than the grid along axis " +
                                           std::to_string(a + 1));
  s->nG = nG;
  s->k1min = lo[0]; s->k2min = lo[1]; s->k3min = lo[2];
  s->nk1 = hi[0] - lo[0] + 1; s->nk2 = hi[1] - lo[1] + 1; s->nk3 = hi[2] - lo[2] + 1;
  s->nk2p = round_up(s->nk2, 4); s->nk3p = round_up(s->nk3, 4);
  std::vector<int> order(nG);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    for (int k : {1, 2, 0}) {
      if (g[3 * a + k] != g[3 * b + k]) return g[3 * a + k] < g[3 * b + k];
    }
    return false;
  });
  std::vector<int> box(nG), k1(nG), jj(nG);
  for (int t = 0; t < nG; ++t) {
    int j = order[t];
    box[t] = (g[3 * j + 1] - s->k2min) * s->nk3 + (g[3 * j + 2] - s->k3min);
    k1[t] = g[3 * j] - s->k1min;
    jj[t] = j;
  }
  // columns: runs of equal box offset in column order
  std::vector<int> col_off, col_start;
  for (int t = 0; t < nG; ++t)
    if (t == 0 || box[t] != box[t - 1]) {
      col_off.push_back(box[t]);
      col_start.push_back(t);
    }
  col_start.push_back(nG);
  s->ncol = (int)col_off.size();
  CK(p, upload(&s->ent_box, box));
  CK(p, upload(&s->ent_k1, k1));
  CK(p, upload(&s->ent_j, jj));
  CK(p, upload(&s->col_off, col_off));
  CK(p, upload(&s->col_start, col_start));
  CK(p, make_table(p->n1, s->k1min, s->nk1, s->nk1, &s->T1d, &s->T1f));
  CK(p, make_table(p->n2, s->k2min, s->nk2, s->nk2p, &s->T2d, &s->T2f));
  CK(p, make_table(p->n3, s->k3min, s->nk3, s->nk3p, &s->T3d, &s->T3f));
  return CHI0_OK;
}

chi0_status analyse_wfn(chi0_plan_s* p, const int32_t* g, int npw) {
  chi0::WfnSphere& w = p->w;
  w.npw = npw;
  if (npw <= 0 || !g) return CHI0_OK;  // wavefunction transform not configured
  int lo[3] = {g[0], g[1], g[2]}, hi[3] = {g[0], g[1], g[2]};
  for (int j = 0; j < npw; ++j)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], g[3 * j + a]);
      hi[a] = std::max(hi[a], g[3 * j + a]);
    }
  const int n[3] = {p->n1, p->n2, p->n3};
  for (int a = 0; a < 3; ++a)
    if (hi[a] - lo[a] + 1 > n[a])
      return fail(p, CHI0_ERR_INVALID, "the wavefunction sphere does not fit the grid");
  w.w1min = lo[0]; w.w2min = lo[1]; w.w3min = lo[2];
  w.nw1 = hi[0] - lo[0] + 1; w.nw2 = hi[1] - lo[1] + 1; w.nw3 = hi[2] - lo[2] + 1;
  const int ncol = w.nw2 * w.nw3;
  std::vector<int> cnt(ncol + 1, 0), start(ncol + 1, 0);
  for (int j = 0; j < npw; ++j) cnt[(g[3 * j + 1] - lo[1]) * w.nw3 + (g[3 * j + 2] - lo[2])]++;
  for (int c = 0; c < ncol; ++c) start[c + 1] = start[c] + cnt[c];
  std::vector<int> fill(start.begin(), start.end() - 1), pw(npw), g1(npw);
  for (int j = 0; j < npw; ++j) {
    int c = (g[3 * j + 1] - lo[1]) * w.nw3 + (g[3 * j + 2] - lo[2]);
    int t = fill[c]++;
    pw[t] = j;
    g1[t] = g[3 * j] - lo[0];
  }
  CK(p, upload(&w.col_start, start));
  CK(p, upload(&w.col_pw, pw));
  CK(p, upload(&w.col_g1, g1));
  CK(p, make_table(p->n1, w.w1min, w.nw1, w.nw1, &w.T1d, &w.T1f));
  CK(p, make_table(p->n2, w.w2min, w.nw2, w.nw2, &w.T2d, &w.T2f));
  CK(p, make_table_t(p->n3, w.w3min, w.nw3, &w.T3d, &w.T3f));
  return CHI0_OK;
}

bool env_fault(const char* what) {
  const char* e = getenv("CHI0_FAULT");
  return e && strcmp(e, what) == 0;
}

chi0_status check_plan(chi0_plan_s* p) {
  if (!p) return CHI0_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
    return fail(p, CHI0_ERR_INVALID, "the current device is not the plan's device");
  return CHI0_OK;
}

}  // namespace

namespace chi0 {

static cudaEvent_t pool_get(chi0_plan_s* p) {
  if (!p->prof_pool.empty()) {
    cudaEvent_t e = p->prof_pool.back();
    p->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

static const char* const kFamilyNames[CHI0_K_COUNT] = {"chi0.wfn_to_grid", "chi0.pair_planes", "chi0.pair_gather",
                                                       "chi0.weights", "chi0.pack", "chi0.contract_tc",
                                                       "chi0.contract_f64", "chi0.epsilon", "chi0.inv_panel",
                                                       "chi0.inv_update"};

ProfScope::ProfScope(chi0_plan_s* plan, int kernel, cudaStream_t st, int launches) : p(plan), k(kernel), s(st) {
  nvtxRangePushA(kFamilyNames[k]);   // host-side range around the launches (visible to nsys / ncu)
  p->prof_launches[k] += launches;
  if (p->prof_timing) {
    e1 = pool_get(p);
    if (e1) cudaEventRecord(e1, s);
  }
}

ProfScope::~ProfScope() {
  nvtxRangePop();
  if (!e1) return;
  cudaEvent_t e2 = pool_get(p);
  if (!e2) {
    p->prof_pool.push_back(e1);
    return;
  }
  cudaEventRecord(e2, s);
  p->prof_events[k].emplace_back(e1, e2);
}

bool is_split(const chi0_plan_s* p) { return p->prec != CHI0_FP64; }
void set_global_error(const std::string& msg) { g_create_err = msg; }
size_t cbytes(const chi0_plan_s* p) { return is_split(p) ? sizeof(float2) : sizeof(double2); }
}  // namespace chi0

// Automatic Hermitian mode pays where the GPU stays full: a launch of one sphere
// has n_freq T^2 work items in plain mode and n_freq T (T + 1) / 2 in Hermitian mode
// (T tiles of 128 along G), one item per SM at a time; a Hermitian item also
// carries its H2 part (taken as a quarter of an item here).  Small spheres with
// few frequencies (fewer items than SMs) run faster in plain mode.
static bool herm_pays(const chi0_plan_s* p, const chi0_plan_desc* d) {
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || n_sm < 1) n_sm = 1;
  double plain = 0.0, herm = 0.0;
  for (int i = 0; i < d->n_q; ++i) {
    const int64_t T = (d->n_G[i] + 127) / 128;
    const int64_t ip = (int64_t)d->n_freq * T * T, ih = (int64_t)d->n_freq * T * (T + 1) / 2;
    plain += (double)((ip + n_sm - 1) / n_sm);
    herm += 1.25 * (double)((ih + n_sm - 1) / n_sm);
  }
  return herm < plain;
}

extern "C" {

const char* chi0_last_error(chi0_plan plan) {
  return plan ? plan->err.c_str() : g_create_err.c_str();
}

size_t chi0_workspace_bytes(chi0_plan plan) { return plan ? plan->ws_bytes : 0; }

chi0_status chi0_plan_create(chi0_plan* out, const chi0_plan_desc* d) {
  if (!out) return fail(nullptr, CHI0_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!d) return fail(nullptr, CHI0_ERR_INVALID, "desc is NULL");
  if (d->n1 < 2 || d->n2 < 2 || d->n3 < 2 || d->n1 > 512 || d->n2 > 512 || d->n3 > 512)
    return fail(nullptr, CHI0_ERR_INVALID, "grid extents must be in [2, 512]");
  if (d->n_q < 1 || !d->n_G || !d->gvec) return fail(nullptr, CHI0_ERR_INVALID, "need n_q >= 1, n_G and gvec");
  if (d->n_freq < 1 || !d->freq_re || !d->freq_im)
    return fail(nullptr, CHI0_ERR_INVALID, "need n_freq >= 1 and frequency arrays");
  if (d->precision != CHI0_FP64 && d->precision != CHI0_SPLIT_BF16 && d->precision != CHI0_SPLIT_FP16)
    return fail(nullptr, CHI0_ERR_INVALID, "unknown precision");
  if (d->npw < 0 || (d->npw > 0 && !d->gw)) return fail(nullptr, CHI0_ERR_INVALID, "bad wavefunction sphere");
  if (d->chain_pairs < 0 || d->chain_pairs % 32 != 0)
    return fail(nullptr, CHI0_ERR_INVALID, "chain_pairs must be a non-negative multiple of 32");
  if (d->max_pairs < 0) return fail(nullptr, CHI0_ERR_INVALID, "max_pairs must be >= 0");
  if (d->n_products != 0 && d->n_products != 3 && d->n_products != 4 && d->n_products != 6)
    return fail(nullptr, CHI0_ERR_INVALID, "n_products must be 0, 3, 4 or 6");
  if (d->hermitian < -1 || d->hermitian > 1)
    return fail(nullptr, CHI0_ERR_INVALID, "hermitian must be -1, 0 or 1");
  for (int i = 0; i < d->n_q; ++i)
    if (d->n_G[i] < 1 || d->n_G[i] > 65536) return fail(nullptr, CHI0_ERR_INVALID, "n_G must be in [1, 65536]");
  if (env_fault("bad_shape")) return fail(nullptr, CHI0_ERR_INVALID, "injected fault: bad_shape");

  chi0_plan_s* p = new chi0_plan_s();
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return fail(nullptr, CHI0_ERR_CUDA, "no CUDA device");
  }
  p->n1 = d->n1; p->n2 = d->n2; p->n3 = d->n3;
  p->nr = (int64_t)d->n1 * d->n2 * d->n3;
  p->prec = d->precision;
  p->n_products = d->n_products ? d->n_products : (d->precision == CHI0_SPLIT_FP16 ? 3 : 6);
  p->delta = d->delta;
  p->n_freq = d->n_freq;
  p->om_re.assign(d->freq_re, d->freq_re + d->n_freq);
  p->om_im.assign(d->freq_im, d->freq_im + d->n_freq);
  p->chain_pairs = d->chain_pairs ? d->chain_pairs : 32;
  p->tc_herm = chi0::is_split(p) && (d->hermitian == 1 || (d->hermitian == 0 && p->n_products != 4 && herm_pays(p, d)));

  chi0_status st = CHI0_OK;
  auto bail = [&](chi0_status s) {
    g_create_err = p->err;
    free_plan(p);
    delete p;
    return s;
  };
  if (chi0::is_split(p)) {
    std::string why;
    if (!chi0::tc_supported(&why)) {
      p->err = "split precision needs the tcgen05 tensor cores of sm_103a: " + why;
      return bail(CHI0_ERR_UNSUPPORTED);
    }
  }
  {
    std::vector<double2> om(p->n_freq);
    for (int i = 0; i < p->n_freq; ++i) om[i] = make_double2(p->om_re[i], p->om_im[i]);
    cudaError_t e = upload(&p->d_omega, om);
    if (e != cudaSuccess) { p->err = cudaGetErrorString(e); return bail(CHI0_ERR_CUDA); }
  }
  int64_t off = 0;
  p->q.resize(d->n_q);
  for (int i = 0; i < d->n_q; ++i) {
    st = analyse_sphere(p, d->gvec + 3 * off, d->n_G[i], &p->q[i]);
    if (st != CHI0_OK) return bail(st);
    p->q[i].goff = off;
    p->q[i].g_host.assign(d->gvec + 3 * off, d->gvec + 3 * (off + d->n_G[i]));
    for (int j = 0; j < d->n_G[i]; ++j)
      if (d->gvec[3 * (off + j)] == 0 && d->gvec[3 * (off + j) + 1] == 0 && d->gvec[3 * (off + j) + 2] == 0) {
        p->q[i].i0 = j;
        break;
      }
    off += d->n_G[i];
    p->max_nG = std::max(p->max_nG, d->n_G[i]);
  }
  st = analyse_wfn(p, d->gw, d->npw);
  if (st != CHI0_OK) return bail(st);

  // workspace
  const size_t cb = chi0::cbytes(p);
  int64_t box = 0;
  for (auto& s : p->q) box = std::max<int64_t>(box, (int64_t)p->n1 * s.nk2 * s.nk3);
  int64_t mp = d->max_pairs ? d->max_pairs : (chi0::is_split(p) ? 8192 : 4096);
  mp = std::max<int64_t>(64, (mp + 63) / 64 * 64);
  p->max_pairs = mp;
  p->block_pairs = mp;
  // D holds the per-plane transforms of up to D_pairs pairs (at most 4 GiB): a whole pair block
  // on the 96^3 grid of the 256-atom-sized workload, so that its pair stage is one launch and each
  // valence plane is read once per block
  p->D_pairs = std::max<int64_t>(64, std::min<int64_t>(mp, ((int64_t)4 << 30) / (box * (int64_t)cb)));
  size_t bytes_D = (size_t)p->D_pairs * box * cb;
  size_t bytes_M = (size_t)mp * p->max_nG * cb;
  size_t bytes_f = (size_t)p->n_freq * mp * sizeof(double2);
  p->pack_bytes = chi0::is_split(p) ? chi0::tc_pack_bytes(p, mp, p->max_nG) : 0;
  const size_t bytes_bwd = (size_t)mp * (1 + (p->max_nG + 63) / 64) * sizeof(double);
  if (env_fault("oom")) { p->err = "injected fault: oom"; return bail(CHI0_ERR_OOM); }
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_D, bytes_D)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_M, bytes_M)) != cudaSuccess ||
      (e = cudaMalloc((void**)&p->d_f, bytes_f)) != cudaSuccess ||
      (p->pack_bytes && (e = cudaMalloc(&p->d_pack, p->pack_bytes)) != cudaSuccess) ||
      (e = cudaMalloc((void**)&p->d_status, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&p->d_bwd, bytes_bwd)) != cudaSuccess ||
      (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) {
    p->err = std::string("workspace allocation: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return bail(e == cudaErrorMemoryAllocation ? CHI0_ERR_OOM : CHI0_ERR_CUDA);
  }
  p->ws_bytes = bytes_D + bytes_M + bytes_f + p->pack_bytes + bytes_bwd + sizeof(int);
  if (chi0::is_split(p) && p->w.npw > 0 && p->n1 == 96 && p->n2 == 96 && p->n3 == 96) {
    // the 96^3 wavefunction transform runs in passes over whole lines: scratch for 128 bands
    p->wfn_ws_bytes = (size_t)128 * 96 * p->w.nw2 * p->w.nw3 * sizeof(float2);
    if ((e = cudaMalloc(&p->wfn_ws, p->wfn_ws_bytes)) != cudaSuccess) {
      p->err = std::string("workspace allocation: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return bail(e == cudaErrorMemoryAllocation ? CHI0_ERR_OOM : CHI0_ERR_CUDA);
    }
    p->ws_bytes += p->wfn_ws_bytes;
  }
  p->bq_M.assign(1, p->d_M);
  p->bq_f.assign(1, p->d_f);
  p->bq_pack.assign(1, p->d_pack);
  if (chi0::is_split(p) && d->n_q > 1) {
    for (int i = 1; i < d->n_q; ++i) {
      void *m = nullptr, *pk = nullptr;
      double2* f = nullptr;
      if ((e = cudaMalloc(&m, bytes_M)) != cudaSuccess || (e = cudaMalloc((void**)&f, bytes_f)) != cudaSuccess ||
          (e = cudaMalloc(&pk, p->pack_bytes)) != cudaSuccess) {
        cudaFree(m);
        cudaFree(f);
        cudaFree(pk);
        p->err = std::string("batched workspace allocation: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return bail(e == cudaErrorMemoryAllocation ? CHI0_ERR_OOM : CHI0_ERR_CUDA);
      }
      p->bq_M.push_back(m);
      p->bq_f.push_back(f);
      p->bq_pack.push_back(pk);
      p->ws_bytes += bytes_M + bytes_f + p->pack_bytes;
    }
  }
  if (chi0::is_split(p)) {
    const char* pe = getenv("CHI0_TC_PAIR");   // contraction variant: CTA pairs (1) or single CTAs (0)
    if (pe && *pe) p->tc_pair = atoi(pe) != 0;
    chi0::tune_apply_cached(p, 0);
  }
  *out = p;
  return CHI0_OK;
}

chi0_status chi0_plan_destroy(chi0_plan p) {
  if (!p) return CHI0_OK;
  cudaDeviceSynchronize();
  free_plan(p);
  delete p;
  return CHI0_OK;
}

chi0_status chi0_sync_status(chi0_plan p, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  CK(p, cudaStreamSynchronize(s));
  int h = 0;
  CK(p, cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(p, cudaMemset(p->d_status, 0, sizeof(int)));
  if (h & 0x100) return fail(p, CHI0_ERR_SINGULAR, "chi0_epsilon_inverse met a zero pivot");
  if (h) return fail(p, CHI0_ERR_TIMEOUT, "a bounded device-side wait ran out (status " + std::to_string(h) + ")");
  return CHI0_OK;
}

// ---------------------------------------------------------------------------
// dielectric matrix
// ---------------------------------------------------------------------------
chi0_status chi0_coulomb(chi0_plan p, int iq, const double* lattice, const double* q_frac, double* v_out) {
  if (!p) return CHI0_ERR_INVALID;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (!lattice || !q_frac || !v_out) return fail(p, CHI0_ERR_INVALID, "NULL argument");
  const double* a = lattice;   // rows a_i
  // cofactor matrix of A: cof[i][j]; det = sum_j a[0][j] cof[0][j]; inv(A)^T = cof / det
  double cof[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cof[i][j] = a[3 * i1 + j1] * a[3 * i2 + j2] - a[3 * i1 + j2] * a[3 * i2 + j1];
    }
  const double det = a[0] * cof[0][0] + a[1] * cof[0][1] + a[2] * cof[0][2];
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return fail(p, CHI0_ERR_INVALID, "singular lattice");
  double b[3][3];   // rows b_i = 2 pi (A^-T) rows
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b[i][j] = 2.0 * M_PI * cof[i][j] / det;
  const double omega_cell = std::fabs(det);
  const chi0::SphereQ& sq = p->q[iq];
  for (int jg = 0; jg < sq.nG; ++jg) {
    double k[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
      const double c = (double)sq.g_host[3 * jg + i] + q_frac[i];
      for (int x = 0; x < 3; ++x) k[x] += c * b[i][x];
    }
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (!(k2 > 0.0)) return fail(p, CHI0_ERR_INVALID, "q + G = 0 at sphere point " + std::to_string(jg));
    v_out[jg] = 4.0 * M_PI / (omega_cell * k2);
  }
  return CHI0_OK;
}

chi0_status chi0_epsilon(chi0_plan p, int iq, const void* chi, const double* v, int symmetric, void* eps,
                         void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (!chi || !v || !eps) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  if (symmetric != 0 && symmetric != 1) return fail(p, CHI0_ERR_INVALID, "symmetric must be 0 or 1");
  CK(p, chi0::launch_epsilon(p, p->q[iq].nG, (const double2*)chi, v, symmetric, (double2*)eps,
                             (cudaStream_t)stream));
  return CHI0_OK;
}

chi0_status chi0_epsilon_inverse(chi0_plan p, int iq, void* eps, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (!eps) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  const int nG = p->q[iq].nG;
  const size_t need = chi0::eps_inverse_ws_bytes(p, nG);
  if (need > p->inv_bytes) {
    CK(p, cudaStreamSynchronize((cudaStream_t)stream));
    cudaFree(p->d_inv);
    p->d_inv = nullptr;
    p->inv_bytes = 0;
    CK(p, cudaMalloc(&p->d_inv, need));
    p->inv_bytes = need;
    p->ws_bytes += need;
  }
  CK(p, chi0::launch_epsilon_inverse(p, nG, (double2*)eps, p->d_inv, (cudaStream_t)stream));
  return CHI0_OK;
}

// reciprocal lattice rows b_i = 2 pi (A^-T) rows and |det A|; false for a singular lattice
static bool recip_lattice(const double* a, double b[3][3], double* omega_cell) {
  double cof[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cof[i][j] = a[3 * i1 + j1] * a[3 * i2 + j2] - a[3 * i1 + j2] * a[3 * i2 + j1];
    }
  const double det = a[0] * cof[0][0] + a[1] * cof[0][1] + a[2] * cof[0][2];
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b[i][j] = 2.0 * M_PI * cof[i][j] / det;
  *omega_cell = std::fabs(det);
  return true;
}

chi0_status chi0_gpp(chi0_plan p, int iq, const void* psi_v, int n_v, const void* eps_inv, const double* lattice,
                     const double* q_frac, double n_el, void* Omega2, void* wt, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (!psi_v || n_v < 1 || !eps_inv || !lattice || !q_frac || !Omega2 || !wt || !(n_el > 0.0))
    return fail(p, CHI0_ERR_INVALID, "bad argument");
  double b[3][3], omega_cell = 0.0;
  if (!recip_lattice(lattice, b, &omega_cell)) return fail(p, CHI0_ERR_INVALID, "singular lattice");
  const chi0::SphereQ& sq = p->q[iq];
  const int nG = sq.nG;
  // distinct differences G_i - G_j through a box index, and the (i, j) -> difference table
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int j = 0; j < nG; ++j)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], sq.g_host[3 * j + a]);
      hi[a] = std::max(hi[a], sq.g_host[3 * j + a]);
    }
  const int ext[3] = {2 * (hi[0] - lo[0]) + 1, 2 * (hi[1] - lo[1]) + 1, 2 * (hi[2] - lo[2]) + 1};
  std::vector<int> box((size_t)ext[0] * ext[1] * ext[2], -1);
  std::vector<int> dvec, idx((size_t)nG * nG);
  for (int i = 0; i < nG; ++i)
    for (int j = 0; j < nG; ++j) {
      int d[3], o[3];
      for (int a = 0; a < 3; ++a) {
        d[a] = sq.g_host[3 * i + a] - sq.g_host[3 * j + a];
        o[a] = d[a] + (hi[a] - lo[a]);
      }
      int& slot = box[((size_t)o[0] * ext[1] + o[1]) * ext[2] + o[2]];
      if (slot < 0) {
        slot = (int)(dvec.size() / 3);
        dvec.insert(dvec.end(), d, d + 3);
      }
      idx[(size_t)i * nG + j] = slot;
    }
  const int nd = (int)(dvec.size() / 3);
  std::vector<double> kvec((size_t)3 * nG);
  for (int j = 0; j < nG; ++j)
    for (int x = 0; x < 3; ++x) {
      double k = 0.0;
      for (int a = 0; a < 3; ++a) k += ((double)sq.g_host[3 * j + a] + q_frac[a]) * b[a][x];
      kvec[3 * j + x] = k;
    }
  for (int j = 0; j < nG; ++j)
    if (!(kvec[3 * j] * kvec[3 * j] + kvec[3 * j + 1] * kvec[3 * j + 1] + kvec[3 * j + 2] * kvec[3 * j + 2] > 0.0))
      return fail(p, CHI0_ERR_INVALID, "q + G = 0 at sphere point " + std::to_string(j));
  const double wp2 = 4.0 * M_PI * n_el / omega_cell;
  cudaStream_t s = (cudaStream_t)stream;
  // offsets spanned by the differences along axes 2 and 3 (the transform is pruned to them)
  const int s2 = hi[1] - lo[1], s3 = hi[2] - lo[2];
  double* dens = nullptr;
  int *d_dvec = nullptr, *d_idx = nullptr;
  double2* rho = nullptr;
  double* d_k = nullptr;
  void* ftw = nullptr;
  auto cleanup = [&]() {
    cudaFree(dens); cudaFree(d_dvec); cudaFree(d_idx); cudaFree(rho); cudaFree(d_k); cudaFree(ftw);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&ftw, chi0::density_ft_ws_bytes(p, s2, s3))) != cudaSuccess ||
      (e = cudaMalloc((void**)&dens, sizeof(double) * p->nr)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d_dvec, sizeof(int) * dvec.size())) != cudaSuccess ||
      (e = cudaMalloc((void**)&d_idx, sizeof(int) * idx.size())) != cudaSuccess ||
      (e = cudaMalloc((void**)&rho, sizeof(double2) * nd)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d_k, sizeof(double) * kvec.size())) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_dvec, dvec.data(), sizeof(int) * dvec.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_k, kvec.data(), sizeof(double) * kvec.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = chi0::launch_density(p, psi_v, n_v, dens, s)) != cudaSuccess ||
      (e = chi0::launch_density_ft(p, dens, d_dvec, nd, s2, s3, ftw, rho, s)) != cudaSuccess ||
      (e = chi0::launch_gpp(nG, (const double2*)eps_inv, rho, d_idx, d_k, wp2, (double2*)Omega2, (double2*)wt, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return fail(p, e == cudaErrorMemoryAllocation ? CHI0_ERR_OOM : CHI0_ERR_CUDA,
                std::string("chi0_gpp: ") + cudaGetErrorString(e));
  }
  cleanup();
  return CHI0_OK;
}

chi0_status chi0_sigma_coh(chi0_plan p, int iq, const void* m, int n_t, int n_b, const double* x, const double* w,
                           const void* Omega2, const void* wt, const double* v, double* sigma, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (n_t < 0 || n_b < 0 || !sigma || ((n_t > 0 && n_b > 0) && (!m || !x || !Omega2 || !wt || !v)))
    return fail(p, CHI0_ERR_INVALID, "bad argument");
  if (n_t > 65535) return fail(p, CHI0_ERR_INVALID, "at most 65535 target bands per call");
  for (int t = 0; t < 2 * n_t; ++t) sigma[t] = 0.0;
  if (n_t == 0 || n_b == 0) return CHI0_OK;
  const int nG = p->q[iq].nG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = chi0::sigma_coh_ws_bytes(p, nG, n_t);
  void* ws = nullptr;
  cudaError_t e = cudaMalloc(&ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, CHI0_ERR_OOM, "chi0_sigma_coh: workspace");
  }
  const size_t cb = chi0::is_split(p) ? sizeof(float2) : sizeof(double2);
  double2* partial = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(ws) + 2 * (size_t)nG * nG * cb);
  int tiles = 0;
  e = chi0::launch_sigma_coh(p, nG, m, n_t, n_b, x, w, (const double2*)Omega2, (const double2*)wt, v, p->delta, ws,
                             partial, &tiles, s);
  std::vector<double2> h((size_t)n_t * tiles);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), partial, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(ws);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, CHI0_ERR_CUDA, std::string("chi0_sigma_coh: ") + cudaGetErrorString(e));
  }
  for (int t = 0; t < n_t; ++t)
    for (int k = 0; k < tiles; ++k) {   // fixed order: deterministic
      sigma[2 * t] += h[(size_t)t * tiles + k].x;
      sigma[2 * t + 1] += h[(size_t)t * tiles + k].y;
    }
  return CHI0_OK;
}

chi0_status chi0_eps_inf(chi0_plan p, int iq, const void* eps_inv, double* out, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (!eps_inv || !out) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  const int i0 = p->q[iq].i0;
  if (i0 < 0) return fail(p, CHI0_ERR_INVALID, "the sphere has no G = 0");
  const size_t nG = (size_t)p->q[iq].nG;
  std::vector<double2> h((size_t)p->n_freq);
  const double2* src = (const double2*)eps_inv + (size_t)i0 * nG + i0;
  CK(p, cudaMemcpy2DAsync(h.data(), sizeof(double2), src, nG * nG * sizeof(double2), sizeof(double2),
                          (size_t)p->n_freq, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(p, cudaStreamSynchronize((cudaStream_t)stream));
  for (int w = 0; w < p->n_freq; ++w) {
    const double d = h[w].x * h[w].x + h[w].y * h[w].y;
    out[2 * w] = h[w].x / d;
    out[2 * w + 1] = -h[w].y / d;
  }
  return CHI0_OK;
}

chi0_status chi0_wfn_to_grid(chi0_plan p, const void* coeff, int nb, void* psi, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (p->w.npw <= 0) return fail(p, CHI0_ERR_INVALID, "the plan has no wavefunction sphere");
  if (nb < 0 || (nb > 0 && (!coeff || !psi))) return fail(p, CHI0_ERR_INVALID, "bad band count or NULL buffer");
  if (nb == 0) return CHI0_OK;
  chi0::ProfScope ps(p, CHI0_K_WFN, (cudaStream_t)stream, 1);
  CK(p, chi0::launch_wfn_to_grid(p, (const double2*)coeff, nb, psi, (cudaStream_t)stream));
  return CHI0_OK;
}

// Pairs of valence rows 0..n_v and conduction columns c_base..c_base+n_c (column ic of the
// index space is band c_idx[ic], or ic when c_idx is NULL); M row = iv*ld_pairs_c + (ic - c_base).
static chi0_status pairs_impl(chi0_plan p, int iq, const void* psi_v, const int32_t* v_idx, int n_v,
                              const void* psi_c, const int32_t* c_idx, int c_base, int n_c, void* M,
                              int64_t ld_pairs_c, cudaStream_t s) {
  // chunk over (v, c) so one chunk's per-plane transforms fit the D buffer
  int vchunk = (int)std::min<int64_t>(n_v, p->D_pairs);
  int cchunk = (int)std::max<int64_t>(1, std::min<int64_t>(n_c, p->D_pairs / vchunk));
  for (int v0 = 0; v0 < n_v; v0 += vchunk) {
    int nv = std::min(vchunk, n_v - v0);
    for (int c0 = 0; c0 < n_c; c0 += cchunk) {
      int nc = std::min(cchunk, n_c - c0);
      {
        chi0::ProfScope ps(p, CHI0_K_PAIR_PLANES, s, 1);
        CK(p, chi0::launch_pair_planes(p, iq, psi_v, v_idx, v0, nv, psi_c, c_idx, c_base + c0, nc, p->d_D, s));
      }
      {
        chi0::ProfScope ps(p, CHI0_K_PAIR_GATHER, s, 1);
        CK(p, chi0::launch_pair_gather(p, iq, p->d_D, nv, nc, (int64_t)v0 * ld_pairs_c + c0, ld_pairs_c, M, s));
      }
    }
  }
  return CHI0_OK;
}

chi0_status chi0_pairs(chi0_plan p, int iq, const void* psi_v, const int32_t* v_idx, int n_v,
                       const void* psi_c, const int32_t* c_idx, int n_c, void* M, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (n_v < 0 || n_c < 0) return fail(p, CHI0_ERR_INVALID, "negative band count");
  if ((int64_t)n_v * n_c == 0) return CHI0_OK;
  if (!psi_v || !psi_c || !M) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  return pairs_impl(p, iq, psi_v, v_idx, n_v, psi_c, c_idx, 0, n_c, M, n_c, (cudaStream_t)stream);
}

static chi0_status accumulate_impl(chi0_plan p, int iq, const void* M, int n_v, int n_c,
                                   const double* E_v, const double* E_col, const double* w_col,
                                   void* chi, cudaStream_t s) {
  const int nG = p->q[iq].nG;
  const int64_t np = (int64_t)n_v * n_c;
  const int64_t blk = p->block_pairs > 0 ? std::min(p->block_pairs, p->max_pairs) : p->max_pairs;
  for (int64_t p0 = 0; p0 < np; p0 += blk) {
    int64_t K = std::min<int64_t>(blk, np - p0);
    {
      chi0::ProfScope ps(p, CHI0_K_WEIGHTS, s, 1);
      CK(p, chi0::launch_weights(p, p0, K, n_c, E_v, E_col, w_col, p->d_f, s));
    }
    if (chi0::is_split(p)) {
      std::string why;
      cudaError_t e = chi0::launch_contract_tc(p, nG, (const float2*)M + p0 * nG, K, p->d_f,
                                               (double2*)chi, s, &why);
      if (e != cudaSuccess)
        return fail(p, CHI0_ERR_CUDA, "tensor-core contraction: " + why + " " + cudaGetErrorString(e));
    } else {
      chi0::ProfScope ps(p, CHI0_K_CONTRACT_F64, s, 1);
      CK(p, chi0::launch_contract_f64(p, nG, (const double2*)M + p0 * nG, K, p->d_f, (double2*)chi, s));
    }
  }
  return CHI0_OK;
}

chi0_status chi0_accumulate(chi0_plan p, int iq, const void* M, int n_v, int n_c, const double* E_v,
                            const double* E_col, const double* w_col, void* chi0, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (n_v < 0 || n_c < 0) return fail(p, CHI0_ERR_INVALID, "negative band count");
  if ((int64_t)n_v * n_c == 0) return CHI0_OK;
  if (!M || !E_v || !E_col || !chi0) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  return accumulate_impl(p, iq, M, n_v, n_c, E_v, E_col, w_col, chi0, (cudaStream_t)stream);
}

// Streams, events and the second workspace set of the pipelined build; on any
// failure the plan falls back to the serial build for good (pipe_state -1).
static bool pipe_setup(chi0_plan p) {
  if (p->pipe_state != 0) return p->pipe_state > 0;
  p->pipe_state = -1;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&p->pipe_lo, cudaStreamNonBlocking, least) != cudaSuccess ||
      cudaStreamCreateWithPriority(&p->pipe_hi, cudaStreamNonBlocking, greatest) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (cudaEvent_t& e : p->pipe_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  const size_t bytes_M = (size_t)p->max_pairs * p->max_nG * chi0::cbytes(p);
  const size_t bytes_f = (size_t)p->n_freq * p->max_pairs * sizeof(double2);
  if (cudaMalloc(&p->pipe_M, bytes_M) != cudaSuccess || cudaMalloc((void**)&p->pipe_f, bytes_f) != cudaSuccess ||
      cudaMalloc(&p->pipe_pack, p->pack_bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->pipe_M); cudaFree(p->pipe_f); cudaFree(p->pipe_pack);
    p->pipe_M = nullptr; p->pipe_f = nullptr; p->pipe_pack = nullptr;
    return false;
  }
  p->ws_bytes += bytes_M + bytes_f + p->pack_bytes;
  p->pipe_state = 1;
  return true;
}

// Split-plan build with two workspace sets: block k's pair stage, factors and
// split planes go on the low-priority stream, its contraction on the
// high-priority one, so the next block's pair stage takes the SMs the
// contraction's last wave leaves idle and never delays a contraction.  Events
// order: packing into set b after the contraction that read set b (two blocks
// earlier), and each contraction after its own packing.  Both streams join the
// caller's stream at the end, also after an error.
static chi0_status build_pipelined(chi0_plan p, int iq, const void* psi_v, int n_v, const double* E_v,
                                   const void* psi_c, const int32_t* c_idx, int n_c, const double* E_col,
                                   const double* w_col, void* chi0, cudaStream_t s, int cb) {
  cudaStream_t lo = p->pipe_lo, hi = p->pipe_hi;
  cudaEvent_t* ev = p->pipe_ev;
  const int nG = p->q[iq].nG;
  chi0_status st = CHI0_OK;
  cudaError_t e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lo, ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hi, ev[0], 0);
  std::string why;
  int k = 0;
  for (int c0 = 0; c0 < n_c && e == cudaSuccess && st == CHI0_OK; c0 += cb, ++k) {
    const int nc = std::min(cb, n_c - c0);
    const int b = k & 1;
    void* M = b ? p->pipe_M : p->d_M;
    double2* f = b ? p->pipe_f : p->d_f;
    void* pk = b ? p->pipe_pack : p->d_pack;
    const int64_t K = (int64_t)n_v * nc;
    st = pairs_impl(p, iq, psi_v, nullptr, n_v, psi_c, c_idx, c0, nc, M, nc, lo);
    if (st != CHI0_OK) break;
    {
      chi0::ProfScope ps(p, CHI0_K_WEIGHTS, lo, 1);
      e = chi0::launch_weights(p, 0, K, nc, E_v, E_col + c0, w_col ? w_col + c0 : nullptr, f, lo);
    }
    if (e == cudaSuccess && k >= 2) e = cudaStreamWaitEvent(lo, ev[3 + b], 0);
    if (e == cudaSuccess) {
      chi0::TcJob jb{nG, (const float2*)M, f, nullptr, pk};
      e = chi0::launch_contract_tc_batch(p, &jb, 1, K, lo, &why, 1);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + b], lo);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hi, ev[1 + b], 0);
    if (e == cudaSuccess) {
      chi0::TcJob jb{nG, nullptr, nullptr, (double2*)chi0, pk};
      e = chi0::launch_contract_tc_batch(p, &jb, 1, K, hi, &why, 2);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[3 + b], hi);
  }
  // join, whatever happened above
  cudaEventRecord(ev[5], lo);
  cudaStreamWaitEvent(s, ev[5], 0);
  cudaEventRecord(ev[6], hi);
  cudaStreamWaitEvent(s, ev[6], 0);
  if (st != CHI0_OK) return st;
  if (e != cudaSuccess)
    return fail(p, CHI0_ERR_CUDA, "pipelined build: " + why + " " + cudaGetErrorString(e));
  return CHI0_OK;
}

chi0_status chi0_build(chi0_plan p, int iq, const void* psi_v, int n_v, const double* E_v,
                       const void* psi_c, const int32_t* c_idx, int n_c, const double* E_col,
                       const double* w_col, void* chi0, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (n_v < 0 || n_c < 0) return fail(p, CHI0_ERR_INVALID, "negative band count");
  if ((int64_t)n_v * n_c == 0) return CHI0_OK;
  if (!psi_v || !psi_c || !E_v || !E_col || !chi0) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  if (n_v > p->max_pairs)
    return fail(p, CHI0_ERR_INVALID, "n_v exceeds the plan's pair block; raise max_pairs");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t blk = p->block_pairs > 0 ? std::min(p->block_pairs, p->max_pairs) : p->max_pairs;
  const int cb = (int)std::max<int64_t>(1, blk / n_v);
  // the pipelined build sets up streams and buffers on first use, which a stream
  // capture does not allow: a captured build stays serial
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;
  }
  if (chi0::is_split(p) && n_c > cb && cap == cudaStreamCaptureStatusNone && pipe_setup(p))
    return build_pipelined(p, iq, psi_v, n_v, E_v, psi_c, c_idx, n_c, E_col, w_col, chi0, s, cb);
  for (int c0 = 0; c0 < n_c; c0 += cb) {
    int nc = std::min(cb, n_c - c0);
    st = pairs_impl(p, iq, psi_v, nullptr, n_v, psi_c, c_idx, c0, nc, p->d_M, nc, s);
    if (st != CHI0_OK) return st;
    st = accumulate_impl(p, iq, p->d_M, n_v, nc, E_v, E_col + c0, w_col ? w_col + c0 : nullptr, chi0, s);
    if (st != CHI0_OK) return st;
  }
  return CHI0_OK;
}

chi0_status chi0_backward(chi0_plan p, int iq, const void* M, int n_v, int n_c, const double* E_v,
                          const double* E_col, const double* w_col, const void* grad_chi0, const double* diag_g,
                          void* grad_M, double* grad_Ev, double* grad_Ecol, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (iq < 0 || iq >= (int)p->q.size()) return fail(p, CHI0_ERR_INVALID, "iq out of range");
  if (n_v < 0 || n_c < 0) return fail(p, CHI0_ERR_INVALID, "negative band count");
  if ((grad_chi0 == nullptr) == (diag_g == nullptr))
    return fail(p, CHI0_ERR_INVALID, "give exactly one of grad_chi0 and diag_g");
  if (diag_g && p->n_freq > chi0::bwd_max_freq())
    return fail(p, CHI0_ERR_INVALID, "the diagonal adjoint supports at most 64 frequencies");
  if ((int64_t)n_v * n_c == 0) return CHI0_OK;
  if (!M || !E_v || !E_col || !grad_M || !grad_Ev || !grad_Ecol) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  const int nG = p->q[iq].nG;
  CK(p, cudaMemsetAsync(grad_Ev, 0, sizeof(double) * n_v, s));
  CK(p, cudaMemsetAsync(grad_Ecol, 0, sizeof(double) * n_c, s));
  const int64_t np = (int64_t)n_v * n_c;
  for (int64_t p0 = 0; p0 < np; p0 += p->max_pairs) {
    const int64_t K = std::min<int64_t>(p->max_pairs, np - p0);
    CK(p, chi0::launch_backward(p, nG, M, p0, K, n_c, E_v, E_col, w_col, (const double2*)grad_chi0, diag_g,
                                grad_M, grad_Ev, grad_Ecol, p->d_bwd, s));
  }
  return CHI0_OK;
}

chi0_status chi0_energy_substitution_estimate(chi0_plan p, const double* E_c, const double* grad_Ecol, int n_c,
                                              int N0, double dE, double E_max, double* E_sub, double* estimate,
                                              void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (n_c < 0 || N0 < 0 || !(dE > 0.0)) return fail(p, CHI0_ERR_INVALID, "need n_c >= 0, N0 >= 0 and dE > 0");
  if (!estimate) return fail(p, CHI0_ERR_INVALID, "estimate is NULL");
  *estimate = 0.0;
  if (n_c == 0) return CHI0_OK;
  if (!E_c || !grad_Ecol) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  CK(p, chi0::launch_energy_substitution(E_c, grad_Ecol, n_c, std::min(N0, n_c), dE, E_max, E_sub, p->d_bwd, s));
  CK(p, cudaMemcpyAsync(estimate, p->d_bwd, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(p, cudaStreamSynchronize(s));
  return CHI0_OK;
}

chi0_status chi0_selftest_wait(chi0_plan p, double budget_ms, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  if (!(budget_ms > 0.0) || budget_ms > 1000.0) return fail(p, CHI0_ERR_INVALID, "budget_ms must be in (0, 1000]");
  CK(p, chi0::launch_wait_selftest(p, budget_ms, (cudaStream_t)stream));
  return CHI0_OK;
}

chi0_status chi0_profile_enable(chi0_plan p, int timing_on) {
  if (!p) return CHI0_ERR_INVALID;
  p->prof_timing = timing_on != 0;
  return CHI0_OK;
}

chi0_status chi0_profile_reset(chi0_plan p) {
  if (!p) return CHI0_ERR_INVALID;
  for (int k = 0; k < CHI0_K_COUNT; ++k) {
    for (auto& e : p->prof_events[k]) {
      cudaEventSynchronize(e.second);
      p->prof_pool.push_back(e.first);
      p->prof_pool.push_back(e.second);
    }
    p->prof_events[k].clear();
    p->prof_launches[k] = 0;
  }
  return CHI0_OK;
}

chi0_status chi0_profile_read(chi0_plan p, double* total_ms, int64_t* launches) {
  if (!p) return CHI0_ERR_INVALID;
  for (int k = 0; k < CHI0_K_COUNT; ++k) {
    double t = 0.0;
    for (auto& e : p->prof_events[k]) {
      if (cudaEventSynchronize(e.second) != cudaSuccess)
        return fail(p, CHI0_ERR_CUDA, "profiling event failed");
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) t += ms;
      cudaGetLastError();
    }
    if (total_ms) total_ms[k] = t;
    if (launches) launches[k] = p->prof_launches[k];
  }
  return CHI0_OK;
}

// enqueue the batched build of every q-point of the plan on stream s
static chi0_status build_batched_enqueue(chi0_plan p, const void* const* psi_v, int n_v, const double* const* E_v,
                                         const void* psi_c, const int32_t* c_idx, int n_c, const double* E_col,
                                         const double* w_col, void* const* chi, cudaStream_t s) {
  const int nq = (int)p->q.size();
  const int64_t blk = p->block_pairs > 0 ? std::min(p->block_pairs, p->max_pairs) : p->max_pairs;
  const int cb = (int)std::max<int64_t>(1, blk / n_v);
  for (int c0 = 0; c0 < n_c; c0 += cb) {
    const int nc = std::min(cb, n_c - c0);
    const int64_t K = (int64_t)n_v * nc;
    if (!chi0::is_split(p)) {
      for (int q = 0; q < nq; ++q) {
        chi0_status st = pairs_impl(p, q, psi_v[q], nullptr, n_v, psi_c, c_idx, c0, nc, p->d_M, nc, s);
        if (st != CHI0_OK) return st;
        st = accumulate_impl(p, q, p->d_M, n_v, nc, E_v[q], E_col + c0, w_col ? w_col + c0 : nullptr, chi[q], s);
        if (st != CHI0_OK) return st;
      }
      continue;
    }
    std::vector<chi0::TcJob> jobs(nq);
    for (int q = 0; q < nq; ++q) {
      chi0_status st = pairs_impl(p, q, psi_v[q], nullptr, n_v, psi_c, c_idx, c0, nc, p->bq_M[q], nc, s);
      if (st != CHI0_OK) return st;
      {
        chi0::ProfScope ps(p, CHI0_K_WEIGHTS, s, 1);
        CK(p, chi0::launch_weights(p, 0, K, nc, E_v[q], E_col + c0, w_col ? w_col + c0 : nullptr, p->bq_f[q], s));
      }
      jobs[q] = chi0::TcJob{p->q[q].nG, (const float2*)p->bq_M[q], p->bq_f[q], (double2*)chi[q], p->bq_pack[q]};
    }
    std::string why;
    cudaError_t e = chi0::launch_contract_tc_batch(p, jobs.data(), nq, K, s, &why);
    if (e != cudaSuccess) return fail(p, CHI0_ERR_CUDA, "batched contraction: " + why + " " + cudaGetErrorString(e));
  }
  return CHI0_OK;
}

chi0_status chi0_build_batched(chi0_plan p, const void* const* psi_v, int n_v, const double* const* E_v,
                               const void* psi_c, const int32_t* c_idx, int n_c, const double* E_col,
                               const double* w_col, void* const* chi, int use_graph, void* stream) {
  chi0_status st = check_plan(p);
  if (st != CHI0_OK) return st;
  const int nq = (int)p->q.size();
  if (!psi_v || !E_v || !chi) return fail(p, CHI0_ERR_INVALID, "NULL host pointer array");
  if (n_v < 0 || n_c < 0) return fail(p, CHI0_ERR_INVALID, "negative band count");
  if ((int64_t)n_v * n_c == 0) return CHI0_OK;
  if (!psi_c || !E_col) return fail(p, CHI0_ERR_INVALID, "NULL buffer");
  for (int q = 0; q < nq; ++q)
    if (!psi_v[q] || !E_v[q] || !chi[q]) return fail(p, CHI0_ERR_INVALID, "NULL buffer in a per-q array");
  if (n_v > p->max_pairs) return fail(p, CHI0_ERR_INVALID, "n_v exceeds the plan's pair block; raise max_pairs");
  if (nq > 16) return fail(p, CHI0_ERR_INVALID, "at most 16 q-points per batched build");
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return build_batched_enqueue(p, psi_v, n_v, E_v, psi_c, c_idx, n_c, E_col, w_col, chi, s);
  // graph mode: capture once per argument set on a plan-owned stream, then launch the graph on `stream`
  std::vector<const void*> key;
  for (int q = 0; q < nq; ++q) { key.push_back(psi_v[q]); key.push_back(E_v[q]); key.push_back(chi[q]); }
  key.push_back(psi_c); key.push_back(c_idx); key.push_back(E_col); key.push_back(w_col);
  key.push_back((const void*)(intptr_t)n_v); key.push_back((const void*)(intptr_t)n_c);
  if (!p->graph_exec || key != p->graph_key) {
    if (p->graph_exec) { cudaGraphExecDestroy(p->graph_exec); p->graph_exec = nullptr; }
    if (!p->cap_stream) CK(p, cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    const bool timing = p->prof_timing;
    p->prof_timing = false;    // no timing events inside the captured graph
    int64_t saved[CHI0_K_COUNT];
    for (int k = 0; k < CHI0_K_COUNT; ++k) saved[k] = p->prof_launches[k];
    CK(p, cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
    st = build_batched_enqueue(p, psi_v, n_v, E_v, psi_c, c_idx, n_c, E_col, w_col, chi, p->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    p->prof_timing = timing;
    // launches are counted when the graph runs, not when it is captured
    for (int k = 0; k < CHI0_K_COUNT; ++k) {
      p->graph_family[k] = p->prof_launches[k] - saved[k];
      p->prof_launches[k] = saved[k];
    }
    if (st != CHI0_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return fail(p, CHI0_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&p->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { p->graph_exec = nullptr; return fail(p, CHI0_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
    p->graph_key = key;
  }
  CK(p, cudaGraphLaunch(p->graph_exec, s));
  for (int k = 0; k < CHI0_K_COUNT; ++k) p->prof_launches[k] += p->graph_family[k];
  return CHI0_OK;
}

int chi0_select_accelerated(const double* E_c, int n_c, int N0, double dE, double dos_A, double dos_V0,
                            double E_max, int32_t* c_sel, double* E_sel, double* w_sel, int cap) {
  if (!E_c || n_c < 0 || N0 < 0 || !(dE > 0.0) || !c_sel || !E_sel || !w_sel || cap < 0) return -1;
  for (int i = 1; i < n_c; ++i)
    if (E_c[i] < E_c[i - 1]) return -1;
  N0 = std::min(N0, n_c);
  int n = 0;
  for (int c = 0; c < N0; ++c) {            // explicit part of Eq. 3
    if (n >= cap) return -1;
    c_sel[n] = c; E_sel[n] = E_c[c]; w_sel[n] = 1.0; ++n;
  }
  if (N0 == 0 || N0 >= n_c) return n;
  const double E0 = E_c[N0 - 1];
  const double span = E_max - E0;
  int NE = (int)ceil(span / dE - 1e-12);
  if (NE < 0) NE = 0;
  for (int i = 0; i < NE; ++i) {            // grid points of Eq. 4
    double lo = std::min(E0 + dE * i, E_max), hi = std::min(E0 + dE * (i + 1), E_max);
    double Ei = 0.5 * (lo + hi), dEi = hi - lo;
    // nearest band above N0; E_c is sorted, so bisect then compare neighbours
    int a = N0, b = n_c;                     // first index with E_c >= Ei
    while (a < b) { int m = (a + b) / 2; if (E_c[m] < Ei) a = m + 1; else b = m; }
    int best = a < n_c ? a : n_c - 1;
    if (a > N0 && (a == n_c || fabs(E_c[a - 1] - Ei) <= fabs(E_c[a] - Ei))) best = a - 1;
    // ties go to the lowest index among equal energies
    while (best > N0 && E_c[best - 1] == E_c[best]) --best;
    double g = (Ei > dos_V0) ? dos_A * sqrt(2.0 * (Ei - dos_V0)) : 0.0;
    if (n >= cap) return -1;
    c_sel[n] = best; E_sel[n] = Ei; w_sel[n] = g * dEi; ++n;
  }
  return n;
}

int chi0_grid_energies(const double* E_c, int n_c, int N0, double dE, double E_max, double* E_out) {
  if (!E_c || !E_out || n_c < 0 || N0 < 0 || !(dE > 0.0)) return -1;
  for (int c = 0; c < n_c; ++c) E_out[c] = E_c[c];
  N0 = std::min(N0, n_c);
  if (N0 == 0 || N0 >= n_c) return 0;
  const double E0 = E_c[N0 - 1];
  const int NE = (int)ceil((E_max - E0) / dE - 1e-12);
  if (NE <= 0) return 0;
  auto edge = [&](int k) { return std::min(E0 + dE * k, E_max); };   // Eq. 4 step edges
  for (int c = N0; c < n_c; ++c) {
    // the step [e_k, e_k+1) holding E_c: last k in [0, NE-1] with e_k <= E_c
    int a = 0, b = NE - 1;
    while (a < b) {
      const int m = (a + b + 1) / 2;
      if (edge(m) <= E_c[c]) a = m; else b = m - 1;
    }
    E_out[c] = 0.5 * (edge(a) + edge(a + 1));
  }
  return 0;
}

int chi0_select_quadrature(const double* E_c, int n_c, int N0, double dE, double dos_A, double dos_V0,
                           double E_max, int grid, int rule, int states, int32_t* c_sel, double* E_sel,
                           double* w_sel, int cap) {
  if (!E_c || n_c < 0 || N0 < 0 || !(dE > 0.0) || !c_sel || !E_sel || !w_sel || cap < 0) return -1;
  if (grid < 0 || grid > 1 || rule < 0 || rule > 2 || states < 1) return -1;
  for (int i = 1; i < n_c; ++i)
    if (E_c[i] < E_c[i - 1]) return -1;
  N0 = std::min(N0, n_c);
  int n = 0;
  for (int c = 0; c < N0; ++c) {            // explicit part of Eq. 3
    if (n >= cap) return -1;
    c_sel[n] = c; E_sel[n] = E_c[c]; w_sel[n] = 1.0; ++n;
  }
  if (N0 == 0 || N0 >= n_c) return n;
  const double E0 = E_c[N0 - 1];
  int NE = (int)ceil((E_max - E0) / dE - 1e-12);
  if (NE <= 0) return n;
  // bin edges: uniform steps of dE (Eq. 4), or equal counts of g(E) = A sqrt(2 (E - V0))
  std::vector<double> edge(NE + 1);
  if (grid == 0) {
    for (int k = 0; k <= NE; ++k) edge[k] = std::min(E0 + dE * k, E_max);
  } else {
    const double c3 = 2.0 * sqrt(2.0) / 3.0;   // int_V0^E g = A c3 (E - V0)^(3/2)
    const double G0 = dos_A * c3 * pow(std::max(E0 - dos_V0, 0.0), 1.5);
    const double G1 = dos_A * c3 * pow(std::max(E_max - dos_V0, 0.0), 1.5);
    for (int k = 0; k <= NE; ++k) {
      const double Gk = G0 + (G1 - G0) * (double)k / (double)NE;
      edge[k] = dos_V0 + pow(Gk / (dos_A * c3), 2.0 / 3.0);
    }
    edge[0] = E0;
    edge[NE] = E_max;
  }
  // nodes and raw weights of the composite rule (ascending)
  std::vector<double> node, raw;
  for (int k = 0; k < NE; ++k) {
    const double a = edge[k], b = edge[k + 1], h = b - a, m = 0.5 * (a + b);
    if (rule == 0) {                        // midpoint
      node.push_back(m); raw.push_back(h);
    } else if (rule == 2) {                 // two-point Gauss-Legendre
      const double d = h / (2.0 * sqrt(3.0));
      node.push_back(m - d); raw.push_back(0.5 * h);
      node.push_back(m + d); raw.push_back(0.5 * h);
    } else {                                // Simpson, shared ends merged
      if (k == 0) { node.push_back(a); raw.push_back(0.0); }
      raw.back() += h / 6.0;
      node.push_back(m); raw.push_back(4.0 * h / 6.0);
      node.push_back(b); raw.push_back(h / 6.0);
    }
  }
  const int avail = n_c - N0, take = std::min(states, avail);
  std::vector<char> used((size_t)avail);
  for (size_t k = 0; k < node.size(); ++k) {
    const double Ek = node[k];
    const double g = (Ek > dos_V0) ? dos_A * sqrt(2.0 * (Ek - dos_V0)) : 0.0;
    const double W = g * raw[k];
    std::fill(used.begin(), used.end(), 0);
    for (int t = 0; t < take; ++t) {        // next nearest band above N0 (ties: lower index)
      int best = -1;
      double bd = 0.0;
      for (int c = N0; c < n_c; ++c) {
        if (used[c - N0]) continue;
        const double d = fabs(E_c[c] - Ek);
        if (best < 0 || d < bd) { best = c; bd = d; }
      }
      used[best - N0] = 1;
      if (n >= cap) return -1;
      c_sel[n] = best; E_sel[n] = Ek; w_sel[n] = W / take; ++n;
    }
  }
  return n;
}

// |sum_c s_c (m - E_c)| over the bands c >= N0 with a <= E_c < b (<= b for the last bin)
static double bin_error_c(const double* E_c, const double* sens, int N0, int n_c, double a, double b, bool last) {
  int lo = N0, hi = n_c;                     // first band with E_c >= a
  while (lo < hi) { int m = (lo + hi) / 2; if (E_c[m] < a) lo = m + 1; else hi = m; }
  const double mid = 0.5 * (a + b);
  double acc = 0.0;
  for (int c = lo; c < n_c && (last ? E_c[c] <= b : E_c[c] < b); ++c) acc += sens[c] * (mid - E_c[c]);
  return fabs(acc);
}

int chi0_select_adaptive(const double* E_c, int n_c, int N0, const double* sens, double dE, double dos_A,
                         double dos_V0, double E_max, int n_split, int states, int32_t* c_sel, double* E_sel,
                         double* w_sel, int cap) {
  if (!E_c || !sens || n_c < 0 || N0 < 0 || !(dE > 0.0) || n_split < 0 || states < 1 || !c_sel || !E_sel ||
      !w_sel || cap < 0)
    return -1;
  for (int i = 1; i < n_c; ++i)
    if (E_c[i] < E_c[i - 1]) return -1;
  N0 = std::min(N0, n_c);
  int n = 0;
  for (int c = 0; c < N0; ++c) {            // explicit part of Eq. 3
    if (n >= cap) return -1;
    c_sel[n] = c; E_sel[n] = E_c[c]; w_sel[n] = 1.0; ++n;
  }
  if (N0 == 0 || N0 >= n_c) return n;
  const double E0 = E_c[N0 - 1];
  const int NE = (int)ceil((E_max - E0) / dE - 1e-12);
  if (NE <= 0) return n;
  std::vector<double> edge(NE + 1);
  for (int k = 0; k <= NE; ++k) edge[k] = std::min(E0 + dE * k, E_max);
  std::vector<double> err(NE);
  for (int k = 0; k < NE; ++k) err[k] = bin_error_c(E_c, sens, N0, n_c, edge[k], edge[k + 1], k == NE - 1);
  for (int t = 0; t < n_split; ++t) {       // split the bin with the largest estimate (lowest on ties)
    int kb = 0;
    for (int k = 1; k < (int)err.size(); ++k)
      if (err[k] > err[kb]) kb = k;
    const bool last = kb == (int)err.size() - 1;
    const double mid = 0.5 * (edge[kb] + edge[kb + 1]);
    edge.insert(edge.begin() + kb + 1, mid);
    err[kb] = bin_error_c(E_c, sens, N0, n_c, edge[kb], edge[kb + 1], false);
    err.insert(err.begin() + kb + 1, bin_error_c(E_c, sens, N0, n_c, edge[kb + 1], edge[kb + 2], last));
  }
  const int avail = n_c - N0, take = std::min(states, avail);
  std::vector<char> used((size_t)avail);
  for (size_t k = 0; k + 1 < edge.size(); ++k) {
    const double Ek = 0.5 * (edge[k] + edge[k + 1]), h = edge[k + 1] - edge[k];
    const double W = ((Ek > dos_V0) ? dos_A * sqrt(2.0 * (Ek - dos_V0)) : 0.0) * h;
    std::fill(used.begin(), used.end(), 0);
    for (int t = 0; t < take; ++t) {        // next nearest band above N0 (ties: lower index)
      int best = -1;
      double bd = 0.0;
      for (int c = N0; c < n_c; ++c) {
        if (used[c - N0]) continue;
        const double d = fabs(E_c[c] - Ek);
        if (best < 0 || d < bd) { best = c; bd = d; }
      }
      used[best - N0] = 1;
      if (n >= cap) return -1;
      c_sel[n] = best; E_sel[n] = Ek; w_sel[n] = W / take; ++n;
    }
  }
  return n;
}

}  // extern "C"
