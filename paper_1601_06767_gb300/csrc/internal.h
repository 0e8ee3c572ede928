// Internal declarations shared by the translation units of libchi0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/chi0.h"

namespace chi0 {

// Pruned-transform structure of one dielectric sphere (one q-point).
// Stage 1 runs along i3 and keeps k3 in [k3min, k3min+nk3); stage 2 along i2
// keeps k2 in [k2min, k2min+nk2); the kept (k2,k3) box of every plane i1 is
// stored; stage 3 runs along i1 for every sphere point.
struct SphereQ {
  int nG = 0;
  int k1min = 0, k2min = 0, k3min = 0;
  int nk1 = 0, nk2 = 0, nk3 = 0;      // kept extents
  int nk2p = 0, nk3p = 0;             // padded to a multiple of 4 (twiddle tables)
  int64_t goff = 0;                   // offset of this sphere in the concatenated list
  std::vector<int32_t> g_host;        // [nG][3] the caller's G vectors (Coulomb, G = 0 index)
  int i0 = -1;                        // index of G = 0, or -1
  // device tables, sphere points sorted by (k2, k3, k1) ("column order")
  int* ent_box = nullptr;             // [nG] (k2-k2min)*nk3 + (k3-k3min)
  int* ent_k1 = nullptr;              // [nG] k1 - k1min
  int* ent_j = nullptr;               // [nG] index of the point in the caller's order
  int ncol = 0;                       // distinct (k2, k3) columns holding sphere points
  int* col_off = nullptr;             // [ncol] (k2-k2min)*nk3 + (k3-k3min) of each column
  int* col_start = nullptr;           // [ncol + 1] first entry of each column (entries in column order)
  double2* T1d = nullptr; float2* T1f = nullptr;   // [n1][nk1]   exp(+2 pi i k1 i1/n1)
  double2* T2d = nullptr; float2* T2f = nullptr;   // [n2][nk2p]  exp(+2 pi i k2 i2/n2)
  double2* T3d = nullptr; float2* T3f = nullptr;   // [n3][nk3p]  exp(+2 pi i k3 i3/n3)
};

// Structure of the wavefunction sphere for chi0_wfn_to_grid.
struct WfnSphere {
  int npw = 0;
  int w1min = 0, w2min = 0, w3min = 0, nw1 = 0, nw2 = 0, nw3 = 0;
  int* col_start = nullptr;           // [nw2*nw3 + 1] start of each (g2,g3) column
  int* col_pw = nullptr;              // [npw] plane-wave index, column order
  int* col_g1 = nullptr;              // [npw] g1 - w1min, column order
  double2* T1d = nullptr; float2* T1f = nullptr;   // [n1][nw1]
  double2* T2d = nullptr; float2* T2f = nullptr;   // [n2][nw2]
  double2* T3d = nullptr; float2* T3f = nullptr;   // [nw3][n3] (transposed)
};

}  // namespace chi0

struct chi0_plan_s {
  int device = 0;
  int n1 = 0, n2 = 0, n3 = 0;
  int64_t nr = 0;
  chi0_precision prec = CHI0_FP64;
  int n_products = 4;
  int64_t max_pairs = 0;     // pairs per accumulate block
  int chain_pairs = 0;       // pairs per TMEM accumulation chain
  int n_freq = 0;
  double delta = 0.0;
  std::vector<double> om_re, om_im;
  double2* d_omega = nullptr;
  std::vector<chi0::SphereQ> q;
  int max_nG = 0;
  chi0::WfnSphere w;
  // workspace
  void* d_D = nullptr;       // per-plane pruned transforms, [pairs][n1][nk2][nk3] complex
  int64_t D_pairs = 0;       // capacity in pairs
  void* d_M = nullptr;       // M block used by chi0_build, [max_pairs][max_nG] complex
  double2* d_f = nullptr;    // frequency factors, [n_freq][max_pairs]
  void* d_pack = nullptr;    // split operands of the tensor-core contraction
  size_t pack_bytes = 0;
  int* d_status = nullptr;   // device status word (bit 0: a bounded wait ran out)
  // per-q workspace sets of the batched build (index 0 aliases d_M / d_f / d_pack)
  std::vector<void*> bq_M;
  std::vector<double2*> bq_f;
  std::vector<void*> bq_pack;
  // graph of the last batched build
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<const void*> graph_key;
  int64_t graph_family[CHI0_K_COUNT] = {};   // kernel launches per family inside the captured graph
  double* d_bwd = nullptr;   // adjoint work: per-pair grad dE and per-tile partial sums
  void* wfn_ws = nullptr;    // scratch of the three-pass wavefunction transform (FP32 plans on 96^3)
  size_t wfn_ws_bytes = 0;
  void* d_inv = nullptr;     // dielectric-inverse workspace (grown on demand)
  // pipelined chi0_build (split plans): the pair stage and packing of block k+1 run on a
  // low-priority stream beside the contraction of block k on a high-priority one, with a
  // second M / factor / split-plane set (allocated on first use)
  cudaStream_t pipe_lo = nullptr, pipe_hi = nullptr;
  cudaEvent_t pipe_ev[7] = {};  // fork, packed[2], contracted[2], join lo, join hi
  void* pipe_M = nullptr;
  double2* pipe_f = nullptr;
  void* pipe_pack = nullptr;
  int pipe_state = 0;           // 0 not set up, 1 ready, -1 unavailable (serial build)
  size_t inv_bytes = 0;
  size_t ws_bytes = 0;
  std::string err;
  bool tc_ready = false;     // tensor-map encoder resolved
  int tc_group = 8;          // tile-row group of the contraction's raster order
  int64_t block_pairs = 0;   // pairs per contraction launch (<= max_pairs); set by the autotuner
  int tc_ctas_per_sm = 1;    // persistent CTAs per SM
  int tc_pair = 0;           // 1: CTA-pair (cta_group::2) contraction
  bool tc_herm = false;      // contract the Hermitian parts H1, H2 on upper-triangle tiles
  // instrumentation
  bool prof_timing = false;
  int64_t prof_launches[CHI0_K_COUNT] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[CHI0_K_COUNT];
  std::vector<cudaEvent_t> prof_pool;
};

namespace chi0 {

bool is_split(const chi0_plan_s* p);
// record the text returned by chi0_last_error(NULL) on this thread
void set_global_error(const std::string& msg);

// Brackets the launches of one kernel family: counts them and, when timing
// is on, records events on the stream before and after.
struct ProfScope {
  chi0_plan_s* p;
  int k;
  cudaStream_t s;
  cudaEvent_t e1 = nullptr;
  ProfScope(chi0_plan_s* plan, int kernel, cudaStream_t st, int launches);
  ~ProfScope();
};
size_t cbytes(const chi0_plan_s* p);   // bytes of one complex element of psi / M

// ---- kernels (launchers return cudaGetLastError()) ----
cudaError_t launch_wfn_to_grid(const chi0_plan_s* p, const double2* coeff, int nb, void* psi,
                               cudaStream_t s);
// stages 1+2 for pairs (v0..v0+nv) x (c0..c0+nc) into D (local pair index iv*nc + ic)
cudaError_t launch_pair_planes(const chi0_plan_s* p, int iq, const void* psi_v, const int32_t* v_idx,
                               int v0, int nv, const void* psi_c, const int32_t* c_idx, int c0,
                               int nc, void* D, cudaStream_t s);
// stage 3: D -> M rows (v0+iv)*ldc + (c0+ic)
cudaError_t launch_pair_gather(const chi0_plan_s* p, int iq, const void* D, int nv, int nc,
                               int64_t row0, int64_t ldv, void* M, cudaStream_t s);
// frequency factors f[w][k] for pairs p0..p0+K of an (n_v x n_c) set
cudaError_t launch_weights(const chi0_plan_s* p, int64_t p0, int64_t K, int n_c, const double* E_v,
                           const double* E_col, const double* w_col, double2* f, cudaStream_t s);
cudaError_t launch_contract_f64(const chi0_plan_s* p, int nG, const double2* M, int64_t K,
                                const double2* f, double2* chi, cudaStream_t s);
// one q-point's share of a batched tensor-core contraction
struct TcJob {
  int nG;
  const float2* M;        // [K][nG]
  const double2* f;       // [n_freq][K]
  double2* chi;           // [n_freq][nG][nG]
  void* pack;             // split-plane workspace (tc_pack_bytes)
};
// mode 0: pack and contract; 1: pack only (absmax, scales, split planes into jobs[].pack);
// 2: contract only, from planes an earlier mode-1 call packed with the same K and shapes
cudaError_t launch_contract_tc_batch(chi0_plan_s* p, const TcJob* jobs, int n_jobs, int64_t K, cudaStream_t s,
                                     std::string* why, int mode = 0);
// split-precision tensor-core path for K pairs of M (float2) with factors f
cudaError_t launch_contract_tc(chi0_plan_s* p, int nG, const float2* M, int64_t K,
                               const double2* f, double2* chi, cudaStream_t s, std::string* why);
size_t tc_pack_bytes(const chi0_plan_s* p, int64_t max_pairs, int max_nG);
// adjoint of the contraction for pairs p0..p0+K (Gamma dense [n_freq][nG][nG] or diag [n_freq][nG])
cudaError_t launch_backward(chi0_plan_s* p, int nG, const void* M, int64_t p0, int64_t K, int n_c,
                            const double* E_v, const double* E_col, const double* w_col, const double2* gamma,
                            const double* diag, void* gM, double* gEv, double* gEc, double* work, cudaStream_t s);
int bwd_max_freq();
// first-order energy-substitution estimate of Eq. 3/4 (one block; writes the grid energy of every
// band to E_sub when it is not NULL and the sum to *out, both device pointers)
cudaError_t launch_energy_substitution(const double* E_c, const double* sens, int n_c, int N0, double dE, double E_max,
                                       double* E_sub, double* out, cudaStream_t s);
// autotuner: apply a cached entry for sphere iq if one exists (returns true if applied)
bool tune_apply_cached(chi0_plan_s* p, int iq);
cudaError_t launch_wait_selftest(chi0_plan_s* p, double budget_ms, cudaStream_t s);
bool tc_supported(std::string* why);
// dielectric matrix: eps = 1 - v chi0 (plain or symmetrised) and its in-place inverse
cudaError_t launch_epsilon(chi0_plan_s* p, int nG, const double2* chi, const double* v, int symmetric,
                           double2* eps, cudaStream_t s);
size_t eps_inverse_ws_bytes(const chi0_plan_s* p, int nG);
// COH self-energy with the plasmon-pole model
cudaError_t launch_density(const chi0_plan_s* p, const void* psi_v, int n_v, double* dens, cudaStream_t s);
size_t density_ft_ws_bytes(const chi0_plan_s* p, int s2, int s3);
cudaError_t launch_density_ft(const chi0_plan_s* p, const double* dens, const int* dvec, int nd, int s2, int s3,
                              void* ws, double2* rho, cudaStream_t s);
cudaError_t launch_gpp(int nG, const double2* eps_inv, const double2* rho, const int* idx, const double* kvec,
                       double wp2, double2* Om2, double2* wt, cudaStream_t s);
size_t sigma_coh_ws_bytes(const chi0_plan_s* p, int nG, int n_t);
cudaError_t launch_sigma_coh(const chi0_plan_s* p, int nG, const void* m, int n_t, int n_b, const double* x,
                             const double* w, const double2* Om2, const double2* wt, const double* v, double delta,
                             void* ws, double2* partial, int* n_tiles, cudaStream_t s);
cudaError_t launch_epsilon_inverse(chi0_plan_s* p, int nG, double2* eps, void* ws, cudaStream_t s);

}  // namespace chi0
