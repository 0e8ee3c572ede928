#!/usr/bin/env python
"""Benchmark of the chi0 hot path on the 256-atom-MgO-sized workload.

Workload (the largest single-GPU configuration): N_v = 512 valence bands,
N_c = 20000 conduction bands, 96^3 grid, N_G = 8000 sphere vectors, one q,
omega = 0 plus 8 imaginary frequencies, delta = 1e-3 Ha.  The full build
streams 1250 conduction blocks of 16 bands (8192 pairs each) through the same
kernels, one after another; one benchmark step builds chi0 over a fixed,
seeded sample of those blocks (--c5-blocks, default 12: 192 conduction bands,
98,304 pairs) from plane-wave coefficients resident in HBM: wavefunctions of
the 512 valence and the sampled conduction bands on the 96^3 grid, pair
matrix elements on the 8000-vector sphere, FP64 frequency factors, split
precision tcgen05 contraction and FP64 merge into chi0 (9.2 GB).  The cost of
a build is linear in the conduction blocks, so the full build time is the
step time x 1250 / blocks (reported as extrapolated).

Metric: effective TFLOP/s = 8 N_G^2 N_pairs n_omega / build time (the
algorithmic work of the contraction only).  Inputs and chi0 (about 15 GB)
exceed L2, so no explicit flush is done between steps.

Legs:
  --impl ours (default): the CUDA path through the C ABI, plus
      e2e (host buffers, every step's coefficient upload and chi0 download
      inside the timed region, pipelined over two buffer sets and a copy
      stream), the plain FP64 GPU path on a sub-sample of the same blocks
      (per-pair cost, so the ratio holds for the whole build), the
      accelerated sum of Eq. 3/4 on the whole 256-atom-sized workload,
      per-kernel device times (roofline) and the FP64 oracle on host cores
      (cpu_baseline, rank 0 only); the 64-atom-sized build (N_G = 2500) with
      its dielectric, quadrature and COH studies under "c2_64atom".
  --impl reference: the FP64 oracle on host cores, one bounded sample of the
      same workload per step.
Multi-GPU: N independent replicas (the build of one q-point is one unit of
work; there is no data-path collective), max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "chi0 build time + effective TFLOP/s, mixed vs FP64 GPU path at ≤1e-6 rel error"
C5_BLOCK_BANDS = 16          # conduction bands per 8192-pair block at 512 valence bands


def c5_workload(n_blocks: int) -> str:
    return ("256-atom-MgO-sized chi0, full band sum (Eq. 1): N_v=512, N_c=20000, grid 96^3, N_G=8000, one "
            "q=(0.001,0,0) bohr^-1, omega = 0 + 8 imaginary (0.01-2 Ha), delta=1e-3 Ha; one step = "
            f"{n_blocks} of the 1250 conduction blocks of 16 bands (seeded sample, "
            f"{n_blocks * C5_BLOCK_BANDS} bands, {512 * n_blocks * C5_BLOCK_BANDS} pairs)")


def c5_sample_bands(n_c: int, n_blocks: int, seed: int) -> np.ndarray:
    """Conduction bands of a fixed, seeded sample of n_blocks blocks of 16
    consecutive bands (the build's own block structure), in ascending order."""
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(n_c // C5_BLOCK_BANDS, size=n_blocks, replace=False))
    return (pick[:, None] * C5_BLOCK_BANDS + np.arange(C5_BLOCK_BANDS)[None, :]).reshape(-1)


# ---------------------------------------------------------------------------
# distributed helpers (replicas); also exercised by the gloo tests on CPU
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend: str):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29531")
        dist.init_process_group(backend, rank=rank, world_size=world)
    return rank, world


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"chi0_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profiled_traffic(kernel_src: str, summary: str):
    """Per-launch DRAM bytes from a committed ncu summary, or None if the kernel
    source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    want = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()[:16]
    src_hash, traffic = None, None
    for line in open(path):
        if line.startswith("source_sha256_16:"):
            src_hash = line.split(":", 1)[1].strip()
        if line.startswith("traffic_bytes_per_full_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if src_hash == want else None


def algorithmic_flops(nG: int, n_pairs: int, n_freq: int) -> float:
    return 8.0 * nG * nG * n_pairs * n_freq


# ---------------------------------------------------------------------------
# the oracle on host cores (cpu_baseline / reference arm)
# ---------------------------------------------------------------------------
def h2_products(Ev, Ec, omega, delta, n_prod, block_cols=None):
    """Products of the H2 part per frequency in Hermitian mode, as the library
    decides them per block of conduction columns (block_cols columns with all
    valence bands; the mean over the blocks): with t the midrange of
    Im f / Re f over the block (when that shrinks the weights) and rho the
    bound on max|Im f - t Re f| / max|Re f|, one product (FP16 operands in both
    precisions) where rho <= 2^-11, three where rho <= 2^-6, else n_prod."""
    Ev, Ec = np.asarray(Ev), np.asarray(Ec)
    block_cols = block_cols or Ec.size
    one = 2.0 ** -11
    out = np.zeros(np.atleast_1d(omega).size)
    blocks = [Ec[c0:c0 + block_cols] for c0 in range(0, Ec.size, block_cols)]
    for blk in blocks:
        dE = (Ev[:, None] - blk[None, :]).reshape(-1)
        for iw, om in enumerate(np.atleast_1d(omega)):
            f = 0.5 * (1.0 / (dE - om + 1j * delta) + 1.0 / (dE + om + 1j * delta))
            fr, fi = np.abs(f.real).max(), np.abs(f.imag).max()
            with np.errstate(divide="ignore", invalid="ignore"):
                t = f.imag / f.real
            half = 0.5 * (t.max() - t.min()) if np.all(np.isfinite(t)) else np.inf
            gmax = half * fr * 1.0001 + fr * 1e-7 if half * fr < fi else fi
            rho = gmax / fr if fr > 0 else 0.0
            out[iw] += 1 if rho <= one else (3 if rho <= 2.0 ** -6 else n_prod)
    return out / len(blocks)


def alu_peaks():
    """Measured FP32 and FP64 FMA throughput of this GPU (chi0_peak_fma, best of
    three launches) with the SM clock sampled meanwhile."""
    import ctypes as C
    import torch
    import paper_1601_06767_gb300 as pkg
    lib = pkg.lib()
    out = {}
    with ClockSampler(torch.cuda.current_device()) as clk:
        for kind, name, iters in ((0, "fp32_tflops", 16384), (1, "fp64_tflops", 512)):
            best = 0.0
            for _ in range(4):                  # the first launch is a warm-up
                ms, fl = C.c_double(0.0), C.c_double(0.0)
                st = lib.chi0_peak_fma(kind, iters, C.byref(ms), C.byref(fl), None)
                if st != 0:
                    raise RuntimeError(lib.chi0_last_error(None))
                best = max(best, fl.value / (ms.value / 1e3) / 1e12)
            out[name] = best
    out["clocks"] = clk.summary()
    out["how"] = "chi0_peak_fma: 8 CTAs x 256 threads per SM, 8 independent FMA chains per thread, best of 3"
    return out


def run_peaks(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps({"case": "peaks", **alu_peaks()}))
    return 0


def coh_study(pkg, prob, plan, chi, psi_v, psi_c, dev, n_t=4):
    """Diagonal COH self-energy of the n_t lowest conduction bands with the
    plasmon-pole model fitted to the static eps^-1 of the benchmark's chi0 (plain form, FP32
    inverse of the split plan): pair elements <t|e^{iG.r}|b> for the valence
    bands and every conduction band (full) or the Eq. 3/4 columns
    (accelerated), then chi0_sigma_coh.  Times are CUDA events around the pair
    elements plus the sum; the accelerated result is compared with the full."""
    import torch
    A = prob.a * np.eye(3)
    v = torch.from_numpy(plan.coulomb(0, A, prob.q_frac[0])).to(dev)
    eps = plan.epsilon(0, chi, v, symmetric=False)
    plan.epsilon_inverse(0, eps)
    eps0 = eps[0].contiguous()
    del eps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Om2, wt = plan.gpp(0, psi_v, eps0, A, prob.q_frac[0], 2.0 * prob.n_v)
    e1.record()
    torch.cuda.synchronize()
    gpp_ms = e0.elapsed_time(e1)
    del eps0
    psi_t = psi_c[:n_t].contiguous()
    E_t = torch.from_numpy(prob.E_c[:n_t]).to(dev)
    Ev = torch.from_numpy(prob.E_v).to(dev)
    c_sel, E_sel, w_sel = pkg.select_accelerated(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max)
    out = {"what": "diagonal Sigma_COH(E_t) of Eq. 2 with the HL plasmon-pole model, targets: the "
                   f"{n_t} lowest conduction bands", "gpp_ms": gpp_ms}
    res = {}
    for label, cidx, Ecol, wcol in (("full", None, prob.E_c, None), ("accelerated", c_sel, E_sel, w_sel)):
        E_b = torch.cat([Ev, torch.as_tensor(Ecol, dtype=torch.float64, device=dev)])
        w_b = None if wcol is None else torch.cat([torch.ones_like(Ev), torch.from_numpy(wcol).to(dev)])
        x = (E_t[:, None] - E_b[None, :]).contiguous()
        ci = None if cidx is None else torch.from_numpy(cidx).to(dev)
        for rep in range(2):                      # the second pass is timed (first-use costs excluded)
            torch.cuda.synchronize()
            e0.record()
            m_v = plan.pairs(0, psi_t, psi_v)
            m_c = plan.pairs(0, psi_t, psi_c, c_idx=ci)
            nG = m_v.shape[-1]
            m = torch.cat([m_v.view(n_t, -1, nG), m_c.view(n_t, -1, nG)], 1).contiguous()
            del m_v, m_c
            sig = plan.sigma_coh(0, m, n_t, int(E_b.numel()), x, Om2, wt, v, w=w_b)
            e1.record()
            torch.cuda.synchronize()
            del m
        ms = e0.elapsed_time(e1)
        terms = float(n_t) * E_b.numel() * nG * nG
        res[label] = sig
        out[label] = {"bands_b": int(E_b.numel()), "ms": ms, "terms_per_s": terms / (ms / 1e3),
                      "sigma_Ha": [[round(float(z.real), 6), round(float(z.imag), 6)] for z in sig]}
        del x
    out["accelerated_rel_diff"] = float(np.max(np.abs(res["accelerated"] - res["full"]) / np.abs(res["full"])))
    return out


def quadrature_study(pkg, prob, plan, chi, psi_v, psi_c, Ev, cv, cc, dev):
    """Eq. 3 with different quadratures of its integral (same N0 and dE): build
    time and relative Frobenius distance of the static chi0 from the full sum
    (both from this GPU path).  With random synthetic wavefunctions M is not
    smooth in energy, so the distance is dominated by the sampling of M, which
    several states per node reduce."""
    import torch
    plan.wfn_to_grid(cv, out=psi_v)
    plan.wfn_to_grid(cc, out=psi_c)
    ref = chi[0]
    ref_norm = float(torch.linalg.vector_norm(ref))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for grid, rule, states in (("uniform", "midpoint", 1), ("quantile", "midpoint", 1), ("uniform", "simpson", 1),
                               ("uniform", "gauss2", 1), ("uniform", "midpoint", 4), ("quantile", "simpson", 2)):
        c_sel, E_sel, w_sel = pkg.select_quadrature(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0,
                                                    prob.E_max, grid, rule, states)
        c_idx = torch.from_numpy(c_sel).to(dev)
        Ecol, wcol = torch.from_numpy(E_sel).to(dev), torch.from_numpy(w_sel).to(dev)
        chi_q = plan.new_chi(0)
        e0.record()
        plan.build(0, psi_v, Ev, psi_c, Ecol, w_col=wcol, c_idx=c_idx, chi=chi_q)
        e1.record()
        torch.cuda.synchronize()
        plan.sync_status()
        err = float(torch.linalg.vector_norm(chi_q[0] - ref)) / ref_norm
        out.append({"grid": grid, "rule": rule, "states": states, "columns": int(c_sel.size),
                    "ms": e0.elapsed_time(e1), "rel_err_static_vs_full": err})
        del chi_q
    # adjoint-driven grid: dL/dE_c of L = sum_G Re(w_G chi0_GG(omega = 0)) from chi0_backward on a proxy
    # (8 valence bands x every conduction band), then as many splits as the uniform grid has bins
    g = torch.Generator(device="cpu").manual_seed(4)
    nv_p = 8
    M = plan.pairs(0, psi_v[:nv_p].contiguous(), psi_c)
    diag = torch.zeros((prob.omega.size, prob.gvec[0].shape[0]), dtype=torch.float64)
    diag[0] = torch.rand(prob.gvec[0].shape[0], generator=g, dtype=torch.float64)
    Ec_d = torch.from_numpy(prob.E_c).to(dev)
    t0 = time.time()
    _, _, gEc = plan.backward(0, M, nv_p, prob.n_c, Ev[:nv_p].contiguous(), Ec_d, diag_g=diag.to(dev))
    sens = gEc.cpu().numpy()
    sens_s = time.time() - t0
    del M
    n_uniform = int(np.ceil((prob.E_max - prob.E_c[prob.N0 - 1]) / prob.dE - 1e-12))
    c_sel, E_sel, w_sel = pkg.select_adaptive(prob.E_c, sens, prob.N0, prob.dE, prob.dos_A, prob.dos_V0,
                                              prob.E_max, n_uniform, 1)
    chi_q = plan.new_chi(0)
    e0.record()
    plan.build(0, psi_v, Ev, psi_c, torch.from_numpy(E_sel).to(dev), w_col=torch.from_numpy(w_sel).to(dev),
               c_idx=torch.from_numpy(c_sel).to(dev), chi=chi_q)
    e1.record()
    torch.cuda.synchronize()
    plan.sync_status()
    out.append({"grid": "adaptive (adjoint)", "rule": "midpoint", "states": 1, "columns": int(c_sel.size),
                "ms": e0.elapsed_time(e1), "sensitivity_s": sens_s,
                "rel_err_static_vs_full": float(torch.linalg.vector_norm(chi_q[0] - ref)) / ref_norm})
    del chi_q
    return out


def dielectric(args, pkg, prob, plan, chi, chi_a, dev):
    """eps = 1 - v^1/2 chi0 v^1/2, its inverse and eps_inf for the full and the
    accelerated chi0 of the benchmark workload (section II, Table III): device
    time of the inverse on the plan's path (FP32 for split plans) and on an FP64
    plan, and the oracle's (LAPACK) inverse of one matrix of the same size on
    the host cores for context."""
    import torch
    nG, nf = chi.shape[-1], chi.shape[0]
    A = prob.a * np.eye(3)
    v = torch.from_numpy(plan.coulomb(0, A, prob.q_frac[0])).to(dev)
    flops = 8.0 * nG ** 3 * nf                 # Gauss-Jordan inverse: N^3 complex MACs per matrix
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_inverse(p, src, reps):
        eps = p.epsilon(0, src, v, symmetric=True)
        p.epsilon_inverse(0, eps)              # first call allocates the workspace
        torch.cuda.synchronize()
        ts = []
        p.profile(True)
        p.profile_reset()
        for _ in range(reps):
            p.epsilon(0, src, v, symmetric=True, out=eps)
            e0.record()
            p.epsilon_inverse(0, eps)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        p.sync_status()
        prof = p.profile_read()
        p.profile(False)
        kern = {k: round(prof[k][0] / reps, 3) for k in ("epsilon", "inv_panel", "inv_update")}
        return eps, statistics.median(ts), kern

    eps, ms, kern = timed_inverse(plan, chi, 3)
    einf = plan.eps_inf(0, eps)
    del eps
    eps_a = plan.epsilon(0, chi_a, v, symmetric=True)
    plan.epsilon_inverse(0, eps_a)
    einf_a = plan.eps_inf(0, eps_a)
    del eps_a
    out = {"what": "eps = 1 - v^1/2 chi0 v^1/2 (v = 4 pi / (Omega |q+G|^2)), eps^-1 by blocked Gauss-Jordan "
                   "with partial pivoting, eps_inf = 1/[eps^-1]_00",
           "matrices": f"{nf} x {nG}^2", "ms_inverse": ms, "tflops": flops / ms / 1e9,
           "precision": "FP32 elimination (split plan)" if plan.precision != "fp64" else "FP64",
           "kernel_ms": kern,
           "eps_inf_full": [round(float(x.real), 6) for x in einf[:3]],
           "eps_inf_accelerated": [round(float(x.real), 6) for x in einf_a[:3]],
           "eps_inf_rel_diff_static": float(abs(einf_a[0] - einf[0]) / abs(einf[0]))}
    if plan.precision != "fp64" and not args.no_fp64:
        p64 = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp64", max_pairs=64)
        eps64, ms64, kern64 = timed_inverse(p64, chi, 1)
        einf64 = p64.eps_inf(0, eps64)
        out.update({"ms_inverse_fp64": ms64, "tflops_fp64": flops / ms64 / 1e9, "kernel_ms_fp64": kern64,
                    "eps_inf_fp64_vs_split_rel": float(abs(einf64[0] - einf[0]) / abs(einf64[0]))})
        del eps64, p64
    if not args.no_cpu:
        from oracle.dielectric import epsilon_inverse
        rng = np.random.default_rng(0)
        E = np.eye(nG) + 0.01 * (rng.standard_normal((nG, nG)) + 1j * rng.standard_normal((nG, nG)))
        t0 = time.time()
        epsilon_inverse(E[None])
        out["cpu_oracle_ms_one_matrix"] = (time.time() - t0) * 1e3
        out["cpu_cores"] = os.cpu_count()
    return out




def tc_tiles(nG: int, herm: bool, cta_pair: bool) -> int:
    """Output tiles (of 128 x 128 elements, 256 x 128 for CTA pairs) one
    frequency of the tensor-core contraction computes: all tiles of the padded
    sphere, or the ones on or above the diagonal in Hermitian mode."""
    rows = 256 if cta_pair else 128
    nGp = (nG + rows - 1) // rows * rows
    TM, TN = nGp // rows, nGp // 128
    return (TN // TM) * TM * (TM + 1) // 2 if herm else TM * TN


def contraction_roofline(prof, alg_flops, pairs, n_prod, n2, nG, nf, herm, cta_pair, traffic, note):
    """Roofline line of k_contract_tc from the launches timed over the region:
    frac = algorithmic flops (8 N_G^2 per pair and frequency) per launch over
    the average launch time, against the measured sustained bf16 peak (fp16
    runs at the same dense rate); the tensor-pipe figures count every MMA the
    kernel issues (split products, padded and mirrored tiles)."""
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    tc_ms, tc_n = prof["contract_tc"]
    tc_n = max(tc_n, 1)
    avg_s = tc_ms / 1e3 / tc_n
    elems = tc_tiles(nG, herm, cta_pair) * (256 if cta_pair else 128) * 128
    # per pair and frequency: products x 4 real products x 2 flops x computed elements
    prods = (np.full(nf, float(n_prod)) + (np.asarray(n2, dtype=np.float64) if herm else 0.0))
    tensor_total = float(np.sum(prods * 8.0 * elems * pairs))
    alg_launch = alg_flops / tc_n
    ach = alg_launch / avg_s / 1e12
    t_ach = tensor_total / tc_n / avg_s / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic, "kernel": "k_contract_tc", "peak_source": f"{pk_kind} bf16_tflops_sustained",
            "flops_per_launch": alg_launch, "flops_kind": "algorithmic, 8 N_G^2 per pair and frequency",
            "launches": tc_n, "avg_launch_ms": avg_s * 1e3,
            "tensor_pipe": {"flops_per_launch": tensor_total / tc_n, "achieved": t_ach, "frac": t_ach / peak,
                            "products_per_frequency": [round(float(x), 3) for x in prods],
                            "hermitian": herm, "cta_pair": bool(cta_pair)},
            "note": note}


def oracle_sample(prob, vb, cb):
    """Time the FP64 oracle on the pairs vb x cb of the workload (wavefunctions,
    pair elements, factors, contraction).  Returns (seconds, flops, chi, coefficients)."""
    from oracle import chi0_from_pairs, freq_factor, pair_elements, wfn_to_grid
    cv, cc = prob.coeff_v(0, vb), prob.coeff_c(cb)
    t0 = time.perf_counter()
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    M = pair_elements(uv, uc, prob.gvec[0], prob.n)
    dE = (prob.E_v[vb][:, None] - prob.E_c[cb][None, :]).reshape(-1)
    chi = chi0_from_pairs(M, freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta))
    dt = time.perf_counter() - t0
    nG = prob.gvec[0].shape[0]
    return dt, algorithmic_flops(nG, vb.size * cb.size, prob.omega.size), chi, (cv, cc)


REF_NV, REF_NC = 2, 8          # pairs per step of the reference arm (256-atom-sized workload)


def run_reference(args):
    from synth import make_problem
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    prob = make_problem("c5")
    bands = c5_sample_bands(prob.n_c, args.c5_blocks, prob.seed + 5)

    def sample(k):
        vb = (np.arange(REF_NV) * 97 + 13 * k) % prob.n_v
        cb = bands[(np.arange(REF_NC) * 23 + 7 * k) % bands.size]
        return vb, np.sort(cb)

    for w in range(args.warmup):
        oracle_sample(prob, *sample(w))
    secs, flops = 0.0, 0.0
    for k in range(args.steps):
        dt, fl, chi, _ = oracle_sample(prob, *sample(args.warmup + k))
        del chi
        secs += dt
        flops += fl
    value = flops / secs / 1e12
    cores = os.cpu_count()
    desc = f"{REF_NV} valence x {REF_NC} conduction bands of the benchmark's sampled blocks per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": c5_workload(args.c5_blocks),
                                            "sample_per_step": f"{REF_NV}x{REF_NC} pairs"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_1601_06767_gb300 as pkg
    from synth import make_problem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist_init("nccl")
    prob = make_problem("c5")
    nG, nf = prob.gvec[0].shape[0], prob.omega.size
    bands = c5_sample_bands(prob.n_c, args.c5_blocks, prob.seed + 5)
    n_pairs = prob.n_v * bands.size
    F = algorithmic_flops(nG, n_pairs, nf)

    t0 = time.time()
    cv_h = _threaded_coeff(prob, 1, np.arange(prob.n_v))
    cc_h = _threaded_coeff(prob, 0, bands)
    gen_s = time.time() - t0
    Ev_h = torch.from_numpy(prob.E_v).pin_memory()
    Ec_h = torch.from_numpy(prob.E_c[bands].copy()).pin_memory()
    cv, cc = cv_h.to(dev), cc_h.to(dev)
    Ev, Ec = Ev_h.to(dev), Ec_h.to(dev)

    herm = {"auto": None, "on": True, "off": False}[args.hermitian]
    plan = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=args.precision, gw=prob.gw,
                        n_products=args.n_products, hermitian=herm)
    tuning = plan.autotune(0)
    psi_v = torch.empty((prob.n_v,) + plan.n, dtype=plan.cdtype, device=dev)
    psi_c = torch.empty((bands.size,) + plan.n, dtype=plan.cdtype, device=dev)
    chi = plan.new_chi(0)

    def step():
        plan.wfn_to_grid(cv, out=psi_v)
        plan.wfn_to_grid(cc, out=psi_c)
        chi.zero_()
        plan.build(0, psi_v, Ev, psi_c, Ec, chi=chi)

    for _ in range(args.warmup):
        step()
    plan.sync_status()
    torch.cuda.synchronize()
    plan.profile(True)
    plan.profile_reset()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dev)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    barrier(dev)
    ms_step = ev0.elapsed_time(ev1) / args.steps
    plan.sync_status()
    prof = plan.profile_read()
    plan.profile(False)
    secs_max = max_over_ranks(ms_step / 1e3, dev)
    value = replica_value(F, world, secs_max) / 1e12
    launches = sum(c for _, c in prof.values())

    # ---- e2e: host buffers, every step's copies inside the timed region ----
    # Through the public API with inputs and chi0 double-buffered and the copies
    # on a second stream: step i+1's upload and step i's chi0 download overlap
    # the neighbouring builds; the region runs from the first upload to the
    # last download, over as many steps as the timed region.
    chi_h = [torch.empty(chi.shape, dtype=chi.dtype).pin_memory() for _ in range(2)]
    ins = [(cv, cc, Ev, Ec), tuple(torch.empty_like(t) for t in (cv, cc, Ev, Ec))]
    chis = [chi, torch.empty_like(chi)]
    cs = torch.cuda.Stream()
    comp = torch.cuda.current_stream()

    def run_e2e(n):
        up = [torch.cuda.Event() for _ in range(n)]
        done = [torch.cuda.Event() for _ in range(n)]
        for i in range(min(2, n)):                     # first two uploads
            with torch.cuda.stream(cs):
                for d, h in zip(ins[i], (cv_h, cc_h, Ev_h, Ec_h)):
                    d.copy_(h, non_blocking=True)
                up[i].record(cs)
        for i in range(n):
            b = i % 2
            comp.wait_event(up[i])
            icv, icc, iEv, iEc = ins[b]
            plan.wfn_to_grid(icv, out=psi_v)
            plan.wfn_to_grid(icc, out=psi_c)
            chis[b].zero_()
            plan.build(0, psi_v, iEv, psi_c, iEc, chi=chis[b])
            done[i].record(comp)
            with torch.cuda.stream(cs):
                cs.wait_event(done[i])
                chi_h[b].copy_(chis[b], non_blocking=True)
                if i + 2 < n:                           # the buffers of step i are free again
                    for d, h in zip(ins[b], (cv_h, cc_h, Ev_h, Ec_h)):
                        d.copy_(h, non_blocking=True)
                    up[i + 2].record(cs)
        comp.wait_stream(cs)

    run_e2e(1)
    torch.cuda.synchronize()
    barrier(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run_e2e(args.steps)
    e1.record()
    torch.cuda.synchronize()
    plan.sync_status()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / args.steps / 1e3, dev)
    h2d = cv_h.nbytes + cc_h.nbytes + Ev_h.nbytes + Ec_h.nbytes
    d2h = chi_h[0].nbytes
    last = (args.steps - 1) % 2
    assert torch.equal(chi_h[last], chis[last].cpu())     # the downloaded result is the build's chi0
    del chis[1], ins[1], chi_h

    # ---- plain FP64 GPU path on a sub-sample of the same blocks ----
    fp64 = None
    if not args.no_fp64:
        plan64 = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp64", gw=prob.gw,
                              max_pairs=1024)
        nc_s = args.fp64_sample
        psi_v64 = plan64.wfn_to_grid(cv)
        cc64 = cc[:nc_s].contiguous()
        psi_c64 = plan64.wfn_to_grid(cc64)
        chi64 = plan64.new_chi(0)
        plan64.build(0, psi_v64, Ev, psi_c64, Ec[:nc_s].contiguous(), chi=chi64)     # warm-up
        torch.cuda.synchronize()
        e0.record()
        plan64.wfn_to_grid(cc64, out=psi_c64)
        chi64.zero_()
        plan64.build(0, psi_v64, Ev, psi_c64, Ec[:nc_s].contiguous(), chi=chi64)
        e1.record()
        torch.cuda.synchronize()
        plan64.sync_status()
        s_ms = e0.elapsed_time(e1)
        e0.record()
        plan64.wfn_to_grid(cv, out=psi_v64)
        e1.record()
        torch.cuda.synchronize()
        step64_s = (s_ms * bands.size / nc_s + e0.elapsed_time(e1)) / 1e3
        fp64 = {"step_s_extrapolated": step64_s, "value_tflops": F / step64_s / 1e12,
                "build_s_extrapolated": step64_s * prob.n_c / bands.size,
                "sample": f"all 512 valence x {nc_s} conduction bands of the first sampled block timed, "
                          f"scaled linearly to the step's {bands.size} bands (cost is linear in the pairs)",
                "mixed_speedup": step64_s / (ms_step / 1e3)}
        del plan64, psi_v64, psi_c64, chi64, cc64

    # ---- accelerated sum of Eq. 3/4 on the whole 256-atom-sized workload ----
    accel = None
    if not args.no_accel:
        c_sel, E_sel, w_sel = pkg.select_accelerated(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0,
                                                     prob.E_max)
        c_uniq, c_inv = np.unique(c_sel, return_inverse=True)
        cc_sel = _threaded_coeff(prob, 0, c_uniq).to(dev)
        psi_sel = plan.wfn_to_grid(cc_sel)
        c_idx = torch.from_numpy(c_inv.astype(np.int32)).to(dev)
        Ecol, wcol = torch.from_numpy(E_sel).to(dev), torch.from_numpy(w_sel).to(dev)
        chi.zero_()
        torch.cuda.synchronize()
        e0.record()
        plan.wfn_to_grid(cv, out=psi_v)
        plan.wfn_to_grid(cc_sel, out=psi_sel)
        plan.build(0, psi_v, Ev, psi_sel, Ecol, w_col=wcol, c_idx=c_idx, chi=chi)
        e1.record()
        torch.cuda.synchronize()
        plan.sync_status()
        acc_s = e0.elapsed_time(e1) / 1e3
        full_s = ms_step / 1e3 * prob.n_c / bands.size
        accel = {"build_s": acc_s, "columns": int(c_sel.size), "bands_transformed": int(c_uniq.size),
                 "pairs": prob.n_v * int(c_sel.size), "N0": prob.N0, "dE_eV": 2.0,
                 "pair_ratio": prob.n_c / c_sel.size, "speedup_vs_full_build": full_s / acc_s}
        del cc_sel, psi_sel

    # ---- roofline of the dominant kernel (tensor-core contraction) ----
    n_prod = {"fp16": 3, "bf16": 6}[args.precision] if args.n_products == 0 else args.n_products
    n2 = h2_products(prob.E_v, prob.E_c[bands], prob.omega, prob.delta, n_prod,
                     max(1, tuning["block_pairs"] // prob.n_v))
    traffic = profiled_traffic("paper_1601_06767_gb300/csrc/kern_tc.cu", f"contract_tc_c5_{args.precision}.md")
    roof = contraction_roofline(prof, F * args.steps, n_pairs * args.steps, n_prod, n2, nG, nf, plan.hermitian,
                                tuning["cta_pair"], traffic,
                                "launch durations inside the pipelined build: the last wave of each launch "
                                "shares the GPU with the next block's pair stage")
    kernel_ms = {k: round(v[0] / args.steps, 3) for k, v in prof.items()}
    full_build_s = ms_step / 1e3 * prob.n_c / bands.size

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": c5_workload(args.c5_blocks), "pairs_per_step": n_pairs, "n_freq": nf,
                       "sampled_conduction_bands": int(bands.size), "sample_fraction": bands.size / prob.n_c,
                       "full_build_s_extrapolated": full_build_s,
                       "precision": f"{args.precision} split x{n_prod} products, FP32 TMEM chains of "
                                    f"32 pairs, FP64 factors and merge"
                                    + ("; Hermitian parts H1 + i H2 on the upper triangle" if plan.hermitian else ""),
                       "l2": "no flush: resident inputs and chi0 (about 15 GB) exceed the 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "kernel_ms_per_step": kernel_ms,
            "kernel_ms_note": "CUDA-event time per kernel family; the build pipelines conduction blocks, "
                              "the pair stage, factors and packing of block k+1 running on a second stream "
                              "beside the contraction of block k, so those families' event times include "
                              "waiting for SMs and the families overlap (their sum exceeds ms_per_step)",
            "gpu_launches": launches,
            "e2e": {"value": replica_value(F, world, e2e_s) / 1e12, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
                    "steps": args.steps},
            "fp64_gpu": fp64, "accelerated": accel, "tuning": tuning, "clocks": clk.summary(),
            "input_gen_s": gen_s}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_c5(prob, plan, psi_v, Ev, bands, dev)
    line["alu_peaks"] = alu_peaks()
    del plan, chi, psi_v, psi_c, cv, cc
    torch.cuda.empty_cache()
    if not args.no_c2:
        line["c2_64atom"] = c2_study(args, pkg, dev, world)
    if rank == 0:
        print(json.dumps(line))
    return 0


def cpu_baseline_c5(prob, plan, psi_v, Ev, bands, dev, nv=4, nc=16, rows=256):
    """The oracle on host cores on a bounded sample of the workload (nv valence
    x nc conduction bands of the sampled blocks, all 9 frequencies), plus the
    GPU result on the same pairs for a parity figure (rows 0..rows-1 of chi0)."""
    import torch
    from oracle import rel_fro
    vb = np.arange(nv) * (prob.n_v // nv)
    cb = np.sort(bands[np.linspace(0, bands.size - 1, nc).round().astype(np.int64)])
    dt, fl, chi_ref, (cv, cc) = oracle_sample(prob, vb, cb)
    ref_rows = np.ascontiguousarray(chi_ref[:, :rows])
    del chi_ref
    psi_c = plan.wfn_to_grid(torch.from_numpy(cc).to(dev))
    vi = torch.from_numpy(vb.astype(np.int32)).to(dev)
    M = plan.pairs(0, psi_v, psi_c, v_idx=vi)
    chi = plan.accumulate(0, M, nv, nc, Ev[vi.long()].contiguous(), torch.from_numpy(prob.E_c[cb]).to(dev))
    got = chi[:, :rows].cpu().numpy()
    del chi, M, psi_c
    err = max(rel_fro(got[i], ref_rows[i]) for i in range(got.shape[0]))
    emax = max(float(np.max(np.abs(got[i] - ref_rows[i])) / np.max(np.abs(ref_rows[i]))) for i in range(got.shape[0]))
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{nv} valence x {nc} conduction bands ({nv * nc} pairs) of the sampled blocks, all 9 "
                      "frequencies, N_G = 8000 (wavefunctions, pair elements, factors, contraction)",
            "seconds": dt, "parity_rows": rows, "parity_rel_fro_max_over_omega": err,
            "parity_rel_max_elem_max_over_omega": emax}


def c2_study(args, pkg, dev, world):
    """The 64-atom-sized build (N_v 128, N_c 6000, 48^3, N_G 2500, 9 frequencies)
    with the studies that use its chi0: accelerated sum, dielectric matrix,
    quadrature variants, COH self-energy, the other split precision and the
    FP64 path on a sample."""
    import torch
    from synth import make_problem
    prob = make_problem("c2")
    nG, nf = prob.gvec[0].shape[0], prob.omega.size
    n_pairs = prob.n_v * prob.n_c
    F = algorithmic_flops(nG, n_pairs, nf)
    cv = _threaded_coeff(prob, 1, np.arange(prob.n_v)).to(dev)
    cc = _threaded_coeff(prob, 0, np.arange(prob.n_c)).to(dev)
    Ev, Ec = torch.from_numpy(prob.E_v).to(dev), torch.from_numpy(prob.E_c).to(dev)
    prec = args.c2_precision
    plan = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=prec, gw=prob.gw)
    tuning = plan.autotune(0)
    psi_v = torch.empty((prob.n_v,) + plan.n, dtype=plan.cdtype, device=dev)
    psi_c = torch.empty((prob.n_c,) + plan.n, dtype=plan.cdtype, device=dev)
    chi = plan.new_chi(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(plan_, chi_, steps):
        def step():
            plan_.wfn_to_grid(cv, out=psi_v)
            plan_.wfn_to_grid(cc, out=psi_c)
            chi_.zero_()
            plan_.build(0, psi_v, Ev, psi_c, Ec, chi=chi_)
        step()
        torch.cuda.synchronize()
        plan_.profile(True)
        plan_.profile_reset()
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        plan_.sync_status()
        pr = plan_.profile_read()
        plan_.profile(False)
        return e0.elapsed_time(e1) / steps, pr

    ms, prof = timed(plan, chi, args.c2_steps)
    n_prod = {"fp16": 3, "bf16": 6}[prec]
    n2 = h2_products(prob.E_v, prob.E_c, prob.omega, prob.delta, n_prod,
                     max(1, tuning["block_pairs"] // prob.n_v))
    roof = contraction_roofline(prof, F * args.c2_steps, n_pairs * args.c2_steps, n_prod, n2, nG, nf,
                                plan.hermitian, tuning["cta_pair"],
                                profiled_traffic("paper_1601_06767_gb300/csrc/kern_tc.cu", f"contract_tc_c2_{prec}.md"),
                                "inside the pipelined build")
    out = {"workload": ("64-atom-MgO-sized chi0, full band sum (Eq. 1): N_v=128, N_c=6000, grid 48^3, N_G=2500, "
                        "omega = 0 + 8 imaginary"),
           "precision": prec, "ms_per_build": ms, "value_tflops": F / (ms / 1e3) / 1e12, "steps": args.c2_steps,
           "roofline": roof, "tuning": tuning,
           "kernel_ms_per_build": {k: round(v[0] / args.c2_steps, 3) for k, v in prof.items()}}

    # accelerated sum (Eq. 3/4): transforms only the bands its columns select
    c_sel, E_sel, w_sel = pkg.select_accelerated(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max)
    c_uniq, c_inv = np.unique(c_sel, return_inverse=True)
    cc_sel = cc.index_select(0, torch.from_numpy(c_uniq.astype(np.int64)).to(dev)).contiguous()
    psi_sel = torch.empty((c_uniq.size,) + plan.n, dtype=plan.cdtype, device=dev)
    c_idx = torch.from_numpy(c_inv.astype(np.int32)).to(dev)
    Ecol, wcol = torch.from_numpy(E_sel).to(dev), torch.from_numpy(w_sel).to(dev)
    chi_a = plan.new_chi(0)

    def step_acc():
        plan.wfn_to_grid(cv, out=psi_v)
        plan.wfn_to_grid(cc_sel, out=psi_sel)
        chi_a.zero_()
        plan.build(0, psi_v, Ev, psi_sel, Ecol, w_col=wcol, c_idx=c_idx, chi=chi_a)

    step_acc()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        step_acc()
    e1.record()
    torch.cuda.synchronize()
    plan.sync_status()
    acc_ms = e0.elapsed_time(e1) / 3
    out["accelerated"] = {"ms": acc_ms, "pairs": prob.n_v * len(c_sel), "columns": len(c_sel),
                          "bands_transformed": int(c_uniq.size), "pair_ratio": prob.n_c / len(c_sel),
                          "speedup_vs_full": ms / acc_ms, "N0": prob.N0, "dE_eV": 2.0}
    if not args.no_eps:
        out["dielectric"] = dielectric(args, pkg, prob, plan, chi, chi_a, dev)
    del chi_a, psi_sel, cc_sel
    if not args.no_quad:
        out["quadrature"] = quadrature_study(pkg, prob, plan, chi, psi_v, psi_c, Ev, cv, cc, dev)
    if not args.no_coh:
        out["coh"] = coh_study(pkg, prob, plan, chi, psi_v, psi_c, dev)
    del plan
    if not args.no_variants:
        other = "fp16" if prec == "bf16" else "bf16"
        plan2 = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=other, gw=prob.gw)
        plan2.autotune(0)
        v_ms, _ = timed(plan2, chi, args.c2_steps)
        out["variants"] = {other: {"ms_per_build": v_ms, "value_tflops": F / (v_ms / 1e3) / 1e12,
                                   "hermitian": plan2.hermitian}}
        del plan2
    if not args.no_fp64:
        plan64 = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp64", gw=prob.gw)
        nc_s = 32
        idx = torch.arange(nc_s, dtype=torch.int32, device=dev)
        psi_v64 = plan64.wfn_to_grid(cv)
        psi_c64 = plan64.wfn_to_grid(cc[:nc_s].contiguous())
        chi64 = plan64.new_chi(0)
        plan64.build(0, psi_v64, Ev, psi_c64, Ec[:nc_s].contiguous(), c_idx=idx, chi=chi64)
        torch.cuda.synchronize()
        e0.record()
        plan64.wfn_to_grid(cc[:nc_s].contiguous(), out=psi_c64)
        chi64.zero_()
        plan64.build(0, psi_v64, Ev, psi_c64, Ec[:nc_s].contiguous(), c_idx=idx, chi=chi64)
        e1.record()
        torch.cuda.synchronize()
        plan64.sync_status()
        full_s = e0.elapsed_time(e1) * prob.n_c / nc_s / 1e3
        out["fp64_gpu"] = {"build_s_extrapolated": full_s, "value_tflops": F / full_s / 1e12,
                           "sample": f"all 128 valence x {nc_s} conduction bands, scaled linearly to 6000",
                           "mixed_speedup": full_s / (ms / 1e3)}
        del plan64, psi_v64, psi_c64, chi64
    del chi, psi_v, psi_c, cv, cc
    torch.cuda.empty_cache()
    return out


def run_case(args):
    """Small fixed cases for ncu captures (no JSON line): 'contract' = two
    accumulate calls of 8192 pairs on the 2500-vector sphere with 9
    frequencies; 'pairs' = two pair-element calls of 128 x 64 pairs on 48^3;
    'wfn' = two grid transforms of 512 conduction bands on 48^3;
    'eps' = two dielectric inverses of 9 matrices of the 2500-vector sphere;
    'coh' = plasmon-pole parameters and COH sums (4 targets x 663 bands);
    'contract5' / 'pairs5' = the same on the 256-atom-sized sphere (N_G 8000,
    8192 = 512 x 16 pairs per call, 96^3 grid) with omega = 0 and one imaginary
    frequency, so that a capture holds a few GB (per-launch counters scale to the
    benchmark's 9 frequencies by 9/2)."""
    import torch
    import paper_1601_06767_gb300 as pkg
    from synth import make_problem
    big = args.case in ("contract5", "pairs5", "wfn5")
    prob = make_problem("c5", n_imag=1) if big else make_problem("c2")
    nG = prob.gvec[0].shape[0]
    K, nv, nc = (8192, 512, 16) if big else (8192, 128, 64)
    if big and args.case_pairs:
        K, nc = args.case_pairs, args.case_pairs // 512
    if big:
        args.case = args.case[:-1]
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    herm = {"auto": None, "on": True, "off": False}[args.hermitian]
    with pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=args.precision, max_pairs=K,
                      gw=prob.gw, n_products=args.n_products, hermitian=herm, chain_pairs=args.chain_pairs) as plan:
        if args.case == "contract" and not args.no_tune:
            plan.autotune(0)          # the variant the benchmark runs
        if args.case == "wfn":
            nb = 256 if big else 512
            cc = torch.from_numpy(prob.coeff_c(np.arange(nb))).cuda()
            psi = torch.empty((nb,) + plan.n, dtype=plan.cdtype, device="cuda")
            plan.wfn_to_grid(cc, out=psi)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            plan.wfn_to_grid(cc, out=psi)
            ev1.record()
            torch.cuda.synchronize()
            plan.sync_status()
            print(json.dumps({"case": "wfn" + ("5" if big else ""), "bands": nb, "ms": ev0.elapsed_time(ev1)}))
            return 0
        if args.case == "coh":
            # plasmon-pole parameters and the COH sums for 4 targets x 663 bands on the 2500-vector sphere
            nb = 663
            psi_v = torch.randn(32, *plan.n, dtype=torch.complex64, device="cuda", generator=g)
            R = torch.randn(nG, nG, dtype=torch.complex128, device="cuda", generator=g) / nG
            eps0 = (torch.eye(nG, dtype=torch.complex128, device="cuda") * 0.6 - 0.05 * (R @ R.conj().T)).contiguous()
            A = prob.a * np.eye(3)
            v = torch.from_numpy(plan.coulomb(0, A, prob.q_frac[0])).cuda()
            m = (torch.randn(4 * nb, nG, dtype=torch.complex64, device="cuda", generator=g) * 0.02).contiguous()
            x = (torch.rand(4, nb, dtype=torch.float64, device="cuda", generator=g) * 4 - 2).contiguous()
            for _ in range(2):
                Om2, wt = plan.gpp(0, psi_v, eps0, A, prob.q_frac[0], 64.0)
                plan.sigma_coh(0, m, 4, nb, x, Om2, wt, v)
            plan.sync_status()
            return 0
        if args.case == "eps":
            # 9 dielectric matrices of the 2500-vector sphere from a rank-600 static-like chi0
            R = torch.randn(600, nG, dtype=torch.complex128, device="cuda", generator=g) / (2 * nG) ** 0.5
            u = torch.rand(600, dtype=torch.float64, device="cuda", generator=g) * 0.9 + 0.1
            chi1 = -(R.T * u) @ R.conj()
            chi = chi1.unsqueeze(0).repeat(prob.omega.size, 1, 1).contiguous()
            v = torch.from_numpy(plan.coulomb(0, prob.a * np.eye(3), prob.q_frac[0])).cuda()
            for _ in range(2):
                eps = plan.epsilon(0, chi, v, symmetric=True)
                plan.epsilon_inverse(0, eps)
            plan.sync_status()
            return 0
        M = torch.randn(K, nG, dtype=torch.complex64, device="cuda", generator=g) * 4e-3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if args.case == "contract":
            # the 256-atom-sized case takes a block of the benchmark's sample from mid-spectrum
            # (nc consecutive bands from the start of that block for --case-pairs)
            cols = c5_sample_bands(prob.n_c, 12, prob.seed + 5)[4 * 16] + np.arange(nc) if big else np.arange(nc)
            Ev = torch.tensor(prob.E_v[:nv], device="cuda")
            Ec = torch.tensor(prob.E_c[cols], device="cuda")
            chi = plan.new_chi(0)

            def call():
                plan.accumulate(0, M, nv, nc, Ev, Ec, chi=chi)
        else:
            psi_v = torch.randn(nv, *plan.n, dtype=torch.complex64, device="cuda", generator=g)
            psi_c = torch.randn(nc, *plan.n, dtype=torch.complex64, device="cuda", generator=g)

            def call():
                plan.pairs(0, psi_v, psi_c, out=M)
        call()
        torch.cuda.synchronize()
        plan.profile(True)
        plan.profile_reset()
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        plan.sync_status()
        prof = {k: v for k, v in plan.profile_read().items() if v[1]}
        print(json.dumps({"case": args.case + ("5" if big else ""), "pairs": K, "ms": e0.elapsed_time(e1),
                          "kernel_ms": {k: round(v[0], 3) for k, v in prof.items()},
                          "launches": {k: v[1] for k, v in prof.items()}}))
    return 0


def _threaded_coeff(prob, stream: int, bands, workers: int = 16):
    """band_coefficients for `bands`, generated by a thread pool (numpy's
    generators release the GIL while filling) into one pinned host tensor."""
    import concurrent.futures as cf
    import numpy as np
    import torch
    from synth import band_coefficients
    bands = np.asarray(bands)
    out = torch.empty((bands.size, prob.npw), dtype=torch.complex128).pin_memory()
    o = out.numpy()
    step = max(1, (bands.size + 4 * workers - 1) // (4 * workers))

    def fill(i0):
        o[i0:i0 + step] = band_coefficients(prob.seed, stream, bands[i0:i0 + step], prob.npw)

    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(fill, range(0, bands.size, step)))
    return out




def run_c3(args):
    """Batched workload: 8 q-points (shifted 2x2x2 grid, N_G 2200-2600), 32
    frequencies, 128 x 4000 bands, split FP16 x3; the whole build as one CUDA
    graph with one persistent contraction launch per conduction block."""
    import numpy as np
    import torch
    import paper_1601_06767_gb300 as pkg
    from oracle import chi0_from_pairs, freq_factor, pair_elements, rel_fro, wfn_to_grid
    from synth import make_problem

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prob = make_problem("c3")
    nGs = [g.shape[0] for g in prob.gvec]
    nf = prob.omega.size
    n_c = max(1, int(round(prob.n_c * args.c5_frac)))
    t0 = time.time()
    cc = _threaded_coeff(prob, 0, np.arange(n_c)).to(dev)
    cvs = [_threaded_coeff(prob, 1 + q, np.arange(prob.n_v)).to(dev) for q in range(prob.n_q)]
    gen_s = time.time() - t0
    plan = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp16", gw=prob.gw, max_pairs=8192)
    tune = plan.autotune(0)
    psi_c = plan.wfn_to_grid(cc)
    psi_vs = [plan.wfn_to_grid(c) for c in cvs]
    Evs = [torch.from_numpy(prob.E_v).to(dev) for _ in range(prob.n_q)]
    Ec = torch.from_numpy(prob.E_c[:n_c]).to(dev)
    chis = [plan.new_chi(q) for q in range(prob.n_q)]
    plan.build_batched(psi_vs, Evs, psi_c, Ec, chis=chis, use_graph=True)    # capture + first run
    torch.cuda.synchronize()
    plan.profile(True)
    plan.profile_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.build_batched(psi_vs, Evs, psi_c, Ec, chis=chis, use_graph=True)
    e1.record()
    torch.cuda.synchronize()
    plan.sync_status()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    F = sum(algorithmic_flops(g, prob.n_v * n_c, nf) for g in nGs)
    # parity: 2 q-points x (2 x 4) pairs, first 300 rows, vs the oracle
    vb, cb = np.arange(2), np.array([0, 1, n_c // 2, n_c - 1])
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    par = 0.0
    for q in (0, prob.n_q - 1):
        cvq, ccq = prob.coeff_v(q, vb), prob.coeff_c(cb)
        Mr = pair_elements(wfn_to_grid(cvq, prob.gw, prob.n), wfn_to_grid(ccq, prob.gw, prob.n), prob.gvec[q], prob.n)
        dE = (prob.E_v[vb][:, None] - prob.E_c[cb][None, :]).reshape(-1)
        fq = freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta)
        Mg = plan.pairs(q, plan.wfn_to_grid(d(cvq)), plan.wfn_to_grid(d(ccq)))
        cg = plan.accumulate(q, Mg, 2, 4, d(prob.E_v[vb]), d(prob.E_c[cb]))
        torch.cuda.synchronize()
        for i in (0, nf // 2, nf - 1):
            ref = (Mr[:, :300].T * fq[i][None, :]) @ Mr.conj()
            par = max(par, rel_fro(cg[i, :300].cpu().numpy(), ref))
    line = {"case": "c3", "workload": ("batched chi0: 8 q-points on a shifted 2x2x2 grid, N_G 2200-2600, "
                                         "32 frequencies, N_v=128, N_c=4000, grid 48^3, split FP16 x3, "
                                         "one CUDA graph, one persistent contraction launch per block"),
            "timed_conduction_bands": n_c, "build_s": ms / 1e3 * prob.n_c / n_c,
            "extrapolated": n_c < prob.n_c, "effective_tflops": F / (ms / 1e3) / 1e12,
            "tensor_tflops_contraction": 3 * F / (prof["contract_tc"][0] / 1e3) / 1e12 if prof["contract_tc"][0] else None,
            "kernel_ms": {k: round(v[0], 2) for k, v in prof.items()},
            "launches_per_build": sum(v[1] for v in prof.values()), "tuning": tune,
            "parity_sample_rel_fro": par, "input_gen_s": gen_s}
    print(json.dumps(line))
    return 0


def run_c4(args):
    """Adjoint workload: L = sum_G Re(w_G chi0_GG(q, 0)), N_v=64, N_c=2000, 36^3,
    N_G=1200: forward + backward of the split FP16 path vs the FP64 path, and
    central finite differences (h = 1e-6 Ha) of the FP64 path."""
    import numpy as np
    import torch
    import paper_1601_06767_gb300 as pkg
    from synth import make_problem

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prob = make_problem("c4")
    nG = prob.gvec[0].shape[0]
    wG = torch.from_numpy(np.random.default_rng(prob.seed + 4).uniform(0, 1, (1, nG))).to(dev)
    cv = _threaded_coeff(prob, 1, np.arange(prob.n_v)).to(dev)
    cc = _threaded_coeff(prob, 0, np.arange(prob.n_c)).to(dev)
    Ev = torch.from_numpy(prob.E_v).to(dev)
    Ec = torch.from_numpy(prob.E_c).to(dev)
    res = {}
    grads = {}
    for prec in ("fp16", "fp64"):
        plan = pkg.Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=prec, gw=prob.gw)
        pv, pc = plan.wfn_to_grid(cv), plan.wfn_to_grid(cc)
        M = plan.pairs(0, pv, pc)
        Mr = M.clone().requires_grad_(True)
        Evr, Ecr = Ev.clone().requires_grad_(True), Ec.clone().requires_grad_(True)
        for _ in range(2):
            L = pkg.Chi0DiagLoss.apply(Mr, Evr, Ecr, None, wG, plan, 0)
            gM, gEv, gEc = torch.autograd.grad(L, (Mr, Evr, Ecr))
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        L = pkg.Chi0DiagLoss.apply(Mr, Evr, Ecr, None, wG, plan, 0)
        e1.record()
        gM, gEv, gEc = torch.autograd.grad(L, (Mr, Evr, Ecr))
        e2.record()
        torch.cuda.synchronize()
        plan.sync_status()
        res[prec] = {"forward_ms": e0.elapsed_time(e1), "backward_ms": e1.elapsed_time(e2), "loss": float(L)}
        grads[prec] = (gM.to(torch.complex128), gEv, gEc, float(L))
        if prec == "fp64":
            h = 1e-6
            fd = []
            for idx in (0, prob.n_v // 2, prob.n_v - 1):
                e = torch.zeros_like(Ev)
                e[idx] = h
                lp = float(pkg.Chi0DiagLoss.apply(M, Ev + e, Ec, None, wG, plan, 0))
                lm = float(pkg.Chi0DiagLoss.apply(M, Ev - e, Ec, None, wG, plan, 0))
                fd.append(abs((lp - lm) / (2 * h) - float(gEv[idx])) / max(1.0, abs(float(gEv[idx]))))
            for idx in (0, prob.n_c // 2, prob.n_c - 1):
                e = torch.zeros_like(Ec)
                e[idx] = h
                lp = float(pkg.Chi0DiagLoss.apply(M, Ev, Ec + e, None, wG, plan, 0))
                lm = float(pkg.Chi0DiagLoss.apply(M, Ev, Ec - e, None, wG, plan, 0))
                fd.append(abs((lp - lm) / (2 * h) - float(gEc[idx])) / max(1.0, abs(float(gEc[idx]))))
            res["fp64"]["fd_max_rel_err"] = max(fd)
        del plan, pv, pc, M, Mr
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    g16, g64 = grads["fp16"], grads["fp64"]
    line = {"case": "c4", "workload": ("adjoint: L = sum_G Re(w_G chi0_GG(q,0)), w_G ~ U(0,1); N_v=64, N_c=2000, "
                                         "grid 36^3, N_G=1200"),
            "timing": res,
            "split_vs_fp64_rel_err": {"grad_M": rel(g16[0], g64[0]), "grad_E_v": rel(g16[1], g64[1]),
                                      "grad_E_c": rel(g16[2], g64[2]), "loss": abs(g16[3] - g64[3]) / abs(g64[3])}}
    print(json.dumps(line))
    return 0



def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16", "fp16"], default="fp16",
                    help="split precision of the headline (256-atom-sized) build")
    ap.add_argument("--n-products", type=int, default=0)
    ap.add_argument("--hermitian", choices=["auto", "on", "off"], default="auto")
    ap.add_argument("--chain-pairs", type=int, default=0,
                    help="pairs per TMEM accumulation chain (multiple of 32; 0 = the library's default)")
    ap.add_argument("--c5-blocks", type=int, default=12,
                    help="conduction blocks (16 bands, 8192 pairs) of the 256-atom-sized workload per step")
    ap.add_argument("--c2-precision", choices=["bf16", "fp16"], default="bf16",
                    help="split precision of the 64-atom-sized build")
    ap.add_argument("--c2-steps", type=int, default=3)
    ap.add_argument("--no-tune", action="store_true",
                    help="--case contract: keep the plan's default tiles (CHI0_TC_PAIR picks the variant)")
    ap.add_argument("--fp64-sample", type=int, default=2,
                    help="conduction bands of the FP64 GPU path's sample (with all 512 valence bands)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accel", action="store_true", help="skip the accelerated 256-atom-sized build")
    ap.add_argument("--no-c2", action="store_true", help="skip the 64-atom-sized build and its studies")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-eps", action="store_true", help="skip the dielectric-matrix measurement")
    ap.add_argument("--no-quad", action="store_true", help="skip the quadrature variants of Eq. 3")
    ap.add_argument("--no-coh", action="store_true", help="skip the COH self-energy measurement")
    ap.add_argument("--case", choices=["contract", "contract5", "pairs", "pairs5", "wfn", "wfn5", "eps", "coh", "c3", "c4",
                                       "peaks"],
                    default=None, help="run a small fixed case for profiling or a separate workload")
    ap.add_argument("--c5-frac", type=float, default=1.0, help="fraction of conduction bands timed in --case c3")
    ap.add_argument("--case-pairs", type=int, default=0,
                    help="--case contract5 / pairs5: pairs per call (a multiple of 512; 0 = 8192)")
    args = ap.parse_args(argv)
    if args.case == "c3":
        return run_c3(args)
    if args.case == "c4":
        return run_c4(args)
    if args.case == "peaks":
        return run_peaks(args)
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
