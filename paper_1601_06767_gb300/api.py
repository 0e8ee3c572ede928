"""Thin PyTorch binding of libchi0 (argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; PyTorch only
provides device memory and the current stream.  Names follow include/chi0.h.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Chi0Plan:
    """A chi0 plan on the current CUDA device (see chi0_plan_create)."""

    def __init__(self, n, gvecs, omega, delta: float, precision: str = "fp64", gw=None,
                 n_products: int = 0, max_pairs: int = 0, chain_pairs: int = 0,
                 hermitian: bool | None = None):
        lib = L.lib()
        n1, n2, n3 = (n, n, n) if np.isscalar(n) else tuple(int(x) for x in n)
        self.n = (n1, n2, n3)
        self.nr = n1 * n2 * n3
        self.precision = precision
        if precision not in L.PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(L.PRECISIONS)}")
        gl = [_i32(g).reshape(-1, 3) for g in gvecs]
        self.n_G = [int(g.shape[0]) for g in gl]
        om = np.atleast_1d(np.asarray(omega, dtype=np.complex128))
        self.n_freq = int(om.size)
        keep = dict(nG=_i32(self.n_G), g=np.ascontiguousarray(np.concatenate(gl, 0)),
                    re=_f64(om.real), im=_f64(om.imag),
                    gw=None if gw is None else _i32(gw).reshape(-1, 3))
        d = L.Chi0PlanDesc()
        d.n1, d.n2, d.n3 = n1, n2, n3
        d.n_q = len(gl)
        d.n_G = keep["nG"].ctypes.data_as(C.POINTER(C.c_int32))
        d.gvec = keep["g"].ctypes.data_as(C.POINTER(C.c_int32))
        d.npw = 0 if gw is None else int(keep["gw"].shape[0])
        d.gw = None if gw is None else keep["gw"].ctypes.data_as(C.POINTER(C.c_int32))
        d.n_freq = self.n_freq
        d.freq_re = keep["re"].ctypes.data_as(C.POINTER(C.c_double))
        d.freq_im = keep["im"].ctypes.data_as(C.POINTER(C.c_double))
        d.delta = float(delta)
        d.precision = L.PRECISIONS[precision]
        d.n_products = int(n_products)
        d.max_pairs = int(max_pairs)
        d.chain_pairs = int(chain_pairs)
        d.hermitian = 0 if hermitian is None else (1 if hermitian else -1)
        h = C.c_void_p()
        L.check(lib.chi0_plan_create(C.byref(h), C.byref(d)), None)
        self._h = h
        on = C.c_int(0)
        L.check(lib.chi0_plan_hermitian(h, C.byref(on)), h)
        self.hermitian = bool(on.value)   # the library's choice (split precisions only)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.cdtype = torch.complex128 if precision == "fp64" else torch.complex64

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            L.lib().chi0_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def workspace_bytes(self) -> int:
        return int(L.lib().chi0_workspace_bytes(self._h))

    def _check(self, st):
        L.check(st, self._h)

    def _c(self, t, name, dtype=None):
        dtype = dtype or self.cdtype
        if t.dtype != dtype or t.device != self.device or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor on {self.device}")
        return t

    # -- autotuner -------------------------------------------------------
    def autotune(self, iq: int = 0, force: bool = False) -> dict:
        best = C.c_double(0.0)
        self._check(L.lib().chi0_autotune(self._h, iq, int(force), C.byref(best), _stream()))
        g, b, pr = C.c_int(0), C.c_int64(0), C.c_int(0)
        self._check(L.lib().chi0_get_tuning(self._h, C.byref(g), C.byref(b), C.byref(pr)))
        return {"group": g.value, "block_pairs": b.value, "cta_pair": pr.value, "us_per_pair": best.value}

    # -- instrumentation -------------------------------------------------
    def profile(self, timing: bool = True):
        self._check(L.lib().chi0_profile_enable(self._h, int(timing)))

    def profile_reset(self):
        self._check(L.lib().chi0_profile_reset(self._h))

    def profile_read(self) -> dict:
        n = len(L.KERNELS)
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.int64)
        self._check(L.lib().chi0_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(L.KERNELS)}

    # -- entry points ----------------------------------------------------
    def sync_status(self):
        self._check(L.lib().chi0_sync_status(self._h, _stream()))

    def wfn_to_grid(self, coeff: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        coeff = self._c(coeff, "coeff", torch.complex128)
        nb = coeff.shape[0]
        if out is None:
            out = torch.empty((nb,) + self.n, dtype=self.cdtype, device=self.device)
        self._c(out, "out")
        self._check(L.lib().chi0_wfn_to_grid(self._h, _ptr(coeff), nb, _ptr(out), _stream()))
        return out

    def pairs(self, iq: int, psi_v, psi_c, v_idx=None, c_idx=None, out=None) -> torch.Tensor:
        self._c(psi_v, "psi_v")
        self._c(psi_c, "psi_c")
        n_v = psi_v.shape[0] if v_idx is None else int(v_idx.numel())
        n_c = psi_c.shape[0] if c_idx is None else int(c_idx.numel())
        for t in (v_idx, c_idx):
            if t is not None:
                self._c(t, "index", torch.int32)
        if out is None:
            out = torch.empty((n_v * n_c, self.n_G[iq]), dtype=self.cdtype, device=self.device)
        self._c(out, "out")
        self._check(L.lib().chi0_pairs(self._h, iq, _ptr(psi_v), _ptr(v_idx), n_v, _ptr(psi_c),
                                       _ptr(c_idx), n_c, _ptr(out), _stream()))
        return out

    def new_chi(self, iq: int) -> torch.Tensor:
        nG = self.n_G[iq]
        return torch.zeros((self.n_freq, nG, nG), dtype=torch.complex128, device=self.device)

    def accumulate(self, iq: int, M, n_v: int, n_c: int, E_v, E_col, w_col=None, chi=None):
        self._c(M, "M")
        for t, nm in ((E_v, "E_v"), (E_col, "E_col"), (w_col, "w_col")):
            if t is not None:
                self._c(t, nm, torch.float64)
        chi = self.new_chi(iq) if chi is None else self._c(chi, "chi", torch.complex128)
        self._check(L.lib().chi0_accumulate(self._h, iq, _ptr(M), n_v, n_c, _ptr(E_v), _ptr(E_col),
                                            _ptr(w_col), _ptr(chi), _stream()))
        return chi

    def build_batched(self, psi_vs, E_vs, psi_c, E_col, w_col=None, c_idx=None, chis=None, use_graph=True):
        """chi0_build_batched over all q-points of the plan; returns the list of chi0[q]."""
        nq = len(self.n_G)
        if len(psi_vs) != nq or len(E_vs) != nq:
            raise ValueError("one valence grid and one energy vector per q-point")
        for t in psi_vs:
            self._c(t, "psi_v")
        self._c(psi_c, "psi_c")
        n_v = psi_vs[0].shape[0]
        n_c = psi_c.shape[0] if c_idx is None else int(c_idx.numel())
        if c_idx is not None:
            self._c(c_idx, "c_idx", torch.int32)
        for t in list(E_vs) + [E_col] + ([w_col] if w_col is not None else []):
            self._c(t, "energies", torch.float64)
        chis = [self.new_chi(q) for q in range(nq)] if chis is None else chis
        for t in chis:
            self._c(t, "chi", torch.complex128)
        arr = lambda ts: (C.c_void_p * nq)(*[t.data_ptr() for t in ts])
        self._check(L.lib().chi0_build_batched(self._h, arr(psi_vs), n_v, arr(E_vs), _ptr(psi_c), _ptr(c_idx), n_c,
                                               _ptr(E_col), _ptr(w_col), arr(chis), int(use_graph), _stream()))
        return chis

    def backward(self, iq: int, M, n_v: int, n_c: int, E_v, E_col, w_col=None, grad_chi=None, diag_g=None):
        """chi0_backward: returns (grad_M, grad_E_v, grad_E_col)."""
        self._c(M, "M")
        for t, nm in ((E_v, "E_v"), (E_col, "E_col"), (w_col, "w_col"), (diag_g, "diag_g")):
            if t is not None:
                self._c(t, nm, torch.float64)
        if grad_chi is not None:
            self._c(grad_chi, "grad_chi", torch.complex128)
        gM = torch.empty_like(M)
        gEv = torch.empty(n_v, dtype=torch.float64, device=self.device)
        gEc = torch.empty(n_c, dtype=torch.float64, device=self.device)
        self._check(L.lib().chi0_backward(self._h, iq, _ptr(M), n_v, n_c, _ptr(E_v), _ptr(E_col), _ptr(w_col),
                                          _ptr(grad_chi), _ptr(diag_g), _ptr(gM), _ptr(gEv), _ptr(gEc),
                                          _stream()))
        return gM, gEv, gEc

    def build(self, iq: int, psi_v, E_v, psi_c, E_col, w_col=None, c_idx=None, chi=None):
        self._c(psi_v, "psi_v")
        self._c(psi_c, "psi_c")
        n_v = psi_v.shape[0]
        n_c = psi_c.shape[0] if c_idx is None else int(c_idx.numel())
        if c_idx is not None:
            self._c(c_idx, "c_idx", torch.int32)
        for t, nm in ((E_v, "E_v"), (E_col, "E_col"), (w_col, "w_col")):
            if t is not None:
                self._c(t, nm, torch.float64)
        chi = self.new_chi(iq) if chi is None else self._c(chi, "chi", torch.complex128)
        self._check(L.lib().chi0_build(self._h, iq, _ptr(psi_v), n_v, _ptr(E_v), _ptr(psi_c), _ptr(c_idx),
                                       n_c, _ptr(E_col), _ptr(w_col), _ptr(chi), _stream()))
        return chi

    # -- dielectric matrix ---------------------------------------------------
    def coulomb(self, iq: int, lattice, q_frac) -> np.ndarray:
        """chi0_coulomb: v(q+G) = 4 pi / (Omega |q+G|^2) on sphere iq (host array)."""
        A = _f64(lattice).reshape(3, 3)
        q = _f64(q_frac).reshape(3)
        v = np.empty(self.n_G[iq], np.float64)
        self._check(L.lib().chi0_coulomb(self._h, iq, A.ctypes.data, q.ctypes.data, v.ctypes.data))
        return v

    def epsilon(self, iq: int, chi, v, symmetric: bool = False, out=None) -> torch.Tensor:
        """chi0_epsilon: eps = 1 - v chi0 (or the symmetrised form); out may be chi."""
        self._c(chi, "chi", torch.complex128)
        self._c(v, "v", torch.float64)
        out = torch.empty_like(chi) if out is None else self._c(out, "out", torch.complex128)
        self._check(L.lib().chi0_epsilon(self._h, iq, _ptr(chi), _ptr(v), int(bool(symmetric)), _ptr(out),
                                         _stream()))
        return out

    def epsilon_inverse(self, iq: int, eps) -> torch.Tensor:
        """chi0_epsilon_inverse: eps is replaced by eps^-1 (and returned)."""
        self._c(eps, "eps", torch.complex128)
        self._check(L.lib().chi0_epsilon_inverse(self._h, iq, _ptr(eps), _stream()))
        return eps

    # -- COH self-energy with the plasmon-pole model ---------------------------
    def gpp(self, iq: int, psi_v, eps_inv0, lattice, q_frac, n_el: float):
        """chi0_gpp: (Omega2, wt) [N_G][N_G] complex128 of sphere iq."""
        self._c(psi_v, "psi_v")
        self._c(eps_inv0, "eps_inv0", torch.complex128)
        nG = self.n_G[iq]
        A = _f64(lattice).reshape(3, 3)
        q = _f64(q_frac).reshape(3)
        Om2 = torch.empty((nG, nG), dtype=torch.complex128, device=self.device)
        wt = torch.empty_like(Om2)
        self._check(L.lib().chi0_gpp(self._h, iq, _ptr(psi_v), int(psi_v.shape[0]), _ptr(eps_inv0), A.ctypes.data,
                                     q.ctypes.data, float(n_el), _ptr(Om2), _ptr(wt), _stream()))
        return Om2, wt

    def sigma_coh(self, iq: int, m, n_t: int, n_b: int, x, Om2, wt, v, w=None) -> np.ndarray:
        """chi0_sigma_coh: diagonal COH self-energy of n_t target bands (host, complex)."""
        self._c(m, "m")
        for t, nm in ((x, "x"), (v, "v"), (w, "w")):
            if t is not None:
                self._c(t, nm, torch.float64)
        self._c(Om2, "Omega2", torch.complex128)
        self._c(wt, "wt", torch.complex128)
        out = np.empty(2 * n_t, np.float64)
        self._check(L.lib().chi0_sigma_coh(self._h, iq, _ptr(m), int(n_t), int(n_b), _ptr(x), _ptr(w), _ptr(Om2),
                                           _ptr(wt), _ptr(v), out.ctypes.data, _stream()))
        return out[0::2] + 1j * out[1::2]

    def eps_inf(self, iq: int, eps_inv) -> np.ndarray:
        """chi0_eps_inf: 1 / [eps^-1]_00 per frequency (complex, host)."""
        self._c(eps_inv, "eps_inv", torch.complex128)
        out = np.empty(2 * self.n_freq, np.float64)
        self._check(L.lib().chi0_eps_inf(self._h, iq, _ptr(eps_inv), out.ctypes.data, _stream()))
        return out[0::2] + 1j * out[1::2]


QUAD_GRIDS = {"uniform": 0, "quantile": 1}
QUAD_RULES = {"midpoint": 0, "simpson": 1, "gauss2": 2}


def select_quadrature(E_c, N0: int, dE: float, dos_A: float, dos_V0: float, E_max: float,
                      grid: str = "uniform", rule: str = "midpoint", states: int = 1):
    """Columns of Eq. 3 with a non-uniform / higher-order quadrature and several
    states per node (chi0_select_quadrature): (band index, energy, weight)."""
    E_c = _f64(E_c)
    n_bins = int(np.ceil(max(E_max - E_c[min(max(N0, 1), E_c.size) - 1], 0) / dE)) + 1 if E_c.size else 0
    cap = int(N0) + (2 * n_bins + 1) * max(int(states), 1) + 2
    c_sel = np.empty(cap, np.int32)
    E_sel = np.empty(cap, np.float64)
    w_sel = np.empty(cap, np.float64)
    n = L.lib().chi0_select_quadrature(E_c.ctypes.data, E_c.size, int(N0), float(dE), float(dos_A),
                                       float(dos_V0), float(E_max), QUAD_GRIDS[grid], QUAD_RULES[rule],
                                       int(states), c_sel.ctypes.data, E_sel.ctypes.data, w_sel.ctypes.data, cap)
    if n < 0:
        raise L.Chi0Error(L.CHI0_ERR_INVALID, "chi0_select_quadrature rejected its input")
    return c_sel[:n].copy(), E_sel[:n].copy(), w_sel[:n].copy()


def select_adaptive(E_c, sens, N0: int, dE: float, dos_A: float, dos_V0: float, E_max: float,
                    n_split: int, states: int = 1):
    """Columns of Eq. 3 on a grid refined where the adjoint's first-order
    estimate of the energy-substitution error is largest (chi0_select_adaptive);
    sens = dL/dE_c, e.g. grad_E_col from Chi0Plan.backward."""
    E_c = _f64(E_c)
    sens = _f64(sens)
    if sens.shape != E_c.shape:
        raise ValueError("one sensitivity per conduction band")
    n_bins = int(np.ceil(max(E_max - E_c[min(max(N0, 1), E_c.size) - 1], 0) / dE)) + 1 if E_c.size else 0
    cap = int(N0) + (n_bins + int(n_split)) * max(int(states), 1) + 2
    c_sel = np.empty(cap, np.int32)
    E_sel = np.empty(cap, np.float64)
    w_sel = np.empty(cap, np.float64)
    n = L.lib().chi0_select_adaptive(E_c.ctypes.data, E_c.size, int(N0), sens.ctypes.data, float(dE),
                                     float(dos_A), float(dos_V0), float(E_max), int(n_split), int(states),
                                     c_sel.ctypes.data, E_sel.ctypes.data, w_sel.ctypes.data, cap)
    if n < 0:
        raise L.Chi0Error(L.CHI0_ERR_INVALID, "chi0_select_adaptive rejected its input")
    return c_sel[:n].copy(), E_sel[:n].copy(), w_sel[:n].copy()


def select_accelerated(E_c, N0: int, dE: float, dos_A: float, dos_V0: float, E_max: float):
    """Columns of Eq. 3/4 from chi0_select_accelerated: (band index, energy, weight)."""
    E_c = _f64(E_c)
    cap = int(N0) + int(np.ceil(max(E_max - E_c[min(max(N0, 1), E_c.size) - 1], 0) / dE)) + 2 if E_c.size else 1
    c_sel = np.empty(cap, np.int32)
    E_sel = np.empty(cap, np.float64)
    w_sel = np.empty(cap, np.float64)
    n = L.lib().chi0_select_accelerated(E_c.ctypes.data, E_c.size, int(N0), float(dE), float(dos_A),
                                        float(dos_V0), float(E_max), c_sel.ctypes.data, E_sel.ctypes.data,
                                        w_sel.ctypes.data, cap)
    if n < 0:
        raise L.Chi0Error(L.CHI0_ERR_INVALID, "chi0_select_accelerated rejected its input")
    return c_sel[:n].copy(), E_sel[:n].copy(), w_sel[:n].copy()


class Chi0Fn(torch.autograd.Function):
    """chi0 = Chi0Fn.apply(M, E_v, E_col, w_col, plan, iq): the contraction of
    Eq. 1 as a differentiable op.  Gradients flow to M, E_v and E_col through
    chi0_backward (dense upstream gradient)."""

    @staticmethod
    def forward(ctx, M, E_v, E_col, w_col, plan, iq):
        n_v, n_c = int(E_v.numel()), int(E_col.numel())
        chi = plan.accumulate(iq, M.contiguous(), n_v, n_c, E_v.contiguous(), E_col.contiguous(),
                              None if w_col is None else w_col.contiguous())
        ctx.save_for_backward(M, E_v, E_col, w_col)
        ctx.plan, ctx.iq = plan, iq
        return chi

    @staticmethod
    def backward(ctx, grad_chi):
        M, E_v, E_col, w_col = ctx.saved_tensors
        gM, gEv, gEc = ctx.plan.backward(ctx.iq, M.contiguous(), int(E_v.numel()), int(E_col.numel()),
                                         E_v.contiguous(), E_col.contiguous(),
                                         None if w_col is None else w_col.contiguous(),
                                         grad_chi=grad_chi.contiguous())
        return gM, gEv, gEc, None, None, None


class Chi0DiagLoss(torch.autograd.Function):
    """L = Chi0DiagLoss.apply(M, E_v, E_col, w_col, g, plan, iq) with
    L = sum_w sum_G g[w][G] Re chi0_w(G, G); the backward uses the fused
    diagonal adjoint of chi0_backward."""

    @staticmethod
    def forward(ctx, M, E_v, E_col, w_col, g, plan, iq):
        n_v, n_c = int(E_v.numel()), int(E_col.numel())
        chi = plan.accumulate(iq, M.contiguous(), n_v, n_c, E_v.contiguous(), E_col.contiguous(),
                              None if w_col is None else w_col.contiguous())
        loss = (g * torch.diagonal(chi, dim1=1, dim2=2).real).sum()
        ctx.save_for_backward(M, E_v, E_col, w_col, g)
        ctx.plan, ctx.iq = plan, iq
        return loss

    @staticmethod
    def backward(ctx, gL):
        M, E_v, E_col, w_col, g = ctx.saved_tensors
        gM, gEv, gEc = ctx.plan.backward(ctx.iq, M.contiguous(), int(E_v.numel()), int(E_col.numel()),
                                         E_v.contiguous(), E_col.contiguous(),
                                         None if w_col is None else w_col.contiguous(),
                                         diag_g=(g * gL).contiguous())
        return gM, gEv, gEc, None, None, None, None


def grid_energies_of_bands(E_c, N0: int, dE: float, E_max: float) -> np.ndarray:
    """chi0_grid_energies: for every conduction band above N0 the energy E_i of
    its Eq. 4 grid point; bands up to N0 keep their own energy (host arrays)."""
    E_c = _f64(E_c)
    out = np.empty_like(E_c)
    if L.lib().chi0_grid_energies(E_c.ctypes.data, E_c.size, int(N0), float(dE), float(E_max), out.ctypes.data) != 0:
        raise L.Chi0Error(L.CHI0_ERR_INVALID, "chi0_grid_energies rejected its input")
    return out


def energy_substitution_estimate(plan, iq: int, M, E_v, E_c, w_col, N0: int, dE: float, E_max: float,
                                 diag_g=None, grad_chi=None):
    """First-order estimate of the change of a loss when every conduction band
    above N0 is given the energy of its Eq. 4 grid point instead of its own:
    chi0_backward on the full band sum for dL/dE_c, then
    chi0_energy_substitution_estimate for sum_c dL/dE_c (E_i(c) - E_c).
    Returns (estimate, grad_E_c)."""
    n_v, n_c = int(E_v.numel()), int(E_c.numel())
    _, _, gEc = plan.backward(iq, M, n_v, n_c, E_v, E_c, w_col, grad_chi=grad_chi, diag_g=diag_g)
    est = C.c_double(0.0)
    plan._check(L.lib().chi0_energy_substitution_estimate(plan._h, _ptr(plan._c(E_c, "E_c", torch.float64)),
                                                          _ptr(gEc), n_c, int(N0), float(dE), float(E_max), None,
                                                          C.byref(est), _stream()))
    return est.value, gEc
