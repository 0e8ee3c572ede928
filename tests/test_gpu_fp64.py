"""GPU parity of the FP64 path (CHI0_FP64 plans) against the FP64 oracle:
wavefunctions on the grid, pair matrix elements, the Eq. 1 contraction and the
streamed whole-path build, on the 8-atom-sized workload and ragged variants.
Bar: relative Frobenius error <= 1e-12."""
import numpy as np
import pytest

from _parity import check_chi
from oracle import (accelerated_pairs, chi0_from_pairs, freq_factor, pair_elements, rel_fro,
                    select_accelerated, wfn_to_grid)
from synth import make_problem

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _torch():
    import torch
    return torch


def _plan(prob, precision="fp64", **kw):
    from paper_1601_06767_gb300 import Chi0Plan
    return Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=precision, gw=prob.gw, **kw)


def _dev(a, dtype=None):
    torch = _torch()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def test_wfn_to_grid_fp64():
    prob = make_problem("c1")
    cc = prob.coeff_c(np.arange(7))
    with _plan(prob) as plan:
        psi = plan.wfn_to_grid(_dev(cc)).cpu().numpy()
    ref = wfn_to_grid(cc, prob.gw, prob.n)
    assert rel_fro(psi, ref) < TOL64


@pytest.mark.parametrize("case", ["c1", "q_shift", "odd"])
def test_pairs_fp64(case):
    if case == "c1":
        prob = make_problem("c1")
        vb, cb = np.arange(5), np.arange(9)
    elif case == "q_shift":   # off-centre sphere (2x2x2 shifted q grid), ragged N_G
        prob = make_problem("c1", n_G=[203], q_frac=[(0.25, 0.75, 0.25)])
        vb, cb = np.arange(3), np.arange(11)
    else:                     # odd grid, small sphere
        prob = make_problem("c1", n=21, n_G=[57], q_bohr=[(0.0, 0.0, 0.0)])
        vb, cb = np.arange(2), np.arange(3)
    cv, cc = prob.coeff_v(0, vb), prob.coeff_c(cb)
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    ref = pair_elements(uv, uc, prob.gvec[0], prob.n)
    with _plan(prob) as plan:
        M = plan.pairs(0, _dev(uv), _dev(uc)).cpu().numpy()
    assert M.shape == ref.shape
    assert rel_fro(M, ref) < TOL64


def test_pairs_with_index_lists_fp64():
    torch = _torch()
    prob = make_problem("c1")
    cv, cc = prob.coeff_v(0, np.arange(6)), prob.coeff_c(np.arange(10))
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    vi, ci = np.array([5, 0, 3]), np.array([9, 2, 2, 7])
    ref = pair_elements(uv[vi], uc[ci], prob.gvec[0], prob.n)
    with _plan(prob) as plan:
        M = plan.pairs(0, _dev(uv), _dev(uc), v_idx=_dev(vi.astype(np.int32)),
                       c_idx=_dev(ci.astype(np.int32))).cpu().numpy()
    assert rel_fro(M, ref) < TOL64
    del torch


def test_accumulate_fp64_matches_eq1():
    prob = make_problem("c1", n_imag=3)
    rng = np.random.default_rng(0)
    nv, nc, nG = 4, 37, prob.gvec[0].shape[0]
    M = (rng.standard_normal((nv * nc, nG)) + 1j * rng.standard_normal((nv * nc, nG))) * 0.05
    Ev = prob.E_v[:nv]
    Ec = prob.E_c[:nc]
    w = rng.uniform(0.5, 2.0, nc)
    dE = (Ev[:, None] - Ec[None, :]).reshape(-1)
    ref = chi0_from_pairs(M, freq_factor(dE, np.tile(w, nv), prob.omega, prob.delta))
    with _plan(prob, max_pairs=64) as plan:       # several internal pair blocks
        chi = plan.accumulate(0, _dev(M), nv, nc, _dev(Ev), _dev(Ec), _dev(w)).cpu().numpy()
    check_chi(chi, ref, TOL64, label="fp64 accumulate")


def test_build_c1_full_fp64():
    """The 8-atom-sized static workload, whole path from coefficients."""
    prob = make_problem("c1")
    cv, cc = prob.coeff_v(0), prob.coeff_c()
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    M = pair_elements(uv, uc, prob.gvec[0], prob.n)
    dE = (prob.E_v[:, None] - prob.E_c[None, :]).reshape(-1)
    ref = chi0_from_pairs(M, freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta))
    with _plan(prob, max_pairs=1024) as plan:
        psi_v = plan.wfn_to_grid(_dev(cv))
        psi_c = plan.wfn_to_grid(_dev(cc))
        chi = plan.build(0, psi_v, _dev(prob.E_v), psi_c, _dev(prob.E_c))
        plan.sync_status()
        chi = chi.cpu().numpy()
    check_chi(chi, ref, TOL64, label="fp64 build c1")


def test_build_accelerated_fp64():
    prob = make_problem("c1", N0=40, dE_eV=3.0)
    sel = select_accelerated(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max)
    c_idx, Ecol, wcol, dEp, wp = accelerated_pairs(prob.E_v, prob.E_c, sel)
    cv, cc = prob.coeff_v(0), prob.coeff_c()
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    M = pair_elements(uv, uc[c_idx], prob.gvec[0], prob.n)
    ref = chi0_from_pairs(M, freq_factor(dEp, wp, prob.omega, prob.delta))
    with _plan(prob, max_pairs=256) as plan:
        psi_v = plan.wfn_to_grid(_dev(cv))
        psi_c = plan.wfn_to_grid(_dev(cc))
        chi = plan.build(0, psi_v, _dev(prob.E_v), psi_c, _dev(Ecol), w_col=_dev(wcol),
                         c_idx=_dev(c_idx.astype(np.int32))).cpu().numpy()
    check_chi(chi, ref, TOL64, label="fp64 accelerated build")


def test_empty_inputs_are_no_ops():
    torch = _torch()
    prob = make_problem("c1")
    with _plan(prob) as plan:
        z = torch.zeros((0,) + plan.n, dtype=torch.complex128, device="cuda")
        assert plan.pairs(0, z, z).shape == (0, 350)
        chi = plan.new_chi(0)
        plan.accumulate(0, torch.zeros((0, 350), dtype=torch.complex128, device="cuda"), 0, 5,
                        _dev(prob.E_v[:1]), _dev(prob.E_c[:5]), chi=chi)
        plan.sync_status()
        assert float(chi.abs().max()) == 0.0


def test_pairs_fp64_large_grid_row_chunks():
    """96^3 grid with the 8000-vector sphere: planes do not fit shared memory in
    FP64, so the row-chunked kernel runs."""
    prob = make_problem("c5")
    cv, cc = prob.coeff_v(0, np.arange(2)), prob.coeff_c(np.arange(2))
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    ref = pair_elements(uv, uc, prob.gvec[0], prob.n)
    with _plan(prob) as plan:
        M = plan.pairs(0, plan.wfn_to_grid(_dev(cv)), plan.wfn_to_grid(_dev(cc)))
        plan.sync_status()
        M = M.cpu().numpy()
    assert rel_fro(M, ref) < TOL64
