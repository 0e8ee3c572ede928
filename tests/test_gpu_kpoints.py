"""Eq. 1's sum over k on the GPU: chi0_build called once per k-point into the
same chi0 (its accumulate semantics), against the oracle's explicit sum over
k; both precisions, full and accelerated (selection per k-point)."""
import numpy as np
import pytest

from oracle import (accelerated_pairs, chi0_from_pairs, chi0_k_points, freq_factor, pair_elements,
                    rel_fro, select_accelerated, wfn_to_grid)
from synth import make_problem

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("bf16", 1e-6)])
def test_k_point_sum_full(precision, tol):
    from paper_1601_06767_gb300 import Chi0Plan
    prob = make_problem("c1", n_imag=2)
    n_k = 3
    ref = chi0_k_points(prob, 0, n_k)
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=precision, gw=prob.gw,
                  max_pairs=1024) as plan:
        chi = plan.new_chi(0)
        for ik in range(n_k):
            psi_v = plan.wfn_to_grid(_dev(prob.coeff_v(0, ik=ik)))
            psi_c = plan.wfn_to_grid(_dev(prob.coeff_c(ik=ik)))
            plan.build(0, psi_v, _dev(prob.E_v), psi_c, _dev(prob.E_c_k(ik)), chi=chi)
        plan.sync_status()
        got = chi.cpu().numpy()
    for iw in range(prob.omega.size):
        assert rel_fro(got[iw], ref[iw]) < tol


def test_k_point_sum_accelerated_bf16():
    from paper_1601_06767_gb300 import Chi0Plan, select_accelerated as lib_select
    prob = make_problem("c1", N0=40, dE_eV=3.0, n_imag=1)
    n_k = 2
    ref = 0
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="bf16", gw=prob.gw,
                  max_pairs=512) as plan:
        chi = plan.new_chi(0)
        for ik in range(n_k):
            E_c = prob.E_c_k(ik)
            sel = select_accelerated(E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0 + 0.004 * ik,
                                     prob.E_max + 0.004 * ik)
            c_idx, Ecol, wcol, dEp, wp = accelerated_pairs(prob.E_v, E_c, sel)
            uv = wfn_to_grid(prob.coeff_v(0, ik=ik), prob.gw, prob.n)
            uc = wfn_to_grid(prob.coeff_c(c_idx, ik=ik), prob.gw, prob.n)
            ref = ref + chi0_from_pairs(pair_elements(uv, uc, prob.gvec[0], prob.n),
                                        freq_factor(dEp, wp, prob.omega, prob.delta))
            c_sel, E_sel, w_sel = lib_select(E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0 + 0.004 * ik,
                                             prob.E_max + 0.004 * ik)
            assert np.array_equal(c_sel, c_idx)
            psi_v = plan.wfn_to_grid(_dev(prob.coeff_v(0, ik=ik)))
            psi_c = plan.wfn_to_grid(_dev(prob.coeff_c(ik=ik)))
            plan.build(0, psi_v, _dev(prob.E_v), psi_c, _dev(E_sel), w_col=_dev(w_sel),
                       c_idx=_dev(c_sel.astype(np.int32)), chi=chi)
        plan.sync_status()
        got = chi.cpu().numpy()
    assert rel_fro(got, ref) < 1e-6
