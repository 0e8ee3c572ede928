"""GPU parity of the FP32 pair stage (register-FFT plane transforms and the
sphere gather) on the grids of every workload, against the FP64 oracle.
Bar: relative Frobenius error of M <= 2e-6 (FP32 transforms of length <= 96)."""
import numpy as np
import pytest

from oracle import pair_elements, rel_fro, wfn_to_grid
from synth import make_problem

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,nv,nc", [("c1", 3, 7), ("c2", 3, 5), ("c4", 2, 5), ("c5", 1, 3),
                                        ("c3", 2, 3)])
def test_pairs_fp32_all_grids(name, nv, nc):
    from paper_1601_06767_gb300 import Chi0Plan
    prob = make_problem(name)
    iq = prob.n_q - 1
    cv, cc = prob.coeff_v(iq, np.arange(nv)), prob.coeff_c(np.arange(nc))
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    ref = pair_elements(uv, uc, prob.gvec[iq], prob.n)
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp16", gw=prob.gw) as plan:
        psi_v = plan.wfn_to_grid(_dev(cv))
        psi_c = plan.wfn_to_grid(_dev(cc))
        M = plan.pairs(iq, psi_v, psi_c)
        plan.sync_status()
        M = M.cpu().numpy()
    err = rel_fro(M, ref)
    print(f"\n{name}: n={prob.n} N_G={ref.shape[1]} pairs rel err {err:.2e}")
    assert err < 2e-6
