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


@pytest.mark.parametrize("lo,ext", [((-14, -20, 3), 29), ((5, -30, -31), 29), ((-31, 4, -8), 29),
                                    ((-16, -9, -23), 32), ((-17, -17, 2), 34)])
def test_pairs_96_shifted_boxes(lo, ext):
    """The 96^3 pair stage (cooperative 96-point lines) on G lists drawn from
    boxes that start at other offsets than a centred sphere, so the kept output
    ranges along i3 and i2 begin anywhere on the grid and wrap past 96, against
    the oracle: extent 29, 32 (the largest the line kernel takes) and 34 (the
    direct row kernel)."""
    from paper_1601_06767_gb300 import Chi0Plan
    prob = make_problem("c5")
    rng = np.random.default_rng(abs(sum(lo)) + 5 + ext)
    axes = [np.arange(l, l + ext) for l in lo]
    box = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    g = box[rng.choice(box.shape[0], 1500, replace=False)].astype(np.int32)
    cv, cc = prob.coeff_v(0, np.arange(2)), prob.coeff_c(np.arange(3))
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    ref = pair_elements(uv, uc, g, prob.n)
    with Chi0Plan(prob.n, [g], prob.omega, prob.delta, precision="fp16", gw=prob.gw) as plan:
        M = plan.pairs(0, plan.wfn_to_grid(_dev(cv)), plan.wfn_to_grid(_dev(cc)))
        plan.sync_status()
        M = M.cpu().numpy()
    err = rel_fro(M, ref)
    emax = np.max(np.abs(M - ref)) / np.max(np.abs(ref))
    print(f"\n96^3 box from {lo}, extent {ext}: rel err {err:.2e}, max abs err / max |M| {emax:.2e}")
    assert err < 2e-6 and emax < 2e-6


@pytest.mark.parametrize("name,n_g", [("c1", 300), ("c2", 900)])
def test_pairs_fp32_scattered_g_list(name, n_g):
    """A G list that is not a sphere: distinct vectors drawn at random from the
    box |g_i| <= n/4 - 1, in random order, so that columns (k2, k3) have holes
    and lone points and the caller's order is unrelated to column order."""
    from paper_1601_06767_gb300 import Chi0Plan
    prob = make_problem(name)
    rng = np.random.default_rng(77)
    r = prob.n // 4 - 1
    box = np.stack(np.meshgrid(*(np.arange(-r, r + 1),) * 3, indexing="ij"), -1).reshape(-1, 3)
    g = box[rng.choice(box.shape[0], n_g, replace=False)].astype(np.int32)
    cv, cc = prob.coeff_v(0, np.arange(2)), prob.coeff_c(np.arange(3))
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    ref = pair_elements(uv, uc, g, prob.n)
    with Chi0Plan(prob.n, [g], prob.omega, prob.delta, precision="bf16", gw=prob.gw) as plan:
        M = plan.pairs(0, plan.wfn_to_grid(_dev(cv)), plan.wfn_to_grid(_dev(cc)))
        plan.sync_status()
        M = M.cpu().numpy()
    err = np.max(np.abs(M - ref)) / np.max(np.abs(ref))
    print(f"\n{name}: scattered G list of {n_g}, max abs err / max |M| {err:.2e}")
    assert err < 2e-6


@pytest.mark.parametrize("name,nb", [("c1", 7), ("c2", 5), ("c4", 4), ("c5", 2)])
def test_wfn_to_grid_fp32_all_grids(name, nb):
    """Split plans put the wavefunctions on the grid in FP32; element by element
    against the FP64 oracle on every workload grid, bar 1e-6 of the largest value."""
    from paper_1601_06767_gb300 import Chi0Plan
    prob = make_problem(name)
    cc = prob.coeff_c(np.arange(nb))
    ref = wfn_to_grid(cc, prob.gw, prob.n)
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="bf16", gw=prob.gw) as plan:
        psi = plan.wfn_to_grid(_dev(cc)).cpu().numpy()
    err = np.max(np.abs(psi.reshape(ref.shape) - ref)) / np.max(np.abs(ref))
    print(f"\n{name}: n={prob.n} wavefunctions max abs err / max |psi| {err:.2e}")
    assert err < 1e-6

