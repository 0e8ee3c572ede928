"""GPU adjoint (chi0_backward) against the FP64 oracle gradient and central
finite differences of the GPU's own FP64 forward.  Bars: FP64 path <= 1e-12
relative to the oracle gradient; FP32 pair elements through the split plans
<= 1e-5; finite differences (h = 1e-6 Ha) <= 1e-6 relative."""
import numpy as np
import pytest

from oracle import chi0_from_pairs, chi0_grad, freq_factor, pair_elements, rel_fro, wfn_to_grid
from synth import make_problem

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(name="c4", nv=4, nc=24, n_imag=0, seed=3):
    prob = make_problem(name, n_imag=n_imag)
    cv, cc = prob.coeff_v(0, np.arange(nv)), prob.coeff_c(np.arange(nc))
    uv, uc = wfn_to_grid(cv, prob.gw, prob.n), wfn_to_grid(cc, prob.gw, prob.n)
    M = pair_elements(uv, uc, prob.gvec[0], prob.n)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, nc)
    return prob, M, prob.E_v[:nv].copy(), prob.E_c[:nc].copy(), w, rng


def _oracle_grads(prob, M, Ev, Ec, w, Gamma):
    nv, nc = Ev.size, Ec.size
    dE = (Ev[:, None] - Ec[None, :]).reshape(-1)
    gM, gd = chi0_grad(M, dE, np.tile(w, nv), prob.omega, prob.delta, Gamma)
    gd = gd.reshape(nv, nc)
    return gM, gd.sum(1), -gd.sum(0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp16", 1e-5), ("bf16", 1e-5)])
def test_backward_diagonal_loss_c4_shape(precision, tol):
    """L = sum_G Re(w_G chi0_GG(q, 0)) with w_G ~ U(0,1) on the 36^3 / 1200-vector sphere."""
    from paper_1601_06767_gb300 import Chi0Plan
    prob, M, Ev, Ec, w, rng = _case()
    nG = M.shape[1]
    wG = rng.uniform(0.0, 1.0, nG)
    Gamma = np.diag(wG).astype(complex)[None]
    ref = _oracle_grads(prob, M, Ev, Ec, w, Gamma)
    cdt = np.complex128 if precision == "fp64" else np.complex64
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=precision, max_pairs=64) as plan:
        gM, gEv, gEc = plan.backward(0, _dev(M.astype(cdt)), Ev.size, Ec.size, _dev(Ev), _dev(Ec), _dev(w),
                                     diag_g=_dev(wG[None]))
        plan.sync_status()
    errs = [rel_fro(gM.cpu().numpy(), ref[0]), rel_fro(gEv.cpu().numpy(), ref[1]), rel_fro(gEc.cpu().numpy(), ref[2])]
    print(f"\n{precision} diag adjoint rel err M/E_v/E_c {['%.1e' % e for e in errs]}")
    assert max(errs) < tol


def test_backward_dense_fp64_matches_oracle():
    from paper_1601_06767_gb300 import Chi0Plan
    prob, M, Ev, Ec, w, rng = _case("c1", nv=3, nc=21, n_imag=2)
    nG = M.shape[1]
    Gamma = rng.standard_normal((prob.omega.size, nG, nG)) + 1j * rng.standard_normal((prob.omega.size, nG, nG))
    ref = _oracle_grads(prob, M, Ev, Ec, w, Gamma)
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp64", max_pairs=64) as plan:
        gM, gEv, gEc = plan.backward(0, _dev(M), Ev.size, Ec.size, _dev(Ev), _dev(Ec), _dev(w),
                                     grad_chi=_dev(Gamma))
        plan.sync_status()
    assert rel_fro(gM.cpu().numpy(), ref[0]) < 1e-12
    assert rel_fro(gEv.cpu().numpy(), ref[1]) < 1e-12
    assert rel_fro(gEc.cpu().numpy(), ref[2]) < 1e-12


def test_autograd_matches_central_differences():
    import torch
    from paper_1601_06767_gb300 import Chi0DiagLoss, Chi0Fn, Chi0Plan
    prob, M, Ev, Ec, w, rng = _case("c1", nv=3, nc=10, n_imag=1)
    nG = M.shape[1]
    Gamma = _dev(rng.standard_normal((prob.omega.size, nG, nG)) + 1j * rng.standard_normal((prob.omega.size, nG, nG)))
    g = _dev(rng.uniform(0, 1, (prob.omega.size, nG)))
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision="fp64") as plan:
        Mt = _dev(M).requires_grad_(True)
        Evt = _dev(Ev).requires_grad_(True)
        Ect = _dev(Ec).requires_grad_(True)
        wt = _dev(w)
        chi = Chi0Fn.apply(Mt, Evt, Ect, wt, plan, 0)
        L = (Gamma.real * chi.real + Gamma.imag * chi.imag).sum()
        L.backward()
        L2 = Chi0DiagLoss.apply(Mt, Evt, Ect, wt, g, plan, 0)
        gEv_d, gEc_d = torch.autograd.grad(L2, (Evt, Ect))

        def loss(Ev_, Ec_, Gam=Gamma):
            c = plan.accumulate(0, _dev(M), Ev.size, Ec.size, _dev(Ev_), _dev(Ec_), wt)
            return float((Gam.real * c.real + Gam.imag * c.imag).sum())

        def loss_d(Ev_, Ec_):
            c = plan.accumulate(0, _dev(M), Ev.size, Ec.size, _dev(Ev_), _dev(Ec_), wt)
            return float((g * torch.diagonal(c, dim1=1, dim2=2).real).sum())

        h = 1e-6
        for fn, gv, gc in ((loss, Evt.grad.cpu().numpy(), Ect.grad.cpu().numpy()),
                           (loss_d, gEv_d.cpu().numpy(), gEc_d.cpu().numpy())):
            for i in range(Ev.size):
                e = np.zeros_like(Ev)
                e[i] = h
                fd = (fn(Ev + e, Ec) - fn(Ev - e, Ec)) / (2 * h)
                assert abs(gv[i] - fd) <= 1e-6 * max(1.0, abs(fd))
            for i in range(0, Ec.size, 3):
                e = np.zeros_like(Ec)
                e[i] = h
                fd = (fn(Ev, Ec + e) - fn(Ev, Ec - e)) / (2 * h)
                assert abs(gc[i] - fd) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("precision", ["fp64", "fp16"])
def test_energy_substitution_estimate_gpu(precision):
    """The adjoint-based first-order estimate of the energy-substitution part of
    the accelerated sum's error, against the actual change of the loss computed
    by two forward builds (Eq. 1 with E_c and with the grid energies)."""
    import torch
    from paper_1601_06767_gb300 import Chi0Plan, energy_substitution_estimate, grid_energies_of_bands
    prob, M, Ev, Ec, w, rng = _case("c1", nv=4, nc=200, seed=5)
    nG = M.shape[1]
    wG = rng.uniform(0, 1, nG)
    cdt = np.complex128 if precision == "fp64" else np.complex64
    N0 = 40
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=precision) as plan:
        Md, Evd, Ecd, gd = _dev(M.astype(cdt)), _dev(Ev), _dev(Ec), _dev(wG[None])

        def loss(E):
            c = plan.accumulate(0, Md, Ev.size, Ec.size, Evd, _dev(E))
            return float((gd[0] * torch.diagonal(c[0]).real).sum())

        rows = []
        for dE in (0.04, 0.02, 0.01):
            est, _ = energy_substitution_estimate(plan, 0, Md, Evd, Ecd, None, N0, dE, prob.E_max, diag_g=gd)
            Esub = grid_energies_of_bands(Ec, N0, dE, prob.E_max)
            rows.append((abs(loss(Esub) - loss(Ec)), abs(loss(Esub) - loss(Ec) - est)))
    for (a1, r1), (a2, r2) in zip(rows, rows[1:]):
        assert r2 < 0.5 * r1
    assert rows[-1][1] < 0.05 * rows[-1][0]


def test_energy_substitution_estimate_matches_oracle():
    """chi0_energy_substitution_estimate against the oracle on the same
    sensitivities: the grid energy of every band bit for bit, the sum to
    rounding (the device sums in a fixed tree order)."""
    import ctypes as C
    import torch
    import paper_1601_06767_gb300 as pkg
    from paper_1601_06767_gb300 import _lib as L
    from oracle import energy_substitution_estimate, grid_energy_of_bands
    from synth import HARTREE_EV
    prob = make_problem("c5")
    rng = np.random.default_rng(21)
    sens = rng.standard_normal(prob.n_c) * np.exp(-prob.E_c)
    small = make_problem("c1")                      # the plan only lends its workspace
    with pkg.Chi0Plan(small.n, small.gvec, [0.0], small.delta, precision="fp64") as plan:
        Ecd, sd = _dev(prob.E_c), _dev(sens)
        for N0, dE_eV in ((prob.N0, 2.0), (prob.N0, 0.31), (1, 4.0), (0, 2.0), (prob.n_c, 2.0)):
            dE = dE_eV / HARTREE_EV
            Esub = torch.empty_like(Ecd)
            est = C.c_double(0.0)
            plan._check(pkg.lib().chi0_energy_substitution_estimate(
                plan._h, C.c_void_p(Ecd.data_ptr()), C.c_void_p(sd.data_ptr()), prob.n_c, N0, dE, prob.E_max,
                C.c_void_p(Esub.data_ptr()), C.byref(est), None))
            ref_E = grid_energy_of_bands(prob.E_c, N0, dE, prob.E_max)
            assert np.array_equal(Esub.cpu().numpy(), ref_E), (N0, dE_eV)
            ref = energy_substitution_estimate(prob.E_c, sens, N0, dE, prob.E_max)
            scale = float(np.sum(np.abs(sens * (ref_E - prob.E_c)))) or 1.0
            assert abs(est.value - ref) <= 1e-13 * scale, (N0, dE_eV, est.value, ref)
        st = pkg.lib().chi0_energy_substitution_estimate(plan._h, None, None, 10, 1, 0.0, 2.2, None,
                                                         C.byref(est), None)
        assert st == L.CHI0_ERR_INVALID
