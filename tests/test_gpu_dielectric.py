"""GPU parity of the dielectric matrix (eps = 1 - v chi0, its inverse by
blocked Gauss-Jordan elimination and eps_inf = 1/[eps^-1]_00) against the FP64
oracle.  Bars: FP64 plans 1e-13 x cond(eps) (relative Frobenius); split
plans (FP32 elimination) 2e-7 x sqrt(N_G) x cond(eps); eps itself to a few
ulps of FP64 (the kernel may fuse the multiply-subtract)."""
import numpy as np
import pytest

from oracle import chi0_full, rel_fro
from oracle.dielectric import coulomb, eps_inf, epsilon, epsilon_inverse
from synth import make_problem

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _plan(n_G, n_freq, precision="fp64", q_frac=((0.0, 0.0, 0.0),), gvec=None, n=24):
    from paper_1601_06767_gb300 import Chi0Plan
    from synth.mgo import g_sphere
    if gvec is None:
        gvec = [g_sphere(n_G, q, n) for q in q_frac]
    omega = np.concatenate([[0.0], 1j * np.linspace(0.1, 1.0, n_freq - 1)]) if n_freq > 1 else np.zeros(1)
    return Chi0Plan(n, gvec, omega, 1e-3, precision=precision)


def _tol(precision, eps):
    cond = max(np.linalg.cond(e) for e in eps)
    n = eps.shape[-1]
    return (1e-13 if precision == "fp64" else 2e-7 * np.sqrt(n)) * cond, cond


_C1 = {}


def _c1():
    if not _C1:
        prob = make_problem("c1", n_imag=2)
        _C1["prob"] = prob
        _C1["chi"] = chi0_full(prob, 0)
    return _C1["prob"], _C1["chi"]


def test_coulomb_matches_oracle():
    prob, _ = _c1()
    with _plan(350, 1, q_frac=prob.q_frac, gvec=prob.gvec) as plan:
        A = prob.a * np.eye(3)
        v = plan.coulomb(0, A, prob.q_frac[0])
    assert rel_fro(v, coulomb(prob.q_frac[0], prob.gvec[0], A)) < 1e-15
    fcc = 0.5 * 7.96 * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=float)
    with _plan(350, 1, q_frac=prob.q_frac, gvec=prob.gvec) as plan:
        v2 = plan.coulomb(0, fcc, (0.1, 0.2, 0.3))
    assert rel_fro(v2, coulomb((0.1, 0.2, 0.3), prob.gvec[0], fcc)) < 1e-14


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
@pytest.mark.parametrize("symmetric", [False, True])
def test_epsilon_inverse_eps_inf_c1(precision, symmetric):
    """chi0 of the 8-atom-sized workload (N_G = 350: ten 32-column panels and a
    ragged one), static and two imaginary frequencies."""
    prob, chi = _c1()
    A = prob.a * np.eye(3)
    v = coulomb(prob.q_frac[0], prob.gvec[0], A)
    eps_ref = epsilon(chi, v, symmetric)
    inv_ref = epsilon_inverse(eps_ref)
    from paper_1601_06767_gb300 import Chi0Plan
    with Chi0Plan(prob.n, prob.gvec, prob.omega, prob.delta, precision=precision) as plan:
        vg = plan.coulomb(0, A, prob.q_frac[0])
        eps = plan.epsilon(0, _dev(chi), _dev(vg), symmetric=symmetric)
        plan.sync_status()
        e_np = eps.cpu().numpy()
        plan.epsilon_inverse(0, eps)
        plan.sync_status()
        inv = eps.cpu().numpy()
        einf = plan.eps_inf(0, eps)
    assert rel_fro(e_np, eps_ref) < 1e-15
    tol, cond = _tol(precision, eps_ref)
    errs = [rel_fro(inv[i], inv_ref[i]) for i in range(inv.shape[0])]
    print(f"\n{precision} sym={symmetric}: cond {cond:.2e}, inverse err {['%.2e' % e for e in errs]}, "
          f"eps_inf {einf}")
    assert max(errs) < tol
    ref_inf = eps_inf(inv_ref, prob.gvec[0].tolist().index([0, 0, 0]))
    assert np.max(np.abs(einf - ref_inf) / np.abs(ref_inf)) < tol


@pytest.mark.parametrize("n_G", [1, 2, 31, 32, 33, 57, 64, 257])
@pytest.mark.parametrize("precision", ["fp64", "fp16"])
def test_inverse_shapes_and_pivoting(n_G, precision):
    """Sizes below, at and above the 32-column panel; a matrix whose diagonal is
    small so that every column needs a row interchange."""
    rng = np.random.default_rng(n_G)
    nf = 2
    P = np.eye(n_G)[rng.permutation(n_G)]
    E = np.empty((nf, n_G, n_G), dtype=np.complex128)
    E[0] = P * (2 + rng.uniform(0, 1, n_G))[:, None] + 0.05 * (rng.standard_normal((n_G, n_G))
                                                             + 1j * rng.standard_normal((n_G, n_G)))
    E[1] = np.eye(n_G) + 0.3 * (rng.standard_normal((n_G, n_G)) + 1j * rng.standard_normal((n_G, n_G))) / np.sqrt(n_G)
    ref = epsilon_inverse(E)
    with _plan(n_G, nf, precision=precision) as plan:
        t = _dev(E)
        plan.epsilon_inverse(0, t)
        plan.sync_status()
        got = t.cpu().numpy()
    tol, cond = _tol("fp64" if precision == "fp64" else "split", E)
    for i in range(nf):
        assert rel_fro(got[i], ref[i]) < tol, (i, rel_fro(got[i], ref[i]), cond)


def test_singular_matrix_reports_status():
    import paper_1601_06767_gb300._lib as L
    E = np.ones((1, 40, 40), dtype=np.complex128)          # rank 1
    E[0, :, 3] = 0.0                                        # and a zero column
    with _plan(40, 1) as plan:
        t = _dev(E)
        plan.epsilon_inverse(0, t)
        with pytest.raises(L.Chi0Error) as ei:
            plan.sync_status()
        assert ei.value.status == L.CHI0_ERR_SINGULAR
        # the plan stays usable
        t = _dev(np.eye(40, dtype=np.complex128)[None] * 2.0)
        plan.epsilon_inverse(0, t)
        plan.sync_status()
        assert np.allclose(t.cpu().numpy()[0], 0.5 * np.eye(40))


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_inverse_c2_size_sampled(precision):
    """The 64-atom-sized sphere (N_G = 2500, 79 panels) on an eps-like matrix
    (identity minus a random negative-semidefinite chi0 of rank 600 scaled by a
    Coulomb-like v); compared with the oracle on one frequency."""
    rng = np.random.default_rng(11)
    nG, K = 2500, 600
    M = (rng.standard_normal((K, nG)) + 1j * rng.standard_normal((K, nG))) / np.sqrt(2 * nG)
    chi = -(M.T * rng.uniform(0.1, 1.0, K)) @ M.conj()
    v = 1.0 / (0.05 + np.arange(nG) / nG)
    E = epsilon(chi[None], v)
    ref = epsilon_inverse(E)
    with _plan(nG, 1, precision=precision, n=48) as plan:
        t = _dev(E)
        plan.epsilon_inverse(0, t)
        plan.sync_status()
        got = t.cpu().numpy()
    tol, cond = _tol(precision, E)
    err = rel_fro(got[0], ref[0])
    print(f"\nN_G 2500 {precision}: cond {cond:.2e} err {err:.2e}")
    assert err < tol
