"""Pins of the oracle's adjoint of Eq. 1 against central finite differences
and against the closed form for a diagonal weighted loss."""
import numpy as np
import pytest

from oracle import chi0_from_pairs, chi0_grad, freq_factor


def _setup(seed=0, n_p=6, n_g=5):
    rng = np.random.default_rng(seed)
    M = (rng.standard_normal((n_p, n_g)) + 1j * rng.standard_normal((n_p, n_g))) / 3
    dE = -rng.uniform(0.2, 2.0, n_p)
    w = rng.uniform(0.5, 2.0, n_p)
    om = np.array([0.0, 0.3j])
    Gam = rng.standard_normal((2, n_g, n_g)) + 1j * rng.standard_normal((2, n_g, n_g))
    return M, dE, w, om, Gam


def _loss(M, dE, w, om, delta, Gam):
    chi = chi0_from_pairs(M, freq_factor(dE, w, om, delta))
    return float(np.sum(Gam.real * chi.real + Gam.imag * chi.imag))


@pytest.mark.parametrize("delta", [1e-3, 0.0])
def test_grad_dE_central_differences(delta):
    M, dE, w, om, Gam = _setup(1)
    _, gd = chi0_grad(M, dE, w, om, delta, Gam)
    h = 1e-6
    for p in range(dE.size):
        e = np.zeros_like(dE)
        e[p] = h
        fd = (_loss(M, dE + e, w, om, delta, Gam) - _loss(M, dE - e, w, om, delta, Gam)) / (2 * h)
        assert abs(gd[p] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_grad_M_central_differences():
    M, dE, w, om, Gam = _setup(2)
    gM, _ = chi0_grad(M, dE, w, om, 1e-3, Gam)
    h = 1e-6
    for p in range(M.shape[0]):
        for g in range(M.shape[1]):
            for unit, part in ((1.0, "re"), (1j, "im")):
                E = np.zeros_like(M)
                E[p, g] = unit * h
                fd = (_loss(M + E, dE, w, om, 1e-3, Gam) - _loss(M - E, dE, w, om, 1e-3, Gam)) / (2 * h)
                got = gM[p, g].real if part == "re" else gM[p, g].imag
                assert abs(got - fd) <= 1e-7 * max(1.0, abs(fd))


def test_diagonal_loss_closed_form():
    M, dE, w, _, _ = _setup(3, n_p=8, n_g=7)
    wG = np.random.default_rng(9).uniform(0, 1, 7)
    Gam = np.diag(wG).astype(complex)[None]
    gM, gd = chi0_grad(M, dE, w, np.array([0.0]), 1e-3, Gam)
    f = freq_factor(dE, w, [0.0], 1e-3)[0]
    fprime = -w / (dE + 1e-3j) ** 2
    assert np.allclose(gM, 2 * f.real[:, None] * wG[None, :] * M, rtol=1e-13, atol=1e-15)
    assert np.allclose(gd, fprime.real * (np.abs(M) ** 2 @ wG), rtol=1e-13, atol=1e-15)


def test_first_order_energy_substitution_estimate():
    """Giving every band above N0 the energy of its Eq. 4 grid point changes a
    loss by sum_c dL/dE_c (E_i(c) - E_c) to first order: the residual of the
    linear estimate falls quadratically with the step while the change itself
    falls linearly."""
    from oracle import energy_substitution_estimate, grid_energy_of_bands, select_accelerated
    rng = np.random.default_rng(11)
    nv, nc, ng = 3, 60, 6
    M = (rng.standard_normal((nv * nc, ng)) + 1j * rng.standard_normal((nv * nc, ng))) / 4
    Ev = np.linspace(-0.25, -0.02, nv)
    Ec = np.sort(rng.uniform(0.17, 2.2, nc))
    wG = rng.uniform(0, 1, ng)
    Gam = np.diag(wG).astype(complex)[None]
    N0 = 10

    def loss(Ec_):
        dE_ = (Ev[:, None] - Ec_[None, :]).reshape(-1)
        chi = chi0_from_pairs(M, freq_factor(dE_, np.ones_like(dE_), [0.0], 1e-3))
        return float(np.sum(wG * np.real(np.diagonal(chi[0]))))

    dEp = (Ev[:, None] - Ec[None, :]).reshape(-1)
    _, gd = chi0_grad(M, dEp, np.ones_like(dEp), np.array([0.0]), 1e-3, Gam)
    gEc = -gd.reshape(nv, nc).sum(0)
    out = []
    for step in (0.08, 0.04, 0.02):
        sel = select_accelerated(Ec, N0, step, 1.0, 0.17, 2.2)
        # brute force: the midpoint of the step whose half-open interval holds E_c
        Esub = Ec.copy()
        for c in range(N0, nc):
            for k in range(sel["E_i"].size):
                last = k == sel["E_i"].size - 1
                if sel["edges"][k] <= Ec[c] and (last or Ec[c] < sel["edges"][k + 1]):
                    Esub[c] = sel["E_i"][k]
                    break
        assert np.array_equal(Esub, grid_energy_of_bands(Ec, N0, step, 2.2))
        actual = loss(Esub) - loss(Ec)
        est = energy_substitution_estimate(Ec, gEc, N0, step, 2.2)
        assert est == pytest.approx(float(np.sum(gEc * (Esub - Ec))), rel=1e-14)
        out.append((abs(actual), abs(actual - est)))
    for (a1, r1), (a2, r2) in zip(out, out[1:]):
        assert r2 < 0.5 * r1            # residual: second order
    assert out[-1][1] < 0.05 * out[-1][0]
