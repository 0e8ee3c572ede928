"""Pins of the oracle's COH self-energy with the HL plasmon-pole model:
the model reproduces the static eps^-1 it is fitted to and satisfies the
f-sum rule it is built from; the closed-form COH kernel equals Eq. 2's
frequency integral done numerically; brute-force loops for the density
ratio and the band/G sums."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle.coh import (coh_kernel, density_ratio, gpp_eps_inv, gpp_parameters, plasma_frequency2,
                        sigma_coh)


def _model(nG=7, seed=0):
    rng = np.random.default_rng(seed)
    kvec = rng.standard_normal((nG, 3)) + np.array([0.3, 0.0, 0.0])
    H = rng.standard_normal((nG, nG)) + 1j * rng.standard_normal((nG, nG))
    eps_inv = np.eye(nG) - 0.3 * (H @ H.conj().T) / nG - 0.2 * np.eye(nG)   # like a static eps^-1
    rho = 0.2 * (rng.standard_normal((nG, nG)) + 1j * rng.standard_normal((nG, nG)))
    rho = 0.5 * (rho + rho.conj().T)
    np.fill_diagonal(rho, 1.0)
    return eps_inv, rho, kvec


def test_model_reproduces_static_inverse_and_diagonal_weight():
    eps_inv, rho, kvec = _model()
    wp2 = plasma_frequency2(16.0, 500.0)
    Omega2, wt = gpp_parameters(eps_inv, rho, kvec, wp2)
    assert np.allclose(gpp_eps_inv(Omega2, wt, 0.0), eps_inv, rtol=0, atol=1e-13)
    assert np.allclose(np.diag(Omega2), wp2, rtol=1e-14)        # (q+G).(q+G)/|q+G|^2 rho(0)/rho(0)
    assert abs(plasma_frequency2(16.0, 500.0) - 4 * np.pi * 16 / 500) < 1e-15


def test_f_sum_rule_of_the_model():
    """int_0^inf w Im eps^-1(w + i eta) dw = -(pi/2) Omega2 for a real pole."""
    Om2, wt, eta = 0.8, 0.6, 1e-4
    f = lambda w: (Om2 / ((w + 1j * eta) ** 2 - wt ** 2)).imag * w
    val = quad(f, 0, 50, points=[wt], limit=400, epsabs=1e-12)[0]
    assert abs(val - (-0.5 * np.pi * Om2)) < 2e-3 * abs(val)


@pytest.mark.parametrize("x", [-1.3, -0.2, 0.9])
def test_coh_kernel_is_eq2_frequency_integral(x):
    """(i/2pi) int_0^inf dE' [eps_r^-1 - eps_a^-1](E') / (x - E' + i delta) with the
    model's pole broadened by eta tends to the closed-form kernel (v = 1, one
    element) as eta -> 0: the difference is O(eta) (1.3e-3 at eta = 1e-3,
    1.3e-4 at 1e-4 for these values), so eta = 1e-4 must agree to 3e-4."""
    Om2, wt, delta, eta = 0.8, 0.6, 2e-2, 1e-4
    d = lambda w: Om2 / ((w + 1j * eta) ** 2 - wt ** 2) - Om2 / ((w - 1j * eta) ** 2 - wt ** 2)
    g = lambda w: (1j / (2 * np.pi)) * d(w) / (x - w + 1j * delta)
    pts = [wt - 100 * eta, wt - 10 * eta, wt, wt + 10 * eta, wt + 100 * eta]
    edges = list(zip([0.0] + pts, pts + [200.0]))
    re = sum(quad(lambda w: g(w).real, a, b, limit=500, epsabs=1e-14, epsrel=1e-12)[0] for a, b in edges)
    im = sum(quad(lambda w: g(w).imag, a, b, limit=500, epsabs=1e-14, epsrel=1e-12)[0] for a, b in edges)
    K = coh_kernel(np.array([[Om2]], complex), np.array([[wt]], complex), np.ones(1), x, delta + eta)[0, 0]
    assert abs((re + 1j * im) - K) < 3e-4 * abs(K)


def test_density_ratio_brute_force():
    rng = np.random.default_rng(1)
    n = 6
    u = rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n))
    d = np.array([[0, 0, 0], [1, 0, 0], [-1, 2, 0], [2, -1, 3]])
    got = density_ratio(u, d)
    dens = 2 * (np.abs(u) ** 2).sum(0)
    j = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij"), -1).reshape(-1, 3)
    for k, dv in enumerate(d):
        want = np.sum(dens.reshape(-1) * np.exp(-2j * np.pi * (j @ dv) / n)) / dens.sum()
        assert abs(got[k] - want) < 1e-13
    assert abs(got[0] - 1) < 1e-15
    assert abs(density_ratio(u, -d[1:2])[0] - np.conj(got[1])) < 1e-14


def test_sigma_coh_brute_force():
    eps_inv, rho, kvec = _model(5, 2)
    Omega2, wt = gpp_parameters(eps_inv, rho, kvec, 0.3)
    rng = np.random.default_rng(3)
    m = rng.standard_normal((4, 5)) + 1j * rng.standard_normal((4, 5))
    x = np.array([-0.7, 0.2, 1.1, -2.0])
    w = np.array([1.0, 1.0, 0.4, 2.5])
    v = rng.uniform(0.2, 3.0, 5)
    delta = 1e-3
    want = 0.0
    for a in range(4):
        for i in range(5):
            for j in range(5):
                want += w[a] * m[a, i] * np.conj(m[a, j]) * Omega2[i, j] * v[j] / (
                    2 * wt[i, j] * (x[a] - wt[i, j] + 1j * delta))
    assert abs(sigma_coh(m, x, w, Omega2, wt, v, delta) - want) < 1e-13 * abs(want)
    from oracle.coh import sigma_coh_abs
    mag = 0.0
    for a in range(4):
        for i in range(5):
            for j in range(5):
                mag += abs(w[a] * m[a, i] * np.conj(m[a, j]) * Omega2[i, j] * v[j] / (
                    2 * wt[i, j] * (x[a] - wt[i, j] + 1j * delta)))
    assert abs(sigma_coh_abs(m, x, w, Omega2, wt, v, delta) - mag) < 1e-13 * mag
    assert mag >= abs(want)


def test_difference_table_and_problem_pipeline():
    """Difference bookkeeping by brute force; Sigma_COH of a small problem equals
    the accelerated form with N0 = N_c (every band explicit) and is linear in
    the column weights."""
    from oracle import chi0_full
    from oracle.coh import difference_table, sigma_coh_problem
    from oracle.dielectric import coulomb, epsilon, epsilon_inverse
    from synth import make_problem
    prob = make_problem("c1", n_v=4, n_c=12, n_G=[27], n_imag=0)
    uniq, idx = difference_table(prob.gvec[0])
    g = prob.gvec[0]
    for i in (0, 5, 26):
        for j in (0, 3, 26):
            assert np.array_equal(uniq[idx[i, j]], g[i] - g[j])
    A = prob.a * np.eye(3)
    eps_inv = epsilon_inverse(epsilon(chi0_full(prob, 0), coulomb(prob.q_frac[0], g, A)))[0]
    full, parts = sigma_coh_problem(prob, [0, 3], eps_inv, A, 2.0 * prob.n_v)
    assert np.all(np.isfinite(full)) and np.all(np.abs(full) > 0)
    same, _ = sigma_coh_problem(prob, [0, 3], eps_inv, A, 2.0 * prob.n_v, cols=np.arange(12),
                                E_cols=prob.E_c, w_cols=np.ones(12))
    assert np.allclose(same, full, rtol=1e-14)
    # the conduction part is linear in the weights: doubling them adds the conduction part again
    dbl, _ = sigma_coh_problem(prob, [0, 3], eps_inv, A, 2.0 * prob.n_v, cols=np.arange(12),
                               E_cols=prob.E_c, w_cols=2 * np.ones(12))
    val, _ = sigma_coh_problem(prob, [0, 3], eps_inv, A, 2.0 * prob.n_v, cols=np.arange(0),
                               E_cols=np.zeros(0), w_cols=np.zeros(0))
    assert np.allclose(dbl - full, full - val, rtol=1e-12)
