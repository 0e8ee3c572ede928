"""Pins of the oracle's Eq. 1 (frequency factor and band-pair contraction)
against closed forms, a direct loop, rank-1 structure and the symmetry /
definiteness properties that Eq. 1 fixes."""
import numpy as np
import pytest

from oracle import chi0_from_pairs, chi0_rows, freq_factor, rel_fro


def _rand_M(n_p, n_g, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_p, n_g)) + 1j * rng.standard_normal((n_p, n_g))) / np.sqrt(2 * n_g)


def _energies(n_p, seed=1):
    rng = np.random.default_rng(seed)
    Ev = rng.uniform(-0.25, 0.0, n_p)
    Ec = rng.uniform(0.17, 2.2, n_p)
    return Ev - Ec


def test_freq_factor_closed_forms():
    dE = _energies(50)
    w = np.random.default_rng(2).uniform(0.5, 3.0, 50)
    d = 1e-3
    # static: both terms equal -> w / (dE + i delta)
    f0 = freq_factor(dE, w, [0.0], d)[0]
    assert np.max(np.abs(f0 - w / (dE + 1j * d))) < 1e-13 * np.max(np.abs(f0))
    # imaginary axis, delta = 0: w dE / (dE^2 + nu^2)
    nu = np.array([0.01, 0.3, 2.0])
    fi = freq_factor(dE, w, 1j * nu, 0.0)
    want = w[None] * dE[None] / (dE[None] ** 2 + nu[:, None] ** 2)
    assert np.max(np.abs(fi - want)) < 1e-13 * np.max(np.abs(want))
    # real axis, delta = 0: w dE / (dE^2 - omega^2)
    om = np.array([0.05, 0.1])
    fr = freq_factor(dE, w, om, 0.0)
    want = w[None] * dE[None] / (dE[None] ** 2 - om[:, None] ** 2)
    assert np.max(np.abs(fr - want)) < 1e-12 * np.max(np.abs(want))


def test_chi0_matches_direct_loop():
    nv, nc, ng = 3, 4, 5
    M = _rand_M(nv * nc, ng, 3)
    dE = _energies(nv * nc, 4)
    om = np.array([0.0, 0.2j])
    f = freq_factor(dE, np.ones_like(dE), om, 1e-3)
    chi = chi0_from_pairs(M, f)
    ref = np.zeros_like(chi)
    for iw in range(2):
        for p in range(nv * nc):
            for a in range(ng):
                for b in range(ng):
                    ref[iw, a, b] += f[iw, p] * M[p, a] * np.conj(M[p, b])
    assert rel_fro(chi, ref) < 1e-14


def test_chi0_rows_match_direct_loop():
    """Rows of Eq. 1 against the quadruple loop, with pair blocks that split
    the sum unevenly and rows given out of order (one repeated)."""
    n_p, ng = 13, 7
    M = _rand_M(n_p, ng, 11)
    dE = _energies(n_p, 12)
    f = freq_factor(dE, np.ones_like(dE), np.array([0.0, 0.3j, 0.1]), 1e-3)
    rows = np.array([6, 0, 3, 3])
    got = chi0_rows(M, f, rows, block=5)
    ref = np.zeros((3, rows.size, ng), dtype=np.complex128)
    for iw in range(3):
        for i, a in enumerate(rows):
            for p in range(n_p):
                for b in range(ng):
                    ref[iw, i, b] += f[iw, p] * M[p, a] * np.conj(M[p, b])
    assert np.max(np.abs(got - ref)) < 1e-14 * np.max(np.abs(ref))
    # complex64 input is widened exactly: the same rows as its complex128 copy
    M32 = M.astype(np.complex64)
    assert np.array_equal(chi0_rows(M32, f, rows), chi0_rows(M32.astype(np.complex128), f, rows))


def test_rank_one_single_pair():
    M = _rand_M(1, 12, 5)
    f = freq_factor(np.array([-0.4]), np.array([1.0]), [0.0], 1e-3)
    chi = chi0_from_pairs(M, f)[0]
    ev = np.linalg.eigvals(chi)
    ev = ev[np.argsort(-np.abs(ev))]
    assert abs(ev[0] - f[0, 0] * np.vdot(M[0], M[0]).real) < 1e-14
    assert np.max(np.abs(ev[1:])) < 1e-14
    assert np.linalg.matrix_rank(chi, tol=1e-12) == 1


def test_hermiticity_and_delta_reflection():
    M = _rand_M(40, 9, 6)
    dE = _energies(40, 7)
    om = np.array([0.0, 0.05j, 1.0j])
    chi_p = chi0_from_pairs(M, freq_factor(dE, np.ones(40), om, 1e-3))
    chi_m = chi0_from_pairs(M, freq_factor(dE, np.ones(40), om, -1e-3))
    chi_0 = chi0_from_pairs(M, freq_factor(dE, np.ones(40), om, 0.0))
    for iw in range(3):
        assert rel_fro(chi_0[iw].conj().T, chi_0[iw]) < 1e-14
        assert rel_fro(chi_p[iw].conj().T, chi_m[iw]) < 1e-14
        # delta > 0 breaks Hermiticity
        assert rel_fro(chi_p[iw].conj().T, chi_p[iw]) > 1e-6


def test_negative_semidefinite_static_and_imaginary_axis():
    M = _rand_M(60, 8, 8)
    dE = _energies(60, 9)
    nus = np.array([0.0, 0.01, 0.1, 0.5, 2.0])
    chi = chi0_from_pairs(M, freq_factor(dE, np.ones(60), 1j * nus, 0.0))
    for iw in range(nus.size):
        ev = np.linalg.eigvalsh(chi[iw])
        assert ev.max() < 1e-14 * abs(ev.min())
    diag = np.abs(np.diagonal(chi, axis1=1, axis2=2))     # [n_freq][N_G]
    assert np.all(np.diff(diag, axis=0) < 0)              # |chi_GG| falls with nu
    # delta > 0 at omega = 0: both Hermitian parts are negative semidefinite
    chd = chi0_from_pairs(M, freq_factor(dE, np.ones(60), [0.0], 1e-2))[0]
    herm = 0.5 * (chd + chd.conj().T)
    anti = (chd - chd.conj().T) / 2j
    assert np.linalg.eigvalsh(herm).max() < 1e-13
    assert np.linalg.eigvalsh(anti).max() < 1e-13


@pytest.mark.parametrize("block", [1, 7, 4096])
def test_linearity_over_pair_blocks(block):
    M = _rand_M(30, 6, 10)
    dE = _energies(30, 11)
    f = freq_factor(dE, np.ones(30), [0.0, 0.3j], 1e-3)
    whole = chi0_from_pairs(M, f, block=block)
    parts = chi0_from_pairs(M[:11], f[:, :11]) + chi0_from_pairs(M[11:], f[:, 11:])
    assert rel_fro(parts, whole) < 1e-14


def test_k_point_sum_is_the_triple_loop():
    """Eq. 1's sum over k: chi0_k_points equals the direct loop over (k, v, c)
    on a tiny case, and its k = 0 term is the single-k chi0."""
    from oracle import chi0_full, chi0_k_points, pair_elements, wfn_to_grid
    from synth import make_problem
    prob = make_problem("c1", n_G=[20], n_imag=1)
    vb, cb = np.arange(2), np.arange(3)
    got = chi0_k_points(prob, 0, 2, v_bands=vb, c_bands=cb)
    ref = np.zeros_like(got)
    for ik in range(2):
        u_v = wfn_to_grid(prob.coeff_v(0, vb, ik=ik), prob.gw, prob.n)
        u_c = wfn_to_grid(prob.coeff_c(cb, ik=ik), prob.gw, prob.n)
        M = pair_elements(u_v, u_c, prob.gvec[0], prob.n).reshape(2, 3, -1)
        for iv in range(2):
            for ic in range(3):
                dE = prob.E_v[iv] - prob.E_c_k(ik)[ic]
                for iw, om in enumerate(prob.omega):
                    f = 0.5 * (1 / (dE - om + 1j * prob.delta) + 1 / (dE + om + 1j * prob.delta))
                    ref[iw] += f * np.outer(M[iv, ic], M[iv, ic].conj())
    assert rel_fro(got, ref) < 1e-14
    one = chi0_k_points(prob, 0, 1, v_bands=vb, c_bands=cb)
    assert rel_fro(one, chi0_full(prob, 0, v_bands=vb, c_bands=cb)) < 1e-15
    # the second k-point brings different states (not a copy of the first)
    assert rel_fro(got - one, one) > 0.1
