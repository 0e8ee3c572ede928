"""Pins of the oracle's dielectric functions (eps = 1 - v chi0 of section II,
eps_inf of Table III) against textbook lattice facts, closed-form inverses,
brute force on tiny matrices, the Schur-complement route to the head of the
inverse and the local-field inequality that a static chi0 fixes."""
import numpy as np
import pytest

from oracle import chi0_from_pairs, freq_factor, rel_fro
from oracle.dielectric import coulomb, eps_inf, epsilon, epsilon_inverse, reciprocal_lattice


def _chi0(n_p=80, n_g=9, omega=(0.0, 0.3j), delta=1e-3, seed=0):
    rng = np.random.default_rng(seed)
    M = (rng.standard_normal((n_p, n_g)) + 1j * rng.standard_normal((n_p, n_g))) / np.sqrt(2 * n_g)
    dE = rng.uniform(-0.25, 0.0, n_p) - rng.uniform(0.17, 2.2, n_p)
    return chi0_from_pairs(M, freq_factor(dE, np.ones(n_p), np.asarray(omega), delta))


def test_coulomb_fcc_textbook_reciprocal_vectors():
    """FCC primitive cell a/2 (0,1,1), ...: b = (2 pi / a) (-1,1,1), ...,
    Omega = a^3 / 4 (textbook values, not derived from the oracle's route)."""
    a = 7.96
    A = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=float)
    B_text = (2 * np.pi / a) * np.array([[-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=float)
    assert np.allclose(reciprocal_lattice(A), B_text, rtol=0, atol=1e-13)
    g = np.array([[1, 0, 0], [0, 0, 0], [1, 1, 1], [-1, 2, 0]], dtype=np.int32)
    q = np.array([0.0, 0.0, 0.25])
    v = coulomb(q, g, A)
    k = (g + q) @ B_text
    want = 4 * np.pi / ((a ** 3 / 4) * (k * k).sum(1))
    assert np.allclose(v, want, rtol=1e-14, atol=0)
    # G = b1 at q = 0: |b1|^2 = 3 (2 pi / a)^2  ->  v = 4 / (3 pi a)
    assert abs(coulomb(np.zeros(3), g[:1], A)[0] - 4 / (3 * np.pi * a)) < 1e-15


def test_coulomb_simple_cubic_and_symmetry():
    a = 15.92
    A = a * np.eye(3)
    g = np.array([[0, 0, 0], [1, 0, 0], [0, -1, 0], [2, 1, -1]], dtype=np.int32)
    q = np.array([0.001 * a / (2 * np.pi), 0.0, 0.0])
    v = coulomb(q, g, A)
    # v(q) of the head: 4 pi / (a^3 q^2) with q = 0.001 bohr^-1
    assert abs(v[0] / (4 * np.pi / (a ** 3 * 1e-6)) - 1) < 1e-12
    # inversion: v(q + G) = v(-q - G)
    assert np.allclose(coulomb(-q, -g, A), v, rtol=1e-15)
    kk = ((g + q) * (2 * np.pi / a)) ** 2
    assert np.all(np.argsort(v) == np.argsort(-kk.sum(1)))


def test_epsilon_identity_and_similarity():
    chi = _chi0()
    v = np.random.default_rng(3).uniform(0.1, 5.0, chi.shape[-1])
    assert np.array_equal(epsilon(np.zeros_like(chi), v), np.broadcast_to(np.eye(9), chi.shape))
    ep, es = epsilon(chi, v), epsilon(chi, v, symmetric=True)
    for iw in range(chi.shape[0]):
        # eps_sym = V^-1/2 eps V^1/2: same spectrum, same diagonal of the inverse
        s = np.sqrt(v)
        assert rel_fro(es[iw], ep[iw] * s[None, :] / s[:, None]) < 1e-14
        e1 = np.sort_complex(np.linalg.eigvals(ep[iw]))
        e2 = np.sort_complex(np.linalg.eigvals(es[iw]))
        assert np.max(np.abs(e1 - e2)) < 1e-12 * np.max(np.abs(e1))
    ip, is_ = epsilon_inverse(ep), epsilon_inverse(es)
    assert np.max(np.abs(np.diagonal(ip, axis1=1, axis2=2) - np.diagonal(is_, axis1=1, axis2=2))) < 1e-13
    assert np.allclose(eps_inf(ip), eps_inf(is_), rtol=1e-13)


def test_inverse_brute_force_adjugate_3x3():
    rng = np.random.default_rng(4)
    E = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)) + 3 * np.eye(3)
    det = (E[0, 0] * (E[1, 1] * E[2, 2] - E[1, 2] * E[2, 1])
           - E[0, 1] * (E[1, 0] * E[2, 2] - E[1, 2] * E[2, 0])
           + E[0, 2] * (E[1, 0] * E[2, 1] - E[1, 1] * E[2, 0]))
    adj = np.empty((3, 3), dtype=complex)
    for i in range(3):
        for j in range(3):
            m = np.delete(np.delete(E, j, 0), i, 1)       # cofactor of (j, i): transpose
            adj[i, j] = (-1) ** (i + j) * (m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0])
    assert rel_fro(epsilon_inverse(E[None])[0], adj / det) < 1e-14


def test_inverse_rank_one_sherman_morrison():
    """chi0 of a single pair is c u u^H; eps = I - c (V u) u^H has the inverse
    I + c (V u) u^H / (1 - c u^H V u)."""
    rng = np.random.default_rng(5)
    n = 11
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    c = -0.7 + 0.002j
    v = rng.uniform(0.2, 3.0, n)
    chi = (c * np.outer(u, u.conj()))[None]
    want = np.eye(n) + c * np.outer(v * u, u.conj()) / (1 - c * np.vdot(u, v * u))
    assert rel_fro(epsilon_inverse(epsilon(chi, v))[0], want) < 1e-13


def test_head_schur_complement_and_one_by_one():
    """1 / [eps^-1]_00 = eps_00 - eps_0r eps_rr^-1 eps_r0 (a linear solve, not an
    inverse); for N_G = 1 it is eps_00 = 1 - v chi0_00."""
    chi = _chi0(n_g=13, omega=(0.0, 0.1j, 1.0j))
    v = np.random.default_rng(6).uniform(0.1, 8.0, 13)
    eps = epsilon(chi, v)
    got = eps_inf(epsilon_inverse(eps))
    for iw in range(eps.shape[0]):
        e = eps[iw]
        want = e[0, 0] - e[0, 1:] @ np.linalg.solve(e[1:, 1:], e[1:, 0])
        assert abs(got[iw] - want) < 1e-13 * abs(want)
    one = chi[:, :1, :1]
    assert np.allclose(eps_inf(epsilon_inverse(epsilon(one, v[:1]))), 1 - v[0] * one[:, 0, 0], rtol=1e-14)


def test_local_fields_lower_eps_inf_for_static_chi0():
    """Static chi0 (delta = 0) is Hermitian negative semidefinite, so the
    symmetrised eps is Hermitian with eigenvalues >= 1 and, by the Schur
    complement, 1/[eps^-1]_00 <= eps_00 with equality only when the head row
    decouples."""
    chi = _chi0(n_g=10, omega=(0.0,), delta=0.0)
    v = np.random.default_rng(7).uniform(0.5, 20.0, 10)
    es = epsilon(chi, v, symmetric=True)[0]
    assert rel_fro(es, es.conj().T) < 1e-14
    assert np.linalg.eigvalsh(es).min() >= 1 - 1e-12
    e_inf = eps_inf(epsilon_inverse(es[None]))[0]
    assert abs(e_inf.imag) < 1e-12 * abs(e_inf)
    assert e_inf.real < es[0, 0].real
    # decoupled head: chi0_0G = 0 for G != 0 -> equality
    chd = chi.copy()
    chd[0, 0, 1:] = 0
    chd[0, 1:, 0] = 0
    ed = epsilon(chd, v, symmetric=True)
    assert abs(eps_inf(epsilon_inverse(ed))[0] - ed[0, 0, 0]) < 1e-13 * abs(ed[0, 0, 0])


@pytest.mark.parametrize("symmetric", [False, True])
def test_inverse_residual_on_eq1_chi0(symmetric):
    chi = _chi0(n_p=300, n_g=40, omega=(0.0, 0.05j, 2.0j))
    v = np.random.default_rng(8).uniform(0.1, 4.0, 40)
    eps = epsilon(chi, v, symmetric=symmetric)
    inv = epsilon_inverse(eps)
    for iw in range(eps.shape[0]):
        assert rel_fro(eps[iw] @ inv[iw], np.eye(40)) < 1e-13
