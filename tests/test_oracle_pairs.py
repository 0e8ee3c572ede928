"""Pins of the oracle's wavefunction and pair-matrix-element code (text after
Eq. 1) against brute force, Parseval, closure and plane-wave special cases."""
import numpy as np
import pytest

from oracle import pair_elements, wfn_to_grid
from synth import band_coefficients, pw_sphere


def _direct_grid(coeff, gw, n, pts):
    out = []
    for j in pts:
        ph = np.exp(2j * np.pi * (gw @ np.asarray(j)) / n)
        out.append(coeff @ ph)
    return np.array(out).T


def test_wfn_to_grid_matches_direct_sum():
    n = 8
    gw = pw_sphere(n, 5.0)
    c = band_coefficients(11, 0, [0, 1, 2], gw.shape[0])
    u = wfn_to_grid(c, gw, n)
    pts = [(0, 0, 0), (1, 2, 3), (7, 0, 5), (3, 3, 3), (6, 1, 4)]
    ref = _direct_grid(c, gw, n, pts)
    got = np.stack([u[:, a, b, d] for (a, b, d) in pts], 1)
    assert np.max(np.abs(got - ref)) < 1e-13
    # normalised bands: mean |u|^2 over the grid is 1
    assert np.allclose(np.mean(np.abs(u) ** 2, axis=(1, 2, 3)), 1.0, atol=1e-13)


def _direct_M(uv, uc, G, n):
    j = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij"), -1).reshape(-1, 3)
    rho = (np.conj(uv) * uc).reshape(-1)
    return np.array([np.sum(rho * np.exp(2j * np.pi * (j @ g) / n)) / n ** 3 for g in G])


def test_pair_elements_match_direct_real_space_sum():
    n = 8
    gw = pw_sphere(n, 3.0)
    cv = band_coefficients(5, 1, [0, 1], gw.shape[0])
    cc = band_coefficients(5, 0, [0, 1, 2], gw.shape[0])
    uv, uc = wfn_to_grid(cv, gw, n), wfn_to_grid(cc, gw, n)
    G = np.array([[0, 0, 0], [1, 0, 0], [0, -1, 2], [-3, 2, 1], [2, 2, -2]], dtype=np.int32)
    M = pair_elements(uv, uc, G, n)
    for iv in range(2):
        for ic in range(3):
            ref = _direct_M(uv[iv], uc[ic], G, n)
            assert np.max(np.abs(M[iv * 3 + ic] - ref)) < 1e-14


def test_pair_elements_match_gspace_convolution():
    # alias-free: n > 2 R_w + R_G  (R_w = sqrt(6) ~ 2.45, R_G = sqrt(3))
    n = 12
    gw = pw_sphere(n, 6.0)
    cv = band_coefficients(7, 1, [0, 1, 2], gw.shape[0])
    cc = band_coefficients(7, 0, [0, 1], gw.shape[0])
    uv, uc = wfn_to_grid(cv, gw, n), wfn_to_grid(cc, gw, n)
    G = pw_sphere(n, 3.0)
    M = pair_elements(uv, uc, G, n)
    index = {tuple(g): k for k, g in enumerate(gw)}
    for iv in range(3):
        for ic in range(2):
            ref = np.zeros(G.shape[0], dtype=np.complex128)
            for jg, g in enumerate(G):
                s = 0j
                for k, gp in enumerate(gw):
                    kk = index.get(tuple(gp + g))
                    if kk is not None:
                        s += np.conj(cv[iv, kk]) * cc[ic, k]
                ref[jg] = s
            assert np.max(np.abs(M[iv * 2 + ic] - ref)) < 1e-14


def test_parseval_full_grid_and_sphere_bound():
    n = 10
    gw = pw_sphere(n, 4.0)
    cv = band_coefficients(3, 1, [0, 1], gw.shape[0])
    cc = band_coefficients(3, 0, [0, 1], gw.shape[0])
    uv, uc = wfn_to_grid(cv, gw, n), wfn_to_grid(cc, gw, n)
    ax = np.arange(n) - n // 2
    full = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    M = pair_elements(uv, uc, full, n)
    small = pair_elements(uv, uc, pw_sphere(n, 5.0), n)
    for iv in range(2):
        for ic in range(2):
            p = iv * 2 + ic
            rhs = np.mean(np.abs(uv[iv]) ** 2 * np.abs(uc[ic]) ** 2)
            assert abs(np.sum(np.abs(M[p]) ** 2) - rhs) < 1e-13 * rhs
            assert np.sum(np.abs(small[p]) ** 2) <= rhs
            # Cauchy-Schwarz for normalised bands: |M| <= 1
            assert np.max(np.abs(M[p])) <= 1.0 + 1e-14


def test_closure_complete_band_set():
    # a complete orthonormal set over the wavefunction sphere (unitary matrix rows)
    n = 12
    gw = pw_sphere(n, 2.0)
    npw = gw.shape[0]
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((npw, npw)) + 1j * rng.standard_normal((npw, npw)))
    bands = Q.T                      # row n = band n; rows orthonormal, columns complete
    cv = band_coefficients(9, 1, [0], npw)
    uv = wfn_to_grid(cv, gw, n)
    un = wfn_to_grid(bands, gw, n)
    G = pw_sphere(n, 2.0)
    M = pair_elements(uv, un, G, n)            # [npw][N_G]
    lhs = M.T @ M.conj()                       # sum_n M_vn(G) conj(M_vn(G'))
    index = {tuple(g): k for k, g in enumerate(gw)}
    rhs = np.zeros_like(lhs)
    for a, Ga in enumerate(G):
        for b, Gb in enumerate(G):
            s = 0j
            for g in gw:
                ka, kb = index.get(tuple(g + Ga)), index.get(tuple(g + Gb))
                if ka is not None and kb is not None:
                    s += np.conj(cv[0, ka]) * cv[0, kb]
            rhs[a, b] = s
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_single_plane_wave_pair_is_kronecker_delta():
    n = 8
    gw = pw_sphere(n, 3.0)
    npw = gw.shape[0]
    a, b = 3, 11
    cv = np.zeros((1, npw), complex)
    cc = np.zeros((1, npw), complex)
    cv[0, a] = 1.0
    cc[0, b] = 1.0
    G = pw_sphere(n, 8.0)
    M = pair_elements(wfn_to_grid(cv, gw, n), wfn_to_grid(cc, gw, n), G, n)[0]
    want = np.array([1.0 if tuple(g) == tuple(gw[a] - gw[b]) else 0.0 for g in G])
    assert want.sum() == 1.0
    assert np.max(np.abs(M - want)) < 1e-15


@pytest.mark.parametrize("c_block", [1, 3, 64])
def test_pair_order_is_valence_major(c_block):
    n = 6
    gw = pw_sphere(n, 2.0)
    uv = wfn_to_grid(band_coefficients(1, 1, [0, 1], gw.shape[0]), gw, n)
    uc = wfn_to_grid(band_coefficients(1, 0, [0, 1, 2], gw.shape[0]), gw, n)
    G = pw_sphere(n, 1.0)
    M = pair_elements(uv, uc, G, n, c_block=c_block)
    one = pair_elements(uv[1:2], uc[2:3], G, n)
    assert np.array_equal(M[1 * 3 + 2], one[0])
