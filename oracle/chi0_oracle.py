"""FP64 CPU oracle: pair matrix elements, Eq. 1 (full band sum), Eq. 3/Eq. 4
(accelerated conduction-band summation) and the adjoint of Eq. 1.

TEST INFRASTRUCTURE ONLY.  Slow, plain NumPy/SciPy in complex128, written to
be checked against the paper by eye.  Imported only by tests, by the smoke
check and by the CPU-baseline legs of the benchmark; the library path never
calls it and it imports nothing from the CUDA package.

Conventions (shared with the library only through its documented interface):
* grid arrays are [band][i1][i2][i3] with i3 fastest; r_j = j/n per axis;
* G vectors are integer triples (units of the reciprocal lattice vectors);
* a pair index is p = iv * n_c + ic (valence-major) over the chosen bands;
* chi0 is stored [n_freq][N_G][N_G] complex128.

Parity status per function: every public function is pinned by
tests/test_oracle_*.py except `accelerated_pairs` and `full_pairs`, which
only reorder inputs (index bookkeeping checked by brute force in the tests).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

_WORKERS = -1  # all host cores for scipy.fft


# --------------------------------------------------------------------------
# wavefunctions and pair matrix elements (text after Eq. 1: M_vc(k,q,G) is the
# matrix element of exp(i(q+G).r) between <v,k+q| and |c,k>; plane-wave basis
# of the computational-details paragraph)
# --------------------------------------------------------------------------
def wfn_to_grid(coeff: np.ndarray, gw: np.ndarray, n: int) -> np.ndarray:
    """u_b(r_j) = sum_g c_b(g) exp(2 pi i g.j / n) on the n^3 grid.

    This is the periodic part of the Bloch function sampled on the FFT grid.
    Written as n^3 * ifftn of the coefficients scattered to (g mod n).
    """
    coeff = np.atleast_2d(np.asarray(coeff, dtype=np.complex128))
    nb = coeff.shape[0]
    grid = np.zeros((nb, n, n, n), dtype=np.complex128)
    i1, i2, i3 = (np.mod(gw[:, k], n) for k in range(3))
    grid[:, i1, i2, i3] = coeff
    return sfft.ifftn(grid, axes=(1, 2, 3), workers=_WORKERS) * float(n ** 3)


def pair_elements(u_v: np.ndarray, u_c: np.ndarray, gvec: np.ndarray, n: int,
                  c_block: int = 64) -> np.ndarray:
    """M_vc(G) = <v,k+q| exp(i(q+G).r) |c,k> for all (v, c), p = iv*n_c + ic.

    With psi_nk = exp(i k.r) u_nk the phases exp(i(k+q).r) cancel, leaving
    M_vc(G) = (1/N_r) sum_r conj(u_v(r)) u_c(r) exp(+i G.r), which is
    numpy's ifftn of the pair product read at (G mod n).
    """
    u_v = np.atleast_2d(u_v.reshape(-1, n, n, n)) if u_v.ndim != 4 else u_v
    u_c = np.atleast_2d(u_c.reshape(-1, n, n, n)) if u_c.ndim != 4 else u_c
    nv, nc = u_v.shape[0], u_c.shape[0]
    g = np.mod(gvec, n)
    out = np.empty((nv, nc, gvec.shape[0]), dtype=np.complex128)
    for iv in range(nv):
        cv = np.conj(u_v[iv])
        for c0 in range(0, nc, c_block):
            rho = cv[None] * u_c[c0:c0 + c_block]
            F = sfft.ifftn(rho, axes=(1, 2, 3), workers=_WORKERS)
            out[iv, c0:c0 + c_block] = F[:, g[:, 0], g[:, 1], g[:, 2]]
    return out.reshape(nv * nc, gvec.shape[0])


# --------------------------------------------------------------------------
# Eq. 1: energy-denominator factor and the band-pair contraction
# --------------------------------------------------------------------------
def freq_factor(dE: np.ndarray, w: np.ndarray, omega: np.ndarray, delta: float) -> np.ndarray:
    """f_p(omega) = (w_p/2) [1/(dE_p - omega + i delta) + 1/(dE_p + omega + i delta)].

    Eq. 1 with dE_p = E_v(k+q) - E_c(k); w_p = 1 for an explicit band pair and
    g(E_i) dE_i for an energy-grid point of Eq. 4.  Shape [n_freq][n_pairs].
    """
    dE = np.asarray(dE, dtype=np.float64)[None, :]
    w = np.asarray(w, dtype=np.float64)[None, :]
    om = np.atleast_1d(np.asarray(omega, dtype=np.complex128))[:, None]
    return 0.5 * w * (1.0 / (dE - om + 1j * delta) + 1.0 / (dE + om + 1j * delta))


def chi0_from_pairs(M: np.ndarray, f: np.ndarray, block: int = 4096) -> np.ndarray:
    """chi0_{G,G'}(omega) = sum_p f_p(omega) M_p(G) conj(M_p(G'))  (Eq. 1).

    M is [n_pairs][N_G]; f is [n_freq][n_pairs].  Summed over pair blocks of
    at most `block` pairs with a ZGEMM each, in FP64.
    """
    M = np.asarray(M, dtype=np.complex128)
    f = np.atleast_2d(np.asarray(f, dtype=np.complex128))
    nG = M.shape[1]
    chi = np.zeros((f.shape[0], nG, nG), dtype=np.complex128)
    for p0 in range(0, M.shape[0], block):
        Mb = M[p0:p0 + block]
        Mc = Mb.conj()
        for iw in range(f.shape[0]):
            chi[iw] += (Mb.T * f[iw, p0:p0 + block][None, :]) @ Mc
    return chi


def chi0_rows(M: np.ndarray, f: np.ndarray, rows, block: int = 4096) -> np.ndarray:
    """Rows G in `rows` of Eq. 1: chi0_{G,G'}(omega) = sum_p f_p(omega) M_p(G)
    conj(M_p(G')) for every G' -> [n_freq][len(rows)][N_G], in FP64.

    For checking chi0 of sizes whose full matrix the host cannot form in
    reasonable time; summed over pair blocks of at most `block` pairs.
    """
    M = np.asarray(M)
    f = np.atleast_2d(np.asarray(f, dtype=np.complex128))
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((f.shape[0], rows.size, M.shape[1]), dtype=np.complex128)
    for p0 in range(0, M.shape[0], block):
        Mb = np.asarray(M[p0:p0 + block], dtype=np.complex128)
        Mc = Mb.conj()
        Mr = Mb[:, rows].T
        for iw in range(f.shape[0]):
            out[iw] += (Mr * f[iw, p0:p0 + block][None, :]) @ Mc
    return out


# --------------------------------------------------------------------------
# Eq. 3 / Eq. 4: accelerated conduction-band summation
# --------------------------------------------------------------------------
def dos(E, A: float, V0: float):
    """Free-electron density of states g(E) = A sqrt(2 (E - V0)), zero below V0.

    Eq. 3's g(E) = (Omega/pi^2) sqrt(2 (E - V_xc(0))) with the prefactor
    Omega/pi^2 passed in as A (bands per Hartree for the synthetic data).
    """
    E = np.asarray(E, dtype=np.float64)
    return A * np.sqrt(np.maximum(2.0 * (E - V0), 0.0))


def select_accelerated(E_c: np.ndarray, N0: int, dE: float, A: float, V0: float,
                       E_max: float) -> dict:
    """Bands and weights of Eq. 3 evaluated with the quadrature of Eq. 4.

    * explicit part: conduction bands 1..N0 (0-based 0..N0-1), weight 1;
    * E_0 is the energy of band N0; the integral runs over (E_0, E_max] on a
      uniform grid of step dE (last interval clipped at E_max), so
      N_E = ceil((E_max - E_0)/dE);
    * E_i is the midpoint of interval i and dE_i its width; the state standing
      for E_i is the conduction band above N0 nearest in energy to E_i (ties
      go to the lower band index); its weight is g(E_i) dE_i and its energy
      denominator uses E_i.
    Returns dict(explicit, rep, E_i, dE_i, w_i, edges, E0).
    """
    E_c = np.asarray(E_c, dtype=np.float64)
    n_c = E_c.size
    if np.any(np.diff(E_c) < 0):
        raise ValueError("conduction energies must be sorted ascending")
    N0 = int(min(max(N0, 0), n_c))
    explicit = np.arange(N0, dtype=np.int64)
    if N0 == 0 or N0 >= n_c or dE <= 0:
        empty = np.zeros(0)
        return dict(explicit=explicit, rep=np.zeros(0, np.int64), E_i=empty, dE_i=empty,
                    w_i=empty, edges=empty, E0=E_c[N0 - 1] if N0 > 0 else V0)
    E0 = E_c[N0 - 1]
    span = E_max - E0
    N_E = max(int(math.ceil(span / dE - 1e-12)), 0)
    edges = np.minimum(E0 + dE * np.arange(N_E + 1), E_max)
    lo, hi = edges[:-1], edges[1:]
    E_i = 0.5 * (lo + hi)
    dE_i = hi - lo
    above = E_c[N0:]
    rep = np.array([N0 + int(np.argmin(np.abs(above - e))) for e in E_i], dtype=np.int64)
    w_i = dos(E_i, A, V0) * dE_i
    return dict(explicit=explicit, rep=rep, E_i=E_i, dE_i=dE_i, w_i=w_i, edges=edges, E0=E0)


def full_pairs(E_v: np.ndarray, E_c: np.ndarray):
    """Pair set of Eq. 1: every (v, c), dE = E_v - E_c, w = 1 (p = iv*n_c + ic)."""
    c_idx = np.arange(E_c.size, dtype=np.int64)
    Ecol = np.asarray(E_c, dtype=np.float64)
    wcol = np.ones(E_c.size)
    dE = (np.asarray(E_v)[:, None] - Ecol[None, :]).reshape(-1)
    w = np.broadcast_to(wcol[None, :], (E_v.size, E_c.size)).reshape(-1)
    return c_idx, Ecol, wcol, dE, w


def accelerated_pairs(E_v: np.ndarray, E_c: np.ndarray, sel: dict):
    """Pair set of Eq. 3/4: columns are the N0 explicit bands, then one state
    per energy-grid point; the column energy is E_c for explicit bands and E_i
    for grid points, the column weight 1 and g(E_i) dE_i respectively."""
    c_idx = np.concatenate([sel["explicit"], sel["rep"]]).astype(np.int64)
    Ecol = np.concatenate([np.asarray(E_c)[sel["explicit"]], sel["E_i"]])
    wcol = np.concatenate([np.ones(sel["explicit"].size), sel["w_i"]])
    dE = (np.asarray(E_v)[:, None] - Ecol[None, :]).reshape(-1)
    w = np.broadcast_to(wcol[None, :], (E_v.size, c_idx.size)).reshape(-1)
    return c_idx, Ecol, wcol, dE, w


def grid_energy_of_bands(E_c: np.ndarray, N0: int, dE: float, E_max: float) -> np.ndarray:
    """The energy each conduction band carries in Eq. 3 with the grid of Eq. 4.

    Bands 1..N0 (0-based 0..N0-1) keep their own energy.  A band above N0
    takes the midpoint E_i of the Eq. 4 step [e_k, e_{k+1}) that holds its
    energy, with the steps of select_accelerated (uniform from E_0, the last
    one clipped at E_max); the last step is closed and also collects energies
    above E_max, the first collects any below E_0.
    """
    E_c = np.asarray(E_c, dtype=np.float64)
    out = E_c.copy()
    sel = select_accelerated(E_c, N0, dE, 1.0, 0.0, E_max)   # A, V0 only enter the weights
    edges = sel["edges"]
    if edges.size < 2:
        return out
    N0 = int(N0)
    k = np.searchsorted(edges, E_c[N0:], side="right") - 1  # last edge <= E_c
    k = np.clip(k, 0, edges.size - 2)
    out[N0:] = sel["E_i"][k]
    return out


def energy_substitution_estimate(E_c: np.ndarray, grad_E_c: np.ndarray, N0: int, dE: float,
                                 E_max: float) -> float:
    """First-order change of a loss L when every band above N0 is given its
    Eq. 4 grid energy in the denominators of Eq. 1 (the energy-substitution
    part of the accelerated sum's error):  sum_c dL/dE_c (E_i(c) - E_c),
    with dL/dE_c from the adjoint (chi0_grad)."""
    E_c = np.asarray(E_c, dtype=np.float64)
    return float(np.sum(np.asarray(grad_E_c, dtype=np.float64) * (grid_energy_of_bands(E_c, N0, dE, E_max) - E_c)))


def chi0_full(prob, iq: int = 0, coeff_v=None, coeff_c=None, v_bands=None, c_bands=None):
    """chi0 of Eq. 1 for q-point iq over the given bands (default: all)."""
    v_bands = np.arange(prob.n_v) if v_bands is None else np.asarray(v_bands)
    c_bands = np.arange(prob.n_c) if c_bands is None else np.asarray(c_bands)
    cv = prob.coeff_v(iq, v_bands) if coeff_v is None else coeff_v
    cc = prob.coeff_c(c_bands) if coeff_c is None else coeff_c
    u_v = wfn_to_grid(cv, prob.gw, prob.n)
    u_c = wfn_to_grid(cc, prob.gw, prob.n)
    M = pair_elements(u_v, u_c, prob.gvec[iq], prob.n)
    dE = (prob.E_v[v_bands][:, None] - prob.E_c[c_bands][None, :]).reshape(-1)
    f = freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta)
    return chi0_from_pairs(M, f)


def chi0_k_points(prob, iq: int = 0, n_k: int = 2, v_bands=None, c_bands=None):
    """Eq. 1 with its sum over k written out: chi0 = sum_k chi0_k, where chi0_k
    pairs the valence set at k + q with the conduction set at k (energies
    prob.E_v and prob.E_c_k(k))."""
    v_bands = np.arange(prob.n_v) if v_bands is None else np.asarray(v_bands)
    c_bands = np.arange(prob.n_c) if c_bands is None else np.asarray(c_bands)
    total = 0
    for ik in range(n_k):
        u_v = wfn_to_grid(prob.coeff_v(iq, v_bands, ik=ik), prob.gw, prob.n)
        u_c = wfn_to_grid(prob.coeff_c(c_bands, ik=ik), prob.gw, prob.n)
        M = pair_elements(u_v, u_c, prob.gvec[iq], prob.n)
        dE = (prob.E_v[v_bands][:, None] - prob.E_c_k(ik)[c_bands][None, :]).reshape(-1)
        total = total + chi0_from_pairs(M, freq_factor(dE, np.ones_like(dE), prob.omega, prob.delta))
    return total


def chi0_accelerated(prob, iq: int = 0, N0=None, dE=None, coeff_v=None):
    """chi0 of Eq. 3 with the integral done by Eq. 4 (frequency factor of Eq. 1
    with E_c replaced by the grid energy E_i for the integration states)."""
    N0 = prob.N0 if N0 is None else N0
    dE = prob.dE if dE is None else dE
    sel = select_accelerated(prob.E_c, N0, dE, prob.dos_A, prob.dos_V0, prob.E_max)
    c_idx, Ecol, wcol, dEp, wp = accelerated_pairs(prob.E_v, prob.E_c, sel)
    cv = prob.coeff_v(iq) if coeff_v is None else coeff_v
    uniq, inv = np.unique(c_idx, return_inverse=True)
    u_v = wfn_to_grid(cv, prob.gw, prob.n)
    u_c = wfn_to_grid(prob.coeff_c(uniq), prob.gw, prob.n)[inv]
    M = pair_elements(u_v, u_c, prob.gvec[iq], prob.n)
    f = freq_factor(dEp, wp, prob.omega, prob.delta)
    return chi0_from_pairs(M, f), sel


# --------------------------------------------------------------------------
# adjoint of Eq. 1
# --------------------------------------------------------------------------
def chi0_grad(M: np.ndarray, dE: np.ndarray, w: np.ndarray, omega, delta: float,
              Gamma: np.ndarray):
    """Gradients of a real loss L(chi0) given Gamma = dL/dRe chi0 + i dL/dIm chi0.

    chi0 = sum_p f_p M_p M_p^H (Eq. 1), so with complex gradients in the
    (dL/dRe + i dL/dIm) convention:
      grad M_p   = conj(f_p) Gamma M_p + f_p Gamma^H M_p       (summed over omega)
      grad dE_p  = Re( f'_p * conj(M_p^H Gamma M_p) ),
      f'_p       = -(w_p/2) [ (dE_p - omega + i delta)^-2 + (dE_p + omega + i delta)^-2 ].
    Gamma is [n_freq][N_G][N_G]; returns (grad_M [n_pairs][N_G], grad_dE [n_pairs]).
    """
    M = np.asarray(M, dtype=np.complex128)
    om = np.atleast_1d(np.asarray(omega, dtype=np.complex128))
    f = freq_factor(dE, w, om, delta)
    d = np.asarray(dE, dtype=np.float64)[None, :]
    fp = -0.5 * np.asarray(w, dtype=np.float64)[None, :] * (
        (d - om[:, None] + 1j * delta) ** -2 + (d + om[:, None] + 1j * delta) ** -2)
    gM = np.zeros_like(M)
    gd = np.zeros(M.shape[0])
    for iw in range(om.size):
        G = Gamma[iw]
        GM = M @ G.T                 # row p: (Gamma M_p)^T
        GHM = M @ G.conj()           # row p: (Gamma^H M_p)^T
        gM += np.conj(f[iw])[:, None] * GM + f[iw][:, None] * GHM
        quad = np.sum(M.conj() * GM, axis=1)      # M_p^H Gamma M_p
        gd += np.real(fp[iw] * np.conj(quad))
    return gM, gd


def loss_diag(chi: np.ndarray, wG: np.ndarray, iw: int = 0) -> float:
    """L = sum_G Re(w_G chi0_GG(omega_iw))."""
    return float(np.sum(np.real(wG * np.diagonal(chi[iw]))))


def rel_fro(a, b) -> float:
    """||a - b||_F / ||b||_F."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))
