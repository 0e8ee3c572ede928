"""FP64 CPU oracle for the Coulomb-hole (COH) self-energy of Eq. 2 with the
Hybertsen-Louie generalised plasmon-pole (HL-GPP) model that the paper uses to
extend the static dielectric matrix to finite frequencies (computational
details), and its accelerated band sum (the same split as Eq. 3 / Eq. 4).

TEST INFRASTRUCTURE ONLY (same rules as chi0_oracle).

Readings (the paper prints Eq. 2 and names HL-GPP; the model's formulas are
those of the plasmon-pole literature, restated here):
* eps^-1_{GG'}(q, w) = delta_{GG'} + Omega2_{GG'} / (w^2 - wt2_{GG'}), with
  Omega2_{GG'} = w_p^2 [(q+G).(q+G') / |q+G|^2] rho(G - G') / rho(0),
  wt2_{GG'}    = Omega2_{GG'} / (delta_{GG'} - eps^-1_{GG'}(q, 0)),
  w_p^2 = 4 pi N_el / Omega (Hartree units) and eps^-1 the inverse of the
  plain eps = 1 - v chi0 (v(q+G) on the row), so the model reproduces
  eps^-1(q, 0) exactly; wt = sqrt(wt2) on the principal branch (complex when
  eps^-1 is); elements with Omega2 = 0 or delta - eps^-1 = 0 carry no pole;
* with that model the frequency integral of Eq. 2 is done in closed form
  (the retarded minus advanced inverse is -i pi (Omega2 / wt) delta(E' - wt)
  for E' > 0), giving
    Sigma_COH^{nn'}(E) = sum_{n''} sum_{GG'} M*_{n''n}(-G) M_{n''n'}(-G')
                         Omega2_{GG'} v(q+G') / (2 wt_{GG'} (E - E_{n''} - wt_{GG'} + i delta));
  with m_{n n''}(G) = <n| e^{iG.r} |n''> (the pair elements of chi0_pairs with
  the target band first) M*_{n''n}(-G) = m_{nn''}(G), so the diagonal element is
    Sigma_n(E) = sum_{n''} w_{n''} sum_{GG'} m(G) K_{GG'}(E - E_{n''}) conj(m(G')),
    K_{GG'}(x) = Omega2_{GG'} v(q+G') / (2 wt_{GG'} (x - wt_{GG'} + i delta)),
  w_{n''} = 1 for explicit bands and g(E_i) dE_i for an energy-grid state of
  the accelerated sum (whose energy E_{n''} is then E_i);
* electron density n(r) = 2 sum_v |u_v(r)|^2 over the valence set (spin 2),
  rho(G) its Fourier coefficient (n(r) = sum_G rho(G) e^{iG.r}); only the ratio
  rho(G)/rho(0) enters, so no cell normalisation is needed there.

Every function is pinned by tests/test_oracle_coh.py.
"""
from __future__ import annotations

import numpy as np


def density_ratio(u_v: np.ndarray, dvec: np.ndarray) -> np.ndarray:
    """rho(d)/rho(0) for integer vectors d (rows of dvec) from the valence
    grids u_v [n_v][n][n][n]: n(r) = 2 sum_v |u_v|^2,
    rho(d) = (1/N_r) sum_r n(r) exp(-2 pi i d.j/n)."""
    u_v = np.asarray(u_v)
    n = u_v.shape[-1]
    dens = 2.0 * np.sum(np.abs(u_v) ** 2, axis=0)
    F = np.fft.fftn(dens) / dens.size            # F[k] = (1/N) sum_j dens_j exp(-2 pi i k.j / n)
    d = np.mod(np.asarray(dvec, dtype=np.int64), n)
    return F[d[:, 0], d[:, 1], d[:, 2]] / F[0, 0, 0]


def plasma_frequency2(n_el: float, omega_cell: float) -> float:
    """w_p^2 = 4 pi N_el / Omega (Hartree atomic units)."""
    return 4.0 * np.pi * n_el / omega_cell


def gpp_parameters(eps_inv0: np.ndarray, rho_ratio: np.ndarray, kvec: np.ndarray, wp2: float):
    """(Omega2, wt) of the HL-GPP model for one q-point.
    eps_inv0 [N_G][N_G]: inverse of the plain static eps; rho_ratio [N_G][N_G]:
    rho(G - G')/rho(0); kvec [N_G][3]: q + G (cartesian, bohr^-1)."""
    kvec = np.asarray(kvec, dtype=np.float64)
    kk = kvec @ kvec.T                                      # (q+G).(q+G')
    k2 = np.einsum("ij,ij->i", kvec, kvec)
    Omega2 = wp2 * (kk / k2[:, None]) * rho_ratio
    den = np.eye(eps_inv0.shape[0]) - eps_inv0
    with np.errstate(divide="ignore", invalid="ignore"):
        wt2 = np.where(den != 0, Omega2 / np.where(den != 0, den, 1.0), 0.0)
    wt = np.sqrt(wt2.astype(np.complex128))
    return Omega2.astype(np.complex128), wt


def gpp_eps_inv(Omega2: np.ndarray, wt: np.ndarray, w: complex) -> np.ndarray:
    """The model's eps^-1(q, w) = I + Omega2 / (w^2 - wt^2) (elements without a pole: I)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(wt != 0, Omega2 / (w * w - wt * wt), 0.0)
    return np.eye(Omega2.shape[0]) + t


def coh_kernel(Omega2: np.ndarray, wt: np.ndarray, v: np.ndarray, x: float, delta: float) -> np.ndarray:
    """K_{GG'}(x) = Omega2 v(q+G') / (2 wt (x - wt + i delta)), zero without a pole."""
    with np.errstate(divide="ignore", invalid="ignore"):
        K = Omega2 * np.asarray(v)[None, :] / (2.0 * wt * (x - wt + 1j * delta))
    return np.where((wt != 0) & (Omega2 != 0), K, 0.0)


def sigma_coh(m: np.ndarray, x: np.ndarray, w: np.ndarray, Omega2: np.ndarray, wt: np.ndarray,
              v: np.ndarray, delta: float) -> complex:
    """Sigma_n = sum_{n''} w_{n''} m_{n''}^T K(x_{n''}) conj(m_{n''}) for one target band;
    m [n''][N_G] = <n| e^{iG.r} |n''>, x [n''] = E_n - E_{n''}."""
    total = 0.0 + 0.0j
    for a in range(m.shape[0]):
        K = coh_kernel(Omega2, wt, v, float(x[a]), delta)
        total += w[a] * (m[a] @ K @ np.conj(m[a]))
    return total


def sigma_coh_abs(m: np.ndarray, x: np.ndarray, w: np.ndarray, Omega2: np.ndarray, wt: np.ndarray,
                  v: np.ndarray, delta: float) -> float:
    """sum_{n''} |w_{n''}| |m_{n''}|^T |K(x_{n''})| |m_{n''}|: the sum of the magnitudes of
    the terms of sigma_coh, the scale against which its rounding errors are measured
    (the terms cancel strongly, so |Sigma| itself can be much smaller)."""
    total = 0.0
    for a in range(m.shape[0]):
        K = np.abs(coh_kernel(Omega2, wt, v, float(x[a]), delta))
        total += abs(w[a]) * (np.abs(m[a]) @ K @ np.abs(m[a]))
    return float(total)


def difference_table(gvec: np.ndarray):
    """The distinct integer vectors G_i - G_j of a sphere and, for each (i, j),
    the index of G_i - G_j in that list (sorted lexicographically)."""
    g = np.asarray(gvec, dtype=np.int64)
    diff = (g[:, None, :] - g[None, :, :]).reshape(-1, 3)
    uniq, inv = np.unique(diff, axis=0, return_inverse=True)
    return uniq, inv.reshape(g.shape[0], g.shape[0])


def sigma_coh_problem(prob, targets, eps_inv0: np.ndarray, A: np.ndarray, n_el: float,
                      cols=None, E_cols=None, w_cols=None, iq: int = 0):
    """Sigma_COH(E_t) of Eq. 2 with the HL-GPP model for target conduction bands
    `targets` of a synthetic problem: the n'' sum runs over the valence set and
    the conduction columns (all bands, or an Eq. 3 selection cols/E_cols/w_cols
    with the energy-grid states carrying their weights and grid energies).
    The valence set of q-point iq stands for the occupied bands (density and
    n''); eps_inv0 is the inverse of the plain static eps of sphere iq."""
    from .chi0_oracle import pair_elements, wfn_to_grid
    from .dielectric import coulomb, reciprocal_lattice
    gvec = prob.gvec[iq]
    u_v = wfn_to_grid(prob.coeff_v(iq), prob.gw, prob.n)
    uniq, idx = difference_table(gvec)
    rho_ratio = density_ratio(u_v, uniq)[idx]
    B = reciprocal_lattice(A)
    kvec = (gvec + prob.q_frac[iq][None, :]) @ B
    wp2 = plasma_frequency2(n_el, abs(np.linalg.det(A)))
    Omega2, wt = gpp_parameters(eps_inv0, rho_ratio, kvec, wp2)
    v = coulomb(prob.q_frac[iq], gvec, A)
    if cols is None:
        cols = np.arange(prob.n_c)
        E_cols = prob.E_c
        w_cols = np.ones(prob.n_c)
    u_c = wfn_to_grid(prob.coeff_c(np.asarray(cols)), prob.gw, prob.n)
    u_b = np.concatenate([u_v, u_c], 0)
    E_b = np.concatenate([prob.E_v, np.asarray(E_cols)])
    w_b = np.concatenate([np.ones(prob.n_v), np.asarray(w_cols)])
    u_t = wfn_to_grid(prob.coeff_c(np.asarray(targets)), prob.gw, prob.n)
    out, mag = [], []
    for it, t in enumerate(targets):
        m = pair_elements(u_t[it:it + 1], u_b, gvec, prob.n)
        out.append(sigma_coh(m, prob.E_c[t] - E_b, w_b, Omega2, wt, v, prob.delta))
        mag.append(sigma_coh_abs(m, prob.E_c[t] - E_b, w_b, Omega2, wt, v, prob.delta))
    return np.asarray(out), dict(Omega2=Omega2, wt=wt, v=v, rho_ratio=rho_ratio, abs_sum=np.asarray(mag))
