"""FP64 CPU oracle for the RPA dielectric matrix built from chi0: the bare
Coulomb interaction v(q+G), epsilon = 1 - v chi0, its inverse and the
macroscopic dielectric constant eps_inf = 1 / [eps^-1]_{00}(q -> 0, omega = 0).

TEST INFRASTRUCTURE ONLY (same rules as chi0_oracle: imported by tests, the
smoke check and the CPU legs of the benchmark; never by the library).

Sources: the RPA relation eps = 1 - v chi0 and W = eps^-1 v stated with Eq. 1
(section II), and the definition of eps_inf given with Table III.  The paper
does not print v or the normalisation of chi0; the readings used here:
* v(q+G) = 4 pi / (Omega |q+G|^2) in Hartree atomic units (e^2 = 1), Omega the
  cell volume, with chi0 exactly as Eq. 1 writes it (no further prefactor);
* eps_{GG'} = delta_{GG'} - v(q+G) chi0_{GG'} ("plain"), or the symmetrised
  form delta_{GG'} - v(q+G)^{1/2} chi0_{GG'} v(q+G')^{1/2}, a similarity
  transform of the plain one with the same eigenvalues and the same diagonal
  of the inverse (so the same eps_inf);
* eps_inf is 1 / [eps^-1]_{00} at the sphere point G = 0, taken at the given
  small q (the limit q -> 0 is not taken numerically); it is returned complex
  (its imaginary part comes from the broadening delta).

Every function is pinned by tests/test_oracle_dielectric.py.
"""
from __future__ import annotations

import numpy as np


def reciprocal_lattice(A: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij for the direct lattice rows a_i."""
    A = np.asarray(A, dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(A).T


def coulomb(q_frac, gvec: np.ndarray, A: np.ndarray) -> np.ndarray:
    """v(q+G) = 4 pi / (Omega |q+G|^2) for q and G given in reciprocal-lattice
    units (q_frac real triple, gvec integer rows); A holds the direct lattice
    vectors as rows (bohr).  Returns [N_G] float64."""
    A = np.asarray(A, dtype=np.float64)
    B = reciprocal_lattice(A)
    k = (np.asarray(gvec, dtype=np.float64) + np.asarray(q_frac, dtype=np.float64)[None, :]) @ B
    omega_cell = abs(np.linalg.det(A))
    return 4.0 * np.pi / (omega_cell * np.einsum("ij,ij->i", k, k))


def epsilon(chi0: np.ndarray, v: np.ndarray, symmetric: bool = False) -> np.ndarray:
    """eps[w] = I - diag(v) chi0[w] (plain) or I - diag(v^1/2) chi0[w] diag(v^1/2)."""
    chi0 = np.asarray(chi0, dtype=np.complex128)
    v = np.asarray(v, dtype=np.float64)
    eye = np.eye(chi0.shape[-1], dtype=np.complex128)
    if symmetric:
        s = np.sqrt(v)
        return eye - s[:, None] * chi0 * s[None, :]
    return eye - v[:, None] * chi0


def epsilon_inverse(eps: np.ndarray) -> np.ndarray:
    """eps^-1 for every frequency (LAPACK LU with partial pivoting)."""
    eps = np.asarray(eps, dtype=np.complex128)
    return np.linalg.inv(eps)


def eps_inf(eps_inv: np.ndarray, i0: int = 0) -> np.ndarray:
    """1 / [eps^-1]_{00} per frequency; i0 is the index of G = 0 in the sphere."""
    return 1.0 / np.asarray(eps_inv)[..., i0, i0]
