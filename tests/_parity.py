"""Comparison helpers of the GPU parity tests (no method arithmetic).

Every chi0 comparison checks, per frequency, both the relative Frobenius
error ||chi - ref||_F / ||ref||_F and the element-wise error
max|chi - ref| / max|ref|: a wrong mirrored element or tile edge moves the
second by its own size while it can hide in the first."""
import numpy as np


def rel_fro(a, b) -> float:
    nb = np.linalg.norm(np.asarray(b).ravel())
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / (nb if nb > 0 else 1.0))


def rel_max(a, b) -> float:
    mb = float(np.max(np.abs(b))) if np.size(b) else 0.0
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / (mb if mb > 0 else 1.0)


def check_chi(got, ref, tol, elem_tol=None, label=""):
    """Assert both bars for every frequency of chi0 [n_freq][N_G][N_G] (or one
    matrix); returns the per-frequency (Frobenius, element-wise) errors."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (label, got.shape, ref.shape)
    if got.ndim == 2:
        got, ref = got[None], ref[None]
    elem_tol = tol if elem_tol is None else elem_tol
    errs = [(rel_fro(got[i], ref[i]), rel_max(got[i], ref[i])) for i in range(got.shape[0])]
    print(f"\n{label}: rel Frobenius {['%.2e' % e[0] for e in errs]}, element-wise {['%.2e' % e[1] for e in errs]}")
    for i, (ef, em) in enumerate(errs):
        assert ef < tol, (label, i, ef)
        assert em < elem_tol, (label, i, em)
    return errs
