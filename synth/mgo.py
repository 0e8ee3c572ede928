"""MgO-shaped synthetic workloads (seeded, deterministic).

Recipe (the paper's DFT wavefunctions are not available, so random data with
the same shapes stands in for them):

* cell: simple cubic, lattice constant a = 7.96 bohr * n/24 (conventional
  8-atom MgO cell at n = 24, scaled so the real-space grid spacing is fixed);
  G vectors are integer triples in units of 2*pi/a;
* wavefunction sphere: all integer g with |g|^2 <= (7 n/24)^2 (1419 points at
  n = 24, an 80 Ry-like cutoff scaled with the cell);
* band coefficients: complex Gaussian (re, im ~ N(0,1)) on that sphere, each
  band normalised to sum |c|^2 = 1; band b of stream s draws from
  numpy.random.default_rng([seed, s, b]) so any subset of bands can be
  regenerated on its own; stream 0 is the conduction set at k, stream 1+iq the
  valence set at k+q;
* dielectric sphere: the N_G integer g with the smallest |q+g|^2, ties broken
  by (g1, g2, g3) ascending;
* energies (Hartree): valence E_v(j) = -0.25 + 0.25 (j-1/2)/N_v, conduction
  E_c(j) = 0.17 + 2.03 ((j-1/2)/N_c)^(2/3), j = 1..N; these are the quantile
  midpoints of a uniform valence band and of a free-electron (square-root)
  conduction density of states starting at V0 = 0.17 Ha and holding N_c states
  up to E_max = 2.2 Ha;
* density-of-states model parameters: g(E) = A sqrt(2 (E - V0)) with
  A = N_c / (sqrt(2) * (2/3) * 2.03^(3/2)) so that g integrates to N_c on
  [V0, E_max];
* frequencies: omega = 0 plus n_imag imaginary frequencies i*w, w log-spaced
  from 0.01 to 2 Ha; broadening delta = 1e-3 Ha;
* k-points (the sum over k of Eq. 1): k-point ik has its own conduction and
  valence streams and conduction energies E_c + 0.004 ik Ha; k-point 0 is the
  single-k workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HARTREE_EV = 27.211386245988
BOHR_A0 = 7.96          # bohr, conventional MgO cell at the 24^3 grid
V0_HA = 0.17
WIDTH_HA = 2.03
DELTA_HA = 1e-3
SEED_BASE = 1601_0000


def _shifted_q_grid():
    return [((i + 0.5) / 2, (j + 0.5) / 2, (l + 0.5) / 2)
            for i in range(2) for j in range(2) for l in range(2)]


# Workload shapes; q is given either in bohr^-1 ("q_bohr") or in units of
# 2 pi / a ("q_frac").
CONFIGS = {
    "c1": dict(idx=1, n_v=16, n_c=240, n=24, n_G=[350], q_bohr=[(0.001, 0.0, 0.0)],
               n_imag=0, N0=None, dE_eV=None),
    "c2": dict(idx=2, n_v=128, n_c=6000, n=48, n_G=[2500], q_bohr=[(0.001, 0.0, 0.0)],
               n_imag=8, N0=512, dE_eV=2.0),
    "c3": dict(idx=3, n_v=128, n_c=4000, n=48,
               n_G=[int(round(2200 + 400 * j / 7)) for j in range(8)],
               q_frac=_shifted_q_grid(), n_imag=31, N0=None, dE_eV=None),
    "c4": dict(idx=4, n_v=64, n_c=2000, n=36, n_G=[1200], q_bohr=[(0.001, 0.0, 0.0)],
               n_imag=0, N0=None, dE_eV=None),
    "c5": dict(idx=5, n_v=512, n_c=20000, n=96, n_G=[8000], q_bohr=[(0.001, 0.0, 0.0)],
               n_imag=8, N0=2048, dE_eV=2.0),
}


def pw_sphere(n: int, r2: float | None = None) -> np.ndarray:
    """Integer g with |g|^2 <= r2 (default (7n/24)^2), sorted by (g1, g2, g3)."""
    if r2 is None:
        r2 = (7.0 * n / 24.0) ** 2
    r = int(np.floor(np.sqrt(r2))) + 1
    ax = np.arange(-r, r + 1)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    g = g[(g * g).sum(1) <= r2 + 1e-9]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0]))
    return np.ascontiguousarray(g[order].astype(np.int32))


def g_sphere(n_G: int, q_frac, n: int | None = None) -> np.ndarray:
    """The n_G integer vectors g with the smallest |q+g|^2 (ties by g1, g2, g3)."""
    q = np.asarray(q_frac, dtype=np.float64)
    r = int(np.ceil((3.0 * n_G / (4.0 * np.pi)) ** (1.0 / 3.0))) + 3
    ax = np.arange(-r, r + 1)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    k2 = np.round(((g + q[None, :]) ** 2).sum(1), 9)
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], k2))
    out = g[order[:n_G]].astype(np.int32)
    if n is not None:
        # the sphere must fit in the grid without wrapping onto itself
        assert (out.max(0) - out.min(0) < n).all(), "G sphere does not fit the grid"
    return np.ascontiguousarray(out)


def valence_energies(n_v: int) -> np.ndarray:
    j = np.arange(1, n_v + 1, dtype=np.float64)
    return -0.25 + 0.25 * (j - 0.5) / n_v


def conduction_energies(n_c: int) -> np.ndarray:
    j = np.arange(1, n_c + 1, dtype=np.float64)
    return V0_HA + WIDTH_HA * ((j - 0.5) / n_c) ** (2.0 / 3.0)


def imag_frequencies(n_imag: int) -> np.ndarray:
    """omega list: 0 followed by n_imag values i*w, w log-spaced 0.01..2 Ha."""
    if n_imag == 0:
        return np.zeros(1, dtype=np.complex128)
    w = np.logspace(np.log10(0.01), np.log10(2.0), n_imag)
    return np.concatenate([[0.0], 1j * w]).astype(np.complex128)


def band_coefficients(seed: int, stream: int, bands, npw: int) -> np.ndarray:
    """Normalised complex Gaussian plane-wave coefficients, one row per band."""
    bands = np.atleast_1d(np.asarray(bands, dtype=np.int64))
    out = np.empty((bands.size, npw), dtype=np.complex128)
    for i, b in enumerate(bands):
        rng = np.random.default_rng([seed, stream, int(b)])
        z = rng.standard_normal((2, npw))
        c = z[0] + 1j * z[1]
        out[i] = c / np.sqrt(np.vdot(c, c).real)
    return out


@dataclass
class Problem:
    name: str
    n: int                      # grid points per axis
    a: float                    # lattice constant (bohr)
    n_v: int
    n_c: int
    gw: np.ndarray              # [npw, 3] int32 wavefunction sphere
    q_frac: np.ndarray          # [n_q, 3] q in units of 2 pi / a
    gvec: list                  # n_q arrays [N_G(q), 3] int32
    omega: np.ndarray           # [n_freq] complex128 (Hartree)
    delta: float                # Hartree
    E_v: np.ndarray             # [n_v]
    E_c: np.ndarray             # [n_c]
    dos_A: float                # g(E) = dos_A * sqrt(2 (E - dos_V0)), states per Hartree
    dos_V0: float
    E_max: float
    N0: int | None = None
    dE: float | None = None     # Hartree
    seed: int = SEED_BASE
    extra: dict = field(default_factory=dict)

    @property
    def npw(self) -> int:
        return int(self.gw.shape[0])

    @property
    def n_q(self) -> int:
        return len(self.gvec)

    def coeff_c(self, bands=None, ik: int = 0) -> np.ndarray:
        bands = np.arange(self.n_c) if bands is None else bands
        return band_coefficients(self.seed, _stream_c(ik), bands, self.npw)

    def coeff_v(self, iq: int = 0, bands=None, ik: int = 0) -> np.ndarray:
        bands = np.arange(self.n_v) if bands is None else bands
        return band_coefficients(self.seed, _stream_v(ik, iq), bands, self.npw)

    def E_c_k(self, ik: int = 0) -> np.ndarray:
        """Conduction energies at k-point ik: E_c shifted by K_SHIFT_HA * ik."""
        return self.E_c + K_SHIFT_HA * ik


# k-points: k-point 0 uses the streams above (0 = conduction at k, 1 + iq =
# valence at k + q); k-point ik > 0 draws from its own streams; its conduction
# energies are shifted by K_SHIFT_HA * ik (a small dispersion), the valence
# energies are shared.
K_SHIFT_HA = 0.004


def _stream_c(ik: int) -> int:
    return 0 if ik == 0 else 100000 + 1000 * ik


def _stream_v(ik: int, iq: int) -> int:
    return 1 + iq if ik == 0 else 100000 + 1000 * ik + 1 + iq


def make_problem(name: str = "custom", *, n_v=None, n_c=None, n=None, n_G=None,
                 q_bohr=None, q_frac=None, n_imag=None, N0=None, dE_eV=None,
                 delta=DELTA_HA, wfn_r2=None, seed=None) -> Problem:
    """Build a named workload (c1..c5) or a custom one with the same recipe."""
    spec = dict(CONFIGS.get(name, {}))
    for k, v in dict(n_v=n_v, n_c=n_c, n=n, n_G=n_G, q_bohr=q_bohr, q_frac=q_frac,
                     n_imag=n_imag, N0=N0, dE_eV=dE_eV).items():
        if v is not None:
            spec[k] = v
    n = int(spec["n"])
    a = BOHR_A0 * n / 24.0
    if spec.get("q_frac") is not None:
        qf = np.asarray(spec["q_frac"], dtype=np.float64).reshape(-1, 3)
    else:
        qb = np.asarray(spec.get("q_bohr", [(0.0, 0.0, 0.0)]), dtype=np.float64).reshape(-1, 3)
        qf = qb * a / (2.0 * np.pi)
    nGs = spec["n_G"]
    nGs = [int(nGs)] * len(qf) if np.isscalar(nGs) else [int(x) for x in nGs]
    gvec = [g_sphere(nG, q, n) for nG, q in zip(nGs, qf)]
    n_c = int(spec["n_c"])
    A = n_c / (np.sqrt(2.0) * (2.0 / 3.0) * WIDTH_HA ** 1.5)
    dE = spec.get("dE_eV")
    idx = int(spec.get("idx", 0))
    return Problem(
        name=name, n=n, a=a, n_v=int(spec["n_v"]), n_c=n_c,
        gw=pw_sphere(n, wfn_r2), q_frac=qf, gvec=gvec,
        omega=imag_frequencies(int(spec.get("n_imag", 0))), delta=float(delta),
        E_v=valence_energies(int(spec["n_v"])), E_c=conduction_energies(n_c),
        dos_A=float(A), dos_V0=V0_HA, E_max=V0_HA + WIDTH_HA,
        N0=spec.get("N0"), dE=None if dE is None else float(dE) / HARTREE_EV,
        seed=SEED_BASE + 100 * idx if seed is None else int(seed))


def _fill_bands(args):
    shm_name, shape, seed, stream, b0, b1 = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        out = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        out[b0:b1] = band_coefficients(seed, stream, np.arange(b0, b1), shape[1])
    finally:
        shm.close()
    return b1 - b0


def band_coefficients_parallel(seed: int, stream: int, n_bands: int, npw: int, workers: int = 0):
    """The same coefficients as band_coefficients(seed, stream, range(n_bands), npw),
    generated by `workers` spawned processes into shared memory.  Returns
    (array, shm); the caller keeps shm alive while the array is in use and
    then calls shm.close(); shm.unlink().  Call before the first CUDA call of
    the process (the workers are spawned, not forked)."""
    import multiprocessing as mp
    import os
    from multiprocessing import shared_memory
    workers = workers or max(1, (os.cpu_count() or 2) - 1)
    shape = (n_bands, npw)
    shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * 16)
    step = max(1, (n_bands + 4 * workers - 1) // (4 * workers))
    jobs = [(shm.name, shape, seed, stream, b, min(n_bands, b + step)) for b in range(0, n_bands, step)]
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_fill_bands, jobs)
    return np.ndarray(shape, dtype=np.complex128, buffer=shm.buf), shm
