"""Non-uniform and higher-order energy quadrature for the integral part of
Eq. 3 (the text after Eq. 4: the integration may use a uniform or non-uniform
energy grid and higher-order rules), with several states per node.

TEST INFRASTRUCTURE ONLY (same rules as chi0_oracle).

Readings (the paper names the options, not their formulas):
* grids on [E_0, E_max], E_0 = energy of band N0, N_E = ceil((E_max - E_0)/dE)
  bins in both cases:
  - "uniform": edges E_0 + k dE, the last clipped at E_max (Eq. 4 as printed);
  - "quantile": edges with equal DOS count between neighbours, i.e.
    G(e_k) - G(E_0) = k (G(E_max) - G(E_0)) / N_E with
    G(E) = int_V0^E g = A (2 sqrt(2) / 3) (E - V0)^(3/2) inverted in closed form;
* rules on each bin [a, b] of width h (raw weights, before the DOS factor):
  - "midpoint": node (a + b)/2, weight h (Eq. 4);
  - "simpson": nodes a, (a + b)/2, b with weights h/6, 4h/6, h/6; the common
    end of neighbouring bins is one node carrying both weights;
  - "gauss2": nodes (a + b)/2 -+ h/(2 sqrt 3), weights h/2 each;
* node weight W_k = g(E_k) x raw weight (g of Eq. 3); the node's states are the
  `states` conduction bands above N0 nearest in energy to E_k (ties to the
  lower index), each carrying W_k / states, with E_k in the denominator as in
  Eq. 4.

Every function is pinned by tests/test_oracle_quadrature.py.
"""
from __future__ import annotations

import math

import numpy as np

from .chi0_oracle import dos

GRIDS = ("uniform", "quantile")
RULES = ("midpoint", "simpson", "gauss2")


def dos_count(E, A: float, V0: float):
    """G(E) = int_V0^E A sqrt(2 (x - V0)) dx = A (2 sqrt 2 / 3) (E - V0)^(3/2)."""
    x = np.maximum(np.asarray(E, dtype=np.float64) - V0, 0.0)
    return A * (2.0 * math.sqrt(2.0) / 3.0) * x ** 1.5


def bin_edges(E0: float, E_max: float, dE: float, A: float, V0: float, grid: str) -> np.ndarray:
    n_bins = max(int(math.ceil((E_max - E0) / dE - 1e-12)), 0)
    if n_bins == 0:
        return np.array([E0], dtype=np.float64)
    if grid == "uniform":
        return np.minimum(E0 + dE * np.arange(n_bins + 1), E_max)
    if grid == "quantile":
        G0, G1 = dos_count(E0, A, V0), dos_count(E_max, A, V0)
        Gk = G0 + (G1 - G0) * np.arange(n_bins + 1) / n_bins
        e = V0 + (Gk / (A * 2.0 * math.sqrt(2.0) / 3.0)) ** (2.0 / 3.0)
        e[0], e[-1] = E0, E_max
        return e
    raise ValueError(grid)


def quadrature_nodes(edges: np.ndarray, rule: str):
    """(nodes, raw weights) of the composite rule over the bins, ascending."""
    a, b = edges[:-1], edges[1:]
    h = b - a
    m = 0.5 * (a + b)
    if rule == "midpoint":
        return m.copy(), h.copy()
    if rule == "gauss2":
        d = h / (2.0 * math.sqrt(3.0))
        nodes = np.stack([m - d, m + d], 1).reshape(-1)
        return nodes, np.repeat(0.5 * h, 2)
    if rule == "simpson":
        nb = h.size
        nodes = np.empty(2 * nb + 1)
        w = np.zeros(2 * nb + 1)
        nodes[0::2] = edges
        nodes[1::2] = m
        w[0:-1:2] += h / 6.0
        w[2::2] += h / 6.0
        w[1::2] += 4.0 * h / 6.0
        return nodes, w
    raise ValueError(rule)


def nearest_bands(E_c: np.ndarray, N0: int, E: float, states: int) -> np.ndarray:
    """The `states` bands with index >= N0 closest in energy to E (ties: lower index)."""
    idx = np.arange(N0, E_c.size)
    order = np.lexsort((idx, np.abs(E_c[N0:] - E)))
    return idx[order[:min(states, idx.size)]]


def select_quadrature(E_c: np.ndarray, N0: int, dE: float, A: float, V0: float, E_max: float,
                      grid: str = "uniform", rule: str = "midpoint", states: int = 1) -> dict:
    """Columns of Eq. 3: N0 explicit bands (weight 1, own energy), then per
    quadrature node its states (band, node energy, node weight / states)."""
    E_c = np.asarray(E_c, dtype=np.float64)
    if np.any(np.diff(E_c) < 0):
        raise ValueError("conduction energies must be sorted ascending")
    n_c = E_c.size
    N0 = int(min(max(N0, 0), n_c))
    cols = list(range(N0))
    Ecol = list(E_c[:N0])
    wcol = [1.0] * N0
    out = dict(nodes=np.zeros(0), raw=np.zeros(0), edges=np.zeros(0))
    if N0 > 0 and N0 < n_c and dE > 0:
        E0 = E_c[N0 - 1]
        edges = bin_edges(E0, E_max, dE, A, V0, grid)
        nodes, raw = quadrature_nodes(edges, rule)
        W = dos(nodes, A, V0) * raw
        for Ek, Wk in zip(nodes, W):
            bands = nearest_bands(E_c, N0, Ek, states)
            for c in bands:
                cols.append(int(c))
                Ecol.append(float(Ek))
                wcol.append(float(Wk) / bands.size)
        out = dict(nodes=nodes, raw=raw, edges=edges)
    out.update(cols=np.asarray(cols, dtype=np.int64), E_col=np.asarray(Ecol, dtype=np.float64),
               w_col=np.asarray(wcol, dtype=np.float64), N0=N0)
    return out


def bin_error(E_c: np.ndarray, sens: np.ndarray, N0: int, a: float, b: float, last: bool) -> float:
    """First-order change of a loss L when the bands above N0 with energy in
    [a, b) (or [a, b] for the last bin) take the bin's midpoint energy:
    |sum_c dL/dE_c (m - E_c)|, the per-bin share of the energy-substitution
    estimate computed with the adjoint of Eq. 1 (sens = dL/dE_c)."""
    E = E_c[N0:]
    s = sens[N0:]
    inside = (E >= a) & ((E <= b) if last else (E < b))
    m = 0.5 * (a + b)
    return float(abs(np.sum(s[inside] * (m - E[inside]))))


def adaptive_edges(E_c: np.ndarray, sens: np.ndarray, N0: int, dE: float, E_max: float, n_split: int) -> np.ndarray:
    """Start from the uniform Eq. 4 grid of step dE on [E_0, E_max] and split,
    n_split times, the bin with the largest bin_error at its midpoint (ties: the
    lowest bin)."""
    E_c = np.asarray(E_c, dtype=np.float64)
    sens = np.asarray(sens, dtype=np.float64)
    E0 = E_c[N0 - 1]
    edges = list(bin_edges(E0, E_max, dE, 1.0, 0.0, "uniform"))
    for _ in range(n_split):
        nb = len(edges) - 1
        if nb <= 0:
            break
        errs = [bin_error(E_c, sens, N0, edges[k], edges[k + 1], k == nb - 1) for k in range(nb)]
        k = int(np.argmax(errs))                      # first maximum = lowest bin on ties
        edges.insert(k + 1, 0.5 * (edges[k] + edges[k + 1]))
    return np.asarray(edges)


def select_adaptive(E_c: np.ndarray, sens: np.ndarray, N0: int, dE: float, A: float, V0: float, E_max: float,
                    n_split: int, states: int = 1) -> dict:
    """Columns of Eq. 3 on the adaptive grid (midpoint rule, `states` states per node)."""
    E_c = np.asarray(E_c, dtype=np.float64)
    n_c = E_c.size
    N0 = int(min(max(N0, 0), n_c))
    cols, Ecol, wcol = list(range(N0)), list(E_c[:N0]), [1.0] * N0
    edges = np.zeros(0)
    if N0 > 0 and N0 < n_c and dE > 0:
        edges = adaptive_edges(E_c, sens, N0, dE, E_max, n_split)
        nodes, raw = quadrature_nodes(edges, "midpoint")
        W = dos(nodes, A, V0) * raw
        for Ek, Wk in zip(nodes, W):
            bands = nearest_bands(E_c, N0, Ek, states)
            for c in bands:
                cols.append(int(c))
                Ecol.append(float(Ek))
                wcol.append(float(Wk) / bands.size)
    return dict(cols=np.asarray(cols, dtype=np.int64), E_col=np.asarray(Ecol), w_col=np.asarray(wcol),
                edges=edges, N0=N0)
