"""Pins of the oracle's accelerated conduction-band summation (Eq. 3 with the
quadrature of Eq. 4): count arithmetic, the N0 = N_c limit, the midpoint-rule
convergence of the integral part, the nearest-state choice and the pair
bookkeeping."""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import (accelerated_pairs, chi0_from_pairs, dos, freq_factor, full_pairs,
                    rel_fro, select_accelerated)
from synth import HARTREE_EV, make_problem

HERE = os.path.dirname(os.path.abspath(__file__))
_A6000 = make_problem("c2").dos_A   # 6000 states on [0.17, 2.2] Ha


def _speedup_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "speedup_tables.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            t, label, nc, nsel, s = line.split()
            rows.append((t, label, int(nc), int(nsel), float(s)))
    return rows


@pytest.mark.parametrize("row", _speedup_rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_printed_speedup_is_pair_count_ratio(row):
    _, _, nc, nsel, printed = row
    assert round(nc / nsel, 1) == pytest.approx(printed, abs=1e-9)


@pytest.mark.parametrize("name,expect", [("c2", 535), ("c5", 2070)])
def test_grid_point_count(name, expect):
    # N_E = ceil((E_max - E_0) / dE) with E_0 the energy of band N0
    prob = make_problem(name)
    sel = select_accelerated(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max)
    assert sel["explicit"].size + sel["rep"].size == expect
    E0 = prob.E_c[prob.N0 - 1]
    assert sel["rep"].size == math.ceil((prob.E_max - E0) / prob.dE)
    # intervals tile (E_0, E_max] exactly; the last one is clipped
    assert sel["edges"][0] == E0 and sel["edges"][-1] == prob.E_max
    assert abs(sel["dE_i"].sum() - (prob.E_max - E0)) < 1e-14
    assert np.all(sel["dE_i"][:-1] == pytest.approx(prob.dE, rel=1e-12))
    assert 0 < sel["dE_i"][-1] <= prob.dE
    assert np.allclose(sel["E_i"], 0.5 * (sel["edges"][:-1] + sel["edges"][1:]), rtol=0, atol=1e-15)


def test_n0_equal_nc_is_full_sum():
    prob = make_problem("c1", n_c=12, n_v=3)
    sel = select_accelerated(prob.E_c, prob.n_c, 0.05, prob.dos_A, prob.dos_V0, prob.E_max)
    c_idx, Ecol, wcol, dE, w = accelerated_pairs(prob.E_v, prob.E_c, sel)
    c_f, E_f, w_f, dE_f, w_ff = full_pairs(prob.E_v, prob.E_c)
    assert np.array_equal(c_idx, c_f) and np.array_equal(dE, dE_f) and np.array_equal(w, w_ff)


def test_representative_is_nearest_state_above_n0():
    rng = np.random.default_rng(3)
    E_c = np.sort(rng.uniform(0.17, 2.2, 300))
    E_c[150] = E_c[151]          # a degenerate pair to exercise the tie rule
    sel = select_accelerated(E_c, 40, 0.037, 100.0, 0.17, 2.2)
    for e, r in zip(sel["E_i"], sel["rep"]):
        dist = np.abs(E_c - e)
        dist[:40] = np.inf
        best = np.flatnonzero(dist == dist.min())
        assert r == best[0]


@pytest.mark.parametrize("omega", [0.0, 0.4j])
def test_integral_part_converges_as_midpoint_rule(omega):
    # All states above E_0 share one matrix element (M = 1 on a 1x1 "sphere"),
    # so Eq. 4 becomes sum_i g(E_i) dE_i h(E_i) and must converge to the
    # integral of g(E) h(E) over (E_0, E_max] with an O(dE^2) error.
    A, V0, Emax, Ev, delta = _A6000, 0.17, 2.2, -0.1, 1e-3
    E_c = 0.17 + 2.03 * ((np.arange(1, 6001) - 0.5) / 6000) ** (2 / 3)
    N0 = 512
    E0 = E_c[N0 - 1]

    def h(E, part):
        z = 0.5 * (1 / (Ev - E - omega + 1j * delta) + 1 / (Ev - E + omega + 1j * delta))
        return (z.real if part == 0 else z.imag) * A * math.sqrt(2 * (E - V0))

    exact = quad(h, E0, Emax, args=(0,), epsabs=1e-12, epsrel=1e-13)[0] + \
        1j * quad(h, E0, Emax, args=(1,), epsabs=1e-12, epsrel=1e-13)[0]
    errs = []
    for dE_eV in (2.0, 1.0, 0.5, 0.25):
        sel = select_accelerated(E_c, N0, dE_eV / HARTREE_EV, A, V0, Emax)
        f = freq_factor(Ev - sel["E_i"], sel["w_i"], [omega], delta)
        got = chi0_from_pairs(np.ones((sel["rep"].size, 1)), f)[0, 0, 0]
        errs.append(abs(got - exact) / abs(exact))
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert errs[0] < 2e-3
    for r in ratios:
        assert 3.0 < r < 5.0


def test_weights_integrate_dos():
    A, V0, Emax = _A6000, 0.17, 2.2
    E_c = 0.17 + 2.03 * ((np.arange(1, 6001) - 0.5) / 6000) ** (2 / 3)
    sel = select_accelerated(E_c, 512, 0.5 / HARTREE_EV, A, V0, Emax)
    E0 = sel["E0"]
    exact = A * math.sqrt(2) * (2 / 3) * ((Emax - V0) ** 1.5 - (E0 - V0) ** 1.5)
    assert abs(sel["w_i"].sum() - exact) / exact < 1e-5
    assert np.allclose(sel["w_i"], dos(sel["E_i"], A, V0) * sel["dE_i"], rtol=1e-15)
    # the synthetic DOS counts N_c states up to E_max
    assert abs(A * math.sqrt(2) * (2 / 3) * (Emax - V0) ** 1.5 - 6000) < 1e-9


def test_explicit_part_is_eq1_restricted_at_static_limit():
    rng = np.random.default_rng(5)
    Ev = np.array([-0.2, -0.05])
    E_c = np.sort(rng.uniform(0.2, 2.0, 40))
    sel = select_accelerated(E_c, 10, 0.2, 50.0, 0.17, 2.2)
    c_idx, Ecol, wcol, dE, w = accelerated_pairs(Ev, E_c, sel)
    nsel = c_idx.size
    M = (rng.standard_normal((2 * nsel, 4)) + 1j * rng.standard_normal((2 * nsel, 4)))
    # explicit columns: dE = E_v - E_c, w = 1 ; grid columns: dE = E_v - E_i, w = g dE_i
    dEm = dE.reshape(2, nsel)
    assert np.allclose(dEm[:, :10], Ev[:, None] - E_c[None, :10], atol=0)
    assert np.allclose(dEm[:, 10:], Ev[:, None] - sel["E_i"][None, :], atol=0)
    assert np.all(w.reshape(2, nsel)[:, :10] == 1.0)
    keep = (np.arange(2 * nsel) % nsel) < 10
    f = freq_factor(dE[keep], w[keep], [0.0], 0.0)
    expl = chi0_from_pairs(M[keep], f)[0]
    direct = sum(M[p][:, None] * M[p].conj()[None, :] / dE[p] for p in np.flatnonzero(keep))
    assert rel_fro(expl, direct) < 1e-14


# ---------------------------------------------------------------------------
# the dE -> 0 limit of Eq. 3/4 with the wavefunctions' own pair elements
# (the text after Eq. 4 and Table I: the accelerated sum approaches the full
# one as the energy grid is refined).  The synthetic conduction energies are
# the DOS-quantile midpoints E_c(j) = F^-1(j - 1/2), F(E) = int_V0^E g, so the
# bins [F^-1(j - 1), F^-1(j)] hold exactly one band each.
# ---------------------------------------------------------------------------
def _one_state_bins(prob, N0):
    from oracle.quadrature import bin_edges, dos_count
    A, V0, Emax = prob.dos_A, prob.dos_V0, prob.E_max
    E_lo = V0 + (N0 / (A * 2.0 * math.sqrt(2.0) / 3.0)) ** (2.0 / 3.0)    # F(E_lo) = N0
    n_bins = prob.n_c - N0
    step = (Emax - E_lo) / n_bins
    edges = bin_edges(E_lo, Emax, step, A, V0, "quantile")
    assert edges.size == n_bins + 1
    assert np.allclose(dos_count(edges, A, V0) - N0, np.arange(n_bins + 1), rtol=0, atol=1e-9)
    return edges, step


def _pairs_of(prob):
    from oracle import pair_elements, wfn_to_grid
    uv = wfn_to_grid(prob.coeff_v(0), prob.gw, prob.n)
    uc = wfn_to_grid(prob.coeff_c(), prob.gw, prob.n)
    return pair_elements(uv, uc, prob.gvec[0], prob.n)


def test_one_state_per_dos_quantile_bin_is_the_full_sum():
    """Nodes at the DOS midpoints F^-1((F(a) + F(b))/2) with weights int_a^b g = 1:
    every bin's state is its own band with its own energy, and Eq. 3/4 gives
    Eq. 1 to rounding."""
    from oracle.quadrature import bin_edges, dos_count, nearest_bands
    prob = make_problem("c1", n_v=4, n_c=96, n_imag=2)
    N0 = 8
    A, V0 = prob.dos_A, prob.dos_V0
    edges, step = _one_state_bins(prob, N0)
    nodes = bin_edges(edges[0], prob.E_max, step / 2, A, V0, "quantile")[1::2]
    w = dos_count(edges[1:], A, V0) - dos_count(edges[:-1], A, V0)
    assert np.allclose(w, 1.0, rtol=0, atol=1e-12)
    assert np.allclose(nodes, prob.E_c[N0:], rtol=0, atol=1e-14)
    rep = np.array([nearest_bands(prob.E_c, N0, e, 1)[0] for e in nodes])
    assert np.array_equal(rep, np.arange(N0, prob.n_c))
    sel = dict(explicit=np.arange(N0), rep=rep, E_i=nodes, w_i=w)
    c_idx, Ecol, wcol, dEp, wp = accelerated_pairs(prob.E_v, prob.E_c, sel)
    assert np.array_equal(c_idx, np.arange(prob.n_c))
    M = _pairs_of(prob)
    _, _, _, dEf, wf = full_pairs(prob.E_v, prob.E_c)
    acc = chi0_from_pairs(M, freq_factor(dEp, wp, prob.omega, prob.delta))
    full = chi0_from_pairs(M, freq_factor(dEf, wf, prob.omega, prob.delta))
    for iw in range(prob.omega.size):
        assert rel_fro(acc[iw], full[iw]) < 1e-14


def test_midpoint_rule_on_one_state_bins_converges_quadratically():
    """Eq. 4's midpoint node and weight g(E_i) dE_i on the same one-state bins:
    the node moves off the band energy and the weight off 1 by O(dE^2) per
    bin, so the distance from the full sum falls as dE^2 (fitted slope) while
    the bands are refined (N0 / N_c fixed, so E_0 stays put)."""
    from oracle.quadrature import nearest_bands, quadrature_nodes
    hs, errs = [], []
    for n_c in (60, 120, 240, 480):
        prob = make_problem("c1", n_v=3, n_c=n_c, n_imag=1)
        N0 = n_c // 10
        edges, step = _one_state_bins(prob, N0)
        nodes, raw = quadrature_nodes(edges, "midpoint")
        rep = np.array([nearest_bands(prob.E_c, N0, e, 1)[0] for e in nodes])
        assert np.array_equal(rep, np.arange(N0, n_c))
        sel = dict(explicit=np.arange(N0), rep=rep, E_i=nodes, w_i=dos(nodes, prob.dos_A, prob.dos_V0) * raw)
        _, _, _, dEp, wp = accelerated_pairs(prob.E_v, prob.E_c, sel)
        _, _, _, dEf, wf = full_pairs(prob.E_v, prob.E_c)
        M = _pairs_of(prob)
        acc = chi0_from_pairs(M, freq_factor(dEp, wp, prob.omega, prob.delta))
        full = chi0_from_pairs(M, freq_factor(dEf, wf, prob.omega, prob.delta))
        errs.append(max(rel_fro(acc[iw], full[iw]) for iw in range(prob.omega.size)))
        hs.append(step)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    print(f"\nmidpoint on one-state bins: errors {['%.2e' % e for e in errs]}, fitted order {slope:.3f}")
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert 1.8 < slope < 2.2
