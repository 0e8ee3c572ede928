"""Pins of the oracle's energy quadrature for the integral part of Eq. 3
(uniform and DOS-quantile grids; midpoint, Simpson and two-point Gauss rules;
several states per node): reduction to the Eq. 4 selection, polynomial
exactness of each rule, equal DOS counts of the quantile bins (numerical
integration), brute-force nearest states, and the convergence order of each
rule on a smooth integrand."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import dos, select_accelerated
from oracle.quadrature import (bin_edges, dos_count, nearest_bands, quadrature_nodes,
                               select_quadrature)
from synth import make_problem


def test_midpoint_uniform_one_state_is_eq4():
    prob = make_problem("c2")
    for N0, dE in ((512, prob.dE), (100, 0.05), (5990, 0.3)):
        ref = select_accelerated(prob.E_c, N0, dE, prob.dos_A, prob.dos_V0, prob.E_max)
        got = select_quadrature(prob.E_c, N0, dE, prob.dos_A, prob.dos_V0, prob.E_max)
        n0 = ref["explicit"].size
        assert np.array_equal(got["cols"][:n0], ref["explicit"])
        assert np.array_equal(got["cols"][n0:], ref["rep"])
        assert np.array_equal(got["E_col"][n0:], ref["E_i"])
        assert np.allclose(got["w_col"][n0:], ref["w_i"], rtol=1e-15, atol=0)


@pytest.mark.parametrize("rule,degree", [("midpoint", 1), ("simpson", 3), ("gauss2", 3)])
def test_rules_exact_to_their_degree(rule, degree):
    edges = np.sort(np.random.default_rng(1).uniform(0.3, 2.1, 9))
    nodes, w = quadrature_nodes(edges, rule)
    a, b = edges[0], edges[-1]
    for d in range(degree + 2):
        exact = (b ** (d + 1) - a ** (d + 1)) / (d + 1)
        err = abs(np.dot(w, nodes ** d) - exact)
        if d <= degree:
            assert err < 1e-13 * max(1.0, abs(exact)), (rule, d, err)
        else:
            assert err > 1e-8, (rule, d, err)
    assert np.all(np.diff(nodes) > 0)


def test_quantile_bins_hold_equal_dos_counts():
    A, V0 = 1234.5, 0.17
    E0, Emax = 0.62, 2.2
    edges = bin_edges(E0, Emax, 0.07, A, V0, "quantile")
    assert edges[0] == E0 and edges[-1] == Emax and np.all(np.diff(edges) > 0)
    assert edges.size - 1 == math.ceil((Emax - E0) / 0.07)
    counts = [quad(lambda e: dos(e, A, V0), lo, hi, epsabs=0, epsrel=1e-13)[0]
              for lo, hi in zip(edges[:-1], edges[1:])]
    assert np.ptp(counts) < 1e-9 * np.mean(counts)
    # closed-form count against numerical integration
    for E in (0.3, 1.0, 2.2):
        assert abs(dos_count(E, A, V0) - quad(lambda e: dos(e, A, V0), V0, E, epsrel=1e-13)[0]) < 1e-9 * dos_count(E, A, V0)


def test_nearest_states_brute_force():
    rng = np.random.default_rng(2)
    E_c = np.sort(np.round(rng.uniform(0.2, 2.0, 60), 2))    # rounded: equal energies occur
    for E in (0.2, 0.95, 1.3333, 2.5):
        for s in (1, 3, 7):
            got = nearest_bands(E_c, 10, E, s)
            cand = sorted(range(10, 60), key=lambda c: (abs(E_c[c] - E), c))[:s]
            assert list(got) == cand


@pytest.mark.parametrize("grid", ["uniform", "quantile"])
@pytest.mark.parametrize("rule,order", [("midpoint", 2), ("simpson", 4), ("gauss2", 4)])
def test_convergence_order_on_a_smooth_integrand(grid, rule, order):
    """sum_k W_k phi(E_k) -> int g phi with error ~ dE^order (phi smooth)."""
    A, V0, E0, Emax = 50.0, 0.17, 0.6, 2.2
    phi = lambda e: 1.0 / (e + 0.25) ** 2          # like 1/(E_v - E)^2 away from the pole
    exact = quad(lambda e: dos(e, A, V0) * phi(e), E0, Emax, epsabs=0, epsrel=2e-14, limit=200)[0]
    errs = []
    for dE in (0.05, 0.025, 0.0125):
        nodes, raw = quadrature_nodes(bin_edges(E0, Emax, dE, A, V0, grid), rule)
        errs.append(abs(np.dot(dos(nodes, A, V0) * raw, phi(nodes)) - exact))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.15 for r in rates), rates


def test_states_share_the_node_weight():
    prob = make_problem("c2")
    for states in (1, 2, 5):
        sel = select_quadrature(prob.E_c, 512, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max,
                                grid="quantile", rule="simpson", states=states)
        n_int = sel["cols"].size - 512
        assert n_int == states * sel["nodes"].size
        W = dos(sel["nodes"], prob.dos_A, prob.dos_V0) * sel["raw"]
        got = sel["w_col"][512:].reshape(-1, states).sum(1)
        assert np.allclose(got, W, rtol=1e-14)
        assert np.all(sel["E_col"][512:].reshape(-1, states) == sel["nodes"][:, None])
        assert np.all(sel["cols"][512:] >= 512)
    # no integration part when N0 covers every band or is zero
    assert select_quadrature(prob.E_c, 0, 0.1, 1.0, 0.17, 2.2)["cols"].size == 0
    assert select_quadrature(prob.E_c, prob.n_c, 0.1, 1.0, 0.17, 2.2)["cols"].size == prob.n_c


def test_bin_error_brute_force_and_adaptive_splits():
    """The per-bin first-order estimate against a plain loop, and the greedy
    refinement: each split halves the bin with the largest estimate (the
    estimate is a signed sum, so a half can exceed its parent), and with zero
    sensitivity above some energy nothing there is split."""
    from oracle.quadrature import adaptive_edges, bin_error
    rng = np.random.default_rng(5)
    E_c = np.sort(rng.uniform(0.17, 2.2, 400))
    N0, dE, Emax = 50, 0.25, 2.2
    sens = rng.standard_normal(400) * np.exp(-3.0 * (E_c - E_c[N0 - 1]))   # large just above E_0
    a, b = 0.9, 1.15
    want = 0.0
    for c in range(N0, 400):
        if a <= E_c[c] < b:
            want += sens[c] * (0.5 * (a + b) - E_c[c])
    assert abs(bin_error(E_c, sens, N0, a, b, False) - abs(want)) < 1e-13
    prev = None
    for n_split in range(0, 12):
        e = adaptive_edges(E_c, sens, N0, dE, Emax, n_split)
        assert e.size == math.ceil((Emax - E_c[N0 - 1]) / dE - 1e-12) + 1 + n_split
        assert np.all(np.diff(e) > 0) and e[0] == E_c[N0 - 1] and e[-1] == Emax
        if prev is not None:
            errs = [bin_error(E_c, sens, N0, prev[k], prev[k + 1], k == prev.size - 2) for k in range(prev.size - 1)]
            k = int(np.argmax(errs))
            added = np.setdiff1d(e, prev)
            assert added.size == 1 and added[0] == 0.5 * (prev[k] + prev[k + 1])
        prev = e
    # zero sensitivity above 1.5 Ha: every split lands below it
    s2 = np.where(E_c < 1.5, sens, 0.0)
    base = adaptive_edges(E_c, s2, N0, dE, Emax, 0)
    e = adaptive_edges(E_c, s2, N0, dE, Emax, 8)
    new = np.setdiff1d(e, base)
    assert new.size == 8 and np.all(new < 1.5)


def test_select_adaptive_reduces_to_eq4_without_splits():
    from oracle.quadrature import select_adaptive
    prob = make_problem("c2")
    sens = np.random.default_rng(6).standard_normal(prob.n_c)
    got = select_adaptive(prob.E_c, sens, prob.N0, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max, 0)
    ref = select_quadrature(prob.E_c, prob.N0, prob.dE, prob.dos_A, prob.dos_V0, prob.E_max)
    assert np.array_equal(got["cols"], ref["cols"])
    assert np.allclose(got["w_col"], ref["w_col"], rtol=1e-15, atol=0)
