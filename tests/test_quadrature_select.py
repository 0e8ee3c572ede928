"""The library's quadrature selection (chi0_select_quadrature, host code)
against the oracle: band indices exactly, node energies and weights to a few
ulps (the two sides evaluate the DOS-quantile edges with differently ordered
products).  No GPU needed."""
import numpy as np
import pytest

from oracle.quadrature import select_quadrature as oracle_select
from synth import make_problem


@pytest.mark.parametrize("grid", ["uniform", "quantile"])
@pytest.mark.parametrize("rule", ["midpoint", "simpson", "gauss2"])
@pytest.mark.parametrize("states", [1, 3])
def test_quadrature_selection_matches_oracle(grid, rule, states):
    import paper_1601_06767_gb300 as P
    pr = make_problem("c2")
    for N0, dE in ((pr.N0, pr.dE), (40, 0.11), (5999, 0.2)):
        c, E, w = P.select_quadrature(pr.E_c, N0, dE, pr.dos_A, pr.dos_V0, pr.E_max, grid, rule, states)
        ref = oracle_select(pr.E_c, N0, dE, pr.dos_A, pr.dos_V0, pr.E_max, grid, rule, states)
        assert np.array_equal(c, ref["cols"]), (grid, rule, states, N0)
        assert np.allclose(E, ref["E_col"], rtol=4e-16 * 8, atol=0)
        assert np.allclose(w, ref["w_col"], rtol=1e-14, atol=0)


def test_quadrature_selection_ties_and_arguments():
    import paper_1601_06767_gb300 as P
    rng = np.random.default_rng(3)
    E_c = np.sort(np.round(rng.uniform(0.2, 2.2, 300), 2))
    for grid in ("uniform", "quantile"):
        for rule in ("midpoint", "simpson", "gauss2"):
            c, E, w = P.select_quadrature(E_c, 25, 0.037, 80.0, 0.17, 2.2, grid, rule, 4)
            ref = oracle_select(E_c, 25, 0.037, 80.0, 0.17, 2.2, grid, rule, 4)
            assert np.array_equal(c, ref["cols"])
    # uniform midpoint with one state is Eq. 4's selection
    a = P.select_quadrature(E_c, 25, 0.037, 80.0, 0.17, 2.2)
    b = P.select_accelerated(E_c, 25, 0.037, 80.0, 0.17, 2.2)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    with pytest.raises(P.Chi0Error):
        P.select_quadrature(E_c[::-1], 25, 0.037, 80.0, 0.17, 2.2)
    with pytest.raises(KeyError):
        P.select_quadrature(E_c, 25, 0.037, 80.0, 0.17, 2.2, rule="trapezoid")


@pytest.mark.parametrize("n_split,states", [(0, 1), (5, 1), (40, 2)])
def test_adaptive_selection_matches_oracle(n_split, states):
    import paper_1601_06767_gb300 as P
    from oracle.quadrature import select_adaptive as oracle_adaptive
    pr = make_problem("c2")
    rng = np.random.default_rng(n_split)
    sens = rng.standard_normal(pr.n_c) * np.exp(-2.0 * (pr.E_c - pr.E_c[pr.N0 - 1]).clip(0))
    c, E, w = P.select_adaptive(pr.E_c, sens, pr.N0, pr.dE, pr.dos_A, pr.dos_V0, pr.E_max, n_split, states)
    ref = oracle_adaptive(pr.E_c, sens, pr.N0, pr.dE, pr.dos_A, pr.dos_V0, pr.E_max, n_split, states)
    assert np.array_equal(c, ref["cols"])
    assert np.allclose(E, ref["E_col"], rtol=1e-15, atol=0)
    assert np.allclose(w, ref["w_col"], rtol=1e-14, atol=0)
    if n_split == 0:
        a = P.select_accelerated(pr.E_c, pr.N0, pr.dE, pr.dos_A, pr.dos_V0, pr.E_max)
        assert all(np.array_equal(x, y) for x, y in zip((c, E, w), a))
