"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/chi0.h declares, and its host-only band selection
(Eq. 3/4) equals the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1601_06767_gb300 as P
from paper_1601_06767_gb300 import _lib as L
from oracle import select_accelerated as oracle_select
from synth import HARTREE_EV, make_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chi0.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chi0_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound():
    names = _declared()
    assert len(names) >= 10
    h = C.CDLL(L.LIB_PATH)
    for n in names:
        assert hasattr(h, n), n
    bound = {s[0] for s in L.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_create_rejects_bad_descriptions_without_a_device():
    lib = P.lib()
    h = C.c_void_p()
    assert lib.chi0_plan_create(C.byref(h), None) == L.CHI0_ERR_INVALID
    assert b"desc" in lib.chi0_last_error(None)
    d = L.Chi0PlanDesc()
    d.n1 = d.n2 = d.n3 = 1
    assert lib.chi0_plan_create(C.byref(h), C.byref(d)) == L.CHI0_ERR_INVALID
    assert h.value is None


def _oracle_columns(E_c, N0, dE, A, V0, Emax):
    o = oracle_select(E_c, N0, dE, A, V0, Emax)
    c = np.concatenate([o["explicit"], o["rep"]])
    E = np.concatenate([np.asarray(E_c)[o["explicit"]], o["E_i"]])
    w = np.concatenate([np.ones(o["explicit"].size), o["w_i"]])
    return c, E, w


@pytest.mark.parametrize("name", ["c2", "c5"])
@pytest.mark.parametrize("dE_eV", [1.5, 2.0, 2.5, 3.0, 3.5, 4.0])
def test_select_matches_oracle(name, dE_eV):
    pr = make_problem(name)
    dE = dE_eV / HARTREE_EV
    c, E, w = P.select_accelerated(pr.E_c, pr.N0, dE, pr.dos_A, pr.dos_V0, pr.E_max)
    oc, oE, ow = _oracle_columns(pr.E_c, pr.N0, dE, pr.dos_A, pr.dos_V0, pr.E_max)
    assert np.array_equal(c, oc)
    assert np.array_equal(E, oE)
    assert np.allclose(w, ow, rtol=1e-15, atol=0)


def test_select_ties_and_degenerate_bands():
    rng = np.random.default_rng(0)
    E_c = np.sort(np.round(rng.uniform(0.17, 2.2, 400), 2))   # many exact degeneracies
    for N0 in (0, 1, 37, 399, 400, 500):
        c, E, w = P.select_accelerated(E_c, N0, 0.031, 80.0, 0.17, 2.2)
        oc, oE, ow = _oracle_columns(E_c, N0, 0.031, 80.0, 0.17, 2.2)
        assert np.array_equal(c, oc) and np.array_equal(E, oE) and np.allclose(w, ow, rtol=1e-15)


def test_select_rejects_unsorted_and_small_capacity():
    lib = P.lib()
    E = np.array([0.3, 0.2, 0.5])
    out_c = np.empty(8, np.int32)
    out_e = np.empty(8)
    out_w = np.empty(8)
    assert lib.chi0_select_accelerated(E.ctypes.data, 3, 1, 0.1, 1.0, 0.17, 2.2, out_c.ctypes.data,
                                       out_e.ctypes.data, out_w.ctypes.data, 8) == -1
    E = np.sort(E)
    assert lib.chi0_select_accelerated(E.ctypes.data, 3, 1, 0.1, 1.0, 0.17, 2.2, out_c.ctypes.data,
                                       out_e.ctypes.data, out_w.ctypes.data, 2) == -1


def test_create_rejects_bad_hermitian_flag_without_a_device():
    import numpy as np
    lib = P.lib()
    g = np.zeros((1, 3), np.int32)
    nG = np.ones(1, np.int32)
    fr = np.zeros(1)
    d = L.Chi0PlanDesc()
    d.n1 = d.n2 = d.n3 = 24
    d.n_q = 1
    d.n_G = nG.ctypes.data_as(C.POINTER(C.c_int32))
    d.gvec = g.ctypes.data_as(C.POINTER(C.c_int32))
    d.n_freq = 1
    d.freq_re = fr.ctypes.data_as(C.POINTER(C.c_double))
    d.freq_im = fr.ctypes.data_as(C.POINTER(C.c_double))
    d.delta = 1e-3
    d.precision = L.CHI0_SPLIT_BF16
    d.hermitian = 5
    h = C.c_void_p()
    assert lib.chi0_plan_create(C.byref(h), C.byref(d)) == L.CHI0_ERR_INVALID
    assert b"hermitian" in lib.chi0_last_error(None)
    assert h.value is None


def test_host_selection_entry_points_reject_bad_arguments():
    import numpy as np
    lib = P.lib()
    E = np.array([0.2, 0.3, 0.5, 0.9])
    s = np.ones(4)
    c = np.empty(256, np.int32)
    e = np.empty(256)
    w = np.empty(256)
    ok = lib.chi0_select_quadrature(E.ctypes.data, 4, 2, 0.1, 1.0, 0.17, 2.2, 1, 1, 2, c.ctypes.data, e.ctypes.data,
                                    w.ctypes.data, 256)
    assert ok == 2 + 2 * 39                 # 19 bins, 39 Simpson nodes, 2 states each
    for grid, rule, states in ((2, 0, 1), (0, 3, 1), (0, 0, 0)):
        assert lib.chi0_select_quadrature(E.ctypes.data, 4, 2, 0.1, 1.0, 0.17, 2.2, grid, rule, states,
                                          c.ctypes.data, e.ctypes.data, w.ctypes.data, 64) == -1
    assert lib.chi0_select_quadrature(E.ctypes.data, 4, 2, 0.1, 1.0, 0.17, 2.2, 0, 0, 1, c.ctypes.data,
                                      e.ctypes.data, w.ctypes.data, 3) == -1          # capacity
    assert lib.chi0_select_adaptive(E.ctypes.data, 4, 2, s.ctypes.data, 0.1, 1.0, 0.17, 2.2, 3, 1,
                                    c.ctypes.data, e.ctypes.data, w.ctypes.data, 64) > 2
    assert lib.chi0_select_adaptive(E.ctypes.data, 4, 2, None, 0.1, 1.0, 0.17, 2.2, 3, 1,
                                    c.ctypes.data, e.ctypes.data, w.ctypes.data, 64) == -1
    assert lib.chi0_select_adaptive(E.ctypes.data, 4, 2, s.ctypes.data, 0.1, 1.0, 0.17, 2.2, -1, 1,
                                    c.ctypes.data, e.ctypes.data, w.ctypes.data, 64) == -1


@pytest.mark.parametrize("name,dE_eV", [("c2", 2.0), ("c5", 2.0), ("c5", 0.37), ("c1", 1.5)])
def test_grid_energies_match_oracle(name, dE_eV):
    """chi0_grid_energies (host C) gives every band the same Eq. 4 grid energy
    as the oracle, bit for bit."""
    from oracle import grid_energy_of_bands
    pr = make_problem(name)
    N0 = pr.N0 if pr.N0 else 40
    dE = dE_eV / HARTREE_EV
    got = P.grid_energies_of_bands(pr.E_c, N0, dE, pr.E_max)
    assert np.array_equal(got, grid_energy_of_bands(pr.E_c, N0, dE, pr.E_max))


def test_grid_energies_edge_cases():
    from oracle import grid_energy_of_bands
    rng = np.random.default_rng(9)
    E = np.sort(rng.uniform(0.2, 2.0, 200))
    E0, dE = E[19], 0.05
    E[60] = E0 + 3 * dE                 # exactly on an interior edge: the upper step holds it
    E[-3:] = [2.3, 2.4, 2.5]            # above E_max: the last step
    E.sort()
    for N0, Emax in ((20, 2.2), (0, 2.2), (200, 2.2), (250, 2.2), (20, E0), (20, E0 - 0.1), (1, 2.2)):
        got = P.grid_energies_of_bands(E, N0, dE, Emax)
        assert np.array_equal(got, grid_energy_of_bands(E, N0, dE, Emax)), (N0, Emax)
    assert np.array_equal(P.grid_energies_of_bands(E[:0], 5, dE, 2.2), E[:0])
    with pytest.raises(L.Chi0Error):
        P.grid_energies_of_bands(E, 5, 0.0, 2.2)
