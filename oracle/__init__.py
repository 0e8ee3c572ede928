"""Plain FP64 CPU oracle for the RPA polarizability hot path (test infrastructure).

This package is test infrastructure only: it is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference legs of
``bench.py``.  The library path never calls it.  It shares no code with the
CUDA path; the only common module is ``synth`` (seeded inputs, no method
arithmetic).

Functions without an independent pin say "parity unpinned" in their
docstring; every other function is pinned by ``tests/test_oracle_*.py``.
"""
from .chi0_oracle import (wfn_to_grid, pair_elements, freq_factor, chi0_from_pairs, chi0_rows,
                          dos, select_accelerated, accelerated_pairs, chi0_full,
                          chi0_accelerated, full_pairs, chi0_grad, loss_diag,
                          rel_fro, chi0_k_points, grid_energy_of_bands,
                          energy_substitution_estimate)

__all__ = ["wfn_to_grid", "pair_elements", "freq_factor", "chi0_from_pairs", "chi0_rows", "dos",
           "select_accelerated", "accelerated_pairs", "chi0_full", "chi0_accelerated",
           "full_pairs", "chi0_grad", "loss_diag", "rel_fro", "chi0_k_points",
           "grid_energy_of_bands", "energy_substitution_estimate"]
