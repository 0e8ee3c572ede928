"""Seeded synthetic inputs shaped like the MgO supercells of the paper.

This package holds input generation only: lattices, plane-wave spheres,
random band coefficients, band energies, frequency lists and the parameters of
the free-electron density-of-states model.  It contains none of the method's
arithmetic (no pair elements, no energy denominators, no polarizability, no
quadrature); both the FP64 oracle and the CUDA path consume what it produces.
"""
from .mgo import (CONFIGS, HARTREE_EV, Problem, band_coefficients, make_problem,
                  pw_sphere, g_sphere, valence_energies, conduction_energies,
                  imag_frequencies)

__all__ = ["CONFIGS", "HARTREE_EV", "Problem", "band_coefficients", "make_problem",
           "pw_sphere", "g_sphere", "valence_energies", "conduction_energies",
           "imag_frequencies"]
