"""GB300-native RPA polarizability (chi0) hot path: pair matrix elements and
the denominator-weighted contraction of Eq. 1, plain and with the accelerated
conduction-band summation of Eq. 3/4.  The compute lives in libchi0.so
(CUDA, sm_103a); this package is a thin binding over its C ABI."""
from ._lib import Chi0Error, lib  # noqa: F401
from .api import (Chi0DiagLoss, Chi0Fn, Chi0Plan, energy_substitution_estimate,  # noqa: F401
                  grid_energies_of_bands, select_accelerated, select_adaptive,
                  select_quadrature)

__all__ = ["Chi0Plan", "Chi0Fn", "Chi0DiagLoss", "Chi0Error", "select_accelerated", "select_quadrature", "select_adaptive", "lib",
           "energy_substitution_estimate", "grid_energies_of_bands"]
