"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds input generators only: triangulations, member parameters
and the closed-form initial, boundary and forcing fields of the experiments
of Section 4.  It contains none of the scheme's arithmetic (no quadrature,
no finite element basis, no assembly, no solve), so that the CPU oracle and
the CUDA path can both consume it without sharing any of the method.
"""
from .mesh import unit_square, channel_step, barycentric_refine, Mesh  # noqa: F401
from .ensembles import (  # noqa: F401
    Ensemble, perturbation_factor, manufactured, config_manufactured_small, lid_cavity,
    channel, sensitivity, convergence_study, energy_study, batched_family,
)
