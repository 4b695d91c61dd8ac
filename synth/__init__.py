"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and assembles arrays: mechanism descriptions
(species formulas, NASA-7 coefficient sets, Arrhenius/third-body/Troe
parameters) and initial fields (temperature and mass-fraction profiles).  It
evaluates no part of the method itself -- no thermodynamic functions, rates,
right-hand sides or integrator steps -- so that neither the CUDA path nor the
oracle can hide a mistake in code the two share.
"""

from .mechanism import Mechanism, generate_mechanism, ELEMENTS, ELEMENT_MASS
from .fields import (
    WORKLOADS,
    Workload,
    workload,
    field_uniform,
    field_tanh_front,
    field_gaussian3d,
)

__all__ = [
    "Mechanism",
    "generate_mechanism",
    "ELEMENTS",
    "ELEMENT_MASS",
    "WORKLOADS",
    "Workload",
    "workload",
    "field_uniform",
    "field_tanh_front",
    "field_gaussian3d",
]
