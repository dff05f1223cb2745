"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark."""
from .fem import (Problem, assemble, poisson_dirichlet, helmholtz_impedance, gaussian_source,  # noqa: F401
                  helmholtz_macro, helmholtz_batch)
