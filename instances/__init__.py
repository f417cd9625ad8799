"""Seeded synthetic SOS programs shared by the oracle and the CUDA path.

This package only *describes* problems: polynomials as sparse
``{exponent tuple: coefficient}`` maps and, for each SOS constraint, which
Gram blocks (basis degree, optional weight polynomial) it uses.  It holds none
of the method's arithmetic: no monomial-basis indexing, no coefficient
matching, no conic data, no ADMM.  Both the CPU oracle and the GPU library
build their own conic form from these descriptions.
"""

from .program import Block, Constraint, SOSProgram  # noqa: F401
from . import workloads  # noqa: F401
