"""FP64 CPU oracle for constant-potential electrostatics (test infrastructure only).

Plain, slow and checkable by eye: direct Ewald sums, a dense Cholesky factorisation and the KKT
system for the electrode charges.  Only the test suite, the smoke check and the benchmark's CPU
baseline leg may import it; the GPU library never does, and the two share no code.
"""
from .ewald import KE  # noqa: F401
from . import ewald, cpm, profile, md  # noqa: F401
