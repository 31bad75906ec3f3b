"""FP64 CPU oracle for the ParaDIAG step with the additive Vanka multigrid.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  `core` wraps the C
oracle (oracle.c), `lfa` is the local Fourier analysis of Sec. 2.1 in numpy.
"""
