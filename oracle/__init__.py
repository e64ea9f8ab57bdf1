"""FP64 CPU oracle of the multi-product imaginary-time propagation method.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the library.
"""
