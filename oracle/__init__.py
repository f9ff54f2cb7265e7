"""FP64 CPU oracle of the MLS-MPM Neo-Hookean step.

TEST INFRASTRUCTURE ONLY: imported by tests/, the package smoke check and
bench.py's CPU-baseline leg; never by the CUDA library or its binding.
"""
