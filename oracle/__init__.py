"""CPU oracle for TSDF-Sampling (arXiv 2311.17878).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg.  The product path never imports it, and it
imports nothing from the product package except the seeded input generators.
"""
