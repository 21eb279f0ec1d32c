"""CPU oracle for the CLoD-GS rasterizer hot path.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg.  Nothing in the product package imports it.
"""
