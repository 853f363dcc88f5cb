"""CPU oracle for the theta-join and k-closest-pairs query.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's
CPU-baseline leg, never by the engine.
"""
