"""CPU oracle for the surfel rendering path (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package. The library itself never does.
"""
