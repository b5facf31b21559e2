"""Plain FP64 CPU oracle of the KPM hot path -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; the product library never does.
"""
