"""Measurement helpers shipped with the library (peak microbenchmarks)."""
