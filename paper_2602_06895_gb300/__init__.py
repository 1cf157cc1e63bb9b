"""GB300-native phase-space hot path (arXiv 2602.06895): batched map from uniform
random numbers to weighted collider events, as sm_103a CUDA behind a C ABI.

The native library is loaded lazily by :mod:`paper_2602_06895_gb300.ps`.
"""
