"""GB300-native HSS-ULV factorization and solve.

The compute path lives in the CUDA library built from ``csrc/`` (loaded on
first use by ``paper_2311_00921_gb300.hss``); ``inputs`` builds seeded
synthetic HSS matrices.
"""
