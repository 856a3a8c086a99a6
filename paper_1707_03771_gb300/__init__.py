"""GB300-native density-fitted RHF hot path: three-index integrals, metric whitening and the
per-iteration J/K contractions, behind a C-ABI library (libdfhf.so) with a thin ctypes binding.

Importing the package loads nothing; `paper_1707_03771_gb300.binding` loads the CUDA library and
fails loudly when it has not been built.
"""
