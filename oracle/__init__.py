"""ORACLE -- test infrastructure only.

A plain, slow FP64 CPU implementation of the density-fitted RHF step: McMurchie-Davidson
integrals in C (md_integrals.c) and the density-fitting / SCF algebra in numpy (dfrhf.py).
Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import it;
the product path (the CUDA library and its binding) never does, and the two share no code.
"""
