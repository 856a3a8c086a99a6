"""ORACLE -- test infrastructure only.

A plain, slow FP64 CPU implementation of the density-fitted RHF step: McMurchie-Davidson
integrals in C (md_integrals.c), the density-fitting / SCF algebra in numpy (dfrhf.py; unrestricted
Hartree-Fock in dfuhf.py, restricted open-shell Hartree-Fock in dfrohf.py, the closed-shell MP2
energy in dfmp2.py, the density-fitting object operations of eqs. (1)-(3) in dfops.py, the DF-RHF
nuclear gradient in dfgrad.py), the
superposition-of-atomic-densities guess (sad.py) and the guess network's forward and backward pass
(mlp.py).
Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import it;
the product path (the CUDA library and its binding) never does, and the two share no code.
"""
