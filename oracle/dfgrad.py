"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Nuclear gradient of the density-fitted RHF energy (the paper lists analytic gradients among the programs,
section "Program features", built on integrals "and their geometric derivatives", section "Molecular
integrals"), plain FP64 numpy.

With A_P,mu nu = (P|mu nu), V = (P|Q), the converged orbitals C (occupied i, j), D = 2 C_occ C_occ^T and
W = 2 sum_i e_i C_i C_i^T, the energy of the RHF functional with the fitted J and exchange is
    E = E_nuc + tr(D H) + 1/2 a^T V^-1 a - sum_ij (P|ij) [V^-1]_PQ (Q|ij),
    a_P = sum_mu nu A_P,mu nu D_mu nu,  (P|ij) = sum_mu nu C_mu i A_P,mu nu C_nu j.
Its derivative along a nuclear coordinate x (the orbitals' response enters only through the
orthonormality constraint, the -tr(W S^x) term):
    dE/dx = dE_nuc/dx + tr(D H^x) - tr(W S^x)
            + c . a^x - 1/2 c^T V^x c                        (c = V^-1 a)
            - 2 sum_P,ij (P|ij)^x Z_P,ij + sum_PQ V^x_PQ sum_ij Z_P,ij Z_Q,ij   (Z = V^-1 (Q|ij))
where a^x, (P|ij)^x use the derivative integrals A^x with D and C held fixed. The derivative integrals
S^x, H^x (basis centres and the moving nucleus' attraction), A^x and V^x are taken as the derivative of
the integral matrices with respect to moving one atom with its orbital and auxiliary shells, by
sixth-order central differences of the integrals (step 5e-4 bohr).
"""
from __future__ import annotations

import copy

import numpy as np

from . import dfrhf


def displaced(sys, atom: int, d: int, h: float):
    """The system with atom `atom` and every orbital and auxiliary shell centred on it moved by h along
    coordinate d."""
    s = copy.deepcopy(sys)
    s.atoms["xyz"][atom, d] += h
    for shells in (s.basis, s.aux):
        sel = shells["atom"] == atom
        shells["center"][sel, d] += h
    return s


def _integrals(sys):
    return dfrhf.overlap(sys), dfrhf.core_hamiltonian(sys), dfrhf.three_center(sys), dfrhf.metric(sys)


def integral_derivatives(sys, atom: int, d: int, h: float = 5e-4):
    """(S^x, H^x, A^x, V^x) for the coordinate (atom, d), sixth-order central differences."""
    f = [_integrals(displaced(sys, atom, d, k * h)) for k in (-3, -2, -1, 1, 2, 3)]
    return tuple((45.0 * (f[3][q] - f[2][q]) - 9.0 * (f[4][q] - f[1][q]) + (f[5][q] - f[0][q])) / (60.0 * h)
                 for q in range(4))


def nuclear_repulsion_gradient(atoms) -> np.ndarray:
    R = np.asarray(atoms["xyz"], dtype=np.float64)
    Z = np.asarray(atoms["Z"], dtype=np.float64)
    g = np.zeros_like(R)
    for i in range(len(Z)):
        for j in range(len(Z)):
            if i != j:
                rij = R[i] - R[j]
                g[i] -= Z[i] * Z[j] * rij / np.linalg.norm(rij) ** 3
    return g


def gradient(sys, res=None, h: float = 5e-4) -> np.ndarray:
    """dE/dR (natom x 3) at the converged DF-RHF solution `res` (dfrhf.scf; computed if None). The metric
    terms are evaluated in the whitened form (triangular solves with the Cholesky factor V = L L^T, the
    way the energy itself is formed): c . a^x - 1/2 c^T V^x c = g . (L^-1 a^x) - 1/2 g^T (L^-1 V^x L^-T) g
    with g = L^-1 a, and likewise for the exchange terms with L^-1 (P|ij); an explicit V^-1 would lose
    kappa(V) eps (about 1e-7 here) of terms that cancel to the gradient."""
    from scipy.linalg import cholesky, solve_triangular
    A = dfrhf.three_center(sys)
    V = dfrhf.metric(sys)
    if res is None:
        res = dfrhf.scf(sys, B=dfrhf.whiten(A, V), conv_E=1e-12, conv_err=1e-9)
    nocc = sys.nocc
    Co = res.C[:, :nocc]
    D = 2.0 * Co @ Co.T
    W = 2.0 * (Co * res.eps[:nocc]) @ Co.T
    L = cholesky(V, lower=True)

    def linv(X):
        return solve_triangular(L, X, lower=True)

    naux = V.shape[0]
    gam = linv(np.einsum("pmn,mn->p", A, D))
    Bij = linv(np.einsum("pmn,mi,nj->pij", A, Co, Co, optimize=True).reshape(naux, -1))
    BB = Bij @ Bij.T
    g = nuclear_repulsion_gradient(sys.atoms)
    for atom in range(len(sys.atoms)):
        for d in range(3):
            Sx, Hx, Ax, Vx = integral_derivatives(sys, atom, d, h)
            Mx = linv(linv(Vx).T)                      # L^-1 V^x L^-T (V^x symmetric)
            gax = linv(np.einsum("pmn,mn->p", Ax, D))
            Bijx = linv(np.einsum("pmn,mi,nj->pij", Ax, Co, Co, optimize=True).reshape(naux, -1))
            g[atom, d] += (np.sum(D * Hx) - np.sum(W * Sx) + gam @ gax - 0.5 * gam @ Mx @ gam
                           - 2.0 * np.sum(Bijx * Bij) + np.sum(Mx * BB))
    return g
