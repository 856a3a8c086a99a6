"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Density-fitted closed-shell MP2 correlation energy (the paper lists MP2 among the programs on the
density-fitting utilities, section "Program features"), plain FP64 numpy:

* the fitted occupied-virtual objects B^P_ia = sum_{mu nu} C_mu i B_P,mu nu C_nu a: two index
  transformations of eq. (1) (first form), applied to both orbital indices;
* the integrals (ia|jb) = sum_P B^P_ia B^P_jb: eq. (2), second form (a contraction of two fitted
  objects into a four-index quantity);
* E2 = sum_{ij ab} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b) over canonical RHF orbitals,
  every orbital correlated (the paper names no frozen core).
"""
from __future__ import annotations

import numpy as np


def ov_objects(B: np.ndarray, C: np.ndarray, nocc: int) -> np.ndarray:
    """B^P_ia (naux, nocc, nvir) from B (naux, n, n) and the orbitals C (n, nmo), occupied first."""
    Co, Cv = C[:, :nocc], C[:, nocc:]
    Y = np.einsum("pmn,mi->pin", B, Co, optimize=True)        # first index transformation
    return np.einsum("pin,na->pia", Y, Cv, optimize=True)     # second


def mp2_energy(B: np.ndarray, C: np.ndarray, eps: np.ndarray, nocc: int) -> float:
    """The closed-shell MP2 correlation energy of the canonical orbitals C with energies eps."""
    Bia = ov_objects(B, C, nocc)
    eo, ev = eps[:nocc], eps[nocc:]
    e2 = 0.0
    for i in range(nocc):
        for j in range(nocc):
            V = Bia[:, i, :].T @ Bia[:, j, :]                  # (ia|jb) over (a, b)
            denom = eo[i] + eo[j] - ev[:, None] - ev[None, :]
            e2 += float(np.sum(V * (2.0 * V - V.T) / denom))
    return e2


def mp2_energy_spin_orbital(B: np.ndarray, C: np.ndarray, eps: np.ndarray, nocc: int) -> float:
    """The same energy from the spin-orbital form 1/4 sum |<ij||ab>|^2 / (e_i + e_j - e_a - e_b) over
    spin orbitals (alpha and beta copies of every spatial orbital), as an independent check of the
    closed-shell spin summation."""
    Bia = ov_objects(B, C, nocc)
    eo, ev = eps[:nocc], eps[nocc:]
    nv = len(ev)
    g = np.einsum("pia,pjb->iajb", Bia, Bia, optimize=True)   # (ia|jb) in spatial orbitals
    so, sv = 2 * nocc, 2 * nv
    occ_sp = np.arange(so) % 2
    vir_sp = np.arange(sv) % 2
    io, iv = np.arange(so) // 2, np.arange(sv) // 2
    e2 = 0.0
    for I in range(so):
        for J in range(so):
            for A in range(sv):
                # <IJ|AB> = (IA|JB) if spin(I) = spin(A) and spin(J) = spin(B)
                s_ia = occ_sp[I] == vir_sp[A]
                coul = np.where(s_ia & (occ_sp[J] == vir_sp), g[io[I], iv[A], io[J], iv], 0.0)
                # <IJ|BA> = (IB|JA) if spin(I) = spin(B) and spin(J) = spin(A)
                exch = np.where((occ_sp[I] == vir_sp) & (occ_sp[J] == vir_sp[A]), g[io[I], iv, io[J], iv[A]], 0.0)
                anti = coul - exch
                denom = eo[io[I]] + eo[io[J]] - ev[iv[A]] - ev[iv]
                e2 += float(np.sum(anti * anti / denom))
    return 0.25 * e2
