"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Density-fitted restricted open-shell Hartree-Fock (the paper lists RHF, UHF and ROHF on the
density-fitted Fock builder, section "Program features", "Standard algorithms"), plain FP64 numpy.
The paper fixes no coupling operator; the reading used here:

* One set of orthonormal orbitals C: n_beta closed (c), n_alpha - n_beta open (o), the rest virtual (v).
  D_a = C[:, :n_alpha] C[:, :n_alpha]^T, D_b = C[:, :n_beta] C[:, :n_beta]^T.
* The Fock matrices and the energy are those of the unrestricted functional (dfuhf):
  F_s = H + J[D_a + D_b] - K_s (eqs. 1-3), E = 1/2 tr(D_a (H + F_a)) + 1/2 tr(D_b (H + F_b)) + E_nuc.
* Effective Fock matrix in the basis of the current orbitals, block by class pair:
  c-o: F_b; o-v: F_a; every other pair (c-c, o-o, v-v, c-v): F_c = (F_a + F_b) / 2.
  Its off-diagonal class blocks are the orbital gradient of E (dE/dk_pq = 2 sum_s (n^s_q - n^s_p) F^s_pq
  for the rotation C -> C exp(k), p < q): -2 F_b on c-o, -2 F_a on o-v, -4 F_c on c-v. The diagonal
  blocks only fix the canonical orbitals, not the converged energy.
* Step: diagonalise the effective matrix (taken to the orthogonal basis X^T S X = 1), occupy by energy.
  A level shift adds lambda to the virtual and lambda / 2 to the open diagonal of the effective matrix
  (in the basis of the current orbitals) before the step: it does not move the stationary point (it
  commutes with the projectors on the current classes) but damps the exchange of open and virtual
  orbitals, without which the iteration on the 2-water doublet cation oscillates for hundreds of steps.
  Pulay DIIS over the shifted effective matrix with the error = its off-diagonal class blocks (same
  basis); converged when |dE| < conv_E and the largest error element is below conv_err.
  Core-Hamiltonian start.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dfrhf
from .dfuhf import spin_contamination


@dataclass
class ROHFResult:
    energy: float
    iterations: int
    converged: bool
    C: np.ndarray
    eps: np.ndarray
    Da: np.ndarray
    Db: np.ndarray
    s2: float


def classes(nmo: int, nalpha: int, nbeta: int) -> np.ndarray:
    """Class of every orbital: 0 closed, 1 open, 2 virtual."""
    c = np.full(nmo, 2)
    c[:nalpha] = 1
    c[:nbeta] = 0
    return c


def uhf_functional(sys, B, H, C, nalpha, nbeta, e_nuc):
    """Energy and spin Fock matrices of the orbitals C (columns) with n_alpha / n_beta occupied."""
    Ca, Cb = C[:, :nalpha], C[:, :nbeta]
    Da, Db = Ca @ Ca.T, Cb @ Cb.T
    J = dfrhf.df_J(B, Da + Db)
    Fa = H + J - dfrhf.df_K(B, Ca)
    Fb = H + J - (dfrhf.df_K(B, Cb) if nbeta > 0 else 0.0)
    E = 0.5 * np.sum(Da * (H + Fa)) + 0.5 * np.sum(Db * (H + Fb)) + e_nuc
    return E, Fa, Fb, Da, Db


def effective_fock_mo(Fa_mo, Fb_mo, nalpha, nbeta):
    """The effective Fock matrix in the orbital basis and its off-diagonal class blocks (the error)."""
    cls = classes(len(Fa_mo), nalpha, nbeta)
    p, q = cls[:, None], cls[None, :]
    F = 0.5 * (Fa_mo + Fb_mo)
    co = ((p == 0) & (q == 1)) | ((p == 1) & (q == 0))
    ov = ((p == 1) & (q == 2)) | ((p == 2) & (q == 1))
    F = np.where(co, Fb_mo, np.where(ov, Fa_mo, F))
    err = np.where(p != q, F, 0.0)
    return F, err


def orbital_gradient(Fa_mo, Fb_mo, nalpha, nbeta):
    """dE/dk_pq (p < q entries; the matrix is antisymmetric) of C -> C exp(k)."""
    nmo = len(Fa_mo)
    na = np.zeros(nmo)
    nb = np.zeros(nmo)
    na[:nalpha] = 1.0
    nb[:nbeta] = 1.0
    G = 2.0 * ((na[None, :] - na[:, None]) * Fa_mo + (nb[None, :] - nb[:, None]) * Fb_mo)
    return np.triu(G, 1) - np.triu(G, 1).T


def rohf(sys, nalpha: int, nbeta: int, conv_E: float = 1e-10, conv_err: float = 1e-7, max_iter: int = 200,
         diis_size: int = 8, B: np.ndarray | None = None, level_shift: float = 0.5) -> ROHFResult:
    if nalpha + nbeta != sys.n_electrons or nalpha < nbeta or nbeta < 0:
        raise ValueError("nalpha + nbeta must equal the electron count, nalpha >= nbeta >= 0")
    S = dfrhf.overlap(sys)
    H = dfrhf.core_hamiltonian(sys)
    if B is None:
        B = dfrhf.whiten(dfrhf.three_center(sys), dfrhf.metric(sys))
    e_nuc = dfrhf.nuclear_repulsion(sys.atoms)
    X, _ = dfrhf.canonical_orthogonalizer(S)
    eps, U = np.linalg.eigh(X.T @ H @ X)            # U: orbitals in the orthogonal basis (columns)
    diis = dfrhf.DIIS(diis_size)
    e_old = None
    energy = 0.0
    converged = False
    it = 0
    Da = Db = None
    for it in range(1, max_iter + 1):
        C = X @ U
        energy, Fa, Fb, Da, Db = uhf_functional(sys, B, H, C, nalpha, nbeta, e_nuc)
        Fe_mo, e_mo = effective_fock_mo(C.T @ Fa @ C, C.T @ Fb @ C, nalpha, nbeta)
        cls = classes(len(Fe_mo), nalpha, nbeta)
        Fe_mo = Fe_mo + np.diag(np.where(cls == 2, level_shift, np.where(cls == 1, 0.5 * level_shift, 0.0)))
        Fe = U @ Fe_mo @ U.T                          # orthogonal basis
        err = U @ e_mo @ U.T
        if e_old is not None and abs(energy - e_old) < conv_E and np.abs(err).max() < conv_err:
            converged = True
            break
        e_old = energy
        diis.push(Fe, err)
        eps, U = np.linalg.eigh(diis.extrapolate() if it >= 2 else Fe)
    C = X @ U
    return ROHFResult(energy=energy, iterations=it, converged=converged, C=C, eps=eps, Da=Da, Db=Db,
                      s2=spin_contamination(Da, Db, S, nalpha, nbeta))
