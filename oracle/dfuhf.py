"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Density-fitted unrestricted Hartree-Fock (the paper lists RHF, UHF and ROHF on the density-fitted Fock
builder, section "Program features", "Standard algorithms"), plain FP64 numpy:

* spin densities D_s = C_s,occ C_s,occ^T (s = alpha, beta; no factor 2);
* J = J[D_a + D_b] (eq. 3), K_s = sum_{P,i in s} Y_P,mu i Y_P,nu i with Y_P = B_P C_s,occ (eqs. 1-2, first
  forms), the full exchange of the spin density D_s;
* F_s = H + J - K_s, E = 1/2 tr(D_a (H + F_a)) + 1/2 tr(D_b (H + F_b)) + E_nuc;
* Pulay DIIS over the pair (F_a, F_b) with the error pair X^T (F_s D_s S - S D_s F_s) X (one set of
  coefficients for both spins), core-Hamiltonian start for both spins, Aufbau per spin;
* converged when |dE| < conv_E and the largest error element of both spins is below conv_err.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dfrhf


@dataclass
class UHFResult:
    energy: float
    iterations: int
    converged: bool
    Da: np.ndarray
    Db: np.ndarray
    eps_a: np.ndarray
    eps_b: np.ndarray
    s2: float


def spin_contamination(Da: np.ndarray, Db: np.ndarray, S: np.ndarray, na: int, nb: int) -> float:
    """<S^2> of the UHF determinant: S_z (S_z + 1) + n_beta - tr(D_a S D_b S), S_z = (n_alpha - n_beta) / 2."""
    sz = 0.5 * (na - nb)
    return sz * (sz + 1.0) + nb - float(np.sum((Da @ S) * (Db @ S).T))


def uhf(sys, nalpha: int, nbeta: int, conv_E: float = 1e-10, conv_err: float = 1e-7, max_iter: int = 200,
        diis_size: int = 8, B: np.ndarray | None = None) -> UHFResult:
    if nalpha + nbeta != sys.n_electrons or nalpha < nbeta or nbeta < 0:
        raise ValueError("nalpha + nbeta must equal the electron count, nalpha >= nbeta >= 0")
    S = dfrhf.overlap(sys)
    H = dfrhf.core_hamiltonian(sys)
    if B is None:
        B = dfrhf.whiten(dfrhf.three_center(sys), dfrhf.metric(sys))
    e_nuc = dfrhf.nuclear_repulsion(sys.atoms)
    X, _ = dfrhf.canonical_orthogonalizer(S)

    def roothaan(F):
        eps, V = np.linalg.eigh(X.T @ F @ X)
        return X @ V, eps

    C, eps = roothaan(H)
    Ca, Cb, ea, eb = C, C, eps, eps
    diis = dfrhf.DIIS(diis_size)
    e_old = None
    energy = 0.0
    it = 0
    converged = False
    Da = Db = None
    for it in range(1, max_iter + 1):
        Coa, Cob = Ca[:, :nalpha], Cb[:, :nbeta]
        Da, Db = Coa @ Coa.T, Cob @ Cob.T
        J = dfrhf.df_J(B, Da + Db)
        Fa = H + J - dfrhf.df_K(B, Coa)
        Fb = H + J - (dfrhf.df_K(B, Cob) if nbeta > 0 else 0.0)
        energy = 0.5 * np.sum(Da * (H + Fa)) + 0.5 * np.sum(Db * (H + Fb)) + e_nuc
        err_a = X.T @ (Fa @ Da @ S - S @ Da @ Fa) @ X
        err_b = X.T @ (Fb @ Db @ S - S @ Db @ Fb) @ X
        err = max(np.abs(err_a).max(), np.abs(err_b).max())
        if e_old is not None and abs(energy - e_old) < conv_E and err < conv_err:
            converged = True
            break
        e_old = energy
        diis.push(np.concatenate([Fa, Fb]), np.concatenate([err_a, err_b]))
        Fx = diis.extrapolate() if it >= 2 else np.concatenate([Fa, Fb])
        n = H.shape[0]
        Ca, ea = roothaan(Fx[:n])
        Cb, eb = roothaan(Fx[n:])
    return UHFResult(energy=energy, iterations=it, converged=converged, Da=Da, Db=Db, eps_a=ea, eps_b=eb,
                     s2=spin_contamination(Da, Db, S, nalpha, nbeta))
