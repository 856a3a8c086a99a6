"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Superposition-of-atomic-densities (SAD) initial guess, plain FP64 numpy. The paper names no initial
guess; the reading used here:

* Every element of the molecule gets a spherically averaged, fractional-occupation restricted DF-HF of
  the neutral atom, in the atom's own orbital and auxiliary shells as the molecule uses them.
* Occupations: Aufbau over the orbital energies; a set of degenerate orbitals (a shell of l > 0 of a
  spherical atom) shares the electrons that reach it equally (occupation <= 2 each), which keeps the
  density spherical.
* The restricted ensemble's Fock matrix is F = H + J[D] - K, with D = sum_i n_i C_i C_i^T and K the
  orbital-form exchange of the weighted orbitals C_i sqrt(n_i / 2) (eqs. 1-2, first forms), i.e. half the
  exchange matrix of D; energy E = 1/2 tr(D (H + F)). For integer occupations this is the closed-shell RHF
  of dfrhf.scf.
* The molecule's guess is the block-diagonal assembly of its atoms' densities, scaled so that
  tr(D S) = N electrons.
"""
from __future__ import annotations

import numpy as np

from . import dfrhf


def aufbau_occupations(eps: np.ndarray, nelec: float, tol: float = 1e-6) -> np.ndarray:
    """Occupations of orbitals with ascending energies eps: sets of degenerate orbitals (energies within
    tol * max(1, |eps|) of the set's first) are filled together, each member taking an equal share of at
    most 2 electrons."""
    occ = np.zeros(len(eps))
    left = float(nelec)
    i = 0
    while left > 0 and i < len(eps):
        j = i + 1
        while j < len(eps) and abs(eps[j] - eps[i]) <= tol * max(1.0, abs(eps[i])):
            j += 1
        take = min(left, 2.0 * (j - i))
        occ[i:j] = take / (j - i)
        left -= take
        i = j
    return occ


def atom_system(sys, a: int):
    """The single atom `a` of `sys` with its own orbital and auxiliary shells (same order as in sys)."""
    from dataclasses import replace
    atoms = sys.atoms[a:a + 1].copy()
    basis = sys.basis[sys.basis["atom"] == a].copy()
    aux = sys.aux[sys.aux["atom"] == a].copy()
    basis["atom"] = 0
    aux["atom"] = 0
    return replace(sys, atoms=atoms, basis=basis, aux=aux, charge=0, label=f"atom{a}")


def atomic_scf(atom, nelec: float | None = None, conv_E: float = 1e-11, conv_err: float = 1e-9,
               max_iter: int = 200, diis_size: int = 8):
    """Fractional-occupation restricted DF-HF of one atom (or any system): returns (D, energy, eps, occ,
    iterations). Core-Hamiltonian start, Pulay DIIS on X^T (F D S - S D F) X as in dfrhf.scf; converged to
    |dE| < 1e-11 Eh and max|e| < 1e-9 (tighter than the molecular SCF: the guess should not carry the
    atoms' convergence noise)."""
    if nelec is None:
        nelec = float(atom.atoms["Z"].sum())
    S = dfrhf.overlap(atom)
    H = dfrhf.core_hamiltonian(atom)
    B = dfrhf.whiten(dfrhf.three_center(atom), dfrhf.metric(atom))
    e_nuc = dfrhf.nuclear_repulsion(atom.atoms)
    X, _ = dfrhf.canonical_orthogonalizer(S)

    def occupy(Fm):
        eps, V = np.linalg.eigh(X.T @ Fm @ X)
        C = X @ V
        occ = aufbau_occupations(eps, nelec)
        m = int(np.count_nonzero(occ))
        Cw = C[:, :m] * np.sqrt(occ[:m] / 2.0)       # weighted orbitals: D = 2 Cw Cw^T
        return 2.0 * Cw @ Cw.T, Cw, eps, occ

    D, Cw, eps, occ = occupy(H)
    diis = dfrhf.DIIS(diis_size)
    e_old = None
    energy = 0.0
    it = 0
    for it in range(1, max_iter + 1):
        F = H + dfrhf.df_J(B, D) - dfrhf.df_K(B, Cw)
        energy = 0.5 * np.sum(D * (H + F)) + e_nuc
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        if e_old is not None and abs(energy - e_old) < conv_E and np.abs(err).max() < conv_err:
            break
        e_old = energy
        diis.push(F, err)
        D, Cw, eps, occ = occupy(diis.extrapolate() if it >= 2 else F)
    return D, energy, eps, occ, it


def sad_density(sys) -> np.ndarray:
    """Block-diagonal superposition of the atoms' fractional-occupation densities (one atomic SCF per
    element, in the molecule's basis order), scaled to tr(D S) = N."""
    n = dfrhf.nfunc(sys.basis)
    off = np.concatenate([[0], np.cumsum(2 * sys.basis["l"] + 1)])
    D0 = np.zeros((n, n))
    cache = {}
    for a in range(len(sys.atoms)):
        shells = np.flatnonzero(sys.basis["atom"] == a)
        if len(shells) == 0:
            continue
        z = int(sys.atoms["Z"][a])
        if z not in cache:
            cache[z] = atomic_scf(atom_system(sys, a))[0]
        lo, hi = off[shells[0]], off[shells[-1] + 1]
        D0[lo:hi, lo:hi] = cache[z]
    S = dfrhf.overlap(sys)
    return D0 * (sys.n_electrons / np.sum(D0 * S))
