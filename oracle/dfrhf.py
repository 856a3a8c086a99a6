"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain FP64 density-fitted restricted Hartree-Fock, written from the definitions:

* Three-index tensor I_{gamma,rs} kept in memory (paper, section "Density fitting utilities"):
  here the Coulomb-metric-whitened B_{P,mu nu} = sum_Q (L^-1)_{PQ} (Q|mu nu), (P|Q) = L L^T,
  i.e. the auxiliary-index transformation of eq. (1) with M' = L^-1.
* Coulomb matrix from eq. (3): gamma_P = sum_{mu nu} B_{P,mu nu} D_{mu nu} (first form),
  J_{mu nu} = sum_P gamma_P B_{P,mu nu} (second form).
* Exchange from eqs. (1)-(2): Y_{P,mu i} = sum_nu B_{P,mu nu} C_{nu i} (first form of eq. 1),
  K_{mu nu} = sum_{P,i} Y_{P,mu i} Y_{P,nu i} (first form of eq. 2). With D = 2 C_occ C_occ^T this K
  is the exchange of the occupied orbitals, half of the exchange matrix of D.
* RHF (paper, section "Standard algorithms": a Fock builder using density fitting):
  F = H + J - K, E = 1/2 tr(D (H + F)) + E_nuc, D = 2 C_occ C_occ^T, Roothaan F C = S C eps with
  Aufbau occupation, core-Hamiltonian guess, Pulay DIIS on X^T (F D S - S D F) X.

Library primitives (numpy matmul, cholesky, triangular solve, eigh) serve as steps; nothing is
blocked or fused. Convergence: |E_n - E_{n-1}| < conv_E and max |X^T(FDS - SDF)X| < conv_err.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile md_integrals.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "md_integrals.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i = ctypes.c_double, ctypes.c_int
        P = ctypes.POINTER
        _lib.or_boys.argtypes = [i, d, P(d)]
        for name in ("or_prim_overlap", "or_prim_kinetic"):
            getattr(_lib, name).restype = d
            getattr(_lib, name).argtypes = [P(i), d, P(d), P(i), d, P(d)]
        _lib.or_prim_potential.restype = d
        _lib.or_prim_potential.argtypes = [P(i), d, P(d), P(i), d, P(d), P(d)]
        _lib.or_prim_eri.restype = d
        _lib.or_prim_eri.argtypes = [P(i), d, P(d), P(i), d, P(d), P(i), d, P(d), P(i), d, P(d)]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------------------------------------
# primitive-level access (used by the pins)
# ---------------------------------------------------------------------------------------------

def boys(mmax: int, T: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    lib().or_boys(mmax, float(T), _dp(out))
    return out


def _pw(p):
    return np.ascontiguousarray(p, dtype=np.int32)


def _xyz(c):
    return np.ascontiguousarray(c, dtype=np.float64)


def prim_overlap(pa, a, A, pb, b, B) -> float:
    pa, pb, A, B = _pw(pa), _pw(pb), _xyz(A), _xyz(B)
    return lib().or_prim_overlap(_ip(pa), a, _dp(A), _ip(pb), b, _dp(B))


def prim_kinetic(pa, a, A, pb, b, B) -> float:
    pa, pb, A, B = _pw(pa), _pw(pb), _xyz(A), _xyz(B)
    return lib().or_prim_kinetic(_ip(pa), a, _dp(A), _ip(pb), b, _dp(B))


def prim_potential(pa, a, A, pb, b, B, C) -> float:
    """<a| 1/|r-C| |b> (positive operator)."""
    pa, pb, A, B, C = _pw(pa), _pw(pb), _xyz(A), _xyz(B), _xyz(C)
    return lib().or_prim_potential(_ip(pa), a, _dp(A), _ip(pb), b, _dp(B), _dp(C))


def prim_eri(pa, a, A, pb, b, B, pc, c, C, pd, d, D) -> float:
    """(ab|cd) over unnormalised Cartesian primitives; exponent 0 with power 0 is 'no function'."""
    args = []
    for p, e, X in ((pa, a, A), (pb, b, B), (pc, c, C), (pd, d, D)):
        p, X = _pw(p), _xyz(X)
        args += [p, X]
        del p, X
    pa_, A_, pb_, B_, pc_, C_, pd_, D_ = args
    return lib().or_prim_eri(_ip(pa_), a, _dp(A_), _ip(pb_), b, _dp(B_), _ip(pc_), c, _dp(C_),
                             _ip(pd_), d, _dp(D_))


def prim_3c(pp, ap, P, pa, a, A, pb, b, B) -> float:
    """(p|ab) over unnormalised Cartesian primitives."""
    return prim_eri(pp, ap, P, (0, 0, 0), 0.0, P, pa, a, A, pb, b, B)


def solid_harmonic_coeffs(l: int) -> tuple[np.ndarray, np.ndarray]:
    """Real solid harmonic coefficients (2l+1, ncart) and the Cartesian powers (ncart, 3)."""
    nc = (l + 1) * (l + 2) // 2
    cs = np.zeros((2 * l + 1) * nc)
    pw = np.zeros(3 * nc, dtype=np.int32)
    L = lib()
    L.or_solid_harmonic_coeffs.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.or_cart_powers.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.or_solid_harmonic_coeffs(l, _dp(cs))
    L.or_cart_powers(l, _ip(pw))
    return cs.reshape(2 * l + 1, nc), pw.reshape(nc, 3)


def sph_norms(l: int, a: float) -> np.ndarray:
    out = np.zeros(2 * l + 1)
    L = lib()
    L.or_sph_norms.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.or_sph_norms(l, a, _dp(out))
    return out


# ---------------------------------------------------------------------------------------------
# matrices over a system (shell arrays come from paper_1707_03771_gb300.clusters)
# ---------------------------------------------------------------------------------------------

def _shell_arrays(shells):
    l = np.ascontiguousarray(shells["l"], dtype=np.int32)
    a = np.ascontiguousarray(shells["exponent"], dtype=np.float64)
    xyz = np.ascontiguousarray(shells["center"], dtype=np.float64).reshape(-1)
    return l, a, xyz


def nfunc(shells) -> int:
    return int((2 * shells["l"] + 1).sum())


def _matrix(fn, shells, *extra):
    l, a, xyz = _shell_arrays(shells)
    n = nfunc(shells)
    out = np.zeros((n, n))
    f = getattr(lib(), fn)
    f.restype = None
    f(ctypes.c_int(len(l)), _ip(l), _dp(a), _dp(xyz), *extra, _dp(out))
    return out


def overlap(sys) -> np.ndarray:
    return _matrix("or_overlap", sys.basis)


def kinetic(sys) -> np.ndarray:
    return _matrix("or_kinetic", sys.basis)


def nuclear(sys) -> np.ndarray:
    Z = np.ascontiguousarray(sys.atoms["Z"], dtype=np.float64)
    R = np.ascontiguousarray(sys.atoms["xyz"], dtype=np.float64).reshape(-1)
    return _matrix("or_nuclear", sys.basis, ctypes.c_int(len(Z)), _dp(Z), _dp(R))


def core_hamiltonian(sys) -> np.ndarray:
    return kinetic(sys) + nuclear(sys)


def metric(sys) -> np.ndarray:
    """(P|Q) two-centre Coulomb metric over the auxiliary basis."""
    return _matrix("or_metric", sys.aux)


def three_center(sys) -> np.ndarray:
    """(P|mu nu) as a dense (naux, n, n) array."""
    la, aa, xa = _shell_arrays(sys.aux)
    l, a, xyz = _shell_arrays(sys.basis)
    naux, n = nfunc(sys.aux), nfunc(sys.basis)
    out = np.zeros((naux, n, n))
    f = lib().or_three_center
    f.restype = None
    f(ctypes.c_int(len(la)), _ip(la), _dp(aa), _dp(xa), ctypes.c_int(len(l)), _ip(l), _dp(a), _dp(xyz),
      _dp(out))
    return out


def three_center_triples(sys, triples) -> list[np.ndarray]:
    """(P|mu nu) blocks for a list of shell triples (P, M, N); each block is (2lP+1, 2lM+1, 2lN+1)."""
    triples = np.ascontiguousarray(triples, dtype=np.int32).reshape(-1, 3)
    la, aa, xa = _shell_arrays(sys.aux)
    l, a, xyz = _shell_arrays(sys.basis)
    sizes = [(2 * sys.aux["l"][p] + 1, 2 * sys.basis["l"][m] + 1, 2 * sys.basis["l"][nn] + 1)
             for p, m, nn in triples]
    counts = np.array([int(np.prod(s)) for s in sizes], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    out = np.zeros(int(counts.sum()))
    f = lib().or_three_center_triples
    f.restype = None
    f(ctypes.c_int(len(la)), _ip(la), _dp(aa), _dp(xa), ctypes.c_int(len(l)), _ip(l), _dp(a), _dp(xyz),
      ctypes.c_int(len(triples)), _ip(triples), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out))
    return [out[o:o + c].reshape(s) for o, c, s in zip(offs, counts, sizes)]


def four_center(sys) -> np.ndarray:
    """Conventional (mu nu|la si) as an (n, n, n, n) array; tiny systems only."""
    l, a, xyz = _shell_arrays(sys.basis)
    n = nfunc(sys.basis)
    out = np.zeros((n, n, n, n))
    f = lib().or_four_center
    f.restype = None
    f(ctypes.c_int(len(l)), _ip(l), _dp(a), _dp(xyz), _dp(out))
    return out


def nuclear_repulsion(atoms) -> float:
    R = np.asarray(atoms["xyz"], dtype=np.float64)
    Z = np.asarray(atoms["Z"], dtype=np.float64)
    e = 0.0
    for i in range(len(Z)):
        for j in range(i):
            e += Z[i] * Z[j] / np.linalg.norm(R[i] - R[j])
    return e


# ---------------------------------------------------------------------------------------------
# density fitting (paper eqs. 1-3)
# ---------------------------------------------------------------------------------------------

def whiten(three: np.ndarray, V: np.ndarray) -> np.ndarray:
    """B = L^-1 (Q|mu nu) with (P|Q) = L L^T (auxiliary-index transform of eq. 1, M' = L^-1)."""
    L = np.linalg.cholesky(V)
    naux, n, _ = three.shape
    from scipy.linalg import solve_triangular
    return solve_triangular(L, three.reshape(naux, n * n), lower=True).reshape(naux, n, n)


def df_J(B: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Eq. (3): gamma_P = sum_{rs} B_{P,rs} D_rs, then J_rs = sum_P gamma_P B_{P,rs}."""
    gamma = np.einsum("prs,rs->p", B, D)
    return np.einsum("p,prs->rs", gamma, B)


def df_Y(B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Eq. (1), first form: Y_{P,mu i} = sum_nu B_{P,mu nu} C_{nu i}."""
    return np.einsum("pmn,ni->pmi", B, C)


def df_K(B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Eq. (2), first form: K_{mu nu} = sum_{P,i} Y_{P,mu i} Y_{P,nu i}."""
    Y = df_Y(B, C)
    return np.einsum("pmi,pni->mn", Y, Y)


def conv_J(eri: np.ndarray, D: np.ndarray) -> np.ndarray:
    return np.einsum("mnls,ls->mn", eri, D)


def conv_K(eri: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Exchange of the occupied orbitals: sum_{l s} (m l|n s) sum_i C_li C_si."""
    P = C @ C.T
    return np.einsum("mlns,ls->mn", eri, P)


# ---------------------------------------------------------------------------------------------
# RHF
# ---------------------------------------------------------------------------------------------

@dataclass
class SCFResult:
    energy: float
    e_nuc: float
    iterations: int
    converged: bool
    D: np.ndarray
    C: np.ndarray
    eps: np.ndarray
    F: np.ndarray
    J: np.ndarray
    K: np.ndarray
    n_dropped: int
    history: list = field(default_factory=list)
    timings: dict = field(default_factory=dict)


def canonical_orthogonalizer(S: np.ndarray, tol: float = 1e-7):
    s, U = np.linalg.eigh(S)
    keep = s > tol
    return U[:, keep] / np.sqrt(s[keep]), int((~keep).sum())


def _solve_roothaan(F, X, nocc):
    e, Cp = np.linalg.eigh(X.T @ F @ X)
    C = X @ Cp
    return C, e


class DIIS:
    """Pulay DIIS: minimise |sum c_i e_i| subject to sum c_i = 1 (Lagrange row)."""

    def __init__(self, size: int = 8):
        self.size = size
        self.F: list[np.ndarray] = []
        self.E: list[np.ndarray] = []

    def push(self, F, err):
        self.F.append(F.copy())
        self.E.append(err.copy())
        if len(self.F) > self.size:
            self.F.pop(0)
            self.E.pop(0)

    def extrapolate(self) -> np.ndarray:
        while True:
            m = len(self.F)
            if m < 2:
                return self.F[-1]
            Bm = -np.ones((m + 1, m + 1))
            Bm[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    Bm[i, j] = np.vdot(self.E[i], self.E[j])
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                c = np.linalg.solve(Bm, rhs)
                if np.all(np.isfinite(c)) and np.linalg.cond(Bm) < 1e14:
                    return sum(ci * Fi for ci, Fi in zip(c[:m], self.F))
            except np.linalg.LinAlgError:
                pass
            self.F.pop(0)
            self.E.pop(0)


def scf(sys, conv_E: float = 1e-10, conv_err: float = 1e-7, max_iter: int = 100, diis_size: int = 8,
        B: np.ndarray | None = None, H: np.ndarray | None = None, S: np.ndarray | None = None,
        jk=None) -> SCFResult:
    """DF-RHF from the core-Hamiltonian guess. `jk(D, C_occ) -> (J, K)` overrides the DF J/K
    (used for the conventional four-index reference)."""
    t0 = time.time()
    if S is None:
        S = overlap(sys)
    if H is None:
        H = core_hamiltonian(sys)
    timings = {"one_electron_s": time.time() - t0}
    if jk is None:
        if B is None:
            t1 = time.time()
            A = three_center(sys)
            timings["three_center_s"] = time.time() - t1
            t1 = time.time()
            B = whiten(A, metric(sys))
            timings["whiten_s"] = time.time() - t1

        def jk(D, Cocc):
            return df_J(B, D), df_K(B, Cocc)
    e_nuc = nuclear_repulsion(sys.atoms)
    nocc = sys.nocc
    X, ndrop = canonical_orthogonalizer(S)
    C, eps = _solve_roothaan(H, X, nocc)
    D = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    diis = DIIS(diis_size)
    e_old = None
    history = []
    converged = False
    J = K = F = None
    t_iter = time.time()
    it = 0
    for it in range(1, max_iter + 1):
        Cocc = C[:, :nocc]
        J, K = jk(D, Cocc)
        F = H + J - K
        energy = 0.5 * np.sum(D * (H + F)) + e_nuc
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        err_max = float(np.abs(err).max())
        dE = None if e_old is None else energy - e_old
        history.append({"iter": it, "energy": energy, "dE": dE, "err": err_max})
        if e_old is not None and abs(dE) < conv_E and err_max < conv_err:
            converged = True
            break
        e_old = energy
        diis.push(F, err)
        Fx = diis.extrapolate() if it >= 2 else F
        C, eps = _solve_roothaan(Fx, X, nocc)
        D = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    timings["iterations_s"] = time.time() - t_iter
    return SCFResult(energy=energy, e_nuc=e_nuc, iterations=it, converged=converged, D=D, C=C, eps=eps,
                     F=F, J=J, K=K, n_dropped=ndrop, history=history, timings=timings)


def conventional_scf(sys, **kw) -> SCFResult:
    """RHF with exact four-index J and K (tiny systems), same SCF driver."""
    eri = four_center(sys)
    return scf(sys, jk=lambda D, Cocc: (conv_J(eri, D), conv_K(eri, Cocc)), **kw)
