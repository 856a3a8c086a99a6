"""Thin ctypes binding of libdfhf.so (include/dfhf.h): argument marshalling only.

Every computation runs in the CUDA library; importing this module raises if the library has not
been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DF_OK, DF_E_ARG, DF_E_NOMEM, DF_E_CUDA, DF_E_NOTCONV, DF_E_STATE, DF_E_NUMERIC, DF_E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
DF_PREC_FP64, DF_PREC_SPLIT = 0, 1
DF_WHITEN_SPLIT, DF_WHITEN_FP64 = 0, 1
DF_GUESS_CORE, DF_GUESS_SAD, DF_GUESS_SPIN = 0, 1, 2

EXPORTED = ["df_init", "df_sizes", "df_build_B", "df_build_B_ex", "df_jk", "scf_run", "df_get_rows", "df_get_matrix", "df_rys",
            "df_prepare", "df_set_stream", "df_timings", "df_free", "df_strerror", "df_last_error",
            "df_coulomb_noalloc", "df_scf_history", "scf_run_batch", "scf_run_guess", "df_mlp_create",
            "df_mlp_free", "df_mlp_nparams", "df_mlp_params", "df_mlp_gradients", "df_mlp_train", "df_mlp_predict",
            "df_water_features", "df_water_blocks", "df_water_density", "df_mlp_guess", "df_rint_pow2",
            "df_fp64_rate", "df_sad_density", "df_build_B_batch",
            "df_init_open", "scf_run_uhf", "scf_run_rohf", "df_water_pairs", "df_pair_blocks", "df_pair_density",
            "df_mlp_guess_pairs", "df_mp2", "df_tensor_create", "df_tensor_from_B", "df_tensor_shape",
            "df_tensor_get", "df_tensor_free", "df_op_transform", "df_op_contract", "df_op_density_fit",
            "df_op_density_back", "df_op_apply_four_index"]
DF_MLP_NFEAT = 57
DF_MLP_NPFEAT = 26
PAIR_CUTOFF = 7.5      # bohr, O-O distance of the water pairs whose blocks the pair network predicts


class Atom(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_double * 3), ("Z", ctypes.c_int)]


class Shell(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("l", ctypes.c_int), ("exponent", ctypes.c_double),
                ("center", ctypes.c_double * 3)]


class Options(ctypes.Structure):
    _fields_ = [("conv_E", ctypes.c_double), ("conv_err", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("diis_size", ctypes.c_int), ("guess", ctypes.c_int), ("precision", ctypes.c_int),
                ("slices", ctypes.c_int), ("incremental", ctypes.c_int), ("screen_tau", ctypes.c_double),
                ("approx_diag", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("e_nuc", ctypes.c_double), ("e_one", ctypes.c_double),
                ("e_coul", ctypes.c_double), ("e_exch", ctypes.c_double), ("last_dE", ctypes.c_double),
                ("last_err", ctypes.c_double), ("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("status", ctypes.c_int), ("n_dropped", ctypes.c_int), ("ramp_iteration", ctypes.c_int),
                ("incremental_builds", ctypes.c_int), ("approx_steps", ctypes.c_int), ("t_build_s", ctypes.c_double),
                ("t_iter_s", ctypes.c_double), ("t_jk_s", ctypes.c_double), ("t_total_s", ctypes.c_double),
                ("s2", ctypes.c_double), ("graph_launches", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libdfhf.so (built by paper_1707_03771_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libdfhf.so not built ({path}); run paper_1707_03771_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, c_int, c_double, c_void_p = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    dp = P(c_double)
    L.df_init.argtypes = [P(Atom), c_int, P(Shell), c_int, P(Shell), c_int, c_int, P(c_void_p)]
    L.df_sizes.argtypes = [c_void_p, P(c_int), P(c_int), P(c_int), P(ctypes.c_longlong)]
    L.df_build_B.argtypes = [c_void_p, c_double, c_int]
    L.df_build_B_ex.argtypes = [c_void_p, c_double, c_int, c_int]
    L.df_jk.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_int, c_int]
    L.scf_run.argtypes = [c_void_p, P(Options), P(Result)]
    L.df_get_rows.argtypes = [c_void_p, c_int, c_int, c_int, dp]
    L.df_get_matrix.argtypes = [c_void_p, c_int, dp]
    L.df_rys.argtypes = [dp, c_int, c_int, dp, dp]
    L.df_rint_pow2.argtypes = [dp, P(c_int), ctypes.c_longlong, P(ctypes.c_longlong)]
    L.df_prepare.argtypes = []
    L.df_fp64_rate.argtypes = [c_int, ctypes.c_longlong, dp, dp]
    L.df_sad_density.argtypes = [c_void_p, dp]
    L.df_build_B_batch.argtypes = [P(c_void_p), c_int, c_double, c_int, c_int]
    L.df_init_open.argtypes = [P(Atom), c_int, P(Shell), c_int, P(Shell), c_int, c_int, P(c_void_p)]
    L.scf_run_uhf.argtypes = [c_void_p, P(Options), c_int, c_int, P(Result)]
    L.scf_run_rohf.argtypes = [c_void_p, P(Options), c_int, c_int, ctypes.c_double, P(Result)]
    L.df_coulomb_noalloc.argtypes = [c_void_p, c_void_p, c_void_p]
    L.df_scf_history.argtypes = [c_void_p, dp, c_int]
    L.scf_run_batch.argtypes = [P(c_void_p), c_int, P(Options), P(Result)]
    L.scf_run_guess.argtypes = [c_void_p, P(Options), dp, P(Result)]
    fp = P(ctypes.c_float)
    L.df_mlp_create.argtypes = [c_int, c_int, c_int, c_int, ctypes.c_ulonglong, P(c_void_p)]
    L.df_mlp_free.argtypes = [c_void_p]
    L.df_mlp_free.restype = None
    L.df_mlp_nparams.argtypes = [c_void_p]
    L.df_mlp_nparams.restype = ctypes.c_longlong
    L.df_mlp_params.argtypes = [c_void_p, fp, c_int]
    L.df_mlp_gradients.argtypes = [c_void_p, fp, fp, c_int, fp, fp]
    L.df_mlp_train.argtypes = [c_void_p, fp, fp, c_int, c_int, c_int, ctypes.c_float, ctypes.c_ulonglong, fp]
    L.df_mlp_predict.argtypes = [c_void_p, fp, c_int, c_int, fp]
    L.df_water_features.argtypes = [P(Atom), c_int, fp]
    L.df_water_blocks.argtypes = [c_void_p, dp, fp]
    L.df_water_density.argtypes = [c_void_p, fp, dp]
    L.df_mlp_guess.argtypes = [c_void_p, c_void_p, c_int, dp]
    ip = P(c_int)
    L.df_water_pairs.argtypes = [P(Atom), c_int, ctypes.c_double, ip, c_int, fp]
    L.df_pair_blocks.argtypes = [c_void_p, dp, ip, c_int, fp]
    L.df_pair_density.argtypes = [c_void_p, fp, ip, c_int, dp]
    L.df_mlp_guess_pairs.argtypes = [c_void_p, c_void_p, c_void_p, ctypes.c_double, c_int, dp]
    L.df_mp2.argtypes = [c_void_p, dp, dp, c_int, c_int, dp]
    L.df_tensor_create.argtypes = [c_void_p, c_int, c_int, c_int, dp, P(c_void_p)]
    L.df_tensor_from_B.argtypes = [c_void_p, P(c_void_p)]
    L.df_tensor_shape.argtypes = [c_void_p, P(c_int), P(c_int), P(c_int)]
    L.df_tensor_get.argtypes = [c_void_p, dp]
    L.df_tensor_free.argtypes = [c_void_p]
    L.df_tensor_free.restype = None
    L.df_op_transform.argtypes = [c_void_p, c_int, dp, c_int, c_int, P(c_void_p)]
    L.df_op_contract.argtypes = [c_void_p, c_void_p, c_int, dp]
    L.df_op_density_fit.argtypes = [c_void_p, dp, dp]
    L.df_op_density_back.argtypes = [c_void_p, dp, dp]
    L.df_op_apply_four_index.argtypes = [c_void_p, dp, c_int, c_int, P(c_void_p)]
    L.df_set_stream.argtypes = [c_void_p, c_void_p]
    L.df_timings.argtypes = [c_void_p, dp, c_int]
    L.df_free.argtypes = [c_void_p]
    L.df_free.restype = None
    L.df_strerror.argtypes = [c_int]
    L.df_strerror.restype = ctypes.c_char_p
    L.df_last_error.argtypes = [c_void_p]
    L.df_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


class DFError(RuntimeError):
    def __init__(self, code, detail=""):
        self.code = code
        super().__init__(f"{load().df_strerror(code).decode()} ({code}) {detail}".strip())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _shells(arr):
    out = (Shell * len(arr))()
    for i, s in enumerate(arr):
        out[i].atom = int(s["atom"])
        out[i].l = int(s["l"])
        out[i].exponent = float(s["exponent"])
        out[i].center[:] = [float(x) for x in s["center"]]
    return out


def _atoms(arr):
    out = (Atom * len(arr))()
    for i, a in enumerate(arr):
        out[i].xyz[:] = [float(x) for x in a["xyz"]]
        out[i].Z = int(a["Z"])
    return out


MATRIX = {"S": 0, "T": 1, "V": 2, "H": 3, "metric": 4, "Linv": 5, "D": 6, "F": 7, "J": 8, "K": 9, "C": 10, "eps": 11,
          "Da": 12, "Db": 13}


class Handle:
    """One molecule on the GPU: wraps df_init ... df_free."""

    def __init__(self, system, open_shell: bool = False):
        """open_shell: df_init_open (any electron count, for scf_uhf)."""
        L = load()
        self.system = system
        h = ctypes.c_void_p()
        atoms, basis, aux = _atoms(system.atoms), _shells(system.basis), _shells(system.aux)
        init = L.df_init_open if open_shell else L.df_init
        rc = init(atoms, len(system.atoms), basis, len(system.basis), aux, len(system.aux), int(system.charge),
                  ctypes.byref(h))
        if rc != DF_OK:
            raise DFError(rc, "df_init")
        self.h = h
        n, na, no, row = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        L.df_sizes(h, ctypes.byref(n), ctypes.byref(na), ctypes.byref(no), ctypes.byref(row))
        self.n, self.naux, self.nocc, self.packed_row = n.value, na.value, no.value, row.value

    def _check(self, rc, what):
        if rc != DF_OK:
            raise DFError(rc, f"{what}: {load().df_last_error(self.h).decode()}")

    def build_B(self, screen_tau: float = 0.0, keep_3c: bool = False, whitening: int | None = None):
        """df_build_B, or df_build_B_ex when `whitening` (DF_WHITEN_*) is given."""
        if whitening is None:
            self._check(load().df_build_B(self.h, screen_tau, int(keep_3c)), "df_build_B")
        else:
            self._check(load().df_build_B_ex(self.h, screen_tau, int(keep_3c), int(whitening)), "df_build_B_ex")

    def jk(self, D, C_occ, precision=DF_PREC_FP64, slices=3):
        """J, K for host arrays D (n x n) and C_occ (n x nocc); returns numpy arrays."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        C = np.ascontiguousarray(C_occ, dtype=np.float64)
        J = np.empty((self.n, self.n))
        K = np.empty((self.n, self.n))
        rc = load().df_jk(self.h, D.ctypes.data, C.ctypes.data, C.shape[1], J.ctypes.data, K.ctypes.data, 0,
                          precision, slices)
        self._check(rc, "df_jk")
        return J, K

    def jk_device(self, D_ptr, C_ptr, nocc, J_ptr, K_ptr, precision=DF_PREC_FP64, slices=3):
        """J, K with device pointers (e.g. torch tensors' data_ptr())."""
        rc = load().df_jk(self.h, D_ptr, C_ptr, nocc, J_ptr, K_ptr, 1, precision, slices)
        self._check(rc, "df_jk")

    def coulomb_noalloc(self, D_ptr, J_ptr):
        """J for device D through df_coulomb_noalloc (no device allocation inside the call)."""
        self._check(load().df_coulomb_noalloc(self.h, D_ptr, J_ptr), "df_coulomb_noalloc")

    def scf(self, conv_E=1e-10, conv_err=1e-7, max_iter=100, diis_size=8, precision=DF_PREC_FP64, slices=3,
            incremental=0, screen_tau=0.0, guess=None, approx_diag=0):
        """SCF from the core-Hamiltonian guess, from the superposition of atomic densities (guess="sad"), or
        from the natural orbitals of a guess density (guess: an n x n array)."""
        sad = isinstance(guess, str)
        if sad and guess != "sad":
            raise ValueError("guess: None, 'sad' or an n x n density")
        o = Options(conv_E, conv_err, max_iter, diis_size, DF_GUESS_SAD if sad else DF_GUESS_CORE, precision, slices,
                    incremental, screen_tau, approx_diag)
        r = Result()
        if guess is None or sad:
            rc = load().scf_run(self.h, ctypes.byref(o), ctypes.byref(r))
        else:
            g = np.ascontiguousarray(guess, dtype=np.float64)
            rc = load().scf_run_guess(self.h, ctypes.byref(o), _dp(g), ctypes.byref(r))
        if rc not in (DF_OK, DF_E_NOTCONV):
            self._check(rc, "scf_run")
        return r.as_dict()

    def water_blocks(self, D):
        """Each water's diagonal block of D in its own frame (upper triangles, float32)."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        nbw = water_nbf(self.system)
        out = np.empty((len(self.system.atoms) // 3, nbw * (nbw + 1) // 2), dtype=np.float32)
        self._check(load().df_water_blocks(self.h, _dp(D), _fp(out)), "df_water_blocks")
        return out

    def water_density(self, blocks):
        blocks = np.ascontiguousarray(blocks, dtype=np.float32)
        D0 = np.empty((self.n, self.n))
        self._check(load().df_water_density(self.h, _fp(blocks), _dp(D0)), "df_water_density")
        return D0

    def mlp_guess(self, mlp, bf16=True, pair_mlp=None, cutoff=PAIR_CUTOFF):
        """Learned D0: diagonal water blocks from `mlp`, plus (if given) the blocks of the water pairs within
        `cutoff` bohr from `pair_mlp` (df_mlp_guess_pairs)."""
        D0 = np.empty((self.n, self.n))
        if pair_mlp is None:
            self._check(load().df_mlp_guess(self.h, mlp.m, int(bf16), _dp(D0)), "df_mlp_guess")
        else:
            self._check(load().df_mlp_guess_pairs(self.h, mlp.m, pair_mlp.m, float(cutoff), int(bf16), _dp(D0)),
                        "df_mlp_guess_pairs")
        return D0

    def mp2(self, C=None, eps=None, nocc=None, n_dropped=0):
        """DF-MP2 correlation energy (df_mp2) of the canonical orbitals C (n x nmo, columns ascending) with
        energies eps; by default those of the last scf() on this handle (n_dropped: its result's
        n_dropped)."""
        if C is None:
            nmo = self.n - n_dropped
            C = self.matrix("C").reshape(-1)[: self.n * nmo].reshape(self.n, nmo)
            eps = self.matrix("eps")[:nmo]
        C = np.ascontiguousarray(C, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        nocc = self.nocc if nocc is None else int(nocc)
        e2 = ctypes.c_double()
        self._check(load().df_mp2(self.h, _dp(C), _dp(eps), C.shape[1], nocc, ctypes.byref(e2)), "df_mp2")
        return e2.value

    def pair_blocks(self, D, pairs):
        """Frame blocks (npairs x nb x nb, float32) of the ordered water pairs `pairs` (npairs x 2) of D."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        nbw = water_nbf(self.system)
        out = np.empty((len(pairs), nbw, nbw), dtype=np.float32)
        self._check(load().df_pair_blocks(self.h, _dp(D), _ip(pairs), len(pairs), _fp(out)), "df_pair_blocks")
        return out

    def pair_density(self, blocks, pairs, D0=None):
        """D0 (zero if not given) plus the laboratory-frame pair blocks (df_pair_density)."""
        blocks = np.ascontiguousarray(blocks, dtype=np.float32)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        D0 = np.zeros((self.n, self.n)) if D0 is None else np.ascontiguousarray(D0, dtype=np.float64).copy()
        self._check(load().df_pair_density(self.h, _fp(blocks), _ip(pairs), len(pairs), _dp(D0)), "df_pair_density")
        return D0

    def scf_uhf(self, nalpha, nbeta, conv_E=1e-10, conv_err=1e-7, max_iter=200, diis_size=8, precision=DF_PREC_FP64,
                slices=3, screen_tau=0.0, guess="core"):
        """Unrestricted Hartree-Fock (scf_run_uhf) with nalpha and nbeta electrons, from the core Hamiltonian
        (guess="core") or from the spin densities of the last open-shell run on this handle (guess="spin")."""
        if guess not in ("core", "spin"):
            raise ValueError("guess: 'core' or 'spin'")
        g = DF_GUESS_CORE if guess == "core" else DF_GUESS_SPIN
        o = Options(conv_E, conv_err, max_iter, diis_size, g, precision, slices, 0, screen_tau, 0)
        r = Result()
        rc = load().scf_run_uhf(self.h, ctypes.byref(o), int(nalpha), int(nbeta), ctypes.byref(r))
        if rc not in (DF_OK, DF_E_NOTCONV):
            self._check(rc, "scf_run_uhf")
        return r.as_dict()

    def scf_rohf(self, nalpha, nbeta, level_shift=0.5, conv_E=1e-10, conv_err=1e-7, max_iter=200, diis_size=8,
                 precision=DF_PREC_FP64, slices=3, screen_tau=0.0):
        """Restricted open-shell Hartree-Fock (scf_run_rohf): nbeta closed and nalpha - nbeta open orbitals."""
        o = Options(conv_E, conv_err, max_iter, diis_size, DF_GUESS_CORE, precision, slices, 0, screen_tau, 0)
        r = Result()
        rc = load().scf_run_rohf(self.h, ctypes.byref(o), int(nalpha), int(nbeta), float(level_shift),
                                 ctypes.byref(r))
        if rc not in (DF_OK, DF_E_NOTCONV):
            self._check(rc, "scf_run_rohf")
        return r.as_dict()

    def sad_density(self):
        """The superposition-of-atomic-densities guess density (n x n), df_sad_density."""
        D0 = np.empty((self.n, self.n))
        self._check(load().df_sad_density(self.h, _dp(D0)), "df_sad_density")
        return D0

    def history(self):
        """Per-iteration rows of the last SCF: iteration, energy, dE, max|e|, slices, J/K ms."""
        L = load()
        n = L.df_scf_history(self.h, None, 0)
        if n < 0:
            raise DFError(n, "df_scf_history")
        out = np.zeros((max(n, 1), 6))
        L.df_scf_history(self.h, _dp(out), n)
        return out[:n]

    def rows(self, which, p0, count):
        out = np.empty((count, self.n, self.n))
        self._check(load().df_get_rows(self.h, which, p0, count, _dp(out)), "df_get_rows")
        return out

    def matrix(self, name):
        which = MATRIX[name]
        if name in ("metric", "Linv"):
            out = np.empty((self.naux, self.naux))
        elif name == "eps":
            out = np.empty(self.n)
        else:
            out = np.empty((self.n, self.n))
        self._check(load().df_get_matrix(self.h, which, _dp(out)), f"df_get_matrix({name})")
        return out

    def timings(self):
        out = np.zeros(20)
        load().df_timings(self.h, _dp(out), 20)
        keys = ["init_ms", "eri3c_ms", "cholesky_ms", "whiten_ms", "gamma_ms", "coulomb_ms", "ytransform_ms",
                "kcontract_ms", "split_ms", "split_y_ms", "split_k_ms", "split_other_ms", "tc_y_tile_n",
                "tc_k_split", "autotune_ms", "tc_k_tile_n", "jk_launches", "potrf_ms", "trtri_ms"]
        return dict(zip(keys, out[:len(keys)]))

    def close(self):
        if getattr(self, "h", None):
            # density-fitting objects made on this handle go first (they use its stream)
            for ref in getattr(self, "_tensors", []):
                t = ref()
                if t is not None:
                    t.close()
            load().df_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def scf_batch(handles, conv_E=1e-10, conv_err=1e-7, max_iter=100, diis_size=8, precision=DF_PREC_FP64, slices=3,
              screen_tau=0.0, incremental=0, approx_diag=0, guess=None):
    """Solve several molecules together (scf_run_batch); guess None (core Hamiltonian) or "sad". Returns one
    result dict per handle."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[hd.h.value for hd in handles])
    if guess not in (None, "sad"):
        raise ValueError("guess: None or 'sad'")
    o = Options(conv_E, conv_err, max_iter, diis_size, DF_GUESS_SAD if guess == "sad" else DF_GUESS_CORE, precision,
                slices, incremental, screen_tau, approx_diag)
    out = (Result * n)()
    rc = load().scf_run_batch(hs, n, ctypes.byref(o), out)
    if rc not in (DF_OK, DF_E_NOTCONV):
        failed = [(i, out[i].status, load().df_last_error(handles[i].h).decode()) for i in range(n)
                  if out[i].status not in (DF_OK, DF_E_NOTCONV)]
        detail = "; ".join(f"molecule {i}: status {st}: {msg}" for i, st, msg in failed[:4])
        raise DFError(rc, f"scf_run_batch: {len(failed)} of {n} failed: {detail}")
    return [out[i].as_dict() for i in range(n)]


def build_B_batch(handles, screen_tau=0.0, keep_3c=False, whitening=DF_WHITEN_SPLIT):
    """B for several molecules (df_build_B_batch): grouped three-centre integrals, then each molecule's
    metric factor and whitening."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[hd.h.value for hd in handles])
    rc = load().df_build_B_batch(hs, n, screen_tau, int(keep_3c), int(whitening))
    if rc != DF_OK:
        raise DFError(rc, "df_build_B_batch: " + load().df_last_error(handles[0].h).decode())


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def water_nbf(system) -> int:
    return int((2 * system.basis["l"][system.basis["atom"] < 3] + 1).sum())


def water_features(system):
    atoms = _atoms(system.atoms)
    nw = len(system.atoms) // 3
    out = np.empty((nw, DF_MLP_NFEAT), dtype=np.float32)
    rc = load().df_water_features(atoms, len(system.atoms), _fp(out))
    if rc < 0:
        raise DFError(rc, "df_water_features")
    return out


def water_pairs(system, cutoff=PAIR_CUTOFF):
    """Ordered water pairs within `cutoff` bohr (O-O), both orders: (pairs int32 (k, 2), features float32
    (k, DF_MLP_NPFEAT))."""
    atoms = _atoms(system.atoms)
    n = load().df_water_pairs(atoms, len(system.atoms), float(cutoff), None, 0, None)
    if n < 0:
        raise DFError(n, "df_water_pairs")
    pairs = np.zeros((n, 2), dtype=np.int32)
    feats = np.zeros((n, DF_MLP_NPFEAT), dtype=np.float32)
    if n:
        rc = load().df_water_pairs(atoms, len(system.atoms), float(cutoff), _ip(pairs), n, _fp(feats))
        if rc < 0:
            raise DFError(rc, "df_water_pairs")
    return pairs, feats


class DFTensor:
    """A density-fitting object I[g][r][s] on the device (df_tensor_*), with the operations of eqs. (1)-(3)
    (df_op_*). Results of eq. (2) and (3) that are matrices or vectors come back as numpy arrays; objects
    as new DFTensor instances. Close (or let go) every tensor before its Handle."""

    def __init__(self, handle, ptr):
        import weakref
        self.handle, self.t = handle, ptr
        if not hasattr(handle, "_tensors"):
            handle._tensors = []
        handle._tensors.append(weakref.ref(self))
        a, r, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        handle._check(load().df_tensor_shape(self.t, ctypes.byref(a), ctypes.byref(r), ctypes.byref(s)),
                      "df_tensor_shape")
        self.shape = (a.value, r.value, s.value)

    @classmethod
    def create(cls, handle, array):
        array = np.ascontiguousarray(array, dtype=np.float64)
        if array.ndim != 3:
            raise ValueError("a density-fitting object is a 3-index array (g, r, s)")
        p = ctypes.c_void_p()
        handle._check(load().df_tensor_create(handle.h, *array.shape, _dp(array), ctypes.byref(p)),
                      "df_tensor_create")
        return cls(handle, p)

    @classmethod
    def from_B(cls, handle):
        p = ctypes.c_void_p()
        handle._check(load().df_tensor_from_B(handle.h, ctypes.byref(p)), "df_tensor_from_B")
        return cls(handle, p)

    def get(self):
        out = np.empty(self.shape)
        self.handle._check(load().df_tensor_get(self.t, _dp(out)), "df_tensor_get")
        return out

    def transform(self, which, M):
        """Eq. (1): which "first" (M: nr x nt), "second" (M: ns x nt) or "aux" (M': naux' x naux)."""
        M = np.ascontiguousarray(M, dtype=np.float64)
        p = ctypes.c_void_p()
        w = {"first": 0, "second": 1, "aux": 2}[which]
        self.handle._check(load().df_op_transform(self.t, w, _dp(M), M.shape[0], M.shape[1], ctypes.byref(p)),
                           "df_op_transform")
        return DFTensor(self.handle, p)

    def contract(self, other, which):
        """Eq. (2): which "first" (ns x nt), "aux" ((nr ns) x (nt nu)) or "pairs" (naux x naux2)."""
        a, r, s = self.shape
        a2, r2, s2 = other.shape
        shape = {"first": (s, s2), "aux": (r * s, r2 * s2), "pairs": (a, a2)}[which]
        out = np.empty(shape)
        w = {"first": 0, "aux": 1, "pairs": 2}[which]
        self.handle._check(load().df_op_contract(self.t, other.t, w, _dp(out)), "df_op_contract")
        return out

    def density_fit(self, M):
        M = np.ascontiguousarray(M, dtype=np.float64)
        D = np.empty(self.shape[0])
        self.handle._check(load().df_op_density_fit(self.t, _dp(M), _dp(D)), "df_op_density_fit")
        return D

    def density_back(self, D):
        D = np.ascontiguousarray(D, dtype=np.float64)
        M = np.empty(self.shape[1:])
        self.handle._check(load().df_op_density_back(self.t, _dp(D), _dp(M)), "df_op_density_back")
        return M

    def apply_four_index(self, G, nt, nu):
        G = np.ascontiguousarray(G, dtype=np.float64)
        p = ctypes.c_void_p()
        self.handle._check(load().df_op_apply_four_index(self.t, _dp(G), int(nt), int(nu), ctypes.byref(p)),
                           "df_op_apply_four_index")
        return DFTensor(self.handle, p)

    def close(self):
        if getattr(self, "t", None):
            load().df_tensor_free(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The density-guess network (df_mlp_*): FP32 weights on the GPU, own training/inference kernels."""

    def __init__(self, nin, nhidden, nlayers, nout, seed=0):
        m = ctypes.c_void_p()
        rc = load().df_mlp_create(nin, nhidden, nlayers, nout, seed, ctypes.byref(m))
        if rc != DF_OK:
            raise DFError(rc, "df_mlp_create")
        self.m = m
        self.nin, self.nout = nin, nout
        self.nparams = load().df_mlp_nparams(m)

    def params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        load().df_mlp_params(self.m, _fp(out), 0)
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        rc = load().df_mlp_params(self.m, _fp(p), 1)
        if rc != DF_OK:
            raise DFError(rc, "df_mlp_params")

    def gradients(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.empty(self.nparams, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        rc = load().df_mlp_gradients(self.m, _fp(X), _fp(Y), X.shape[0], _fp(g), _fp(loss))
        if rc != DF_OK:
            raise DFError(rc, "df_mlp_gradients")
        return float(loss[0]), g

    def train(self, X, Y, epochs, batch, lr, seed=0):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        hist = np.zeros(epochs, dtype=np.float32)
        rc = load().df_mlp_train(self.m, _fp(X), _fp(Y), X.shape[0], epochs, batch, lr, seed, _fp(hist))
        if rc != DF_OK:
            raise DFError(rc, "df_mlp_train")
        return hist

    def predict(self, X, bf16=False):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.empty((X.shape[0], self.nout), dtype=np.float32)
        rc = load().df_mlp_predict(self.m, _fp(X), X.shape[0], int(bf16), _fp(Y))
        if rc != DF_OK:
            raise DFError(rc, "df_mlp_predict")
        return Y

    def close(self):
        if getattr(self, "m", None):
            load().df_mlp_free(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_bytes(system, precision=DF_PREC_FP64, slices=5) -> int:
    """Device memory one molecule needs for its B tensors (and split slices), for wave planning."""
    n, naux, nocc = system.nbf, system.naux, system.nocc
    nt = (n + 63) // 64
    npad = nt * 64
    row = nt * (nt + 1) // 2 * 64 * 64
    total = 2 * naux * row * 8 + 40 * n * n * 8
    if precision == DF_PREC_SPLIT:
        # B slices as packed lower 128-tiles (the tensor-core layout), Y and its slices
        ldy = (nocc + 31) // 32 * 32
        nb = (n + 127) // 128
        total += slices * naux * (nb * (nb + 1) // 2) * 128 * 128 * 2 + naux * npad * ldy * (8 + 2 * slices)
    return int(total)


def scf_waves(systems, budget_bytes, precision=DF_PREC_FP64, slices=3, on_done=None, **kw):
    """Solve many molecules in waves whose estimated device memory fits `budget_bytes`; each wave is
    one scf_run_batch. on_done(index, handle, result), if given, is called for every molecule before its
    handle is closed. Returns one result dict per system, in order."""
    results = [None] * len(systems)
    order = list(range(len(systems)))
    i = 0
    while i < len(order):
        wave, used = [], 0
        while i < len(order):
            need = estimate_bytes(systems[order[i]], precision, 5)
            if wave and used + need > budget_bytes:
                break
            wave.append(order[i])
            used += need
            i += 1
        handles = [Handle(systems[k]) for k in wave]
        try:
            res = scf_batch(handles, precision=precision, slices=slices, **kw)
            if on_done is not None:
                for k, hd, r in zip(wave, handles, res):
                    on_done(k, hd, r)
        finally:
            for h in handles:
                h.close()
        for k, r in zip(wave, res):
            results[k] = r
    return results


def rint_pow2(v, k):
    """rint(v 2^k), ties to even, by the library's splitting routine run on the host (test hook)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    k = np.ascontiguousarray(np.broadcast_to(k, v.shape), dtype=np.int32)
    out = np.empty(v.shape, dtype=np.int64)
    rc = load().df_rint_pow2(_dp(v), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), v.size,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    if rc != DF_OK:
        raise DFError(rc, "df_rint_pow2")
    return out


def rys(T, nroots):
    T = np.ascontiguousarray(T, dtype=np.float64)
    x = np.empty((len(T), nroots))
    w = np.empty((len(T), nroots))
    rc = load().df_rys(_dp(T), len(T), nroots, _dp(x), _dp(w))
    if rc != DF_OK:
        raise DFError(rc, "df_rys")
    return x, w


def fp64_rate(kind: int = 0, iters: int = 100000):
    """Measured FP64 rate (TFLOP/s) of the current device: kind 0 a DFMA loop, 1 an FP64 mma.sync loop.
    Returns (tflops, milliseconds of the timed launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    rc = load().df_fp64_rate(int(kind), int(iters), ctypes.byref(t), ctypes.byref(ms))
    if rc != DF_OK:
        raise DFError(rc, "df_fp64_rate")
    return t.value, ms.value
