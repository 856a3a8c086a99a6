"""GPU parity on the 8-water cluster (n=400, naux=1096, nocc=40) against the CPU oracle, element by element.

* B from both whitenings (the default 7-slice tensor-core product and the FP64 product) against the oracle's
  B = L^-1 (Q|mu nu) (eq. 1, third form), every row. Both GPU whitenings multiply by an explicitly inverted
  Cholesky factor; the oracle substitutes (scipy's triangular solve). The forward error of a product with a
  computed triangular inverse is bounded by a multiple of n eps kappa(L) |B| (Higham, Accuracy and Stability
  of Numerical Algorithms, ch. 14), so two correct FP64 whitenings of this metric (condition number 5.5e11,
  kappa(L) = 7.4e5) may differ by up to naux eps kappa(L) = 1.8e-7 of max|B|; measured: 6.6e-8, and the
  two GPU whitenings agree with each other to 3e-10.
* J and K (eqs. 1-3) against the oracle's contractions applied to the GPU's own B: the FP64 kernels to
  1e-12 relative; the split exchange at S slices to its splitting bound 2^(7 - 7S) relative to max|K|
  (each operand is cut into S digits of 7 bits, the pairs beyond S are dropped).
* J and K of the default path against the oracle's J and K on the oracle's B (whole path, the whitening
  bar).
"""
import numpy as np
import pytest

from oracle import dfrhf
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def w8():
    return clusters.workload("water8")


@pytest.fixture(scope="module")
def oracle8(w8):
    M = dfrhf.metric(w8)
    B = dfrhf.whiten(dfrhf.three_center(w8), M)
    ev = np.linalg.eigvalsh(M)
    tol = len(M) * np.finfo(float).eps * np.sqrt(ev[-1] / ev[0])
    return {"M": M, "B": B, "tol": tol}


@pytest.fixture(scope="module")
def density(w8):
    rng = np.random.default_rng(88)
    C = np.linalg.qr(rng.normal(size=(w8.nbf, w8.nocc)))[0]
    return C, 2 * C @ C.T


@pytest.fixture(scope="module")
def gpu8(lib, w8):
    """Two handles on the same cluster: B whitened on the tensor cores (default) and in FP64."""
    tc = lib.Handle(w8)
    tc.build_B()
    fp = lib.Handle(w8)
    fp.build_B(whitening=lib.DF_WHITEN_FP64)
    yield tc, fp
    tc.close()
    fp.close()


def test_whitened_B_both_whitenings_match_oracle(gpu8, oracle8):
    tc, fp = gpu8
    Bref = oracle8["B"]
    scale = np.abs(Bref).max()
    B_tc = tc.rows(1, 0, tc.naux)
    B_fp = fp.rows(1, 0, fp.naux)
    d_tc = np.abs(B_tc - Bref).max()
    d_fp = np.abs(B_fp - Bref).max()
    d_tf = np.abs(B_tc - B_fp).max()
    print(f"max|B| {scale:.3e}; tensor-core vs oracle {d_tc / scale:.2e}, FP64 vs oracle {d_fp / scale:.2e}, "
          f"tensor-core vs FP64 {d_tf / scale:.2e} (bar {oracle8['tol']:.2e})")
    assert d_tc <= oracle8["tol"] * scale
    assert d_fp <= oracle8["tol"] * scale
    # the 7-slice product against the FP64 product of the same L^-1 and integrals: an exact CPU emulation
    # of the splitting gives 2.8e-10 of max|B| on this cluster
    assert d_tf <= 2e-9 * scale


def test_jk_on_gpu_B_match_oracle_contractions(lib, gpu8, density):
    """FP64 J and K and split K at 3 and 5 slices, against eqs. (1)-(3) applied to the same B."""
    _, fp = gpu8
    C, D = density
    B = fp.rows(1, 0, fp.naux)
    Jr = dfrhf.df_J(B, D)
    Kr = dfrhf.df_K(B, C)
    del B
    J, K = fp.jk(D, C)
    assert np.abs(J - Jr).max() <= 1e-12 * np.abs(Jr).max()
    assert np.abs(K - Kr).max() <= 1e-12 * np.abs(Kr).max()
    kmax = np.abs(Kr).max()
    for S in (3, 5):
        Js, Ks = fp.jk(D, C, lib.DF_PREC_SPLIT, S)
        rel = np.abs(Ks - Kr).max() / kmax
        print(f"split S={S}: max|dK|/max|K| {rel:.2e} (bound {2.0 ** (7 - 7 * S):.2e})")
        assert rel <= 2.0 ** (7 - 7 * S)
        assert np.abs(Js - Jr).max() <= 1e-12 * np.abs(Jr).max()   # J stays FP64 in split mode
        assert np.abs(Ks - Ks.T).max() == 0.0


def test_jk_default_path_against_oracle_B(gpu8, oracle8, density):
    tc, _ = gpu8
    C, D = density
    J, K = tc.jk(D, C)
    Jr = dfrhf.df_J(oracle8["B"], D)
    Kr = dfrhf.df_K(oracle8["B"], C)
    dJ = np.abs(J - Jr).max() / np.abs(Jr).max()
    dK = np.abs(K - Kr).max() / np.abs(Kr).max()
    print(f"default path vs oracle: J {dJ:.2e}, K {dK:.2e} relative (bar {oracle8['tol']:.2e})")
    assert dJ <= oracle8["tol"] and dK <= oracle8["tol"]
