"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances: integrals, metric and B to 1e-11 absolute ((P|mu nu) bar of the FP64 path); J and K to
1e-11 relative to their largest element; SCF energy to 1e-9 Eh.
"""
import numpy as np
import pytest

from oracle import dfrhf
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu

TOL_INT = 1e-11
TOL_E = 1e-9


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def water2():
    return clusters.workload("water2")


@pytest.fixture(scope="module")
def water2_oracle(water2):
    S = dfrhf.overlap(water2)
    T = dfrhf.kinetic(water2)
    V = dfrhf.nuclear(water2)
    M = dfrhf.metric(water2)
    A = dfrhf.three_center(water2)
    B = dfrhf.whiten(A, M)
    return dict(S=S, T=T, V=V, M=M, A=A, B=B)


@pytest.fixture(scope="module")
def water2_gpu(lib, water2):
    h = lib.Handle(water2)
    h.build_B(keep_3c=True)
    yield h
    h.close()


def test_rys_rule_reproduces_boys_moments(lib):
    T = np.concatenate([[0.0, 1e-9, 1e-3], np.linspace(0.01, 59.99, 97), [60.0, 75.0, 300.0, 5e4]])
    for n in range(1, 5):
        x, w = lib.rys(T, n)
        for t, xr, wr in zip(T, x, w):
            F = dfrhf.boys(2 * n - 1, t)
            for k in range(2 * n):
                q = np.sum(wr * xr ** k)
                assert abs(q - F[k]) <= 2e-13 * F[k], (n, t, k, q, F[k])


def test_one_electron_matrices(water2_gpu, water2_oracle):
    for name, key in (("S", "S"), ("T", "T"), ("V", "V")):
        d = np.abs(water2_gpu.matrix(name) - water2_oracle[key]).max()
        assert d <= TOL_INT, (name, d)


def test_metric(water2_gpu, water2_oracle):
    d = np.abs(water2_gpu.matrix("metric") - water2_oracle["M"]).max()
    assert d <= TOL_INT, d


def test_three_center_all_rows(water2_gpu, water2_oracle):
    A = water2_gpu.rows(0, 0, water2_gpu.naux)
    d = np.abs(A - water2_oracle["A"]).max()
    assert d <= TOL_INT, d


def _whitening_tol(M):
    """Relative tolerance between two correct FP64 whitenings: the oracle solves L B = A by
    substitution, the GPU multiplies by an explicitly inverted L; the two differ by a small multiple
    of eps * kappa(L) |B| with kappa(L) = sqrt(kappa(M)) (the factor covers the summation-order growth
    over naux terms)."""
    ev = np.linalg.eigvalsh(M)
    return max(TOL_INT, 300 * np.finfo(float).eps * np.sqrt(ev[-1] / ev[0]))


def test_whitened_B(water2_gpu, water2_oracle):
    B = water2_gpu.rows(1, 0, water2_gpu.naux)
    scale = max(1.0, np.abs(water2_oracle["B"]).max())
    d = np.abs(B - water2_oracle["B"]).max()
    assert d <= _whitening_tol(water2_oracle["M"]) * scale, d
    # whitening preserves the Coulomb metric of the fit: B^T B = A^T V^-1 A (pairwise products)
    Bf, Af = B.reshape(B.shape[0], -1)[:, :400], water2_oracle["A"].reshape(B.shape[0], -1)[:, :400]
    G_gpu = Bf.T @ Bf
    G_ref = Af.T @ np.linalg.solve(water2_oracle["M"], Af)
    assert np.abs(G_gpu - G_ref).max() <= _whitening_tol(water2_oracle["M"]) * np.abs(G_ref).max()


@pytest.mark.parametrize("seed", [3, 4])
def test_random_shells_every_class(lib, seed):
    """Random exponents (0.05-500), random centres, every (lP, la, lb) class, several 64-wide tiles
    and a ragged tail."""
    rng = clusters.SplitMix64(seed)
    basis = clusters.random_shells(rng, 60, 2, box=3.0, natom=2)
    aux = clusters.random_shells(rng, 24, 3, box=3.0, natom=2)
    # make sure every class appears at least once
    basis["l"][:3] = [0, 1, 2]
    aux["l"][:4] = [0, 1, 2, 3]
    atoms = np.zeros(2, dtype=clusters.ATOM_DTYPE)
    atoms["xyz"] = [[0.1, 0.2, -0.3], [1.0, -0.7, 0.5]]
    atoms["Z"] = [3, 3]
    system = clusters.System(atoms=atoms, basis=basis, aux=aux)
    assert system.nbf > 128 and system.nbf % 64 != 0
    ref3 = dfrhf.three_center(system)
    refS = dfrhf.overlap(system)
    refV = dfrhf.nuclear(system)
    refM = dfrhf.metric(system)
    with lib.Handle(system) as h:
        assert np.abs(h.matrix("S") - refS).max() <= TOL_INT
        assert np.abs(h.matrix("V") - refV).max() <= TOL_INT * max(1, np.abs(refV).max())
        assert np.abs(h.matrix("metric") - refM).max() <= TOL_INT * max(1, np.abs(refM).max())
        h.build_B(keep_3c=True)
        A = h.rows(0, 0, h.naux)
    scale = max(1.0, np.abs(ref3).max())
    d = np.abs(A - ref3).max()
    assert d <= TOL_INT * scale, (d, scale)


def test_jk_kernels_exact(water2_gpu, water2):
    """J and K kernels against the oracle's eq. (1)-(3) contractions applied to the same B."""
    rng = np.random.default_rng(7)
    n, nocc = water2.nbf, water2.nocc
    C = rng.normal(size=(n, nocc)) * 0.3
    D = 2 * C @ C.T
    J, K = water2_gpu.jk(D, C)
    B = water2_gpu.rows(1, 0, water2_gpu.naux)
    Jr = dfrhf.df_J(B, D)
    Kr = dfrhf.df_K(B, C)
    assert np.abs(J - Jr).max() <= 1e-12 * np.abs(Jr).max()
    assert np.abs(K - Kr).max() <= 1e-12 * np.abs(Kr).max()
    assert np.abs(K - K.T).max() == 0.0
    assert np.abs(J - J.T).max() <= 1e-13 * np.abs(J).max()


def test_jk_against_oracle_end_to_end(water2_gpu, water2_oracle, water2):
    rng = np.random.default_rng(8)
    n, nocc = water2.nbf, water2.nocc
    C = np.linalg.qr(rng.normal(size=(n, nocc)))[0]
    D = 2 * C @ C.T
    J, K = water2_gpu.jk(D, C)
    Jr = dfrhf.df_J(water2_oracle["B"], D)
    Kr = dfrhf.df_K(water2_oracle["B"], C)
    tol = _whitening_tol(water2_oracle["M"])
    assert np.abs(J - Jr).max() <= tol * np.abs(Jr).max()
    assert np.abs(K - Kr).max() <= tol * np.abs(Kr).max()


def test_scf_energy_matches_oracle(lib, water2):
    ref = dfrhf.scf(water2)
    with lib.Handle(water2) as h:
        res = h.scf()
        D = h.matrix("D")
        S = h.matrix("S")
    assert res["converged"]
    assert abs(res["energy"] - ref.energy) <= TOL_E, (res["energy"], ref.energy)
    assert abs(np.trace(D @ S) - water2.n_electrons) < 1e-9
    assert np.abs(D - ref.D).max() < 1e-6


def test_invalid_inputs_rejected(lib, water2):
    import copy
    bad = copy.deepcopy(water2)
    bad.basis = bad.basis.copy()
    bad.basis["exponent"][0] = -1.0
    with pytest.raises(lib.DFError) as e:
        lib.Handle(bad)
    assert e.value.code == lib.DF_E_ARG
    bad2 = copy.deepcopy(water2)
    bad2.aux = bad2.aux.copy()
    bad2.aux["l"][0] = 4
    with pytest.raises(lib.DFError):
        lib.Handle(bad2)
    odd = copy.deepcopy(water2)
    odd.charge = 1
    with pytest.raises(lib.DFError):
        lib.Handle(odd)
    with lib.Handle(water2) as h:
        with pytest.raises(lib.DFError) as e:
            h.jk(np.eye(h.n), np.zeros((h.n, h.nocc)))
        assert e.value.code == lib.DF_E_STATE
