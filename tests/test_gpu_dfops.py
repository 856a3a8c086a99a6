"""The density-fitting object operations of eqs. (1)-(3) on the GPU (df_tensor_*, df_op_*) against
oracle/dfops.py, element by element on ragged random tensors (no dimension a multiple of the 64-wide GEMM
tiles), and on the 2-water B: J and K composed from the operations against the oracle's DF J and K."""
import numpy as np
import pytest

from oracle import dfops, dfrhf
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def _close(a, b):
    scale = max(1.0, float(np.abs(b).max()))
    return float(np.abs(a - b).max()) <= 1e-12 * scale


def test_operations_against_oracle(lib):
    r = np.random.default_rng(41)
    g, nr, ns, nt, nu = 37, 23, 19, 11, 7
    I = r.normal(size=(g, nr, ns))
    I2 = r.normal(size=(g, nr, nt))
    I3 = r.normal(size=(g, nt, nu))
    I4 = r.normal(size=(13, nr, ns))
    Mr, Ms, Mp = r.normal(size=(nr, nt)), r.normal(size=(ns, nt)), r.normal(size=(29, g))
    Mrs, D, G = r.normal(size=(nr, ns)), r.normal(size=g), r.normal(size=(nr * ns, nt * nu))
    with lib.Handle(clusters.workload("water2")) as h:
        t, t2, t3, t4 = (lib.DFTensor.create(h, x) for x in (I, I2, I3, I4))
        assert t.shape == (g, nr, ns) and np.array_equal(t.get(), I)
        assert _close(t.transform("first", Mr).get(), dfops.transform_first(I, Mr))
        assert _close(t.transform("second", Ms).get(), dfops.transform_second(I, Ms))
        assert _close(t.transform("aux", Mp).get(), dfops.transform_aux(I, Mp))
        assert _close(t.contract(t2, "first"), dfops.contract_first(I, I2))
        assert _close(t.contract(t3, "aux"), dfops.contract_aux(I, I3))
        assert _close(t.contract(t4, "pairs"), dfops.contract_pairs(I, I4))
        assert _close(t.density_fit(Mrs), dfops.density_fit(I, Mrs))
        assert _close(t.density_back(D), dfops.density_back(I, D))
        assert _close(t.apply_four_index(G, nt, nu).get(), dfops.apply_four_index(I, G, nt, nu))
        with pytest.raises(lib.DFError) as e:
            t.transform("first", Ms)                    # M must have nr rows
        assert e.value.code == lib.DF_E_ARG
        with pytest.raises(lib.DFError):
            t.contract(t3, "first")                     # first indices differ in length


def test_coulomb_and_exchange_from_operations(lib):
    """On the 2-water B (df_tensor_from_B): J = density_back(density_fit(D)) and K = contract_first(Y, Y)
    with Y = transform_first(B, C_occ), against the oracle's DF J and K on the same B."""
    system = clusters.workload("water2")
    rng = np.random.default_rng(42)
    with lib.Handle(system) as h:
        h.build_B(whitening=lib.DF_WHITEN_FP64)
        C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
        D = 2 * C @ C.T
        B = h.rows(1, 0, h.naux)
        tb = lib.DFTensor.from_B(h)
        assert np.array_equal(tb.get(), B)
        J = tb.density_back(tb.density_fit(D))
        Y = tb.transform("first", C)
        K = Y.contract(Y, "first")
        Jh, Kh = h.jk(D, C)
    assert _close(J, dfrhf.df_J(B, D)) and _close(K, dfrhf.df_K(B, C))
    assert np.abs(J - Jh).max() <= 1e-12 * np.abs(Jh).max() and np.abs(K - Kh).max() <= 1e-12 * np.abs(Kh).max()
