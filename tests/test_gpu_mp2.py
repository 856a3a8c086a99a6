"""DF-MP2 on the GPU (df_mp2) against the oracle (oracle/dfmp2.py): the correlation energy of the same
canonical orbitals, at 2 waters from the oracle's own B and at 8 waters from the GPU's B (the MP2 step
alone), and at 2 waters end to end from the oracle's own SCF orbitals."""
import numpy as np
import pytest

from oracle import dfmp2, dfrhf
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def _orbitals(h, r):
    nmo = h.n - r["n_dropped"]
    C = h.matrix("C").reshape(-1)[: h.n * nmo].reshape(h.n, nmo)
    return C, h.matrix("eps")[:nmo]


def test_mp2_water2_against_oracle(lib):
    system = clusters.workload("water2")
    B = dfrhf.whiten(dfrhf.three_center(system), dfrhf.metric(system))
    with lib.Handle(system) as h:
        r = h.scf(conv_E=1e-12, conv_err=1e-9)
        C, eps = _orbitals(h, r)
        e2 = h.mp2(C, eps)
        e2_default = h.mp2(n_dropped=r["n_dropped"])
        with pytest.raises(lib.DFError):
            h.mp2(C, eps, nocc=C.shape[1])             # no virtual orbital
    ref_same = dfmp2.mp2_energy(B, C, eps, system.nocc)
    ro = dfrhf.scf(system, B=B, conv_E=1e-12, conv_err=1e-9)
    ref_own = dfmp2.mp2_energy(B, ro.C, ro.eps, system.nocc)
    print(f"water2 E2: GPU {e2:.12f}, oracle on the GPU orbitals {ref_same:.12f}, oracle end to end {ref_own:.12f}")
    assert e2 < 0 and e2 == e2_default
    assert abs(e2 - ref_same) <= 1e-11 * abs(ref_same)
    assert abs(e2 - ref_own) <= 1e-8


def test_mp2_water8_against_oracle_on_gpu_B(lib):
    system = clusters.workload("water8")
    with lib.Handle(system) as h:
        r = h.scf()
        C, eps = _orbitals(h, r)
        e2 = h.mp2(C, eps)
        B = h.rows(1, 0, h.naux)
    ref = dfmp2.mp2_energy(B, C, eps, system.nocc)
    print(f"water8 E2: GPU {e2:.12f}, oracle {ref:.12f}")
    assert e2 < 0 and abs(e2 - ref) <= 1e-11 * abs(ref)
