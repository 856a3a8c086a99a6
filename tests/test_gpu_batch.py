"""Batched SCF (scf_run_batch): molecules of uneven size solved together on one GPU give the same
energies as separate runs (FP64: same arithmetic; split precision: within 1e-6 Eh of FP64)."""
import numpy as np
import pytest

from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def _systems():
    rng = clusters.SplitMix64(77)
    return [clusters.water_cluster(1 + int(rng.uniform() * 4), 1000 + k) for k in range(6)]


def test_batch_fp64_equals_single_runs(lib):
    systems = _systems()
    singles = []
    for s in systems:
        with lib.Handle(s) as h:
            singles.append(h.scf()["energy"])
    handles = [lib.Handle(s) for s in systems]
    try:
        res = lib.scf_batch(handles)
    finally:
        for h in handles:
            h.close()
    for r, e in zip(res, singles):
        assert r["converged"]
        assert abs(r["energy"] - e) <= 1e-10, (r["energy"], e)


def test_batch_split_matches_fp64(lib):
    systems = _systems()[:4]
    handles = [lib.Handle(s) for s in systems]
    try:
        e64 = [r["energy"] for r in lib.scf_batch(handles)]
        es = lib.scf_batch(handles, precision=lib.DF_PREC_SPLIT, slices=3)
    finally:
        for h in handles:
            h.close()
    for r, e in zip(es, e64):
        assert r["converged"]
        assert abs(r["energy"] - e) <= 1e-6, (r["energy"], e)


def test_batch_rejects_duplicate_handles(lib):
    s = clusters.workload("water2")
    with lib.Handle(s) as h:
        with pytest.raises(lib.DFError) as e:
            lib.scf_batch([h, h])
        assert e.value.code == lib.DF_E_ARG


@pytest.mark.parametrize("whitening", [0, 1])
def test_grouped_integrals_equal_single_builds(lib, whitening):
    """df_build_B_batch (one persistent launch per class over all molecules' work items) gives the integrals,
    and B, of each molecule's own df_build_B_ex to rounding: both kernels run the same per-triple code, which
    the compiler may contract into fused multiply-adds differently in the two kernels; molecules of uneven
    size."""
    systems = [clusters.water_cluster(w, 500 + w) for w in (3, 1, 5, 2)]
    ref3, refB = [], []
    for s in systems:
        with lib.Handle(s) as h:
            h.build_B(keep_3c=True, whitening=whitening)
            ref3.append(h.rows(0, 0, h.naux))
            refB.append(h.rows(1, 0, h.naux))
    handles = [lib.Handle(s) for s in systems]
    try:
        lib.build_B_batch(handles, keep_3c=True, whitening=whitening)
        for h, a, b in zip(handles, ref3, refB):
            assert np.abs(h.rows(0, 0, h.naux) - a).max() <= 1e-14 * np.abs(a).max()
            # the whitening amplifies last-bit differences of the integrals (the tensor-core form can also move
            # a digit of its slices): held to the whitening's own error level
            assert np.abs(h.rows(1, 0, h.naux) - b).max() <= 1e-9 * np.abs(b).max()
    finally:
        for h in handles:
            h.close()
