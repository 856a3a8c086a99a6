"""Metric whitening B = L^-1 (Q|mu nu) (eq. 1, third form) on the tensor cores (7 Ozaki slices) against
the float-float FP32-pipe whitening on the same integrals, and the SCF energies each gives."""
import os

import numpy as np
import pytest

from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def _build(lib, system, mode, keep):
    old = os.environ.pop("DFHF_WHITEN", None)
    if mode:
        os.environ["DFHF_WHITEN"] = mode
    try:
        h = lib.Handle(system)
        h.build_B(keep_3c=keep)
    finally:
        os.environ.pop("DFHF_WHITEN", None)
        if old is not None:
            os.environ["DFHF_WHITEN"] = old
    return h


@pytest.fixture(scope="module")
def water8_pair(lib):
    system = clusters.workload("water8")
    tc = _build(lib, system, None, keep=False)       # in place over the unwhitened tensor
    ff = _build(lib, system, "ff", keep=True)
    yield system, tc, ff
    tc.close()
    ff.close()


def test_tensor_core_whitening_matches_float_float(water8_pair):
    system, tc, ff = water8_pair
    rng = np.random.default_rng(3)
    rows = sorted(set(rng.integers(0, system.naux, 24).tolist()) | {0, system.naux - 1})
    scale = 0.0
    worst = 0.0
    for p in rows:
        a, b = tc.rows(1, p, 1)[0], ff.rows(1, p, 1)[0]
        scale = max(scale, np.abs(b).max())
        worst = max(worst, np.abs(a - b).max())
    print(f"max|dB| {worst:.3e}, max|B| {scale:.3e}, rel {worst / scale:.3e}")
    # 7 slices: the splitting error is ~2^-49 of the row and column scales summed over naux terms; an
    # exact CPU emulation of the same splitting on this cluster gives 2.8e-10 of max|B|
    assert worst <= 2e-9 * scale


def test_tensor_core_whitening_scf_energy(water8_pair):
    _, tc, ff = water8_pair
    e_tc, e_ff = tc.scf()["energy"], ff.scf()["energy"]
    print(f"E(tcgen05 whitening) {e_tc:.12f}  E(float-float) {e_ff:.12f}  dE {e_tc - e_ff:.3e}")
    assert abs(e_tc - e_ff) <= 1e-8


def test_keep_and_in_place_agree(lib):
    system = clusters.workload("water2")
    a = _build(lib, system, None, keep=True)
    b = _build(lib, system, None, keep=False)
    try:
        assert np.array_equal(a.rows(1, 0, 4), b.rows(1, 0, 4))
        assert np.array_equal(a.rows(1, system.naux - 3, 3), b.rows(1, system.naux - 3, 3))
    finally:
        a.close()
        b.close()


def test_whitening_tile_widths_identical(lib):
    """The 64- and 32-column whitening tiles do the same per-element arithmetic: bitwise equal B."""
    system = clusters.workload("water8")
    out = []
    for t in ("64", "32"):
        os.environ["DFHF_WHITEN_TILE"] = t
        try:
            h = _build(lib, system, None, keep=False)
            out.append(h.rows(1, 0, 3))
            out.append(h.rows(1, system.naux - 2, 2))
            h.close()
        finally:
            del os.environ["DFHF_WHITEN_TILE"]
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[3])


def test_blocked_triangular_inverse_matches_cusolver(lib):
    """The blocked recursive inverse of the metric's Cholesky factor (the default) agrees with cuSOLVER's
    trtri (DFHF_TRTRI=cusolver) and satisfies L^-1 (P|Q) L^-T = I to the metric's conditioning."""
    system = clusters.workload("water8")
    with lib.Handle(system) as h:
        h.build_B()
        L_blk = h.matrix("Linv")
        M = h.matrix("metric")
    os.environ["DFHF_TRTRI"] = "cusolver"
    try:
        with lib.Handle(system) as h:
            h.build_B()
            L_ref = h.matrix("Linv")
    finally:
        del os.environ["DFHF_TRTRI"]
    ev = np.linalg.eigvalsh(M)
    kappa_L = np.sqrt(ev[-1] / ev[0])
    tol = 100 * np.finfo(float).eps * kappa_L
    assert np.abs(np.triu(L_blk, 1)).max() == 0.0
    assert np.abs(L_blk - L_ref).max() <= tol * np.abs(L_ref).max()
    # L^-1 (P|Q) L^-T - I, formed in FP64, carries the metric's own conditioning kappa(L)^2 eps; the
    # blocked inverse's residual stays at that level and at the level of cuSOLVER's
    resid = np.abs(L_blk @ M @ L_blk.T - np.eye(len(M))).max()
    resid_ref = np.abs(L_ref @ M @ L_ref.T - np.eye(len(M))).max()
    print(f"kappa(L) {kappa_L:.2e}, max|L^-1 M L^-T - I| {resid:.2e} (cuSOLVER inverse {resid_ref:.2e})")
    assert resid <= max(10 * resid_ref, 100 * np.finfo(float).eps * kappa_L ** 2)
