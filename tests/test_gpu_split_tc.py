"""The tcgen05 (TMEM + TMA) split-precision kernels against the mma.sync split kernels and the FP64
path on the same B and C. B's slices are full rows with one exponent per (P, mu) where they fit in HBM
(every size here) and packed lower 128 x 128 tiles with one exponent per auxiliary row otherwise (the
tiles above the diagonal read transposed; forced with DFHF_TC_PACKED=1); C is cut the same way. They re-slice Y with exponents over different
blocks of the (P, i) contraction (the tensor-core contraction over chunks of the contiguous index
P ldy + i, the mma.sync one over whole auxiliary rows), so their K differ by the splitting error: each is
held to the bound 2^(7 - 7S) against FP64, and the two to twice it."""
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


def _k(h, lib, D, C, slices, tc):
    old = os.environ.get("DFHF_SPLIT_TC")
    os.environ["DFHF_SPLIT_TC"] = "1" if tc else "0"
    try:
        return h.jk(D, C, lib.DF_PREC_SPLIT, slices)[1]
    finally:
        if old is None:
            del os.environ["DFHF_SPLIT_TC"]
        else:
            os.environ["DFHF_SPLIT_TC"] = old


@pytest.mark.parametrize("name", ["water2", "water8"])
@pytest.mark.parametrize("slices", [3, 5])
def test_tensor_core_split_matches_mma_sync_and_fp64(lib, name, slices):
    system = clusters.workload(name)
    rng = np.random.default_rng(12)
    with lib.Handle(system) as h:
        h.build_B()
        C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
        D = 2 * C @ C.T
        K64 = h.jk(D, C, lib.DF_PREC_FP64)[1]
        Kms = _k(h, lib, D, C, slices, tc=False)
        Ktc = _k(h, lib, D, C, slices, tc=True)
        Ktc2 = _k(h, lib, D, C, slices, tc=True)
    scale = np.abs(K64).max()
    bound = 2.0 ** (7 - 7 * slices)
    print(f"{name} S={slices}: tcgen05 {np.abs(Ktc - K64).max() / scale:.2e}, mma.sync "
          f"{np.abs(Kms - K64).max() / scale:.2e} relative to FP64")
    assert np.array_equal(Ktc, Ktc2)
    assert np.abs(Ktc - K64).max() <= bound * scale
    assert np.abs(Kms - K64).max() <= bound * scale
    assert np.abs(Ktc - Kms).max() <= 2 * bound * scale


def test_autotuner_choice_is_valid_and_cached(lib):
    """The autotuner picks a Y tile width dividing the occupied width and a K split of at least one
    auxiliary block; a second molecule of the same size bucket reuses the choice without tuning."""
    system = clusters.workload("water8")
    rng = np.random.default_rng(4)
    with lib.Handle(system) as h:
        h.build_B()
        C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
        D = 2 * C @ C.T
        K1 = _k(h, lib, D, C, 5, tc=True)
        t1 = h.timings()
    ldy = (system.nocc + 31) // 32 * 32
    assert t1["tc_y_tile_n"] in (32, 64, 80) and ldy % int(t1["tc_y_tile_n"]) == 0
    assert t1["tc_k_split"] >= 1
    assert t1["autotune_ms"] > 0
    with lib.Handle(system) as h:
        h.build_B()
        K2 = _k(h, lib, D, C, 5, tc=True)
        t2 = h.timings()
    assert t2["autotune_ms"] == t1["autotune_ms"]          # no new tuning for the same bucket
    assert (t2["tc_y_tile_n"], t2["tc_k_split"]) == (t1["tc_y_tile_n"], t1["tc_k_split"])
    assert np.array_equal(K1, K2)


@pytest.mark.parametrize("slices", [3, 5])
def test_tile_widths_give_identical_exchange(lib, slices):
    """Every tile width and split of the tensor-core kernels performs the same per-element arithmetic
    (same exact chunk sums, same drain order), so K is bitwise identical across tilings."""
    system = clusters.workload("water8")
    rng = np.random.default_rng(6)
    out = {}
    with lib.Handle(system) as h:
        h.build_B()
        C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
        D = 2 * C @ C.T
        for tiles in ("32,64,4", "64,32,4", "32,32,4"):
            os.environ["DFHF_TC_TILES"] = tiles
            try:
                out[tiles] = _k(h, lib, D, C, slices, tc=True)
            finally:
                del os.environ["DFHF_TC_TILES"]
    ref = out["32,64,4"]
    for k, v in out.items():
        assert np.array_equal(v, ref), k


@pytest.mark.parametrize("packed", ["0", "1"])
@pytest.mark.parametrize("rows", ["100", "1"])
def test_blocked_slices_match_resident_slices(lib, rows, packed):
    """When B's slices do not fit in HBM they are cut per block of auxiliary rows at every build; at 5
    slices the digits are the same as with every row resident, so K is bitwise identical. Blocks of 100
    rows (ragged last block: 1096 = 10 * 100 + 96) and of 1 row; the second build reuses the buffer; full
    rows and packed tiles (whose zero padding must survive the ragged last block)."""
    system = clusters.workload("water8")
    rng = np.random.default_rng(8)
    os.environ["DFHF_TC_PACKED"] = packed
    try:
        with lib.Handle(system) as h:
            h.build_B()
            C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
            D = 2 * C @ C.T
            K64 = h.jk(D, C, lib.DF_PREC_FP64)[1]
            resident = _k(h, lib, D, C, 5, tc=True)
        with lib.Handle(system) as h:
            h.build_B()
            os.environ["DFHF_SPLIT_BLOCK_ROWS"] = rows
            try:
                blocked5 = _k(h, lib, D, C, 5, tc=True)
                blocked3 = _k(h, lib, D, C, 3, tc=True)
                again5 = _k(h, lib, D, C, 5, tc=True)
            finally:
                del os.environ["DFHF_SPLIT_BLOCK_ROWS"]
    finally:
        del os.environ["DFHF_TC_PACKED"]
    assert np.array_equal(blocked5, resident)
    assert np.array_equal(again5, resident)
    scale = np.abs(K64).max()
    assert np.abs(blocked3 - K64).max() <= 2.0 ** (7 - 21) * scale


@pytest.mark.parametrize("name", ["water2", "water8"])
def test_packed_and_full_slice_layouts(lib, name):
    """B's slices as packed lower 128-tiles (one exponent per auxiliary row; tiles above the diagonal read as
    MN-major operands; at 8 waters np = 448 leaves a zero-padded half tile) against full rows (one exponent
    per (P, mu)): both within the splitting bound 2^(7 - 7S) of FP64, within twice it of each other, and
    the packed path bitwise reproducible."""
    system = clusters.workload(name)
    rng = np.random.default_rng(21)
    out = {}
    with lib.Handle(system) as h:
        h.build_B()
        C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
        D = 2 * C @ C.T
        K64 = h.jk(D, C, lib.DF_PREC_FP64)[1]
        for packed in ("1", "0", "1"):
            os.environ["DFHF_TC_PACKED"] = packed
            try:
                out.setdefault(packed, []).append({S: _k(h, lib, D, C, S, tc=True) for S in (3, 5)})
            finally:
                del os.environ["DFHF_TC_PACKED"]
    scale = np.abs(K64).max()
    for S in (3, 5):
        bound = 2.0 ** (7 - 7 * S)
        kp, kf = out["1"][0][S], out["0"][0][S]
        print(f"{name} S={S}: packed {np.abs(kp - K64).max() / scale:.2e}, full rows {np.abs(kf - K64).max() / scale:.2e}")
        assert np.abs(kp - K64).max() <= bound * scale
        assert np.abs(kf - K64).max() <= bound * scale
        assert np.abs(kp - kf).max() <= 2 * bound * scale
        assert np.array_equal(kp, out["1"][1][S])
        assert np.abs(kp - kp.T).max() == 0.0
