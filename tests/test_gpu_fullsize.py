"""Parity at the benchmark's full size (32-water cluster, n=1600, naux=4384, nocc=160) in the launch
configuration bench.py times: sampled three-centre integrals against the oracle one block at a
time, and properties that hold at any size for J and K."""
import numpy as np
import pytest

from oracle import dfrhf
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    system = clusters.workload("water32")
    h = binding.Handle(system)
    h.build_B(keep_3c=True)
    yield binding, system, h
    h.close()


def test_sampled_three_center_blocks(big):
    binding, system, h = big
    rng = np.random.default_rng(32)
    aux_off = np.concatenate([[0], np.cumsum(2 * system.aux["l"] + 1)])
    bas_off = np.concatenate([[0], np.cumsum(2 * system.basis["l"] + 1)])
    # every angular-momentum class at least once, plus random triples
    triples = []
    for lp in range(4):
        for la in range(3):
            for lb in range(3):
                P = rng.choice(np.flatnonzero(system.aux["l"] == lp))
                M = rng.choice(np.flatnonzero(system.basis["l"] == la))
                N = rng.choice(np.flatnonzero(system.basis["l"] == lb))
                triples.append((P, M, N))
    for _ in range(60):
        triples.append((rng.integers(len(system.aux)), rng.integers(len(system.basis)), rng.integers(len(system.basis))))
    ref = dfrhf.three_center_triples(system, triples)
    worst = 0.0
    for (P, M, N), blk in zip(triples, ref):
        np_ = blk.shape[0]
        rows = h.rows(0, int(aux_off[P]), np_)
        got = rows[:, bas_off[M]:bas_off[M] + blk.shape[1], bas_off[N]:bas_off[N] + blk.shape[2]]
        worst = max(worst, np.abs(got - blk).max())
    assert worst <= 1e-11, worst


def test_full_size_jk_properties(big):
    binding, system, h = big
    rng = np.random.default_rng(33)
    C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
    D = 2 * C @ C.T
    J, K = h.jk(D, C)
    assert np.abs(J - J.T).max() <= 1e-13 * np.abs(J).max()
    assert np.abs(K - K.T).max() == 0.0
    # Coulomb energy 1/2 tr(DJ) = 1/2 |gamma|^2 >= 0; exchange tr(DK) = 2 sum_P |C^T B_P C|^2 >= 0
    assert np.sum(D * J) > 0 and np.sum(D * K) > 0
    # exchange is invariant under a rotation of the occupied orbitals
    Q = np.linalg.qr(rng.normal(size=(h.nocc, h.nocc)))[0]
    _, K2 = h.jk(D, C @ Q)
    assert np.abs(K2 - K).max() <= 1e-11 * np.abs(K).max()
    # split-precision K agrees with the FP64 K
    _, Ks = h.jk(D, C, binding.DF_PREC_SPLIT, 3)
    assert np.abs(Ks - K).max() <= 2e-5 * np.abs(K).max()


def test_full_size_jk_sampled_against_oracle(big):
    """J and K at full size against the oracle's eqs. (1)-(3) applied to the GPU's own B, which is streamed
    to the host in blocks of auxiliary rows: J in full (eq. 3 is a sum over rows), and K on a sampled index
    set I (K_II = sum_{P,i} Y_P,Ii Y_P,Ii^T needs only the rows I of every B_P: eq. 2 applied to B[:, I, :]).
    I spans the first and last functions, tile edges and the ragged tail. The split exchange runs at 5
    slices in the tile configuration of the benchmark (the widths the autotuner picks give bitwise the same
    K; the split over auxiliary blocks is the occupancy heuristic the benchmark uses)."""
    binding, system, h = big
    rng = np.random.default_rng(34)
    n = h.n
    C = np.linalg.qr(rng.normal(size=(n, h.nocc)))[0]
    D = 2 * C @ C.T
    J64, K64 = h.jk(D, C)
    _, K5 = h.jk(D, C, binding.DF_PREC_SPLIT, 5)
    t = h.timings()
    print(f"split tiles: Y {t['tc_y_tile_n']:.0f}, K {t['tc_k_tile_n']:.0f}, K split {t['tc_k_split']:.0f}")
    idx = sorted({0, 1, 63, 64, 127, 128, 511, 512, n // 2, n - 65, n - 64, n - 2, n - 1}
                 | set(rng.choice(n, 19, replace=False).tolist()))
    Jr = np.zeros((n, n))
    Kr = np.zeros((len(idx), len(idx)))
    step = 48
    for p0 in range(0, h.naux, step):
        Bb = h.rows(1, p0, min(step, h.naux - p0))
        Jr += dfrhf.df_J(Bb, D)
        Kr += dfrhf.df_K(np.ascontiguousarray(Bb[:, idx, :]), C)
    kmax = np.abs(Kr).max()
    dJ = np.abs(J64 - Jr).max() / np.abs(Jr).max()
    dK64 = np.abs(K64[np.ix_(idx, idx)] - Kr).max() / kmax
    dK5 = np.abs(K5[np.ix_(idx, idx)] - Kr).max() / kmax
    print(f"32 waters vs oracle: J {dJ:.2e}, K FP64 {dK64:.2e}, K split S=5 {dK5:.2e} (relative to max)")
    assert dJ <= 1e-11
    assert dK64 <= 1e-11
    assert dK5 <= 2.0 ** (7 - 7 * 5)
