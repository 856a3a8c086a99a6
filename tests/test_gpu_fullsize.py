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
