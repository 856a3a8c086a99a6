"""Learned initial guess: network gradients against the FP64 oracle, BF16 inference, rotation of the
frame blocks, and an SCF started from the learned density reaching the same energy."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def test_mlp_gradients_match_oracle(lib):
    dims = [6, 16, 16, 16, 5]
    net = lib.Mlp(6, 16, 3, 5, seed=3)
    rs = np.random.default_rng(4)
    p = (rs.normal(size=net.nparams) * 0.4).astype(np.float32)
    net.set_params(p)
    X = rs.normal(size=(9, 6)).astype(np.float32)
    Y = rs.normal(size=(9, 5)).astype(np.float32)
    loss, g = net.gradients(X, Y)
    ref = omlp.gradient(p.astype(np.float64), dims, X.astype(np.float64), Y.astype(np.float64))
    ref_loss = omlp.loss(p.astype(np.float64), dims, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max()
    net.close()


def test_bf16_inference_close_to_fp32(lib):
    net = lib.Mlp(57, 64, 3, 40, seed=5)
    X = np.random.default_rng(6).normal(size=(11, 57)).astype(np.float32)
    y32 = net.predict(X, bf16=False)
    y16 = net.predict(X, bf16=True)
    assert np.abs(y16 - y32).max() <= 3e-2 * np.abs(y32).max()
    net.close()


def _rotate(system, R, t):
    atoms = system.atoms.copy()
    atoms["xyz"] = atoms["xyz"] @ R.T + t
    return clusters.make_system(atoms)


def test_frame_blocks_are_rotation_invariant(lib):
    s1 = clusters.workload("water2")
    q, r = np.linalg.qr(np.random.default_rng(8).normal(size=(3, 3)))
    R = q * np.sign(np.diag(r))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    s2 = _rotate(s1, R, np.array([0.3, -1.2, 2.0]))
    blocks = []
    for s in (s1, s2):
        with lib.Handle(s) as h:
            h.scf()
            D = h.matrix("D")
            b = h.water_blocks(D)
            blocks.append(b)
            # round trip: frame blocks back to the laboratory frame reproduce the diagonal blocks of D
            D0 = h.water_density(b)
            for w in range(len(s.atoms) // 3):
                sl = slice(50 * w, 50 * w + 50)
                assert np.abs(D0[sl, sl] - D[sl, sl]).max() <= 1e-5 * np.abs(D[sl, sl]).max()
    assert np.abs(blocks[0] - blocks[1]).max() <= 1e-6 * np.abs(blocks[0]).max()


def test_learned_guess_scf_same_energy_fewer_iterations(lib):
    train = [clusters.water_cluster(w, 10000 + k) for k, w in enumerate([2, 3, 4, 3, 2, 4])]
    X, Y = [], []
    for s in train:
        with lib.Handle(s) as h:
            h.scf()
            Y.append(h.water_blocks(h.matrix("D")))
        X.append(lib.water_features(s))
    X = np.concatenate(X)
    Y = np.concatenate(Y)
    net = lib.Mlp(lib.DF_MLP_NFEAT, 64, 3, Y.shape[1], seed=11)
    nout = Y.shape[1]
    p = net.params()
    p[-nout:] = Y.mean(axis=0)              # start from the mean block (superposed monomer density):
    p[-nout - nout * 64:-nout] = 0.0        # output bias = mean, last-layer weights zero
    net.set_params(p)
    hist = net.train(X, Y, epochs=150, batch=8, lr=1e-3, seed=1)
    assert hist[-1] < hist[0]
    test = clusters.water_cluster(5, 20000)
    with lib.Handle(test) as h:
        core = h.scf()
        D0 = h.mlp_guess(net, bf16=True)
        learned = h.scf(guess=D0)
    net.close()
    print(f"iterations core-H {core['iterations']} learned {learned['iterations']}, "
          f"dE {learned['energy'] - core['energy']:.2e}")
    assert learned["converged"] and core["converged"]
    assert abs(learned["energy"] - core["energy"]) <= 1e-8
    assert learned["iterations"] < core["iterations"]


def test_pair_blocks_round_trip_and_rotation_invariant(lib):
    """Pair blocks (df_pair_blocks) of a converged density, put back by df_pair_density, reproduce D's
    off-diagonal water blocks; the frame blocks do not change when the cluster is rotated."""
    s1 = clusters.water_cluster(4, 77)
    q, r = np.linalg.qr(np.random.default_rng(9).normal(size=(3, 3)))
    R = q * np.sign(np.diag(r))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    s2 = _rotate(s1, R, np.array([-0.4, 2.2, 0.9]))
    out = []
    for s in (s1, s2):
        pairs, _ = lib.water_pairs(s, cutoff=100.0)          # every pair, both orders
        assert len(pairs) == 12
        with lib.Handle(s) as h:
            h.scf()
            D = h.matrix("D")
            b = h.pair_blocks(D, pairs)
            D0 = h.pair_density(b, pairs)
        for w1, w2 in pairs:
            blk = (slice(50 * w1, 50 * w1 + 50), slice(50 * w2, 50 * w2 + 50))
            assert np.abs(D0[blk] - D[blk]).max() <= 1e-5 * np.abs(D).max()
        for w in range(4):
            assert np.abs(D0[50 * w:50 * w + 50, 50 * w:50 * w + 50]).max() == 0.0
        out.append(b)
    assert np.abs(out[0] - out[1]).max() <= 1e-6 * np.abs(out[0]).max()


def test_learned_guess_with_pair_blocks(lib):
    """Diagonal and pair networks trained on a few small clusters: the SCF from the guess with pair blocks
    converges to the core-Hamiltonian energy in fewer iterations."""
    train = [clusters.water_cluster(w, 10000 + k) for k, w in enumerate([2, 3, 4, 3, 2, 4])]
    X, Y, XP, YP = [], [], [], []
    for s in train:
        pairs, pf = lib.water_pairs(s)
        with lib.Handle(s) as h:
            h.scf()
            D = h.matrix("D")
            Y.append(h.water_blocks(D))
            if len(pairs):
                YP.append(h.pair_blocks(D, pairs).reshape(len(pairs), -1))
                XP.append(pf)
        X.append(lib.water_features(s))
    nets = []
    for Xs, Ys, nin in ((X, Y, lib.DF_MLP_NFEAT), (XP, YP, lib.DF_MLP_NPFEAT)):
        Xs, Ys = np.concatenate(Xs), np.concatenate(Ys)
        net = lib.Mlp(nin, 64, 3, Ys.shape[1], seed=11)
        nout = Ys.shape[1]
        p = net.params()
        p[-nout:] = Ys.mean(axis=0)
        p[-nout - nout * 64:-nout] = 0.0
        net.set_params(p)
        hist = net.train(Xs, Ys, epochs=150, batch=8, lr=1e-3, seed=1)
        assert hist[-1] < hist[0]
        nets.append(net)
    test = clusters.water_cluster(5, 20000)
    with lib.Handle(test) as h:
        core = h.scf()
        D0 = h.mlp_guess(nets[0], bf16=True, pair_mlp=nets[1])
        learned = h.scf(guess=D0)
    for n in nets:
        n.close()
    print(f"iterations core-H {core['iterations']} learned with pairs {learned['iterations']}, "
          f"dE {learned['energy'] - core['energy']:.2e}")
    assert learned["converged"] and core["converged"]
    assert abs(learned["energy"] - core["energy"]) <= 1e-8
    assert learned["iterations"] < core["iterations"]
