"""CPU-side checks of the CUDA library: it builds, loads without a GPU and exports every entry
point declared in include/dfhf.h (no compute calls here)."""
import ctypes
import os
import re

from paper_1707_03771_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == declared


def test_strerror_without_gpu():
    lib = binding.load()
    assert lib.df_strerror(0) == b"ok"
    assert lib.df_strerror(-1) == b"invalid argument"


def test_water_pair_features_are_rigid_motion_invariant():
    """Host logic of the learned guess's pair list (df_water_pairs, no GPU): both orders of every pair within
    the cutoff, nothing beyond it, and features unchanged under a rotation and translation of the cluster."""
    import numpy as np

    from paper_1707_03771_gb300 import clusters
    s = clusters.water_cluster(12, 31)
    pairs, feats = binding.water_pairs(s)
    O = s.atoms["xyz"][0::3]
    d = np.linalg.norm(O[:, None] - O[None], axis=-1)
    expect = [(a, b) for a in range(len(O)) for b in range(len(O)) if a != b and d[a, b] <= binding.PAIR_CUTOFF]
    assert [tuple(p) for p in pairs.tolist()] == expect and len(expect) > 0
    q, r = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    R = q * np.sign(np.diag(r))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    atoms = s.atoms.copy()
    atoms["xyz"] = atoms["xyz"] @ R.T + np.array([1.5, -0.7, 3.0])
    pairs2, feats2 = binding.water_pairs(clusters.make_system(atoms))
    assert np.array_equal(pairs, pairs2)
    assert np.abs(feats - feats2).max() <= 1e-5
    # the O-O distance expansion peaks at the distance
    r_oo = d[pairs[:, 0], pairs[:, 1]]
    centre = 4.5 + 0.5 * np.argmax(feats[:, 18:], axis=1)
    assert np.all(np.abs(centre - np.clip(r_oo, 4.5, 8.0)) <= 0.25 + 1e-9)
