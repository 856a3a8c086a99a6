"""SCF iterations replayed from captured CUDA graphs: after the first occurrence of each kind of step, the
J/K build and the Fock / energy / DIIS-error part of an iteration are captured from the stream and replayed
(the DIIS slot is read from device memory). Replays run the same kernels with the same arguments, so the
energies and iteration counts equal those of direct launches (DFHF_SCF_GRAPHS=0) bit for bit."""
import os

import pytest

from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def _scf(h, graphs, **kw):
    old = os.environ.pop("DFHF_SCF_GRAPHS", None)
    if not graphs:
        os.environ["DFHF_SCF_GRAPHS"] = "0"
    try:
        return h.scf(**kw)
    finally:
        os.environ.pop("DFHF_SCF_GRAPHS", None)
        if old is not None:
            os.environ["DFHF_SCF_GRAPHS"] = old


@pytest.mark.parametrize("mode", ["fp64", "split_inc_approx", "sad_split"])
def test_graph_replay_equals_direct_launches(lib, mode):
    kw = {"fp64": {}, "split_inc_approx": dict(precision=lib.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1),
          "sad_split": dict(precision=lib.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1, guess="sad")}[mode]
    with lib.Handle(clusters.workload("water8")) as h:
        h.build_B()
        direct = _scf(h, False, **kw)
        graph = _scf(h, True, **kw)
    print(f"{mode}: iterations {graph['iterations']}, graph launches {graph['graph_launches']}")
    assert direct["converged"] and graph["converged"]
    assert direct["graph_launches"] == 0 and graph["graph_launches"] > 0
    assert graph["energy"] == direct["energy"] and graph["iterations"] == direct["iterations"]
