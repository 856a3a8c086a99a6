"""Superposition-of-atomic-densities guess on the GPU (df_sad_density, options.guess = DF_GUESS_SAD) against
the oracle (oracle/sad.py): the atoms' fractional-occupation DF-HF densities assembled block-diagonally,
element by element; SCF from the SAD guess reaches the core-Hamiltonian guess's energy (the converged state
does not depend on the guess), in FP64, in split precision and in the batched driver."""
import numpy as np
import pytest

from oracle import sad
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


def test_sad_density_matches_oracle(lib):
    system = clusters.workload("water2")
    ref = sad.sad_density(system)
    with lib.Handle(system) as h:
        D0 = h.sad_density()
        S = h.matrix("S")
    d = np.abs(D0 - ref).max()
    print(f"max|D0 - D0(oracle)| {d:.2e} (max|D0| {np.abs(ref).max():.2f})")
    assert d <= 5e-8 * np.abs(ref).max()
    assert abs(np.sum(D0 * S) - system.n_electrons) <= 1e-10


@pytest.mark.parametrize("name", ["water2", "water8"])
def test_scf_from_sad_reaches_core_guess_energy(lib, name):
    with lib.Handle(clusters.workload(name)) as h:
        h.build_B()
        core = h.scf()
        sadr = h.scf(guess="sad")
        split = h.scf(guess="sad", precision=lib.DF_PREC_SPLIT, slices=3, incremental=1, approx_diag=1)
    print(f"{name}: iterations core-H {core['iterations']}, SAD {sadr['iterations']}, SAD split {split['iterations']}")
    assert core["converged"] and sadr["converged"] and split["converged"]
    assert abs(sadr["energy"] - core["energy"]) <= 1e-9
    assert abs(split["energy"] - core["energy"]) <= 1e-6


def test_batched_sad_equals_single_runs(lib):
    systems = [clusters.water_cluster(w, 300 + w) for w in (1, 3, 2)]
    singles = []
    for s in systems:
        with lib.Handle(s) as h:
            singles.append(h.scf(guess="sad"))
    handles = [lib.Handle(s) for s in systems]
    try:
        res = lib.scf_batch(handles, guess="sad")
    finally:
        for h in handles:
            h.close()
    for a, b in zip(singles, res):
        assert b["converged"] and abs(a["energy"] - b["energy"]) <= 1e-9
