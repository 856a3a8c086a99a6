"""Incremental Fock builds: late iterations take K = K[D_ref] + K[D - D_ref], the density change
factorised exactly from the occupied orbitals of both densities, with a full build every 8 iterations.

In FP64 the change is built exactly, so the SCF must land on the full-build energy; in split mode the
change is built at 3 slices on top of a 5-slice reference and must stay within the split tolerance of
the FP64 energy on the same B."""
import numpy as np
import pytest

from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def water8_runs(lib):
    system = clusters.workload("water8")
    with lib.Handle(system) as h:
        runs = {"fp64": h.scf(), "fp64_inc": h.scf(incremental=1),
                "split": h.scf(precision=lib.DF_PREC_SPLIT, slices=3),
                "split_inc": h.scf(precision=lib.DF_PREC_SPLIT, slices=3, incremental=1)}
        runs["history"] = h.history()
    for k, r in runs.items():
        if k != "history":
            print(f"{k}: E {r['energy']:.10f} it {r['iterations']} incremental {r['incremental_builds']} "
                  f"t_jk {r['t_jk_s']:.3f}s")
    return runs


def test_fp64_incremental_equals_full_builds(water8_runs):
    full, inc = water8_runs["fp64"], water8_runs["fp64_inc"]
    assert full["converged"] and inc["converged"]
    assert full["incremental_builds"] == 0
    assert inc["incremental_builds"] > 0
    assert abs(inc["energy"] - full["energy"]) <= 1e-9


def test_split_incremental_within_split_tolerance(water8_runs):
    e64, inc = water8_runs["fp64"]["energy"], water8_runs["split_inc"]
    assert inc["converged"] and inc["incremental_builds"] > 0
    assert abs(inc["energy"] - e64) <= 1e-6
    assert abs(inc["energy"] - water8_runs["split"]["energy"]) <= 1e-8


def test_incremental_resets_every_eight_iterations(water8_runs):
    inc = water8_runs["split_inc"]
    late = inc["iterations"] - inc["ramp_iteration"] + 1     # iterations from the first 5-slice build on
    full_late = late - inc["incremental_builds"]
    # one full (reference) build opens each block of 8 late iterations
    assert full_late == int(np.ceil(late / 8))
