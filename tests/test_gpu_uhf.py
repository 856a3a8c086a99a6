"""DF-UHF on the GPU (scf_run_uhf) against the oracle (oracle/dfuhf.py): the closed-shell reduction to the RHF
energy, the one-electron hydrogen atom (lowest eigenvalue of the core Hamiltonian, <S^2> = 3/4), and the
doublet cation and triplet of the 2-water cluster, energy, <S^2> and spin densities element by element;
the split-precision exchange within 1e-6 Eh. DF-ROHF (scf_run_rohf) against oracle/dfrohf.py the same way,
with <S^2> = S(S+1) and E_UHF <= E_ROHF."""
import numpy as np
import pytest

from oracle import dfuhf, sad
from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def water2():
    return clusters.workload("water2")


def test_closed_shell_uhf_equals_rhf(lib, water2):
    with lib.Handle(water2) as h:
        h.build_B()
        r = h.scf()
        u = h.scf_uhf(10, 10)
    assert u["converged"] and abs(u["energy"] - r["energy"]) <= 1e-9, (u["energy"], r["energy"])
    assert abs(u["s2"]) <= 1e-9


def test_hydrogen_atom(lib, water2):
    from scipy.linalg import eigh

    from oracle import dfrhf
    atom = sad.atom_system(water2, 1)
    e0 = eigh(dfrhf.core_hamiltonian(atom), dfrhf.overlap(atom), eigvals_only=True)[0]
    with lib.Handle(atom, open_shell=True) as h:
        u = h.scf_uhf(1, 0)
        with pytest.raises(lib.DFError) as e:
            h.scf()                          # restricted SCF refuses an odd electron count
        assert e.value.code == lib.DF_E_STATE
    assert u["converged"] and abs(u["energy"] - e0) <= 1e-10, (u["energy"], e0)
    assert abs(u["s2"] - 0.75) <= 1e-10


@pytest.mark.parametrize("charge,na,nb", [(1, 10, 9), (0, 11, 9)])
def test_open_shell_against_oracle(lib, water2, charge, na, nb):
    import copy
    system = copy.deepcopy(water2)
    system.charge = charge
    ref = dfuhf.uhf(system, na, nb)
    assert ref.converged
    with lib.Handle(system, open_shell=True) as h:
        h.build_B(whitening=lib.DF_WHITEN_FP64)
        u = h.scf_uhf(na, nb)
        Da, Db = h.matrix("Da"), h.matrix("Db")
        us = h.scf_uhf(na, nb, precision=lib.DF_PREC_SPLIT, slices=3)
    print(f"charge {charge} ({na}, {nb}): GPU {u['energy']:.10f} ({u['iterations']} it), oracle {ref.energy:.10f} "
          f"({ref.iterations} it), <S^2> {u['s2']:.6f} vs {ref.s2:.6f}; split {us['energy'] - u['energy']:+.2e}")
    assert u["converged"] and us["converged"]
    assert abs(u["energy"] - ref.energy) <= 1e-9
    assert abs(u["s2"] - ref.s2) <= 1e-6
    assert np.abs(Da - ref.Da).max() <= 1e-6 and np.abs(Db - ref.Db).max() <= 1e-6
    assert abs(us["energy"] - u["energy"]) <= 1e-6


@pytest.mark.parametrize("charge,na,nb", [(1, 10, 9), (0, 11, 9)])
def test_rohf_against_oracle(lib, water2, charge, na, nb):
    """ROHF (scf_run_rohf) against oracle/dfrohf.py on the same FP64 B: energy, <S^2> = S(S+1), spin
    densities; above the UHF energy; the split-precision exchange within 1e-6 Eh; closed shell = RHF."""
    import copy

    from oracle import dfrhf, dfrohf
    system = copy.deepcopy(water2)
    system.charge = charge
    ref = dfrohf.rohf(system, na, nb)
    assert ref.converged
    with lib.Handle(system, open_shell=True) as h:
        h.build_B(whitening=lib.DF_WHITEN_FP64)
        ro = h.scf_rohf(na, nb)
        Da, Db = h.matrix("Da"), h.matrix("Db")
        u = h.scf_uhf(na, nb)
        rs = h.scf_rohf(na, nb, precision=lib.DF_PREC_SPLIT, slices=3)
        with pytest.raises(lib.DFError) as e:
            h.scf_rohf(na, nb, level_shift=-1.0)
        assert e.value.code == lib.DF_E_ARG
    S = 0.5 * (na - nb)
    print(f"ROHF charge {charge} ({na}, {nb}): GPU {ro['energy']:.10f} ({ro['iterations']} it), oracle "
          f"{ref.energy:.10f} ({ref.iterations} it), UHF {u['energy']:.10f}; <S^2> {ro['s2']:.8f}; "
          f"split {rs['energy'] - ro['energy']:+.2e}")
    assert ro["converged"] and rs["converged"]
    assert abs(ro["energy"] - ref.energy) <= 1e-9
    assert abs(ro["s2"] - S * (S + 1)) <= 1e-9
    assert np.abs(Da - ref.Da).max() <= 1e-6 and np.abs(Db - ref.Db).max() <= 1e-6
    assert u["energy"] <= ro["energy"] + 1e-10
    assert abs(rs["energy"] - ro["energy"]) <= 1e-6


def test_closed_shell_rohf_equals_rhf(lib, water2):
    with lib.Handle(water2) as h:
        h.build_B()
        r = h.scf()
        ro = h.scf_rohf(10, 10)
    assert ro["converged"] and abs(ro["energy"] - r["energy"]) <= 1e-9, (ro["energy"], r["energy"])


def test_uhf_from_rohf_spin_densities(lib, water2):
    """UHF started from the ROHF solution (DF_GUESS_SPIN): the ROHF determinant is one of UHF's, so the run
    descends to an energy at or below ROHF's; a handle without an earlier open-shell run refuses the guess."""
    import copy
    system = copy.deepcopy(water2)
    system.charge = 1
    with lib.Handle(system, open_shell=True) as h:
        h.build_B(whitening=lib.DF_WHITEN_FP64)
        with pytest.raises(lib.DFError) as e:
            h.scf_uhf(10, 9, guess="spin")
        assert e.value.code == lib.DF_E_STATE
        ro = h.scf_rohf(10, 9)
        us = h.scf_uhf(10, 9, guess="spin")
        uc = h.scf_uhf(10, 9)
    print(f"ROHF {ro['energy']:.10f}, UHF from ROHF {us['energy']:.10f} ({us['iterations']} it), "
          f"UHF from core-H {uc['energy']:.10f}")
    assert ro["converged"] and us["converged"]
    assert us["energy"] <= ro["energy"] + 1e-10
    assert us["s2"] >= 0.75 - 1e-9
