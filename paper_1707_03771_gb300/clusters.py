"""Seeded synthetic workloads: water clusters and their even-tempered Gaussian bases.

This module is the one input generator that both the CUDA path and the CPU oracle read.
It holds geometry and basis *data* only -- atoms, shell angular momenta, exponents and
centres -- and none of the method's arithmetic (no normalisation, no integrals).

Workload recipe (the paper names no molecules for this path; it states only that every
algorithm rests on density fitting with the three-index tensor held in memory, section
"Density fitting utilities"):

* Monomer: O at the origin, two H at 0.96 Angstrom, H-O-H angle 104.5 degrees.
* Orientation: uniform random rotation from a Shoemake unit quaternion (3 uniforms).
* Placement: O uniform in a cube of side (n_water * 29.9 A^3)^(1/3) (liquid-water number
  density); a molecule is rejected if any O-O distance is < 2.6 A or any intermolecular
  atom pair is < 1.5 A.
* PRNG: SplitMix64, doubles in [0, 1) from the top 53 bits.
* Orbital basis (uncontracted, spherical): O 8 s (0.15*2.8^k), 4 p (0.2*3^k), 2 d (0.8, 2.4);
  H 4 s (0.1*3^k), 2 p (0.5, 1.5)  -> 50 functions per water.
* Auxiliary basis: exponents 0.1*2^k per angular momentum; O 12 s, 8 p, 6 d, 3 f;
  H 6 s, 3 p, 2 d  -> 137 functions per water.
* Units: the generator works in Angstrom and returns bohr (1 bohr = 0.529177210903 A).
* Shell order: atom order; within an atom by l ascending, then exponent descending.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then a 3-step mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


# --- basis definitions (exponents only; per element: list of (l, [exponents])) -----------------

def _even(alpha0: float, ratio: float, count: int) -> list[float]:
    return [alpha0 * ratio ** k for k in range(count)]


ORBITAL_BASIS = {
    8: [(0, _even(0.15, 2.8, 8)), (1, _even(0.2, 3.0, 4)), (2, [0.8, 2.4])],
    1: [(0, _even(0.1, 3.0, 4)), (1, [0.5, 1.5])],
}
AUX_BASIS = {
    8: [(0, _even(0.1, 2.0, 12)), (1, _even(0.1, 2.0, 8)), (2, _even(0.1, 2.0, 6)),
        (3, _even(0.1, 2.0, 3))],
    1: [(0, _even(0.1, 2.0, 6)), (1, _even(0.1, 2.0, 3)), (2, _even(0.1, 2.0, 2))],
}

SHELL_DTYPE = np.dtype([("atom", np.int32), ("l", np.int32), ("exponent", np.float64),
                        ("center", np.float64, (3,))])
ATOM_DTYPE = np.dtype([("xyz", np.float64, (3,)), ("Z", np.int32)])


@dataclass
class System:
    """A molecule with its orbital and auxiliary shell lists (bohr)."""
    atoms: np.ndarray        # ATOM_DTYPE
    basis: np.ndarray        # SHELL_DTYPE
    aux: np.ndarray          # SHELL_DTYPE
    charge: int = 0
    label: str = ""

    @property
    def n_electrons(self) -> int:
        return int(self.atoms["Z"].sum()) - self.charge

    @property
    def nocc(self) -> int:
        return self.n_electrons // 2

    @property
    def nbf(self) -> int:
        return int((2 * self.basis["l"] + 1).sum())

    @property
    def naux(self) -> int:
        return int((2 * self.aux["l"] + 1).sum())


def shells_for(atoms: np.ndarray, table: dict) -> np.ndarray:
    """Shell list for `atoms` from a per-element table; order: atom, l ascending, exponent descending."""
    rows = []
    for ia, atom in enumerate(atoms):
        for l, exps in sorted(table[int(atom["Z"])], key=lambda t: t[0]):
            for a in sorted(exps, reverse=True):
                rows.append((ia, l, a, tuple(atom["xyz"])))
    return np.array(rows, dtype=SHELL_DTYPE)


def make_system(atoms: np.ndarray, basis_table=ORBITAL_BASIS, aux_table=AUX_BASIS,
                charge: int = 0, label: str = "") -> System:
    return System(atoms=atoms, basis=shells_for(atoms, basis_table),
                  aux=shells_for(atoms, aux_table), charge=charge, label=label)


# --- water cluster geometry ---------------------------------------------------------------------

R_OH = 0.96          # Angstrom
HOH_DEG = 104.5
MIN_OO = 2.6
MIN_INTER = 1.5
VOLUME_PER_WATER = 29.9


def _monomer() -> np.ndarray:
    half = math.radians(HOH_DEG / 2.0)
    return np.array([[0.0, 0.0, 0.0],
                     [R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
                     [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)]])


def _quat_rotation(u1: float, u2: float, u3: float) -> np.ndarray:
    """Rotation matrix from Shoemake's uniform unit quaternion (Graphics Gems III, 1992)."""
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_cluster_atoms(n_water: int, seed: int, reject_inter: bool = True,
                        max_attempts: int = 200000) -> np.ndarray:
    """Seeded water cluster (atoms in bohr): O, H, H per molecule in placement order."""
    if n_water < 1:
        raise ValueError("n_water must be >= 1")
    rng = SplitMix64(seed)
    side = (n_water * VOLUME_PER_WATER) ** (1.0 / 3.0)
    mono = _monomer()
    placed: list[np.ndarray] = []
    attempts = 0
    while len(placed) < n_water:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError(f"could not place {n_water} waters (seed {seed})")
        o = np.array([rng.uniform() * side for _ in range(3)])
        rot = _quat_rotation(rng.uniform(), rng.uniform(), rng.uniform())
        mol = o + mono @ rot.T
        ok = True
        for other in placed:
            if np.linalg.norm(other[0] - mol[0]) < MIN_OO:
                ok = False
                break
            if reject_inter:
                d = np.linalg.norm(other[:, None, :] - mol[None, :, :], axis=-1)
                if d.min() < MIN_INTER:
                    ok = False
                    break
        if ok:
            placed.append(mol)
    xyz = np.concatenate(placed, axis=0) * BOHR_PER_ANGSTROM
    atoms = np.zeros(3 * n_water, dtype=ATOM_DTYPE)
    atoms["xyz"] = xyz
    atoms["Z"] = np.tile(np.array([8, 1, 1], dtype=np.int32), n_water)
    return atoms


def water_cluster(n_water: int, seed: int) -> System:
    return make_system(water_cluster_atoms(n_water, seed), label=f"water{n_water}_seed{seed}")


# Named workloads (sizes in functions: orbital n, auxiliary naux, occupied nocc).
WORKLOADS = {
    "water2": dict(n_water=2, seed=0),     # n=100,  naux=274,  nocc=10
    "water8": dict(n_water=8, seed=8),     # n=400,  naux=1096, nocc=40
    "water16": dict(n_water=16, seed=16),  # n=800,  naux=2192, nocc=80
    "water32": dict(n_water=32, seed=1),   # n=1600, naux=4384, nocc=160
    "water40": dict(n_water=40, seed=2),   # n=2000, naux=5480, nocc=200
}


def workload(name: str) -> System:
    spec = WORKLOADS[name]
    return water_cluster(spec["n_water"], spec["seed"])


def h2_system(r_bohr: float, alpha: float = 1.0) -> System:
    """H2 along z with one s Gaussian per atom; the auxiliary set is the product-complete set
    (s Gaussians of exponent 2*alpha on each atom and one of exponent 2*alpha at the bond midpoint),
    which spans every orbital product exactly."""
    atoms = np.zeros(2, dtype=ATOM_DTYPE)
    atoms["xyz"] = [[0, 0, 0], [0, 0, r_bohr]]
    atoms["Z"] = [1, 1]
    basis = np.array([(0, 0, alpha, (0, 0, 0)), (1, 0, alpha, (0, 0, r_bohr))], dtype=SHELL_DTYPE)
    aux = np.array([(0, 0, 2 * alpha, (0, 0, 0)), (1, 0, 2 * alpha, (0, 0, r_bohr)),
                    (0, 0, 2 * alpha, (0, 0, r_bohr / 2))], dtype=SHELL_DTYPE)
    return System(atoms=atoms, basis=basis, aux=aux, label="h2")


def random_shells(rng: SplitMix64, count: int, lmax: int, box: float = 3.0,
                  amin: float = 0.05, amax: float = 500.0, natom: int = 1) -> np.ndarray:
    """Random shells for parity tests: l uniform in 0..lmax, log-uniform exponents, centres in a box."""
    rows = []
    for _ in range(count):
        l = min(int(rng.uniform() * (lmax + 1)), lmax)
        a = amin * (amax / amin) ** rng.uniform()
        c = tuple((rng.uniform() - 0.5) * box for _ in range(3))
        rows.append((min(int(rng.uniform() * natom), natom - 1), l, a, c))
    return np.array(rows, dtype=SHELL_DTYPE)
