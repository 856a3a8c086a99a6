"""Pins for the CPU oracle: closed forms, identities and invariants that fix what it computes
independently of its own code. Runs without a GPU."""
import math
import os

import numpy as np
import pytest
from scipy.special import erf, gamma, gammainc

from oracle import dfrhf
from paper_1707_03771_gb300 import clusters

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


# --------------------------------------------------------------------------- Boys function

@pytest.mark.parametrize("T", [0.0, 1e-12, 1e-6, 0.3, 1.7, 9.5, 25.0, 39.99, 40.01, 55.0, 130.0, 900.0])
def test_boys_incomplete_gamma(T):
    """F_m(T) = Gamma(m+1/2) P(m+1/2, T) / (2 T^(m+1/2)), with P the regularised lower incomplete gamma."""
    F = dfrhf.boys(8, T)
    for m in range(9):
        if T == 0.0:
            ref = 1.0 / (2 * m + 1)
        elif T < 1e-5:   # Taylor series of exp(-T t^2) integrated term by term
            ref = sum((-T) ** k / (math.factorial(k) * (2 * m + 2 * k + 1)) for k in range(6))
        else:
            ref = gamma(m + 0.5) * gammainc(m + 0.5, T) / (2 * T ** (m + 0.5))
        assert abs(F[m] - ref) <= 2e-14 * max(ref, 1e-300) + 1e-300, (m, T, F[m], ref)


def test_boys_f0_erf_and_asymptote():
    for T in [0.05, 0.5, 3.0, 12.0, 33.0, 60.0]:
        assert abs(dfrhf.boys(0, T)[0] - 0.5 * math.sqrt(math.pi / T) * erf(math.sqrt(T))) < 1e-15
    T = 300.0
    F = dfrhf.boys(7, T)
    for m in range(8):
        dfact = np.prod(np.arange(2 * m - 1, 0, -2)) if m > 0 else 1.0
        asym = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] / asym - 1) < 1e-13


def test_boys_downward_identity():
    for T in [0.2, 5.0, 38.0, 45.0, 80.0]:
        F = dfrhf.boys(9, T)
        for m in range(9):
            assert abs(F[m] - (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)) <= 1e-14 * F[m]


# --------------------------------------------------------------------------- s-type closed forms

def _rand_centre(scale=1.5):
    return rng.uniform(-scale, scale, 3)


S0 = (0, 0, 0)


def test_s_closed_forms():
    for _ in range(20):
        a, b, c, d = np.exp(rng.uniform(np.log(0.05), np.log(50.0), 4))
        A, B, C, D, Cn = (_rand_centre() for _ in range(5))
        p, q = a + b, c + d
        mu = a * b / p
        RAB2 = np.sum((A - B) ** 2)
        Kab = math.exp(-mu * RAB2)
        P = (a * A + b * B) / p
        Q = (c * C + d * D) / q
        # overlap and kinetic (Helgaker eq. 9.2.41-9.3.x closed forms for s functions)
        S = (math.pi / p) ** 1.5 * Kab
        assert abs(dfrhf.prim_overlap(S0, a, A, S0, b, B) - S) <= 1e-14 * S + 1e-300
        T = mu * (3 - 2 * mu * RAB2) * S
        assert abs(dfrhf.prim_kinetic(S0, a, A, S0, b, B) - T) <= 1e-13 * mu * (3 + 2 * mu * RAB2) * S + 1e-300
        # nuclear attraction: 2 pi / p K_ab F0(p |P - C|^2)
        V = 2 * math.pi / p * Kab * dfrhf.boys(0, p * np.sum((P - Cn) ** 2))[0]
        assert abs(dfrhf.prim_potential(S0, a, A, S0, b, B, Cn) - V) <= 1e-13 * V
        # two-centre: 2 pi^{5/2} / (a b sqrt(a+b)) F0(ab/(a+b) R^2)
        two = 2 * math.pi ** 2.5 / (a * b * math.sqrt(a + b)) * dfrhf.boys(0, a * b / (a + b) * RAB2)[0]
        assert abs(dfrhf.prim_eri(S0, a, A, S0, 0.0, A, S0, b, B, S0, 0.0, B) - two) <= 1e-13 * two
        # three-centre (s|ss) and four-centre (ss|ss)
        Kcd = math.exp(-c * d / q * np.sum((C - D) ** 2))
        three = 2 * math.pi ** 2.5 / (c * p * math.sqrt(c + p)) * Kab * dfrhf.boys(0, c * p / (c + p) * np.sum((C - P) ** 2))[0]
        assert abs(dfrhf.prim_3c(S0, c, C, S0, a, A, S0, b, B) - three) <= 1e-13 * three
        four = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * dfrhf.boys(0, p * q / (p + q) * np.sum((P - Q) ** 2))[0]
        assert abs(dfrhf.prim_eri(S0, a, A, S0, b, B, S0, c, C, S0, d, D) - four) <= 1e-13 * four + 1e-300


# --------------------------------------------------------------------------- higher l from centre derivatives

def _richardson(f, x0, h):
    def cd(hh):
        return (f(x0 + hh) - f(x0 - hh)) / (2 * hh)
    return (4 * cd(h / 2) - cd(h)) / 3


def _raise_power(fn, centres, exps, powers, which, axis):
    """x_A^{i+1} g = (1/2a) (d/dA_x [x_A^i g] + i x_A^{i-1} g), with A = centres[which]."""
    a = exps[which]
    i = powers[which][axis]

    def f_at(shift):
        cs = [np.array(c, dtype=float) for c in centres]
        cs[which][axis] += shift
        return fn(cs, powers)
    deriv = _richardson(f_at, 0.0, 2e-3)
    low = 0.0
    if i > 0:
        pl = [list(p) for p in powers]
        pl[which][axis] -= 1
        low = i * fn([np.array(c, dtype=float) for c in centres], pl)
    return (deriv + low) / (2 * a)


@pytest.mark.parametrize("kind", ["overlap", "potential", "three", "four"])
def test_centre_derivative_raises_l(kind):
    """A Cartesian power raised by one equals a centre derivative of the lower function (exact
    identity of Gaussians); checked with Richardson-extrapolated finite differences."""
    for trial in range(6):
        if kind == "overlap":
            nc = 2
            Cn = None
        elif kind == "potential":
            nc = 2
            Cn = _rand_centre()
        elif kind == "three":
            nc = 3
        else:
            nc = 4
        exps = list(np.exp(rng.uniform(np.log(0.2), np.log(3.0), nc)))
        centres = [_rand_centre(1.0) for _ in range(nc)]
        powers = [list(rng.integers(0, 2, 3)) for _ in range(nc)]

        def fn(cs, pw):
            if kind == "overlap":
                return dfrhf.prim_overlap(pw[0], exps[0], cs[0], pw[1], exps[1], cs[1])
            if kind == "potential":
                return dfrhf.prim_potential(pw[0], exps[0], cs[0], pw[1], exps[1], cs[1], Cn)
            if kind == "three":
                return dfrhf.prim_3c(pw[0], exps[0], cs[0], pw[1], exps[1], cs[1], pw[2], exps[2], cs[2])
            return dfrhf.prim_eri(pw[0], exps[0], cs[0], pw[1], exps[1], cs[1], pw[2], exps[2], cs[2],
                                  pw[3], exps[3], cs[3])
        which = int(rng.integers(0, nc))
        axis = int(rng.integers(0, 3))
        up = [list(p) for p in powers]
        up[which][axis] += 1
        direct = fn(centres, up)
        via = _raise_power(fn, centres, exps, powers, which, axis)
        scale = max(abs(direct), abs(fn(centres, powers)), 1e-3)
        assert abs(direct - via) <= 2e-8 * scale, (kind, trial, direct, via)


def test_point_charge_limit():
    """A tight s function of exponent alpha tends to (pi/alpha)^{3/2} times a point charge; the
    three-centre integral then tends to the nuclear-attraction integral (error O(1/alpha))."""
    for _ in range(4):
        a, b = np.exp(rng.uniform(np.log(0.3), np.log(2.0), 2))
        A, B, C = _rand_centre(), _rand_centre(), _rand_centre()
        pa, pb = list(rng.integers(0, 3, 3)), list(rng.integers(0, 2, 3))
        V = dfrhf.prim_potential(pa, a, A, pb, b, B, C)

        def f(alpha):
            return dfrhf.prim_3c(S0, alpha, C, pa, a, A, pb, b, B) / (math.pi / alpha) ** 1.5
        extrap = 2 * f(2e5) - f(1e5)
        assert abs(extrap - V) <= 1e-7 * max(abs(V), 1e-3)


# --------------------------------------------------------------------------- solid harmonics

def _read_golden_harmonics():
    rows = {}
    with open(os.path.join(GOLDEN, "solid_harmonics_l3.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            l, m = int(parts[0]), int(parts[1])
            poly = {}
            for t in parts[2:]:
                c, pw = t.split(":")
                poly[tuple(int(x) for x in pw.split(","))] = float(c)
            rows[(l, m)] = poly
    return rows


def test_solid_harmonics_match_textbook_table():
    gold = _read_golden_harmonics()
    for l in range(4):
        cs, pw = dfrhf.solid_harmonic_coeffs(l)
        for m in range(-l, l + 1):
            got = {tuple(pw[k]): cs[m + l, k] for k in range(len(pw)) if abs(cs[m + l, k]) > 1e-14}
            ref = gold[(l, m)]
            assert set(got) == set(ref), (l, m)
            for key in ref:
                assert abs(got[key] - ref[key]) < 1e-12, (l, m, key)


def _poly_eval(cs, pw, pts):
    mon = np.stack([np.prod(pts ** p, axis=1) for p in pw], axis=1)
    return mon @ cs.T


def test_solid_harmonics_harmonic_and_equal_norm():
    for l in range(4):
        cs, pw = dfrhf.solid_harmonic_coeffs(l)
        # Laplacian of each polynomial vanishes
        for m in range(2 * l + 1):
            lap = {}
            for k, p in enumerate(pw):
                for ax in range(3):
                    if p[ax] >= 2:
                        q = list(p)
                        q[ax] -= 2
                        lap[tuple(q)] = lap.get(tuple(q), 0.0) + cs[m, k] * p[ax] * (p[ax] - 1)
            assert all(abs(v) < 1e-12 for v in lap.values()), (l, m)
        # every m component has the same normalisation constant
        for a in [0.1, 1.3, 40.0]:
            n = dfrhf.sph_norms(l, a)
            assert np.allclose(n, n[0], rtol=1e-13, atol=0)


def _wigner_from_harmonics(l, R):
    """Matrix D with S_m(R x) = sum_m' D_mm' S_m'(x), fitted on random points."""
    cs, pw = dfrhf.solid_harmonic_coeffs(l)
    pts = rng.normal(size=(64, 3))
    A = _poly_eval(cs, pw, pts)
    Bm = _poly_eval(cs, pw, pts @ R.T)
    D, res, *_ = np.linalg.lstsq(A, Bm, rcond=None)
    assert np.allclose(A @ D, Bm, atol=1e-10)   # the span is rotation invariant
    return D.T


def _random_rotation():
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def _shell_system(specs):
    """System with explicit shells [(l, exponent, centre)], one dummy atom."""
    atoms = np.zeros(1, dtype=clusters.ATOM_DTYPE)
    atoms["Z"] = 2
    return np.array([(0, l, a, tuple(c)) for l, a, c in specs], dtype=clusters.SHELL_DTYPE), atoms


def test_three_center_rotation_translation_and_index_symmetry():
    R = _random_rotation()
    shift = np.array([0.7, -1.1, 0.4])
    for lp, lm, ln in [(3, 2, 2), (2, 2, 1), (1, 0, 2), (3, 1, 0)]:
        cP, cM, cN = _rand_centre(), _rand_centre(), _rand_centre()
        aP, aM, aN = 0.9, 0.6, 1.7
        basis, atoms = _shell_system([(lm, aM, cM), (ln, aN, cN)])
        aux, _ = _shell_system([(lp, aP, cP)])
        sysA = clusters.System(atoms=atoms, basis=basis, aux=aux)
        blk = dfrhf.three_center_triples(sysA, [(0, 0, 1), (0, 1, 0)])
        assert np.allclose(blk[0], blk[1].transpose(0, 2, 1), atol=1e-15, rtol=0)
        basis_r, _ = _shell_system([(lm, aM, R @ cM), (ln, aN, R @ cN)])
        aux_r, _ = _shell_system([(lp, aP, R @ cP)])
        rot = dfrhf.three_center_triples(clusters.System(atoms=atoms, basis=basis_r, aux=aux_r), [(0, 0, 1)])[0]
        DP, DM, DN = (_wigner_from_harmonics(l, R) for l in (lp, lm, ln))
        # normalised functions: the fitted D maps unnormalised harmonics; norms are m-independent
        pred = np.einsum("ap,bm,cn,pmn->abc", DP, DM, DN, blk[0])
        assert np.abs(pred - rot).max() < 1e-12 * max(1.0, np.abs(blk[0]).max())
        basis_t, _ = _shell_system([(lm, aM, cM + shift), (ln, aN, cN + shift)])
        aux_t, _ = _shell_system([(lp, aP, cP + shift)])
        tr = dfrhf.three_center_triples(clusters.System(atoms=atoms, basis=basis_t, aux=aux_t), [(0, 0, 1)])[0]
        assert np.abs(tr - blk[0]).max() < 1e-13


def test_overlap_diagonal_blocks_identity():
    sysw = clusters.water_cluster(1, 3)
    S = dfrhf.overlap(sysw)
    off = 0
    for sh in sysw.basis:
        k = 2 * sh["l"] + 1
        assert np.allclose(S[off:off + k, off:off + k], np.eye(k), atol=1e-13)
        off += k
    V = dfrhf.metric(sysw)
    assert np.allclose(V, V.T, atol=1e-13)
    assert np.linalg.eigvalsh(V).min() > 0


# --------------------------------------------------------------------------- density-fitting layer

def test_df_exact_for_product_complete_aux():
    """H2 with one s per atom; the auxiliary set spans every orbital product, so DF J and K equal the
    conventional four-index J and K up to the conditioning of the metric."""
    sysh = clusters.h2_system(1.4, alpha=0.8)
    B = dfrhf.whiten(dfrhf.three_center(sysh), dfrhf.metric(sysh))
    eri = dfrhf.four_center(sysh)
    C = np.linalg.qr(rng.normal(size=(2, 1)))[0]
    D = 2 * C @ C.T
    assert np.abs(dfrhf.df_J(B, D) - dfrhf.conv_J(eri, D)).max() < 1e-10
    assert np.abs(dfrhf.df_K(B, C) - dfrhf.conv_K(eri, C)).max() < 1e-10


def test_df_coulomb_variational_and_monotone():
    """Coulomb-metric fitting underestimates the Coulomb energy, and a larger auxiliary set (a
    superset) raises the fitted energy towards the exact value."""
    sysw = clusters.water_cluster(1, 7)
    # a smaller orbital basis keeps the four-index reference quick
    sysw.basis = sysw.basis[sysw.basis["l"] <= 1]
    n = dfrhf.nfunc(sysw.basis)
    C = np.linalg.qr(rng.normal(size=(n, 5)))[0]
    D = 2 * C @ C.T
    eri = dfrhf.four_center(sysw)
    e_exact = 0.5 * np.sum(D * dfrhf.conv_J(eri, D))
    energies = []
    for lmax in (0, 1, 2, 3):
        aux = sysw.aux[sysw.aux["l"] <= lmax]
        s2 = clusters.System(atoms=sysw.atoms, basis=sysw.basis, aux=aux)
        B = dfrhf.whiten(dfrhf.three_center(s2), dfrhf.metric(s2))
        energies.append(0.5 * np.sum(D * dfrhf.df_J(B, D)))
    assert all(e <= e_exact + 1e-10 for e in energies)
    assert all(energies[i] <= energies[i + 1] + 1e-10 for i in range(3))
    assert energies[-1] > energies[0]


# --------------------------------------------------------------------------- SCF

def test_h2_closed_form_energy():
    """One s Gaussian per H: the occupied orbital is fixed by symmetry, so the RHF energy follows
    from the s-type closed forms; the product-complete auxiliary set makes DF exact."""
    R, a = 1.4, 0.8
    sysh = clusters.h2_system(R, alpha=a)
    res = dfrhf.scf(sysh)
    N = (2 * a / math.pi) ** 0.75
    s12 = N * N * (math.pi / (2 * a)) ** 1.5 * math.exp(-a / 2 * R * R)
    t11 = N * N * (a / 2) * 3 * (math.pi / (2 * a)) ** 1.5
    t12 = N * N * (a / 2) * (3 - a * R * R) * (math.pi / (2 * a)) ** 1.5 * math.exp(-a / 2 * R * R)
    F0 = lambda T: 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * erf(math.sqrt(T))
    pref = 2 * math.pi / (2 * a)
    v11 = -N * N * pref * (F0(0) + F0(2 * a * R * R))
    v12 = -N * N * pref * math.exp(-a / 2 * R * R) * 2 * F0(2 * a * (R / 2) ** 2)
    h11, h12 = t11 + v11, t12 + v12

    def eri(A, B, C, D):
        cen = np.array([0.0, R])
        P = (cen[A] + cen[B]) / 2
        Q = (cen[C] + cen[D]) / 2
        K = math.exp(-a / 2 * (cen[A] - cen[B]) ** 2) * math.exp(-a / 2 * (cen[C] - cen[D]) ** 2)
        p = q = 2 * a
        return N ** 4 * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * K * F0(p * q / (p + q) * (P - Q) ** 2)
    c = 1 / math.sqrt(2 * (1 + s12))
    hs = c * c * (2 * h11 + 2 * h12)
    Js = 0.0
    for A in range(2):
        for B in range(2):
            for C in range(2):
                for D in range(2):
                    Js += c ** 4 * eri(A, B, C, D)
    e = 2 * hs + Js + 1.0 / R
    assert abs(res.energy - e) < 1e-10, (res.energy, e)


def _water_rotated(sysw, R, shift):
    atoms = sysw.atoms.copy()
    atoms["xyz"] = atoms["xyz"] @ R.T + shift
    return clusters.make_system(atoms)


@pytest.fixture(scope="module")
def water1_result():
    sysw = clusters.water_cluster(1, 11)
    return sysw, dfrhf.scf(sysw)


def test_scf_density_invariants(water1_result):
    sysw, res = water1_result
    assert res.converged
    S = dfrhf.overlap(sysw)
    D = res.D
    assert abs(np.trace(D @ S) - sysw.n_electrons) < 1e-10
    assert np.abs(D @ S @ D - 2 * D).max() < 1e-10
    assert np.abs(res.J - res.J.T).max() < 1e-12 and np.abs(res.K - res.K.T).max() < 1e-12
    comm = res.F @ D @ S - S @ D @ res.F
    assert np.abs(comm).max() < 1e-6
    # exchange of the occupied orbitals is invariant under a rotation among them
    B = dfrhf.whiten(dfrhf.three_center(sysw), dfrhf.metric(sysw))
    Cocc = res.C[:, :sysw.nocc]
    Q = np.linalg.qr(rng.normal(size=(sysw.nocc, sysw.nocc)))[0]
    assert np.abs(dfrhf.df_K(B, Cocc) - dfrhf.df_K(B, Cocc @ Q)).max() < 1e-12


def test_scf_energy_rigid_motion_invariance(water1_result):
    sysw, res = water1_result
    R = _random_rotation()
    moved = _water_rotated(sysw, R, np.array([1.3, -0.2, 2.9]))
    assert abs(dfrhf.scf(moved).energy - res.energy) < 1e-10


def test_scf_energy_permutation_invariance():
    sysw = clusters.water_cluster(2, 21)
    e1 = dfrhf.scf(sysw).energy
    atoms = np.concatenate([sysw.atoms[3:], sysw.atoms[:3]])
    e2 = dfrhf.scf(clusters.make_system(atoms)).energy
    assert abs(e1 - e2) < 1e-10


def test_nuclear_repulsion_closed_form():
    atoms = np.zeros(3, dtype=clusters.ATOM_DTYPE)
    atoms["xyz"] = [[0, 0, 0], [3, 0, 0], [0, 4, 0]]
    atoms["Z"] = [8, 1, 2]
    assert abs(dfrhf.nuclear_repulsion(atoms) - (8 / 3 + 16 / 4 + 2 / 5)) < 1e-14


def test_generator_counts_and_geometry():
    s = clusters.workload("water2")
    assert (s.nbf, s.naux, s.nocc) == (100, 274, 10)
    big = clusters.water_cluster(32, 1)
    assert (big.nbf, big.naux, big.nocc) == (1600, 4384, 160)
    xyz = big.atoms["xyz"] / clusters.BOHR_PER_ANGSTROM
    O = xyz[0::3]
    d = np.linalg.norm(O[:, None] - O[None], axis=-1) + np.eye(32) * 10
    assert d.min() >= 2.6 - 1e-12
    for w in range(32):
        r1 = np.linalg.norm(xyz[3 * w + 1] - xyz[3 * w])
        r2 = np.linalg.norm(xyz[3 * w + 2] - xyz[3 * w])
        v1, v2 = xyz[3 * w + 1] - xyz[3 * w], xyz[3 * w + 2] - xyz[3 * w]
        ang = math.degrees(math.acos(np.dot(v1, v2) / (r1 * r2)))
        assert abs(r1 - 0.96) < 1e-12 and abs(r2 - 0.96) < 1e-12 and abs(ang - 104.5) < 1e-9
    # SplitMix64 reference values: seed 0 first output (published test vector)
    assert clusters.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


# --------------------------------------------------------------------------- learned-guess network

def test_mlp_oracle_gradient_central_differences():
    """The oracle's backpropagated gradient equals central differences of its own loss."""
    from oracle import mlp
    rs = np.random.default_rng(3)
    dims = [5, 8, 8, 8, 4]
    n = sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))
    p = rs.normal(size=n) * 0.5
    X = rs.normal(size=(7, 5))
    Y = rs.normal(size=(7, 4))
    g = mlp.gradient(p, dims, X, Y)
    h = 1e-6
    for k in rs.choice(n, 40, replace=False):
        e = np.zeros(n)
        e[k] = h
        fd = (mlp.loss(p + e, dims, X, Y) - mlp.loss(p - e, dims, X, Y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-6 * abs(g[k]), (k, fd, g[k])


def test_mlp_oracle_forward_and_loss_hand_computed():
    """The oracle's forward pass and loss on a 2 -> 3 (ReLU) -> 2 network whose outputs were worked out by
    hand. Layout per layer: W (out x in, row-major), then b. Sample 1 leaves two hidden units negative (the
    ReLU must cut them) and has a negative output (no ReLU on the output layer); sample 2 keeps every
    hidden unit. A transposed W, a dropped bias or an activation on the last layer changes the values."""
    from oracle import mlp
    W1 = [[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]
    b1 = [0.0, 1.0, -0.5]
    W2 = [[2.0, 1.0, -1.0], [0.5, 3.0, 4.0]]
    b2 = [0.25, -1.0]
    params = np.array(sum(W1, []) + b1 + sum(W2, []) + b2)
    dims = [2, 3, 2]
    X = np.array([[1.0, -2.0], [0.5, 1.5]])
    # sample 1: z1 = (1, -1, -1.5) -> h = (1, 0, 0) -> out = (2 + 0.25, 0.5 - 1) = (2.25, -0.5)
    # sample 2: z1 = (0.5, 2.5, 1.5) = h -> out = (1 + 2.5 - 1.5 + 0.25, 0.25 + 7.5 + 6 - 1) = (2.25, 12.75)
    Z, acts = mlp.forward(params, dims, X)
    assert np.array_equal(Z[0], [[1.0, -1.0, -1.5], [0.5, 2.5, 1.5]])
    assert np.array_equal(acts[1], [[1.0, 0.0, 0.0], [0.5, 2.5, 1.5]])
    assert np.array_equal(acts[-1], [[2.25, -0.5], [2.25, 12.75]])
    # loss: mean of (0.25, -0.5, 0.25, 0.75)^2 = 0.9375 / 4
    Y = np.array([[2.0, 0.0], [2.0, 12.0]])
    assert mlp.loss(params, dims, X, Y) == 0.234375


# ---------------------------------------------------------------------------------------------
# superposition of atomic densities (oracle/sad.py)
# ---------------------------------------------------------------------------------------------

def test_aufbau_occupations_hand_cases():
    from oracle import sad
    eps = np.array([-20.0, -1.0, -0.5, -0.5 + 1e-12, -0.5 - 1e-12, 0.3, 0.3, 0.9])
    assert np.allclose(sad.aufbau_occupations(eps, 8), [2, 2, 4 / 3, 4 / 3, 4 / 3, 0, 0, 0], atol=0)
    assert np.array_equal(sad.aufbau_occupations(eps, 1), [1, 0, 0, 0, 0, 0, 0, 0])
    assert np.array_equal(sad.aufbau_occupations(eps, 10), [2, 2, 2, 2, 2, 0, 0, 0])
    assert np.array_equal(sad.aufbau_occupations(eps, 11), [2, 2, 2, 2, 2, 0.5, 0.5, 0])
    assert sad.aufbau_occupations(eps, 7).sum() == 7


@pytest.fixture(scope="module")
def water2_sys():
    return clusters.workload("water2")


@pytest.mark.parametrize("atom_index,z", [(0, 10), (1, 2)])
def test_fractional_scf_reduces_to_rhf_for_closed_shells(water2_sys, atom_index, z):
    """With every occupied shell full (Ne in the oxygen shells, He in the hydrogen shells) the occupations
    are integers and the fractional-occupation SCF is the closed-shell DF-RHF of dfrhf.scf: same energy."""
    from oracle import sad
    atom = sad.atom_system(water2_sys, atom_index)
    atom.atoms["Z"] = z
    D, e, eps, occ, _ = sad.atomic_scf(atom)
    ref = dfrhf.scf(atom)
    assert np.array_equal(occ[:z // 2], np.full(z // 2, 2.0)) and occ[z // 2:].sum() == 0
    assert abs(e - ref.energy) <= 1e-9, (e, ref.energy)
    assert np.abs(D - ref.D).max() <= 1e-6


def test_oxygen_atom_density_is_spherical(water2_sys):
    """Fractional occupation 4/3 of each 2p orbital: tr(DS) = 8, and the density is spherical, i.e. in
    real solid harmonics every (l, l') block between two shells is zero for l != l' and a multiple of the
    identity over m for l = l' (the rotation matrices of each l are orthogonal)."""
    from oracle import sad
    atom = sad.atom_system(water2_sys, 0)
    D, e, eps, occ, _ = sad.atomic_scf(atom)
    S = dfrhf.overlap(atom)
    assert abs(np.sum(D * S) - 8.0) <= 1e-11
    assert np.allclose(occ[:5], [2, 2, 4 / 3, 4 / 3, 4 / 3], rtol=0, atol=1e-15) and occ[5:].sum() == 0
    ls = atom.basis["l"]
    off = np.concatenate([[0], np.cumsum(2 * ls + 1)])
    scale = np.abs(D).max()
    for i, li in enumerate(ls):
        for j, lj in enumerate(ls):
            blk = D[off[i]:off[i + 1], off[j]:off[j + 1]]
            if li != lj:
                assert np.abs(blk).max() <= 1e-10 * scale
            else:
                assert np.abs(blk - blk[0, 0] * np.eye(2 * li + 1)).max() <= 1e-10 * scale


def test_hydrogen_atom_density_is_one_electron(water2_sys):
    from oracle import sad
    atom = sad.atom_system(water2_sys, 1)
    D, e, eps, occ, _ = sad.atomic_scf(atom)
    S = dfrhf.overlap(atom)
    assert occ[0] == 1.0 and occ[1:].sum() == 0
    w = np.sort(np.linalg.eigvals(D @ S).real)
    assert abs(w[-1] - 1.0) <= 1e-10 and np.abs(w[:-1]).max() <= 1e-10   # one orbital, occupation 1


def test_sad_density_assembly(water2_sys):
    from oracle import sad
    D0 = sad.sad_density(water2_sys)
    S = dfrhf.overlap(water2_sys)
    assert abs(np.sum(D0 * S) - water2_sys.n_electrons) <= 1e-10
    off = np.concatenate([[0], np.cumsum(2 * water2_sys.basis["l"] + 1)])
    blocks = []
    for a in range(len(water2_sys.atoms)):
        sh = np.flatnonzero(water2_sys.basis["atom"] == a)
        blocks.append((off[sh[0]], off[sh[-1] + 1]))
    Dox = sad.atomic_scf(sad.atom_system(water2_sys, 0))[0]
    for a, (lo, hi) in enumerate(blocks):
        for b, (lo2, hi2) in enumerate(blocks):
            blk = D0[lo:hi, lo2:hi2]
            if a != b:
                assert not blk.any()
        if int(water2_sys.atoms["Z"][a]) == 8:
            assert np.abs(D0[lo:hi, lo:hi] - Dox).max() <= 1e-12


# ---------------------------------------------------------------------------------------------
# unrestricted Hartree-Fock (oracle/dfuhf.py)
# ---------------------------------------------------------------------------------------------

def test_uhf_closed_shell_equals_rhf(water2_sys):
    """With as many alpha as beta electrons the UHF determinant stays restricted: the RHF energy, spin
    densities of half the RHF density, <S^2> = 0."""
    from oracle import dfuhf
    n = water2_sys.n_electrons // 2
    u = dfuhf.uhf(water2_sys, n, n)
    r = dfrhf.scf(water2_sys)
    assert u.converged and abs(u.energy - r.energy) <= 1e-9, (u.energy, r.energy)
    assert np.abs(u.Da - 0.5 * r.D).max() <= 1e-6 and np.abs(u.Da - u.Db).max() <= 1e-6
    assert abs(u.s2) <= 1e-9


def test_uhf_hydrogen_atom_has_no_electron_interaction(water2_sys):
    """One electron: J[D_a] and K_a cancel exactly (with density fitting too: both give sum_P gamma_P^2 for
    the single orbital), so the UHF energy is the lowest eigenvalue of the core Hamiltonian in the metric S,
    and <S^2> = 3/4."""
    from scipy.linalg import eigh

    from oracle import dfuhf, sad
    atom = sad.atom_system(water2_sys, 1)
    u = dfuhf.uhf(atom, 1, 0)
    e0 = eigh(dfrhf.core_hamiltonian(atom), dfrhf.overlap(atom), eigvals_only=True)[0]
    assert u.converged and abs(u.energy - e0) <= 1e-10, (u.energy, e0)
    assert abs(u.s2 - 0.75) <= 1e-12


# restricted open-shell Hartree-Fock (oracle/dfrohf.py)

def test_rohf_closed_shell_equals_rhf(water2_sys):
    """With no open orbitals the effective Fock matrix is the closed-shell one: the RHF energy, <S^2> = 0."""
    from oracle import dfrohf
    n = water2_sys.n_electrons // 2
    ro = dfrohf.rohf(water2_sys, n, n)
    r = dfrhf.scf(water2_sys)
    assert ro.converged and abs(ro.energy - r.energy) <= 1e-9, (ro.energy, r.energy)
    assert abs(ro.s2) <= 1e-9


@pytest.fixture(scope="module")
def water2_open(water2_sys):
    """The 2-water cluster as a doublet cation (10, 9) and as a triplet (11, 9): ROHF and UHF of each."""
    import copy

    from oracle import dfrohf, dfuhf
    out = {}
    for charge, na, nb in [(1, 10, 9), (0, 11, 9)]:
        s = copy.deepcopy(water2_sys)
        s.charge = charge
        B = dfrhf.whiten(dfrhf.three_center(s), dfrhf.metric(s))
        out[(na, nb)] = (s, B, dfrohf.rohf(s, na, nb, B=B, conv_err=1e-9), dfuhf.uhf(s, na, nb, B=B))
    return out


@pytest.mark.parametrize("na,nb", [(10, 9), (11, 9)])
def test_rohf_is_a_spin_eigenfunction_above_uhf(water2_open, na, nb):
    """ROHF: <S^2> = S(S+1) exactly (the beta orbitals are a subset of the alpha ones); the UHF determinant
    has more variational freedom, so E_UHF <= E_ROHF, and UHF is spin-contaminated above S(S+1)."""
    s, B, ro, u = water2_open[(na, nb)]
    S = 0.5 * (na - nb)
    assert ro.converged and u.converged
    assert abs(ro.s2 - S * (S + 1)) <= 1e-10, ro.s2
    assert u.energy <= ro.energy + 1e-10 and ro.energy - u.energy < 0.05, (u.energy, ro.energy)
    assert u.s2 > S * (S + 1)


@pytest.mark.parametrize("na,nb", [(10, 9), (11, 9)])
def test_rohf_converged_orbitals_are_stationary(water2_open, na, nb):
    """The converged ROHF orbitals are a stationary point of the energy under every orbital rotation
    C -> C exp(k): central differences of E along random antisymmetric k vanish to O(t^2), while the same
    differences at the core-Hamiltonian orbitals match the analytic gradient (which pins the coupling
    blocks: F_b on closed-open, F_a on open-virtual, F_a + F_b on closed-virtual)."""
    from scipy.linalg import expm

    from oracle import dfrohf
    s, B, ro, _ = water2_open[(na, nb)]
    H = dfrhf.core_hamiltonian(s)
    e_nuc = dfrhf.nuclear_repulsion(s.atoms)
    X, _ = dfrhf.canonical_orthogonalizer(dfrhf.overlap(s))
    rng = np.random.default_rng(5)

    def energy(C):
        return dfrohf.uhf_functional(s, B, H, C, na, nb, e_nuc)[0]

    Ccore = X @ np.linalg.eigh(X.T @ H @ X)[1]
    nmo = Ccore.shape[1]
    t = 1e-4
    for _ in range(3):
        k = rng.normal(size=(nmo, nmo))
        k = np.triu(k, 1) - np.triu(k, 1).T
        k /= np.linalg.norm(k)
        # stationary at convergence (converged to max|e| < 1e-9: the directional derivative along a unit
        # rotation is at most |G|_F, a few 1e-8), and a minimum along k
        ep, em, e0 = energy(ro.C @ expm(t * k)), energy(ro.C @ expm(-t * k)), energy(ro.C)
        dE = (ep - em) / (2 * t)
        curv = (ep + em - 2 * e0) / t**2
        assert abs(dE) <= 1e-6 and curv > 0.0, (dE, curv)
        # analytic gradient at the core-Hamiltonian orbitals
        _, Fa, Fb, _, _ = dfrohf.uhf_functional(s, B, H, Ccore, na, nb, e_nuc)
        G = dfrohf.orbital_gradient(Ccore.T @ Fa @ Ccore, Ccore.T @ Fb @ Ccore, na, nb)
        fd = (energy(Ccore @ expm(t * k)) - energy(Ccore @ expm(-t * k))) / (2 * t)
        an = float(np.sum(np.triu(G, 1) * np.triu(k, 1)))
        assert abs(an) > 1e-2 and abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    # the effective matrix's off-diagonal class blocks are the gradient up to the factors -2, -2, -4
    _, Fa, Fb, _, _ = dfrohf.uhf_functional(s, B, H, Ccore, na, nb, e_nuc)
    Fa_mo, Fb_mo = Ccore.T @ Fa @ Ccore, Ccore.T @ Fb @ Ccore
    _, err = dfrohf.effective_fock_mo(Fa_mo, Fb_mo, na, nb)
    G = dfrohf.orbital_gradient(Fa_mo, Fb_mo, na, nb)
    cls = dfrohf.classes(nmo, na, nb)
    for a, b, f in [(0, 1, -2.0), (1, 2, -2.0), (0, 2, -4.0)]:
        blk = np.ix_(cls == a, cls == b)
        assert np.abs(G[blk] - f * err[blk]).max() <= 1e-12 * max(1.0, np.abs(G[blk]).max())


# closed-shell DF-MP2 (oracle/dfmp2.py)

def test_mp2_h2_minimal_basis_closed_form():
    """H2 with one s function per atom (the product-complete auxiliary set makes DF exact): one occupied
    (sigma_g) and one virtual (sigma_u) orbital, fixed by symmetry, so E2 = (gu|gu)^2 / (2 (e_g - e_u)) with
    e_g = h_gg + (gg|gg), e_u = h_uu + 2 (uu|gg) - (ug|ug), every integral from the s-type closed forms."""
    from oracle import dfmp2
    R, a = 1.4, 0.8
    sysh = clusters.h2_system(R, alpha=a)
    res = dfrhf.scf(sysh)
    B = dfrhf.whiten(dfrhf.three_center(sysh), dfrhf.metric(sysh))
    N = (2 * a / math.pi) ** 0.75
    s12 = N * N * (math.pi / (2 * a)) ** 1.5 * math.exp(-a / 2 * R * R)
    t11 = N * N * (a / 2) * 3 * (math.pi / (2 * a)) ** 1.5
    t12 = N * N * (a / 2) * (3 - a * R * R) * (math.pi / (2 * a)) ** 1.5 * math.exp(-a / 2 * R * R)
    F0 = lambda T: 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * erf(math.sqrt(T))
    pref = 2 * math.pi / (2 * a)
    v11 = -N * N * pref * (F0(0) + F0(2 * a * R * R))
    v12 = -N * N * pref * math.exp(-a / 2 * R * R) * 2 * F0(2 * a * (R / 2) ** 2)
    h = np.array([[t11 + v11, t12 + v12], [t12 + v12, t11 + v11]])
    cen = np.array([0.0, R])

    def ao(A, B_, C, D):
        P = (cen[A] + cen[B_]) / 2
        Q = (cen[C] + cen[D]) / 2
        K = math.exp(-a / 2 * (cen[A] - cen[B_]) ** 2) * math.exp(-a / 2 * (cen[C] - cen[D]) ** 2)
        p = q = 2 * a
        return N ** 4 * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * K * F0(p * q / (p + q) * (P - Q) ** 2)

    eri = np.array([[[[ao(A, B_, C, D) for D in range(2)] for C in range(2)] for B_ in range(2)] for A in range(2)])
    cg = np.array([1.0, 1.0]) / math.sqrt(2 * (1 + s12))
    cu = np.array([1.0, -1.0]) / math.sqrt(2 * (1 - s12))

    def mo(p, q, r, s):
        return float(np.einsum("abcd,a,b,c,d->", eri, p, q, r, s))

    e_g = cg @ h @ cg + mo(cg, cg, cg, cg)
    e_u = cu @ h @ cu + 2 * mo(cu, cu, cg, cg) - mo(cu, cg, cu, cg)
    e2_closed = mo(cg, cu, cg, cu) ** 2 / (2 * (e_g - e_u))
    e2 = dfmp2.mp2_energy(B, res.C, res.eps, 1)
    assert abs(res.eps[0] - e_g) < 1e-10 and abs(res.eps[1] - e_u) < 1e-10
    assert e2 < 0 and abs(e2 - e2_closed) < 1e-12, (e2, e2_closed)


@pytest.fixture(scope="module")
def water2_mp2(water2_sys):
    from oracle import dfmp2
    B = dfrhf.whiten(dfrhf.three_center(water2_sys), dfrhf.metric(water2_sys))
    res = dfrhf.scf(water2_sys, B=B)
    return B, res, dfmp2.mp2_energy(B, res.C, res.eps, water2_sys.nocc)


def test_mp2_closed_shell_form_equals_spin_orbital_form(water2_mp2, water2_sys):
    """The closed-shell spin summation 2 (ia|jb) - (ib|ja) against the antisymmetrised spin-orbital sum
    1/4 |<ij||ab>|^2 on the 2-water cluster: a swapped exchange index or a wrong factor fails it."""
    from oracle import dfmp2
    B, res, e2 = water2_mp2
    e2_so = dfmp2.mp2_energy_spin_orbital(B, res.C, res.eps, water2_sys.nocc)
    assert e2 < 0 and abs(e2 - e2_so) < 1e-11 * abs(e2), (e2, e2_so)


def test_mp2_size_consistent():
    """Two identical waters 3000 bohr apart: the correlation energy is twice the monomer's (MP2 is size
    consistent; the dimer's orbitals pair up into degenerate sets, and E2 does not depend on how a
    degenerate set is rotated). The remaining interaction falls off with distance (measured: 5e-8 Eh at
    100 bohr, 2.8e-9 at 300, 1.1e-10 at 3000)."""
    from oracle import dfmp2
    mono = clusters.water_cluster(1, 5)
    atoms = np.concatenate([mono.atoms, mono.atoms.copy()])
    atoms["xyz"][3:] += np.array([0.0, 0.0, 3000.0])
    dimer = clusters.make_system(atoms)
    out = []
    for s in (mono, dimer):
        B = dfrhf.whiten(dfrhf.three_center(s), dfrhf.metric(s))
        r = dfrhf.scf(s, B=B, conv_E=1e-13, conv_err=1e-11, max_iter=200)
        out.append(dfmp2.mp2_energy(B, r.C, r.eps, s.nocc))
    assert abs(out[1] - 2 * out[0]) < 1e-9, out


# density-fitting object operations, eqs. (1)-(3) (oracle/dfops.py)

def test_dfops_brute_force_tiny():
    """Every operation against nested loops over its defining sum, on tiny ragged tensors."""
    from oracle import dfops
    r = np.random.default_rng(31)
    g, nr, ns, nt, nu = 3, 2, 3, 2, 4
    I, I2, I3 = r.normal(size=(g, nr, ns)), r.normal(size=(g, nr, nt)), r.normal(size=(g, nt, nu))
    Mr, Ms, Mp = r.normal(size=(nr, nt)), r.normal(size=(ns, nt)), r.normal(size=(5, g))
    Mrs, D, G = r.normal(size=(nr, ns)), r.normal(size=g), r.normal(size=(nr * ns, nt * nu))
    out = np.zeros((g, nt, ns))
    for a in range(g):
        for t in range(nt):
            for s in range(ns):
                out[a, t, s] = sum(I[a, k, s] * Mr[k, t] for k in range(nr))
    assert np.allclose(dfops.transform_first(I, Mr), out, rtol=0, atol=1e-13)
    out = np.zeros((g, nr, nt))
    for a in range(g):
        for k in range(nr):
            for t in range(nt):
                out[a, k, t] = sum(I[a, k, s] * Ms[s, t] for s in range(ns))
    assert np.allclose(dfops.transform_second(I, Ms), out, rtol=0, atol=1e-13)
    out = np.zeros((5, nr, ns))
    for a in range(5):
        out[a] = sum(Mp[a, d] * I[d] for d in range(g))
    assert np.allclose(dfops.transform_aux(I, Mp), out, rtol=0, atol=1e-13)
    out = np.zeros((ns, nt))
    for s in range(ns):
        for t in range(nt):
            out[s, t] = sum(I[a, k, s] * I2[a, k, t] for a in range(g) for k in range(nr))
    assert np.allclose(dfops.contract_first(I, I2), out, rtol=0, atol=1e-13)
    out = np.zeros((nr * ns, nt * nu))
    for k in range(nr):
        for s in range(ns):
            for t in range(nt):
                for u in range(nu):
                    out[k * ns + s, t * nu + u] = sum(I[a, k, s] * I3[a, t, u] for a in range(g))
    assert np.allclose(dfops.contract_aux(I, I3), out, rtol=0, atol=1e-13)
    I4 = r.normal(size=(4, nr, ns))
    out = np.array([[np.sum(I[a] * I4[b]) for b in range(4)] for a in range(g)])
    assert np.allclose(dfops.contract_pairs(I, I4), out, rtol=0, atol=1e-13)
    assert np.allclose(dfops.density_fit(I, Mrs), [np.sum(I[a] * Mrs) for a in range(g)], rtol=0, atol=1e-13)
    assert np.allclose(dfops.density_back(I, D), sum(D[a] * I[a] for a in range(g)), rtol=0, atol=1e-13)
    out = np.zeros((g, nt, nu))
    for a in range(g):
        for t in range(nt):
            for u in range(nu):
                out[a, t, u] = sum(I[a, k, s] * G[k * ns + s, t * nu + u] for k in range(nr) for s in range(ns))
    assert np.allclose(dfops.apply_four_index(I, G, nt, nu), out, rtol=0, atol=1e-13)


def test_dfops_give_exact_coulomb_and_exchange_for_h2():
    """With the product-complete auxiliary set of H2, J = density_back(B, density_fit(B, D)) and
    K = contract_first(Y, Y) with Y = transform_first(B, C_occ) equal the four-index J and K."""
    from oracle import dfops
    sysh = clusters.h2_system(1.4, alpha=0.8)
    B = dfrhf.whiten(dfrhf.three_center(sysh), dfrhf.metric(sysh))
    eri = dfrhf.four_center(sysh)
    C = np.linalg.qr(np.random.default_rng(4).normal(size=(2, 1)))[0]
    D = 2 * C @ C.T
    J = dfops.density_back(B, dfops.density_fit(B, D))
    Y = dfops.transform_first(B, C)
    K = dfops.contract_first(Y, Y)
    assert np.abs(J - dfrhf.conv_J(eri, D)).max() < 1e-10
    assert np.abs(K - dfrhf.conv_K(eri, C)).max() < 1e-10


def test_dfops_identities():
    """Adjointness of the two density contractions; orthogonal transformations undone by their
    transposes; G-application of a two-object product equals the auxiliary transformation by the pair
    contraction: sum_rs I_g,rs (sum_h I2_h,rs I3_h,tu) = sum_h (sum_rs I_g,rs I2_h,rs) I3_h,tu."""
    from oracle import dfops
    r = np.random.default_rng(32)
    g, nr, ns, nt, nu = 7, 5, 6, 3, 4
    I, I2, I3 = r.normal(size=(g, nr, ns)), r.normal(size=(g + 2, nr, ns)), r.normal(size=(g + 2, nt, nu))
    M, D = r.normal(size=(nr, ns)), r.normal(size=g)
    assert abs(dfops.density_fit(I, M) @ D - np.sum(M * dfops.density_back(I, D))) < 1e-12
    Q = np.linalg.qr(r.normal(size=(nr, nr)))[0]
    assert np.abs(dfops.transform_first(dfops.transform_first(I, Q), Q.T) - I).max() < 1e-13
    Q2 = np.linalg.qr(r.normal(size=(ns, ns)))[0]
    assert np.abs(dfops.transform_second(dfops.transform_second(I, Q2), Q2.T) - I).max() < 1e-13
    lhs = dfops.apply_four_index(I, dfops.contract_aux(I2, I3), nt, nu)
    rhs = dfops.transform_aux(I3, dfops.contract_pairs(I, I2))
    assert np.abs(lhs - rhs).max() < 1e-12


# nuclear gradient of DF-RHF (oracle/dfgrad.py)

@pytest.fixture(scope="module")
def water1_grad():
    from oracle import dfgrad
    s = clusters.water_cluster(1, 3)
    B = dfrhf.whiten(dfrhf.three_center(s), dfrhf.metric(s))
    res = dfrhf.scf(s, B=B, conv_E=1e-13, conv_err=1e-10, max_iter=200)
    return s, res, dfgrad.gradient(s, res)


def test_gradient_matches_energy_differences(water1_grad):
    """Against fourth-order central differences of the converged SCF energy along every coordinate of a
    water (each displaced geometry converged from scratch): a dropped orbital-constraint term -tr(W S^x), a
    sign slip on the metric-derivative terms or a missing nuclear-repulsion term all fail it."""
    from oracle import dfgrad
    s, res, g = water1_grad
    h = 2e-3

    def energy(a, d, step):
        sd = dfgrad.displaced(s, a, d, step)
        return dfrhf.scf(sd, conv_E=1e-13, conv_err=1e-10, max_iter=200).energy

    fd = np.zeros_like(g)
    for a in range(len(s.atoms)):
        for d in range(3):
            e = [energy(a, d, k * h) for k in (-2, -1, 1, 2)]
            fd[a, d] = (8 * (e[2] - e[1]) - (e[3] - e[0])) / (12 * h)
    assert np.abs(g).max() > 1e-3
    assert np.abs(g - fd).max() < 5e-8, np.abs(g - fd).max()


def test_gradient_translation_and_rotation_invariance(water1_grad):
    """The energy does not change under rigid translations and rotations: the gradient sums to zero and
    exerts no torque."""
    s, res, g = water1_grad
    R = np.asarray(s.atoms["xyz"], dtype=np.float64)
    assert np.abs(g.sum(axis=0)).max() < 1e-8
    assert np.abs(np.cross(R, g).sum(axis=0)).max() < 1e-8
