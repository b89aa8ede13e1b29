"""Pins of the FP64 CPU oracle against things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle -- a wrong sign of
a field, a transposed C gamma5, a wrong permutation sign, a wrong split of the
source tensor, a shift in the wrong direction -- fails at least one of them:

* the worked example the paper prints (Eq. (2.7), 370 vs 3456);
* the textbook determinant form of the Wick contraction (tests/wick_brute.py);
* the naive permutation sum of Eq. (2.4) without effective blocks;
* exact symmetries: colour gauge invariance, u<->d relabelling, SU(3) flavour,
  B1 <-> B2 exchange, translations, site-constant propagators.
"""

import itertools
import os

import numpy as np
import pytest

import nbs_inputs as I
from oracle import nbs_oracle as O
from wick_brute import correlator_brute, dirac_cg5

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def props3(seed, L, t=0):
    return {f: I.propagator(seed, f, L, t) for f in "uds"}


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --- conventions ---------------------------------------------------------------

def test_cg5_is_c_gamma5_of_dirac_matrices():
    assert np.allclose(dirac_cg5(), O.CG5, atol=1e-15)
    assert np.allclose(O.CG5, -O.CG5.T)
    assert np.count_nonzero(O.CG5) == 4   # N_alpha = 4 of Sec. 2


def test_perm_sign_is_determinant_of_permutation_matrix():
    for p in itertools.permutations(range(5)):
        assert O.perm_sign(p) == round(np.linalg.det(np.eye(5)[list(p)]))


def test_levi_civita():
    assert O.EPS[0, 1, 2] == 1 and O.EPS[1, 0, 2] == -1 and O.EPS[2, 0, 1] == 1
    assert np.count_nonzero(O.EPS) == 6


# --- the worked example of Eq. (2.7) -------------------------------------------

def _golden_terms():
    rows, scalars = [], {}
    with open(os.path.join(GOLDEN, "worked_example_pLambda_pXu.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if "|" in line:
                _, idx, size, h1, h2 = [s.strip() for s in line.split("|")]
                norm = lambda s: frozenset() if s == "-" else frozenset(s.split())
                rows.append((norm(idx), int(size), norm(h1), norm(h2)))
            else:
                k, v = line.split()
                scalars[k] = int(v)
    return rows, scalars


def _paper_name(letter):
    if letter in O._SPIN:
        return "a%d" % (O._SPIN.index(letter) + 1)
    if letter in O._COL:
        return "c%d" % (O._COL.index(letter) + 1)
    return {"p": "a3", "q": "a4"}[letter]


def test_worked_example_pLambda_pXu_matches_paper():
    rows, scalars = _golden_terms()
    terms = O.topologies("p", "Lambda", "p", "Xu")
    got = sorted(
        (frozenset(_paper_name(c) for c in t.xi), O.xi_size(t),
         frozenset(_paper_name(c) for c in t.held1), frozenset(_paper_name(c) for c in t.held2))
        for t in terms)
    # held spins are named by the source slot they sit on (a3 = slot 3, a4 = slot 6 in the paper)
    fix = lambda s: frozenset({"a3": "a3", "a4": "a4"}[x] for x in s)
    want = sorted((r[0], r[1], fix(r[2]), fix(r[3])) for r in rows)
    assert [g[:2] for g in got] == [w[:2] for w in want]
    assert got == want
    assert sum(O.xi_size(t) for t in terms) == scalars["total_effective_iterations"] == 370
    # (N_c! N_alpha)^B per topology of Eq. (2.4): 576 source-tensor terms each
    assert len(terms) * (6 * 4) ** 2 == scalars["naive_iterations"] == 3456
    # N_u! N_d! N_s! flavour-respecting permutations per sink monomial pair
    for _, m in O.FIELDS["Lambda"]:
        assert len(O.wick_permutations("udu" + m, "udu" + "dsu")) == 6 * 2 * 1


def test_pn_topology_count():
    terms = O.topologies("p", "n", "p", "n")
    assert len(terms) == 9
    assert sum(O.xi_size(t) for t in terms) == 586


# --- the determinant definition ------------------------------------------------

CHANNELS_L1 = [("p", "n", "p", "n"), ("p", "Lambda", "p", "Xu"), ("Sigma+", "Sigma-", "p", "Xi-"),
               ("n", "Sigma+", "p", "Sigma0"), ("Xi0", "Xi-", "Xi0", "Xi-")]


@pytest.mark.parametrize("channel", CHANNELS_L1)
def test_oracle_equals_determinant_wick_L1(channel):
    props = props3(11, 1)
    F = O.correlator(channel, props, 1)
    for spins in [(0, 1, 0, 1), (2, 3, 1, 0), (3, 0, 1, 1)]:
        b = correlator_brute(channel, props, 1, (0, 0, 0), spins)
        assert abs(F[spins][0] - b) <= 1e-12 * abs(b)


@pytest.mark.parametrize("block", [(1, 0), (0, 1), (1, 1)])
def test_oracle_other_source_spins_equal_determinant_wick_L1(block):
    """Source spins outside the upper components (alpha3, alpha4 in {2 o3, 2 o3 + 1} x {2 o4, 2 o4 + 1})
    against the determinant definition, which takes any source spins."""
    props = props3(13, 1)
    for channel in CHANNELS_L1[:3]:
        F = O.correlator(channel, props, 1, block=block)
        for a1, a2, j3, j4 in [(0, 1, 0, 1), (2, 3, 1, 0), (3, 0, 1, 1)]:
            b = correlator_brute(channel, props, 1, (0, 0, 0), (a1, a2, 2 * block[0] + j3, 2 * block[1] + j4))
            assert abs(F[a1, a2, j3, j4][0] - b) <= 1e-12 * abs(b), (channel, block)


def test_oracle_equals_determinant_wick_L2_shift():
    props = props3(12, 2)
    r = (1, 0, 1)
    F = O.correlator(("p", "n", "p", "n"), props, 2, [r])
    spins = (1, 2, 0, 1)
    b = correlator_brute(("p", "n", "p", "n"), props, 2, r, spins)
    assert abs(F[spins][0] - b) <= 1e-12 * abs(b)


# --- naive Eq. (2.4): permutations without effective blocks ---------------------

def naive_eq24(channel, props, L):
    """sum_X sum_P sigma_P sum_{xi'} W(xi') N1(X+r; xi'_P1..3) N2(X; xi'_P4..6), every r."""
    B1, B2, B3, B4 = channel
    V = L ** 3
    W = []
    for c in itertools.product(range(3), repeat=6):
        e = O.EPS[c[0], c[1], c[2]] * O.EPS[c[3], c[4], c[5]]
        if e == 0:
            continue
        for s in itertools.product(range(4), repeat=6):
            if s[2] > 1 or s[5] > 1:
                continue
            g = O.CG5[s[0], s[1]] * O.CG5[s[3], s[4]]
            if g:
                W.append((e * g, c, s))
    F = np.zeros((V, 4, 4, 2, 2), dtype=np.complex128)
    blocks = {}
    for (c1, m1), (c2, m2), (c3, m3), (c4, m4) in itertools.product(
            O.FIELDS[B1], O.FIELDS[B2], O.FIELDS[B3], O.FIELDS[B4]):
        for m in (m1, m2):
            if m not in blocks:
                blocks[m] = O.normal_block(props[m[0]], props[m[1]], props[m[2]])
        N1, N2 = blocks[m1], blocks[m2]
        for P, sgn in O.wick_permutations(m1 + m2, m3 + m4):
            for w, c, s in W:
                a = N1[:, :, s[P[0]], c[P[0]], s[P[1]], c[P[1]], s[P[2]], c[P[2]]]   # [V, 4]
                b = N2[:, :, s[P[3]], c[P[3]], s[P[4]], c[P[4]], s[P[5]], c[P[5]]]
                coef = c1 * c2 * c3 * c4 * sgn * w
                for r in range(V):
                    idx = O.shifted_sites(L, (r % L, (r // L) % L, r // (L * L)))
                    F[r, :, :, s[2], s[5]] += coef * a[idx].T @ b
    return np.moveaxis(F, 0, -1)


@pytest.mark.parametrize("channel", [("p", "n", "p", "n"), ("Lambda", "Sigma0", "p", "Xi-")])
def test_effective_blocks_equal_naive_permutation_sum_L2(channel):
    props = props3(13, 2)
    F = O.correlator(channel, props, 2)
    Fn = naive_eq24(channel, props, 2)
    assert rel(F, Fn) < 1e-13


# --- exact symmetries ----------------------------------------------------------

SYM_CHANNELS = [("p", "n", "p", "n"), ("Lambda", "Lambda", "Sigma0", "Sigma0"), ("p", "Xi-", "Sigma+", "Sigma-"),
                ("Sigma0", "Xi0", "Lambda", "Xi0")]


@pytest.mark.parametrize("channel", SYM_CHANNELS)
def test_sink_colour_gauge_invariance(channel):
    L = 2
    props = props3(21, L)
    U = I.haar_su3(99, L)
    assert np.allclose(np.linalg.det(U), 1.0)
    assert np.allclose(np.einsum("xab,xcb->xac", U, U.conj()), np.eye(3)[None])
    rot = {f: I.rotate_sink_colour(S, U) for f, S in props.items()}
    F, Fr = O.correlator(channel, props, L), O.correlator(channel, rot, L)
    assert rel(Fr, F) < 1e-12


def test_global_source_colour_invariance():
    L = 2
    props = props3(22, L)
    U = I.haar_su3(5, 1)[0]
    rot = {f: I.rotate_source_colour(S, U) for f, S in props.items()}
    for ch in SYM_CHANNELS[:2]:
        assert rel(O.correlator(ch, rot, L), O.correlator(ch, props, L)) < 1e-12


def test_colour_rotation_is_not_trivial():
    """A U(3) phase (det != 1) must change a baryon correlator: the checks above are not vacuous."""
    L = 1
    props = props3(23, L)
    U = np.exp(0.3j) * np.eye(3)[None]
    rot = {f: I.rotate_sink_colour(S, U) for f, S in props.items()}
    F, Fr = O.correlator(("p", "n", "p", "n"), props, L), O.correlator(("p", "n", "p", "n"), rot, L)
    assert rel(Fr, F) > 0.1


#: operator identity under u <-> d: field -> (image, sign), from Eqs. (2.2)-(2.3)
UD_IMAGE = {"p": ("n", 1), "n": ("p", 1), "Sigma+": ("Sigma-", 1), "Sigma-": ("Sigma+", 1),
            "Xi0": ("Xi-", -1), "Xi-": ("Xi0", -1), "Xu": ("Xd", -1), "Xd": ("Xu", -1),
            "Xs": ("Xs", -1), "Lambda": ("Lambda", -1), "Sigma0": ("Sigma0", 1)}


@pytest.mark.parametrize("channel", [("p", "n", "p", "n"), ("p", "Lambda", "n", "Sigma+"),
                                     ("Xi0", "Xi-", "Xi0", "Xi-"), ("Lambda", "Sigma0", "Sigma+", "Sigma-")])
def test_u_d_relabelling(channel):
    L = 2
    props = props3(31, L)
    swapped = {"u": props["d"], "d": props["u"], "s": props["s"]}
    img = [UD_IMAGE[b] for b in channel]
    sign = np.prod([s for _, s in img])
    F = O.correlator(channel, props, L)
    Fi = O.correlator(tuple(b for b, _ in img), swapped, L)
    assert rel(F, sign * Fi) < 1e-12


def test_isospin_pp_equals_nn():
    L = 2
    S = I.propagator(32, "u", L, 0)
    props = {"u": S, "d": S, "s": I.propagator(32, "s", L, 0)}
    Fpp = O.correlator(("p", "p", "p", "p"), props, L)
    Fnn = O.correlator(("n", "n", "n", "n"), props, L)
    assert np.linalg.norm(Fpp) > 0
    assert rel(Fnn, Fpp) < 1e-12


def test_su3_flavour_symmetric_point():
    L = 1
    S = I.propagator(33, "u", L, 0)
    props = {"u": S, "d": S, "s": S}
    Fpp = O.correlator(("p", "p", "p", "p"), props, L)
    for ch in [("Sigma+", "Sigma+", "Sigma+", "Sigma+"), ("Xi0", "Xi0", "Xi0", "Xi0"), ("n", "n", "n", "n")]:
        assert rel(O.correlator(ch, props, L), Fpp) < 1e-12


@pytest.mark.parametrize("channel", [("p", "Lambda", "p", "Lambda"), ("Sigma+", "Xi-", "Lambda", "Xi0")])
def test_exchange_relation(channel):
    """Baryon operators anticommute: F^{B1B2}_{a1a2}(r) = -F^{B2B1}_{a2a1}(-r)."""
    L = 2
    props = props3(41, L)
    B1, B2, B3, B4 = channel
    F = O.correlator(channel, props, L)
    G = O.correlator((B2, B1, B3, B4), props, L)
    idx = np.array([((-(r % L)) % L) + L * ((-((r // L) % L)) % L) + L * L * ((-(r // (L * L))) % L)
                    for r in range(L ** 3)])
    assert rel(F, -np.transpose(G, (1, 0, 2, 3, 4))[..., idx]) < 1e-12
    # source swap: Jbar(B3 B4)_{a3 a4} = -Jbar(B4 B3)_{a4 a3}
    H = O.correlator((B1, B2, B4, B3), props, L)
    assert rel(F, -np.transpose(H, (0, 1, 3, 2, 4))) < 1e-12


def test_translation_invariance():
    L = 3
    props = props3(51, L)
    a = (1, 2, 0)
    moved = {f: I.translate(S, L, a) for f, S in props.items()}
    ch = ("p", "Sigma0", "n", "Sigma+")
    assert rel(O.correlator(ch, moved, L), O.correlator(ch, props, L)) < 1e-12


def test_site_constant_propagators():
    L = 2
    one = props3(52, 1)
    const = {f: np.repeat(S, L ** 3, axis=0) for f, S in one.items()}
    ch = ("Lambda", "Lambda", "p", "Xi-")
    F1 = O.correlator(ch, one, 1)[..., 0]
    F = O.correlator(ch, const, L)
    assert rel(F, (L ** 3) * F1[..., None] * np.ones(L ** 3)) < 1e-12


def test_zero_momentum_is_sum_over_r():
    L = 2
    props = props3(53, L)
    ch = ("Sigma0", "Sigma0", "Lambda", "Sigma0")
    assert rel(O.zero_momentum(ch, props, L), O.correlator(ch, props, L).sum(-1)) < 1e-13


def test_momentum_projection_is_dft_of_direct_sum():
    """The momentum projection (correlation theorem of Eq. (2.6) on phase-weighted site sums of the normal
    blocks, accumulated in chunks with a ragged last chunk) against the explicit DFT of the direct O(V^2)
    sum, for distinct u, d, s propagators and several momenta; n = 0 is the zero-momentum sum."""
    L = 3
    props = props3(61, L)
    ns = [(0, 0, 0), (1, 0, 0), (0, 2, 1), (1, 2, 2)]
    sums = O.PhaseSums(props, L, ns, chunk=10)
    s = np.arange(L ** 3)
    x, y, z = s % L, (s // L) % L, s // (L * L)
    for ch in [("p", "n", "p", "n"), ("Lambda", "Sigma0", "Sigma+", "Sigma-"), ("Xi0", "Xi-", "Sigma0", "Xi0")]:
        F = O.correlator(ch, props, L)
        got = O.momentum_projection(ch, sums, ns)
        for k, n in enumerate(ns):
            want = F @ np.exp(-2j * np.pi * (n[0] * x + n[1] * y + n[2] * z) / L)
            assert rel(got[k], want) < 1e-13, (ch, n)
        assert rel(got[0], O.zero_momentum(ch, props, L)) < 1e-13


def test_momentum_projection_other_source_spins():
    L = 2
    props = props3(62, L)
    sums = O.PhaseSums(props, L, [(1, 0, 1)], chunk=3)
    s = np.arange(L ** 3)
    ph = np.exp(-2j * np.pi * ((s % L) + (s // (L * L))) / L)
    ch = ("p", "Sigma0", "n", "Sigma+")
    for block in [(1, 0), (1, 1)]:
        want = O.correlator(ch, props, L, block=block) @ ph
        assert rel(O.momentum_projection(ch, sums, [(1, 0, 1)], block=block)[0], want) < 1e-13


def test_channel_table_and_the_four_that_vanish():
    """52 of the 56 sector pairs; the four left out are identically zero when u = d (the oracle computes
    them directly, never identifying u with d), the 52 kept are not, and with u != d none vanishes."""
    table, all56 = O.channel_table(), O.channel_table_56()
    assert len(all56) == 56 and len(set(all56)) == 56
    assert len(table) == 52 and table[0] == ("p", "n", "p", "n") and table[-1] == ("Xi0", "Xi-", "Xi0", "Xi-")
    dropped = [ch for ch in all56 if ch not in table]
    assert sorted(dropped) == sorted([("Lambda", "Lambda", "Lambda", "Sigma0"), ("Lambda", "Sigma0", "Lambda", "Lambda"),
                                      ("Lambda", "Sigma0", "Sigma0", "Sigma0"), ("Sigma0", "Sigma0", "Lambda", "Sigma0")])
    Sl, Ss = I.propagator(63, "l", 1, 0), I.propagator(63, "s", 1, 0)
    equal = {"u": Sl, "d": Sl.copy(), "s": Ss}
    unequal = props3(64, 1)
    for ch in all56:
        if "Lambda" not in ch and "Sigma0" not in ch:
            continue
        F = O.correlator(ch, equal, 1)
        scale = np.linalg.norm(O.correlator(("Lambda", "Lambda", "Lambda", "Lambda"), equal, 1))
        if ch in dropped:
            assert np.linalg.norm(F) < 1e-13 * scale, ch
            assert np.linalg.norm(O.correlator(ch, unequal, 1)) > 1e-3 * scale, ch
        else:
            assert np.linalg.norm(F) > 1e-3 * scale, ch


def test_direct_sum_paths_agree():
    rng = np.random.default_rng(0)
    L, m, n, K = 3, 4, 8, 5
    E1 = rng.normal(size=(L ** 3, m, K)) + 1j * rng.normal(size=(L ** 3, m, K))
    E2 = rng.normal(size=(L ** 3, n, K)) + 1j * rng.normal(size=(L ** 3, n, K))
    rs = [(1, 0, 2), (2, 2, 2), (0, 0, 0)]
    a = O.direct_sum(E1, E2, L, rs)
    want = np.zeros((len(rs), m, n), dtype=complex)
    for ir, (rx, ry, rz) in enumerate(rs):
        for z, y, x in itertools.product(range(L), repeat=3):
            Y = (x + rx) % L + L * ((y + ry) % L) + L * L * ((z + rz) % L)
            X = x + L * (y + L * z)
            want[ir] += E1[Y] @ E2[X].T
    assert rel(a, want) < 1e-13
    b = O.direct_sum(E1, E2, L, rs, table_bytes=0)   # the per-r branch
    assert rel(b, want) < 1e-13


# --- the potential stencil against closed forms ------------------------------------

def test_potential_stencil_closed_forms():
    """R = exp(i k.r - E t): the lattice Laplacian multiplies by -sum_i 2 (1 - cos k_i), the central first
    difference by -sinh(E), the second difference by 2 (cosh(E) - 1); each coefficient separately."""
    L = 6
    k = 2 * np.pi * np.array([1, 2, 5]) / L
    E = 0.37
    x = np.arange(L ** 3) % L
    y = (np.arange(L ** 3) // L) % L
    z = np.arange(L ** 3) // (L * L)
    phase = np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))
    R = [phase * np.exp(-E * t) for t in (2, 3, 4)]
    lam = -2.0 * np.sum(1.0 - np.cos(k))
    for (a, b, c), want in [((0, 0, 1), lam), ((0, 1, 0), -np.sinh(E)), ((1, 0, 0), 2 * (np.cosh(E) - 1))]:
        K, P = O.potential_stencil(R[0], R[1], R[2], L, a, b, c)
        assert np.allclose(K, want * R[1], rtol=0, atol=1e-12)
        assert np.allclose(P, want, rtol=0, atol=1e-12)
    # a constant field has no Laplacian; linear combination of the three
    Rc = np.full(L ** 3, 2.0 + 1.0j)
    K, _ = O.potential_stencil(0.5 * Rc, Rc, 2.0 * Rc, L, 0.3, -1.0, 0.7)
    assert np.allclose(K, (0.3 * (2.0 - 2.0 + 0.5) - 1.0 * 0.5 * 1.5) * Rc)
