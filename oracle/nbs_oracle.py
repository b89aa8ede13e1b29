"""Plain FP64 CPU oracle for the octet-octet NBS four-point correlators.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py use it.  It shares no code with the
CUDA library (paper_1604_07983_gb300) and imports nothing from it.

What it computes (Nemura, LATTICE 2015, arXiv:1604.07983):

  F^{<B1 B2 B3bar B4bar>}_{a1 a2, a3 a4}(r) = sum_X < B1_a1(X+r) B2_a2(X) Jbar_{a3 a4} >   (Sec. 2, first equation)

evaluated the way Sec. 2 writes it:
  * interpolating fields expanded into flavour monomials, Eqs. (2.2)-(2.3);
  * normal baryon blocks per site by explicit epsilon / C gamma5 sums,
    Eq. (2.5) (the kernel equation of Sec. 4 (i));
  * the Wick sum over permutations P of the six source slots with sign
    sigma_P and the source tensor eps eps (Cg5)(Cg5) delta delta, Eq. (2.4);
  * the permutations grouped by which source slots feed B1 (the topologies of
    Eq. (2.7)), with the source tensor absorbed into effective blocks so that
    only the shared source indices xi~ connect B1 and B2 (Sec. 2 after
    Eq. (2.6); Sec. 4 (ii));
  * the spatial sum over X done DIRECTLY, O(V^2), instead of by the FFT of
    Eq. (2.6).

Conventions (readings where the paper is silent):
  * Dirac representation, C = gamma4 gamma2; C gamma5 is the real
    antisymmetric matrix CG5 below (4 non-zeros, the paper's N_alpha = 4).
  * Source spins a3, a4 projected to the upper Dirac components {0, 1}.
  * The source operator is the mirror of the sink: qbar6 ... qbar1, so the
    direct pairing has sign +1 and sigma_P = sign(P).
  * Propagator S_f[x][i][j], i = 3*alpha + a (sink), j = 3*alpha' + a' (source).
  * X + r is taken modulo L componentwise; site = x + L*(y + L*z).
  * Every flavour uses its own propagator: u and d are never identified
    here, so the isospin identities tested against this oracle are not built in.
"""

from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# --- Dirac / colour tensors -------------------------------------------------

#: C gamma5 in the Dirac representation (reading of Eq. (2.2)).
CG5 = np.array(
    [[0, 1, 0, 0],
     [-1, 0, 0, 0],
     [0, 0, 0, 1],
     [0, 0, -1, 0]], dtype=np.float64)

#: Levi-Civita symbol eps_abc.
EPS = np.zeros((3, 3, 3))
for _a, _b, _c in itertools.permutations(range(3)):
    EPS[_a, _b, _c] = np.linalg.det(np.eye(3)[[_a, _b, _c]])

#: delta(alpha', alpha) restricted to the projected source spins alpha in {0,1}.
PROJ = np.zeros((4, 2))
PROJ[0, 0] = PROJ[1, 1] = 1.0


def projector(offset: int) -> np.ndarray:
    """delta(alpha', alpha) for the source spin pair alpha in {2 offset, 2 offset + 1} (offset 0: PROJ)."""
    P = np.zeros((4, 2))
    P[2 * offset, 0] = P[2 * offset + 1, 1] = 1.0
    return P

# --- interpolating fields, Eqs. (2.2) and (2.3) ------------------------------

_R6 = 1.0 / math.sqrt(6.0)
_R2 = 1.0 / math.sqrt(2.0)

#: field -> list of (coefficient, (q1, q2, q3)) for eps_abc (q1_a Cg5 q2_b) q3_c.
FIELDS: dict[str, list[tuple[float, str]]] = {
    "p": [(+1.0, "udu")],
    "n": [(-1.0, "udd")],
    "Sigma+": [(-1.0, "usu")],
    "Sigma-": [(-1.0, "dsd")],
    "Xi0": [(+1.0, "uss")],
    "Xi-": [(-1.0, "dss")],
    "Xu": [(1.0, "dsu")],
    "Xd": [(1.0, "sud")],
    "Xs": [(1.0, "uds")],
    "Lambda": [(_R6, "dsu"), (_R6, "sud"), (-2.0 * _R6, "uds")],
    "Sigma0": [(_R2, "dsu"), (-_R2, "sud")],
}


def perm_sign(p) -> int:
    """Sign of a permutation given as a sequence of distinct integers."""
    p = list(p)
    inv = sum(1 for i in range(len(p)) for j in range(i + 1, len(p)) if p[i] > p[j])
    return -1 if inv % 2 else 1


# --- normal baryon blocks, Eq. (2.5) -----------------------------------------

def normal_block(S1: np.ndarray, S2: np.ndarray, S3: np.ndarray) -> np.ndarray:
    """[B_alpha^(0)](x; xi1', xi2', xi3') for sink quarks q1 q2 q3 with propagators S1 S2 S3.

    N[x, alpha, s1, c1, s2, c2, s3, c3] =
        sum_abc eps_abc sum_{beta gamma} (Cg5)_{beta gamma}
            S1[x](beta,a; s1,c1) S2[x](gamma,b; s2,c2) S3[x](alpha,c; s3,c3)
    where (s_k, c_k) is the source spin and colour paired with sink quark k.
    """
    V = S1.shape[0]
    r = lambda S: S.reshape(V, 4, 3, 4, 3)  # [x, sink spin, sink colour, src spin, src colour]
    return np.einsum("abc,BG,xBaPQ,xGbRS,xAcTU->xAPQRSTU",
                     EPS, CG5, r(S1), r(S2), r(S3), optimize=True)


# --- Wick permutations and topologies, Eqs. (2.4), (2.7) ---------------------

def wick_permutations(sink: str, src: str):
    """All P in S6 with flavour(sink quark k) == flavour(source slot P(k)), with sign(P)."""
    out = []
    for P in itertools.permutations(range(6)):
        if all(sink[k] == src[P[k]] for k in range(6)):
            out.append((P, perm_sign(P)))
    return out


@dataclass
class Term:
    """One topology of Eq. (2.7): fixed source monomials and the source slots feeding B1."""
    c34: float                   # product of the source monomial coefficients
    sign0: int                   # sign of the reference permutation (sorted S, sorted complement)
    S: tuple                     # source slots (0..5) paired with B1's quarks, sorted
    Sc: tuple                    # the complement, paired with B2's quarks
    side1: list = field(default_factory=list)   # (coef, monomial, slot of each sink quark)
    side2: list = field(default_factory=list)
    xi: tuple = ()               # shared index letters, canonical order
    held1: str = ""              # projected source spins carried by the B1 block
    held2: str = ""
    factors1: list = field(default_factory=list)  # (einsum letters, tensor)
    factors2: list = field(default_factory=list)


_SPIN = "ABCDEF"     # einsum letter of the source spin of slot k
_COL = "GHIJKL"      # einsum letter of the source colour of slot k
_OUT = "pq"          # projected source spins alpha3 (slot 2), alpha4 (slot 5)


def _letter_size(ch: str) -> int:
    return 4 if ch in _SPIN else 3


def source_factors(block=(0, 0)):
    """The source tensor of Eq. (2.4) as (baryon, letters, tensor) factors.

    eps_{c1 c2 c3} eps_{c4 c5 c6} (Cg5)_{a1 a2} (Cg5)_{a4 a5} delta_{a3 alpha3} delta_{a6 alpha4}
    with alpha3 in {2 block[0], 2 block[0] + 1} and alpha4 in {2 block[1], 2 block[1] + 1}
    (block (0, 0): the upper Dirac components).
    """
    fs = []
    for b in range(2):
        k = 3 * b
        fs.append((b, "eps", _COL[k] + _COL[k + 1] + _COL[k + 2], EPS))
        fs.append((b, "cg5", _SPIN[k] + _SPIN[k + 1], CG5))
        fs.append((b, "proj", _SPIN[k + 2] + _OUT[b], projector(block[b])))
    return fs


def _factor_slots(letters: str):
    out = []
    for ch in letters:
        if ch in _SPIN:
            out.append(_SPIN.index(ch))
        elif ch in _COL:
            out.append(_COL.index(ch))
    return out


def topologies(B1: str, B2: str, B3: str, B4: str, block=(0, 0)) -> list[Term]:
    """Group the Wick permutations of Eq. (2.4) into the effective-block terms of Eq. (2.7).

    For every pair of source monomials and every set S of three source slots,
    the permutations with P({1,2,3}) = S factor as sign(P) = sign(P0_S) *
    sign(tau1) * sign(tau2), tau1 (tau2) acting inside B1 (B2).  The source
    tensor is split between the two blocks: each source baryon's epsilon and
    C gamma5 go to the block that holds at least two of its three slots, and
    its projector goes with the slot it acts on.  The indices of one block's
    slots that appear in a factor of the other block are the shared indices
    xi~ (the index sets listed in Sec. 4 (ii)).
    """
    terms = []
    for (c3, m3), (c4, m4) in itertools.product(FIELDS[B3], FIELDS[B4]):
        src = m3 + m4
        groups: dict[tuple, Term] = {}
        for (c1, m1), (c2, m2) in itertools.product(FIELDS[B1], FIELDS[B2]):
            for P, sgn in wick_permutations(m1 + m2, src):
                S = tuple(sorted(P[:3]))
                Sc = tuple(sorted(P[3:]))
                P0 = S + Sc
                tau1 = [S.index(P[k]) for k in range(3)]
                tau2 = [Sc.index(P[k]) for k in range(3, 6)]
                s0 = perm_sign(P0)
                assert sgn == s0 * perm_sign(tau1) * perm_sign(tau2)
                t = groups.get(S)
                if t is None:
                    t = groups[S] = Term(c34=c3 * c4, sign0=s0, S=S, Sc=Sc)
                e1 = (c1 * perm_sign(tau1), m1, tuple(P[:3]))
                e2 = (c2 * perm_sign(tau2), m2, tuple(P[3:]))
                if e1 not in t.side1:
                    t.side1.append(e1)
                if e2 not in t.side2:
                    t.side2.append(e2)
        for S, t in sorted(groups.items()):
            _assign_factors(t, block)
            terms.append(t)
    return terms


def _assign_factors(t: Term, block=(0, 0)) -> None:
    in1 = set(t.S)
    xi = set()
    for b, kind, letters, tensor in source_factors(block):
        slots = _factor_slots(letters)
        if kind == "proj":
            side1 = slots[0] in in1
        else:
            side1 = sum(1 for k in range(3 * b, 3 * b + 3) if k in in1) >= 2
        (t.factors1 if side1 else t.factors2).append((letters, tensor))
        for ch in letters:
            if ch in _OUT:
                if side1:
                    t.held1 += ch
                else:
                    t.held2 += ch
                continue
            k = _factor_slots(ch)[0]
            if (k in in1) != side1:
                xi.add(ch)
    t.xi = tuple(sorted(xi))


def xi_size(t: Term) -> int:
    return int(np.prod([_letter_size(ch) for ch in t.xi])) if t.xi else 1


# --- effective blocks and the correlator ------------------------------------

class _Blocks:
    """Normal blocks per sink monomial, computed on first use."""

    def __init__(self, props: dict):
        self.props = props
        self.cache: dict[str, np.ndarray] = {}

    def __call__(self, mono: str) -> np.ndarray:
        if mono not in self.cache:
            p = self.props
            self.cache[mono] = normal_block(p[mono[0]], p[mono[1]], p[mono[2]])
        return self.cache[mono]


def effective_block(t: Term, side: int, blocks: _Blocks) -> np.ndarray:
    """Effective baryon block of one side of a topology, per site.

    Returns E[x, alpha, held..., xi~...] flattened to [V, 4*2^len(held), |xi~|]:
    sum over the side's monomials and intra-block assignments of
    coef * sign(tau) * (normal block contracted with the side's source factors).
    """
    entries = t.side1 if side == 1 else t.side2
    factors = t.factors1 if side == 1 else t.factors2
    held = t.held1 if side == 1 else t.held2
    out = "xz" + held + "".join(t.xi)
    E = None
    for coef, mono, slots in entries:
        N = blocks(mono)
        spec = "xz" + "".join(_SPIN[k] + _COL[k] for k in slots)
        specs = [spec] + [f[0] for f in factors]
        ops = [N] + [f[1] for f in factors]
        e = coef * np.einsum(",".join(specs) + "->" + out, *ops, optimize=True)
        E = e if E is None else E + e
    V = E.shape[0]
    return E.reshape(V, 4 * 2 ** len(held), -1)


def _place(Ft: np.ndarray, t: Term) -> np.ndarray:
    """[..., alpha1, held1, alpha2, held2] -> [..., alpha1, alpha2, alpha3, alpha4]."""
    lead = Ft.shape[:-2]
    h1 = (2,) * len(t.held1)
    h2 = (2,) * len(t.held2)
    F = Ft.reshape(lead + (4,) + h1 + (4,) + h2)
    n = len(lead)
    src = "".join(chr(ord("a") + i) for i in range(n))
    spec = src + "w" + t.held1 + "v" + t.held2
    return np.einsum(spec + "->" + src + "wvpq", F)


def shifted_sites(L: int, r) -> np.ndarray:
    """Site index of X + r (mod L componentwise) for every site X."""
    s = np.arange(L ** 3)
    x, y, z = s % L, (s // L) % L, s // (L * L)
    return (x + r[0]) % L + L * ((y + r[1]) % L) + L * L * ((z + r[2]) % L)


def direct_sum(E1: np.ndarray, E2: np.ndarray, L: int, r_list, table_bytes: int = 1 << 30) -> np.ndarray:
    """sum_X sum_xi E1[X+r, m, xi] E2[X, n, xi] for each r: complex128 [n_r, m, n].

    When the site-pair table fits in memory it is formed once,
    G[Y, m, X, n] = sum_xi E1[Y, m, xi] E2[X, n, xi], and summed along Y = X + r;
    otherwise each r gathers E1[X + r] and contracts over (X, xi).
    """
    V, m, K = E1.shape
    n = E2.shape[1]
    s = np.arange(V)
    out = np.empty((len(r_list), m, n), dtype=np.complex128)
    if V * m * V * n * 16 <= table_bytes:
        G = (E1.reshape(V * m, K) @ E2.reshape(V * n, K).T).reshape(V, m, V, n)
        for ir, r in enumerate(r_list):
            out[ir] = G[shifted_sites(L, r), :, s, :].sum(axis=0)
    else:
        for ir, r in enumerate(r_list):
            out[ir] = np.tensordot(E1[shifted_sites(L, r)], E2, axes=([0, 2], [0, 2]))
    return out


def all_r(L: int):
    """Every separation r in site order (rx fastest)."""
    return [(x, y, z) for z in range(L) for y in range(L) for x in range(L)]


def correlator(channel, props: dict, L: int, r_list=None, block=(0, 0)) -> np.ndarray:
    """F^{<B1 B2 B3bar B4bar>}_{a1 a2, a3 a4}(r) for one timeslice, by direct sum over X.

    channel: (B1, B2, B3, B4) field names (keys of FIELDS).
    props:   {'u': S_u, 'd': S_d, 's': S_s}, complex128 [V, 12, 12] each.
    r_list:  None for every r (site order), else a list of (rx, ry, rz).
    block:   source spin pair (o3, o4): alpha3 = 2 o3 + j3, alpha4 = 2 o4 + j4 for j in {0, 1}.
    Returns complex128 [4, 4, 2, 2, n_r]  (alpha1, alpha2, j3, j4, r).
    """
    B1, B2, B3, B4 = channel
    if r_list is None:
        r_list = all_r(L)
    blocks = _Blocks(props)
    F = np.zeros((len(r_list), 4, 4, 2, 2), dtype=np.complex128)
    for t in topologies(B1, B2, B3, B4, block):
        E1 = effective_block(t, 1, blocks)
        E2 = effective_block(t, 2, blocks)
        F += t.sign0 * t.c34 * _place(direct_sum(E1, E2, L, r_list), t)
    return np.moveaxis(F, 0, -1)


def zero_momentum(channel, props: dict, L: int, block=(0, 0)) -> np.ndarray:
    """sum_r F(r) = sum_terms sign (sum_x E1)(sum_y E2): complex128 [4, 4, 2, 2]."""
    B1, B2, B3, B4 = channel
    blocks = _Blocks(props)
    F = np.zeros((4, 4, 2, 2), dtype=np.complex128)
    for t in topologies(B1, B2, B3, B4, block):
        s1 = effective_block(t, 1, blocks).sum(axis=0)
        s2 = effective_block(t, 2, blocks).sum(axis=0)
        F += t.sign0 * t.c34 * _place((s1 @ s2.T)[None], t)[0]
    return F


class PhaseSums:
    """Phase-weighted site sums of the normal blocks, sum_x e^{i sign 2 pi n.x / L} N^m(x), per monomial.

    For a momentum q = 2 pi n / L the correlation theorem of Eq. (2.6) gives
        sum_r e^{-i q.r} F(r) = sum_terms (sum_Y e^{-i q.Y} E1(Y)) (sum_X e^{+i q.X} E2(X)),
    and an effective block is linear in the normal block of each site (the source tensor of Eq. (2.4)
    acts site by site, Eq. (2.7)), so sum_x w(x) E(x) is the effective block built from
    sum_x w(x) N(x).  The sums are accumulated over chunks of sites, so no full-volume normal block is
    held; each one is returned as a one-site block [1, 4, 4, 3, 4, 3, 4, 3] that effective_block()
    takes in place of the per-site blocks.
    """

    def __init__(self, props: dict, L: int, n_list, chunk: int = 1024):
        self.props, self.L, self.chunk = props, L, chunk
        self.n_list = [tuple(int(v) for v in n) for n in n_list]
        self.cache: dict[str, dict] = {}

    def _fill(self, mono: str) -> dict:
        L, V = self.L, self.L ** 3
        s = np.arange(V)
        x, y, z = s % L, (s // L) % L, s // (L * L)
        keys = [(n, sign) for n in self.n_list for sign in (-1, 1)]
        acc = None
        for c0 in range(0, V, self.chunk):
            sl = slice(c0, min(V, c0 + self.chunk))
            N = normal_block(self.props[mono[0]][sl], self.props[mono[1]][sl], self.props[mono[2]][sl])
            # one row of weights e^{i sign q.x} per (n, sign) over this chunk's sites
            W = np.stack([np.exp(1j * sign * 2.0 * math.pi * (n[0] * x[sl] + n[1] * y[sl] + n[2] * z[sl]) / L)
                          for n, sign in keys])
            part = W @ N.reshape(N.shape[0], -1)
            acc = part if acc is None else acc + part
        shape = (1,) + N.shape[1:]
        return {k: acc[i].reshape(shape) for i, k in enumerate(keys)}

    def blocks(self, n, sign: int):
        """A blocks callable (monomial -> one-site block) for the weight e^{i sign 2 pi n.x / L}."""
        n = tuple(int(v) for v in n)

        def get(mono: str) -> np.ndarray:
            if mono not in self.cache:
                self.cache[mono] = self._fill(mono)
            return self.cache[mono][(n, sign)]
        return get


def momentum_projection(channel, sums: PhaseSums, n_list, block=(0, 0)) -> np.ndarray:
    """F~(q) = sum_r e^{-i q.r} F(r) at q = 2 pi n / L for each n of n_list, by the correlation theorem of
    Eq. (2.6): sum over terms of (sum_Y e^{-i q.Y} E1(Y)) (sum_X e^{+i q.X} E2(X)).
    complex128 [len(n_list), 4, 4, 2, 2]; n = (0, 0, 0) is the zero-momentum sum of zero_momentum()."""
    B1, B2, B3, B4 = channel
    F = np.zeros((len(n_list), 4, 4, 2, 2), dtype=np.complex128)
    for t in topologies(B1, B2, B3, B4, block):
        for k, n in enumerate(n_list):
            s1 = effective_block(t, 1, sums.blocks(n, -1))[0]
            s2 = effective_block(t, 2, sums.blocks(n, +1))[0]
            F[k] += t.sign0 * t.c34 * _place((s1 @ s2.T)[None], t)[0]
    return F


#: strangeness sectors S = 0 .. -4 and their particle-basis pairs of smallest |I3|
SECTORS = [
    [("p", "n")],
    [("p", "Lambda"), ("p", "Sigma0"), ("n", "Sigma+")],
    [("p", "Xi-"), ("n", "Xi0"), ("Lambda", "Lambda"), ("Lambda", "Sigma0"), ("Sigma+", "Sigma-"),
     ("Sigma0", "Sigma0")],
    [("Lambda", "Xi0"), ("Sigma+", "Xi-"), ("Sigma0", "Xi0")],
    [("Xi0", "Xi-")],
]


def channel_table_56() -> list[tuple[str, str, str, str]]:
    """Every (sink pair, source pair) of one sector, in sector order, sink-major: 1 + 9 + 36 + 9 + 1 = 56."""
    return [sink + src for sector in SECTORS for sink in sector for src in sector]


def vanishes_for_equal_light(channel) -> bool:
    """True for a channel that is identically zero when u and d share a propagator.

    Lambda and Sigma0 are the only fields of the list that the exchange u <-> d maps to themselves
    (Lambda to -Lambda, Sigma0 to +Sigma0, Eq. (2.3)), so a channel made of them alone with an odd
    number of Lambdas equals minus itself.
    """
    return all(f in ("Lambda", "Sigma0") for f in channel) and sum(f == "Lambda" for f in channel) % 2 == 1


def channel_table() -> list[tuple[str, str, str, str]]:
    """The 52 octet-octet channels "from NN to Xi Xi" (Sec. 1; Sec. 4 (iii)), reconstructed.

    The paper takes its list from tables of another paper that are not available here, so the list is
    rebuilt from its description: in each strangeness sector the particle-basis sink pairs of smallest
    |I3| (SECTORS), each with every pair of its sector as the source (channel_table_56), without the
    four that vanish identically for u = d (vanishes_for_equal_light): 52 remain.
    """
    return [ch for ch in channel_table_56() if not vanishes_for_equal_light(ch)]


def flavour_content(channel) -> tuple[int, int]:
    """(number of light quarks, number of strange quarks) of the sink pair."""
    m = FIELDS[channel[0]][0][1] + FIELDS[channel[1]][0][1]
    return 6 - m.count("s"), m.count("s")


# --- from correlators to a local potential (the step Sec. 1 motivates) --------

def potential_stencil(R_prev: np.ndarray, R_cur: np.ndarray, R_next: np.ndarray, L: int, a: float, b: float,
                      c: float):
    """K = a d_t^2 R + b d_t R + c lap R and K / R(t) for cubes R[..., V] (site = x + L (y + L z)), periodic.

    Central differences in t (second difference and half the difference of the neighbours); the lattice
    Laplacian sums the six nearest neighbours minus 6 R.  The caller normalises R and picks a, b, c.
    """
    shape = R_cur.shape
    cube = lambda R: R.reshape(shape[:-1] + (L, L, L))  # axes (z, y, x)
    Rc = cube(R_cur)
    lap = -6.0 * Rc
    for ax in (-1, -2, -3):
        lap = lap + np.roll(Rc, 1, axis=ax) + np.roll(Rc, -1, axis=ax)
    K = a * (R_next - 2.0 * R_cur + R_prev) + b * 0.5 * (R_next - R_prev) + c * lap.reshape(shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        return K, K / R_cur
