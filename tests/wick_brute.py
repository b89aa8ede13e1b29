"""Brute-force Wick contraction by determinants (test-only pin for the oracle).

Knows nothing about baryon blocks, permutations or topologies.  Each
interpolating field is expanded into its quark terms

    B_alpha(x) = sum coef * q1[(beta, a)] q2[(gamma, b)] q3[(alpha, c)],
    coef = (monomial coefficient) * eps_abc * (C gamma5)_{beta gamma},

the two-baryon source likewise into antiquark terms with the tensor of
Eq. (2.4), and each product of six quarks and six antiquarks is evaluated by
the textbook identity for Gaussian Grassmann integrals

    < q_1 ... q_6 qbar_6 ... qbar_1 > = det[ M ],
    M[k][l] = delta(flavour_k, flavour_l) * S_flavour(x_k; i_k, j_l).

The six antiquarks are ordered qbar_6 ... qbar_1 (slot 6 leftmost), the
mirror of the sink, which is the reading of Eq. (2.5) the oracle uses.  C
gamma5 is built here from explicit Euclidean Dirac matrices, independently of
the oracle's table.
"""

from __future__ import annotations

import itertools
import math

import numpy as np


def dirac_cg5() -> np.ndarray:
    """C gamma5 with C = gamma4 gamma2, Euclidean Dirac representation."""
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    Z, I = np.zeros((2, 2)), np.eye(2)
    g = [np.block([[Z, -1j * sk], [1j * sk, Z]]) for sk in s]
    g4 = np.block([[I, Z], [Z, -I]])
    g5 = g[0] @ g[1] @ g[2] @ g4
    return (g4 @ g[1] @ g5)


_CG5 = dirac_cg5()
_r6, _r2 = 1 / math.sqrt(6), 1 / math.sqrt(2)

# Eqs. (2.2), (2.3): field -> list of (coefficient, flavours of (q1 Cg5 q2) q3)
OPERATORS = {
    "p": [(1.0, ("u", "d", "u"))],
    "n": [(-1.0, ("u", "d", "d"))],
    "Sigma+": [(-1.0, ("u", "s", "u"))],
    "Sigma-": [(-1.0, ("d", "s", "d"))],
    "Xi0": [(1.0, ("u", "s", "s"))],
    "Xi-": [(-1.0, ("d", "s", "s"))],
    "Xu": [(1.0, ("d", "s", "u"))],
    "Xd": [(1.0, ("s", "u", "d"))],
    "Xs": [(1.0, ("u", "d", "s"))],
    "Lambda": [(_r6, ("d", "s", "u")), (_r6, ("s", "u", "d")), (-2 * _r6, ("u", "d", "s"))],
    "Sigma0": [(_r2, ("d", "s", "u")), (-_r2, ("s", "u", "d"))],
}


def _eps_terms():
    out = []
    for p in itertools.permutations(range(3)):
        sgn = 1 if sum(p[i] > p[j] for i in range(3) for j in range(i + 1, 3)) % 2 == 0 else -1
        out.append((p, sgn))
    return out


def _quark_terms(field: str, alpha: int):
    """(coef, [(flavour, spin, colour)] * 3) for B_alpha, or for a source baryon with open spin alpha."""
    out = []
    for cm, fl in OPERATORS[field]:
        for (a, b, c), e in _eps_terms():
            for beta in range(4):
                for gamma in range(4):
                    g = _CG5[beta, gamma]
                    if g == 0:
                        continue
                    out.append((cm * e * g, [(fl[0], beta, a), (fl[1], gamma, b), (fl[2], alpha, c)]))
    return out


_FL = {"u": 0, "d": 1, "s": 2}


def correlator_brute(channel, props: dict, L: int, r, spins, X_list=None) -> complex:
    """F_{a1 a2, a3 a4}(r) = sum_X < B1_a1(X+r) B2_a2(X) Jbar_{a3 a4} > by determinants.

    props: {'u','d','s'} -> complex128 [V, 12, 12]; spins = (a1, a2, a3, a4) with a3, a4 in {0, 1}.
    X_list restricts the sum over X (default: every site).
    """
    B1, B2, B3, B4 = channel
    a1, a2, a3, a4 = spins
    V = L ** 3
    Sall = np.stack([props["u"], props["d"], props["s"]])  # [flav, V, 12, 12]
    sink1, sink2 = _quark_terms(B1, a1), _quark_terms(B2, a2)
    src3, src4 = _quark_terms(B3, a3), _quark_terms(B4, a4)

    def arr(terms1, terms2):
        coef = np.array([c1 * c2 for c1, _ in terms1 for c2, _ in terms2])
        q = [t1 + t2 for _, t1 in terms1 for _, t2 in terms2]
        fl = np.array([[_FL[f] for f, _, _ in qq] for qq in q])
        idx = np.array([[3 * s + c for _, s, c in qq] for qq in q])
        return coef, fl, idx

    ck, fk, ik = arr(sink1, sink2)     # sink quark k = 0..5
    cl, fl, jl = arr(src3, src4)       # source slot l = 0..5
    if X_list is None:
        X_list = range(V)
    total = 0.0 + 0.0j
    for X in X_list:
        x, y, z = X % L, (X // L) % L, X // (L * L)
        Y = (x + r[0]) % L + L * ((y + r[1]) % L) + L * L * ((z + r[2]) % L)
        site = np.array([Y] * 3 + [X] * 3)
        for s0 in range(0, len(ck), 64):
            sl = slice(s0, s0 + 64)
            f_k = fk[sl][:, None, :, None]
            f_l = fl[None, :, None, :]
            M = Sall[f_k, site[None, None, :, None], ik[sl][:, None, :, None], jl[None, :, None, :]]
            M = np.where(f_k == f_l, M, 0.0)
            d = np.linalg.det(M)
            total += np.einsum("s,t,st->", ck[sl], cl, d)
    return total
