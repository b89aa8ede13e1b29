"""Step-by-step numpy re-execution of the device program from the exported plan tables.

Test-only: it lets the CPU suite check the host channel compiler (block
recipes, packing signs, gather tables, term shapes) against the oracle
without a GPU.  It follows the same stages as the kernels (field blocks,
FFT, table-driven contraction at q and -q, inverse FFT) with numpy.
"""

import numpy as np

from paper_1604_07983_gb300 import plan_tables

_G = np.array([[0, 1, 0, 0], [-1, 0, 0, 0], [0, 0, 0, 1], [0, 0, -1, 0]], float)
_E = np.zeros((3, 3, 3))
for (a, b, c), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (1, 0, 2): -1, (0, 2, 1): -1, (2, 1, 0): -1}.items():
    _E[a, b, c] = s


def _normal(S1, S2, S3):
    V = S1.shape[0]
    r = lambda S: S.reshape(V, 4, 3, 12)
    # N[x, alpha, j1, j2, j3] = sum eps_abc G_bg S1(b a; j1) S2(g b; j2) S3(alpha c; j3)
    return np.einsum("abc,BG,xBaI,xGbJ,xAcK->xAIJK", _E, _G, r(S1), r(S2), r(S3), optimize=True)


#: diquark flavour pairs of the normal-block patterns (pattern = diquark * nflav + third flavour)
_DIQUARKS = {2: [(0, 0), (0, 1)], 3: [(0, 0), (0, 1), (1, 1), (0, 2), (1, 2)]}


def emulate(channel_ids, Sl, Ss, L, Sd=None):
    """F[ch, alpha1, alpha2, alpha3, alpha4, r] for one timeslice.  Sd given: the three-flavour tables
    (propagators u = Sl, d = Sd, s = Ss); else the two-flavour tables (l = Sl, s = Ss)."""
    V = L ** 3
    nf = 2 if Sd is None else 3
    tb = plan_tables(channel_ids, flavours=nf)
    S = [Sl, Ss] if nf == 2 else [Sl, Sd, Ss]
    N = {}
    for d, (f0, f1) in enumerate(_DIQUARKS[nf]):
        for f2 in range(nf):
            N[d * nf + f2] = _normal(S[f0], S[f1], S[f2])
    ncell = len(tb["cells"])
    FB = np.zeros((ncell, 4, V), dtype=complex)
    for ti, (off, nc, toff, nt) in enumerate(tb["types"]):
        for c in range(nc):
            code = tb["cells"][off + c]
            y = (code % 12, (code // 12) % 12, code // 144)
            acc = np.zeros((V, 4), dtype=complex)
            for k in range(toff, toff + nt):
                pat, a0, a1, a2 = tb["typeterms"][k]
                acc += tb["typecoef"][k] * N[pat][:, :, y[a0], y[a1], y[a2]]
            FB[off + c] = acc.T
    FBt = np.fft.fftn(FB.reshape(ncell, 4, L, L, L), axes=(2, 3, 4)).reshape(ncell, 4, V)
    q = np.arange(V)
    qx, qy, qz = q % L, (q // L) % L, q // (L * L)
    qm = (-qx) % L + L * ((-qy) % L) + L * L * ((-qz) % L)
    nch = len(channel_ids)
    Ft = np.zeros((nch, 4, 4, 2, 2, V), dtype=complex)
    for (ch, K, shape, n1, n2, off1, off2, _) in tb["terms"]:
        nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
        nh2 = 4 // nh1
        # entries of step k are ordered [i][h]
        c1 = tb["ent1_cell"][off1:off1 + K * nh1 * n1].reshape(K, n1, nh1).transpose(0, 2, 1)
        w1 = tb["ent1_coef"][off1:off1 + K * nh1 * n1].reshape(K, n1, nh1).transpose(0, 2, 1)
        c2 = tb["ent2_cell"][off2:off2 + K * nh2 * n2].reshape(K, n2, nh2).transpose(0, 2, 1)
        w2 = tb["ent2_coef"][off2:off2 + K * nh2 * n2].reshape(K, n2, nh2).transpose(0, 2, 1)
        e1 = np.einsum("khi,khiaq->khaq", w1, FBt[c1])
        e2 = np.einsum("khi,khibq->khbq", w2, FBt[c2][..., qm])
        prod = np.einsum("kiaq,kjbq->abijq", e1, e2)  # [a, b, h1, h2, q]
        for h1 in range(nh1):
            for h2 in range(nh2):
                if shape == 0:
                    s = h2
                elif shape == 3:
                    s = h1
                elif shape == 1:
                    s = h1 + 2 * h2
                else:
                    s = h2 + 2 * h1
                Ft[ch, :, :, s % 2, s // 2] += prod[:, :, h1, h2]
    return np.fft.ifftn(Ft.reshape(nch, 4, 4, 2, 2, L, L, L), axes=(5, 6, 7)).reshape(nch, 4, 4, 2, 2, V)
