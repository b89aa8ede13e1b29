"""CPU checks of the C ABI library: exports, argument errors, and the host
channel compiler re-executed step by step against the oracle (no GPU)."""

import ctypes
import os
import re

import numpy as np
import pytest

import nbs_inputs as I
from oracle import nbs_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
nbs = pytest.importorskip("paper_1604_07983_gb300.nbs")


@pytest.fixture(scope="module")
def lib():
    try:
        return nbs.lib()
    except ImportError:
        pytest.skip("libnbs.so not built")


def header_functions():
    src = open(os.path.join(ROOT, "include", "nbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nbs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = header_functions()
    assert declared == sorted(nbs.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_channel_table(lib):
    names = nbs.channel_names()
    assert len(names) == 52
    assert names[0] == ("p", "n", "p", "n")
    assert len(set(names)) == 52
    for c, ch in enumerate(names):
        _, nl = nbs.channel_info(c)
        assert (nl, 6 - nl) == O.flavour_content(ch)
    # isospin-forbidden Lambda/Sigma0 transitions are not in the table
    assert ("Lambda", "Lambda", "Lambda", "Sigma0") not in names
    assert ("Sigma0", "Sigma0", "Lambda", "Sigma0") not in names


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.nbs_create(ctypes.byref(h), 8, 8, 4) == nbs.NBS_EINVAL
    assert b"flavours" in lib.nbs_last_error(None)
    assert lib.nbs_create(ctypes.byref(h), 5, 8, 2) == nbs.NBS_EINVAL
    assert lib.nbs_create(ctypes.byref(h), 8, 0, 2) == nbs.NBS_EINVAL
    p = ctypes.c_void_p()
    for bad in (4 * 52, -1):  # ids run over 52 channels x 4 source spin pairs
        ids = (ctypes.c_int * 1)(bad)
        assert lib.nbs_plan_create(ctypes.byref(p), ids, 1) == nbs.NBS_EINVAL
    ids = (ctypes.c_int * 1)(99)  # channel 47, source spins alpha3 in {2, 3}, alpha4 in {0, 1}
    assert lib.nbs_plan_create(ctypes.byref(p), ids, 1) == nbs.NBS_OK
    lib.nbs_plan_destroy(p)
    assert lib.nbs_channel_info(52, None, 0) == nbs.NBS_EINVAL
    assert lib.nbs_set_precision(None, 0) == nbs.NBS_EINVAL


def test_block_types_share_isospin_partners(lib):
    tb = nbs.plan_tables(list(range(52)))
    # p/n, Sigma+/Sigma-, Xi0/Xi-, Lambda, Sigma0: five stored types; of their 4104 cells (3 x 792 + 792 +
    # 936, 16416 components) the 52 channels' gathers read 3547, and only those are kept
    assert len(tb["types"]) == 5
    assert len(tb["cells"]) == 3547
    used = np.zeros(len(tb["cells"]), bool)
    used[tb["ent1_cell"]] = True
    used[tb["ent2_cell"]] = True
    assert used.all()


def test_gather_entries_stay_inside_their_slabs(lib):
    """Every gather entry (padding included) reads a cell of its side's stored type."""
    names = nbs.channel_names()
    tb = nbs.plan_tables(list(range(52)))
    types = tb["types"]
    tpl = nbs.plan_tables([0])   # p/n type is type 0 in every plan
    assert tpl["types"][0][0] == 0
    # the stored type of each sink field, from a one-channel plan per field pair
    for c, (ch, K, shape, n1, n2, off1, off2, local) in enumerate(tb["terms"]):
        nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
        nh2 = 4 // nh1
        cells1 = tb["ent1_cell"][off1:off1 + K * nh1 * n1]
        cells2 = tb["ent2_cell"][off2:off2 + K * nh2 * n2]
        for cells in (cells1, cells2):
            t = np.searchsorted(types[:, 0], cells, side="right") - 1
            assert (t == t[0]).all(), names[ch]
            assert ((cells >= types[t, 0]) & (cells < types[t, 0] + types[t, 1])).all()
        assert n1 % 2 == 0 and n2 % 2 == 0


@pytest.mark.parametrize("ids", [list(range(52)), [0], [3, 17, 40]])
def test_slab_work_split_covers_every_term_once(lib, ids):
    """Re-run, on the host, the bookkeeping of the momentum-slab contraction:
    every shared index of every term is visited once, by a warp whose
    partial-sum slot range holds the term's channel, and every read stays
    inside the group's two slabs."""
    tb = nbs.plan_tables(ids)
    W = 4
    terms, items, groups, gch = tb["terms"], tb["items"], tb["groups"], tb["group_ch"]
    seen = np.zeros(len(terms), dtype=int)
    assert sorted(gch.tolist()) == list(range(len(ids)))
    for g in groups:
        base1, n1, base2, n2, ch_off, nch, item_off, nslot = g[:8]
        warp_off, out_base, cfirst = g[8:13], g[13:18], g[18:22]
        assert warp_off[0] == 0 and (np.diff(warp_off) >= 0).all() and out_base[W] == nslot
        for w in range(W):
            for it in range(item_off + warp_off[w], item_off + warp_off[w + 1]):
                t, k0 = items[it]
                ch, K, shape, nn1, nn2, off1, off2, local = terms[t]
                assert gch[ch_off + local] == ch and 0 <= local < nch
                r = local - cfirst[w]
                assert 0 <= r < out_base[w + 1] - out_base[w]
                assert k0 % 32 == 0 and k0 < K
                seen[t] += min(32, K - k0)
                nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
                nh2 = 4 // nh1
                c1 = tb["ent1_cell"][off1 + k0 * nh1 * nn1: off1 + min(K, k0 + 32) * nh1 * nn1]
                c2 = tb["ent2_cell"][off2 + k0 * nh2 * nn2: off2 + min(K, k0 + 32) * nh2 * nn2]
                assert ((c1 >= base1) & (c1 < base1 + n1)).all()
                assert ((c2 >= base2) & (c2 < base2 + n2)).all()
                assert off1 % 2 == 0 and off2 % 2 == 0
    assert (seen == terms[:, 1]).all()


@pytest.mark.parametrize("ids", [list(range(52)), [0], [24, 25, 51]])
def test_chunk_tables_decode_to_the_gather_tables(lib, ids):
    """The 16-bit shared-memory tables of the chunk contraction decode to the
    full gather tables up to the order of the shared indices (the same on both
    sides; terms of one channel and form may exchange them) and of the entries
    of each sum, every read stays in its slab, every shared index of every term
    is visited once, and the shared memory fits a GB300 block."""
    tb = nbs.plan_tables(ids)
    chunks, ctab, items, toff, codes = tb["chunks"], tb["chunk_tab"], tb["chunk_items"], tb["term_tab_off"], tb["codes"]
    terms = tb["terms"]
    assert len(chunks) > 0 and codes[31] == 0
    seen = np.zeros(len(terms), dtype=int)
    for ck in chunks:
        base1, n1, base2, n2, ch_off, nch, tab_off, tab_len, item_off, nslot = ck[:10]
        warp_off, out_base, cfirst, local0 = ck[10:19], ck[19:28], ck[28:36], ck[36]
        assert tab_off % 8 == 0 and tab_len % 8 == 0 and tab_len <= 45056
        assert out_base[8] == nslot
        smem = tab_len * 2 + 2 * (2 * 936 + 2 * 936) * 16 + nslot * 64 * 8 + 128
        assert smem <= 227 * 1024
        for w in range(8):
            for it in range(item_off + warp_off[w], item_off + warp_off[w + 1]):
                t, k0 = items[it]
                ch, K, shape, nn1, nn2, off1, off2, gl = terms[t]
                r = gl - local0 - cfirst[w]
                assert 0 <= gl - local0 < nch and 0 <= r < out_base[w + 1] - out_base[w]
                seen[t] += min(32, K - k0)
        got_keys, want_keys = {}, {}
        for t in set(int(x) for x in items[item_off:item_off + warp_off[8], 0]):
            ch, K, shape, nn1, nn2, off1, off2, gl = terms[t]
            nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
            nh2 = 4 // nh1
            got = [[] for _ in range(K)]
            want = [[] for _ in range(K)]
            got_keys.setdefault((ch, shape, nn1, nn2), []).append(got)
            want_keys.setdefault((ch, shape, nn1, nn2), []).append(want)
            for side, (nn, nh, off, base, ncell) in enumerate([(nn1, nh1, off1, base1, n1), (nn2, nh2, off2, base2, n2)]):
                n = K * nh * nn
                o = toff[t, side]
                assert o % 8 == 0 and o + n <= tab_len
                e = ctab[tab_off + o: tab_off + o + n].astype(np.int64)
                assert ((e & 1023) < ncell).all()
                cell = ((e & 1023) + base).reshape(K, nn, nh)
                coef = (codes[e >> 11] * np.where(e & 1024, -1.0, 1.0)).reshape(K, nn, nh)
                want_cell = tb["ent%d_cell" % (side + 1)][off: off + n].reshape(K, nn, nh)
                want_coef = tb["ent%d_coef" % (side + 1)][off: off + n].reshape(K, nn, nh)
                for k in range(K):
                    for h in range(nh):
                        for keys, c, f in ((got, cell, coef), (want, want_cell, want_coef)):
                            keys[k].append(tuple(sorted((int(c[k, i, h]), round(float(f[k, i, h]), 9))
                                                        for i in range(nn) if f[k, i, h] != 0)))
        # the terms of one channel and form may share their shared indices (one table run)
        for key in want_keys:
            flat = lambda lists: sorted(tuple(x) for lst in lists for x in lst)
            assert flat(got_keys[key]) == flat(want_keys[key]), key
    assert (seen == terms[:, 1]).all()


def test_worked_counts_pn(lib):
    tb = nbs.plan_tables([0])
    terms = tb["terms"]
    assert len(terms) == 9
    assert int(terms[:, 1].sum()) == 586


@pytest.mark.parametrize("L,ids", [(2, list(range(52))), (3, [0, 5, 17, 30, 47, 51])])
def test_compiled_tables_reproduce_oracle(lib, L, ids):
    from plan_emulator import emulate
    names = nbs.channel_names()
    Sl, Ss = I.propagator(61, "l", L, 0), I.propagator(61, "s", L, 0)
    props = {"u": Sl, "d": Sl, "s": Ss}
    F = emulate(ids, Sl, Ss, L)
    for k, c in enumerate(ids):
        Fo = O.correlator(names[c], props, L)
        assert np.linalg.norm(F[k] - Fo) <= 1e-12 * np.linalg.norm(Fo), names[c]


def test_source_spin_blocks_reproduce_oracle(lib):
    """Ids c + k * 52 (k = 1, 2, 3) project the source spins onto the other three pairs
    (alpha3 in {2 (k & 1), +1}, alpha4 in {2 (k >> 1), +1}); the compiled tables, run by the
    emulator, equal the oracle's correlator for that pair (itself pinned to the determinant
    definition at those spins)."""
    from plan_emulator import emulate
    names = nbs.channel_names()
    n = len(names)
    L = 2
    Sl, Ss = I.propagator(62, "l", L, 0), I.propagator(62, "s", L, 0)
    props = {"u": Sl, "d": Sl, "s": Ss}
    base = [0, 9, 24, 33, 51]
    ids = [c + k * n for k in (1, 2, 3) for c in base]
    F = emulate(ids, Sl, Ss, L)
    for j, vid in enumerate(ids):
        c, k = vid % n, vid // n
        Fo = O.correlator(names[c], props, L, block=(k & 1, k >> 1))
        assert np.linalg.norm(Fo) > 0
        assert np.linalg.norm(F[j] - Fo) <= 1e-12 * np.linalg.norm(Fo), (names[c], k)
    with pytest.raises(nbs.NBSError):
        nbs.plan_tables([4 * n])


def test_three_flavours_reproduce_oracle(lib):
    """u != d (flavours = 3): separate stored blocks per sink field, the 15 normal-block patterns over the
    diquarks uu, ud, dd, us, ds; the compiled tables, run by the emulator on distinct u, d, s
    propagators, equal the oracle (which never identifies u with d)."""
    from plan_emulator import emulate
    names = nbs.channel_names()
    L = 2
    Su, Sd, Ss = (I.propagator(63, f, L, 0) for f in ("u", "d", "s"))
    props = {"u": Su, "d": Sd, "s": Ss}
    ids = [0, 1, 4, 9, 12, 24, 33, 39, 51]
    tb = nbs.plan_tables(ids, flavours=3)
    assert len(tb["types"]) > len(nbs.plan_tables(ids)["types"])   # no isospin sharing
    F = emulate(ids, Su, Ss, L, Sd=Sd)
    for j, c in enumerate(ids):
        Fo = O.correlator(names[c], props, L)
        assert np.linalg.norm(F[j] - Fo) <= 1e-12 * np.linalg.norm(Fo), names[c]
    # with u = d the three-flavour tables give the two-flavour result
    Fl = emulate(ids, Su, Ss, L, Sd=Su)
    F2 = emulate(ids, Su, Ss, L)
    assert np.linalg.norm(Fl - F2) <= 1e-12 * np.linalg.norm(F2)


def test_quad_runs_cover_every_step_once(lib):
    """The quad-lane kernels walk each chunk's table runs (a channel's terms of one fixed form back to
    back, or one term) in 8-index steps cut into 16 warp ranges: every shared index of every run is taken
    by exactly one warp, each segment stays inside one run and names the run's form, lengths and channel
    (shapes 0 and 2 with the sides exchanged), and each warp's channels fit its partial-sum slots.  The runs
    are the terms' tables laid end to end."""
    tb = nbs.plan_tables(list(range(52)))
    T, toff, segs = tb["terms"], tb["term_tab_off"], tb["quad_segs"]
    fixed = {(0, 8, 2): 4, (1, 2, 2): 5, (2, 2, 2): 6, (3, 2, 8): 7}
    assert len(segs) == tb["quad_chunks"][-1][43 + 16]
    for ck, qk in zip(tb["chunks"], tb["quad_chunks"]):
        item_off, nit, local0 = ck[8], ck[10 + 8], ck[36]
        nslot, out_base, cfirst, seg_base = qk[8], qk[10:27], qk[27:43], qk[43:60]
        assert qk[9] == local0 and nslot == out_base[16]
        terms_here = sorted(set(int(t) for t in tb["chunk_items"][item_off:item_off + nit, 0]))
        # runs: maximal chains of terms whose side-1 and side-2 tables continue each other
        start = {}
        for t in terms_here:
            ch, K, shape, n1, n2 = T[t][:5]
            nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
            start[(toff[t][0], toff[t][1])] = (t, K, nh1 * n1, (4 // nh1) * n2)
        runs = {}
        for (o1, o2), (t, K, r1, r2) in start.items():
            if any(o1 == p1 + k * a and o2 == p2 + k * b for (p1, p2), (_, k, a, b) in start.items() if (p1, p2) != (o1, o2)):
                continue  # continues another member
            members, k_tot, c1, c2 = [t], K, o1 + K * r1, o2 + K * r2
            while (c1, c2) in start:
                t2, K2, _, _ = start[(c1, c2)]
                members.append(t2)
                k_tot += K2
                c1, c2 = c1 + K2 * r1, c2 + K2 * r2
            runs[(o1, o2)] = (members, k_tot)
        assert sum(len(m) for m, _ in runs.values()) == len(terms_here)
        seen = {key: np.zeros(k, dtype=int) for key, (_, k) in runs.items()}
        for w in range(16):
            keys = []
            for form, t1, t2, kbeg, kend, local, n1, n2 in segs[seg_base[w]:seg_base[w + 1]]:
                swapped = bool(form & 8)
                if swapped:  # shapes 0 and 2 run as 3 and 1 with B2's list first
                    t1, t2, n1, n2 = t2, t1, n2, n1
                members, k_tot = runs[(t1, t2)]
                shapes = {tuple(T[m][2:5]) for m in members}
                assert len(shapes) == 1 and len({T[m][7] for m in members}) == 1
                shape, nn1, nn2 = shapes.pop()
                assert swapped == (shape % 2 == 0)
                want = fixed.get((shape, n1, n2), shape)
                assert (n1, n2) == (nn1, nn2) and form == (want ^ 3 | 8 if swapped else want)
                assert (form & 3) in (1, 3)
                assert len(members) == 1 or want >= 4
                assert local == T[members[0]][7] - local0
                assert 0 <= local - cfirst[w] < out_base[w + 1] - out_base[w]
                assert kbeg % 8 == 0 and kbeg < kend <= k_tot
                seen[(t1, t2)][kbeg:kend] += 1
                keys.append((local, swapped))
            # a warp's runs visit each (channel, side order) once: one flush each
            assert len(set(keys)) == len([k for i, k in enumerate(keys) if i == 0 or keys[i - 1] != k])
        assert all((v == 1).all() for v in seen.values())


@pytest.mark.parametrize("ids", [list(range(52)), list(range(208)), [0], [24, 25, 51], list(range(0, 208, 5))])
def test_quad_kernels_fit_one_block_of_shared_memory(lib, ids):
    """The quad-lane kernels hold a chunk's table and runs, two double-buffered slabs of 2 x 944 cells, the
    partial-sum slots and the per-channel slot lists in one block's shared memory; for the channel sets used
    here that fits a GB300 block (227 KB), so they run instead of the pair-lane fallback."""
    tb = nbs.plan_tables(ids)
    qc = tb["quad_chunks"]
    assert len(qc) > 0
    max_tab, max_slot = int(qc[:, 7].max()), int(qc[:, 8].max())
    max_segs = max(int(q[43 + 16] - q[43]) for q in qc)
    smem = 128 + 2 * 2 * 2 * 944 * 16 + (max_tab + 128) * 2 + max_slot * 64 * 8 + 64 * 4 + max_segs * 32 + \
        (3 * max_slot + 1) * 4 + 8 + 16
    assert smem <= 227 * 1024, smem


def _halfwarp_passes(tb):
    """Shared-memory passes of the quad kernels' gathers under the bank model the compiler orders for: per
    entry slot, the four consecutive shared indices of a half-warp read 32-byte cell rows that take one pass
    per cell of the most frequent (cell mod 4), identical cells counting once.  Returns (passes, ideal)."""
    tab, T, toff, qc, items = tb["chunk_tab"], tb["terms"], tb["term_tab_off"], tb["chunks"], tb["chunk_items"]
    passes = ideal = 0
    seen = set()
    for ck in qc:
        tab_off, item_off, nit = ck[6], ck[8], ck[10 + 8]
        for t in sorted(set(int(x) for x in items[item_off:item_off + nit, 0])):
            ch, K, shape, n1, n2 = T[t][:5]
            nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
            for side, (nn, nh) in enumerate(((n1, nh1), (n2, 4 // nh1))):
                o = tab_off + toff[t][side]
                if (o, side) in seen:
                    continue
                seen.add((o, side))
                e = tab[o:o + K * nn * nh].astype(np.int64).reshape(K, nn * nh)
                for g in range(0, K, 4):
                    for j in range(nn * nh):
                        cells = set(int(c) & 1023 for c in e[g:g + 4, j])
                        passes += max(sum(1 for c in cells if c % 4 == r) for r in range(4))
                        ideal += 1
    return passes, ideal


def test_gather_tables_are_ordered_for_the_banks(lib):
    """The compiler groups each table run's shared indices four at a time so that a half-warp's gathers hit
    distinct bank groups where it can: the 52-channel tables need at most 1.3x the conflict-free number of
    shared-memory passes (the unordered tables needed about 2.6x)."""
    passes, ideal = _halfwarp_passes(nbs.plan_tables(list(range(52))))
    assert passes <= 1.3 * ideal, (passes, ideal)


def test_quad_warp_split_is_balanced_under_its_cost_model(lib):
    """Each chunk's steps are cut into 16 warp ranges whose largest cost (per-form step costs plus a cost per
    run start and per flush, the compiler's model) is within 10 % of the mean over the chunks' warps."""
    tb = nbs.plan_tables(list(range(52)))
    qc, segs = tb["quad_chunks"], tb["quad_segs"]
    worst = mean = 0.0
    for q in qc:
        costs = []
        for w in range(16):
            x, cur = 0.0, None
            for form, t1, t2, kb, ke, local, n1, n2 in segs[q[43 + w]:q[43 + w + 1]]:
                sh = form & 3
                nh1 = 1 << ((sh & 1) + ((sh >> 1) & 1))
                ent = nh1 * n1 + (4 // nh1) * n2
                step = {5: 799.0, 7: 1035.0}.get(form & 7, 926.0 + 43.0 * ent)
                x += ((ke - kb + 7) // 8) * step + 671.0
                if (local, form >> 3) != cur:
                    x += 893.0
                    cur = (local, form >> 3)
            costs.append(x)
        worst += max(costs)
        mean += sum(costs) / 16
    assert worst <= 1.10 * mean, worst / mean


def _held(shape):
    nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1))
    return nh1, 4 // nh1


def _s_index(shape, h1, h2):  # alpha3 + 2 alpha4 of a product, by the term's shape
    return {0: h2, 3: h1, 1: h1 + 2 * h2, 2: h2 + 2 * h1}[shape]


@pytest.mark.parametrize("ids", [list(range(52)), [0, 17, 47], [5, 60, 130, 199, 207], [51, 3, 29, 104, 8]])
def test_quad_runs_reproduce_the_term_products(lib, ids):
    """The quad-lane kernels' walk of the compiled runs, emulated in FP64 on random slab values (one momentum):
    lane spin a gathers its own list, the exchanged list's rows are taken for every alpha, runs with exchanged
    sides (shapes 0 and 2 as 3 and 1) read B2's list first and flush transposed in (alpha1, alpha2), and the s
    index follows the run's shape.  Every channel equals the plain sum over its terms of E1 E2 built from the
    uncompressed gather lists."""
    tb = nbs.plan_tables(ids)
    T, codes, tab = tb["terms"], tb["codes"], tb["chunk_tab"]
    rng = np.random.default_rng(7)
    ncells = int(tb["cells"].shape[0])
    A = rng.standard_normal((ncells, 4)) + 1j * rng.standard_normal((ncells, 4))  # B1's blocks at q
    B = rng.standard_normal((ncells, 4)) + 1j * rng.standard_normal((ncells, 4))  # B2's blocks at -q
    nch = len(ids)
    want = np.zeros((nch, 4, 4, 4), complex)
    for t in range(len(T)):
        ch, K, shape, n1, n2, off1, off2 = (int(x) for x in T[t][:7])
        nh1, nh2 = _held(shape)
        c1 = tb["ent1_cell"][off1:off1 + K * n1 * nh1].reshape(K, n1, nh1)
        f1 = tb["ent1_coef"][off1:off1 + K * n1 * nh1].reshape(K, n1, nh1)
        c2 = tb["ent2_cell"][off2:off2 + K * n2 * nh2].reshape(K, n2, nh2)
        f2 = tb["ent2_coef"][off2:off2 + K * n2 * nh2].reshape(K, n2, nh2)
        E1 = np.einsum("kih,kiha->kha", f1, A[c1])  # [xi][h1][alpha1]
        E2 = np.einsum("kih,kiha->kha", f2, B[c2])
        for h1 in range(nh1):
            for h2 in range(nh2):
                want[ch, :, :, _s_index(shape, h1, h2)] += np.einsum("ka,kb->ab", E1[:, h1], E2[:, h2])
    got = np.zeros_like(want)
    for ck, q in zip(tb["chunks"], tb["quad_chunks"]):
        base1, base2, ch_off, tab_off = ck[0], ck[2], ck[4], ck[6]
        for w in range(16):
            for form, t1, t2, kb, ke, local, n1, n2 in tb["quad_segs"][q[43 + w]:q[43 + w + 1]]:
                swapped, shape = bool(form & 8), int(form & 3)
                nh1, nh2 = _held(shape)
                Sa, ba, Sb, bb = (B, base2, A, base1) if swapped else (A, base1, B, base2)
                def gather(off, n, nh, S, base):
                    e = tab[tab_off + off + kb * n * nh: tab_off + off + ke * n * nh].astype(np.int64)
                    e = e.reshape(ke - kb, n, nh)
                    c = codes[e >> 11] * np.where(e & 1024, -1.0, 1.0)
                    return np.einsum("kih,kiha->kha", c, S[base + (e & 1023)])
                Eo, Ex = gather(t1, n1, nh1, Sa, ba), gather(t2, n2, nh2, Sb, bb)
                ch = tb["group_ch"][ch_off + local]
                for h1 in range(nh1):
                    for h2 in range(nh2):
                        P = np.einsum("ka,kb->ab", Eo[:, h1], Ex[:, h2])  # [own spin][exchanged spin]
                        got[ch, :, :, _s_index(shape, h1, h2)] += P.T if swapped else P
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("ids", [list(range(52)), [0], [24, 25, 51], list(range(0, 208, 5)), list(range(208))])
def test_row_tables_reproduce_the_term_products(lib, ids):
    """The two-phase contraction's tables, executed in FP64 on random stored blocks (one momentum q and its
    mirror -q) the way the kernels do: phase A builds every row of every stored type at both momenta (sum of
    +-1 / +-2 times the type's cells), phase B walks each chunk's warp segments, lane (kq, s) of step st
    takes record (8 st + kq, s): scale times the outer product of its B1 row (of type1, at q) and B2 row
    (of type2, at -q) into output pair s.  Every channel equals the plain sum over its terms of E1 E2 built
    from the uncompressed gather lists; every step is walked by exactly one warp, inside one channel, and
    each warp's channels fit its slots."""
    tb = nbs.plan_tables(ids)
    rt = tb["rows"]
    assert rt is not None
    T = tb["terms"]
    rng = np.random.default_rng(8)
    ncells = int(tb["cells"].shape[0])
    A = rng.standard_normal((ncells, 4)) + 1j * rng.standard_normal((ncells, 4))  # stored blocks at q
    B = rng.standard_normal((ncells, 4)) + 1j * rng.standard_normal((ncells, 4))  # at -q
    nch = len(ids)
    want = np.zeros((nch, 4, 4, 4), complex)
    for t in range(len(T)):
        ch, K, shape, n1, n2, off1, off2 = (int(x) for x in T[t][:7])
        nh1, nh2 = _held(shape)
        c1 = tb["ent1_cell"][off1:off1 + K * n1 * nh1].reshape(K, n1, nh1)
        f1 = tb["ent1_coef"][off1:off1 + K * n1 * nh1].reshape(K, n1, nh1)
        c2 = tb["ent2_cell"][off2:off2 + K * n2 * nh2].reshape(K, n2, nh2)
        f2 = tb["ent2_coef"][off2:off2 + K * n2 * nh2].reshape(K, n2, nh2)
        E1 = np.einsum("kih,kiha->kha", f1, A[c1])
        E2 = np.einsum("kih,kiha->kha", f2, B[c2])
        for h1 in range(nh1):
            for h2 in range(nh2):
                want[ch, :, :, _s_index(shape, h1, h2)] += np.einsum("ka,kb->ab", E1[:, h1], E2[:, h2])
    coef = np.array([1.0, -1.0, 2.0, -2.0])
    # phase A: the rows of every type, at q (from A) and at -q (from B); padding rows stay NaN (no record
    # may name them)
    types = rt["types"]
    NR = len(rt["desc"])
    Rq = np.full((NR, 4), np.nan, complex)
    Rm = np.full((NR, 4), np.nan, complex)
    roff = 0
    for t, (base, ncell, tr, nrow) in enumerate(types[:, :4].astype(int)):
        assert tr == roff and tr % 8 == 0 and nrow % 8 == 0 and nrow <= 4095
        roff += nrow
        for r in range(tr, tr + nrow):
            d = int(rt["desc"][r])
            off, cnt, ty = d & 0xFFFFFF, (d >> 24) & 31, d >> 29
            assert ty == t
            if cnt == 0:
                continue
            e = rt["ent"][off:off + cnt].astype(np.int64)
            cell = e & 0xFFF
            assert np.all(cell < ncell) and np.all(np.diff(cell) > 0)
            c = coef[(e >> 12) & 3][:, None]
            Rq[r] = (c * A[base + cell]).sum(axis=0)
            Rm[r] = (c * B[base + cell]).sum(axis=0)
    assert roff == NR
    got = np.zeros_like(want)
    Z = len(rt["scales"]) - 1  # the zero code (padding records)
    assert Z == 63 and rt["scales"][Z] == 0
    W = rt["warps"]
    for ck in rt["chunks"]:
        t1, t2, roff1, nrow1, roff2, nrow2, rec_off, nstep, ch_off, nch_c, nslot, seg_off, smem = \
            (int(x) for x in ck[:13])
        seg_base, out_base, cfirst = ck[14:15 + W], ck[15 + W:16 + 2 * W], ck[16 + 2 * W:16 + 3 * W]
        assert (roff1, nrow1, roff2, nrow2) == (types[t1, 2], types[t1, 3], types[t2, 2], types[t2, 3])
        assert smem <= rt["smem"] <= 232448
        rec = rt["rec"][rec_off: rec_off + 32 * nstep].astype(np.int64).reshape(nstep, 4, 8)  # [step][g][kq]
        seen = np.zeros(nstep, int)
        for w in range(W):
            segs = rt["segs"][seg_off + seg_base[w]: seg_off + seg_base[w + 1]]
            for sb, se, local, gmap in segs:
                assert cfirst[w] <= local < cfirst[w] + out_base[w + 1] - out_base[w]
                # the flush's turns: group g's rank among the lower groups of its s, and the largest count
                sg = [(gmap >> 2 * g) & 3 for g in range(4)]
                ranks = [sum(sg[h] == sg[g] for h in range(g)) for g in range(4)]
                assert [(gmap >> 8 + 2 * g) & 3 for g in range(4)] == ranks
                assert gmap >> 16 == max(ranks) + 1
                seen[sb:se] += 1
                ch = rt["ch"][ch_off + local]
                for st in range(sb, se):
                    for kq in range(8):
                        for g in range(4):  # lane group g holds records of output pair s
                            s = (gmap >> 2 * g) & 3
                            wd = rec[st, g, kq]
                            r1, r2, code = wd & 0xFFF, (wd >> 12) & 0xFFF, wd >> 24
                            if code == Z:
                                continue
                            assert r1 < nrow1 and r2 < nrow2
                            x, y = Rq[roff1 + r1], Rm[roff2 + r2]
                            assert np.isfinite(x).all() and np.isfinite(y).all()
                            got[ch, :, :, s] += rt["scales"][code] * np.outer(x, y)
        assert np.all(seen == 1)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_row_loads_spread_over_the_banks_per_quarter_warp(lib):
    """Shared-memory wavefronts of the product kernel's 16-byte row loads: a warp's load is served in four
    phases of eight lanes (one lane group of one step, lanes 8 g .. 8 g + 7), and a phase takes as many
    wavefronts as its fullest 16-byte bank group (row mod 8) has distinct rows; ideal one.  Rows are
    numbered by colouring and each (channel, s) list's records regrouped over its quarters so that a
    quarter's rows fall in distinct bank groups: the loads stay within 1.12x of ideal for the 52-channel
    tables (quarters of consecutive records, rows numbered in first-use order, give about 1.6x)."""
    rt = nbs.plan_tables(list(range(52)))["rows"]
    Z = len(rt["scales"]) - 1
    act = ideal = 0
    for ck in rt["chunks"]:
        rec_off, nstep = int(ck[6]), int(ck[7])
        rec = rt["rec"][rec_off: rec_off + 32 * nstep].astype(np.int64).reshape(nstep * 4, 8)
        for q in rec:
            q = q[(q >> 24) != Z]
            if not len(q):
                continue
            for rows in (q & 0xFFF, (q >> 12) & 0xFFF):
                act += np.bincount(np.unique(rows) % 8).max()
                ideal += 1
    assert act / ideal <= 1.12, act / ideal

