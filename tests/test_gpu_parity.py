"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (normwise per channel and timeslice, ||F_gpu - F_ref|| / ||F_ref||):
FP64 path 1e-12, FP32 path 2e-5.
"""

import os

import numpy as np
import pytest

import nbs_inputs as I
from oracle import nbs_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def nbs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07983_gb300 as P
    P.lib()
    return P


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def gpu_correlate(nbs, ids, L, props, precision, t_range=None, host_out=False, c64=False, cfg=0):
    """props: list over t of (S_l, S_s) numpy complex128 arrays."""
    T = len(props)
    t0, t1 = t_range or (0, T)
    V = L ** 3
    with nbs.Context(L, T, precision=precision) as ctx:
        ctx.set_param(ctx.PARAM_CONTRACT_CFG, cfg)
        for t, (Sl, Ss) in enumerate(props):
            dt = torch.complex64 if c64 else torch.complex128
            ctx.load_props(torch.from_numpy(Sl).to("cuda", dt), torch.from_numpy(Ss).to("cuda", dt), t)
        shape = (len(ids), t1 - t0, 4, 4, 2, 2, V)
        if host_out:
            out = torch.empty(shape, dtype=torch.complex128).pin_memory()
        else:
            out = torch.empty(shape, dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, t0, t1, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def seeded(seed, L, T, decay=0.0):
    return [(I.propagator(seed, "l", L, t, decay), I.propagator(seed, "s", L, t, decay)) for t in range(T)]


def oracle(name, Sl, Ss, L, r_list=None):
    return O.correlator(name, {"u": Sl, "d": Sl, "s": Ss}, L, r_list)


def test_fp64_all_channels_L2(nbs):
    L, T = 2, 2
    props = seeded(1701, L, T)
    names = nbs.channel_names()
    ids = list(range(len(names)))
    F = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64)
    for c in ids:
        for t in range(T):
            assert rel(F[c, t], oracle(names[c], *props[t], L)) < FP64_TOL, (names[c], t)


@pytest.mark.parametrize("L", [1, 3, 4, 6])
def test_fp64_sizes(nbs, L):
    props = seeded(1702 + L, L, 1)
    names = nbs.channel_names()
    ids = [0, 3, 9, 17, 24, 40, 47, 51]
    F = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64)
    for k, c in enumerate(ids):
        assert rel(F[k, 0], oracle(names[c], *props[0], L)) < FP64_TOL, names[c]


def test_config1_pn_8cube_all_timeslices(nbs):
    """8^3 x 8, pn channel, full O(V^2) oracle at every r and t."""
    L, T = 8, 8
    props = seeded(1605, L, T)
    F = gpu_correlate(nbs, [0], L, props, nbs.NBS_FP64)
    for t in range(T):
        assert rel(F[0, t], oracle(("p", "n", "p", "n"), *props[t], L)) < FP64_TOL, t


def test_fp32_decaying_propagators(nbs):
    """FP32 path with a per-timeslice rescale: late timeslices (|S| ~ e^-15.5) must not underflow."""
    L, T = 4, 32
    props = seeded(1607, L, T, decay=0.5)
    names = nbs.channel_names()
    ids = [0, 9, 24, 51]
    F = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP32, t_range=(28, 32))
    for k, c in enumerate(ids):
        for tt, t in enumerate(range(28, 32)):
            ref = oracle(names[c], *props[t], L)
            assert np.linalg.norm(ref) < 1e-25   # |S|^6 ~ e^-84: FP32 would underflow without the rescale
            assert rel(F[k, tt], ref) < FP32_TOL, (names[c], t)


def test_fp32_all_channels_L4(nbs):
    L = 4
    props = seeded(1711, L, 1)
    names = nbs.channel_names()
    ids = list(range(len(names)))
    F32 = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP32)
    F64 = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64)
    for c in ids:
        ref = oracle(names[c], *props[0], L)
        assert rel(F64[c, 0], ref) < FP64_TOL, names[c]
        assert rel(F32[c, 0], ref) < FP32_TOL, names[c]


@pytest.mark.parametrize("cfg", [0, 4, 22, 11])
def test_contraction_variants_all_channels(nbs, cfg):
    """Every contraction kernel and launch shape against the oracle, FP64 and FP32, all 52 channels: the
    default (FP32: the row kernels; FP64: thread per momentum), the quad-lane kernel (config 4; FP64 takes
    its default) and two thread-per-momentum shapes."""
    L = 3
    props = seeded(1721, L, 1)
    names = nbs.channel_names()
    ids = list(range(len(names)))
    F64 = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64, cfg=cfg)
    F32 = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP32, cfg=cfg)
    for c in ids:
        ref = oracle(names[c], *props[0], L)
        assert rel(F64[c, 0], ref) < FP64_TOL, (cfg, names[c])
        assert rel(F32[c, 0], ref) < FP32_TOL, (cfg, names[c])


def test_row_contraction_ragged_block_deterministic(nbs):
    """The row contraction with a momentum block (24) that leaves a ragged last block at 4^3: two runs
    give identical results (the slot sums are deterministic), and they agree with the quad-lane kernel
    (config 4, another summation order) to FP32 rounding."""
    L = 4
    props = seeded(1723, L, 1, decay=0.5)
    ids = list(range(nbs.channel_count()))
    out = []
    for cfg in (0, 0, 4):
        with nbs.Context(L, 1, precision=nbs.NBS_FP32) as ctx:
            ctx.set_param(ctx.PARAM_CONTRACT_CFG, cfg)
            ctx.set_param(ctx.PARAM_CHUNK_QBLOCK, 24)
            ctx.load_props(torch.from_numpy(props[0][0]).cuda(), torch.from_numpy(props[0][1]).cuda(), 0)
            o = torch.empty((len(ids), 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
            ctx.correlate(ids, 0, 1, o)
            torch.cuda.synchronize()
            out.append(o.cpu().numpy())
    assert np.isfinite(out[0]).all()
    assert np.array_equal(out[0], out[1])
    for c in ids:
        assert rel(out[2][c], out[0][c]) < 1e-6, c


@pytest.mark.parametrize("cfg", [0])
def test_bf16x3_tensor_core_path_all_channels(nbs, cfg):
    """Split-BF16 x 3 contraction on the tensor cores (quad-lane fragments by movmatrix): every channel
    against the oracle at 2e-5."""
    L = 4
    props = seeded(1722, L, 2, decay=0.5)
    names = nbs.channel_names()
    ids = list(range(len(names)))
    F = gpu_correlate(nbs, ids, L, props, nbs.NBS_BF16X3, cfg=cfg)
    for c in ids:
        for t in range(2):
            assert rel(F[c, t], oracle(names[c], *props[t], L)) < FP32_TOL, (names[c], t)


def expected(L):
    """The oracle's stored values for the L^3 parity case (tests/golden/make_expected.py: momentum
    projections of every channel, direct O(V^2) sums at sampled r for a few channels) and the case's
    propagators, regenerated from the same seeded recipe."""
    e = np.load(os.path.join(os.path.dirname(__file__), "golden", "expected_%dcube_t%d.npz" % (L, {32: 12, 48: 5}[L])))
    assert int(e["L"]) == L
    seed, t, decay = int(e["seed"]), int(e["t"]), float(e["decay"])
    Sl, Ss = I.propagator(seed, "l", L, t, decay), I.propagator(seed, "s", L, t, decay)
    if bool(e["c64"]):
        Sl = Sl.astype(np.complex64).astype(np.complex128)
        Ss = Ss.astype(np.complex64).astype(np.complex128)
    return e, Sl, Ss


def check_against_expected(nbs, e, F, L, tol, what):
    """F [channel, 1, 4, 4, 2, 2, V] from the GPU against the stored oracle values: for every channel and
    stored momentum n, sum_r e^{-2 pi i n.r / L} F(r) normwise over the 64 spins; for the stored channels,
    F at the sampled separations normwise over spins and separations."""
    names = nbs.channel_names()
    assert [" ".join(n) for n in names] == [str(x) for x in e["names"]]   # the oracle's own table
    V = L ** 3
    s = np.arange(V)
    x, y, z = s % L, (s // L) % L, s // (L * L)
    n_list = e["n_list"]
    ph = np.stack([np.exp(-2j * np.pi * (n[0] * x + n[1] * y + n[2] * z) / L) for n in n_list], axis=1)
    got = F[:, 0].reshape(len(names), 64, V) @ ph                     # [channel, 64, n]
    want = e["proj"].reshape(len(names), len(n_list), 64)
    for c in range(len(names)):
        for k in range(len(n_list)):
            assert rel(got[c, :, k], want[c, k]) < tol, (what, names[c], tuple(n_list[k]))
    idx = [int(r[0] + L * (r[1] + L * r[2])) for r in e["r_list"]]
    for j, c in enumerate(e["direct_ids"]):
        assert rel(F[int(c), 0][..., idx], e["direct"][j]) < tol, (what, names[int(c)], "direct sum")


def test_precision_table_32cube(nbs, capsys):
    """The metric's configuration (32^3, seed 1607, t = 12, exp(-0.5 t)) against the oracle directly: the
    FP64, FP32 and split-BF16x3 GPU paths, every one of the 52 channels at five momenta (including q = 0,
    the self-mirror (16, 16, 16) and the contraction's last momentum (31, 31, 31)) and four channels in
    different chunks at five separations (two seeded at random) by the oracle's direct O(V^2) sum; FP64
    within 1e-12, the others within 2e-5.  Also the per-channel normwise error table of FP32 and
    split-BF16x3 against the FP64 GPU path over all r."""
    L = 32
    e, Sl, Ss = expected(L)
    t = int(e["t"])
    names = nbs.channel_names()
    ids = list(range(len(names)))
    F64 = gpu_correlate(nbs, ids, L, [(Sl, Ss)], nbs.NBS_FP64)
    check_against_expected(nbs, e, F64, L, FP64_TOL, "FP64")
    rows = []
    for mode in (nbs.NBS_FP32, nbs.NBS_BF16X3):
        F = gpu_correlate(nbs, ids, L, [(Sl, Ss)], mode)
        check_against_expected(nbs, e, F, L, FP32_TOL, mode)
        errs = [rel(F[c, 0], F64[c, 0]) for c in ids]
        rows.append(errs)
        assert max(errs) < FP32_TOL, (mode, names[int(np.argmax(errs))], max(errs))
        del F
    with capsys.disabled():
        print("\nprecision table 32^3 t=%d: channel, FP32 err, BF16x3 err" % t)
        for c in ids:
            print("%-32s %.3e %.3e" % (" ".join(names[c]), rows[0][c], rows[1][c]))
        print("max FP32 %.3e  max BF16x3 %.3e" % (max(rows[0]), max(rows[1])))


def test_host_output_and_timeslice_split(nbs):
    L, T = 4, 5
    props = seeded(1712, L, T)
    ids = [0, 7, 30]
    Fd = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64)
    Fh = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64, host_out=True)
    assert np.array_equal(Fd, Fh)
    Fa = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64, t_range=(0, 2))
    Fb = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64, t_range=(2, 5))
    assert np.array_equal(np.concatenate([Fa, Fb], axis=1), Fd)


def test_complex64_input(nbs):
    L = 4
    props = seeded(1713, L, 1)
    props32 = [(a.astype(np.complex64).astype(np.complex128), b.astype(np.complex64).astype(np.complex128))
               for a, b in props]
    names = nbs.channel_names()
    ids = [0, 24]
    F = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP32, c64=True)
    for k, c in enumerate(ids):
        assert rel(F[k, 0], oracle(names[c], *props32[0], L)) < FP32_TOL


def test_16cube_gauge_invariance_and_samples(nbs):
    """16^3: every channel invariant under site-local SU(3) sink-colour rotations;
    sampled r and the zero-momentum sum against the oracle for two channels."""
    L = 16
    Sl, Ss = I.propagator(1606, "l", L, 0), I.propagator(1606, "s", L, 0)
    U = I.haar_su3(1606, L)
    names = nbs.channel_names()
    ids = list(range(len(names)))
    F = gpu_correlate(nbs, ids, L, [(Sl, Ss)], nbs.NBS_FP64)
    Fr = gpu_correlate(nbs, ids, L, [(I.rotate_sink_colour(Sl, U), I.rotate_sink_colour(Ss, U))], nbs.NBS_FP64)
    for c in ids:
        assert rel(Fr[c, 0], F[c, 0]) < FP64_TOL, names[c]
    rs = [(0, 0, 0), (1, 0, 0), (0, 15, 0), (8, 8, 8), (3, 11, 5)]
    idx = [x + L * (y + L * z) for x, y, z in rs]
    props = {"u": Sl, "d": Sl, "s": Ss}
    for c in (0, 51):
        ref = O.correlator(names[c], props, L, rs)
        assert rel(F[c, 0][..., idx], ref) < FP64_TOL, names[c]
        zm = O.zero_momentum(names[c], props, L)
        assert rel(F[c, 0].sum(-1), zm) < FP64_TOL


def test_zero_momentum_call(nbs):
    L = 4
    props = seeded(1714, L, 1)
    ids = [0, 24, 51]
    with nbs.Context(L, 1, precision=nbs.NBS_FP64) as ctx:
        ctx.load_props(torch.from_numpy(props[0][0]).cuda(), torch.from_numpy(props[0][1]).cuda(), 0)
        out = torch.empty((3, 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, 0, 1, out)
        zm = ctx.zero_momentum(3)
    assert rel(zm, out.cpu().numpy()[:, 0].sum(-1)) < FP64_TOL


def test_state_and_nan_errors(nbs):
    L = 2
    with nbs.Context(L, 2) as ctx:
        out = torch.empty((1, 1, 4, 4, 2, 2, 8), dtype=torch.complex128, device="cuda")
        with pytest.raises(nbs.NBSError) as e:
            ctx.correlate([0], 0, 1, out)
        assert e.value.code == -4
        Sl, Ss = I.propagator(1, "l", L, 0), I.propagator(1, "s", L, 0)
        Sl[3, 4, 5] = np.nan
        ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), 0)
        with pytest.raises(nbs.NBSError) as e:
            ctx.correlate([0], 0, 1, out)
        assert e.value.code == -6
        with pytest.raises(nbs.NBSError) as e:
            ctx.correlate([4 * 52], 0, 1, out)  # ids run over 52 channels x 4 source spin pairs
        assert e.value.code == -1


def test_graph_replay_matches_correlate(nbs):
    """A captured CUDA graph of nbs_correlate replays the same kernels: identical output; a replay after
    new propagators are loaded gives the new correlators; buffer reallocation and NaN inputs are errors."""
    L, T = 4, 3
    props = seeded(1731, L, T, decay=0.5)
    ids = [0, 9, 24, 51]
    shape = (len(ids), T, 4, 4, 2, 2, L ** 3)
    with nbs.Context(L, T, precision=nbs.NBS_FP32) as ctx:
        for t, (Sl, Ss) in enumerate(props):
            ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), t)
        ref = torch.empty(shape, dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, 0, T, ref)
        out = torch.full(shape, float("nan"), dtype=torch.complex128, device="cuda")
        g = ctx.capture(ids, 0, T, out)
        torch.cuda.synchronize()
        assert torch.isnan(out).all()          # capturing runs nothing
        g.launch()
        assert torch.equal(out, ref)
        # new propagators in slot 1, replay
        Sl, Ss = I.propagator(1732, "l", L, 1, 0.5), I.propagator(1732, "s", L, 1, 0.5)
        ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), 1)
        g.launch()
        one = torch.empty((len(ids), 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, 1, 2, one)
        assert torch.equal(out[:, 1:2], one) and torch.equal(out[:, 0], ref[:, 0])
        names = nbs.channel_names()
        got = out.cpu().numpy()
        for k, c in enumerate(ids):
            assert rel(got[k, 1], oracle(names[c], Sl, Ss, L)) < FP32_TOL, names[c]
        # NaN propagators are reported by a waited replay
        bad = torch.from_numpy(Sl).cuda()
        bad[3, 2, 1] = float("nan")
        ctx.load_props(bad, torch.from_numpy(Ss).cuda(), 2)
        with pytest.raises(nbs.NBSError) as ei:
            g.launch()
        assert ei.value.code == -6
        # more channels reallocate the context's buffers: the graph refuses to run
        ctx.load_props(torch.from_numpy(props[2][0]).cuda(), torch.from_numpy(props[2][1]).cuda(), 2)
        big = torch.empty((52, 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
        ctx.correlate(list(range(52)), 0, 1, big)
        with pytest.raises(nbs.NBSError) as ei:
            g.launch()
        assert ei.value.code == -4


def test_full_source_spin(nbs):
    """All 4 x 4 source spins (ids c + k * 52) through the GPU path, FP64 and FP32, against the
    oracle's correlator for each source spin pair."""
    L = 4
    props = seeded(1741, L, 1, decay=0.5)
    names = nbs.channel_names()
    chans = [0, 24, 51]
    ids = nbs.full_spin_ids(chans)
    F64 = nbs.assemble_full_spin(gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64))
    F32 = nbs.assemble_full_spin(gpu_correlate(nbs, ids, L, props, nbs.NBS_FP32))
    assert F64.shape == (len(chans), 1, 4, 4, 4, 4, L ** 3)
    for j, c in enumerate(chans):
        for k in range(4):
            o3, o4 = k & 1, k >> 1
            ref = oracle(names[c], *props[0], L) if k == 0 else \
                O.correlator(names[c], {"u": props[0][0], "d": props[0][0], "s": props[0][1]}, L, block=(o3, o4))
            sl = (j, 0, slice(None), slice(None), slice(2 * o3, 2 * o3 + 2), slice(2 * o4, 2 * o4 + 2))
            assert rel(F64[sl], ref) < FP64_TOL, (names[c], k)
            assert rel(F32[sl], ref) < FP32_TOL, (names[c], k)


def test_three_flavours_u_ne_d(nbs):
    """flavours = 3 (u != d): FP64 and FP32 against the oracle with distinct u, d, s propagators, and with
    u = d equal to the two-flavour path."""
    L = 4
    names = nbs.channel_names()
    ids = [0, 4, 9, 24, 39, 51]
    Su, Sd, Ss = (I.propagator(1751, f, L, 0, 0.5) for f in ("u", "d", "s"))
    shape = (len(ids), 1, 4, 4, 2, 2, L ** 3)
    res = {}
    for prec in (nbs.NBS_FP64, nbs.NBS_FP32):
        with nbs.Context(L, 1, flavours=3, precision=prec) as ctx:
            ctx.load_props3(torch.from_numpy(Su).cuda(), torch.from_numpy(Sd).cuda(), torch.from_numpy(Ss).cuda(), 0)
            out = torch.empty(shape, dtype=torch.complex128, device="cuda")
            ctx.correlate(ids, 0, 1, out)
            res[prec] = out.cpu().numpy()
            with pytest.raises(nbs.NBSError):
                ctx.load_props(torch.from_numpy(Su).cuda(), torch.from_numpy(Ss).cuda(), 0)
    props = {"u": Su, "d": Sd, "s": Ss}
    for k, c in enumerate(ids):
        ref = O.correlator(names[c], props, L)
        assert rel(res[nbs.NBS_FP64][k, 0], ref) < FP64_TOL, names[c]
        assert rel(res[nbs.NBS_FP32][k, 0], ref) < FP32_TOL, names[c]
    with nbs.Context(L, 1, flavours=3, precision=nbs.NBS_FP64) as ctx:
        u = torch.from_numpy(Su).cuda()
        ctx.load_props3(u, u, torch.from_numpy(Ss).cuda(), 0)
        out3 = torch.empty(shape, dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, 0, 1, out3)
    two = gpu_correlate(nbs, ids, L, [(Su, Ss)], nbs.NBS_FP64)
    assert rel(out3.cpu().numpy(), two) < FP64_TOL


def test_48cube_complex64_storage(nbs):
    """The 48^3 configuration (complex64 propagator storage, e^{-0.4 t} decay) against the oracle: every
    channel at five momenta and pn at two separations by the direct O(V^2) sum, for the FP64 GPU path
    (1e-12) and the FP32 and split-BF16x3 paths on complex64 storage (2e-5); FP32 and split-BF16x3 against
    the FP64 GPU path over all r within 2e-5; and the FP32 result unchanged by a site-local SU(3) rotation
    of the sink colour (the blocks are colour singlets)."""
    L = 48
    e, Sl128, Ss128 = expected(L)
    names = nbs.channel_names()
    ids = list(range(len(names)))
    props = [(Sl128, Ss128)]
    F64 = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP64)
    check_against_expected(nbs, e, F64, L, FP64_TOL, "FP64")
    F32 = gpu_correlate(nbs, ids, L, props, nbs.NBS_FP32, c64=True)
    check_against_expected(nbs, e, F32, L, FP32_TOL, "FP32")
    F16 = gpu_correlate(nbs, ids, L, props, nbs.NBS_BF16X3, c64=True)
    check_against_expected(nbs, e, F16, L, FP32_TOL, "BF16X3")
    for c in ids:
        assert rel(F32[c, 0], F64[c, 0]) < FP32_TOL, names[c]
        assert rel(F16[c, 0], F64[c, 0]) < FP32_TOL, names[c]
    U = I.haar_su3(1615, L)
    rot = [(I.rotate_sink_colour(props[0][0], U), I.rotate_sink_colour(props[0][1], U))]
    sub = [0, 24, 51]
    G32 = gpu_correlate(nbs, sub, L, rot, nbs.NBS_FP32, c64=True)
    for k, c in enumerate(sub):
        assert rel(G32[k, 0], F64[c, 0]) < FP32_TOL, names[c]


def test_potential_stencil(nbs):
    """nbs_potential against the oracle's stencil: random cubes at 5^3 and 8^3, and the correlators of one
    channel on three consecutive timeslices (FP64 path) at 4^3."""
    rng = np.random.default_rng(1761)
    for L, n in ((5, 3), (8, 2)):
        R = [rng.standard_normal((n, L ** 3)) + 1j * rng.standard_normal((n, L ** 3)) for _ in range(3)]
        a, b, c = 0.125, -1.0, 0.25
        K, P = nbs.potential(*(torch.from_numpy(x).cuda() for x in R), L, a, b, c)
        Ko, Po = O.potential_stencil(R[0], R[1], R[2], L, a, b, c)
        assert rel(K.cpu().numpy(), Ko) < 1e-14 and rel(P.cpu().numpy(), Po) < 1e-13
    L = 4
    props = seeded(1762, L, 3, decay=0.5)
    F = gpu_correlate(nbs, [0], L, props, nbs.NBS_FP64)[0]          # [t, 4, 4, 2, 2, V]
    R = [F[t].reshape(64, L ** 3) for t in range(3)]
    K = nbs.potential(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in R), L, 0.1, -1.0, 0.2,
                      ratio=False)
    Ko, _ = O.potential_stencil(R[0], R[1], R[2], L, 0.1, -1.0, 0.2)
    assert rel(K.cpu().numpy(), Ko) < 1e-13


def test_24cube_sampled_r(nbs):
    """24^3 (radix-3 FFT, the fused y/z pass with 3 x-values per block; the batched workload's size):
    FP64 and FP32 against the oracle on sampled separations for the pn channel."""
    L = 24
    Sl, Ss = I.propagator(1608, "l", L, 3, 0.5), I.propagator(1608, "s", L, 3, 0.5)
    F64 = gpu_correlate(nbs, [0], L, [(Sl, Ss)], nbs.NBS_FP64)
    F32 = gpu_correlate(nbs, [0], L, [(Sl, Ss)], nbs.NBS_FP32)
    rs = [(0, 0, 0), (1, 0, 0), (0, 23, 0), (12, 12, 12), (5, 17, 9)]
    idx = [x + L * (y + L * z) for x, y, z in rs]
    ref = O.correlator(("p", "n", "p", "n"), {"u": Sl, "d": Sl, "s": Ss}, L, rs)
    assert rel(F64[0, 0][..., idx], ref) < FP64_TOL
    assert rel(F32[0, 0][..., idx], ref) < FP32_TOL


def test_slab_wait_timeout_is_reported_and_recoverable(nbs):
    """The failure path of the contraction's bounded slab wait, without a device fault: the test switch
    NBS_PARAM_TEST_SKIP_SLAB makes the TMA-staged FP32 quad-lane kernel (contraction config 4) arm each
    block's first slab wait and issue no copy, so nothing is in flight when the wait runs out (about a
    second).  nbs_correlate returns NBS_ETIMEOUT, a waited replay of a graph captured with the switch on
    returns NBS_ETIMEOUT, and with the switch off the same context gives the oracle's correlators again,
    through that kernel and through the default one."""
    L = 8
    props = seeded(1771, L, 1, decay=0.5)
    names = nbs.channel_names()
    ids = [0, 9, 24, 51]
    with nbs.Context(L, 1, precision=nbs.NBS_FP32) as ctx:
        ctx.load_props(torch.from_numpy(props[0][0]).cuda(), torch.from_numpy(props[0][1]).cuda(), 0)
        out = torch.empty((len(ids), 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
        ctx.set_param(0, 4)             # NBS_PARAM_CONTRACT_CFG: the quad-lane kernel
        ctx.correlate(ids, 0, 1, out)   # allocates every buffer before the capture below
        ctx.set_param(3, 1)             # NBS_PARAM_TEST_SKIP_SLAB
        with pytest.raises(nbs.NBSError) as ei:
            ctx.correlate(ids, 0, 1, out)
        assert ei.value.code == -5      # NBS_ETIMEOUT
        g = ctx.capture(ids, 0, 1, out)
        with pytest.raises(nbs.NBSError) as ei:
            g.launch()
        assert ei.value.code == -5
        g.close()
        ctx.set_param(3, 0)
        ctx.correlate(ids, 0, 1, out)
        torch.cuda.synchronize()
        F = out.cpu().numpy()
        ctx.set_param(0, 0)
        ctx.correlate(ids, 0, 1, out)
        torch.cuda.synchronize()
        F0 = out.cpu().numpy()
    for k, c in enumerate(ids):
        want = oracle(names[c], *props[0], L)
        assert rel(F[k, 0], want) < FP32_TOL, names[c]
        assert rel(F0[k, 0], want) < FP32_TOL, names[c]


def test_batched_graph_replay_uneven_sizes_against_the_oracle(nbs):
    """The batched workload's form: contexts of uneven size (16^3 and 24^3, two timeslices each), one CUDA
    graph per (context, timeslice) captured once and all replayed back to back without waiting; every replay
    equals a direct nbs_correlate of the same timeslice bit for bit, and its zero-momentum sum sum_r F(r)
    equals the oracle's (momentum projection at q = 0) within the FP32 tolerance."""
    names = nbs.channel_names()
    ids = [0, 9, 24, 33, 51]
    ctxs, jobs = [], []
    try:
        for L, seed in ((16, 1791), (24, 1792)):
            props = seeded(seed, L, 2, decay=0.5)
            ctx = nbs.Context(L, 2, precision=nbs.NBS_FP32)
            for t, (Sl, Ss) in enumerate(props):
                ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), t)
            ref = torch.empty((len(ids), 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
            ctx.correlate(ids, 0, 1, ref)   # allocates before the captures
            for t in range(2):
                out = torch.full((len(ids), 1, 4, 4, 2, 2, L ** 3), float("nan"), dtype=torch.complex128,
                                 device="cuda")
                jobs.append((ctx, L, t, props[t], out, ctx.capture(ids, t, t + 1, out)))
            ctxs.append(ctx)
        for job in jobs:
            job[5].launch(wait=False)
        torch.cuda.synchronize()
        for ctx, L, t, (Sl, Ss), out, g in jobs:
            direct = torch.empty_like(out)
            ctx.correlate(ids, t, t + 1, direct)
            torch.cuda.synchronize()
            assert torch.equal(out, direct), (L, t)
            zm = out.cpu().numpy()[:, 0].sum(axis=-1)
            sums = O.PhaseSums({"u": Sl, "d": Sl, "s": Ss}, L, [(0, 0, 0)])
            for k, c in enumerate(ids):
                assert rel(zm[k], O.momentum_projection(names[c], sums, [(0, 0, 0)])[0]) < FP32_TOL, (L, t, names[c])
    finally:
        for job in jobs:
            job[5].close()
        for c in ctxs:
            c.close()
