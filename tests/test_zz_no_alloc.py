"""The allocation-free entry point nbs_correlate_static against nbs_correlate.

nbs_correlate_static exists for callers that cannot call cudaMalloc (a host
that owns all device memory in its own pool, a locked allocator, a loop that
must not allocate): it keeps every intermediate in one static device array.
Its result must equal the ordinary context path's within the FP64 tolerance
of the other parity tests, on two calls in a row (the second call reuses the
array the first one left behind).  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import nbs_inputs as I
from oracle import nbs_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07983_gb300 as pkg
    pkg.lib()
    return pkg


def context_result(P, Sl, Ss, L, cid):
    with P.Context(L, 1, precision=P.NBS_FP64) as ctx:
        ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), 0)
        out = torch.empty((1, 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
        ctx.correlate([cid], 0, 1, out)
        torch.cuda.synchronize()
    return out.cpu().numpy()[0, 0]


def static_call(P, Sl, Ss, L, cid):
    """nbs_correlate_static on device copies of Sl, Ss (complex128 or complex64): (return code, output)."""
    out = torch.full((4, 4, 2, 2, L ** 3), float("nan"), dtype=torch.complex128, device="cuda")
    u = torch.from_numpy(Sl).cuda()
    s = torch.from_numpy(Ss).cuda()
    dtype = 1 if Sl.dtype == np.complex64 else 0   # NBS_C64 / NBS_C128
    rc = P.lib().nbs_correlate_static(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(s.data_ptr()), L, dtype, cid,
                                      ctypes.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def static_result(P, Sl, Ss, L, cid):
    rc, out = static_call(P, Sl, Ss, L, cid)
    assert rc == 0, P.lib().nbs_last_error(None)
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_static_entry_matches_context_path_twice(P):
    cases = [(4, 0, 1801), (3, 24, 1802)]   # (L, channel id, seed): pn at 4^3, Lambda Lambda at 3^3
    for L, cid, seed in cases:
        Sl, Ss = I.propagator(seed, "l", L, 0), I.propagator(seed, "s", L, 0)
        got = static_result(P, Sl, Ss, L, cid)
        want = context_result(P, Sl, Ss, L, cid)
        assert np.isfinite(got).all()
        assert rel(got, want) < FP64_TOL, (L, cid)


def test_static_entry_complex64_inputs_and_the_oracle(P):
    """Complex64 propagators through the static entry equal the context path on the same values (FP64,
    1e-12), and both equal the FP64 oracle; so do complex128 inputs for two more channels, twice."""
    names = P.channel_names()
    L = 4
    Sl, Ss = I.propagator(1803, "l", L, 0, 0.5), I.propagator(1803, "s", L, 0, 0.5)
    Sl32, Ss32 = Sl.astype(np.complex64), Ss.astype(np.complex64)
    up = {"u": Sl32.astype(np.complex128), "d": Sl32.astype(np.complex128), "s": Ss32.astype(np.complex128)}
    got = static_result(P, Sl32, Ss32, L, 9)
    assert rel(got, context_result(P, up["u"], up["s"], L, 9)) < FP64_TOL
    assert rel(got, O.correlator(names[9], up, L)) < FP64_TOL
    props = {"u": Sl, "d": Sl, "s": Ss}
    for cid in (33, 51):
        for _ in range(2):
            assert rel(static_result(P, Sl, Ss, L, cid), O.correlator(names[cid], props, L)) < FP64_TOL, cid


def test_static_entry_reports_nan_and_bad_channels(P):
    L = 3
    Sl, Ss = I.propagator(1804, "l", L, 0), I.propagator(1804, "s", L, 0)
    bad = Sl.copy()
    bad[5, 7, 2] = np.nan
    rc, _ = static_call(P, bad, Ss, L, 0)
    assert rc == -6   # NBS_ENAN
    rc, _ = static_call(P, Sl, Ss, L, 52)
    assert rc == -1   # NBS_EINVAL: ids of the static entry are the 52 built-in channels
    assert b"channel" in P.lib().nbs_last_error(None)
    # the array is usable again after the errors
    assert rel(static_result(P, Sl, Ss, L, 0), context_result(P, Sl, Ss, L, 0)) < FP64_TOL


def test_static_entry_rejects_lattices_beyond_its_array(P):
    L = 6
    u = torch.zeros((L ** 3, 12, 12), dtype=torch.complex128, device="cuda")
    out = torch.zeros((4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
    rc = P.lib().nbs_correlate_static(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), L, 0, 0,
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1   # NBS_EINVAL
    assert b"L must be" in P.lib().nbs_last_error(None)
