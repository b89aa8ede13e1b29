"""The launch-shape autotuner's host logic on the CPU, with a stand-in context that records the parameters
it is given and reports stage times from a table (no GPU): it times every candidate, keeps the fastest
contraction shape and FFT block, applies them, writes them to its cache under the key of (GPU, L,
precision, channel list), and on a second call applies the cached choice without timing anything."""

import json

import pytest

nbs = pytest.importorskip("paper_1604_07983_gb300.nbs")
from paper_1604_07983_gb300 import autotune as A  # noqa: E402


class FakeContext:
    """Stage times depend on the parameters set: the contraction on (config, momentum block), the FFTs on
    the FFT block."""

    PARAM_CONTRACT_CFG, PARAM_CHUNK_QBLOCK, PARAM_FFT_BLOCK = 0, 1, 2

    def __init__(self, L, contract_ms, fft_ms):
        self.L, self.V = L, L ** 3
        self.params = {}
        self.calls = []
        self.contract_ms, self.fft_ms = contract_ms, fft_ms
        self.prof = False
        self.acc = {}

    def set_param(self, p, v):
        self.params[p] = v
        self.calls.append(("param", p, v))

    def _stage(self, name, ms):
        if self.prof:
            self.acc[name] = self.acc.get(name, 0.0) + ms

    def correlate(self, ids, t0, t1, out):
        self.calls.append(("correlate", t0))
        cfg, qb = self.params.get(0, 0), self.params.get(1, 32)
        self._stage("contract", self.contract_ms[(cfg, qb)])
        self._stage("fft_inv", 0.5 * self.fft_ms[self.params.get(2, 128)])

    def blocks(self, t):
        self.calls.append(("blocks", t))
        self._stage("fft_fwd", 0.5 * self.fft_ms[self.params.get(2, 128)])

    def set_profiling(self, on):
        self.prof = bool(on)
        self.acc = {}

    def profile(self):
        return dict(self.acc), 0


def test_cache_key_names_gpu_size_precision_and_channels():
    k = A.cache_key("NVIDIA GB300", 32, nbs.NBS_FP32, range(52))
    assert k.startswith("NVIDIA GB300|L=32|prec=1|ch=")
    assert k != A.cache_key("NVIDIA GB300", 32, nbs.NBS_FP32, range(51))
    assert k != A.cache_key("NVIDIA GB300", 24, nbs.NBS_FP32, range(52))
    assert k != A.cache_key("NVIDIA GB300", 32, nbs.NBS_BF16X3, range(52))
    assert k == A.cache_key("NVIDIA GB300", 32, nbs.NBS_FP32, list(range(52)))


def test_candidates_are_valid_contraction_configs():
    for prec, cands in A.CANDIDATES.items():
        assert cands, prec
        for cfg, qb in cands:
            a, w = cfg // 10, cfg % 10
            assert 0 <= cfg <= 4 or (a in (1, 2, 4) and w in (1, 2, 4)), (prec, cfg)
            assert qb == 0 or 1 <= qb <= 1 << 20
    assert (0, 32) in A.CANDIDATES[nbs.NBS_FP32] and (4, 32) in A.CANDIDATES[nbs.NBS_FP32]


def test_tune_picks_the_fastest_applies_and_caches(tmp_path):
    prec = nbs.NBS_FP32
    times = {c: 30.0 + i for i, c in enumerate(A.CANDIDATES[prec])}
    fastest = A.CANDIDATES[prec][2]
    times[fastest] = 20.0
    ctx = FakeContext(16, times, {64: 3.0, 128: 2.5, 256: 2.8})
    path = str(tmp_path / "tune.json")
    best = A.tune(ctx, list(range(52)), prec, reps=2, out=object(), key="k", cache_path=path)
    assert (best["cfg"], best["qb"]) == fastest and best["ms"] == pytest.approx(20.0)
    assert best["fft_block"] == 128 and best["fft_ms"] == pytest.approx(2.5)
    assert len(best["timings"]) == len(A.CANDIDATES[prec]) and len(best["fft_timings"]) == 3
    # the choice is the context's final state
    assert ctx.params[0] == fastest[0] and ctx.params[2] == 128
    if fastest[1]:
        assert ctx.params[1] == fastest[1]
    cached = json.load(open(path))["k"]
    assert (cached["cfg"], cached["qb"], cached["fft_block"]) == (fastest[0], fastest[1], 128)
    # second call: the cached choice, applied without timing
    ctx2 = FakeContext(16, times, {64: 3.0, 128: 2.5, 256: 2.8})
    again = A.tune(ctx2, list(range(52)), prec, out=object(), key="k", cache_path=path)
    assert (again["cfg"], again["qb"]) == fastest
    assert not [c for c in ctx2.calls if c[0] != "param"]
    assert ctx2.params[0] == fastest[0] and ctx2.params[2] == 128
