"""Launch-shape autotuner for the contraction and the 3-D FFTs.

For a context with propagators loaded, it times each candidate kernel / launch
shape of the effective-block contraction on one timeslice with the library's
own CUDA-event stage timing (nbs_set_profiling / nbs_profile) and keeps the
fastest, then does the same for the block size of the FFTs' strided passes
(forward and inverse stage times), and caches the choice in a JSON file keyed
by (GPU name, L, precision, channel set).  Results do not depend on the choice
beyond rounding; every candidate is covered by the parity tests.
"""

from __future__ import annotations

import hashlib
import json
import os

from .nbs import NBS_BF16X3, NBS_FP32, NBS_FP64, Context

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "nbs_gb300", "autotune.json")

#: (contraction config, momentum block) candidates per precision mode: FP32 the two-phase row kernel
#: (config 0) at three momentum blocks and the quad-lane kernel (config 4); BF16X3 its quad-lane
#: tensor-core kernel; FP64 the thread-per-momentum shapes
CANDIDATES = {
    NBS_FP32: [(0, 32), (0, 64), (0, 16), (4, 32)],
    NBS_BF16X3: [(0, 16), (0, 32), (0, 64)],
    NBS_FP64: [(21, 0), (12, 0), (22, 0), (11, 0)],
}


def cache_key(device_name: str, L: int, precision: int, ids) -> str:
    """Cache key of a tuning: GPU name, lattice size, precision mode and a hash of the channel list."""
    h = hashlib.sha1(",".join(map(str, ids)).encode()).hexdigest()[:12]
    return "%s|L=%d|prec=%d|ch=%s" % (device_name, L, precision, h)


def _key(ctx: Context, ids, precision: int) -> str:
    import torch
    return cache_key(torch.cuda.get_device_name(), ctx.L, precision, ids)


def _load(path=None):
    try:
        with open(path or CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


FFT_BLOCKS = (64, 128, 256)


def _apply(ctx: Context, cfg: int, qb: int, fft_block: int = 0):
    ctx.set_param(Context.PARAM_CONTRACT_CFG, cfg)
    if qb:
        ctx.set_param(Context.PARAM_CHUNK_QBLOCK, qb)
    if fft_block:
        ctx.set_param(Context.PARAM_FFT_BLOCK, fft_block)


def tune(ctx: Context, ids, precision: int, t: int = 0, reps: int = 2, use_cache: bool = True, out=None,
         key: str = None, cache_path: str = None) -> dict:
    """Pick the fastest contraction shape and FFT block for (ctx.L, precision, ids) and apply them to ctx.

    Propagators for timeslice t must be loaded.  out: a device tensor [len(ids), 1, 4, 4, 2, 2, V] to
    correlate into (allocated when None); key, cache_path: the cache key and file (defaults: cache_key()
    of this GPU, CACHE).  Returns {"cfg", "qb", "ms", "timings", "fft_block", "fft_ms", "fft_timings"}.
    """
    key = key or _key(ctx, ids, precision)
    cache_path = cache_path or CACHE
    cache = _load(cache_path) if use_cache else {}
    if key in cache and "fft_block" in cache[key]:
        best = cache[key]
        _apply(ctx, best["cfg"], best["qb"], best["fft_block"])
        return best
    if out is None:
        import torch
        out = torch.empty((len(ids), 1, 4, 4, 2, 2, ctx.V), dtype=torch.complex128, device="cuda")
    timings = []
    for cfg, qb in CANDIDATES[precision]:
        _apply(ctx, cfg, qb)
        ctx.correlate(ids, t, t + 1, out)  # warm-up (and block build)
        ctx.set_profiling(True)
        for _ in range(reps):
            ctx.correlate(ids, t, t + 1, out)
        stages, _ = ctx.profile()
        ctx.set_profiling(False)
        timings.append({"cfg": cfg, "qb": qb, "ms": stages["contract"] / reps})
    best = dict(min(timings, key=lambda r: r["ms"]))
    best["timings"] = timings
    _apply(ctx, best["cfg"], best["qb"])
    fft_timings = []
    for fb in FFT_BLOCKS:
        ctx.set_param(Context.PARAM_FFT_BLOCK, fb)
        ctx.blocks(t)  # warm-up
        ctx.set_profiling(True)
        for _ in range(reps):
            ctx.blocks(t)                     # rescale, blocks, forward FFT (always rebuilt)
            ctx.correlate(ids, t, t + 1, out)  # contraction and inverse FFT on those blocks
        stages, _ = ctx.profile()
        ctx.set_profiling(False)
        fft_timings.append({"fft_block": fb, "ms": (stages["fft_fwd"] + stages["fft_inv"]) / reps})
    fbest = min(fft_timings, key=lambda r: r["ms"])
    best["fft_block"], best["fft_ms"], best["fft_timings"] = fbest["fft_block"], fbest["ms"], fft_timings
    _apply(ctx, best["cfg"], best["qb"], best["fft_block"])
    if use_cache:
        cache[key] = best
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best
