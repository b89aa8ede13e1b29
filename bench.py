"""Throughput of the NBS correlator path on GB300: 52-channel correlators per second at 32^3.

One step = one full pass of the hot path -- propagator rescale, baryon blocks,
forward FFT, effective blocks and their product in momentum space, inverse
FFT, FP64 restore -- for every one of the 52 channels on one timeslice of a
32^3 x 32 lattice (synthetic seeded propagators with exp(-0.5 t) decay).
Step k processes timeslice (W + k) mod 32.  A correlator is one
(channel, timeslice): 64 spin components x 32^3 separations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on the host
cores on a bounded sample of the same workload, scaled to the same unit.
Under torchrun every rank runs its own 32^3 x 32 lattice (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_DEFAULT, T_DEFAULT, DECAY, SEED = 32, 32, 0.5, 1607
METRIC = "52-channel NBS correlators/sec/timeslice at 32^3"
UNIT = "correlators/s"
FP32_LANES, SM_MAX_MHZ = 128, 2070.0   # FP32 lanes per SM; the clock used when no sample is available
# DRAM bytes per momentum of the FP32 contraction kernels, from one ncu capture of
# `python bench.py --L 16 --T 2 --steps 1 --warmup 1 --e2e-steps 1 --no-cpu-baseline`
# (dram__bytes_read.sum + dram__bytes_write.sum over 4096 momenta); an entry is dropped
# whenever its kernel changes, until it is captured again
DRAM_BYTES_PER_Q = {"k_contract_qseg": 1.255847e9 / 4096, "k_contract_rows": 0.631365e9 / 4096,
                    "k_eff_rows": 0.900618e9 / 4096}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["fp32", "fp64", "bf16x3"], default="fp32")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--L", type=int, default=L_DEFAULT)
    ap.add_argument("--T", type=int, default=T_DEFAULT)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-legs", action="store_true",
                    help="skip the FP64 / split-BF16x3 timing and error legs of the FP32 line")
    ap.add_argument("--contract-cfg", type=int, default=0, help="NBS_PARAM_CONTRACT_CFG (kernel / launch shape)")
    ap.add_argument("--qblock", type=int, default=0, help="NBS_PARAM_CHUNK_QBLOCK (0 = library default)")
    ap.add_argument("--c64", action="store_true", help="store the propagators as complex64 (the 48^3 x 64 config)")
    ap.add_argument("--decay", type=float, default=DECAY)
    ap.add_argument("--autotune", action="store_true", help="pick the contraction shape with the autotuner first")
    ap.add_argument("--no-graphs", action="store_true", help="batched workload without CUDA graphs")
    ap.add_argument("--workload", choices=["single", "batched", "potential", "stream"], default="single",
                    help="batched: six configurations 2x16^3x32, 2x24^3x48, 2x32^3x32, every timeslice; "
                         "potential: the stencil from correlators to a local potential (nbs_potential); "
                         "stream: 48^3 x 64 with complex64 propagators streamed through HBM one timeslice at a "
                         "time and every correlator copied to pinned host memory")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ---- clocks during the timed region ---------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---- the CPU oracle arm ------------------------------------------------------------------

def oracle_sample_setup(L, seed=SEED, t=3):
    """Oracle state for the bounded sample: one 144-index topology of the pn channel at L^3."""
    import numpy as np
    import nbs_inputs as I
    from oracle import nbs_oracle as O
    Sl, Ss = I.propagator(seed, "l", L, t, DECAY), I.propagator(seed, "s", L, t, DECAY)
    props = {"u": Sl, "d": Sl, "s": Ss}
    blocks = O._Blocks(props)
    terms = O.topologies("p", "n", "p", "n")
    term = max(terms, key=O.xi_size)
    t0 = time.perf_counter()
    E1 = O.effective_block(term, 1, blocks)
    E2 = O.effective_block(term, 2, blocks)
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    return dict(O=O, E1=E1, E2=E2, term=term, L=L, rng=rng, setup_s=setup_s)


def oracle_cmac_per_correlator(L):
    """Complex multiply-adds of the oracle's direct sum for one correlator, averaged over the 52 channels
    (the oracle's own channel table: this arm never loads the library)."""
    from oracle import nbs_oracle as O
    names = O.channel_table()
    V = L ** 3
    tot = sum(sum(O.xi_size(t) for t in O.topologies(*ch)) for ch in names)
    return 64.0 * tot / len(names) * V * V


def oracle_step(st, n_r=1):
    """Direct sum of the sampled topology for n_r random separations; returns the CMAC done."""
    L = st["L"]
    rs = [tuple(int(v) for v in st["rng"].integers(0, L, 3)) for _ in range(n_r)]
    st["O"].direct_sum(st["E1"], st["E2"], L, rs, table_bytes=0)
    return 64.0 * st["O"].xi_size(st["term"]) * L ** 3 * n_r


def host_cores():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("internal_api") == "openblas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


def cpu_baseline(L, budget_s=15.0):
    st = oracle_sample_setup(L)
    cmac, el, n = 0.0, 0.0, 0
    t0 = time.perf_counter()
    while el < budget_s or n < 2:
        cmac += oracle_step(st)
        n += 1
        el = time.perf_counter() - t0
    rate = cmac / el
    per_corr = oracle_cmac_per_correlator(L)
    return {"value": rate / per_corr, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": ("FP64 oracle direct sum over X (O(V^2)) of the largest pn topology (|xi|=144) at %d^3, "
                       "%d separations r in %.1f s after %.1f s of block setup; %.3g CMAC/s scaled by the "
                       "oracle's CMAC per correlator averaged over the 52 channels (%.3g)"
                       % (L, n, el, st["setup_s"], rate, per_corr))}


def run_reference(args, rank):
    if rank != 0:
        return
    L = args.L
    st = oracle_sample_setup(L)
    per_corr = oracle_cmac_per_correlator(L)
    for _ in range(args.warmup):
        oracle_step(st)
    cmac = 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cmac += oracle_step(st)
    el = time.perf_counter() - t0
    value = cmac / el / per_corr
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "%d^3 x %d lattice, 52 channels, exp(-0.5 t) seeded propagators" % (L, args.T),
                       "precision": "fp64 oracle", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": "each step: oracle direct sum of the largest pn topology at one random r "
                                       "at %d^3, scaled by the oracle's CMAC per correlator (%.3g)" % (L, per_corr)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- host logic of the multi-rank (replica) path --------------------------------------------

def rank_seed(rank):
    """Seed of the lattice a rank processes: every rank runs its own configuration (weak scaling)."""
    return SEED + rank


def batched_seed(ci, rank, nconf=6):
    return 1608 + ci + nconf * rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of the ranks' values of x (the job ends when its slowest rank does)."""
    if dist is None:
        return float(x)
    import torch
    tt = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the max-over-ranks time."""
    return units_per_rank * world / seconds


# ---- the GPU arm ---------------------------------------------------------------------------

def make_props_host(L, T, seed, decay=DECAY, c64=False):
    import numpy as np
    import nbs_inputs as I
    dt = np.complex64 if c64 else np.complex128
    return [(I.propagator(seed, "l", L, t, decay).astype(dt), I.propagator(seed, "s", L, t, decay).astype(dt))
            for t in range(T)]


def contraction_flops(ids):
    from paper_1604_07983_gb300 import plan_tables
    tb = plan_tables(ids)
    return 8.0 * 64.0 * float(tb["terms"][:, 1].sum()), tb


def precision_legs(P, ctx, ids, T, out, t_err=12, steps64=3, steps16=8):
    """The second half of the metric on the same context and workload: per-channel normwise error of
    the FP32 and split-BF16x3 paths against the plain FP64 GPU path on one timeslice, and the device
    throughput of the FP64 and BF16x3 paths (each step one timeslice, all channels)."""
    import torch
    nch, V = len(ids), ctx.V
    t_err = t_err % T
    res = {}
    for name, mode in (("fp64", P.NBS_FP64), ("fp32", P.NBS_FP32), ("bf16x3", P.NBS_BF16X3)):
        ctx.set_precision(mode)
        o = torch.empty((nch, 1, 4, 4, 2, 2, V), dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, t_err, t_err + 1, o)
        res[name] = o.reshape(nch, -1)
    torch.cuda.synchronize()
    ref = res.pop("fp64")
    norm = torch.linalg.vector_norm(ref, dim=1)
    err = {k: (torch.linalg.vector_norm(v - ref, dim=1) / norm).cpu().tolist() for k, v in res.items()}
    del res, ref
    rates = {}
    for name, mode, steps, warm in (("fp64", P.NBS_FP64, steps64, 1), ("bf16x3", P.NBS_BF16X3, steps16, 2)):
        ctx.set_precision(mode)
        for k in range(warm):
            ctx.correlate(ids, k % T, k % T + 1, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            t = (warm + k) % T
            ctx.correlate(ids, t, t + 1, out)
        e1.record()
        torch.cuda.synchronize()
        rates[name] = (nch * steps / (e0.elapsed_time(e1) / 1e3), steps)
    ctx.set_precision(P.NBS_FP32)
    return err, rates, t_err


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_1604_07983_gb300 as P
    try:
        P.lib()
    except ImportError:
        from paper_1604_07983_gb300 import build as B
        B.build()
        P.lib()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    L, T = args.L, args.T
    V = L ** 3
    prec = {"fp32": P.NBS_FP32, "fp64": P.NBS_FP64, "bf16x3": P.NBS_BF16X3}[args.precision]
    ids = list(range(P.channel_count()))
    nch = len(ids)
    seed = rank_seed(rank)
    if args.workload == "batched":
        run_batched(args, rank, world, P, prec, ids, dist)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "potential":
        run_potential(args, rank, world, P, dist)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "stream":
        run_stream(args, rank, world, P, prec, ids, dist)
        if dist:
            dist.destroy_process_group()
        return
    host_props = make_props_host(L, T, seed, args.decay, args.c64)

    ctx = P.Context(L, T, precision=prec)
    ctx.set_param(ctx.PARAM_CONTRACT_CFG, args.contract_cfg)
    if args.qblock:
        ctx.set_param(ctx.PARAM_CHUNK_QBLOCK, args.qblock)
    for t, (Sl, Ss) in enumerate(host_props):
        ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), t)
    out = torch.empty((nch, 1, 4, 4, 2, 2, V), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    tuned = None
    if args.autotune:
        from paper_1604_07983_gb300 import autotune
        tuned = autotune.tune(ctx, ids, prec, t=0, use_cache=False)

    for k in range(args.warmup):
        ctx.correlate(ids, k % T, k % T + 1, out)
    torch.cuda.synchronize()

    ctx.set_profiling(True)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record()
        for k in range(args.steps):
            t = (args.warmup + k) % T
            ctx.correlate(ids, t, t + 1, out)
        stop.record()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda")
    stages, launches = ctx.profile()
    value = job_rate(nch * args.steps, world, ms / 1e3)

    # ---- end to end through the public API with host buffers ----
    # every step's propagators are copied in from pinned host memory (nbs_load_props), then one
    # nbs_correlate call over those timeslices writes every result to pinned host memory; inside
    # the call the copy-out of timeslice t overlaps the compute of t + 1
    e2e_steps = max(1, min(args.e2e_steps, args.steps, T))
    pin_u = [torch.from_numpy(Sl).pin_memory() for Sl, _ in host_props[:e2e_steps]]
    pin_s = [torch.from_numpy(Ss).pin_memory() for _, Ss in host_props[:e2e_steps]]
    out_h = torch.empty((nch, e2e_steps, 4, 4, 2, 2, V), dtype=torch.complex128).pin_memory()
    out_w = torch.empty((nch, 1, 4, 4, 2, 2, V), dtype=torch.complex128).pin_memory()
    ctx.set_profiling(False)
    ctx.load_props(pin_u[0], pin_s[0], 0)
    ctx.correlate(ids, 0, 1, out_w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # five repetitions of the whole sequence (load and correlate, each including its copies); the median
    # is reported, all five are listed
    reps = []
    for _ in range(5):
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            ctx.load_props(pin_u[k], pin_s[k], k)
        ctx.correlate(ids, 0, e2e_steps, out_h)
        torch.cuda.synchronize()
        reps.append(max_over_ranks(time.perf_counter() - t0, dist, "cuda"))
    e2e_s = sorted(reps)[len(reps) // 2]
    e2e_value = job_rate(nch * e2e_steps, world, e2e_s)
    e2e_reps = [job_rate(nch * e2e_steps, world, r) for r in reps]
    h2d = 2 * V * 144 * (8 if args.c64 else 16)
    d2h = nch * 64 * V * 16
    legs = None
    if world == 1 and prec == P.NBS_FP32 and not args.no_precision_legs:
        legs = precision_legs(P, ctx, ids, T, out)
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    ctx.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ----
    peaks = measured_peaks()
    fl, tb = contraction_flops(ids)
    flops_per_launch = fl * V
    ncomp = 4 * len(tb["cells"])
    csz = 16 if prec == P.NBS_FP64 else 8
    # stage "eff_rows" (the FP32 path's effective-block row kernel) is part of stage "contract"
    dominant = max((k for k in stages if k != "eff_rows"), key=lambda k: stages[k])
    per_launch_ms = {k: v / args.steps for k, v in stages.items()}
    rows_ms = per_launch_ms.get("eff_rows", 0.0)
    contract_ms = per_launch_ms["contract"] - rows_ms  # the product kernel alone
    if dominant == "contract" and prec == P.NBS_BF16X3:
        peak = peaks.get("bf16_tflops", 1900.0)
        ach = 3 * flops_per_launch / (per_launch_ms["contract"] / 1e3) / 1e12
        roof = {"kernel": "k_contract_tcq", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)" if "bf16_tflops" in peaks else "fallback",
                "work_per_launch": "3 bf16 products x 8 flop x 64 x sum|xi~| (=%d) x V complex MACs of Eq. (4.3)"
                                   % int(tb["terms"][:, 1].sum())}
    elif dominant == "contract":
        if prec == P.NBS_FP32:
            mhz = clocks.summary().get("sm_mhz") or SM_MAX_MHZ
            peak = n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12
            peak_src = ("derived, not measured: %d SMs (device) x %d FP32 lanes x 2 flop x %.0f MHz (median "
                        "sampled SM clock)" % (n_sm, FP32_LANES, mhz))
        else:
            peak = 1.25
            peak_src = "nominal GB300 FP64 1.25 TFLOP/s"
        ach = flops_per_launch / (contract_ms / 1e3) / 1e12
        cfg = tuned["cfg"] if tuned else args.contract_cfg
        kname = {0: "k_contract_rows", 4: "k_contract_qseg"}.get(cfg, "k_contract") if prec == P.NBS_FP32 else \
            "k_contract"
        traffic = None
        if kname in DRAM_BYTES_PER_Q and prec == P.NBS_FP32:
            traffic = DRAM_BYTES_PER_Q[kname] * V
        roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic, "traffic_unit": "DRAM bytes per launch",
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at 16^3, "
                                   "scaled by V" if traffic else None),
                "peak_source": peak_src,
                "work_per_launch": "8 flop x 64 x sum|xi~| (=%d) x V complex MACs of Eq. (4.3)"
                                   % int(tb["terms"][:, 1].sum())}
        if kname == "k_contract_rows" and tb.get("rows") is not None:
            # what the kernel issues: products of one channel that name the same two rows are merged, so it
            # runs fewer multiply-adds than the terms of Eq. (4.3) count (every record of every step, padding
            # records included, is a 4 x 4 complex outer product)
            nstep = int(sum(int(c[7]) for c in tb["rows"]["chunks"]))
            issued = 128.0 * 32 * nstep * V
            roof["issued"] = {"achieved": issued / (contract_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                              "work_per_launch": "8 flop x 16 x 32 records x %d steps x V" % nstep}
    else:
        hbm = peaks.get("hbm_gbs", 6800.0)
        if dominant == "fft_fwd":
            nbytes = 2.0 * ncomp * V * csz
        elif dominant == "fft_inv":
            nbytes = 2.0 * nch * 64 * V * csz
        elif dominant == "blocks":
            nbytes = ncomp * V * csz + 2 * 144 * V * csz
        else:
            nbytes = 2 * 144 * V * (16 + csz)
        ach = nbytes / (per_launch_ms[dominant] / 1e3) / 1e9
        roof = {"kernel": dominant, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    roof_rows = None
    if rows_ms > 0 and tb.get("rows") is not None:
        # effective-block rows (Eq. (4.2)): the stored blocks read once, the rows of every type written once
        nr = len(tb["rows"]["desc"])
        nbytes = V * (len(tb["cells"]) * 32.0 + nr * 32.0)
        hbm = peaks.get("hbm_gbs", 6800.0)
        ach = nbytes / (rows_ms / 1e3) / 1e9
        traffic = DRAM_BYTES_PER_Q.get("k_eff_rows", 0) * V or None
        roof_rows = {"kernel": "k_eff_rows", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm, "ms": rows_ms, "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at 16^3, "
                                       "scaled by V" if traffic else None,
                     "work_per_launch": "%d stored cells + %d rows x 32 bytes x V" % (len(tb["cells"]), nr),
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {P.NBS_FP32: "f32", P.NBS_FP64: "f64", P.NBS_BF16X3: "bf16x3"}[prec],
        "data": "synthetic seeded Gaussian propagators, exp(-0.5 t) decay",
        "config": {"workload": "%d^3 x %d lattice, all %d channels, one timeslice per step%s"
                               % (L, T, nch, ", complex64 propagator storage" if args.c64 else ""),
                   "precision": {P.NBS_FP32: "fp64 rescale -> fp32 blocks/FFT/contraction -> fp64 restore",
                                 P.NBS_FP64: "fp64",
                                 P.NBS_BF16X3: "fp64 rescale -> fp32 blocks/FFT -> split-bf16x3 tensor-core "
                                               "contraction (fp32 accumulate) -> fp64 restore"}[prec], "l2": "inputs larger than L2 (blocks %.2f GB/step)"
                   % (ncomp * V * csz / 1e9), "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": roof,
        "roofline_eff_rows": roof_rows,
        "stages_ms_per_step": {k: round(v, 4) for k, v in per_launch_ms.items()},
        "gpu_launches": int(launches),
        "contraction_shape": {"cfg": tuned["cfg"], "qb": tuned["qb"], "timings": tuned["timings"],
                              "fft_block": tuned["fft_block"], "fft_timings": tuned["fft_timings"]} if tuned else
                             {"cfg": args.contract_cfg, "qb": args.qblock},
        "clocks": clocks.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "repetitions": [round(x, 1) for x in e2e_reps], "reported": "median"},
    }
    if legs:
        err, rates, t_err = legs
        v64, v16 = rates["fp64"][0], rates["bf16x3"][0]
        line["fp64_value"] = v64
        line["mixed_over_fp64"] = value / v64
        line["bf16x3_value"] = v16
        line["bf16x3_over_fp64"] = v16 / v64
        line["error_vs_fp64"] = {
            "what": "normwise ||F - F_fp64|| / ||F_fp64|| per channel over all r and 64 spins, timeslice %d, "
                    "against the plain FP64 GPU path in this run" % t_err,
            "tolerance": 2e-5, "fp32_max": max(err["fp32"]), "bf16x3_max": max(err["bf16x3"]),
            "fp32_per_channel": [float("%.3g" % e) for e in err["fp32"]],
            "bf16x3_per_channel": [float("%.3g" % e) for e in err["bf16x3"]],
            "steps": {"fp64": rates["fp64"][1], "bf16x3": rates["bf16x3"][1]}}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(L)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


BATCH = [(16, 32), (16, 32), (24, 48), (24, 48), (32, 32), (32, 32)]


def run_batched(args, rank, world, P, prec, ids, dist=None):
    """Six configurations of uneven size (seeds 1608..1613), every timeslice of each, one
    context per configuration; a step is one timeslice of one configuration.  Each
    (configuration, timeslice) is captured once as a CUDA graph (nbs_graph_capture) and the
    timed region replays the 224 graphs back to back (--no-graphs: plain nbs_correlate calls)."""
    import torch
    nch = len(ids)
    ctxs, outs, jobs = [], [], []
    for ci, (L, T) in enumerate(BATCH):
        ctx = P.Context(L, T, precision=prec)
        ctx.set_param(ctx.PARAM_CONTRACT_CFG, args.contract_cfg)
        for t, (Sl, Ss) in enumerate(make_props_host(L, T, batched_seed(ci, rank), args.decay)):
            ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), t)
        ctxs.append(ctx)
        outs.append(torch.empty((nch, 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda"))
        jobs += [(ci, t) for t in range(T)]
    for ci in range(len(BATCH)):  # warm-up (allocates every buffer): one timeslice per configuration
        ctxs[ci].correlate(ids, 0, 1, outs[ci])
    graphs = None
    if not args.no_graphs:
        graphs = [ctxs[ci].capture(ids, t, t + 1, outs[ci]) for ci, t in jobs]
        for ci in range(len(BATCH)):
            graphs[jobs.index((ci, 0))].launch()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record()
        if graphs:
            for g in graphs:
                g.launch(wait=False)
        else:
            for ci, t in jobs:
                ctxs[ci].correlate(ids, t, t + 1, outs[ci])
        stop.record()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda")
    value = job_rate(nch * len(jobs), world, ms / 1e3)
    for c in ctxs:
        c.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC + " (batched: 2x16^3x32, 2x24^3x48, 2x32^3x32)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": len(jobs), "warmup": len(BATCH), "ms_per_step": ms / len(jobs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec != P.NBS_FP64 else "f64", "data": "synthetic, seeds 1608-1613",
            "config": {"workload": "6 configurations, %d timeslices, all %d channels" % (len(jobs), nch),
                       "launch": "one captured CUDA graph per (configuration, timeslice)" if graphs else
                                 "nbs_correlate per (configuration, timeslice)"},
            "gpu_launches": sum((9 if BATCH[ci][0] >= 16 and prec != P.NBS_FP64 else 11) for ci, _ in jobs),
            "clocks": clocks.summary()}), flush=True)


STREAM_L, STREAM_T, STREAM_DECAY, STREAM_SEED, STREAM_BASE = 48, 64, 0.4, 1614, 4


def run_stream(args, rank, world, P, prec, ids, dist=None):
    """The 48^3 x 64 configuration streamed: timeslice t's complex64 propagators are copied from pinned host
    memory into one of two propagator slots (nbs_load_props), its correlators for all channels computed and
    copied to pinned host memory (nbs_correlate with a host output) -- a step is one timeslice, the whole path
    including both copies, 64 steps in all, taken in pairs (one call over two propagator slots).  The host holds STREAM_BASE seeded timeslices (t = 0..3, decay
    exp(-0.4 t)) and timeslice t streams base t mod 4: generating all 64 at 48^3 would take minutes of host
    time, and every step moves and computes the same amount either way."""
    import numpy as np
    import torch
    L, T = STREAM_L, STREAM_T
    V = L ** 3
    nch = len(ids)
    seed = STREAM_SEED + 1000 * rank
    base = [(torch.from_numpy(I_prop(seed, "l", L, t, STREAM_DECAY).astype(np.complex64)).pin_memory(),
             torch.from_numpy(I_prop(seed, "s", L, t, STREAM_DECAY).astype(np.complex64)).pin_memory())
            for t in range(STREAM_BASE)]
    out = torch.empty((nch, 2, 4, 4, 2, 2, V), dtype=torch.complex128).pin_memory()
    ctx = P.Context(L, 2, precision=prec)
    ctx.set_param(ctx.PARAM_CONTRACT_CFG, args.contract_cfg)

    def pair(t):
        # timeslices t, t + 1 into the two slots, then one call over both: inside it the copy-out of the
        # first overlaps the compute of the second
        for k in range(2):
            u, s = base[(t + k) % STREAM_BASE]
            ctx.load_props(u, s, k)
        ctx.correlate(ids, 0, 2, out)
    for t in range(0, 2 * max(2, (args.warmup + 1) // 2), 2):
        pair(t)
    torch.cuda.synchronize()
    steps = T
    ctx.set_profiling(True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(0, steps, 2):
            pair(t)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if dist:
            dist.barrier()
    el = max_over_ranks(el, dist, "cuda")
    stages, launches = ctx.profile()
    ctx.close()
    h2d = 2 * V * 144 * 8
    d2h = nch * 64 * V * 16
    value = job_rate(nch * steps, world, el)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC.replace("32^3", "48^3") + " (48^3 x 64, propagators streamed)", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": 2 * max(2, (args.warmup + 1) // 2),
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {P.NBS_FP32: "f32", P.NBS_FP64: "f64", P.NBS_BF16X3: "bf16x3"}[prec],
            "data": "synthetic: %d seeded complex64 Gaussian timeslices with exp(-0.4 t) decay, timeslice t streams "
                    "base t mod %d" % (STREAM_BASE, STREAM_BASE),
            "config": {"workload": "48^3 x 64 lattice, all %d channels, one timeslice per step: H2D of its "
                                   "complex64 propagators (%.0f MB), the path, D2H of its complex128 correlators "
                                   "(%.2f GB) to pinned host memory" % (nch, h2d / 1e6, d2h / 1e9),
                       "timing": "host clock around the 64 steps (every copy inside), synchronised",
                       "l2": "inputs larger than L2"},
            "stages_ms_per_step": {k: round(v / steps, 4) for k, v in stages.items()},
            "gpu_launches": int(launches), "clocks": clocks.summary(),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}),
            flush=True)


def I_prop(seed, flavour, L, t, decay):
    import nbs_inputs as I
    return I.propagator(seed, flavour, L, t, decay)


def run_potential(args, rank, world, P, dist=None):
    """nbs_potential on the 52 x 64 correlator components of one timeslice at L^3 (FP64, three timeslices
    resident): 3 reads and 2 writes of 16 bytes per point, about 45 FP64 operations per point."""
    import torch
    L = args.L
    V = L ** 3
    n = 52 * 64
    g = torch.Generator(device="cuda").manual_seed(1763 + rank)
    R = [torch.randn((n, V), dtype=torch.complex128, device="cuda", generator=g) for _ in range(3)]
    for _ in range(args.warmup):
        P.potential(*R, L, 0.125, -1.0, 0.25)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record()
        for _ in range(args.steps):
            P.potential(*R, L, 0.125, -1.0, 0.25)
        stop.record()
        torch.cuda.synchronize()
    ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda") / args.steps
    nbytes = 5 * 16.0 * n * V
    gbs = nbytes / (ms / 1e3) / 1e9
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    # FP64 operations per point: Laplacian 14, time differences 6, combination 8, ratio K/R 17
    tflops = 45.0 * n * V / (ms / 1e3) / 1e12
    if rank == 0:
        print(json.dumps({
            "metric": "NBS potential stencil (K = a d_t^2 R + b d_t R + c lap R and K/R), points/s at %d^3" % L,
            "value": job_rate(n * V, world, ms / 1e3), "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic complex Gaussian cubes",
            "config": {"workload": "52 channels x 64 spin components, %d^3, one timeslice per step" % L},
            "roofline": {"kernel": "k_potential", "bound": "alu", "achieved": tflops, "peak": 1.25, "unit": "TFLOP/s",
                         "frac": tflops / 1.25, "traffic": None, "peak_source": "nominal GB300 FP64 1.25 TFLOP/s",
                         "work_per_launch": "45 FP64 operations x %d points" % (n * V),
                         "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                                 "bytes_per_launch": "3 reads + 2 writes x 16 B per point"}},
            "gpu_launches": args.steps, "clocks": clocks.summary()}), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
