"""Write the oracle's expected values for the large-lattice GPU parity tests.

Calls only the FP64 CPU oracle (oracle/) and the seeded input generator
(nbs_inputs); nothing here touches the CUDA library.  The values are too slow
to recompute inside every GPU test run (the direct O(V^2) sum at 32^3 and 48^3
takes minutes per channel), so they are computed once here and stored:

  expected_32cube_t12.npz  32^3, seed 1607, timeslice 12, exp(-0.5 t) decay,
                           complex128 propagators (the metric's configuration)
  expected_48cube_t5.npz   48^3, seed 1614, timeslice 5, exp(-0.4 t) decay,
                           propagators rounded to complex64 (complex64 storage)

Each file holds, for the oracle's 52-channel table, the momentum projections
F~(q) = sum_r e^{-i q.r} F(r) at a few momenta (correlation theorem of
Eq. (2.6) on phase-weighted site sums of the normal blocks), and the direct
O(V^2) sum of the first equation of Sec. 2 at sampled separations r for a few
channels.

  python tests/golden/make_expected.py 32     # about 40 minutes on 8 cores (Lambda Lambda: 33)
  python tests/golden/make_expected.py 48     # about 12 minutes, 40 GB of memory
"""

from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import nbs_inputs as I  # noqa: E402
from oracle import nbs_oracle as O  # noqa: E402

CASES = {
    32: dict(seed=1607, t=12, decay=0.5, c64=False,
             n_list=[(0, 0, 0), (1, 0, 0), (16, 16, 16), (31, 31, 31), (5, 16, 27)],
             direct_ids=[0, 9, 24, 51], n_random_r=2,
             r_fixed=[(0, 0, 0), (1, 0, 0), (16, 16, 16)]),
    48: dict(seed=1614, t=5, decay=0.4, c64=True,
             n_list=[(0, 0, 0), (1, 0, 0), (24, 24, 24), (47, 47, 47), (7, 24, 41)],
             direct_ids=[0], n_random_r=1,
             r_fixed=[(24, 24, 24)]),
}


def path(L: int) -> str:
    c = CASES[L]
    return os.path.join(HERE, "expected_%dcube_t%d.npz" % (L, c["t"]))


def inputs(L: int):
    """The case's propagators as the GPU test loads them (complex64-rounded where the case stores c64)."""
    c = CASES[L]
    Sl = I.propagator(c["seed"], "l", L, c["t"], c["decay"])
    Ss = I.propagator(c["seed"], "s", L, c["t"], c["decay"])
    if c["c64"]:
        Sl = Sl.astype(np.complex64).astype(np.complex128)
        Ss = Ss.astype(np.complex64).astype(np.complex128)
    return Sl, Ss


def r_list(L: int):
    c = CASES[L]
    rng = np.random.default_rng(c["seed"])
    rs = list(c["r_fixed"])
    rs += [tuple(int(v) for v in rng.integers(0, L, 3)) for _ in range(c["n_random_r"])]
    return rs


def make(L: int) -> None:
    c = CASES[L]
    Sl, Ss = inputs(L)
    props = {"u": Sl, "d": Sl, "s": Ss}
    names = O.channel_table()
    t0 = time.time()
    sums = O.PhaseSums(props, L, c["n_list"])
    proj = np.array([O.momentum_projection(ch, sums, c["n_list"]) for ch in names])
    print("%d^3: momentum projections of %d channels in %.0f s" % (L, len(names), time.time() - t0), flush=True)
    del sums
    rs = r_list(L)
    direct = []
    for cid in c["direct_ids"]:
        t0 = time.time()
        direct.append(O.correlator(names[cid], props, L, rs))
        print("%d^3: direct sum of %s at %d separations in %.0f s" % (L, " ".join(names[cid]), len(rs),
                                                                      time.time() - t0), flush=True)
    np.savez(path(L), L=L, seed=c["seed"], t=c["t"], decay=c["decay"], c64=c["c64"],
             names=np.array([" ".join(ch) for ch in names]), n_list=np.array(c["n_list"]), proj=proj,
             direct_ids=np.array(c["direct_ids"]), r_list=np.array(rs), direct=np.array(direct))
    print("wrote", path(L), flush=True)


if __name__ == "__main__":
    for arg in sys.argv[1:]:
        make(int(arg))
