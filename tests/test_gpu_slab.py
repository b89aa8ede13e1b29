"""The L-parallel path (nbs_slab_*) on one GPU: the ranks run one after another in this process, each on its
own context, and their exchanges are device-to-device copies between their buffers (exactly what an
all-to-all delivers: from each source rank, in rank order, the block it addressed to the receiver).  No
kernel waits on another rank.  The assembled F(r) must equal the single-GPU FP32 path (the same FP32
arithmetic in another order) and the FP64 oracle.
"""

import numpy as np
import pytest

import nbs_inputs as I
from oracle import nbs_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def exchange(sends, counts):
    """recv[r] = the blocks sends[s] holds for r, for s in rank order (counts[s][r] values each)."""
    n = len(sends)
    offs = [np.concatenate([[0], np.cumsum(c)]) for c in counts]
    return [torch.cat([sends[s][int(offs[s][r]):int(offs[s][r + 1])] for s in range(n)]) for r in range(n)]


def slab_path(nbs, L, nranks, ids, Sl, Ss):
    """F [channel, 4, 4, 2, 2, V] through nranks L-parallel contexts on this GPU."""
    ctxs = [nbs.SlabContext(L, nranks, r, ids) for r in range(nranks)]
    try:
        props = []
        for c in ctxs:
            a, b = c.z_begin * L * L, c.z_end * L * L
            props.append((torch.from_numpy(Sl[a:b]).cuda(), torch.from_numpy(Ss[a:b]).cuda()))
        mb = np.maximum.reduce([c.begin(u, s) for c, (u, s) in zip(ctxs, props)])
        sends = [torch.empty(sum(c.send_blocks), dtype=torch.complex64, device="cuda") for c in ctxs]
        for c, buf in zip(ctxs, sends):
            c.blocks(mb, buf)
        recvs = exchange(sends, [c.send_blocks for c in ctxs])
        for c, buf in zip(ctxs, recvs):
            assert buf.numel() == sum(c.recv_blocks)
        sends2 = [torch.empty(sum(c.send_corr), dtype=torch.complex64, device="cuda") for c in ctxs]
        for c, rb, sb in zip(ctxs, recvs, sends2):
            c.contract(rb, sb)
        recvs2 = exchange(sends2, [c.send_corr for c in ctxs])
        outs = []
        for c, rb in zip(ctxs, recvs2):
            assert rb.numel() == sum(c.recv_corr)
            o = torch.empty((len(ids), 4, 4, 2, 2, c.z_end - c.z_begin, L, L), dtype=torch.complex128, device="cuda")
            c.finish(rb, o)
            outs.append(o)
        torch.cuda.synchronize()
        return torch.cat(outs, dim=5).reshape(len(ids), 4, 4, 2, 2, L ** 3).cpu().numpy()
    finally:
        for c in ctxs:
            c.close()


def single_gpu(nbs, L, ids, Sl, Ss):
    with nbs.Context(L, 1, precision=nbs.NBS_FP32) as ctx:
        ctx.load_props(torch.from_numpy(Sl).cuda(), torch.from_numpy(Ss).cuda(), 0)
        out = torch.empty((len(ids), 1, 4, 4, 2, 2, L ** 3), dtype=torch.complex128, device="cuda")
        ctx.correlate(ids, 0, 1, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()[:, 0]


@pytest.mark.parametrize("L,nranks,seed", [(8, 2, 1781), (12, 3, 1782), (16, 2, 1783), (16, 4, 1784)])
def test_slab_ranks_equal_the_single_gpu_path(nbs, L, nranks, seed):
    Sl, Ss = I.propagator(seed, "l", L, 2, 0.5), I.propagator(seed, "s", L, 2, 0.5)
    ids = list(range(nbs.channel_count()))
    F = slab_path(nbs, L, nranks, ids, Sl, Ss)
    G = single_gpu(nbs, L, ids, Sl, Ss)
    for c in ids:
        assert rel(F[c], G[c]) < 1e-5, (L, nranks, c)


def test_slab_ranks_against_the_oracle(nbs):
    L = 8
    Sl, Ss = I.propagator(1785, "l", L, 0), I.propagator(1785, "s", L, 0)
    names = nbs.channel_names()
    ids = [0, 9, 51]
    F = slab_path(nbs, L, 2, ids, Sl, Ss)
    props = {"u": Sl, "d": Sl, "s": Ss}
    for k, c in enumerate(ids):
        assert rel(F[k], O.correlator(names[c], props, L)) < FP32_TOL, names[c]
