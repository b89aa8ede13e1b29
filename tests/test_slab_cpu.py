"""The L-parallel path's layout and data movement on the CPU (no GPU).

The library gives each rank its z-planes and a y-set closed under y -> -y (mod L).  These tests check the
layout's invariants, and run the path's partition and transposes on world-size 2 and 3 gloo ranks: every
rank transforms its z-planes along x and y with numpy, packs the lines by the owner of their y (the index
map of the library's forward pack), exchanges them with all_to_all_single, unpacks by the owner of their z,
transforms along z -- and then holds exactly the full lattice's 3-D FFT on its momenta (every x and z, its
y-set), including -q of each of its q; the inverse runs the same way back to the z-planes.
"""

import os

import numpy as np
import pytest

nbs = pytest.importorskip("paper_1604_07983_gb300.nbs")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    try:
        return nbs.lib()
    except ImportError:
        pytest.skip("libnbs.so not built")


@pytest.mark.parametrize("L,P", [(2, 2), (3, 2), (4, 3), (8, 2), (8, 4), (12, 3), (16, 2), (16, 4), (24, 5),
                                 (32, 8), (48, 6)])
def test_layout_is_a_mirror_closed_partition(lib, L, P):
    zs, ys = [], []
    for r in range(P):
        zb, ze, y = nbs.slab_layout(L, P, r)
        assert zb == r * L // P and ze == (r + 1) * L // P and ze > zb
        assert y == sorted(y) and len(y) > 0
        assert set((L - v) % L for v in y) == set(y)      # closed under y -> -y
        zs.append((zb, ze))
        ys.append(y)
    assert sorted(v for y in ys for v in y) == list(range(L))
    sizes = [len(y) for y in ys]
    assert max(sizes) - min(sizes) <= 2


def test_layout_rejects_too_many_ranks(lib):
    with pytest.raises(nbs.NBSError):
        nbs.slab_layout(4, 4, 0)     # the units {0}, {2}, {1, 3}: three ranks at most
    with pytest.raises(nbs.NBSError):
        nbs.slab_layout(8, 2, 2)


# ---- the exchange on gloo ranks --------------------------------------------------------------------

def _offsets(counts):
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def _rank_main(rank, world, L, ncomp, port, errq):
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        lay = [nbs.slab_layout(L, world, p) for p in range(world)]
        zb, ze, ymine = lay[rank]
        lz = ze - zb
        ny = [len(l[2]) for l in lay]
        yowner = np.empty(L, int)
        yloc = np.empty(L, int)
        for p, (_, _, y) in enumerate(lay):
            yowner[y] = p
            yloc[y] = np.arange(len(y))
        rng = np.random.default_rng(5)
        full = rng.standard_normal((ncomp, L, L, L)) + 1j * rng.standard_normal((ncomp, L, L, L))   # [c][z][y][x]
        slab = full[:, zb:ze].copy()
        # x and y on the z-planes
        slab = np.fft.fft(np.fft.fft(slab, axis=3), axis=2)
        # forward pack: element (c, zl, y, x) -> block of y's owner d, [c][zl][yl_d][x]
        send_counts = [ncomp * lz * ny[d] * L for d in range(world)]
        off = _offsets(send_counts)
        send = np.empty(off[-1], complex)
        for c in range(ncomp):
            for zl in range(lz):
                for y in range(L):
                    d = yowner[y]
                    o = off[d] + ((c * lz + zl) * ny[d] + yloc[y]) * L
                    send[o:o + L] = slab[c, zl, y]
        recv_counts = [ncomp * (lay[s][1] - lay[s][0]) * ny[rank] * L for s in range(world)]
        recv = torch.empty(sum(recv_counts) * 2, dtype=torch.float64)
        dist.all_to_all_single(recv, torch.from_numpy(send.view(np.float64).copy()), [2 * n for n in recv_counts],
                               [2 * n for n in send_counts])
        recv = recv.numpy().view(complex)
        # forward unpack: element (c, z, yl, x) <- block of z's owner s, [c][zl][yl][x]
        roff = _offsets(recv_counts)
        mom = np.empty((ncomp, L, ny[rank], L), complex)
        for s in range(world):
            zbs, zes, _ = lay[s]
            blk = recv[roff[s]:roff[s + 1]].reshape(ncomp, zes - zbs, ny[rank], L)
            mom[:, zbs:zes] = blk
        mom = np.fft.fft(mom, axis=1)   # z
        want = np.fft.fftn(full, axes=(1, 2, 3))[:, :, ymine, :]
        assert np.abs(mom - want).max() <= 1e-10 * np.abs(want).max()
        # -q of every local q is local: (-z, -y, -x) of the full transform
        mir = [ymine.index((L - y) % L) for y in ymine]
        qm = mom[:, (-np.arange(L)) % L][:, :, mir][:, :, :, (-np.arange(L)) % L]
        wantm = np.fft.fftn(full, axes=(1, 2, 3))[:, (-np.arange(L)) % L][:, :, [(L - y) % L for y in ymine]]
        wantm = wantm[:, :, :, (-np.arange(L)) % L]
        assert np.abs(qm - wantm).max() <= 1e-10 * np.abs(want).max()
        # inverse: z on the y-set, pack by z's owner, exchange, unpack by y's owner, then y and x
        mom = np.fft.ifft(mom, axis=1)
        send2_counts = [ncomp * (lay[d][1] - lay[d][0]) * ny[rank] * L for d in range(world)]
        off2 = _offsets(send2_counts)
        send2 = np.empty(off2[-1], complex)
        for d in range(world):
            zbd, zed, _ = lay[d]
            send2[off2[d]:off2[d + 1]] = mom[:, zbd:zed].ravel()
        recv2_counts = [ncomp * lz * ny[s] * L for s in range(world)]
        recv2 = torch.empty(sum(recv2_counts) * 2, dtype=torch.float64)
        dist.all_to_all_single(recv2, torch.from_numpy(send2.view(np.float64).copy()), [2 * n for n in recv2_counts],
                               [2 * n for n in send2_counts])
        recv2 = recv2.numpy().view(complex)
        roff2 = _offsets(recv2_counts)
        back = np.empty((ncomp, lz, L, L), complex)
        for s in range(world):
            back[:, :, lay[s][2], :] = recv2[roff2[s]:roff2[s + 1]].reshape(ncomp, lz, ny[s], L)
        back = np.fft.ifft(np.fft.ifft(back, axis=2), axis=3)
        assert np.abs(back - full[:, zb:ze]).max() <= 1e-10 * np.abs(full).max()
        dist.destroy_process_group()
    except Exception as e:  # report to the parent
        errq.put("rank %d: %r" % (rank, e))
        raise


@pytest.mark.parametrize("world,L", [(2, 8), (3, 12)])
def test_partition_and_transposes_on_gloo_ranks(lib, world, L):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    errq = ctx.Queue()
    port = 29650 + world
    procs = [ctx.Process(target=_rank_main, args=(r, world, L, 3, port, errq)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    errs = []
    while not errq.empty():
        errs.append(errq.get())
    assert not errs, errs
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
