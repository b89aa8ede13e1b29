"""Thin ctypes binding of the C ABI in include/nbs.h (argument marshalling only).

Every step of the correlator path runs in libnbs.so; this module only turns
Python/torch objects into pointers and sizes and raises on error codes.  If
the library is missing, importing the binding raises: there is no fallback.
PyTorch provides device memory (through the allocator hook) and streams.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbs.so")

NBS_OK, NBS_EINVAL, NBS_ENOMEM, NBS_ECUDA, NBS_ESTATE, NBS_ETIMEOUT, NBS_ENAN = 0, -1, -2, -3, -4, -5, -6
NBS_FP64, NBS_FP32, NBS_BF16X3 = 0, 1, 2
NBS_C128, NBS_C64 = 0, 1
NBS_NSPIN = 64
ERRORS = {NBS_EINVAL: "EINVAL", NBS_ENOMEM: "ENOMEM", NBS_ECUDA: "ECUDA", NBS_ESTATE: "ESTATE",
          NBS_ETIMEOUT: "ETIMEOUT", NBS_ENAN: "ENAN"}

#: every symbol include/nbs.h declares
EXPORTS = ["nbs_set_allocator", "nbs_create", "nbs_destroy", "nbs_set_precision", "nbs_set_stream",
           "nbs_load_props", "nbs_blocks", "nbs_correlate", "nbs_zero_momentum", "nbs_set_param", "nbs_set_profiling",
           "nbs_profile", "nbs_channel_count",
           "nbs_channel_info", "nbs_last_error", "nbs_plan_create", "nbs_plan_destroy", "nbs_plan_sizes",
           "nbs_plan_export", "nbs_correlate_static", "nbs_graph_capture", "nbs_graph_launch", "nbs_graph_destroy",
           "nbs_load_props3", "nbs_plan_create_flavours", "nbs_potential", "nbs_plan_row_sizes",
           "nbs_slab_layout", "nbs_slab_create", "nbs_slab_sizes", "nbs_slab_begin", "nbs_slab_blocks",
           "nbs_slab_contract", "nbs_slab_finish"]


class NBSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lib = None
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def lib():
    """The loaded libnbs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libnbs.so not built: run python -c 'import __graft_entry__ as g; g.build()'")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    sig = {
        "nbs_set_allocator": (i, [ALLOC_FN, FREE_FN, vp]),
        "nbs_create": (i, [ctypes.POINTER(vp), i, i, i]),
        "nbs_destroy": (i, [vp]),
        "nbs_set_precision": (i, [vp, i]),
        "nbs_set_stream": (i, [vp, vp]),
        "nbs_load_props": (i, [vp, vp, vp, i, i, i]),
        "nbs_blocks": (i, [vp, i]),
        "nbs_correlate": (i, [vp, ctypes.POINTER(i), i, i, i, vp, i]),
        "nbs_zero_momentum": (i, [vp, ctypes.POINTER(ctypes.c_double)]),
        "nbs_set_param": (i, [vp, i, i]),
        "nbs_set_profiling": (i, [vp, i]),
        "nbs_profile": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ll)]),
        "nbs_channel_count": (i, []),
        "nbs_channel_info": (i, [i, ctypes.c_char_p, i]),
        "nbs_last_error": (ctypes.c_char_p, [vp]),
        "nbs_plan_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(i), i]),
        "nbs_plan_destroy": (i, [vp]),
        "nbs_plan_sizes": (i, [vp, ctypes.POINTER(ll)]),
        "nbs_plan_row_sizes": (i, [vp, ctypes.POINTER(ll)]),
        "nbs_plan_export": (i, [vp, i, vp]),
        "nbs_correlate_static": (i, [vp, vp, i, i, i, vp, vp]),
        "nbs_graph_capture": (i, [vp, ctypes.POINTER(i), i, i, i, vp, ctypes.POINTER(vp)]),
        "nbs_graph_launch": (i, [vp, i]),
        "nbs_graph_destroy": (i, [vp]),
        "nbs_load_props3": (i, [vp, vp, vp, vp, i, i, i]),
        "nbs_plan_create_flavours": (i, [ctypes.POINTER(vp), ctypes.POINTER(i), i, i]),
        "nbs_potential": (i, [vp, vp, vp, i, ll, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, vp, vp]),
        "nbs_slab_layout": (i, [i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "nbs_slab_create": (i, [ctypes.POINTER(vp), i, i, i, ctypes.POINTER(i), i]),
        "nbs_slab_sizes": (i, [vp, ctypes.POINTER(ll), ctypes.POINTER(ll), ctypes.POINTER(ll), ctypes.POINTER(ll)]),
        "nbs_slab_begin": (i, [vp, vp, vp, i, ctypes.POINTER(ctypes.c_ulonglong)]),
        "nbs_slab_blocks": (i, [vp, ctypes.POINTER(ctypes.c_ulonglong), vp]),
        "nbs_slab_contract": (i, [vp, vp, vp]),
        "nbs_slab_finish": (i, [vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc, h=None):
    if rc != NBS_OK:
        msg = lib().nbs_last_error(h)
        raise NBSError(rc, msg.decode() if msg else "")
    return rc


# ---- channel table -----------------------------------------------------------

def channel_count() -> int:
    return lib().nbs_channel_count()


def channel_info(cid: int):
    """((B1, B2, B3, B4), n_light) of a built-in channel id."""
    buf = ctypes.create_string_buffer(128)
    nl = lib().nbs_channel_info(cid, buf, 128)
    _check(nl if nl < 0 else 0)
    sink, src = buf.value.decode().split("|")
    return tuple(sink.split()) + tuple(src.split()), nl


def channel_names():
    return [channel_info(c)[0] for c in range(channel_count())]


# ---- host-only plan introspection ---------------------------------------------

PX = dict(TYPES=0, TYPETERMS=1, TYPECOEF=2, CELLS=3, TERMS=4, ENT1_CELL=5, ENT1_COEF=6, ENT2_CELL=7,
          ENT2_COEF=8, CHANNELS=9, GROUPS=10, GROUPCH=11, ITEMS=12, CHUNKS=13, CHUNKTAB=14, CHUNKITEMS=15,
          QUADCHUNKS=18, QUADSEGS=19, ROWCHUNKS=20, ROWENT=21, ROWDESC=22, ROWREC=23, ROWCH=24, ROWSEGS=25,
          ROWSCALES=26, ROWTYPES=27,
          TERMTABOFF=16, CODES=17)


def plan_tables(channel_ids, flavours: int = 2):
    """Compile the channel tables on the host (2 or 3 propagator flavours) and return them as numpy arrays."""
    import numpy as np
    L = lib()
    ids = (ctypes.c_int * len(channel_ids))(*channel_ids)
    p = ctypes.c_void_p()
    _check(L.nbs_plan_create_flavours(ctypes.byref(p), ids, len(channel_ids), flavours))
    try:
        s = (ctypes.c_longlong * 12)()
        _check(L.nbs_plan_sizes(p, s))
        ntypes, ncells, ntt, nterm, ne1, ne2, nch, ngr, nit, nck, nctab, ncit = list(s)

        def get(what, shape, dtype):
            a = np.zeros(shape, dtype=dtype)
            _check(L.nbs_plan_export(p, PX[what], a.ctypes.data_as(ctypes.c_void_p)))
            return a

        return dict(
            types=get("TYPES", (ntypes, 4), np.int32), typeterms=get("TYPETERMS", (ntt, 4), np.int32),
            typecoef=get("TYPECOEF", (ntt,), np.float64), cells=get("CELLS", (ncells,), np.int32),
            terms=get("TERMS", (nterm, 8), np.int32), ent1_cell=get("ENT1_CELL", (ne1,), np.int32),
            ent1_coef=get("ENT1_COEF", (ne1,), np.float64), ent2_cell=get("ENT2_CELL", (ne2,), np.int32),
            ent2_coef=get("ENT2_COEF", (ne2,), np.float64), channels=get("CHANNELS", (nch, 4), np.int32),
            groups=get("GROUPS", (ngr, 24), np.int32), items=get("ITEMS", (nit, 2), np.int32),
            group_ch=get("GROUPCH", (nch,), np.int32), chunks=get("CHUNKS", (nck, 40), np.int32),
            quad_chunks=(qc := get("QUADCHUNKS", (nck, 64), np.int32)),
            quad_segs=get("QUADSEGS", (int(qc[-1, 43 + 16]) if nck else 0, 8), np.int32),
            chunk_tab=get("CHUNKTAB", (max(nctab, 1),), np.uint16), chunk_items=get("CHUNKITEMS", (ncit, 2), np.int32),
            term_tab_off=get("TERMTABOFF", (nterm, 2), np.int32), codes=get("CODES", (32,), np.float64),
            rows=row_tables(L, p, get))
    finally:
        L.nbs_plan_destroy(p)


def row_tables(L, p, get):
    """The two-phase contraction's tables (None where they do not fit shared memory)."""
    import numpy as np
    rs = (ctypes.c_longlong * 10)()
    _check(L.nbs_plan_row_sizes(p, rs))
    ok, nck, nent, nrows, nrec, nch, nseg, smem, warps, ntypes = list(rs)
    if not ok:
        return None
    return dict(warps=warps, chunks=get("ROWCHUNKS", (nck, 96), np.int32), ent=get("ROWENT", (max(nent, 1),), np.uint16),
                desc=get("ROWDESC", (max(nrows, 1),), np.uint32), rec=get("ROWREC", (max(nrec, 1),), np.uint32),
                ch=get("ROWCH", (max(nch, 1),), np.int32), segs=get("ROWSEGS", (max(nseg, 1), 4), np.int32),
                scales=get("ROWSCALES", (64,), np.float64), types=get("ROWTYPES", (max(ntypes, 1), 8), np.int32),
                smem=smem)


# ---- torch-backed device allocator -------------------------------------------

_alloc_refs = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    import torch

    def _a(nbytes, user):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:
            return None

    def _f(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_refs = (ALLOC_FN(_a), FREE_FN(_f))
    _check(lib().nbs_set_allocator(_alloc_refs[0], _alloc_refs[1], None))


# ---- correlator without device allocation ------------------------------------

STATIC_MAX_L = 4


def correlate_static(u, s, L: int, channel_id: int, out, stream=None):
    """One channel, one timeslice, FP64, L <= 4, every intermediate in the library's static device array.

    u, s: device tensors [V,12,12] (complex128 or complex64); out: device complex128 [4,4,2,2,V].
    """
    c64 = "complex64" in str(u.dtype)
    h = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().nbs_correlate_static(_ptr(u), _ptr(s), L, NBS_C64 if c64 else NBS_C128, channel_id, _ptr(out),
                                      ctypes.c_void_p(h)))
    return out


def full_spin_ids(channel_ids):
    """The ids that cover the full 4 x 4 source spin of the given channels: for each channel c the
    four source spin pairs c + k * channel_count(), k = o3 + 2 o4 (alpha3 in {2 o3, 2 o3 + 1},
    alpha4 in {2 o4, 2 o4 + 1}), in the order [k][channel]."""
    n = channel_count()
    return [c + k * n for k in range(4) for c in channel_ids]


def assemble_full_spin(out):
    """[4 * n, nt, 4, 4, 2, 2, V] (ids from full_spin_ids) -> [n, nt, 4, 4, 4, 4, V]
    (alpha1, alpha2, alpha3, alpha4)."""
    k4 = out.shape[0]
    n = k4 // 4
    parts = out.reshape((4, n) + tuple(out.shape[1:]))  # [k][c][t][a1][a2][j3][j4][V]
    shape = (n, out.shape[1], 4, 4, 4, 4, out.shape[-1])
    full = out.new_empty(shape) if hasattr(out, "new_empty") else __import__("numpy").empty(shape, out.dtype)
    for k in range(4):
        o3, o4 = k & 1, k >> 1
        full[:, :, :, :, 2 * o3:2 * o3 + 2, 2 * o4:2 * o4 + 2] = parts[k]
    return full


def potential(r_prev, r_cur, r_next, L: int, a: float, b: float, c: float, ratio: bool = True, stream=None):
    """nbs_potential on device complex128 tensors [..., L^3] (same shape): returns K (and K / R(t))."""
    import torch
    n = r_cur.numel() // (L ** 3)
    K = torch.empty_like(r_cur)
    P = torch.empty_like(r_cur) if ratio else None
    h = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().nbs_potential(_ptr(r_prev), _ptr(r_cur), _ptr(r_next), L, n, a, b, c, _ptr(K),
                               _ptr(P) if P is not None else None, ctypes.c_void_p(h)))
    return (K, P) if ratio else K


# ---- context -----------------------------------------------------------------

def _ptr(x):
    """Device or host address of a torch tensor or numpy array."""
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


class Context:
    """One L^3 x T lattice on the current CUDA device (nbs_create ... nbs_destroy)."""

    def __init__(self, L: int, T: int, flavours: int = 2, precision: int = NBS_FP64, stream=None):
        self._lib = lib()
        h = ctypes.c_void_p()
        _check(self._lib.nbs_create(ctypes.byref(h), L, T, flavours))
        self.h = h
        self.L, self.T, self.V = L, T, L ** 3
        self.set_precision(precision)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        for g in getattr(self, "_graphs", []):
            g.close()
        self._graphs = []
        if getattr(self, "h", None):
            self._lib.nbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_precision(self, mode: int):
        _check(self._lib.nbs_set_precision(self.h, mode), self.h)

    def set_stream(self, stream):
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(self._lib.nbs_set_stream(self.h, ctypes.c_void_p(handle)), self.h)

    def load_props(self, u, s, t: int):
        """u, s: complex128/complex64 [V,12,12] torch tensors (device or host) or numpy arrays (host)."""
        import numpy as np
        dt = str(getattr(u, "dtype", ""))
        c64 = "complex64" in dt
        on_dev = bool(getattr(u, "is_cuda", False))
        if not hasattr(u, "data_ptr"):
            u = np.ascontiguousarray(u)
            s = np.ascontiguousarray(s)
        _check(self._lib.nbs_load_props(self.h, _ptr(u), _ptr(s), t, NBS_C64 if c64 else NBS_C128, int(on_dev)),
               self.h)
        self._keep = (u, s)

    def load_props3(self, u, d, s, t: int):
        """u, d, s propagators (u != d) for a context created with flavours=3; arrays as in load_props."""
        import numpy as np
        c64 = "complex64" in str(getattr(u, "dtype", ""))
        on_dev = bool(getattr(u, "is_cuda", False))
        if not hasattr(u, "data_ptr"):
            u, d, s = (np.ascontiguousarray(x) for x in (u, d, s))
        _check(self._lib.nbs_load_props3(self.h, _ptr(u), _ptr(d), _ptr(s), t, NBS_C64 if c64 else NBS_C128,
                                         int(on_dev)), self.h)
        self._keep = (u, d, s)

    def blocks(self, t: int):
        _check(self._lib.nbs_blocks(self.h, t), self.h)

    def correlate(self, channel_ids, t_begin: int, t_end: int, out):
        """out: complex128 [n_ch, t_end - t_begin, 4, 4, 2, 2, V] (torch device tensor, or host tensor/array)."""
        ids = (ctypes.c_int * len(channel_ids))(*channel_ids)
        on_dev = bool(getattr(out, "is_cuda", False))
        _check(self._lib.nbs_correlate(self.h, ids, len(channel_ids), t_begin, t_end, _ptr(out), int(on_dev)),
               self.h)
        return out

    def capture(self, channel_ids, t_begin: int, t_end: int, out) -> "Graph":
        """CUDA graph of correlate(channel_ids, t_begin, t_end, out) for a device tensor out (nbs_graph_capture)."""
        if not getattr(out, "is_cuda", False):
            raise ValueError("graph capture needs a device output tensor")
        ids = (ctypes.c_int * len(channel_ids))(*channel_ids)
        g = ctypes.c_void_p()
        _check(self._lib.nbs_graph_capture(self.h, ids, len(channel_ids), t_begin, t_end, _ptr(out), ctypes.byref(g)),
               self.h)
        graph = Graph(self, g)
        if not hasattr(self, "_graphs"):
            self._graphs = []
        self._graphs.append(graph)
        return graph

    PARAM_CONTRACT_CFG = 0
    PARAM_CHUNK_QBLOCK = 1
    PARAM_FFT_BLOCK = 2

    def set_param(self, param: int, value: int):
        _check(self._lib.nbs_set_param(self.h, param, value), self.h)

    STAGES = ("rescale", "blocks", "fft_fwd", "contract", "fft_inv", "restore_copy", "eff_rows")

    def set_profiling(self, on: bool = True):
        _check(self._lib.nbs_set_profiling(self.h, int(on)), self.h)

    def profile(self):
        """(dict stage -> accumulated device ms, number of kernel launches)."""
        ms = (ctypes.c_double * 7)()
        n = ctypes.c_longlong()
        _check(self._lib.nbs_profile(self.h, ms, ctypes.byref(n)), self.h)
        return dict(zip(self.STAGES, list(ms))), n.value

    def zero_momentum(self, n_channels: int):
        import numpy as np
        out = np.zeros((n_channels, 4, 4, 2, 2), dtype=np.complex128)
        _check(self._lib.nbs_zero_momentum(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), self.h)
        return out


class Graph:
    """A captured correlator work list (nbs_graph_*); keeps its context alive."""

    def __init__(self, ctx: "Context", g):
        self.ctx, self.g = ctx, g

    def launch(self, wait: bool = True):
        if not self.g or not self.ctx.h:
            raise NBSError(-4, "graph or context closed")
        _check(self.ctx._lib.nbs_graph_launch(self.g, int(wait)), self.ctx.h)

    def close(self):
        if self.g:
            self.ctx._lib.nbs_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- L-parallel path (nbs_slab_*) ----------------------------------------------

def slab_layout(L: int, nranks: int, rank: int):
    """(z_begin, z_end, y values) of rank `rank` of nranks on an L^3 lattice (host only)."""
    zb, ze, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ys = (ctypes.c_int * max(L, 1))()
    _check(lib().nbs_slab_layout(L, nranks, rank, ctypes.byref(zb), ctypes.byref(ze), ys, ctypes.byref(n)))
    return zb.value, ze.value, list(ys[:n.value])


class SlabContext:
    """One rank of the L-parallel path (nbs_slab_create ... nbs_destroy): the steps of a timeslice, with the
    exchanges left to the caller (slab_correlate does them with torch.distributed)."""

    def __init__(self, L: int, nranks: int, rank: int, channel_ids):
        self._lib = lib()
        self.L, self.nranks, self.rank = L, nranks, rank
        self.ids = list(channel_ids)
        h = ctypes.c_void_p()
        ids = (ctypes.c_int * len(self.ids))(*self.ids)
        _check(self._lib.nbs_slab_create(ctypes.byref(h), L, nranks, rank, ids, len(self.ids)))
        self.h = h
        self.z_begin, self.z_end, self.ys = slab_layout(L, nranks, rank)
        c = [(ctypes.c_longlong * nranks)() for _ in range(4)]
        _check(self._lib.nbs_slab_sizes(self.h, *c), self.h)
        self.send_blocks, self.recv_blocks, self.send_corr, self.recv_corr = ([int(v) for v in a] for a in c)

    def close(self):
        if getattr(self, "h", None):
            self._lib.nbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def begin(self, u, s):
        """u, s: device tensors [sites of the rank's z-planes, 12, 12], complex128 or complex64; returns the two
        max|S| bit patterns (numpy uint64[2]) to be max-reduced over the ranks."""
        import numpy as np
        mb = (ctypes.c_ulonglong * 2)()
        c64 = "complex64" in str(u.dtype)
        _check(self._lib.nbs_slab_begin(self.h, _ptr(u), _ptr(s), NBS_C64 if c64 else NBS_C128, mb), self.h)
        self._keep = (u, s)
        return np.array([mb[0], mb[1]], dtype=np.uint64)

    def blocks(self, maxbits, send):
        """send: complex64 device tensor of sum(send_blocks) values."""
        mb = (ctypes.c_ulonglong * 2)(int(maxbits[0]), int(maxbits[1]))
        _check(self._lib.nbs_slab_blocks(self.h, mb, _ptr(send)), self.h)

    def contract(self, recv, send):
        _check(self._lib.nbs_slab_contract(self.h, _ptr(recv), _ptr(send)), self.h)

    def finish(self, recv, out):
        """out: complex128 device tensor [n_channels, 4, 4, 2, 2, z_end - z_begin, L, L]."""
        _check(self._lib.nbs_slab_finish(self.h, _ptr(recv), _ptr(out)), self.h)


def slab_correlate(ctx: SlabContext, u, s, out, group=None):
    """One timeslice of the L-parallel path on this rank, the exchanges done with torch.distributed (the
    default group, or `group`): MAX-reduce of the propagator maxima, two all-to-alls."""
    import numpy as np
    import torch
    import torch.distributed as dist
    mb = ctx.begin(u, s)
    m = torch.from_numpy(mb.astype(np.int64)).to(u.device)   # positive doubles order like their bit patterns
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    mb = m.cpu().numpy().astype(np.uint64)
    dev = u.device
    send = torch.empty(sum(ctx.send_blocks), dtype=torch.complex64, device=dev)
    recv = torch.empty(sum(ctx.recv_blocks), dtype=torch.complex64, device=dev)
    ctx.blocks(mb, send)
    dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), ctx.recv_blocks, ctx.send_blocks,
                           group=group)
    send2 = torch.empty(sum(ctx.send_corr), dtype=torch.complex64, device=dev)
    recv2 = torch.empty(sum(ctx.recv_corr), dtype=torch.complex64, device=dev)
    ctx.contract(recv, send2)
    dist.all_to_all_single(torch.view_as_real(recv2), torch.view_as_real(send2), ctx.recv_corr, ctx.send_corr,
                           group=group)
    ctx.finish(recv2, out)
    return out
