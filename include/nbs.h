/*
 * nbs.h -- C ABI of the GB300 library for octet-octet Nambu-Bethe-Salpeter
 * four-point correlators by the effective baryon block algorithm
 * (H. Nemura, arXiv:1604.07983, LATTICE 2015).
 *
 * Computes, for every requested channel <B1 B2 | B3bar B4bar> and timeslice t,
 *
 *   F_{a1 a2, a3 a4}(r, t) = sum_X < B1_a1(X + r, t) B2_a2(X, t) Jbar_{B3 a3, B4 a4}(t0) >
 *
 * (Sec. 2, first equation) from wall-source light (u = d) and strange quark
 * propagators (or separate u, d, s propagators: flavours = 3), following the
 * paper's pipeline: baryon blocks per site
 * (Eq. (4.1), Sec. 4 (i)), a forward 3-D FFT per block component (Eq. (2.6)),
 * effective blocks and their product in momentum space (Eqs. (4.2)-(4.3),
 * Sec. 4 (ii)-(iii)) and an inverse FFT.
 *
 * Conventions: Dirac representation with C gamma5 =
 * [[0,1,0,0],[-1,0,0,0],[0,0,0,1],[0,0,-1,0]]; source spins a3, a4 in {0,1}
 * (upper components) for channel ids below nbs_channel_count(), the other
 * three pairs for ids c + k nbs_channel_count() (k = 1, 2, 3; see
 * nbs_correlate); forward FFT e^{-iq.x} unnormalised, inverse
 * e^{+iq.r}/V; X + r periodic; site = x + L*(y + L*z).
 *
 * Errors: every call returns NBS_OK (0) or a negative NBS_E* code; the text of
 * the last error of a context is nbs_last_error().  No call aborts the process.
 * Threading: a context is used by one host thread at a time.
 * Memory: the context owns every device buffer it allocates (through the
 * allocator hook when one is installed, else cudaMalloc); callers own the
 * buffers they pass in.
 */
#ifndef NBS_H
#define NBS_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define NBS_OK        0
#define NBS_EINVAL   -1   /* bad argument (size, id, null pointer, range)      */
#define NBS_ENOMEM   -2   /* device or host allocation failed                   */
#define NBS_ECUDA    -3   /* a CUDA runtime call or kernel launch failed         */
#define NBS_ESTATE   -4   /* call out of order (e.g. no propagators for t)       */
#define NBS_ETIMEOUT -5   /* a bounded device wait gave up                       */
#define NBS_ENAN     -6   /* non-finite value in the propagators                 */

/* ---- precision modes (nbs_set_precision) ------------------------------- */
#define NBS_FP64   0   /* blocks, FFTs and contraction in complex FP64           */
#define NBS_FP32   1   /* FP64 rescale -> FP32 blocks/FFT/contraction -> FP64 restore */
#define NBS_BF16X3 2   /* as NBS_FP32, with the effective-block product on the tensor
                          cores: split-BF16 x 3 (hi*hi + hi*lo + lo*hi), FP32 accumulation */

/* ---- propagator element types (nbs_load_props) ------------------------- */
#define NBS_C128   0   /* interleaved complex double */
#define NBS_C64    1   /* interleaved complex float  */

/* ---- number of output spin components per (channel, t, r) -------------- */
#define NBS_NSPIN  64  /* a1 (4) x a2 (4) x a3 (2) x a4 (2) */

typedef struct nbs_ctx nbs_ctx;
typedef struct nbs_plan nbs_plan;
typedef struct nbs_graph nbs_graph;

/* Device allocator hook: alloc(bytes, user) returns a device pointer or NULL;
 * free(ptr, user).  Installed per process before nbs_create; NULL restores
 * cudaMalloc/cudaFree. */
typedef void* (*nbs_alloc_fn)(unsigned long long bytes, void* user);
typedef void (*nbs_free_fn)(void* ptr, void* user);
int nbs_set_allocator(nbs_alloc_fn alloc, nbs_free_fn free_fn, void* user);

/* Create a context for an L^3 x T lattice on the current CUDA device.
 * flavours: 2 = {light (u = d), strange} (isospin limit, Sec. 4 (i): the
 * blocks of n, Sigma-, Xi- are shared with p, Sigma+, Xi0); 3 = {u, d, s}
 * with u != d (every sink field gets its own stored blocks, propagators
 * loaded with nbs_load_props3); any other value is rejected with NBS_EINVAL.
 * 1 <= L <= 64, 1 <= T <= 4096.  Allocates the propagator store
 * (flavours x T timeslices). */
int nbs_create(nbs_ctx** out, int L, int T, int flavours);
/* Wait for the context's stream, then release every device and host buffer
 * of the context (propagator store, blocks, tables, the L-parallel buffers).
 * Graphs captured from it must be destroyed first.  NULL is a no-op. */
int nbs_destroy(nbs_ctx* h);

/* Select the arithmetic of the path (NBS_FP64 default, NBS_FP32 or NBS_BF16X3).
 * The paper computes in FP64 throughout (Sec. 3, Sec. 5); NBS_FP32 and
 * NBS_BF16X3 rescale each timeslice's propagators by a power of two in FP64
 * and undo it exactly in FP64 after the inverse FFT of Eq. (2.6).  Blocks
 * built in another mode are rebuilt by the next nbs_correlate; NBS_EINVAL
 * for another mode. */
int nbs_set_precision(nbs_ctx* h, int mode);

/* Run every later call of the context on this cudaStream_t (0 = legacy default). */
int nbs_set_stream(nbs_ctx* h, void* stream);

/* Copy one timeslice of the light (u) and strange (s) propagators into the
 * context: the wall-source quark propagators S(x, t; t0) from which the
 * blocks of Eq. (4.1) are built (Sec. 2; u = d in the isospin limit).  Layout of each: [z][y][x][i = 3*alpha + a][j = 3*alpha' + a'],
 * V*144 complex numbers of `dtype`; on_device selects device or host
 * pointers.  The library copies; the caller keeps ownership.  0 <= t < T.
 * A host copy is issued on the context's own load stream after the work
 * already enqueued on the context's stream, so that it overlaps the compute
 * of timeslices loaded before it; the blocks of t wait for it, and host
 * memory given to it must stay unchanged until the next nbs_correlate,
 * nbs_blocks or nbs_graph_launch (with wait) returns.  A device copy is
 * issued on the context's stream. */
int nbs_load_props(nbs_ctx* h, const void* u, const void* s, int t, int dtype, int on_device);
/* The same for a context with flavours = 3: the u, d and s propagators
 * (same layout and dtype).  NBS_EINVAL on a flavours = 2 context (and
 * nbs_load_props on a flavours = 3 one). */
int nbs_load_props3(nbs_ctx* h, const void* u, const void* d, const void* s, int t, int dtype, int on_device);

/* Build the momentum-space baryon blocks of timeslice t: per-timeslice
 * power-of-two rescale of the propagators, blocks of Eq. (4.1) for every
 * sink field, forward 3-D FFT of every component (Sec. 4 (i)).  Replaces the
 * blocks of any earlier timeslice.  NBS_ESTATE if no propagators for t. */
int nbs_blocks(nbs_ctx* h, int t);

/* Correlators of n_channels channels (ids of the built-in table, see
 * nbs_channel_info) for timeslices t_begin <= t < t_end.  For each t the
 * blocks are (re)built when needed, the effective blocks are formed and
 * multiplied in momentum space (Eqs. (4.2)-(4.3)), and the inverse FFT
 * gives F(r).  Source spins: id c (0 <= c < nbs_channel_count()) projects
 * them onto the upper components, alpha3, alpha4 in {0, 1}; id c + k *
 * nbs_channel_count() with k = 1, 2, 3 onto alpha3 in {2 (k & 1),
 * 2 (k & 1) + 1} and alpha4 in {2 (k >> 1), 2 (k >> 1) + 1}, so the four
 * ids c + k n cover the full 4 x 4 source spin of Eq. (2.4).
 * out: caller-allocated complex128
 *   [n_channels][t_end - t_begin][a1][a2][a3][a4][z][y][x]
 * (a3, a4 in {0, 1} relative to the id's source spin pair)
 * on the device (out_on_device = 1) or on the host (0; pinned memory is
 * copied asynchronously per timeslice).  Returns when `out` is complete.
 * NBS_ENAN if a propagator held a non-finite value; NBS_ETIMEOUT if a
 * bounded wait of the contraction on its TMA slab copies gave up (the
 * output is then incomplete; the context stays usable). */
int nbs_correlate(nbs_ctx* h, const int* channel_ids, int n_channels,
                  int t_begin, int t_end, void* out, int out_on_device);

/* CUDA-graph form of nbs_correlate for repeated work lists (the paper
 * launches the same kernels for every timeslice and configuration).
 * nbs_graph_capture records, without running it, the device work that
 * nbs_correlate(h, channel_ids, n_channels, t_begin, t_end, out, 1) would
 * do -- rescale, blocks, forward FFT, contraction, inverse FFT, restore for
 * every timeslice of the range -- into a CUDA graph that the context's stream
 * replays with nbs_graph_launch.  A replay reads the propagators loaded in
 * the context at that time (load new ones with nbs_load_props between
 * replays, same storage type) and writes the same device buffer `out`
 * (complex128, layout of nbs_correlate).  The caller owns the graph
 * (nbs_graph_destroy) and must destroy it before the context.
 * Preconditions: profiling off; propagators loaded for every t of the
 * range.  Every buffer the path needs is allocated before the capture.
 * nbs_graph_launch returns NBS_ESTATE if the context's buffers were
 * reallocated (a later call with more channels or another precision) or a
 * timeslice's storage type changed since the capture, NBS_ENAN after a
 * waited replay whose propagators held a non-finite value, NBS_ETIMEOUT
 * after a waited replay in which a contraction's slab wait gave up.  wait = 0 returns
 * after the launch; synchronise the context's stream before reading `out`. */
int nbs_graph_capture(nbs_ctx* h, const int* channel_ids, int n_channels, int t_begin, int t_end,
                      void* out, nbs_graph** graph);
int nbs_graph_launch(nbs_graph* graph, int wait);
int nbs_graph_destroy(nbs_graph* graph);

/* The stencil from NBS correlators to a local potential (the step that
 * Sec. 1 motivates: the potential follows from the NBS wave function).  For
 * n_components cubes R(r, t) (complex128, [component][z][y][x], periodic),
 * given at t - 1, t, t + 1, writes
 *   K = a (R(t+1) - 2 R(t) + R(t-1)) + b (R(t+1) - R(t-1)) / 2
 *     + c sum_{i=x,y,z} (R(r + e_i) + R(r - e_i) - 2 R(r))
 * and, if ratio_out is not NULL, K / R(t) (IEEE division: infinite or NaN
 * where R(t) = 0).  All pointers are device pointers; the caller normalises
 * R (e.g. by the single-baryon correlators) and picks a, b, c (for the
 * time-dependent method of the paper's Refs. [Ishii:2006ec, Aoki:2009ji]
 * they carry the reduced mass).  Runs on `stream` (a cudaStream_t, 0 for the
 * legacy default) and returns when K is written.  No context is needed. */
int nbs_potential(const void* r_prev, const void* r_cur, const void* r_next, int L, long long n_components,
                  double a, double b, double c, void* k_out, void* ratio_out, void* stream);

/* Zero-momentum projection of the last nbs_correlate's final timeslice,
 * sum_r F(r) = F~(q = 0), complex128 [n_channels][64] on the host. */
int nbs_zero_momentum(nbs_ctx* h, double* out);

/* Launch-shape parameters (for tuning; results agree to rounding).
 * NBS_PARAM_CONTRACT_CFG selects the contraction kernel:
 *   0 = default: in FP32, when its tables fit shared memory, the two-kernel
 *       row contraction (every distinct effective-block row of every stored
 *       type built once per momentum, Eq. (4.2), then per chunk of channels
 *       the 4 x 4 sink-spin outer products of each shared index and
 *       source-spin pair from bulk-copied rows, Eq. (4.3)), else config 4;
 *       in BF16X3 the quad-lane tensor-core form; in FP64 the
 *       thread-per-momentum kernel (A = 2, W = 1);
 *   4 = the quad-lane chunk kernel (FP32; persistent blocks of 16 warps,
 *       four lanes per shared index, one sink spin each, gathers straight
 *       from TMA-staged slabs; each warp walks its share of the steps as runs
 *       of one table run), else the default;
 *   A*10 + W = the thread-per-momentum kernel with A sink spins alpha1 per
 *       thread (1, 2 or 4) and W warps per block (1, 2 or 4); in FP32 also
 *       the kernel where neither the row nor the quad-lane tables fit.
 * In NBS_BF16X3 mode the quad-lane tensor-core kernel runs (fragments by
 * movmatrix, no shared-memory staging); a channel set whose tables do not fit
 * it is rejected with NBS_EINVAL.
 * NBS_EINVAL for any other value. */
#define NBS_PARAM_CONTRACT_CFG 0
/* NBS_PARAM_CHUNK_QBLOCK: momenta per block of the chunk contractions (default 32). */
#define NBS_PARAM_CHUNK_QBLOCK 1
/* NBS_PARAM_FFT_BLOCK: threads per block of the strided (y, z) passes of the
 * 3-D FFTs: 64, 128 (default) or 256. */
#define NBS_PARAM_FFT_BLOCK 2
/* NBS_PARAM_TEST_SKIP_SLAB (test switch, 0 by default): 1 makes the
 * TMA-staged quad-lane contraction (FP32, NBS_PARAM_CONTRACT_CFG 4) arm its
 * first slab wait in every block without issuing the copy, so that the
 * bounded wait runs out with no copy in flight and nbs_correlate (or a
 * waited nbs_graph_launch of a graph captured meanwhile) returns
 * NBS_ETIMEOUT; it exercises the failure path without a device fault.  Each
 * block waits about one second before it gives up.  (The default two-phase
 * kernel stages its slabs with cp.async gathers and has no bounded wait.) */
#define NBS_PARAM_TEST_SKIP_SLAB 3
int nbs_set_param(nbs_ctx* h, int param, int value);

/* Profiling (stage timing with CUDA events on the context's stream).
 * nbs_set_profiling(h, 1) clears the counters and records an event pair around
 * every stage of later calls; nbs_profile() returns the accumulated device
 * milliseconds per stage, stage_ms[NBS_NSTAGES] = {rescale (a0), blocks (a1),
 * forward FFT (a2), effective blocks + contraction (a3, a4), inverse FFT (a5),
 * restore + output copy (a5), effective-block rows (a3, where the FP32
 * two-phase contraction builds them in a kernel of their own; this time is
 * also part of stage 3)}, and the number of kernels launched. */
#define NBS_NSTAGES 7
int nbs_set_profiling(nbs_ctx* h, int on);
int nbs_profile(nbs_ctx* h, double* stage_ms, long long* launches);

/* Built-in channel table: the 52 octet-octet channels from NN to XiXi
 * (Sec. 1 and Sec. 4 (iii)), reconstructed as the sink x source pairs of
 * each strangeness sector at minimal |I3| without the four that vanish
 * identically for u = d. */
int nbs_channel_count(void);
/* Writes "B1 B2 | B3 B4" into buf (len bytes incl. NUL); returns the
 * number of light quarks n_l (n_s = 6 - n_l) or a negative error. */
int nbs_channel_info(int id, char* buf, int len);

/* Text of the last error on this context (or of the last context-less call
 * when h is NULL).  Never NULL. */
const char* nbs_last_error(const nbs_ctx* h);

/* ---- correlator without any device allocation ----------------------------
 * Not part of the paper's method (it has no counterpart there): an entry
 * point for callers that cannot call cudaMalloc -- a host application that
 * owns all device memory through its own pool, a process whose allocator is
 * locked, a loop that must not allocate.  It computes, in FP64, the
 * correlator of ONE built-in channel on ONE timeslice of an L^3 lattice with
 * L <= NBS_STATIC_MAX_L, exactly as nbs_correlate would, but every
 * intermediate buffer lives in one static device array of
 * NBS_STATIC_SCRATCH_BYTES bytes that each GPU loading the library keeps
 * until the process exits.
 *   u, s: device pointers, V*144 complex values of `dtype` each, layout as
 *         in nbs_load_props; out: device pointer, complex128 [a1][a2][a3][a4][V].
 *   stream: cudaStream_t (0 = legacy default).  Returns after `out` is written.
 * Errors: NBS_EINVAL for L > NBS_STATIC_MAX_L, an unknown channel or null
 * pointers (text in nbs_last_error(NULL)); NBS_ENAN; NBS_ECUDA.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and uploads the FFT twiddles; make that first call
 * before any stream capture.  That set-up is kept for the life of the
 * process: after cudaDeviceReset the entry is not usable again in the same
 * process.  Every call reuses the same array and leaves
 * its contents behind; calls that overlap on the GPU (other streams or host
 * threads) race on it and must be serialised by the caller. */
#define NBS_STATIC_MAX_L 4
#define NBS_STATIC_SCRATCH_BYTES 12582912
int nbs_correlate_static(const void* u, const void* s, int L, int dtype, int channel_id, void* out, void* stream);

/* ---- L-parallel path: the lattice split over ranks ------------------------
 * The paper's second parallelisation (Sec. 4 (i): the FFTs need an all-to-all
 * between the nodes that hold parts of the lattice; Sec. 5 compares it with
 * the T-parallel mode).  nranks ranks share one L^3 timeslice: rank r holds
 * the z-planes [z_begin, z_end) of the propagators (z0[p] = floor(p L /
 * nranks)) and, in momentum space, every z and x of a set of y values closed
 * under y -> -y (mod L), so that q and -q of each momentum it owns are local
 * and the contraction of Eq. (4.3) needs no exchange.  Per timeslice:
 *   1. nbs_slab_begin: max|S| of the rank's propagators -> maxbits[2] (bit
 *      patterns of the two maxima: the caller reduces them over the ranks with
 *      MAX, as 64-bit integers);
 *   2. nbs_slab_blocks(maxbits of all ranks): common power-of-two rescale,
 *      blocks of Eq. (4.1) on the rank's sites, FFT along x and y, packed into
 *      `send` for the forward exchange;
 *   3. the caller's all-to-all (send counts / receive counts per peer from
 *      nbs_slab_sizes, complex64 values, blocks of peer order);
 *   4. nbs_slab_contract(recv, send): FFT along z, the two-phase contraction on
 *      the rank's momenta, inverse FFT along z, packed for the inverse exchange;
 *   5. the caller's all-to-all (the correlator counts);
 *   6. nbs_slab_finish(recv, out): inverse FFT along y and x, FP64 restore:
 *      out = complex128 [n_channels][a1][a2][a3][a4][z_begin..z_end)[y][x],
 *      the rank's z-planes of F(r) (device pointer).
 * FP32 arithmetic (the two-phase contraction), two propagators (u = d, s).
 * All pointers are device pointers the caller owns; the propagators passed to
 * nbs_slab_begin must stay valid until nbs_slab_blocks returns.  Every call
 * returns after its device work; NBS_ENAN (begin) and NBS_ETIMEOUT (contract)
 * as for nbs_correlate. */
/* The layout of rank `rank` of nranks on an L^3 lattice: its z range and its
 * y values (ys must hold L ints).  Host only. */
int nbs_slab_layout(int L, int nranks, int rank, int* z_begin, int* z_end, int* ys, int* n_ys);
/* A context for rank `rank` of nranks for the given channels (ids as in
 * nbs_correlate); destroyed with nbs_destroy.  NBS_EINVAL where no layout
 * exists (each rank needs a z-plane and a y pair) or the two-phase tables do
 * not fit shared memory. */
int nbs_slab_create(nbs_ctx** out, int L, int nranks, int rank, const int* channel_ids, int n_channels);
/* Per-peer element counts (complex64 values) of the four exchange buffers:
 * forward send / receive (blocks), inverse send / receive (correlators); each
 * array has nranks entries (NULL to skip). */
int nbs_slab_sizes(const nbs_ctx* h, long long* send_blocks, long long* recv_blocks, long long* send_corr,
                   long long* recv_corr);
int nbs_slab_begin(nbs_ctx* h, const void* u, const void* s, int dtype, unsigned long long* maxbits);
int nbs_slab_blocks(nbs_ctx* h, const unsigned long long* maxbits, void* send);
int nbs_slab_contract(nbs_ctx* h, const void* recv, void* send);
int nbs_slab_finish(nbs_ctx* h, const void* recv, void* out);

/* ---- host-only introspection of the compiled channel tables ------------
 * nbs_plan_create runs the host "channel compiler" (Sec. 4 (ii)-(iii): the
 * diagrammatic classification done on the CPU and packed as structures of
 * arrays) for a channel list without touching a GPU.  Tests use it to check
 * the tables on the CPU.  nbs_plan_create_flavours compiles for 2 or 3
 * propagator flavours (nbs_create's meaning); nbs_plan_create uses 2. */
int nbs_plan_create(nbs_plan** out, const int* channel_ids, int n_channels);
int nbs_plan_create_flavours(nbs_plan** out, const int* channel_ids, int n_channels, int flavours);
int nbs_plan_destroy(nbs_plan* p);
/* sizes[0..NBS_PLAN_NSIZES-1]: see NBS_PS_* below */
#define NBS_PS_NTYPES     0   /* stored block types                          */
#define NBS_PS_NCELLS     1   /* total cells (components = 4 * cells)        */
#define NBS_PS_NTYPETERMS 2   /* recipe terms over all types                 */
#define NBS_PS_NTERMS     3   /* contraction terms                           */
#define NBS_PS_NENT1      4   /* side-1 gather entries                       */
#define NBS_PS_NENT2      5   /* side-2 gather entries                       */
#define NBS_PS_NCH        6   /* channels                                    */
#define NBS_PS_NGROUPS    7   /* slab groups                                 */
#define NBS_PS_NITEMS     8   /* slab work items                             */
#define NBS_PS_NCHUNKS    9   /* table chunks (0 when the chunk kernel cannot run) */
#define NBS_PS_NCHUNKTAB 10   /* 16-bit chunk-table entries                  */
#define NBS_PS_NCHUNKITEMS 11 /* chunk work items                            */
#define NBS_PLAN_NSIZES  12
int nbs_plan_sizes(const nbs_plan* p, long long* sizes);
/* what: NBS_PX_* ; dst must hold the documented number of int32/double */
#define NBS_PX_TYPES      0   /* int32 [ntypes][4]: cell_off, ncell, term_off, nterm   */
#define NBS_PX_TYPETERMS  1   /* int32 [nterms][4]: pattern, a0, a1, a2                */
#define NBS_PX_TYPECOEF   2   /* double [nterms]                                        */
#define NBS_PX_CELLS      3   /* int32 [ncells]: y0 + 12*y1 + 144*y2                    */
#define NBS_PX_TERMS      4   /* int32 [nterm][8]: ch, K, shape, n1, n2, off1, off2, slot in group */
#define NBS_PX_ENT1_CELL  5   /* int32 [nent1]  */
#define NBS_PX_ENT1_COEF  6   /* double [nent1] */
#define NBS_PX_ENT2_CELL  7   /* int32 [nent2]  */
#define NBS_PX_ENT2_COEF  8   /* double [nent2] */
#define NBS_PX_CHANNELS   9   /* int32 [nch][4]: term_begin, term_end, n_l, n_s         */
#define NBS_PX_GROUPS    10   /* int32 [ngroups][24]: base1, ncell1, base2, ncell2, ch_off, nch,
                                 item_off, nslot, warp_off[5], out_base[5], cfirst[4], 0, 0 */
#define NBS_PX_GROUPCH   11   /* int32 [sum of nch]: request-order channel of each group slot */
#define NBS_PX_ITEMS     12   /* int32 [nitems][2]: term, first shared index                 */
#define NBS_PX_CHUNKS    13   /* int32 [nchunks][40]: base1, ncell1, base2, ncell2, ch_off, nch,
                                 tab_off, tab_len, item_off, nslot, warp_off[9], out_base[9],
                                 cfirst[8], ch_local0, 0, 0, 0 */
#define NBS_PX_CHUNKTAB  14   /* uint16 [nchunktab]: cell - base | sign << 10 | code << 11   */
#define NBS_PX_CHUNKITEMS 15  /* int32 [nchunkitems][2]: term, first shared index            */
#define NBS_PX_TERMTABOFF 16  /* int32 [nterms][2]: side-1, side-2 offset in the chunk table */
#define NBS_PX_CODES     17   /* double [32]: |coefficient| of each code (code 31 = 0)       */
#define NBS_PX_QUADCHUNKS 18  /* int32 [nchunks][64]: the chunks split over the 16 warps of the
                                 quad-lane kernels: base1, ncell1, base2, ncell2, ch_off, nch,
                                 tab_off, tab_len, nslot, ch_local0, out_base[17], cfirst[16],
                                 seg_base[17] (warp w walks the quad segments seg_base[w] ..
                                 seg_base[w+1]), padding                                      */
#define NBS_PX_QUADSEGS  19   /* int32 [quad_chunks[nchunks-1].seg_base[16]][8]: per-warp runs of
                                 steps of one table run (a channel's terms of one fixed form,
                                 back to back, or one term): form (0..3 shape, 4..7 the fixed
                                 forms), side-1 and side-2 table offsets, first and end shared
                                 index, chunk-local channel, n1, n2                            */
#define NBS_PX_ROWCHUNKS 20   /* int32 [nchunks][96]: the product kernel's chunks: type1, type2, roff1,
                                 nrow1, roff2, nrow2, rec_off, nstep, ch_off, nch, nslot, seg_off, smem, 0,
                                 seg_base[W + 1], out_base[W + 1], cfirst[W], padding (W = the kernel's
                                 record-walking warps, NBS_PRS_WARPS)                                      */
#define NBS_PX_ROWENT    21   /* uint16: row entries, cell of the row's stored type (bits 0..11) | code
                                 (bits 12..13: +1, -1, +2, -2)                                             */
#define NBS_PX_ROWDESC   22   /* uint32 per row (all types, row order): entry offset (bits 0..23) |
                                 count << 24 | type << 29; padding rows have count 0                      */
#define NBS_PX_ROWREC    23   /* uint32 [step][4 g][8]: B1 row (bits 0..11, of type1) | B2 row << 12 (of
                                 type2) | scale code << 24; one record per distinct (s, B1 row, B2 row)
                                 of a channel, its scale the sum over the products that name them; four
                                 padding steps follow the last chunk                                      */
#define NBS_PX_ROWCH     24   /* int32: request-order channel of each chunk channel                       */
#define NBS_PX_ROWSEGS   25   /* int32 [nsegs][4]: first step, end step, chunk-local channel, lane-group
                                 map (records of lane group g, lanes 8 g + kq, are for output source-spin
                                 pair (map >> 2 g) & 3; bits 8 + 2 g: the group's turn among the groups
                                 of its s when the warp adds them into the slot, bits 16..18: the turns) */
#define NBS_PX_ROWSCALES 26   /* double [64]: the scale of each code (code 63 = 0)                          */
#define NBS_PX_ROWTYPES  27   /* int32 [ntypes][8]: stored type's first cell, cells, first row, rows, 0... */
int nbs_plan_export(const nbs_plan* p, int what, void* dst);
/* Sizes of the two-phase contraction's tables (the rows of the effective
 * blocks per stored type, Eq. (4.2), and the product records per chunk of
 * channels, Eq. (4.3)): sizes[0..NBS_PRS_N-1]. */
#define NBS_PRS_OK       0   /* 1 if every chunk fits a block's shared memory     */
#define NBS_PRS_NCHUNKS  1
#define NBS_PRS_NENT     2   /* row entries                                      */
#define NBS_PRS_NROWS    3   /* rows per momentum, all stored types              */
#define NBS_PRS_NREC     4
#define NBS_PRS_NCH      5
#define NBS_PRS_NSEGS    6
#define NBS_PRS_SMEM     7   /* the largest chunk's shared memory (bytes)        */
#define NBS_PRS_WARPS    8   /* record-walking (consumer) warps per block of the
                                product kernel; four helper warps copy the rows
                                and sum the slots                               */
#define NBS_PRS_NTYPES   9   /* stored types with rows                          */
#define NBS_PRS_N       10
int nbs_plan_row_sizes(const nbs_plan* p, long long* sizes);

#ifdef __cplusplus
}
#endif
#endif /* NBS_H */
