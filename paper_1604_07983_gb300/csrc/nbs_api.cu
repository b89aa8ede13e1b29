// nbs_api.cu -- the C ABI (include/nbs.h): context, memory, orchestration.
//
// Per timeslice the path is (arXiv:1604.07983, Sec. 4):
//   a0  max|S| per flavour -> power-of-two rescale + transpose       (kernels_blocks.cu)
//   a1  diquarks -> field blocks of Eq. (4.1)                        (kernels_blocks.cu)
//   a2  forward 3-D FFT of every block component                      (fft.cu)
//   a3+a4 effective blocks and their product in q-space, Eq. (4.3)    (kernels_contract.cu)
//   a5  inverse 3-D FFT, FP64 restore, copy to the caller             (fft.cu, kernels_contract.cu)
// all on one stream; host outputs leave through a second stream from two
// alternating staging buffers so that the copy of t overlaps work on t+1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nbs.h"
#include "common.cuh"
#include "plan.h"

using namespace nbs;

namespace {

nbs_alloc_fn g_alloc = nullptr;
nbs_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;
thread_local std::string g_err;

void* dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) return g_alloc((unsigned long long)bytes, g_alloc_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(void* p, nbs_free_fn f, void* user) {
  if (!p) return;
  if (f) f(p, user);
  else cudaFree(p);
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct nbs_plan {
  Plan plan;
};

struct nbs_ctx {
  int L = 0, T = 0, V = 0, device = 0;
  int nflav = 2;                 // propagators per timeslice: 2 (l = u = d, s) or 3 (u, d, s)
  unsigned buf_gen = 0;          // bumped by every device (re)allocation
  bool capturing = false;        // enqueueing into a CUDA graph: no allocation, no host synchronisation
  cudaStream_t gst = nullptr;    // capture stream
  int mode = NBS_FP64;
  cudaStream_t st = 0;
  cudaStream_t cst = nullptr;
  cudaEvent_t ev_done[2] = {nullptr, nullptr};   // staging buffer b copied out
  // host-to-device propagator loads run on their own stream, after everything already on st; the blocks of
  // timeslice t wait for ev_loaded[t] while load_pending[t] is set
  cudaStream_t lst = nullptr;
  cudaEvent_t ev_mark = nullptr;
  std::vector<cudaEvent_t> ev_loaded;
  std::vector<char> load_pending;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr};  // staging buffer b written
  std::string err;
  nbs_free_fn free_fn = nullptr;  // allocator at creation
  void* free_user = nullptr;

  DevBuf props;                 // [T][2][V*144] complex128 slots
  std::vector<signed char> have;  // -1 none, NBS_C128, NBS_C64
  DevBuf propsT, FB, Ft, zm, small;
  DevBuf stage[2];
  unsigned long long* maxbits = nullptr;  // [2]
  int* flags = nullptr;                   // [1]
  int* exps = nullptr;                    // [2]
  int* host_flags = nullptr;              // pinned copy of flags

  // compiled channel tables
  bool plan_ok = false;
  std::vector<int> plan_ids;
  Plan plan;
  int plan_gen = 0;
  DevBuf d_terms, d_chtb, d_chnl, d_e1, d_e2, d_cells, d_gch;
  DevBuf d_qchunks, d_qsegs, d_ctab, d_codes;
  int chunk_st1 = 0, chunk_st2 = 0, chunk_tab = 0, chunk_row = 0, quad_slot = 0;
  int chunk_qb = 32;
  DevBuf d_rchunks, d_rtypes, d_rdesc, d_rent, d_rrec, d_rsegs, d_rch, d_rscales;  // two-phase contraction tables
  DevBuf d_qlist;  // momenta in the product kernel's visiting order
  DevBuf RQ;       // effective-block rows of every stored type, momentum-major (FP32 two-phase path)
  int test_skip_slab = 0;  // NBS_PARAM_TEST_SKIP_SLAB (test switch)
  // one rank of the L-parallel path (nbs_slab_create): its z-planes, its mirror-closed y-set
  bool slab = false;
  SlabGeom sg;
  int srank = 0, slz = 0, sny = 0, snch = 0;
  long long svs = 0, svm = 0;       // sites of its z-planes, momenta of its y-set
  MomGeom smg;
  SlabOff soff[4];                  // send / receive offsets of the forward and the inverse exchange
  DevBuf s_FB, s_FBm, s_Ft, s_F;    // blocks [c][zl][y][x], [c][z][yl][x]; correlators [n][z][yl][x], [n][zl][y][x]
  const void* s_u = nullptr;        // the rank's propagators of the current timeslice (caller's)
  const void* s_s = nullptr;
  int s_c64 = 0;
  int fft_block = 128;  // NBS_PARAM_FFT_BLOCK
  int tables_mode = -1;
  TypeRecipeSet recipes;

  int blocks_t = -1, blocks_mode = -1, blocks_gen = -1;
  int last_nch = 0;
  int contract_cfg = 0;  // NBS_PARAM_CONTRACT_CFG, 0 = default
  int smem_optin = 0;    // the device's shared memory per block (opt-in)
  int nsm = 0;           // the device's multiprocessors

  // profiling: CUDA events around each stage, resolved after the final sync
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  double stage_ms[NBS_NSTAGES] = {};
  long long launches = 0;
};

namespace {

int fail(nbs_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

int cuda_fail(nbs_ctx* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(h, NBS_ECUDA, m);
}

cudaEvent_t prof_event(nbs_ctx* h) {
  if (h->evnext == h->evpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->evpool.push_back(e);
  }
  return h->evpool[h->evnext++];
}

// record the start of a stage; returns the event (or null when profiling is off)
cudaEvent_t stage_begin(nbs_ctx* h) {
  if (!h->prof) return nullptr;
  cudaEvent_t e = prof_event(h);
  if (e) cudaEventRecord(e, h->st);
  return e;
}
void stage_end(nbs_ctx* h, int stage, cudaEvent_t begin) {
  if (!h->prof || !begin) return;
  cudaEvent_t e = prof_event(h);
  if (!e) return;
  cudaEventRecord(e, h->st);
  h->marks.push_back({stage, {begin, e}});
}
// after a synchronisation: accumulate the stage times and recycle the events
void prof_resolve(nbs_ctx* h) {
  for (auto& m : h->marks) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, m.second.first, m.second.second) == cudaSuccess) h->stage_ms[m.first] += ms;
  }
  h->marks.clear();
  h->evnext = 0;
  cudaGetLastError();
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(h, _e, where); \
  } while (0)

int ensure(nbs_ctx* h, DevBuf& b, size_t bytes, const char* what) {
  if (b.bytes >= bytes && b.p) return NBS_OK;
  if (h->capturing)
    return fail(h, NBS_ESTATE, std::string("buffer for ") + what + " would be allocated while capturing");
  ++h->buf_gen;
  if (b.p) {
    cudaStreamSynchronize(h->st);
    dev_free(b.p, h->free_fn, h->free_user);
    b.p = nullptr;
    b.bytes = 0;
  }
  b.p = dev_alloc(bytes);
  if (!b.p) return fail(h, NBS_ENOMEM, std::string("cannot allocate ") + std::to_string(bytes) + " bytes for " + what);
  b.bytes = bytes;
  return NBS_OK;
}

// kernel launches of one 3-D FFT (fft.cu): x pass, then y and z fused for FP32 and L >= 16
int fft_passes(int L, bool f32) { return L == 1 ? 0 : (L >= 16 && f32 ? 2 : 3); }

// FP32 and BF16X3 share the FP32 blocks and FFTs
bool is_f32(int mode) { return mode == NBS_FP32 || mode == NBS_BF16X3; }

int upload_tables(nbs_ctx* h) {
  const Plan& P = h->plan;
  int rc;
  std::vector<DevTerm> terms(P.terms.size());
  for (size_t i = 0; i < P.terms.size(); ++i) {
    const TermHdr& t = P.terms[i];
    terms[i] = {t.ch, t.K, t.shape, t.n1, t.n2, t.off1, t.off2, t.pad};
  }
  if ((rc = ensure(h, h->d_gch, std::max<size_t>(P.group_ch.size(), 1) * sizeof(int), "group channels"))) return rc;
  if (P.chunks_ok) {
    h->chunk_st1 = h->chunk_st2 = h->chunk_tab = 0;
    for (const ChunkHdr& c : P.chunks) {
      h->chunk_st1 = std::max(h->chunk_st1, c.ncell1);
      h->chunk_st2 = std::max(h->chunk_st2, c.ncell2);
      h->chunk_tab = std::max(h->chunk_tab, c.tab_len);
    }
    h->quad_slot = 0;
    for (const QuadChunkHdr& c : P.quad_chunks) h->quad_slot = std::max(h->quad_slot, c.nslot);
    h->chunk_row = 0;
    for (const TermHdr& t : P.terms) {
      const int nh1 = 1 << ((t.shape & 1) + ((t.shape >> 1) & 1));
      h->chunk_row = std::max(h->chunk_row, std::max(t.n1 * nh1, t.n2 * (4 / nh1)));
    }
    float codes[32] = {};
    for (size_t i = 0; i < P.coef_codes.size() && i < 31; ++i) codes[i] = (float)P.coef_codes[i];
    if ((rc = ensure(h, h->d_qchunks, std::max<size_t>(P.quad_chunks.size(), 1) * sizeof(QuadChunkHdr), "quad chunks")))
      return rc;
    if ((rc = ensure(h, h->d_qsegs, std::max<size_t>(P.quad_segs.size(), 1) * sizeof(QuadSeg), "quad segments")))
      return rc;
    if ((rc = ensure(h, h->d_ctab, std::max<size_t>(P.chunk_tab.size(), 8) * 2, "chunk tables"))) return rc;
    if ((rc = ensure(h, h->d_codes, sizeof(codes), "coefficient codes"))) return rc;
    CK(cudaMemcpyAsync(h->d_qchunks.p, P.quad_chunks.data(), P.quad_chunks.size() * sizeof(QuadChunkHdr),
                       cudaMemcpyHostToDevice, h->st),
       "upload quad chunks");
    CK(cudaMemcpyAsync(h->d_qsegs.p, P.quad_segs.data(), P.quad_segs.size() * sizeof(QuadSeg), cudaMemcpyHostToDevice,
                       h->st),
       "upload quad segments");
    CK(cudaMemcpyAsync(h->d_ctab.p, P.chunk_tab.data(), P.chunk_tab.size() * 2, cudaMemcpyHostToDevice, h->st), "upload chunk tables");
    CK(cudaMemcpyAsync(h->d_codes.p, codes, sizeof(codes), cudaMemcpyHostToDevice, h->st), "upload codes");
    CK(cudaStreamSynchronize(h->st), "upload sync");
  }
  if (P.rows_ok) {
    float sc[NBS_ROW_SCALES];
    for (int i = 0; i < NBS_ROW_SCALES; ++i) sc[i] = (float)P.row_scales[i];
    if ((rc = ensure(h, h->d_rchunks, P.row_chunks.size() * sizeof(RowChunkHdr), "row chunks"))) return rc;
    if ((rc = ensure(h, h->d_rtypes, P.row_types.size() * sizeof(RowTypeHdr), "row types"))) return rc;
    if ((rc = ensure(h, h->d_rdesc, std::max<size_t>(P.row_desc.size(), 8) * 4, "row descriptors"))) return rc;
    if ((rc = ensure(h, h->d_rent, std::max<size_t>(P.row_ent.size(), 8) * 2, "row entries"))) return rc;
    if ((rc = ensure(h, h->d_rrec, std::max<size_t>(P.row_rec.size(), 32) * 4, "row records"))) return rc;
    if ((rc = ensure(h, h->d_rsegs, std::max<size_t>(P.row_segs.size(), 1) * sizeof(RowSeg), "row segments"))) return rc;
    if ((rc = ensure(h, h->d_rch, std::max<size_t>(P.row_ch.size(), 1) * sizeof(int), "row channels"))) return rc;
    if ((rc = ensure(h, h->d_rscales, sizeof(sc), "row scales"))) return rc;
    CK(cudaMemcpyAsync(h->d_rchunks.p, P.row_chunks.data(), P.row_chunks.size() * sizeof(RowChunkHdr),
                       cudaMemcpyHostToDevice, h->st), "upload row chunks");
    CK(cudaMemcpyAsync(h->d_rtypes.p, P.row_types.data(), P.row_types.size() * sizeof(RowTypeHdr),
                       cudaMemcpyHostToDevice, h->st), "upload row types");
    CK(cudaMemcpyAsync(h->d_rdesc.p, P.row_desc.data(), P.row_desc.size() * 4, cudaMemcpyHostToDevice, h->st),
       "upload row descriptors");
    CK(cudaMemcpyAsync(h->d_rent.p, P.row_ent.data(), P.row_ent.size() * 2, cudaMemcpyHostToDevice, h->st),
       "upload row entries");
    CK(cudaMemcpyAsync(h->d_rrec.p, P.row_rec.data(), P.row_rec.size() * 4, cudaMemcpyHostToDevice, h->st),
       "upload row records");
    CK(cudaMemcpyAsync(h->d_rsegs.p, P.row_segs.data(), P.row_segs.size() * sizeof(RowSeg), cudaMemcpyHostToDevice,
                       h->st), "upload row segments");
    CK(cudaMemcpyAsync(h->d_rch.p, P.row_ch.data(), P.row_ch.size() * sizeof(int), cudaMemcpyHostToDevice, h->st),
       "upload row channels");
    CK(cudaMemcpyAsync(h->d_rscales.p, sc, sizeof(sc), cudaMemcpyHostToDevice, h->st), "upload row scales");
    const std::vector<int2> qo = momentum_order(h->slab ? h->smg : full_geom(h->L));
    if (qo.empty()) return fail(h, NBS_EINVAL, "no momentum order for this geometry");
    if ((rc = ensure(h, h->d_qlist, qo.size() * sizeof(int2), "momentum order"))) return rc;
    CK(cudaMemcpyAsync(h->d_qlist.p, qo.data(), qo.size() * sizeof(int2), cudaMemcpyHostToDevice, h->st),
       "upload momentum order");
    CK(cudaStreamSynchronize(h->st), "upload sync");
  }
  CK(cudaMemcpyAsync(h->d_gch.p, P.group_ch.data(), P.group_ch.size() * sizeof(int), cudaMemcpyHostToDevice, h->st), "upload group channels");
  if ((rc = ensure(h, h->d_terms, std::max<size_t>(terms.size(), 1) * sizeof(DevTerm), "terms"))) return rc;
  if ((rc = ensure(h, h->d_chtb, P.ch_term_begin.size() * sizeof(int), "term ranges"))) return rc;
  if ((rc = ensure(h, h->d_chnl, std::max<size_t>(P.ch_fl.size(), 3) * sizeof(int), "flavour content"))) return rc;
  std::vector<int> cells(P.ncells);
  for (size_t ti = 0; ti < P.types.size(); ++ti) {
    const BlockType& bt = P.types[ti];
    for (int c = 0; c < bt.ncell; ++c) cells[bt.cell_off + c] = bt.cells[c] | ((int)ti << 11);
  }
  if ((rc = ensure(h, h->d_cells, std::max<size_t>(cells.size(), 1) * sizeof(int), "cells"))) return rc;
  CK(cudaMemcpyAsync(h->d_terms.p, terms.data(), terms.size() * sizeof(DevTerm), cudaMemcpyHostToDevice, h->st), "upload terms");
  CK(cudaMemcpyAsync(h->d_chtb.p, P.ch_term_begin.data(), P.ch_term_begin.size() * sizeof(int), cudaMemcpyHostToDevice, h->st), "upload ranges");
  CK(cudaMemcpyAsync(h->d_chnl.p, P.ch_fl.data(), P.ch_fl.size() * sizeof(int), cudaMemcpyHostToDevice, h->st),
     "upload flavour content");
  CK(cudaMemcpyAsync(h->d_cells.p, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice, h->st), "upload cells");
  std::memset(&h->recipes, 0, sizeof(h->recipes));
  if (P.types.size() > NBS_MAX_TYPES) return fail(h, NBS_EINVAL, "too many block types");
  for (size_t ti = 0; ti < P.types.size(); ++ti) {
    const BlockType& bt = P.types[ti];
    TypeRecipe& r = h->recipes.t[ti];
    if (bt.terms.size() > NBS_MAX_TYPE_TERMS) return fail(h, NBS_EINVAL, "block type with too many terms");
    r.nterms = (int)bt.terms.size();
    r.cell_off = bt.cell_off;
    r.ncell = bt.ncell;
    for (size_t k = 0; k < bt.terms.size(); ++k) {
      r.pat[k] = bt.terms[k].pat;
      r.arg[k] = bt.terms[k].a[0] | (bt.terms[k].a[1] << 2) | (bt.terms[k].a[2] << 4);
      r.coef[k] = bt.terms[k].c;
    }
  }
  // gather entries in the arithmetic of the current mode
  const size_t n1 = P.ent1_cell.size(), n2 = P.ent2_cell.size();
  if (is_f32(h->mode)) {
    std::vector<Ent<float>> a(n1), b(n2);
    for (size_t i = 0; i < n1; ++i) a[i] = {P.ent1_cell[i], (float)P.ent1_coef[i]};
    for (size_t i = 0; i < n2; ++i) b[i] = {P.ent2_cell[i], (float)P.ent2_coef[i]};
    if ((rc = ensure(h, h->d_e1, std::max<size_t>(n1, 1) * sizeof(Ent<float>), "gathers"))) return rc;
    if ((rc = ensure(h, h->d_e2, std::max<size_t>(n2, 1) * sizeof(Ent<float>), "gathers"))) return rc;
    CK(cudaMemcpyAsync(h->d_e1.p, a.data(), n1 * sizeof(Ent<float>), cudaMemcpyHostToDevice, h->st), "upload e1");
    CK(cudaMemcpyAsync(h->d_e2.p, b.data(), n2 * sizeof(Ent<float>), cudaMemcpyHostToDevice, h->st), "upload e2");
    CK(cudaStreamSynchronize(h->st), "upload sync");
  } else {
    std::vector<Ent<double>> a(n1), b(n2);
    for (size_t i = 0; i < n1; ++i) { a[i].cell = P.ent1_cell[i]; a[i].pad = 0; a[i].coef = P.ent1_coef[i]; }
    for (size_t i = 0; i < n2; ++i) { b[i].cell = P.ent2_cell[i]; b[i].pad = 0; b[i].coef = P.ent2_coef[i]; }
    if ((rc = ensure(h, h->d_e1, std::max<size_t>(n1, 1) * sizeof(Ent<double>), "gathers"))) return rc;
    if ((rc = ensure(h, h->d_e2, std::max<size_t>(n2, 1) * sizeof(Ent<double>), "gathers"))) return rc;
    CK(cudaMemcpyAsync(h->d_e1.p, a.data(), n1 * sizeof(Ent<double>), cudaMemcpyHostToDevice, h->st), "upload e1");
    CK(cudaMemcpyAsync(h->d_e2.p, b.data(), n2 * sizeof(Ent<double>), cudaMemcpyHostToDevice, h->st), "upload e2");
    CK(cudaStreamSynchronize(h->st), "upload sync");
  }
  h->tables_mode = h->mode;
  return NBS_OK;
}

int ensure_plan(nbs_ctx* h, const std::vector<int>& ids) {
  if (h->plan_ok && h->plan_ids == ids) {
    if (h->tables_mode != h->mode) return upload_tables(h);
    return NBS_OK;
  }
  std::string e = compile_plan(ids, h->plan, h->nflav);
  if (!e.empty()) {
    h->plan_ok = false;
    return fail(h, NBS_EINVAL, e);
  }
  h->plan_ids = ids;
  h->plan_ok = true;
  ++h->plan_gen;
  return upload_tables(h);
}

std::vector<int> all_channels() {
  std::vector<int> ids(channel_table().size());
  for (size_t i = 0; i < ids.size(); ++i) ids[i] = (int)i;
  return ids;
}

template <typename T>
int build_blocks(nbs_ctx* h, int t) {
  const int V = h->V;
  const Plan& P = h->plan;
  int rc;
  const int nf = h->nflav;
  if ((rc = ensure(h, h->propsT, (size_t)nf * 144 * V * sizeof(C<T>), "scaled propagators"))) return rc;
  if ((rc = ensure(h, h->FB, 4ull * P.ncells * V * sizeof(C<T>), "baryon blocks"))) return rc;
  const char* base = (const char*)h->props.p + (size_t)t * nf * V * 144 * sizeof(double2);
  if (h->load_pending[t]) {  // its propagators are still being copied in on the load stream
    CK(cudaStreamWaitEvent(h->st, h->ev_loaded[t], 0), "wait load");
    h->load_pending[t] = 0;
  }
  PropPtrs pp = {};
  for (int f = 0; f < nf; ++f) pp.p[f] = base + (size_t)f * V * 144 * sizeof(double2);
  const int c64 = h->have[t] == NBS_C64;
  cudaEvent_t e0 = stage_begin(h);
  CK(cudaMemsetAsync(h->small.p, 0, 32, h->st), "clear max|S|");  // the NaN flag accumulates over a call
  CK(launch_props_maxabs(pp, nf, c64, V, h->maxbits, h->flags, h->st), "max|S|");
  CK(launch_props_scale<T>(pp, nf, c64, V, h->maxbits, h->exps, (C<T>*)h->propsT.p, h->st), "rescale");
  stage_end(h, 0, e0);
  cudaEvent_t e1 = stage_begin(h);
  CK(launch_blocks_tiled<T>((const C<T>*)h->propsT.p, (const int*)h->d_cells.p, P.ncells, h->recipes, V, nf,
                            (C<T>*)h->FB.p, h->st),
     "diquarks and field blocks");
  stage_end(h, 1, e1);
  cudaEvent_t e2 = stage_begin(h);
  CK(fft3d_blocks<T>((C<T>*)h->FB.p, P.ncells, h->L, h->st, h->fft_block), "forward FFT");
  stage_end(h, 2, e2);
  h->launches += 3 + fft_passes(h->L, sizeof(T) == 4);  // max|S|, rescale, tiled blocks, forward FFT
  h->blocks_t = t;
  h->blocks_mode = h->mode;
  h->blocks_gen = h->plan_gen;
  return NBS_OK;
}

// every device buffer nbs_correlate(nch channels) needs, allocated now
// the two-phase FP32 contraction runs: FP32 mode, the default contraction, tables that fit the device
bool rows_path(const nbs_ctx* h) {
  return h->mode == NBS_FP32 && h->contract_cfg == 0 && h->plan.rows_ok && h->plan.row_smem <= h->smem_optin;
}

template <typename T>
int prepare(nbs_ctx* h, int nch) {
  const int V = h->V;
  int rc;
  if ((rc = ensure(h, h->propsT, (size_t)h->nflav * 144 * V * sizeof(C<T>), "scaled propagators"))) return rc;
  if ((rc = ensure(h, h->FB, 4ull * h->plan.ncells * V * sizeof(C<T>), "baryon blocks"))) return rc;
  if ((rc = ensure(h, h->Ft, (size_t)nch * 64 * V * sizeof(C<T>), "momentum-space correlators"))) return rc;
  if (sizeof(T) == 4 && rows_path(h) &&
      (rc = ensure(h, h->RQ, (size_t)V * h->plan.row_nr * 32, "effective-block rows")))
    return rc;
  return ensure(h, h->zm, (size_t)nch * 64 * sizeof(C<T>), "zero momentum");
}

template <typename T>
int correlate(nbs_ctx* h, int nch, int t0, int t1, void* out, int on_dev) {
  const int V = h->V;
  const long long nt = t1 - t0;
  int rc;
  if ((rc = ensure(h, h->Ft, (size_t)nch * 64 * V * sizeof(C<T>), "momentum-space correlators"))) return rc;
  if ((rc = ensure(h, h->zm, (size_t)nch * 64 * sizeof(C<T>), "zero momentum"))) return rc;
  if (sizeof(T) == 4 && rows_path(h) &&
      (rc = ensure(h, h->RQ, (size_t)V * h->plan.row_nr * 32, "effective-block rows")))
    return rc;
  const size_t per_t = (size_t)nch * 64 * V * sizeof(double2);
  CK(cudaMemsetAsync(h->flags, 0, sizeof(int), h->st), "clear NaN flag");
  if (!on_dev) {
    for (int b = 0; b < 2; ++b)
      if ((rc = ensure(h, h->stage[b], per_t, "output staging"))) return rc;
  }
  for (int t = t0; t < t1; ++t) {
    if (h->have[t] < 0) return fail(h, NBS_ESTATE, "no propagators loaded for timeslice " + std::to_string(t));
    if (h->capturing || !(h->blocks_t == t && h->blocks_mode == h->mode && h->blocks_gen == h->plan_gen)) {
      if ((rc = build_blocks<T>(h, t))) return rc;
    }
    cudaEvent_t e3 = stage_begin(h);
    // default in FP32: the quad-lane chunk kernel when the tables fit; FP64: the thread-per-momentum kernel
    const bool f32_chunks = sizeof(T) == 4 && h->plan.chunks_ok;
    // the quad-lane kernels: where their shared memory (table, slabs, slots, runs) fits the device
    const bool quad_fits = h->plan.chunks_ok &&
                           qseg_smem_bytes(h->quad_slot, h->chunk_tab, h->plan.max_quad_segs) <= (size_t)h->smem_optin &&
                           tcq_smem_bytes(h->quad_slot, h->chunk_tab, h->plan.max_quad_segs) <= (size_t)h->smem_optin;
    // the two-phase row kernel: FP32 default where its tables fit the device's shared memory
    const bool rows_fit = sizeof(T) == 4 && h->plan.rows_ok && h->plan.row_smem <= h->smem_optin;
    const bool use_rows = sizeof(T) == 4 && rows_path(h);
    const bool use_qseg = f32_chunks && quad_fits && (h->contract_cfg == 4 || (h->contract_cfg == 0 && !rows_fit));
    if (use_rows) {
      cudaEvent_t e6 = stage_begin(h);
      CK(launch_eff_rows((const float2*)h->FB.p, V, h->d_rtypes.p, (int)h->plan.row_types.size(),
                         (const unsigned*)h->d_rdesc.p, (const unsigned short*)h->d_rent.p,
                         (int)h->plan.row_ent.size(), h->plan.row_nr, (float2*)h->RQ.p, h->nsm, h->st),
         "effective-block rows");
      stage_end(h, 6, e6);
      CK(launch_contract_rows((const float2*)h->RQ.p, full_geom(h->L), h->plan.row_nr, (const int2*)h->d_qlist.p,
                              (int)h->plan.row_chunks.size(), h->chunk_qb, h->d_rchunks.p, (const unsigned*)h->d_rrec.p,
                              h->d_rsegs.p, (const int*)h->d_rch.p, (const float*)h->d_rscales.p, h->plan.row_smem,
                              (float2*)h->Ft.p, h->flags, h->st),
         "contraction (rows)");
    } else if (h->mode == NBS_BF16X3 && quad_fits && h->contract_cfg != 2) {
      CK(launch_contract_tcq((const float2*)h->FB.p, h->plan.ncells, h->L, (int)h->plan.quad_chunks.size(),
                             h->chunk_qb, h->d_qchunks.p, h->d_qsegs.p, h->plan.max_quad_segs,
                             (const int*)h->d_gch.p, (const unsigned short*)h->d_ctab.p, (const float*)h->d_codes.p,
                             std::max(h->chunk_st1, h->chunk_st2), h->quad_slot, h->chunk_tab, h->chunk_row,
                             (float2*)h->Ft.p, h->flags, h->st),
         "contraction (tensor cores)");
    } else if (h->mode == NBS_BF16X3) {
      return fail(h, NBS_EINVAL, "BF16X3 needs channel tables that fit the quad-lane kernel");
    } else if (use_qseg) {
      CK(launch_contract_qseg((const float2*)h->FB.p, h->plan.ncells, h->L, (int)h->plan.quad_chunks.size(),
                              h->chunk_qb, h->d_qchunks.p, h->d_qsegs.p, h->plan.max_quad_segs,
                              (const int*)h->d_gch.p, (const unsigned short*)h->d_ctab.p, (const float*)h->d_codes.p,
                              std::max(h->chunk_st1, h->chunk_st2), h->quad_slot, h->chunk_tab, h->chunk_row,
                              (float2*)h->Ft.p, h->flags, h->test_skip_slab, h->st),
         "contraction");
    } else {
      // the thread-per-momentum kernel: FP64, and FP32 where neither the row nor the quad-lane tables fit;
      // configs below 10 (0, 4) take its default shape
      const int cfg = h->contract_cfg < 10 ? 0 : h->contract_cfg;
      CK(launch_contract<T>((const C<T>*)h->FB.p, h->L, (const DevTerm*)h->d_terms.p, (const int*)h->d_chtb.p, nch,
                            (const Ent<T>*)h->d_e1.p, (const Ent<T>*)h->d_e2.p, (C<T>*)h->Ft.p, cfg, h->st),
         "contraction");
    }
    stage_end(h, 3, e3);
    h->launches += 1 + fft_passes(h->L, sizeof(T) == 4) + 1;  // contraction, inverse FFT, restore
    if (t == t1 - 1) {
      // F~(q = 0) of every (channel, spin) before the inverse transform
      CK(cudaMemcpy2DAsync(h->zm.p, sizeof(C<T>), h->Ft.p, (size_t)V * sizeof(C<T>), sizeof(C<T>), (size_t)nch * 64,
                           cudaMemcpyDeviceToDevice, h->st),
         "zero momentum");
    }
    cudaEvent_t e4 = stage_begin(h);
    CK(fft3d_inverse<T>((C<T>*)h->Ft.p, (long long)nch * 64, h->L, h->st, h->fft_block), "inverse FFT");
    stage_end(h, 4, e4);
    cudaEvent_t e5 = stage_begin(h);
    const long long tt = t - t0;
    if (on_dev) {
      double2* o = (double2*)out + tt * 64 * V;
      CK(launch_restore<T>((const C<T>*)h->Ft.p, V, nch, (const int*)h->d_chnl.p, h->exps, h->nflav, o, nt * 64 * V,
                           h->st),
         "restore");
    } else {
      const int b = (int)(tt & 1);
      if (tt >= 2) CK(cudaStreamWaitEvent(h->st, h->ev_done[b], 0), "wait staging");
      CK(launch_restore<T>((const C<T>*)h->Ft.p, V, nch, (const int*)h->d_chnl.p, h->exps, h->nflav,
                           (double2*)h->stage[b].p,
                           64LL * V, h->st),
         "restore");
      CK(cudaEventRecord(h->ev_ready[b], h->st), "event");
      CK(cudaStreamWaitEvent(h->cst, h->ev_ready[b], 0), "wait restore");
      char* dst = (char*)out + tt * 64 * V * sizeof(double2);
      CK(cudaMemcpy2DAsync(dst, (size_t)nt * 64 * V * sizeof(double2), h->stage[b].p, 64 * V * sizeof(double2),
                           64 * V * sizeof(double2), nch, cudaMemcpyDeviceToHost, h->cst),
         "copy out");
      CK(cudaEventRecord(h->ev_done[b], h->cst), "event");
    }
    stage_end(h, 5, e5);
  }
  CK(cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->st), "NaN flag");
  if (h->capturing) {  // a replay leaves other blocks behind than the ones last built here
    h->blocks_t = -1;
    h->last_nch = nch;
    return NBS_OK;
  }
  if (!on_dev) CK(cudaStreamSynchronize(h->cst), "copy sync");
  CK(cudaStreamSynchronize(h->st), "sync");
  CK(cudaStreamSynchronize(h->lst), "load sync");  // every load issued before the call has landed
  prof_resolve(h);
  if (*h->host_flags) {
    h->blocks_t = -1;
    if (*h->host_flags & 2) return fail(h, NBS_ETIMEOUT, "a bounded wait in the contraction gave up");
    return fail(h, NBS_ENAN, "non-finite value in the propagators");
  }
  h->last_nch = nch;
  return NBS_OK;
}

}  // namespace

void nbs::set_global_error(const std::string& msg) { g_err = msg; }

extern "C" {

int nbs_set_allocator(nbs_alloc_fn alloc, nbs_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(nullptr, NBS_EINVAL, "allocator needs both functions");
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return NBS_OK;
}

namespace {
int create_ctx(nbs_ctx** out, int L, int T, int flavours, bool store);
}

int nbs_create(nbs_ctx** out, int L, int T, int flavours) { return create_ctx(out, L, T, flavours, true); }

namespace {
// store: allocate the propagator store of T timeslices (the L-parallel ranks take the caller's)
int create_ctx(nbs_ctx** out, int L, int T, int flavours, bool store) {
  if (!out) return fail(nullptr, NBS_EINVAL, "null output pointer");
  *out = nullptr;
  if (flavours != 2 && flavours != 3)
    return fail(nullptr, NBS_EINVAL, "flavours must be 2 (light u = d, strange) or 3 (u, d, s)");
  if (L < 1 || L > 64 || !fft_supported(L))
    return fail(nullptr, NBS_EINVAL, "L must be one of 1 2 3 4 6 8 12 16 24 32 48");
  if (T < 1 || T > 4096) return fail(nullptr, NBS_EINVAL, "T must be in [1, 4096]");
  nbs_ctx* h = new nbs_ctx();
  h->L = L;
  h->T = T;
  h->V = L * L * L;
  h->nflav = flavours;
  h->free_fn = g_free;
  h->free_user = g_alloc_user;
  h->have.assign(T, -1);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "cudaGetDevice"); }
  if ((e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
    delete h;
    return cuda_fail(nullptr, e, "device attributes");
  }
  if ((e = fft_init()) != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "FFT twiddles"); }
  if ((e = cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking)) != cudaSuccess) {
    delete h;
    return cuda_fail(nullptr, e, "copy stream");
  }
  for (int b = 0; b < 2; ++b) {
    cudaEventCreateWithFlags(&h->ev_done[b], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&h->ev_ready[b], cudaEventDisableTiming);
  }
  if ((e = cudaStreamCreateWithFlags(&h->lst, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_mark, cudaEventDisableTiming)) != cudaSuccess) {
    nbs_destroy(h);
    return cuda_fail(nullptr, e, "load stream");
  }
  h->ev_loaded.assign(T, nullptr);
  h->load_pending.assign(T, 0);
  if (cudaMallocHost(&h->host_flags, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    nbs_destroy(h);
    return fail(nullptr, NBS_ENOMEM, "pinned flag");
  }
  *h->host_flags = 0;
  int rc = store ? ensure(h, h->props, (size_t)T * flavours * h->V * 144 * sizeof(double2), "propagator store") : 0;
  if (!rc) rc = ensure(h, h->small, 256, "scale scratch");
  if (rc) {
    std::string m = h->err;
    nbs_destroy(h);
    return fail(nullptr, rc, m);
  }
  h->maxbits = (unsigned long long*)h->small.p;  // one per flavour (<= 3)
  h->flags = (int*)((char*)h->small.p + 32);
  h->exps = (int*)((char*)h->small.p + 64);      // one per flavour
  *out = h;
  return NBS_OK;
}
}  // namespace

int nbs_destroy(nbs_ctx* h) {
  if (!h) return NBS_OK;
  cudaStreamSynchronize(h->st);
  if (h->cst) cudaStreamSynchronize(h->cst);
  if (h->lst) cudaStreamSynchronize(h->lst);
  DevBuf* bufs[] = {&h->props, &h->propsT, &h->FB, &h->Ft, &h->zm, &h->small, &h->stage[0], &h->stage[1],
                    &h->d_terms, &h->d_chtb, &h->d_chnl, &h->d_e1, &h->d_e2, &h->d_cells,
                    &h->d_gch, &h->d_qchunks, &h->d_qsegs, &h->d_ctab,
                    &h->d_codes, &h->d_rchunks, &h->d_rtypes, &h->d_rdesc, &h->d_rent, &h->d_rrec, &h->d_rsegs,
                    &h->d_rch, &h->d_rscales, &h->d_qlist, &h->RQ, &h->s_FB, &h->s_FBm, &h->s_Ft, &h->s_F};
  for (DevBuf* b : bufs) dev_free(b->p, h->free_fn, h->free_user);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    if (h->ev_done[b]) cudaEventDestroy(h->ev_done[b]);
    if (h->ev_ready[b]) cudaEventDestroy(h->ev_ready[b]);
  }
  if (h->cst) cudaStreamDestroy(h->cst);
  if (h->gst) cudaStreamDestroy(h->gst);
  for (cudaEvent_t e : h->ev_loaded)
    if (e) cudaEventDestroy(e);
  if (h->ev_mark) cudaEventDestroy(h->ev_mark);
  if (h->lst) cudaStreamDestroy(h->lst);
  if (h->host_flags) cudaFreeHost(h->host_flags);
  delete h;
  return NBS_OK;
}

int nbs_set_precision(nbs_ctx* h, int mode) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (mode != NBS_FP64 && mode != NBS_FP32 && mode != NBS_BF16X3) return fail(h, NBS_EINVAL, "unknown precision mode");
  h->mode = mode;
  return NBS_OK;
}

int nbs_set_stream(nbs_ctx* h, void* stream) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  h->st = (cudaStream_t)stream;
  return NBS_OK;
}

namespace {
int load_props(nbs_ctx* h, const void* const* src, int n, int t, int dtype, int on_device) {
  for (int f = 0; f < n; ++f)
    if (!src[f]) return fail(h, NBS_EINVAL, "null propagator pointer");
  if (t < 0 || t >= h->T) return fail(h, NBS_EINVAL, "timeslice out of range");
  if (dtype != NBS_C128 && dtype != NBS_C64) return fail(h, NBS_EINVAL, "dtype must be NBS_C128 or NBS_C64");
  const size_t bytes = (size_t)h->V * 144 * (dtype == NBS_C128 ? sizeof(double2) : sizeof(float2));
  char* base = (char*)h->props.p + (size_t)t * h->nflav * h->V * 144 * sizeof(double2);
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // from the host: on the load stream, after the work already on st (which may still read this slot), so
  // that the copies overlap the compute of the timeslices loaded before; from the device: on st itself
  // (the caller's producers of the source are ordered there)
  cudaStream_t ls = h->st;
  if (!on_device) {
    if (!h->ev_loaded[t]) CK(cudaEventCreateWithFlags(&h->ev_loaded[t], cudaEventDisableTiming), "load event");
    CK(cudaEventRecord(h->ev_mark, h->st), "load mark");
    CK(cudaStreamWaitEvent(h->lst, h->ev_mark, 0), "load after st");
    ls = h->lst;
  } else if (h->load_pending[t]) {  // a host load of this slot still in flight
    CK(cudaStreamWaitEvent(h->st, h->ev_loaded[t], 0), "wait load");
    h->load_pending[t] = 0;
  }
  for (int f = 0; f < n; ++f)
    CK(cudaMemcpyAsync(base + (size_t)f * h->V * 144 * sizeof(double2), src[f], bytes, k, ls), "copy propagator");
  if (!on_device) {
    CK(cudaEventRecord(h->ev_loaded[t], h->lst), "loaded");
    h->load_pending[t] = 1;
  }
  h->have[t] = (signed char)dtype;
  if (h->blocks_t == t) h->blocks_t = -1;
  return NBS_OK;
}
}  // namespace

int nbs_load_props(nbs_ctx* h, const void* u, const void* s, int t, int dtype, int on_device) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (h->nflav != 2) return fail(h, NBS_EINVAL, "a context with flavours = 3 takes nbs_load_props3");
  const void* src[2] = {u, s};
  return load_props(h, src, 2, t, dtype, on_device);
}

int nbs_load_props3(nbs_ctx* h, const void* u, const void* d, const void* s, int t, int dtype, int on_device) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (h->nflav != 3) return fail(h, NBS_EINVAL, "nbs_load_props3 needs a context created with flavours = 3");
  const void* src[3] = {u, d, s};
  return load_props(h, src, 3, t, dtype, on_device);
}

int nbs_blocks(nbs_ctx* h, int t) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (t < 0 || t >= h->T) return fail(h, NBS_EINVAL, "timeslice out of range");
  if (h->have[t] < 0) return fail(h, NBS_ESTATE, "no propagators loaded for timeslice " + std::to_string(t));
  int rc;
  if (!h->plan_ok && (rc = ensure_plan(h, all_channels()))) return rc;
  if (h->tables_mode != h->mode && (rc = upload_tables(h))) return rc;
  CK(cudaMemsetAsync(h->flags, 0, sizeof(int), h->st), "clear NaN flag");
  rc = is_f32(h->mode) ? build_blocks<float>(h, t) : build_blocks<double>(h, t);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->st), "NaN flag");
  CK(cudaStreamSynchronize(h->st), "sync");
  CK(cudaStreamSynchronize(h->lst), "load sync");
  prof_resolve(h);
  if (*h->host_flags) {
    h->blocks_t = -1;
    return fail(h, NBS_ENAN, "non-finite value in the propagators");
  }
  return NBS_OK;
}

int nbs_correlate(nbs_ctx* h, const int* channel_ids, int n_channels, int t_begin, int t_end, void* out,
                  int out_on_device) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (!channel_ids || n_channels < 1 || n_channels > 65535) return fail(h, NBS_EINVAL, "bad channel list");
  if (t_begin < 0 || t_end > h->T || t_begin >= t_end) return fail(h, NBS_EINVAL, "bad timeslice range");
  if (!out) return fail(h, NBS_EINVAL, "null output");
  std::vector<int> ids(channel_ids, channel_ids + n_channels);
  int rc = ensure_plan(h, ids);
  if (rc) return rc;
  return is_f32(h->mode) ? correlate<float>(h, n_channels, t_begin, t_end, out, out_on_device)
                         : correlate<double>(h, n_channels, t_begin, t_end, out, out_on_device);
}

struct nbs_graph {
  nbs_ctx* h = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned buf_gen = 0;
  int mode = 0, t0 = 0, t1 = 0;
  std::vector<signed char> have;  // propagator storage types of [t0, t1) at capture
};

int nbs_graph_capture(nbs_ctx* h, const int* channel_ids, int n_channels, int t_begin, int t_end, void* out,
                      nbs_graph** graph) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (!graph) return fail(h, NBS_EINVAL, "null graph pointer");
  *graph = nullptr;
  if (!channel_ids || n_channels < 1 || n_channels > 65535) return fail(h, NBS_EINVAL, "bad channel list");
  if (t_begin < 0 || t_end > h->T || t_begin >= t_end) return fail(h, NBS_EINVAL, "bad timeslice range");
  if (!out) return fail(h, NBS_EINVAL, "null output");
  if (h->prof) return fail(h, NBS_EINVAL, "profiling must be off while capturing");
  for (int t = t_begin; t < t_end; ++t)
    if (h->have[t] < 0) return fail(h, NBS_ESTATE, "no propagators loaded for timeslice " + std::to_string(t));
  std::vector<int> ids(channel_ids, channel_ids + n_channels);
  int rc = ensure_plan(h, ids);
  if (!rc) rc = is_f32(h->mode) ? prepare<float>(h, n_channels) : prepare<double>(h, n_channels);
  if (rc) return rc;
  cudaError_t e;
  if (!h->gst && (e = cudaStreamCreateWithFlags(&h->gst, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(h, e, "capture stream");
  CK(cudaStreamSynchronize(h->st), "sync before capture");
  CK(cudaStreamSynchronize(h->lst), "loads before capture");  // no wait on a load event inside the capture
  std::fill(h->load_pending.begin(), h->load_pending.end(), 0);
  cudaStream_t user = h->st;
  h->st = h->gst;
  if ((e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
    h->st = user;
    return cuda_fail(h, e, "begin capture");
  }
  h->capturing = true;
  rc = is_f32(h->mode) ? correlate<float>(h, n_channels, t_begin, t_end, out, 1)
                       : correlate<double>(h, n_channels, t_begin, t_end, out, 1);
  h->capturing = false;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(h->st, &g);
  h->st = user;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "instantiate graph");
  nbs_graph* G = new nbs_graph();
  G->h = h;
  G->exec = exec;
  G->buf_gen = h->buf_gen;
  G->mode = h->mode;
  G->t0 = t_begin;
  G->t1 = t_end;
  G->have.assign(h->have.begin() + t_begin, h->have.begin() + t_end);
  *graph = G;
  return NBS_OK;
}

int nbs_graph_launch(nbs_graph* graph, int wait) {
  if (!graph || !graph->h) return fail(nullptr, NBS_EINVAL, "null graph");
  nbs_ctx* h = graph->h;
  if (graph->buf_gen != h->buf_gen || graph->mode != h->mode)
    return fail(h, NBS_ESTATE, "the context's buffers or precision changed since the capture; capture again");
  for (int t = graph->t0; t < graph->t1; ++t)
    if (h->have[t] != graph->have[t - graph->t0])
      return fail(h, NBS_ESTATE, "propagator storage of timeslice " + std::to_string(t) + " changed since the capture");
  *h->host_flags = 0;
  for (int t = graph->t0; t < graph->t1; ++t)  // propagators loaded since the capture
    if (h->load_pending[t]) {
      CK(cudaStreamWaitEvent(h->st, h->ev_loaded[t], 0), "wait load");
      h->load_pending[t] = 0;
    }
  CK(cudaGraphLaunch(graph->exec, h->st), "graph launch");
  h->blocks_t = -1;
  if (!wait) return NBS_OK;
  CK(cudaStreamSynchronize(h->st), "sync");
  CK(cudaStreamSynchronize(h->lst), "load sync");
  if (*h->host_flags & 2) return fail(h, NBS_ETIMEOUT, "a slab copy wait in the contraction gave up");
  if (*h->host_flags) return fail(h, NBS_ENAN, "non-finite value in the propagators");
  return NBS_OK;
}

int nbs_graph_destroy(nbs_graph* graph) {
  if (!graph) return NBS_OK;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  delete graph;
  return NBS_OK;
}

int nbs_potential(const void* r_prev, const void* r_cur, const void* r_next, int L, long long n_components, double a,
                  double b, double c, void* k_out, void* ratio_out, void* stream) {
  if (!r_prev || !r_cur || !r_next || !k_out) return fail(nullptr, NBS_EINVAL, "null array");
  if (L < 1 || L > 64) return fail(nullptr, NBS_EINVAL, "L must be in [1, 64]");
  if (n_components < 0 || n_components > (1LL << 40) / ((long long)L * L * L))
    return fail(nullptr, NBS_EINVAL, "bad number of components");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_potential((const double2*)r_prev, (const double2*)r_cur, (const double2*)r_next, L,
                                   n_components, a, b, c, (double2*)k_out, (double2*)ratio_out, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "potential stencil");
  return NBS_OK;
}

int nbs_set_param(nbs_ctx* h, int param, int value) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  switch (param) {
    case NBS_PARAM_CONTRACT_CFG: {
      const int a = value / 10, w = value % 10;
      if (!(value == 0 || value == 4) && !((a == 1 || a == 2 || a == 4) && (w == 1 || w == 2 || w == 4)))
        return fail(h, NBS_EINVAL, "contraction config must be 0, 4 or A*10+W with A, W in {1, 2, 4}");
      h->contract_cfg = value;
      return NBS_OK;
    }
    case NBS_PARAM_CHUNK_QBLOCK:
      if (value < 1 || value > (1 << 20)) return fail(h, NBS_EINVAL, "momentum block must be in [1, 2^20]");
      h->chunk_qb = value;
      return NBS_OK;
    case NBS_PARAM_FFT_BLOCK:
      if (value != 64 && value != 128 && value != 256) return fail(h, NBS_EINVAL, "FFT block must be 64, 128 or 256");
      h->fft_block = value;
      return NBS_OK;
    case NBS_PARAM_TEST_SKIP_SLAB:
      if (value != 0 && value != 1) return fail(h, NBS_EINVAL, "the slab-skip test switch is 0 or 1");
      h->test_skip_slab = value;
      return NBS_OK;
    default: return fail(h, NBS_EINVAL, "unknown parameter");
  }
}

int nbs_set_profiling(nbs_ctx* h, int on) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  h->prof = on != 0;
  for (double& v : h->stage_ms) v = 0;
  h->launches = 0;
  return NBS_OK;
}

int nbs_profile(nbs_ctx* h, double* stage_ms, long long* launches) {
  if (!h) return fail(nullptr, NBS_EINVAL, "null context");
  if (stage_ms)
    for (int i = 0; i < NBS_NSTAGES; ++i) stage_ms[i] = h->stage_ms[i];
  if (launches) *launches = h->launches;
  return NBS_OK;
}

int nbs_zero_momentum(nbs_ctx* h, double* out) {
  if (!h || !out) return fail(h, NBS_EINVAL, "null argument");
  if (h->last_nch == 0) return fail(h, NBS_ESTATE, "no correlator computed yet");
  const int n = h->last_nch * 64;
  std::vector<double> tmp(2 * n);
  if (is_f32(h->mode)) {
    std::vector<float2> f(n);
    CK(cudaMemcpy(f.data(), h->zm.p, n * sizeof(float2), cudaMemcpyDeviceToHost), "zero momentum");
    for (int i = 0; i < n; ++i) { tmp[2 * i] = f[i].x; tmp[2 * i + 1] = f[i].y; }
  } else {
    CK(cudaMemcpy(tmp.data(), h->zm.p, n * sizeof(double2), cudaMemcpyDeviceToHost), "zero momentum");
  }
  int e[3] = {0, 0, 0};
  CK(cudaMemcpy(e, h->exps, h->nflav * sizeof(int), cudaMemcpyDeviceToHost), "exponents");
  for (int c = 0; c < h->last_nch; ++c) {
    const int* fl = &h->plan.ch_fl[3 * c];
    const double sc = std::ldexp(1.0, e[0] * fl[0] + e[1] * fl[1] + e[2] * fl[2]);
    for (int k = 0; k < 128; ++k) out[c * 128 + k] = tmp[c * 128 + k] * sc;
  }
  return NBS_OK;
}

int nbs_channel_count(void) { return (int)channel_table().size(); }

int nbs_channel_info(int id, char* buf, int len) {
  const auto& tab = channel_table();
  if (id < 0 || id >= (int)tab.size()) return fail(nullptr, NBS_EINVAL, "channel id out of range");
  const ChannelDef& c = tab[id];
  std::string s = std::string(field_name(c.b[0])) + " " + field_name(c.b[1]) + " | " + field_name(c.b[2]) + " " +
                  field_name(c.b[3]);
  if (buf && len > 0) {
    std::strncpy(buf, s.c_str(), (size_t)len - 1);
    buf[len - 1] = 0;
  }
  int nl = 0;
  for (int b = 0; b < 2; ++b)
    for (const Mono& m : {field_monomials(c.b[b])[0]})
      for (int k = 0; k < 3; ++k) nl += m.q[k] != FS;
  return nl;
}

const char* nbs_last_error(const nbs_ctx* h) { return h ? h->err.c_str() : g_err.c_str(); }

int nbs_plan_create(nbs_plan** out, const int* channel_ids, int n_channels) {
  return nbs_plan_create_flavours(out, channel_ids, n_channels, 2);
}

int nbs_plan_create_flavours(nbs_plan** out, const int* channel_ids, int n_channels, int flavours) {
  if (!out || !channel_ids || n_channels < 1) return fail(nullptr, NBS_EINVAL, "bad arguments");
  nbs_plan* p = new nbs_plan();
  std::string e = compile_plan(std::vector<int>(channel_ids, channel_ids + n_channels), p->plan, flavours);
  if (!e.empty()) {
    delete p;
    *out = nullptr;
    return fail(nullptr, NBS_EINVAL, e);
  }
  *out = p;
  return NBS_OK;
}

int nbs_plan_destroy(nbs_plan* p) {
  delete p;
  return NBS_OK;
}

int nbs_plan_sizes(const nbs_plan* p, long long* s) {
  if (!p || !s) return fail(nullptr, NBS_EINVAL, "bad arguments");
  const Plan& P = p->plan;
  long long nterm = 0;
  for (auto& t : P.types) nterm += (long long)t.terms.size();
  s[NBS_PS_NTYPES] = (long long)P.types.size();
  s[NBS_PS_NCELLS] = P.ncells;
  s[NBS_PS_NTYPETERMS] = nterm;
  s[NBS_PS_NTERMS] = (long long)P.terms.size();
  s[NBS_PS_NENT1] = (long long)P.ent1_cell.size();
  s[NBS_PS_NENT2] = (long long)P.ent2_cell.size();
  s[NBS_PS_NCH] = (long long)P.channels.size();
  s[NBS_PS_NGROUPS] = (long long)P.groups.size();
  s[NBS_PS_NITEMS] = (long long)P.items.size() / 2;
  s[NBS_PS_NCHUNKS] = P.chunks_ok ? (long long)P.chunks.size() : 0;
  s[NBS_PS_NCHUNKTAB] = (long long)P.chunk_tab.size();
  s[NBS_PS_NCHUNKITEMS] = (long long)P.chunk_items.size() / 2;
  return NBS_OK;
}

int nbs_plan_row_sizes(const nbs_plan* p, long long* s) {
  if (!p || !s) return fail(nullptr, NBS_EINVAL, "bad arguments");
  const Plan& P = p->plan;
  s[NBS_PRS_OK] = P.rows_ok ? 1 : 0;
  s[NBS_PRS_NCHUNKS] = (long long)P.row_chunks.size();
  s[NBS_PRS_NENT] = (long long)P.row_ent.size();
  s[NBS_PRS_NROWS] = (long long)P.row_desc.size();
  s[NBS_PRS_NREC] = (long long)P.row_rec.size();
  s[NBS_PRS_NCH] = (long long)P.row_ch.size();
  s[NBS_PRS_NSEGS] = (long long)P.row_segs.size();
  s[NBS_PRS_SMEM] = P.row_smem;
  s[NBS_PRS_WARPS] = NBS_ROW_WARPS;
  s[NBS_PRS_NTYPES] = (long long)P.row_types.size();
  return NBS_OK;
}

int nbs_plan_export(const nbs_plan* p, int what, void* dst) {
  if (!p || !dst) return fail(nullptr, NBS_EINVAL, "bad arguments");
  const Plan& P = p->plan;
  int* I = (int*)dst;
  double* D = (double*)dst;
  switch (what) {
    case NBS_PX_TYPES: {
      int toff = 0;
      for (auto& t : P.types) {
        *I++ = t.cell_off; *I++ = t.ncell; *I++ = toff; *I++ = (int)t.terms.size();
        toff += (int)t.terms.size();
      }
      return NBS_OK;
    }
    case NBS_PX_TYPETERMS:
      for (auto& t : P.types)
        for (auto& tt : t.terms) { *I++ = tt.pat; *I++ = tt.a[0]; *I++ = tt.a[1]; *I++ = tt.a[2]; }
      return NBS_OK;
    case NBS_PX_TYPECOEF:
      for (auto& t : P.types)
        for (auto& tt : t.terms) *D++ = tt.c;
      return NBS_OK;
    case NBS_PX_CELLS:
      for (auto& t : P.types)
        for (int c : t.cells) *I++ = c;
      return NBS_OK;
    case NBS_PX_TERMS:
      for (auto& t : P.terms) {
        *I++ = t.ch; *I++ = t.K; *I++ = t.shape; *I++ = t.n1; *I++ = t.n2; *I++ = t.off1; *I++ = t.off2; *I++ = t.pad;
      }
      return NBS_OK;
    case NBS_PX_ENT1_CELL: std::memcpy(I, P.ent1_cell.data(), P.ent1_cell.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_ENT1_COEF: std::memcpy(D, P.ent1_coef.data(), P.ent1_coef.size() * sizeof(double)); return NBS_OK;
    case NBS_PX_ENT2_CELL: std::memcpy(I, P.ent2_cell.data(), P.ent2_cell.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_ENT2_COEF: std::memcpy(D, P.ent2_coef.data(), P.ent2_coef.size() * sizeof(double)); return NBS_OK;
    case NBS_PX_CHANNELS:
      for (size_t c = 0; c < P.channels.size(); ++c) {
        *I++ = P.ch_term_begin[c]; *I++ = P.ch_term_begin[c + 1]; *I++ = P.ch_nl[c]; *I++ = 6 - P.ch_nl[c];
      }
      return NBS_OK;
    case NBS_PX_GROUPS:
      static_assert(sizeof(GroupHdr) == 24 * sizeof(int), "group header layout");
      std::memcpy(I, P.groups.data(), P.groups.size() * sizeof(GroupHdr));
      return NBS_OK;
    case NBS_PX_GROUPCH: std::memcpy(I, P.group_ch.data(), P.group_ch.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_ITEMS: std::memcpy(I, P.items.data(), P.items.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_CHUNKS:
      static_assert(sizeof(ChunkHdr) == 40 * sizeof(int), "chunk header layout");
      if (P.chunks_ok) std::memcpy(I, P.chunks.data(), P.chunks.size() * sizeof(ChunkHdr));
      return NBS_OK;
    case NBS_PX_CHUNKTAB: std::memcpy(dst, P.chunk_tab.data(), P.chunk_tab.size() * 2); return NBS_OK;
    case NBS_PX_CHUNKITEMS: std::memcpy(I, P.chunk_items.data(), P.chunk_items.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_TERMTABOFF: std::memcpy(I, P.term_tab_off.data(), P.term_tab_off.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_CODES:
      for (int i = 0; i < 32; ++i) D[i] = i < (int)P.coef_codes.size() && i < 31 ? P.coef_codes[i] : 0.0;
      return NBS_OK;
    case NBS_PX_QUADCHUNKS:
      static_assert(sizeof(QuadChunkHdr) == 64 * sizeof(int), "quad chunk header layout");
      if (P.chunks_ok) std::memcpy(I, P.quad_chunks.data(), P.quad_chunks.size() * sizeof(QuadChunkHdr));
      return NBS_OK;
    case NBS_PX_QUADSEGS:
      static_assert(sizeof(QuadSeg) == 8 * sizeof(int), "quad segment layout");
      if (P.chunks_ok) std::memcpy(I, P.quad_segs.data(), P.quad_segs.size() * sizeof(QuadSeg));
      return NBS_OK;
    case NBS_PX_ROWCHUNKS:
      static_assert(sizeof(RowChunkHdr) == 96 * sizeof(int), "row chunk header layout");
      std::memcpy(I, P.row_chunks.data(), P.row_chunks.size() * sizeof(RowChunkHdr));
      return NBS_OK;
    case NBS_PX_ROWENT: std::memcpy(dst, P.row_ent.data(), P.row_ent.size() * 2); return NBS_OK;
    case NBS_PX_ROWTYPES:
      static_assert(sizeof(RowTypeHdr) == 8 * sizeof(int), "row type header layout");
      std::memcpy(I, P.row_types.data(), P.row_types.size() * sizeof(RowTypeHdr));
      return NBS_OK;
    case NBS_PX_ROWDESC: std::memcpy(dst, P.row_desc.data(), P.row_desc.size() * 4); return NBS_OK;
    case NBS_PX_ROWREC: std::memcpy(dst, P.row_rec.data(), P.row_rec.size() * 4); return NBS_OK;
    case NBS_PX_ROWCH: std::memcpy(I, P.row_ch.data(), P.row_ch.size() * sizeof(int)); return NBS_OK;
    case NBS_PX_ROWSEGS:
      static_assert(sizeof(RowSeg) == 4 * sizeof(int), "row segment layout");
      std::memcpy(I, P.row_segs.data(), P.row_segs.size() * sizeof(RowSeg));
      return NBS_OK;
    case NBS_PX_ROWSCALES:
      for (int i = 0; i < NBS_ROW_SCALES; ++i) D[i] = i < (int)P.row_scales.size() ? P.row_scales[i] : 0.0;
      return NBS_OK;
    default: return fail(nullptr, NBS_EINVAL, "unknown export");
  }
}

// ---- L-parallel path ------------------------------------------------------------------------

int nbs_slab_layout(int L, int nranks, int rank, int* z_begin, int* z_end, int* ys, int* n_ys) {
  SlabGeom g;
  if (!z_begin || !z_end || !ys || !n_ys) return fail(nullptr, NBS_EINVAL, "null output");
  if (!fft_supported(L) || !slab_layout(L, nranks, g) || rank < 0 || rank >= nranks)
    return fail(nullptr, NBS_EINVAL, "no layout of this many ranks on this lattice (L must be a supported FFT "
                                     "size; each rank needs a z-plane and a y pair)");
  *z_begin = g.z0[rank];
  *z_end = g.z0[rank + 1];
  const std::vector<int> y = slab_yset(g, rank);
  *n_ys = (int)y.size();
  std::copy(y.begin(), y.end(), ys);
  return NBS_OK;
}

int nbs_slab_create(nbs_ctx** out, int L, int nranks, int rank, const int* channel_ids, int n_channels) {
  if (!out || !channel_ids || n_channels < 1) return fail(nullptr, NBS_EINVAL, "null argument or no channels");
  *out = nullptr;
  SlabGeom g;
  if (!fft_supported(L) || !slab_layout(L, nranks, g) || rank < 0 || rank >= nranks)
    return fail(nullptr, NBS_EINVAL, "no layout of this many ranks on this lattice");
  nbs_ctx* h = nullptr;
  int rc = create_ctx(&h, L, 1, 2, false);
  if (rc) return rc;
  h->mode = NBS_FP32;
  h->slab = true;
  h->sg = g;
  h->srank = rank;
  h->slz = g.z0[rank + 1] - g.z0[rank];
  h->sny = g.ny[rank];
  h->svs = (long long)h->slz * L * L;
  h->svm = (long long)L * h->sny * L;
  h->smg.L = L;
  h->smg.Ly = h->sny;
  const std::vector<int> ys = slab_yset(g, rank);
  for (int i = 0; i < 64; ++i) h->smg.ymir[i] = 0;
  for (int i = 0; i < h->sny; ++i) h->smg.ymir[i] = g.yloc[(L - ys[i]) % L];
  std::vector<int> ids(channel_ids, channel_ids + n_channels);
  if ((rc = ensure_plan(h, ids))) {
    std::string m = h->err;
    nbs_destroy(h);
    return fail(nullptr, rc, m);
  }
  if (!h->plan.rows_ok || h->plan.row_smem > h->smem_optin) {
    nbs_destroy(h);
    return fail(nullptr, NBS_EINVAL, "the L-parallel path needs the two-phase contraction tables");
  }
  h->snch = n_channels;
  const long long nc = h->plan.ncells, n64 = 64LL * n_channels;
  // exchange offsets in elements of the moved data (32-byte cells, complex FP32 correlators)
  for (int p = 0; p < 4; ++p) {
    h->soff[p].rank = rank;
    h->soff[p].off[0] = 0;
  }
  for (int p = 0; p < nranks; ++p) {
    const int lz = g.z0[p + 1] - g.z0[p];
    h->soff[0].off[p + 1] = h->soff[0].off[p] + nc * h->slz * g.ny[p] * L;     // forward send: y-set of p
    h->soff[1].off[p + 1] = h->soff[1].off[p] + nc * lz * h->sny * L;          // forward receive: z-planes of p
    h->soff[2].off[p + 1] = h->soff[2].off[p] + n64 * lz * h->sny * L;         // inverse send: z-planes of p
    h->soff[3].off[p + 1] = h->soff[3].off[p] + n64 * h->slz * g.ny[p] * L;    // inverse receive: y-set of p
  }
  if ((rc = ensure(h, h->propsT, 2ull * 144 * h->svs * sizeof(float2), "scaled propagators")) ||
      (rc = ensure(h, h->s_FB, 4ull * nc * h->svs * sizeof(float2), "slab blocks")) ||
      (rc = ensure(h, h->s_FBm, 4ull * nc * h->svm * sizeof(float2), "momentum-set blocks")) ||
      (rc = ensure(h, h->s_Ft, (size_t)n64 * h->svm * sizeof(float2), "momentum-set correlators")) ||
      (rc = ensure(h, h->s_F, (size_t)n64 * h->svs * sizeof(float2), "slab correlators")) ||
      (rc = ensure(h, h->RQ, (size_t)h->svm * h->plan.row_nr * 32, "effective-block rows"))) {
    std::string m = h->err;
    nbs_destroy(h);
    return fail(nullptr, rc, m);
  }
  *out = h;
  return NBS_OK;
}

int nbs_slab_sizes(const nbs_ctx* h, long long* send_blocks, long long* recv_blocks, long long* send_corr,
                   long long* recv_corr) {
  if (!h || !h->slab) return fail(nullptr, NBS_EINVAL, "not an L-parallel context");
  long long* outs[4] = {send_blocks, recv_blocks, send_corr, recv_corr};
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    const long long per = k < 2 ? 4 : 1;  // complex values per moved element
    for (int p = 0; p < h->sg.P; ++p) outs[k][p] = (h->soff[k].off[p + 1] - h->soff[k].off[p]) * per;
  }
  return NBS_OK;
}

int nbs_slab_begin(nbs_ctx* h, const void* u, const void* s, int dtype, unsigned long long* maxbits) {
  if (!h || !h->slab) return fail(h, NBS_EINVAL, "not an L-parallel context");
  if (!u || !s || !maxbits) return fail(h, NBS_EINVAL, "null pointer");
  if (dtype != NBS_C128 && dtype != NBS_C64) return fail(h, NBS_EINVAL, "dtype must be NBS_C128 or NBS_C64");
  h->s_u = u;
  h->s_s = s;
  h->s_c64 = dtype == NBS_C64;
  const PropPtrs pp = {{u, s, nullptr}};
  CK(cudaMemsetAsync(h->small.p, 0, 64, h->st), "clear max|S|");
  CK(launch_props_maxabs(pp, 2, h->s_c64, (int)h->svs, h->maxbits, h->flags, h->st), "max|S|");
  unsigned long long mb[2];
  CK(cudaMemcpyAsync(mb, h->maxbits, sizeof(mb), cudaMemcpyDeviceToHost, h->st), "max|S| to host");
  CK(cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->st), "NaN flag");
  CK(cudaStreamSynchronize(h->st), "sync");
  if (*h->host_flags) return fail(h, NBS_ENAN, "non-finite value in the propagators");
  maxbits[0] = mb[0];
  maxbits[1] = mb[1];
  return NBS_OK;
}

int nbs_slab_blocks(nbs_ctx* h, const unsigned long long* maxbits, void* send) {
  if (!h || !h->slab || !h->s_u) return fail(h, NBS_EINVAL, "not an L-parallel context, or no nbs_slab_begin");
  if (!maxbits || !send) return fail(h, NBS_EINVAL, "null pointer");
  const Plan& P = h->plan;
  const int L = h->L;
  const long long nc = P.ncells;
  const PropPtrs pp = {{h->s_u, h->s_s, nullptr}};
  CK(cudaMemcpyAsync(h->maxbits, maxbits, 2 * sizeof(unsigned long long), cudaMemcpyHostToDevice, h->st),
     "max|S| of all ranks");
  CK(launch_props_scale<float>(pp, 2, h->s_c64, (int)h->svs, h->maxbits, h->exps, (float2*)h->propsT.p, h->st),
     "rescale");
  CK(launch_blocks_tiled<float>((const float2*)h->propsT.p, (const int*)h->d_cells.p, P.ncells, h->recipes,
                                (int)h->svs, 2, (float2*)h->s_FB.p, h->st),
     "diquarks and field blocks");
  float2* fb = (float2*)h->s_FB.p;
  CK(fft_rows<float>(fb, nc * h->slz * L, L, 4, -1, h->st), "x pass");
  CK(fft_lines<float>(fb, nc * h->slz * 4LL * L, 4 * L, 4LL * L * L, 4LL * L, L, -1, h->fft_block, h->st), "y pass");
  CK(launch_slab_move(SLAB_PACK_BLOCKS, fb, send, nc, h->sg, h->soff[0], h->st), "pack for the forward exchange");
  CK(cudaStreamSynchronize(h->st), "sync");
  return NBS_OK;
}

int nbs_slab_contract(nbs_ctx* h, const void* recv, void* send) {
  if (!h || !h->slab) return fail(h, NBS_EINVAL, "not an L-parallel context");
  if (!recv || !send) return fail(h, NBS_EINVAL, "null pointer");
  const Plan& P = h->plan;
  const int L = h->L, ny = h->sny;
  const long long nc = P.ncells, n64 = 64LL * h->snch;
  float2* fbm = (float2*)h->s_FBm.p;
  float2* ft = (float2*)h->s_Ft.p;
  CK(launch_slab_move(SLAB_UNPACK_BLOCKS, recv, fbm, nc, h->sg, h->soff[1], h->st), "unpack the forward exchange");
  CK(fft_lines<float>(fbm, nc * ny * 4LL * L, 4 * L * ny, 4LL * L * ny * L, 4LL * L * ny, L, -1, h->fft_block, h->st),
     "z pass");
  CK(cudaMemsetAsync(h->flags, 0, sizeof(int), h->st), "clear flags");
  CK(launch_eff_rows(fbm, h->svm, h->d_rtypes.p, (int)P.row_types.size(), (const unsigned*)h->d_rdesc.p,
                     (const unsigned short*)h->d_rent.p, (int)P.row_ent.size(), P.row_nr, (float2*)h->RQ.p, h->nsm,
                     h->st),
     "effective-block rows on the momentum set");
  CK(launch_contract_rows((const float2*)h->RQ.p, h->smg, P.row_nr, (const int2*)h->d_qlist.p,
                          (int)P.row_chunks.size(), h->chunk_qb, h->d_rchunks.p, (const unsigned*)h->d_rrec.p,
                          h->d_rsegs.p, (const int*)h->d_rch.p, (const float*)h->d_rscales.p, P.row_smem, ft,
                          h->flags, h->st),
     "contraction on the momentum set");
  CK(fft_lines<float>(ft, n64 * ny * L, L * ny, (long long)L * ny * L, (long long)L * ny, L, 1, h->fft_block, h->st),
     "inverse z pass");
  CK(launch_slab_move(SLAB_PACK_CORR, ft, send, n64, h->sg, h->soff[2], h->st), "pack for the inverse exchange");
  CK(cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->st), "flags");
  CK(cudaStreamSynchronize(h->st), "sync");
  if (*h->host_flags & 2) return fail(h, NBS_ETIMEOUT, "a bounded wait in the contraction gave up");
  return NBS_OK;
}

int nbs_slab_finish(nbs_ctx* h, const void* recv, void* out) {
  if (!h || !h->slab) return fail(h, NBS_EINVAL, "not an L-parallel context");
  if (!recv || !out) return fail(h, NBS_EINVAL, "null pointer");
  const int L = h->L;
  const long long n64 = 64LL * h->snch;
  float2* f = (float2*)h->s_F.p;
  CK(launch_slab_move(SLAB_UNPACK_CORR, recv, f, n64, h->sg, h->soff[3], h->st), "unpack the inverse exchange");
  CK(fft_lines<float>(f, n64 * h->slz * L, L, (long long)L * L, L, L, 1, h->fft_block, h->st), "inverse y pass");
  CK(fft_rows<float>(f, n64 * h->slz * L, L, 1, 1, h->st), "inverse x pass");
  CK(launch_restore<float>(f, (int)h->svs, h->snch, (const int*)h->d_chnl.p, h->exps, 2, (double2*)out, 64LL * h->svs,
                           h->st, (long long)L * L * L),
     "restore");
  CK(cudaStreamSynchronize(h->st), "sync");
  return NBS_OK;
}

}  // extern "C"
