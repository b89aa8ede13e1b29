// noalloc.cu -- nbs_correlate_static: the correlator of one channel on one
// small timeslice with no device allocation at all.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- inside a host that owns every byte of device memory through its
// own pool, a process whose allocator is locked, or a path that must not
// allocate (a timing-critical loop, a checker running next to a production
// job).  Such callers pass their inputs and outputs; every intermediate
// buffer (rescaled propagators, diquarks, momentum-space blocks, correlators
// in momentum space, the gather tables) lives in the file-scope array
// g_static_scratch below, which every GPU that loads the library keeps until
// the process exits.
//
// The array is shared by every call: a call overwrites what the last call
// left, clears the reduction words it needs at zero, and calls whose work
// overlaps on the GPU (two streams, two host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/nbs.h"
#include "common.cuh"
#include "plan.h"

using namespace nbs;

namespace {

constexpr int kMaxL = NBS_STATIC_MAX_L;
constexpr long long kMaxV = (long long)kMaxL * kMaxL * kMaxL;
constexpr int kMaxCells = 2 * 936;        // the two largest stored block types
constexpr int kMaxTerms = 512;
constexpr int kMaxEntries = 1 << 16;      // per side

// byte offsets of the regions inside the static scratch
constexpr size_t kSmall = 0;                                           // maxima, flag, exponents
constexpr size_t kProps = 256;                                         // [2][144][V] complex128
constexpr size_t kQ = kProps + 2 * 144 * kMaxV * 16;                   // [6][144][V]
constexpr size_t kFB = kQ + 6 * 144 * kMaxV * 16;                      // [cells][V][4]
constexpr size_t kFt = kFB + (size_t)kMaxCells * kMaxV * 4 * 16;       // [64][V]
constexpr size_t kTerms = kFt + 64 * kMaxV * 16;                       // DevTerm[kMaxTerms]
constexpr size_t kChtb = kTerms + kMaxTerms * sizeof(DevTerm);         // int[2]
constexpr size_t kChnl = kChtb + 16;                                   // int[3]
constexpr size_t kCells = kChnl + 16;                                  // int[kMaxCells]
constexpr size_t kE1 = (kCells + kMaxCells * 4 + 255) / 256 * 256;     // Ent<double>[kMaxEntries]
constexpr size_t kE2 = kE1 + (size_t)kMaxEntries * sizeof(Ent<double>);
constexpr size_t kTotal = kE2 + (size_t)kMaxEntries * sizeof(Ent<double>);
static_assert(kTotal <= NBS_STATIC_SCRATCH_BYTES, "static scratch too small");

__device__ __align__(256) unsigned char g_static_scratch[NBS_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
unsigned char* g_addr[64] = {};   // device address of g_static_scratch per device

// the text nbs_last_error(NULL) returns
int err(int code, const std::string& m) {
  set_global_error(m);
  return code;
}

// once per device, with that device current: the array's device address
int setup(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return err(NBS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    e = fft_init();
    if (e != cudaSuccess) {
      cudaGetLastError();
      return err(NBS_ECUDA, std::string("FFT twiddles: ") + cudaGetErrorString(e));
    }
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return NBS_OK;
}

#define SCK(call, where)                                                                  \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) {                                                              \
      cudaGetLastError();                                                                 \
      return err(NBS_ECUDA, std::string(where) + ": " + cudaGetErrorString(_e));          \
    }                                                                                     \
  } while (0)

}  // namespace

extern "C" int nbs_correlate_static(const void* u, const void* s, int L, int dtype, int channel_id, void* out,
                                    void* stream) {
  if (!u || !s || !out) return err(NBS_EINVAL, "null pointer");
  if (L < 1 || L > kMaxL || !fft_supported(L))
    return err(NBS_EINVAL, "nbs_correlate_static: L must be 1, 2, 3 or 4 (static scratch holds L <= " +
                               std::to_string(kMaxL) + ")");
  if (dtype != NBS_C128 && dtype != NBS_C64) return err(NBS_EINVAL, "dtype must be NBS_C128 or NBS_C64");
  if (channel_id < 0 || channel_id >= (int)channel_table().size()) return err(NBS_EINVAL, "channel id out of range");
  Plan P;
  std::string e = compile_plan(std::vector<int>{channel_id}, P);
  if (!e.empty()) return err(NBS_EINVAL, e);
  if (P.ncells > kMaxCells || (int)P.terms.size() > kMaxTerms || (long long)P.ent1_cell.size() > kMaxEntries ||
      (long long)P.ent2_cell.size() > kMaxEntries || P.types.size() > NBS_MAX_TYPES)
    return err(NBS_EINVAL, "nbs_correlate_static: channel tables exceed the static scratch");

  int dev = 0;
  SCK(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) return err(NBS_EINVAL, "device index above 63");
  unsigned char* base = nullptr;
  int rc = setup(dev, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int V = L * L * L;

  // tables of this channel into the scratch
  std::vector<DevTerm> terms(P.terms.size());
  for (size_t i = 0; i < P.terms.size(); ++i) {
    const TermHdr& t = P.terms[i];
    terms[i] = {t.ch, t.K, t.shape, t.n1, t.n2, t.off1, t.off2, 0};
  }
  std::vector<int> cells(P.ncells);
  TypeRecipeSet rs = {};
  for (size_t ti = 0; ti < P.types.size(); ++ti) {
    const BlockType& bt = P.types[ti];
    for (int c = 0; c < bt.ncell; ++c) cells[bt.cell_off + c] = bt.cells[c] | ((int)ti << 11);
    if (bt.terms.size() > NBS_MAX_TYPE_TERMS) return err(NBS_EINVAL, "block type with too many terms");
    TypeRecipe& r = rs.t[ti];
    r.nterms = (int)bt.terms.size();
    r.cell_off = bt.cell_off;
    r.ncell = bt.ncell;
    for (size_t k = 0; k < bt.terms.size(); ++k) {
      r.pat[k] = bt.terms[k].pat;
      r.arg[k] = bt.terms[k].a[0] | (bt.terms[k].a[1] << 2) | (bt.terms[k].a[2] << 4);
      r.coef[k] = bt.terms[k].c;
    }
  }
  std::vector<Ent<double>> e1(P.ent1_cell.size()), e2(P.ent2_cell.size());
  for (size_t i = 0; i < e1.size(); ++i) { e1[i].cell = P.ent1_cell[i]; e1[i].pad = 0; e1[i].coef = P.ent1_coef[i]; }
  for (size_t i = 0; i < e2.size(); ++i) { e2[i].cell = P.ent2_cell[i]; e2[i].pad = 0; e2[i].coef = P.ent2_coef[i]; }
  SCK(cudaMemcpyAsync(base + kTerms, terms.data(), terms.size() * sizeof(DevTerm), cudaMemcpyHostToDevice, st), "terms");
  SCK(cudaMemcpyAsync(base + kChtb, P.ch_term_begin.data(), 2 * sizeof(int), cudaMemcpyHostToDevice, st), "ranges");
  SCK(cudaMemcpyAsync(base + kChnl, P.ch_fl.data(), 3 * sizeof(int), cudaMemcpyHostToDevice, st), "flavours");
  SCK(cudaMemcpyAsync(base + kCells, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice, st), "cells");
  SCK(cudaMemcpyAsync(base + kE1, e1.data(), e1.size() * sizeof(Ent<double>), cudaMemcpyHostToDevice, st), "e1");
  SCK(cudaMemcpyAsync(base + kE2, e2.data(), e2.size() * sizeof(Ent<double>), cudaMemcpyHostToDevice, st), "e2");

  // the path, FP64, every buffer inside the scratch
  unsigned long long* maxbits = (unsigned long long*)(base + kSmall);
  int* flags = (int*)(base + kSmall + 16);
  int* exps = (int*)(base + kSmall + 64);
  double2* props = (double2*)(base + kProps);
  double2* Q = (double2*)(base + kQ);
  double2* FB = (double2*)(base + kFB);
  double2* Ft = (double2*)(base + kFt);
  const int c64 = dtype == NBS_C64;
  SCK(cudaMemsetAsync(base + kSmall, 0, 64, st), "clear reduction words");
  const PropPtrs pp = {{u, s, nullptr}};
  SCK(launch_props_maxabs(pp, 2, c64, V, maxbits, flags, st), "max|S|");
  SCK(launch_props_scale<double>(pp, 2, c64, V, maxbits, exps, props, st), "rescale");
  SCK(launch_diquarks<double>(props, V, 2, Q, st), "diquarks");
  SCK(launch_field_blocks<double>(props, Q, (const int*)(base + kCells), P.ncells, rs, V, 2, FB, st), "field blocks");
  SCK(fft3d_blocks<double>(FB, P.ncells, L, st), "forward FFT");
  SCK(launch_contract<double>(FB, L, (const DevTerm*)(base + kTerms), (const int*)(base + kChtb), 1,
                              (const Ent<double>*)(base + kE1), (const Ent<double>*)(base + kE2), Ft, 0, st),
      "contraction");
  SCK(fft3d_inverse<double>(Ft, 64, L, st), "inverse FFT");
  SCK(launch_restore<double>(Ft, V, 1, (const int*)(base + kChnl), exps, 2, (double2*)out, 64LL * V, st), "restore");
  int flag = 0;
  SCK(cudaMemcpyAsync(&flag, flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
  SCK(cudaStreamSynchronize(st), "sync");
  if (flag) return err(NBS_ENAN, "non-finite value in the propagators");
  return NBS_OK;
}
