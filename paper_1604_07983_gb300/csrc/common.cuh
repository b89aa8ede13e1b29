// common.cuh -- complex helpers and launch declarations shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace nbs {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> cmake(T re, T im) { C<T> z; z.x = re; z.y = im; return z; }
template <typename T> __host__ __device__ __forceinline__ C<T> czero() { return cmake<T>(T(0), T(0)); }
template <typename T> __host__ __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return cmake<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return cmake<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return cmake<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(C<T>& acc, C<T> a, C<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += s * a   (s real)
template <typename T> __host__ __device__ __forceinline__ void crfma(C<T>& acc, T s, C<T> a) {
  acc.x = fma(s, a.x, acc.x);
  acc.y = fma(s, a.y, acc.y);
}

// Gather-table entry of the contraction: stored cell and real coefficient.
template <typename T> struct Ent { int cell; T coef; };
template <> struct __align__(16) Ent<double> { int cell; int pad; double coef; };

struct DevTerm { int ch, K, shape, n1, n2, off1, off2, pad; };

// Block-type recipe for the field-block kernel (constant memory).
#define NBS_MAX_TYPES 8
#define NBS_MAX_TYPE_TERMS 8
struct TypeRecipe {
  int nterms;
  int cell_off;
  int ncell;
  int pad;
  int pat[NBS_MAX_TYPE_TERMS];
  int arg[NBS_MAX_TYPE_TERMS];       // a0 + 4*a1 + 16*a2
  double coef[NBS_MAX_TYPE_TERMS];
};

// ---- launchers (defined in the .cu files) ----------------------------------
// kernels_blocks.cu
// the propagators of one timeslice, one pointer per flavour (nflav = 2: l, s; 3: u, d, s)
struct PropPtrs { const void* p[3]; };
cudaError_t launch_props_maxabs(const PropPtrs& props, int nflav, int in_c64, int V,
                                unsigned long long* maxbits, int* flags, cudaStream_t st);
template <typename T>
cudaError_t launch_props_scale(const PropPtrs& props, int nflav, int in_c64, int V,
                               const unsigned long long* maxbits, int* exps, C<T>* out, cudaStream_t st);
// Q[(d*3 + c)*144 + j1*12 + j2][site] for the n_diquarks(nflav) diquarks of plan.h
template <typename T>
cudaError_t launch_diquarks(const C<T>* props, int V, int nflav, C<T>* Q, cudaStream_t st);
struct TypeRecipeSet { TypeRecipe t[NBS_MAX_TYPES]; };
template <typename T>
cudaError_t launch_field_blocks(const C<T>* props, const C<T>* Q, const int* cells, int ncells,
                                const TypeRecipeSet& recipes, int V, int nflav, C<T>* FB, cudaStream_t st);
// diquarks and field blocks in one site-tiled kernel (no diquark array in HBM)
template <typename T>
cudaError_t launch_blocks_tiled(const C<T>* props, const int* cells, int ncells, const TypeRecipeSet& recipes, int V,
                                int nflav, C<T>* FB, cudaStream_t st);
// fft.cu
cudaError_t fft_init();
bool fft_supported(int L);
// forward FFT of the stored blocks, layout [cell][z][y][x][alpha]
template <typename T>
cudaError_t fft3d_blocks(C<T>* data, long long ncells, int L, cudaStream_t st, int sb = 128);
// inverse FFT of nbatch contiguous cubes [batch][z][y][x]
template <typename T>
cudaError_t fft3d_inverse(C<T>* data, long long nbatch, int L, cudaStream_t st, int sb = 128);
// kernels_contract.cu
template <typename T>
cudaError_t launch_contract(const C<T>* FB, int L, const DevTerm* terms, const int* ch_tb, int nch,
                            const Ent<T>* e1, const Ent<T>* e2, C<T>* Ft, int cfg, cudaStream_t st);
// quad-lane chunk contraction (FP32): chunks points to QuadChunkHdr[nchunks],
// segs to the per-warp runs QuadSeg[] (plan.h), max_segs = the most runs of one
// chunk; max_cells = the largest stored type's cell count (<= 944)
size_t qseg_smem_bytes(int max_slot, int max_tab, int max_segs);
// ncells: the stored block array's cells (the TMA tensor extent); flags: bit 1
// set if a slab wait gave up
cudaError_t launch_contract_qseg(const float2* FB, long long ncells, int L, int nchunks, int qb, const void* chunks,
                                 const void* segs, int max_segs, const int* group_ch, const unsigned short* tab,
                                 const float* codes, int max_cells, int max_slot, int max_tab, int max_row, float2* Ft,
                                 int* flags, int skip_first, cudaStream_t st);
// quad-lane tensor-core contraction (split-BF16 x 3): same arguments
size_t tcq_smem_bytes(int max_slot, int max_tab, int max_segs);
cudaError_t launch_contract_tcq(const float2* FB, long long ncells, int L, int nchunks, int qb, const void* chunks,
                                const void* segs, int max_segs, const int* group_ch, const unsigned short* tab,
                                const float* codes, int max_cells, int max_slot, int max_tab, int max_row, float2* Ft,
                                int* flags, cudaStream_t st);
// Momenta of a contraction launch: q = x + L (y + Ly z), x and z over [0, L), y over Ly values of a set
// that contains -y (mod L) with every y; the index of -y is ymir[y].  The full cube: Ly = L,
// ymir[y] = (L - y) mod L.
struct MomGeom {
  int L, Ly;
  int ymir[64];
};
inline MomGeom full_geom(int L) {
  MomGeom g;
  g.L = L;
  g.Ly = L;
  for (int y = 0; y < 64; ++y) g.ymir[y] = y < L ? (L - y) % L : 0;
  return g;
}
// phase A of the FP32 contraction: the rows of every stored type at every momentum (RQ: 2 NR 16-byte units
// per momentum); types, desc, ent: Plan::row_types, row_desc, row_ent in device memory
cudaError_t launch_eff_rows(const float2* FB, long long V, const void* types, int ntypes, const unsigned* desc,
                            const unsigned short* ent, int nent, int NR, float2* RQ, int nsm, cudaStream_t st);
// phase B; qlist: the momenta in visiting order as (q, -q) pairs (momentum_order), device memory
cudaError_t launch_contract_rows(const float2* RQ, const MomGeom& geom, int NR, const int2* qlist, int nchunks, int qb,
                                 const void* chunks, const unsigned* rec, const void* segs, const int* row_ch,
                                 const float* scales, int smem, float2* Ft, int* flags, cudaStream_t st);
std::vector<int2> momentum_order(const MomGeom& g);
// ---- L-parallel path (slab.cu) -------------------------------------------------------
#define NBS_SLAB_MAX_RANKS 64
// ranks' z-planes [z0[p], z0[p+1]); y-sets: owner rank and local index of each y, set sizes
struct SlabGeom {
  int L = 0, P = 0;
  int z0[NBS_SLAB_MAX_RANKS + 1] = {};
  int zowner[64] = {};
  int ny[NBS_SLAB_MAX_RANKS] = {};
  int yowner[64] = {}, yloc[64] = {};
};
// this rank and the element offset of each peer's block in an exchange buffer
struct SlabOff {
  int rank = 0;
  long long off[NBS_SLAB_MAX_RANKS + 1] = {};
};
bool slab_layout(int L, int nranks, SlabGeom& g);
std::vector<int> slab_yset(const SlabGeom& g, int p);
enum SlabMove { SLAB_PACK_BLOCKS = 0, SLAB_UNPACK_BLOCKS = 1, SLAB_PACK_CORR = 2, SLAB_UNPACK_CORR = 3 };
// the four moves around the exchanges: blocks [c][zl][y][x] (32-byte cells) -> by y-owner, by z-owner ->
// [c][z][yl][x]; correlators [c][z][yl][x] (complex FP32) -> by z-owner, by y-owner -> [c][zl][y][x]
cudaError_t launch_slab_move(int kind, const void* src, void* dst, long long ncomp, const SlabGeom& g,
                             const SlabOff& o, cudaStream_t st);
// one pass of the FFT over arbitrary lines: line l starts at (l / inner) * group + l % inner, its L points
// `stride` apart (fft.cu)
template <typename T>
cudaError_t fft_lines(C<T>* data, long long nlines, int inner, long long group, long long stride, int L, int dir,
                      int sb, cudaStream_t st);
// the x pass: nrows contiguous rows of L * IL values, IL interleaved lines each (IL = 1 or 4)
template <typename T>
cudaError_t fft_rows(C<T>* data, long long nrows, int L, int IL, int dir, cudaStream_t st);
// ch_fl: per channel the quarks of each propagator (3 ints); exps: per propagator
// norm: the volume of the inverse transform's 1/V (0: V, the values per channel and spin)
template <typename T>
cudaError_t launch_restore(const C<T>* Ft, int V, int nch, const int* ch_fl, const int* exps, int nflav,
                           double2* out, long long ch_stride, cudaStream_t st, long long norm = 0);

// kernels_potential.cu: K = a d_t^2 R + b d_t R + c lap R, P = K / R (P may be null)
cudaError_t launch_potential(const double2* Rm, const double2* R0, const double2* Rp, int L, long long ncomp, double a,
                             double b, double c, double2* K, double2* P, cudaStream_t st);

}  // namespace nbs
