// kernels_contract.cu -- effective blocks and their product in momentum space
// (Sec. 4 (ii)-(iii), Eqs. (4.2)-(4.3) of arXiv:1604.07983), and the restore
// of the correlator after the inverse FFT.
//
// One thread owns one momentum q (and A1 of the four sink spins alpha1); the
// threads of a warp own 32 consecutive q, so every gather of a stored block
// cell reads one contiguous run of 32 x 4 spins (FP32: 1 KB) and every thread
// runs the same table-driven program (the SoA layout the paper uses against
// warp divergence).  For each term of the channel and each shared source index
// xi~ the thread forms
//   e1[alpha1][h1] = sum_i coef1_i * FB~[cell1_i](q)     (B1 block at  q)
//   e2[alpha2][h2] = sum_i coef2_i * FB~[cell2_i](-q)    (B2 block at -q)
// and accumulates F~[alpha1][alpha2][alpha3][alpha4](q) += e1 * e2, the
// held spins (h1, h2) carrying alpha3 / alpha4 as the term's shape says.
#include "common.cuh"
#include "plan.h"

#include <algorithm>

namespace nbs {

namespace {

// N consecutive complex values (the sink spins of one stored cell and site),
// from a 16-byte aligned address, with 16-byte loads through the read-only path
template <typename T, int N> struct AlphaLoad;
template <int N> struct AlphaLoad<float, N> {
  static __device__ __forceinline__ void run(const float2* p, float2 (&x)[N]) {
    if constexpr (N == 1) {
      x[0] = __ldg(p);
    } else {
#pragma unroll
      for (int v = 0; v < N / 2; ++v) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(p) + v);
        x[2 * v] = make_float2(w.x, w.y);
        x[2 * v + 1] = make_float2(w.z, w.w);
      }
    }
  }
};
template <int N> struct AlphaLoad<double, N> {
  static __device__ __forceinline__ void run(const double2* p, double2 (&x)[N]) {
#pragma unroll
    for (int v = 0; v < N; ++v) x[v] = __ldg(p + v);
  }
};

// one term: for each shared index k, the two effective blocks from their
// gather lists (ordered [i][h], i even) and their outer product into acc
template <typename T, int A1, int SHAPE>
__device__ __forceinline__ void run_term(const DevTerm& h, const C<T>* __restrict__ FB, long long cs, long long qoff,
                                         long long qmoff, const Ent<T>* __restrict__ E1,
                                         const Ent<T>* __restrict__ E2, C<T> (&acc)[A1][4][4]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  const int n1 = h.n1, n2 = h.n2;
  const Ent<T>* p1 = E1 + h.off1;
  const Ent<T>* p2 = E2 + h.off2;
  for (int k = 0; k < h.K; ++k) {
    C<T> v1[NH1][A1];
    C<T> v2[NH2][4];
#pragma unroll
    for (int hh = 0; hh < NH1; ++hh)
#pragma unroll
      for (int a = 0; a < A1; ++a) v1[hh][a] = czero<T>();
#pragma unroll
    for (int hh = 0; hh < NH2; ++hh)
#pragma unroll
      for (int b = 0; b < 4; ++b) v2[hh][b] = czero<T>();
    for (int i = 0; i < n1; i += 2, p1 += 2 * NH1) {
      int cell[2 * NH1];
      T coef[2 * NH1];
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j) { cell[j] = __ldg(&p1[j].cell); coef[j] = __ldg(&p1[j].coef); }
      C<T> x[2 * NH1][A1];
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j) AlphaLoad<T, A1>::run(FB + cell[j] * cs + qoff, x[j]);
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j)
#pragma unroll
        for (int a = 0; a < A1; ++a) crfma<T>(v1[j % NH1][a], coef[j], x[j][a]);
    }
    for (int i = 0; i < n2; i += 2, p2 += 2 * NH2) {
      int cell[2 * NH2];
      T coef[2 * NH2];
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j) { cell[j] = __ldg(&p2[j].cell); coef[j] = __ldg(&p2[j].coef); }
      C<T> x[2 * NH2][4];
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j) AlphaLoad<T, 4>::run(FB + cell[j] * cs + qmoff, x[j]);
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j)
#pragma unroll
        for (int b = 0; b < 4; ++b) crfma<T>(v2[j % NH2][b], coef[j], x[j][b]);
    }
#pragma unroll
    for (int a = 0; a < A1; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int h1 = 0; h1 < NH1; ++h1)
#pragma unroll
          for (int h2 = 0; h2 < NH2; ++h2) {
            // spin slot s = alpha3 + 2 alpha4
            int s;
            if (SHAPE == 0) s = h2;                 // both on the B2 block
            else if (SHAPE == 3) s = h1;            // both on the B1 block
            else if (SHAPE == 1) s = h1 + 2 * h2;   // alpha3 on B1, alpha4 on B2
            else s = h2 + 2 * h1;                   // alpha4 on B1, alpha3 on B2
            cfma<T>(acc[a][b][s], v1[h1][a], v2[h2][b]);
          }
  }
}

// grid.x = channel x alpha1-group (fastest, so that every channel of a q-tile
// runs at the same time and the tile's stored blocks are reused from L2),
// grid.y = q-tile of NT consecutive momenta.  Stored blocks: FB[cell][q][alpha].
template <typename T, int A1, int NT>
__global__ void __launch_bounds__(NT) k_contract(const C<T>* __restrict__ FB, int L, const DevTerm* __restrict__ terms,
                                                 const int* __restrict__ ch_tb, const Ent<T>* __restrict__ E1,
                                                 const Ent<T>* __restrict__ E2, C<T>* __restrict__ Ft) {
  const long long V = (long long)L * L * L;
  const int q = blockIdx.y * NT + threadIdx.x;
  if (q >= V) return;
  constexpr int NG = 4 / A1;
  const int ch = blockIdx.x / NG;
  const int a0 = (blockIdx.x % NG) * A1;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int qm = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  C<T> acc[A1][4][4];
#pragma unroll
  for (int a = 0; a < A1; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[a][b][s] = czero<T>();
  const long long cs = 4 * V, qoff = 4LL * q + a0, qmoff = 4LL * qm;
  const int t1 = ch_tb[ch + 1];
  for (int t = ch_tb[ch]; t < t1; ++t) {
    DevTerm h = terms[t];
    switch (h.shape) {
      case 0: run_term<T, A1, 0>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
      case 1: run_term<T, A1, 1>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
      case 2: run_term<T, A1, 2>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
      default: run_term<T, A1, 3>(h, FB, cs, qoff, qmoff, E1, E2, acc); break;
    }
  }
  C<T>* o = Ft + (long long)ch * 64 * V + q;
#pragma unroll
  for (int a = 0; a < A1; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        // acc holds s = alpha3 + 2 alpha4; the output layout is [alpha1][alpha2][alpha3][alpha4]
        const int spin = ((a0 + a) * 4 + b) * 4 + 2 * (s & 1) + (s >> 1);
        o[(long long)spin * V] = acc[a][b][s];
      }
}

// ---- momentum-slab contraction ----------------------------------------------
//
// One CTA per (q, group of channels that read the same two stored block
// types).  The CTA first copies the two momentum slabs it needs -- every cell
// of B1's type at q and of B2's type at -q, four spins each -- from HBM into
// shared memory with cp.async, so that the ~100 reads of every stored value
// that the effective blocks of all terms make are served from shared memory.
// The slab of a type is stored as planes of 16 bytes per cell (FP32: spins
// 0,1 | 2,3; FP64: one spin per plane) so that random cells spread over the
// banks.  Warps take items (term, 32 consecutive shared indices xi~): lane j
// forms the two effective blocks of shared index k0 + j and accumulates its
// 64 products in registers; a warp reduce-scatter then leaves two of the 64
// sums per lane, and the per-warp partials are added in a fixed order.

template <typename T> struct SlabTraits;
template <> struct SlabTraits<float> { static constexpr int NP = 2; };   // planes of float4
template <> struct SlabTraits<double> { static constexpr int NP = 4; };  // planes of double2

template <typename T>
__device__ __forceinline__ void slab_load(const uint4* S, int stride, int cell, C<T> (&x)[4]);
template <>
__device__ __forceinline__ void slab_load<float>(const uint4* S, int stride, int cell, float2 (&x)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(S + cell);
  const float4 b = *reinterpret_cast<const float4*>(S + stride + cell);
  x[0] = make_float2(a.x, a.y);
  x[1] = make_float2(a.z, a.w);
  x[2] = make_float2(b.x, b.y);
  x[3] = make_float2(b.z, b.w);
}
template <>
__device__ __forceinline__ void slab_load<double>(const uint4* S, int stride, int cell, double2 (&x)[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) x[a] = *reinterpret_cast<const double2*>(S + a * stride + cell);
}

// A1 sink spins alpha1 per lane: lane = ag * KPW + kk, alpha1 = ag * A1 + a'
template <typename T, int A1>
__device__ __forceinline__ void slab_load_a1(const uint4* S, int stride, int cell, int ag, C<T> (&x)[A1]);
template <>
__device__ __forceinline__ void slab_load_a1<float, 2>(const uint4* S, int stride, int cell, int ag, float2 (&x)[2]) {
  const float4 a = *reinterpret_cast<const float4*>(S + ag * stride + cell);
  x[0] = make_float2(a.x, a.y);
  x[1] = make_float2(a.z, a.w);
}
template <>
__device__ __forceinline__ void slab_load_a1<double, 1>(const uint4* S, int stride, int cell, int ag, double2 (&x)[1]) {
  x[0] = *reinterpret_cast<const double2*>(S + ag * stride + cell);
}

// N gather entries (N even) from a 16-byte aligned run: cell - base and coefficient
template <typename T, int N>
__device__ __forceinline__ void load_entries(const Ent<T>* p, int base, int (&cell)[N], T (&coef)[N]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int j = 0; j < N; j += 2) {
      const int4 w = __ldg(reinterpret_cast<const int4*>(p + j));
      cell[j] = w.x - base;
      coef[j] = __int_as_float(w.y);
      cell[j + 1] = w.z - base;
      coef[j + 1] = __int_as_float(w.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int4 w = __ldg(reinterpret_cast<const int4*>(p + j));
      cell[j] = w.x - base;
      coef[j] = __hiloint2double(w.w, w.z);
    }
  }
}

template <typename T, int A1, int SHAPE>
__device__ __forceinline__ void slab_item(const DevTerm& h, int k, bool active, int ag, const uint4* S1, int st1,
                                          int base1, const uint4* S2, int st2, int base2,
                                          const Ent<T>* __restrict__ E1, const Ent<T>* __restrict__ E2,
                                          T (&acc)[A1 * 32]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  C<T> v1[NH1][A1], v2[NH2][4];
#pragma unroll
  for (int hh = 0; hh < NH1; ++hh)
#pragma unroll
    for (int a = 0; a < A1; ++a) v1[hh][a] = czero<T>();
#pragma unroll
  for (int hh = 0; hh < NH2; ++hh)
#pragma unroll
    for (int a = 0; a < 4; ++a) v2[hh][a] = czero<T>();
  if (active) {
    const Ent<T>* p1 = E1 + h.off1 + (long long)k * NH1 * h.n1;
    for (int i = 0; i < h.n1; i += 2, p1 += 2 * NH1) {
      int cell[2 * NH1];
      T coef[2 * NH1];
      load_entries<T, 2 * NH1>(p1, base1, cell, coef);
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j) {
        C<T> x[A1];
        slab_load_a1<T, A1>(S1, st1, cell[j], ag, x);
#pragma unroll
        for (int a = 0; a < A1; ++a) crfma<T>(v1[j % NH1][a], coef[j], x[a]);
      }
    }
    const Ent<T>* p2 = E2 + h.off2 + (long long)k * NH2 * h.n2;
    for (int i = 0; i < h.n2; i += 2, p2 += 2 * NH2) {
      int cell[2 * NH2];
      T coef[2 * NH2];
      load_entries<T, 2 * NH2>(p2, base2, cell, coef);
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j) {
        C<T> x[4];
        slab_load<T>(S2, st2, cell[j], x);
#pragma unroll
        for (int b = 0; b < 4; ++b) crfma<T>(v2[j % NH2][b], coef[j], x[b]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < A1; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h1 = 0; h1 < NH1; ++h1)
#pragma unroll
        for (int h2 = 0; h2 < NH2; ++h2) {
          int s;  // alpha3 + 2 alpha4
          if (SHAPE == 0) s = h2;
          else if (SHAPE == 3) s = h1;
          else if (SHAPE == 1) s = h1 + 2 * h2;
          else s = h2 + 2 * h1;
          const int m = (a * 4 + b) * 4 + s;
          C<T> z = cmake<T>(acc[2 * m], acc[2 * m + 1]);
          cfma<T>(z, v1[h1][a], v2[h2][b]);
          acc[2 * m] = z.x;
          acc[2 * m + 1] = z.y;
        }
}

// Sum acc over the KPW lanes that share a spin group (lane bits below KPW);
// lane kk ends with the sums of acc[4 kk .. 4 kk + 3] in acc[0..3].  One
// stage per lane bit, from the highest: keep the half selected by the bit,
// send the other half to the partner lane.
template <typename T, int LEN, int S>
struct ReduceScatter {
  static __device__ __forceinline__ void run(T (&acc)[LEN], int lane) {
    if constexpr (S >= 1) {
      constexpr int n = 2 * S;  // live length after this stage = 4 * S; before it 8 * S
      const bool up = lane & S;
#pragma unroll
      for (int j = 0; j < 2 * n; ++j) {
        const T keep = up ? acc[2 * n + j] : acc[j];
        const T give = up ? acc[j] : acc[2 * n + j];
        acc[j] = keep + __shfl_xor_sync(0xffffffffu, give, S);
      }
      ReduceScatter<T, LEN, S / 2>::run(acc, lane);
    }
  }
};
template <typename T, int LEN, int KPW>
__device__ __forceinline__ void warp_reduce_scatter(T (&acc)[LEN], int lane) {
  static_assert(LEN == 4 * KPW, "four values per lane remain");
  ReduceScatter<T, LEN, KPW / 2>::run(acc, lane);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <typename T, int NW, int A1>
__global__ void __launch_bounds__(NW * 32) k_contract_slab(const C<T>* __restrict__ FB, int L, int ngroups,
                                                          const GroupHdr* __restrict__ groups,
                                                          const int* __restrict__ group_ch, const int* __restrict__ items,
                                                          const DevTerm* __restrict__ terms,
                                                          const Ent<T>* __restrict__ E1, const Ent<T>* __restrict__ E2,
                                                          int st1, int st2, int max_slot, C<T>* __restrict__ Ft) {
  constexpr int NP = SlabTraits<T>::NP;
  constexpr int NT = NW * 32;
  constexpr int KPW = 32 * A1 / 4;      // shared indices per warp pass
  constexpr int LEN = A1 * 32;          // accumulator values per lane
  static_assert(LEN / KPW == 4, "reduce-scatter leaves two complex sums per lane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint4* S1 = reinterpret_cast<uint4*>(smem_raw);
  uint4* S2 = S1 + NP * st1;
  C<T>* OUT = reinterpret_cast<C<T>*>(S2 + NP * st2);
  const long long V = (long long)L * L * L;
  const int q = blockIdx.x / ngroups;
  const int g = blockIdx.x % ngroups;
  const int qx = q % L, qy = (q / L) % L, qz = q / (L * L);
  const int qm = (L - qx) % L + L * ((L - qy) % L + L * ((L - qz) % L));
  const GroupHdr& gh = groups[g];
  const int base1 = gh.base1, n1 = gh.ncell1, base2 = gh.base2, n2 = gh.ncell2, nch = gh.nch, nslot = gh.nslot;
  // slabs: cell c, plane p = 16 bytes at ((base + c) * V + q) * 4 complex + 16 p bytes
  for (int i = threadIdx.x; i < NP * n1; i += NT) {
    const int c = i / NP, p = i % NP;
    cp_async16(S1 + p * st1 + c, reinterpret_cast<const char*>(FB + ((long long)(base1 + c) * V + q) * 4) + 16 * p);
  }
  for (int i = threadIdx.x; i < NP * n2; i += NT) {
    const int c = i / NP, p = i % NP;
    cp_async16(S2 + p * st2 + c, reinterpret_cast<const char*>(FB + ((long long)(base2 + c) * V + qm) * 4) + 16 * p);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < nslot * 64; i += NT) OUT[i] = czero<T>();
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ag = lane / KPW, kk = lane % KPW;
  T acc[LEN];
#pragma unroll
  for (int j = 0; j < LEN; ++j) acc[j] = T(0);
  int cur = -1;
  const int it0 = gh.item_off + gh.warp_off[w], it1 = gh.item_off + gh.warp_off[w + 1];
  for (int it = it0; it < it1; ++it) {
    const int term = items[2 * it], k0 = items[2 * it + 1];
    const DevTerm h = terms[term];
    if (h.pad != cur) {
      if (cur >= 0) {
        warp_reduce_scatter<T, LEN, KPW>(acc, lane);
        // lane (ag, kk) holds products 2 kk, 2 kk + 1 of spin group ag
        C<T>* o = OUT + (gh.out_base[w] + cur - gh.cfirst[w]) * 64 + ag * (A1 * 16) + 2 * kk;
        o[0] = cadd<T>(o[0], cmake<T>(acc[0], acc[1]));
        o[1] = cadd<T>(o[1], cmake<T>(acc[2], acc[3]));
#pragma unroll
        for (int j = 0; j < LEN; ++j) acc[j] = T(0);
      }
      cur = h.pad;
    }
    for (int kb = 0; kb < 32 && k0 + kb < h.K; kb += KPW) {
      const int k = k0 + kb + kk;
      const bool active = (kb + kk < 32) && k < h.K;
      switch (h.shape) {
        case 0: slab_item<T, A1, 0>(h, k, active, ag, S1, st1, base1, S2, st2, base2, E1, E2, acc); break;
        case 1: slab_item<T, A1, 1>(h, k, active, ag, S1, st1, base1, S2, st2, base2, E1, E2, acc); break;
        case 2: slab_item<T, A1, 2>(h, k, active, ag, S1, st1, base1, S2, st2, base2, E1, E2, acc); break;
        default: slab_item<T, A1, 3>(h, k, active, ag, S1, st1, base1, S2, st2, base2, E1, E2, acc); break;
      }
    }
  }
  if (cur >= 0) {
    warp_reduce_scatter<T, LEN, KPW>(acc, lane);
    C<T>* o = OUT + (gh.out_base[w] + cur - gh.cfirst[w]) * 64 + ag * (A1 * 16) + 2 * kk;
    o[0] = cadd<T>(o[0], cmake<T>(acc[0], acc[1]));
    o[1] = cadd<T>(o[1], cmake<T>(acc[2], acc[3]));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nch * 64; i += NT) {
    const int c = i / 64, m = i % 64;
    C<T> sum = czero<T>();
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {  // fixed order: the result does not depend on scheduling
      const int r = c - gh.cfirst[ww];
      if (r >= 0 && r < gh.out_base[ww + 1] - gh.out_base[ww]) sum = cadd<T>(sum, OUT[(gh.out_base[ww] + r) * 64 + m]);
    }
    // m = (alpha1*4 + alpha2)*4 + alpha3 + 2 alpha4  ->  output [alpha1][alpha2][alpha3][alpha4]
    const int spin = (m & ~3) + 2 * (m & 1) + ((m >> 1) & 1);
    Ft[((long long)group_ch[gh.ch_off + c] * 64 + spin) * V + q] = sum;
  }
}

// ---- persistent chunk contraction (FP32) -----------------------------------------
//
// A CTA owns one chunk (whole channels of a slab group whose gather tables,
// 16 bits per entry, fit in shared memory) and a block of consecutive
// momenta.  It loads the chunk's table once, then for each momentum waits for
// the two slabs (prefetched with cp.async into the other half of a double
// buffer while the previous momentum was being contracted), builds the
// effective blocks from shared memory and accumulates their products.
// Lane l owns shared index k0 + (l >> 1) and the sink spins alpha1 of pair
// (l & 1), so the two lanes reading the same B2 cell sit in one quarter-warp
// and their loads are one broadcast.

template <int NH>
__device__ __forceinline__ void load_codes(const unsigned short* p, unsigned (&e)[2 * NH]) {
  if constexpr (NH == 1) {
    const unsigned w = *reinterpret_cast<const unsigned*>(p);
    e[0] = w & 0xffffu; e[1] = w >> 16;
  } else if constexpr (NH == 2) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    e[0] = w.x & 0xffffu; e[1] = w.x >> 16; e[2] = w.y & 0xffffu; e[3] = w.y >> 16;
  } else {
    const uint4 w = *reinterpret_cast<const uint4*>(p);
    e[0] = w.x & 0xffffu; e[1] = w.x >> 16; e[2] = w.y & 0xffffu; e[3] = w.y >> 16;
    e[4] = w.z & 0xffffu; e[5] = w.z >> 16; e[6] = w.w & 0xffffu; e[7] = w.w >> 16;
  }
}

__device__ __forceinline__ float decode_coef(unsigned e, const float* codes) {
  const float a = codes[e >> 11];
  return (e & 1024u) ? -a : a;
}

template <int SHAPE>
__device__ __forceinline__ void chunk_item(const DevTerm& h, int k, bool active, int ag, const unsigned short* T1,
                                           const unsigned short* T2, const uint4* S1, int st1, const uint4* S2,
                                           int st2, const float* cc, float (&acc)[64]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  float2 v1[NH1][2], v2[NH2][4];
#pragma unroll
  for (int hh = 0; hh < NH1; ++hh) v1[hh][0] = v1[hh][1] = make_float2(0.f, 0.f);
#pragma unroll
  for (int hh = 0; hh < NH2; ++hh)
#pragma unroll
    for (int b = 0; b < 4; ++b) v2[hh][b] = make_float2(0.f, 0.f);
  if (active) {
    const unsigned short* p1 = T1 + k * NH1 * h.n1;
    for (int i = 0; i < h.n1; i += 2, p1 += 2 * NH1) {
      unsigned e[2 * NH1];
      load_codes<NH1>(p1, e);
#pragma unroll
      for (int j = 0; j < 2 * NH1; ++j) {
        const float c = decode_coef(e[j], cc);
        const float4 x = *reinterpret_cast<const float4*>(S1 + ag * st1 + (e[j] & 1023u));
        v1[j % NH1][0].x = fmaf(c, x.x, v1[j % NH1][0].x);
        v1[j % NH1][0].y = fmaf(c, x.y, v1[j % NH1][0].y);
        v1[j % NH1][1].x = fmaf(c, x.z, v1[j % NH1][1].x);
        v1[j % NH1][1].y = fmaf(c, x.w, v1[j % NH1][1].y);
      }
    }
    const unsigned short* p2 = T2 + k * NH2 * h.n2;
    for (int i = 0; i < h.n2; i += 2, p2 += 2 * NH2) {
      unsigned e[2 * NH2];
      load_codes<NH2>(p2, e);
#pragma unroll
      for (int j = 0; j < 2 * NH2; ++j) {
        const float c = decode_coef(e[j], cc);
        const unsigned cell = e[j] & 1023u;
        const float4 x = *reinterpret_cast<const float4*>(S2 + cell);
        const float4 y = *reinterpret_cast<const float4*>(S2 + st2 + cell);
        crfma<float>(v2[j % NH2][0], c, make_float2(x.x, x.y));
        crfma<float>(v2[j % NH2][1], c, make_float2(x.z, x.w));
        crfma<float>(v2[j % NH2][2], c, make_float2(y.x, y.y));
        crfma<float>(v2[j % NH2][3], c, make_float2(y.z, y.w));
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h1 = 0; h1 < NH1; ++h1)
#pragma unroll
        for (int h2 = 0; h2 < NH2; ++h2) {
          int s;  // alpha3 + 2 alpha4
          if (SHAPE == 0) s = h2;
          else if (SHAPE == 3) s = h1;
          else if (SHAPE == 1) s = h1 + 2 * h2;
          else s = h2 + 2 * h1;
          const int m = (a * 4 + b) * 4 + s;
          float2 z = make_float2(acc[2 * m], acc[2 * m + 1]);
          cfma<float>(z, v1[h1][a], v2[h2][b]);
          acc[2 * m] = z.x;
          acc[2 * m + 1] = z.y;
        }
}

// reduce 64 values over the 16 lanes of one spin pair (xor masks 16, 8, 4, 2);
// lane l ends with the sums of acc[4 (l >> 1) .. 4 (l >> 1) + 3]
template <int M>
__device__ __forceinline__ void pair_reduce_stage(float (&acc)[64], int lane) {
  if constexpr (M >= 2) {
    constexpr int n = 2 * M;  // kept length after this stage
    const bool up = lane & M;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const float keep = up ? acc[n + j] : acc[j];
      const float give = up ? acc[j] : acc[n + j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, give, M);
    }
    pair_reduce_stage<M / 2>(acc, lane);
  }
}

__device__ __forceinline__ void cp_async16b(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_chunk(
    const float2* __restrict__ FB, int L, int nchunks, int qb, const ChunkHdr* __restrict__ chunks,
    const int* __restrict__ group_ch, const int* __restrict__ items, const DevTerm* __restrict__ terms,
    const int* __restrict__ tab_off, const unsigned short* __restrict__ tab, const float* __restrict__ codes, int st1,
    int st2,
    int max_slot, int max_tab, float2* __restrict__ Ft) {
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned short* TAB = reinterpret_cast<unsigned short*>(smem_raw);
  uint4* SB = reinterpret_cast<uint4*>(smem_raw + (size_t)max_tab * 2);  // max_tab is a multiple of 8
  const int slab = 2 * st1 + 2 * st2;                                     // uint4 per buffer
  float2* OUT = reinterpret_cast<float2*>(SB + 2 * slab);
  float* CODES = reinterpret_cast<float*>(OUT + max_slot * 64);
  if (threadIdx.x < 32) CODES[threadIdx.x] = codes[threadIdx.x];
  const long long V = (long long)L * L * L;
  const int ci = blockIdx.x % nchunks;
  const long long q_begin = (long long)(blockIdx.x / nchunks) * qb;
  const long long q_end = min(V, q_begin + qb);
  const ChunkHdr& ck = chunks[ci];
  const int base1 = ck.base1, n1 = ck.ncell1, base2 = ck.base2, n2 = ck.ncell2;

  auto issue_slabs = [&](long long q, uint4* S) {
    const int qx = (int)(q % L), qy = (int)((q / L) % L), qz = (int)(q / ((long long)L * L));
    const long long qm = (L - qx) % L + L * ((L - qy) % L + (long long)L * ((L - qz) % L));
    for (int i = threadIdx.x; i < 2 * n1; i += NT) {
      const int c = i >> 1, p = i & 1;
      cp_async16b(S + p * st1 + c, reinterpret_cast<const char*>(FB + ((long long)(base1 + c) * V + q) * 4) + 16 * p);
    }
    uint4* S2 = S + 2 * st1;
    for (int i = threadIdx.x; i < 2 * n2; i += NT) {
      const int c = i >> 1, p = i & 1;
      cp_async16b(S2 + p * st2 + c, reinterpret_cast<const char*>(FB + ((long long)(base2 + c) * V + qm) * 4) + 16 * p);
    }
  };

  for (int i = threadIdx.x; i < ck.tab_len / 8; i += NT)
    cp_async16b(TAB + 8 * i, tab + ck.tab_off + 8 * i);
  if (q_begin < q_end) issue_slabs(q_begin, SB);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < ck.nslot * 64; i += NT) OUT[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ag = lane & 1, kk = lane >> 1;
  const int it0 = ck.item_off + ck.warp_off[w], it1 = ck.item_off + ck.warp_off[w + 1];
  for (long long q = q_begin; q < q_end; ++q) {
    uint4* S = SB + ((q - q_begin) & 1) * slab;
    if (q + 1 < q_end) issue_slabs(q + 1, SB + ((q + 1 - q_begin) & 1) * slab);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const uint4* S1 = S;
    const uint4* S2 = S + 2 * st1;
    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.f;
    int cur = -1;
    for (int it = it0; it < it1; ++it) {
      const int term = items[2 * it], k0 = items[2 * it + 1];
      const DevTerm h = terms[term];
      const int local = h.pad - ck.ch_local0;
      if (local != cur) {
        if (cur >= 0) {
          pair_reduce_stage<16>(acc, lane);
          float2* o = OUT + (ck.out_base[w] + cur - ck.cfirst[w]) * 64 + ag * 32 + 2 * kk;
          o[0].x += acc[0]; o[0].y += acc[1]; o[1].x += acc[2]; o[1].y += acc[3];
#pragma unroll
          for (int j = 0; j < 64; ++j) acc[j] = 0.f;
        }
        cur = local;
      }
      const unsigned short* T1 = TAB + tab_off[2 * term];
      const unsigned short* T2 = TAB + tab_off[2 * term + 1];
      for (int kb = 0; kb < 32 && k0 + kb < h.K; kb += 16) {
        const int k = k0 + kb + kk;
        const bool active = k < h.K;
        switch (h.shape) {
          case 0: chunk_item<0>(h, k, active, ag, T1, T2, S1, st1, S2, st2, CODES, acc); break;
          case 1: chunk_item<1>(h, k, active, ag, T1, T2, S1, st1, S2, st2, CODES, acc); break;
          case 2: chunk_item<2>(h, k, active, ag, T1, T2, S1, st1, S2, st2, CODES, acc); break;
          default: chunk_item<3>(h, k, active, ag, T1, T2, S1, st1, S2, st2, CODES, acc); break;
        }
      }
    }
    if (cur >= 0) {
      pair_reduce_stage<16>(acc, lane);
      float2* o = OUT + (ck.out_base[w] + cur - ck.cfirst[w]) * 64 + ag * 32 + 2 * kk;
      o[0].x += acc[0]; o[0].y += acc[1]; o[1].x += acc[2]; o[1].y += acc[3];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ck.nch * 64; i += NT) {
      const int c = i / 64, m = i % 64;
      float2 sum = make_float2(0.f, 0.f);
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) {  // fixed order
        const int r = c - ck.cfirst[ww];
        if (r >= 0 && r < ck.out_base[ww + 1] - ck.out_base[ww]) {
          float2& v = OUT[(ck.out_base[ww] + r) * 64 + m];
          sum.x += v.x;
          sum.y += v.y;
          v = make_float2(0.f, 0.f);
        }
      }
      const int spin = (m & ~3) + 2 * (m & 1) + ((m >> 1) & 1);
      Ft[((long long)group_ch[ck.ch_off + c] * 64 + spin) * V + q] = sum;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
  }
}

// ---- persistent chunk contraction, second form (FP32) -------------------------------------
//
// Same work split and output order as k_contract_chunk; the inner loops are
// cheaper per table entry:
//  * the coefficient comes from a 64-entry signed table indexed by the top six
//    bits of the entry (code * 2 + sign), one shared load and no select;
//  * the two 16-byte halves of a cell's four spins sit next to each other in
//    the slab, so one base address serves both;
//  * lanes past the end of a term read a row of zero-coefficient entries
//    instead of branching, so the warp never diverges.

constexpr int CHUNK2_ZROW = 128;  // zero-coefficient entries (>= max over terms of n * held spins)
// slab plane stride (16-byte units): a compile-time constant so that the second
// plane of a cell is an immediate offset; >= the cells of any stored type, and 4
// mod 8 so that the two planes of one cell fall in different bank groups
constexpr int CHUNK2_ST = 948;

template <int SHAPE>
__device__ __forceinline__ void chunk2_item(int n1, int n2, const unsigned short* p1, const unsigned short* p2,
                                            const uint4* S1a, const uint4* S2, const float* sc, float (&acc)[64]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  float2 v1[NH1][2], v2[NH2][4];
#pragma unroll
  for (int hh = 0; hh < NH1; ++hh) v1[hh][0] = v1[hh][1] = make_float2(0.f, 0.f);
#pragma unroll
  for (int hh = 0; hh < NH2; ++hh)
#pragma unroll
    for (int b = 0; b < 4; ++b) v2[hh][b] = make_float2(0.f, 0.f);
  for (int i = 0; i < n1; i += 2, p1 += 2 * NH1) {
    unsigned e[2 * NH1];
    load_codes<NH1>(p1, e);
#pragma unroll
    for (int j = 0; j < 2 * NH1; ++j) {
      const float c = sc[e[j] >> 10];
      const float4 x = *reinterpret_cast<const float4*>(S1a + (e[j] & 1023u));
      v1[j % NH1][0].x = fmaf(c, x.x, v1[j % NH1][0].x);
      v1[j % NH1][0].y = fmaf(c, x.y, v1[j % NH1][0].y);
      v1[j % NH1][1].x = fmaf(c, x.z, v1[j % NH1][1].x);
      v1[j % NH1][1].y = fmaf(c, x.w, v1[j % NH1][1].y);
    }
  }
  for (int i = 0; i < n2; i += 2, p2 += 2 * NH2) {
    unsigned e[2 * NH2];
    load_codes<NH2>(p2, e);
#pragma unroll
    for (int j = 0; j < 2 * NH2; ++j) {
      const float c = sc[e[j] >> 10];
      const uint4* b = S2 + (e[j] & 1023u);
      const float4 x = *reinterpret_cast<const float4*>(b);
      const float4 y = *reinterpret_cast<const float4*>(b + CHUNK2_ST);
      crfma<float>(v2[j % NH2][0], c, make_float2(x.x, x.y));
      crfma<float>(v2[j % NH2][1], c, make_float2(x.z, x.w));
      crfma<float>(v2[j % NH2][2], c, make_float2(y.x, y.y));
      crfma<float>(v2[j % NH2][3], c, make_float2(y.z, y.w));
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h1 = 0; h1 < NH1; ++h1)
#pragma unroll
        for (int h2 = 0; h2 < NH2; ++h2) {
          int s;  // alpha3 + 2 alpha4
          if (SHAPE == 0) s = h2;
          else if (SHAPE == 3) s = h1;
          else if (SHAPE == 1) s = h1 + 2 * h2;
          else s = h2 + 2 * h1;
          const int m = (a * 4 + b) * 4 + s;
          float2 z = make_float2(acc[2 * m], acc[2 * m + 1]);
          cfma<float>(z, v1[h1][a], v2[h2][b]);
          acc[2 * m] = z.x;
          acc[2 * m + 1] = z.y;
        }
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_chunk2(
    const float2* __restrict__ FB, int L, int nchunks, int qb, const ChunkHdr* __restrict__ chunks,
    const int* __restrict__ group_ch, const int* __restrict__ items, const DevTerm* __restrict__ terms,
    const int* __restrict__ tab_off, const unsigned short* __restrict__ tab, const float* __restrict__ codes, int st1,
    int st2, int max_slot, int max_tab, float2* __restrict__ Ft) {
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned short* TAB = reinterpret_cast<unsigned short*>(smem_raw);
  unsigned short* ZROW = TAB + max_tab;                                               // max_tab % 8 == 0
  uint4* SB = reinterpret_cast<uint4*>(smem_raw + (size_t)(max_tab + CHUNK2_ZROW) * 2);
  constexpr int slab = 4 * CHUNK2_ST;                                                 // uint4 per buffer
  float2* OUT = reinterpret_cast<float2*>(SB + 2 * slab);
  float* SC = reinterpret_cast<float*>(OUT + max_slot * 64);
  if (threadIdx.x < 64) {
    const float a = codes[threadIdx.x >> 1];
    SC[threadIdx.x] = (threadIdx.x & 1) ? -a : a;
  }
  for (int i = threadIdx.x; i < CHUNK2_ZROW; i += NT) ZROW[i] = (unsigned short)(31u << 11);
  const long long V = (long long)L * L * L;
  const int ci = blockIdx.x % nchunks;
  const long long q_begin = (long long)(blockIdx.x / nchunks) * qb;
  const long long q_end = min(V, q_begin + qb);
  const ChunkHdr& ck = chunks[ci];
  const int base1 = ck.base1, n1c = ck.ncell1, base2 = ck.base2, n2c = ck.ncell2;

  // slab layout: four planes of CHUNK2_ST 16-byte slots (side 1 spins 0-1, side 1
  // spins 2-3, side 2 spins 0-1, side 2 spins 2-3), indexed by cell
  auto issue_slabs = [&](long long q, uint4* S) {
    const int qx = (int)(q % L), qy = (int)((q / L) % L), qz = (int)(q / ((long long)L * L));
    const long long qm = (L - qx) % L + L * ((L - qy) % L + (long long)L * ((L - qz) % L));
    for (int i = threadIdx.x; i < 2 * n1c; i += NT) {
      const int c = i >> 1, p = i & 1;
      cp_async16b(S + p * CHUNK2_ST + c,
                  reinterpret_cast<const char*>(FB + ((long long)(base1 + c) * V + q) * 4) + 16 * p);
    }
    uint4* S2 = S + 2 * CHUNK2_ST;
    for (int i = threadIdx.x; i < 2 * n2c; i += NT) {
      const int c = i >> 1, p = i & 1;
      cp_async16b(S2 + p * CHUNK2_ST + c,
                  reinterpret_cast<const char*>(FB + ((long long)(base2 + c) * V + qm) * 4) + 16 * p);
    }
  };

  for (int i = threadIdx.x; i < ck.tab_len / 8; i += NT)
    cp_async16b(TAB + 8 * i, tab + ck.tab_off + 8 * i);
  if (q_begin < q_end) issue_slabs(q_begin, SB);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < ck.nslot * 64; i += NT) OUT[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ag = lane & 1, kk = lane >> 1;
  const int it0 = ck.item_off + ck.warp_off[w], it1 = ck.item_off + ck.warp_off[w + 1];
  for (long long q = q_begin; q < q_end; ++q) {
    uint4* S = SB + ((q - q_begin) & 1) * slab;
    if (q + 1 < q_end) issue_slabs(q + 1, SB + ((q + 1 - q_begin) & 1) * slab);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const uint4* S1a = S + ag * CHUNK2_ST;
    const uint4* S2 = S + 2 * CHUNK2_ST;
    float acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.f;
    int cur = -1;
    for (int it = it0; it < it1; ++it) {
      const int term = items[2 * it], k0 = items[2 * it + 1];
      const DevTerm h = terms[term];
      const int local = h.pad - ck.ch_local0;
      if (local != cur) {
        if (cur >= 0) {
          pair_reduce_stage<16>(acc, lane);
          float2* o = OUT + (ck.out_base[w] + cur - ck.cfirst[w]) * 64 + ag * 32 + 2 * kk;
          o[0].x += acc[0]; o[0].y += acc[1]; o[1].x += acc[2]; o[1].y += acc[3];
#pragma unroll
          for (int j = 0; j < 64; ++j) acc[j] = 0.f;
        }
        cur = local;
      }
      const unsigned short* T1 = TAB + tab_off[2 * term];
      const unsigned short* T2 = TAB + tab_off[2 * term + 1];
      const int nh1 = 1 << ((h.shape & 1) + ((h.shape >> 1) & 1));
      for (int kb = 0; kb < 32 && k0 + kb < h.K; kb += 16) {
        const int k = k0 + kb + kk;
        const bool active = k < h.K;
        const unsigned short* p1 = active ? T1 + k * nh1 * h.n1 : ZROW;
        const unsigned short* p2 = active ? T2 + k * (4 / nh1) * h.n2 : ZROW;
        switch (h.shape) {
          case 0: chunk2_item<0>(h.n1, h.n2, p1, p2, S1a, S2, SC, acc); break;
          case 1: chunk2_item<1>(h.n1, h.n2, p1, p2, S1a, S2, SC, acc); break;
          case 2: chunk2_item<2>(h.n1, h.n2, p1, p2, S1a, S2, SC, acc); break;
          default: chunk2_item<3>(h.n1, h.n2, p1, p2, S1a, S2, SC, acc); break;
        }
      }
    }
    if (cur >= 0) {
      pair_reduce_stage<16>(acc, lane);
      float2* o = OUT + (ck.out_base[w] + cur - ck.cfirst[w]) * 64 + ag * 32 + 2 * kk;
      o[0].x += acc[0]; o[0].y += acc[1]; o[1].x += acc[2]; o[1].y += acc[3];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ck.nch * 64; i += NT) {
      const int c = i / 64, m = i % 64;
      float2 sum = make_float2(0.f, 0.f);
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) {  // fixed order
        const int r = c - ck.cfirst[ww];
        if (r >= 0 && r < ck.out_base[ww + 1] - ck.out_base[ww]) {
          float2& v = OUT[(ck.out_base[ww] + r) * 64 + m];
          sum.x += v.x;
          sum.y += v.y;
          v = make_float2(0.f, 0.f);
        }
      }
      const int spin = (m & ~3) + 2 * (m & 1) + ((m >> 1) & 1);
      Ft[((long long)group_ch[ck.ch_off + c] * 64 + spin) * V + q] = sum;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
  }
}

// f * 2^ex as a double, by integer operations on the bit pattern (exact): a
// normal FP32 value keeps its sign and mantissa and gets the FP64 exponent
// E - 127 + 1023 + ex; zeros stay zeros; FP32 subnormals, infinities, NaNs
// and results outside the FP64 normal range go through ldexp.
__device__ __forceinline__ double scaled_double(float f, int ex) {
  const unsigned b = __float_as_uint(f);
  const unsigned E = (b >> 23) & 255u;
  const int DE = (int)E + (1023 - 127) + ex;
  if (E - 1u < 254u && DE > 0 && DE < 2047) {
    // high word: sign, 11-bit exponent, top 20 mantissa bits; low word: last 3 mantissa bits
    const unsigned hi = (b & 0x80000000u) | ((unsigned)DE << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return ldexp((double)f, ex);
}

// out[ch * ch_stride + c*V + r] = Ft[ch][c][r] * 2^(sum_f e_f n_f) / V
// FP32 input: 1/V applied in FP32, the power of two added to the exponent
// (no FP64 arithmetic, which is scarce on GB300); two complex values per
// 16-byte load and RS independent loads in flight per thread.  FP64 input:
// FP64 multiply.
template <typename T>
__global__ void __launch_bounds__(256) k_restore(const C<T>* __restrict__ Ft, long long V, const int* __restrict__ ch_fl,
                                                 const int* __restrict__ exps, int nflav, double2* __restrict__ out,
                                                 long long ch_stride, long long norm) {
  const int ch = blockIdx.y;
  int ex = 0;  // sum over the propagators of (their exponent) x (their quarks in the sink pair)
  for (int f = 0; f < nflav; ++f) ex += exps[f] * ch_fl[3 * ch + f];
  const long long n = 64 * V;
  const C<T>* src = Ft + ch * n;
  double2* dst = out + ch * ch_stride;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(T) == 4) {
    constexpr int RS = 4;
    const float inv = 1.0f / (float)norm;
    const float4* s4 = reinterpret_cast<const float4*>(src);  // n is even, Ft 16-byte aligned
    const long long n2 = n / 2;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n2; i0 += RS * stride) {
      float4 z[RS];
#pragma unroll
      for (int u = 0; u < RS; ++u) {
        const long long i = i0 + u * stride;
        z[u] = i < n2 ? __ldcs(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < RS; ++u) {
        const long long i = i0 + u * stride;
        if (i < n2) {
          dst[2 * i] = make_double2(scaled_double(z[u].x * inv, ex), scaled_double(z[u].y * inv, ex));
          dst[2 * i + 1] = make_double2(scaled_double(z[u].z * inv, ex), scaled_double(z[u].w * inv, ex));
        }
      }
    }
  } else {
    const double scale = ldexp(1.0, ex) / (double)norm;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const C<T> z = src[i];
      dst[i] = make_double2((double)z.x * scale, (double)z.y * scale);
    }
  }
}

}  // namespace

template <typename T, int A1, int NT>
cudaError_t launch_contract_cfg(const C<T>* FB, int L, const DevTerm* terms, const int* ch_tb, int nch,
                                const Ent<T>* e1, const Ent<T>* e2, C<T>* Ft, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  dim3 grid((unsigned)(nch * (4 / A1)), (unsigned)((V + NT - 1) / NT));
  k_contract<T, A1, NT><<<grid, NT, 0, st>>>(FB, L, terms, ch_tb, e1, e2, Ft);
  return cudaGetLastError();
}

// cfg: alpha1 values per thread (1, 2, 4) x 10 + threads per block / 32 (1, 2, 4)
template <typename T>
cudaError_t launch_contract(const C<T>* FB, int L, const DevTerm* terms, const int* ch_tb, int nch, const Ent<T>* e1,
                            const Ent<T>* e2, C<T>* Ft, int cfg, cudaStream_t st) {
  if (cfg == 0) cfg = sizeof(T) == 4 ? 42 : 21;
  if (nch * 4 > 2147483647 / 4) return cudaErrorInvalidValue;
  switch (cfg) {
#define NBS_CFG(a, w) \
  case a * 10 + w: return launch_contract_cfg<T, a, 32 * w>(FB, L, terms, ch_tb, nch, e1, e2, Ft, st);
    NBS_CFG(1, 1) NBS_CFG(1, 2) NBS_CFG(1, 4)
    NBS_CFG(2, 1) NBS_CFG(2, 2) NBS_CFG(2, 4)
    NBS_CFG(4, 1) NBS_CFG(4, 2) NBS_CFG(4, 4)
#undef NBS_CFG
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
size_t slab_smem_bytes(int st1, int st2, int max_slot) {
  return (size_t)SlabTraits<T>::NP * 16 * (st1 + st2) + (size_t)max_slot * 64 * sizeof(C<T>);
}

template <typename T>
cudaError_t launch_contract_slab(const C<T>* FB, int L, int ngroups, const void* groups, const int* group_ch,
                                 const int* items, const DevTerm* terms, const Ent<T>* e1, const Ent<T>* e2, int st1,
                                 int st2, int max_slot, C<T>* Ft, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  const size_t sm = slab_smem_bytes<T>(st1, st2, max_slot);
  auto kern = k_contract_slab<T, NBS_SLAB_WARPS, sizeof(T) == 4 ? 2 : 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nblk = V * ngroups;
  if (nblk > 2147483647LL) return cudaErrorInvalidValue;
  kern<<<(unsigned)nblk, NBS_SLAB_WARPS * 32, sm, st>>>(FB, L, ngroups, (const GroupHdr*)groups, group_ch, items,
                                                       terms, e1, e2, st1, st2, max_slot, Ft);
  return cudaGetLastError();
}

size_t chunk_smem_bytes(int st1, int st2, int max_slot, int max_tab) {
  return (size_t)max_tab * 2 + (size_t)2 * (2 * st1 + 2 * st2) * 16 + (size_t)max_slot * 64 * sizeof(float2) + 128;
}

cudaError_t launch_contract_chunk(const float2* FB, int L, int nchunks, int qb, const void* chunks, const int* group_ch,
                                  const int* items, const DevTerm* terms, const int* tab_off, const unsigned short* tab,
                                  const float* codes, int st1, int st2, int max_slot, int max_tab, float2* Ft,
                                  cudaStream_t st) {
  const long long V = (long long)L * L * L;
  const size_t sm = chunk_smem_bytes(st1, st2, max_slot, max_tab);
  auto kern = k_contract_chunk<NBS_CHUNK_WARPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL || max_tab % 8) return cudaErrorInvalidValue;
  kern<<<(unsigned)(nqb * nchunks), NBS_CHUNK_WARPS * 32, sm, st>>>(FB, L, nchunks, qb, (const ChunkHdr*)chunks,
                                                                    group_ch, items, terms, tab_off, tab, codes, st1, st2,
                                                                    max_slot, max_tab, Ft);
  return cudaGetLastError();
}

size_t chunk2_smem_bytes(int st1, int st2, int max_slot, int max_tab) {
  (void)st1;
  (void)st2;
  return (size_t)(max_tab + CHUNK2_ZROW) * 2 + (size_t)2 * 4 * CHUNK2_ST * 16 +
         (size_t)max_slot * 64 * sizeof(float2) + 64 * sizeof(float);
}

cudaError_t launch_contract_chunk2(const float2* FB, int L, int nchunks, int qb, const void* chunks,
                                   const int* group_ch, const int* items, const DevTerm* terms, const int* tab_off,
                                   const unsigned short* tab, const float* codes, int st1, int st2, int max_slot,
                                   int max_tab, int max_row, float2* Ft, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  const size_t sm = chunk2_smem_bytes(st1, st2, max_slot, max_tab);
  if (max_row > CHUNK2_ZROW || max_tab % 8 || st1 > CHUNK2_ST || st2 > CHUNK2_ST) return cudaErrorInvalidValue;
  auto kern = k_contract_chunk2<NBS_CHUNK_WARPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL) return cudaErrorInvalidValue;
  kern<<<(unsigned)(nqb * nchunks), NBS_CHUNK_WARPS * 32, sm, st>>>(FB, L, nchunks, qb, (const ChunkHdr*)chunks,
                                                                    group_ch, items, terms, tab_off, tab, codes, st1, st2,
                                                                    max_slot, max_tab, Ft);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restore(const C<T>* Ft, int V, int nch, const int* ch_fl, const int* exps, int nflav, double2* out,
                           long long ch_stride, cudaStream_t st, long long norm) {
  long long n = 64LL * V;
  if (sizeof(T) == 4) n /= 8;  // 16-byte loads, four per thread per pass
  int bx = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096));
  dim3 grid(bx, nch);
  k_restore<T><<<grid, 256, 0, st>>>(Ft, (long long)V, ch_fl, exps, nflav, out, ch_stride, norm ? norm : (long long)V);
  return cudaGetLastError();
}

template cudaError_t launch_contract<float>(const float2*, int, const DevTerm*, const int*, int, const Ent<float>*,
                                            const Ent<float>*, float2*, int, cudaStream_t);
template cudaError_t launch_contract<double>(const double2*, int, const DevTerm*, const int*, int, const Ent<double>*,
                                             const Ent<double>*, double2*, int, cudaStream_t);
template cudaError_t launch_contract_slab<float>(const float2*, int, int, const void*, const int*, const int*,
                                                 const DevTerm*, const Ent<float>*, const Ent<float>*, int, int, int,
                                                 float2*, cudaStream_t);
template cudaError_t launch_contract_slab<double>(const double2*, int, int, const void*, const int*, const int*,
                                                  const DevTerm*, const Ent<double>*, const Ent<double>*, int, int, int,
                                                  double2*, cudaStream_t);
template size_t slab_smem_bytes<float>(int, int, int);
template size_t slab_smem_bytes<double>(int, int, int);
template cudaError_t launch_restore<float>(const float2*, int, int, const int*, const int*, int, double2*, long long,
                                           cudaStream_t, long long);
template cudaError_t launch_restore<double>(const double2*, int, int, const int*, const int*, int, double2*, long long,
                                            cudaStream_t, long long);

}  // namespace nbs
