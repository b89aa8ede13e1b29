// kernels_quad.cu -- the effective-block product of Eq. (4.3), FP32, with four
// lanes per shared index (the quad-lane contraction).
//
// A CTA of 16 warps keeps one chunk of channels' compressed gather tables in
// shared memory and sweeps a block of momenta, staging the two momentum slabs
// of each q (B1's stored type at q, B2's at -q) into a double buffer with TMA
// boxes issued by one thread (tma.cuh; 16-byte cp.async by all threads where
// the tensor map cannot be encoded).  Inside a warp, lane 4 kq + a owns shared index k0 + kq of the
// current 8-index step and spin a: it builds E1[alpha1 = a][h1] and
// E2[alpha2 = a][h2] (one 8-byte load and two FMAs per gather entry), takes
// the other three alpha2 rows of E2 from the lanes of its quad by warp
// shuffles, and accumulates its 16 complex products F[alpha1 = a][alpha2]
// [alpha3 alpha4] += E1 E2 in 32 registers.  The small accumulator keeps a
// thread under 128 registers, so one CTA of 16 warps fits an SM.  Each warp
// walks its range of steps as runs of one table run (QuadSeg, plan.h), staged
// in shared memory once per CTA, so the term form is dispatched once per run;
// when a warp moves to another channel it sums its partial products over the
// eight shared-index lanes and adds them to the channel's slot in shared
// memory; the slots of all warps are added in a fixed order.
#include <cstring>

#include "common.cuh"
#include "plan.h"
#include "tma.cuh"

namespace nbs {

namespace {

constexpr int QUAD_ZROW = 128;  // zero-coefficient entries (>= max over terms of n * held spins)
constexpr int QUAD_ST = 944;    // cells per slab side (>= the cells of any stored type)

__device__ __forceinline__ void cp_async16q(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// 2 NH consecutive 16-bit entries (shared index row, pair of i) in one load
template <int NH>
__device__ __forceinline__ void load_entries(const unsigned short* p, unsigned (&e)[2 * NH]) {
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

// one 8-index step of one term: gather this lane's rows of E1 and E2 (entries
// ordered [i][h], coefficient = sc[entry >> 10] (signed code), cell = entry &
// 1023), exchange E2 rows inside the quad, accumulate the products.  Lane-
// relative alpha2: acc[d][s] holds alpha2 = a ^ d.
// I1, I2 > 0: the gather lists hold exactly 2 I1 (2 I2) entries per held spin,
// and the loops are unrolled into straight-line code (the common term forms);
// 0: lengths n1, n2 at run time
template <int SHAPE, int I1, int I2>
__device__ __forceinline__ void quad_step(int n1, int n2, const unsigned short* p1, const unsigned short* p2,
                                          const float2* S1a, const float2* S2a, const float* sc, float (&acc)[32]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  float2 v1[NH1], v2[4][NH2];
#pragma unroll
  for (int h = 0; h < NH1; ++h) v1[h] = make_float2(0.f, 0.f);
#pragma unroll
  for (int h = 0; h < NH2; ++h) v2[0][h] = make_float2(0.f, 0.f);
  if (I1) n1 = 2 * I1;
  if (I2) n2 = 2 * I2;
#pragma unroll
  for (int i = 0; i < (I1 ? 2 * I1 : n1); i += 2, p1 += 2 * NH1) {
    unsigned e[2 * NH1];
    load_entries<NH1>(p1, e);
#pragma unroll
    for (int j = 0; j < 2 * NH1; ++j) {
      const float c = sc[e[j] >> 10];
      const float2 x = S1a[4 * (e[j] & 1023u)];
      v1[j % NH1].x = fmaf(c, x.x, v1[j % NH1].x);
      v1[j % NH1].y = fmaf(c, x.y, v1[j % NH1].y);
    }
  }
#pragma unroll
  for (int i = 0; i < (I2 ? 2 * I2 : n2); i += 2, p2 += 2 * NH2) {
    unsigned e[2 * NH2];
    load_entries<NH2>(p2, e);
#pragma unroll
    for (int j = 0; j < 2 * NH2; ++j) {
      const float c = sc[e[j] >> 10];
      const float2 x = S2a[4 * (e[j] & 1023u)];
      v2[0][j % NH2].x = fmaf(c, x.x, v2[0][j % NH2].x);
      v2[0][j % NH2].y = fmaf(c, x.y, v2[0][j % NH2].y);
    }
  }
#pragma unroll
  for (int d = 1; d < 4; ++d)
#pragma unroll
    for (int h = 0; h < NH2; ++h) {
      v2[d][h].x = __shfl_xor_sync(0xffffffffu, v2[0][h].x, d);
      v2[d][h].y = __shfl_xor_sync(0xffffffffu, v2[0][h].y, d);
    }
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int h1 = 0; h1 < NH1; ++h1)
#pragma unroll
      for (int h2 = 0; h2 < NH2; ++h2) {
        int s;  // alpha3 + 2 alpha4
        if (SHAPE == 0) s = h2;
        else if (SHAPE == 3) s = h1;
        else if (SHAPE == 1) s = h1 + 2 * h2;
        else s = h2 + 2 * h1;
        float2 z = make_float2(acc[2 * (4 * d + s)], acc[2 * (4 * d + s) + 1]);
        cfma<float>(z, v1[h1], v2[d][h2]);
        acc[2 * (4 * d + s)] = z.x;
        acc[2 * (4 * d + s) + 1] = z.y;
      }
}

// sum a lane's 32 partial floats over the eight lanes of equal spin a (xor 4,
// 8, 16), halving the kept length each stage: lane 4 kq + a ends with floats
// 4 kq .. 4 kq + 3 (complex 2 kq, 2 kq + 1 of its 16) summed over kq
template <int M>
__device__ __forceinline__ void quad_reduce(float (&acc)[32], int lane) {
  if constexpr (M >= 4) {
    constexpr int n = M;  // kept length after this stage
    const bool up = lane & M;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const float keep = up ? acc[n + j] : acc[j];
      const float give = up ? acc[j] : acc[n + j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, give, M);
    }
    quad_reduce<M / 2>(acc, lane);
  }
}

// ---- runs, flush, kernel -----------------------------------------------------
// The step loop of a run only advances two table pointers; the channel flush
// indexes alpha2 = a ^ d directly (the reduction never mixes spins a).

template <int SHAPE, int I1, int I2>
__device__ __forceinline__ void qseg_run(const QuadSeg& sg, int kq, const unsigned short* TAB,
                                         const unsigned short* ZROW, const float2* S1a, const float2* S2a,
                                         const float* sc, float (&acc)[32]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  const int n1 = I1 ? 2 * I1 : sg.n1, n2 = I2 ? 2 * I2 : sg.n2;
  const int r1 = NH1 * n1, r2 = NH2 * n2;  // entries per shared index
  const unsigned short* p1 = TAB + sg.t1 + (sg.kbeg + kq) * r1;
  const unsigned short* p2 = TAB + sg.t2 + (sg.kbeg + kq) * r2;
#pragma unroll 1
  for (int k0 = sg.kbeg; k0 < sg.kend; k0 += 8, p1 += 8 * r1, p2 += 8 * r2) {
    const bool active = k0 + kq < sg.kend;  // the four lanes of a quad agree
    quad_step<SHAPE, I1, I2>(n1, n2, active ? p1 : ZROW, active ? p2 : ZROW, S1a, S2a, sc, acc);
  }
}

// reduce over the eight shared-index lanes, add into slot [alpha1][alpha2][s];
// acc holds complex 4 d + s with (alpha1, alpha2) = (a, a ^ d), or
// (a ^ d, a) after a run with exchanged sides (swapped)
__device__ __forceinline__ void qseg_flush(float (&acc)[32], int lane, bool swapped, float2* slot) {
  const int a = lane & 3, kq = lane >> 2;
  quad_reduce<16>(acc, lane);  // lane keeps complex 2 kq, 2 kq + 1: d = kq >> 1, s = 2 (kq & 1) + {0, 1}
  const int b = a ^ (kq >> 1);
  float2* o = slot + (swapped ? 16 * b + 4 * a : 16 * a + 4 * b) + 2 * (kq & 1);
  o[0].x += acc[0];
  o[0].y += acc[1];
  o[1].x += acc[2];
  o[1].y += acc[3];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
}

// TMA: slabs staged by the tensor memory accelerator (one thread issues the
// boxes, an mbarrier per buffer counts the bytes); else 16-byte cp.async by all
// threads.  flags: bit 1 is set if a slab wait gave up (the CTA then returns).
template <int NW, bool TMA>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_qseg(
    const __grid_constant__ CUtensorMap fbmap, const float2* __restrict__ FB, int L, int nchunks, int qb,
    const QuadChunkHdr* __restrict__ chunks, const QuadSeg* __restrict__ segs, const int* __restrict__ group_ch,
    const unsigned short* __restrict__ tab, const float* __restrict__ codes, int max_slot, int max_tab, int max_segs,
    float2* __restrict__ Ft, int* __restrict__ flags, int skip_first) {
  constexpr int NT = NW * 32;
  constexpr int slab = 2 * 2 * QUAD_ST;  // uint4 per buffer: two sides x cells x 32 bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // slabs first, on a 128-byte boundary (TMA destinations), then the rest
  const unsigned pad = (128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u;
  uint4* SB = reinterpret_cast<uint4*>(smem_raw + pad);
  unsigned short* TAB = reinterpret_cast<unsigned short*>(SB + 2 * slab);
  unsigned short* ZROW = TAB + max_tab;  // max_tab % 8 == 0
  float2* OUT = reinterpret_cast<float2*>(ZROW + QUAD_ZROW);
  float* SC = reinterpret_cast<float*>(OUT + max_slot * 64);
  QuadSeg* SEG = reinterpret_cast<QuadSeg*>(SC + 64);
  // per chunk-local channel c: its partial-sum slots SL[CS[c] .. CS[c + 1]) in
  // warp order, and its request-order channel GC[c]
  int* CS = reinterpret_cast<int*>(SEG + max_segs);
  int* SL = CS + max_slot + 1;
  int* GC = SL + max_slot;
  unsigned long long* MB = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(GC + max_slot) + 7) & ~static_cast<uintptr_t>(7));  // one mbarrier per buffer
  const unsigned mb0 = (unsigned)__cvta_generic_to_shared(MB);
  if (threadIdx.x < 64) {
    const float m = codes[threadIdx.x >> 1];
    SC[threadIdx.x] = (threadIdx.x & 1) ? -m : m;
  }
  for (int i = threadIdx.x; i < QUAD_ZROW; i += NT) ZROW[i] = (unsigned short)(31u << 11);
  const long long V = (long long)L * L * L;
  const int ci = blockIdx.x % nchunks;
  const long long q_begin = (long long)(blockIdx.x / nchunks) * qb;
  const long long q_end = min(V, q_begin + qb);
  const QuadChunkHdr& ck = chunks[ci];
  const int base1 = ck.base1, n1c = ck.ncell1, base2 = ck.base2, n2c = ck.ncell2;
  const int seg0 = ck.seg_base[0], nseg = ck.seg_base[NW] - seg0;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int c = 0; c < ck.nch; ++c) {
      CS[c] = n;
      for (int ww = 0; ww < NW; ++ww) {
        const int r = c - ck.cfirst[ww];
        if (r >= 0 && r < ck.out_base[ww + 1] - ck.out_base[ww]) SL[n++] = ck.out_base[ww] + r;
      }
      GC[c] = group_ch[ck.ch_off + c];
    }
    CS[ck.nch] = n;
  }

  // coordinates of the next momentum to stage (slabs are issued for q_begin,
  // q_begin + 1, ... in order)
  int nqx = (int)(q_begin % L), nqy = (int)((q_begin / L) % L), nqz = (int)(q_begin / ((long long)L * L));
  auto issue_slabs = [&](long long q, uint4* S) {
    const long long qm = (nqx ? L - nqx : 0) + L * ((nqy ? L - nqy : 0) + (long long)L * (nqz ? L - nqz : 0));
    if (++nqx == L) {
      nqx = 0;
      if (++nqy == L) {
        nqy = 0;
        ++nqz;
      }
    }
    if constexpr (TMA) {
      if (threadIdx.x == 0) {
        if (skip_first && q == q_begin)  // test switch: arm the wait, issue no box (nothing in flight)
          mbar_expect_tx(mb0, 32u);
        else
          tma_issue_slabs(&fbmap, (unsigned)__cvta_generic_to_shared(S), 2 * QUAD_ST * 16, mb0 + (S == SB ? 0u : 8u),
                          base1, n1c, (int)q, base2, n2c, (int)qm);
      }
      return;
    }
    for (int i = threadIdx.x; i < 2 * n1c; i += NT)
      cp_async16q(S + i, reinterpret_cast<const char*>(FB + ((long long)(base1 + (i >> 1)) * V + q) * 4) + 16 * (i & 1));
    uint4* S2 = S + 2 * QUAD_ST;
    for (int i = threadIdx.x; i < 2 * n2c; i += NT)
      cp_async16q(S2 + i, reinterpret_cast<const char*>(FB + ((long long)(base2 + (i >> 1)) * V + qm) * 4) + 16 * (i & 1));
  };

  if constexpr (TMA) {
    // once a CTA of this launch has given up on a slab wait, the others leave at once
    if (__syncthreads_or(threadIdx.x == 0 && (*reinterpret_cast<volatile int*>(flags) & 2))) return;
    if (threadIdx.x == 0) {
      mbar_init(mb0, 1);
      mbar_init(mb0 + 8, 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
  }
  for (int i = threadIdx.x; i < ck.tab_len / 8; i += NT) cp_async16q(TAB + 8 * i, tab + ck.tab_off + 8 * i);
  for (int i = threadIdx.x; i < 2 * nseg; i += NT)
    cp_async16q(reinterpret_cast<uint4*>(SEG) + i, reinterpret_cast<const uint4*>(segs + seg0) + i);
  if (q_begin < q_end) issue_slabs(q_begin, SB);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < ck.nslot * 64; i += NT) OUT[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // a slab wait that gave up: flag it, let thread 0 wait (bounded) for
  // the boxes in flight, and leave together
  auto give_up = [&](unsigned mb, unsigned parity, bool in_flight) {
    if (threadIdx.x == 0) {
      atomicOr(flags, 2);
      // the boxes of the buffer given up on may still be in flight: wait for them (up to eight more
      // seconds of the global timer) before the block's shared memory is released
      for (int k = 0; in_flight && k < 8 && !mbar_wait_timed(mb, parity, 1000000000ull); ++k) {
      }
    }
  };
  if constexpr (TMA) {
    // the test switch's withheld copy: a wait of one second of the global timer
    const bool ok = q_begin >= q_end || (skip_first ? mbar_wait_timed(mb0, 0, 1000000000ull) : mbar_wait(mb0, 0));
    if (__syncthreads_or(!ok)) {
      give_up(mb0, 0, !skip_first);
      return;
    }
  }

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = lane & 3, kq = lane >> 2;
  const int s_begin = ck.seg_base[w] - seg0, s_end = ck.seg_base[w + 1] - seg0;
  float2* const out_w = OUT + (ck.out_base[w] - ck.cfirst[w]) * 64;
  for (long long q = q_begin; q < q_end; ++q) {
    uint4* S = SB + ((q - q_begin) & 1) * slab;
    if (q + 1 < q_end) issue_slabs(q + 1, SB + ((q + 1 - q_begin) & 1) * slab);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const float2* S1a = reinterpret_cast<const float2*>(S) + a;
    const float2* S2a = reinterpret_cast<const float2*>(S + 2 * QUAD_ST) + a;
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    int cur = -1;  // 2 * channel + sides exchanged, of the accumulated products
    for (int si = s_begin;; ++si) {
      // one flush site: on a change of channel or of side order, and after the last run
      const int key = si < s_end ? 2 * SEG[si].local + ((SEG[si].form >> 3) & 1) : -1;
      if (key != cur) {
        if (cur >= 0) qseg_flush(acc, lane, cur & 1, out_w + (cur >> 1) * 64);
        cur = key;
      }
      if (si >= s_end) break;
      const QuadSeg sg = SEG[si];
      const bool sw = sg.form & 8;
      const float2* Sa = sw ? S2a : S1a;  // the lanes' own list
      const float2* Sb = sw ? S1a : S2a;  // the exchanged list
      switch (sg.form & 7) {
        case 5: qseg_run<1, 1, 1>(sg, kq, TAB, ZROW, Sa, Sb, SC, acc); break;
        case 7: qseg_run<3, 1, 4>(sg, kq, TAB, ZROW, Sa, Sb, SC, acc); break;
        case 1: qseg_run<1, 0, 0>(sg, kq, TAB, ZROW, Sa, Sb, SC, acc); break;
        default: qseg_run<3, 0, 0>(sg, kq, TAB, ZROW, Sa, Sb, SC, acc); break;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ck.nch * 64; i += NT) {
      const int c = i >> 6, m = i & 63;
      float2 sum = make_float2(0.f, 0.f);
      for (int k = CS[c]; k < CS[c + 1]; ++k) {  // warp order: a fixed summation order
        float2& v = OUT[SL[k] * 64 + m];
        sum.x += v.x;
        sum.y += v.y;
        v = make_float2(0.f, 0.f);
      }
      const int spin = (m & ~3) + 2 * (m & 1) + ((m >> 1) & 1);
      Ft[((long long)GC[c] * 64 + spin) * V + q] = sum;
    }
    if constexpr (TMA) {
      // the next momentum's slabs: buffer (u + 1) & 1, its fill number (u + 1) >> 1
      const long long u = q + 1 - q_begin;
      const unsigned mb = mb0 + 8u * (unsigned)(u & 1), parity = (unsigned)((u >> 1) & 1);
      const bool ok = q + 1 >= q_end || mbar_wait(mb, parity);
      if (__syncthreads_or(!ok)) {
        give_up(mb, parity, true);
        return;
      }
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
    }
  }
}

}  // namespace

size_t qseg_smem_bytes(int max_slot, int max_tab, int max_segs) {
  return 128 + (size_t)2 * 2 * 2 * QUAD_ST * 16 + (size_t)(max_tab + QUAD_ZROW) * 2 +
         (size_t)max_slot * 64 * sizeof(float2) + 64 * sizeof(float) + (size_t)max_segs * sizeof(QuadSeg) +
         (size_t)(3 * max_slot + 1) * sizeof(int) + 8 + 2 * sizeof(unsigned long long);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

bool encode_fb_map(CUtensorMap* map, const float2* FB, long long V, long long ncells) {
  const EncodeTiled fn = encode_tiled();
  if (!fn || !FB || (reinterpret_cast<uintptr_t>(FB) & 15) || V <= 0 || ncells <= 0 || V > (1LL << 31)) return false;
  const cuuint64_t dim[3] = {8, (cuuint64_t)V, (cuuint64_t)ncells};
  const cuuint64_t stride[2] = {32, (cuuint64_t)V * 32};
  const cuuint32_t box[3] = {8, 1, (cuuint32_t)QUAD_BOX};
  const cuuint32_t estride[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(FB), dim, stride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_contract_qseg(const float2* FB, long long ncells, int L, int nchunks, int qb, const void* chunks,
                                 const void* segs, int max_segs, const int* group_ch, const unsigned short* tab,
                                 const float* codes, int max_cells, int max_slot, int max_tab, int max_row, float2* Ft,
                                 int* flags, int skip_first, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  if (max_row > QUAD_ZROW || max_tab % 8 || max_cells > QUAD_ST || max_cells > 1024 || max_segs < 0 || !flags)
    return cudaErrorInvalidValue;
  const size_t sm = qseg_smem_bytes(max_slot, max_tab, max_segs);
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL) return cudaErrorInvalidValue;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const bool tma = encode_fb_map(&map, FB, V, ncells);
  auto kern = tma ? k_contract_qseg<NBS_QUAD_WARPS, true> : k_contract_qseg<NBS_QUAD_WARPS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(nqb * nchunks), NBS_QUAD_WARPS * 32, sm, st>>>(map, FB, L, nchunks, qb, (const QuadChunkHdr*)chunks,
                                                                   (const QuadSeg*)segs, group_ch, tab, codes,
                                                                   max_slot, max_tab, max_segs, Ft, flags,
                                                                   tma ? skip_first : 0);
  return cudaGetLastError();
}

}  // namespace nbs
