// kernels_tcq.cu -- the effective-block product of Eq. (4.3) on the tensor
// cores (split-BF16 x 3, FP32 accumulation) with the quad-lane work split.
//
// Work split (per-warp runs), tables, slabs and zero row as in the quad-lane
// FP32 contraction (kernels_quad.cu): lane 4 kq + a gathers, for shared index k0 + kq of an
// 8-index step, the rows E1[alpha1 = a][h1] and E2[alpha2 = a][h2].  Seen
// across the warp, the complex rows of one held spin h form an 8 x 8 matrix
// M[k][2 alpha + re/im] whose row k is held by the lanes of quad k in exactly
// the register layout of an m8n8 b16 fragment once (re, im) are packed as
// bf16x2.  movmatrix.trans turns it into M^T, which is both an A-fragment
// register (rows 2 alpha + re/im, 8 shared indices) and the B fragment of
// mma.m16n8k8, so each 8-index step is one k8 product with no shared-memory
// staging.  With real rows (re, im) on both sides, P = A B holds the
// four real products; Re F = P[re,re] - P[im,im], Im F = P[re,im] + P[im,re]
// are formed when a warp flushes a channel.  Each value x is split into
// hi = rn_bf16(x), lo = rn_bf16(x - hi); the product is hi hi + hi lo + lo hi.
// Tiles per step: shapes 1, 2 (2 x 2 held spins): A = E1 (16 rows), one n8
// tile per h2; shape 3: two m16 tiles of E1, B = E2; shape 0: two m16 tiles
// of E2, B = E1 (the transposed product).  One instantiation per shape with
// run-time gather lengths keeps the loop inside the instruction cache.
#include <cuda_bf16.h>

#include <cstring>

#include "common.cuh"
#include "plan.h"
#include "tma.cuh"

namespace nbs {

namespace {

constexpr int TCQ_ZROW = 128;  // zero-coefficient entries (>= max over terms of n * held spins)
constexpr int TCQ_ST = 944;    // cells per slab side (>= the cells of any stored type)

__device__ __forceinline__ void cp_async16t(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <int NH>
__device__ __forceinline__ void tcq_entries(const unsigned short* p, unsigned (&e)[2 * NH]) {
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

// rows of NH held spins of one side: v[h] = sum_i coef * slab[cell][a]
template <int NH, int I>
__device__ __forceinline__ void tcq_gather(int n, const unsigned short* p, const float2* Sa, const float* sc,
                                           float2 (&v)[NH]) {
#pragma unroll
  for (int h = 0; h < NH; ++h) v[h] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int i = 0; i < (I ? 2 * I : n); i += 2, p += 2 * NH) {
    unsigned e[2 * NH];
    tcq_entries<NH>(p, e);
#pragma unroll
    for (int j = 0; j < 2 * NH; ++j) {
      const float c = sc[e[j] >> 10];
      const float2 x = Sa[4 * (e[j] & 1023u)];
      v[j % NH].x = fmaf(c, x.x, v[j % NH].x);
      v[j % NH].y = fmaf(c, x.y, v[j % NH].y);
    }
  }
}

__device__ __forceinline__ unsigned mov_trans(unsigned x) {
  unsigned y;
  asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(y) : "r"(x));
  return y;
}

__device__ __forceinline__ unsigned bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<unsigned*>(&v); }

// (re, im) -> transposed hi and lo fragments
__device__ __forceinline__ void split_frag(float2 v, unsigned& hi, unsigned& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
  hi = mov_trans(bf2_bits(h));
  lo = mov_trans(bf2_bits(l));
}

__device__ __forceinline__ void mma1688(float (&d)[4], unsigned a0, unsigned a1, unsigned b0) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

// two independent tiles (rows: the held-spin pairs (x0, x1) and (y0, y1); columns
// b0, b1), each hi hi + hi lo + lo hi, issued interleaved so the chains overlap
__device__ __forceinline__ void mma2_bf16x3(float (&d0)[4], float (&d1)[4], unsigned ah00, unsigned ah01,
                                            unsigned al00, unsigned al01, unsigned ah10, unsigned ah11,
                                            unsigned al10, unsigned al11, unsigned bh0, unsigned bl0, unsigned bh1,
                                            unsigned bl1) {
  mma1688(d0, ah00, ah01, bh0);
  mma1688(d1, ah10, ah11, bh1);
  mma1688(d0, ah00, ah01, bl0);
  mma1688(d1, ah10, ah11, bl1);
  mma1688(d0, al00, al01, bh0);
  mma1688(d1, al10, al11, bh1);
}

// one 8-index step: gather this lane's rows, split, transpose, and multiply on
// the tensor cores (mma.m16n8k8: the step's 8 shared indices are the k dimension)
template <int SHAPE>
__device__ __forceinline__ void tcq_step(int n1, int n2, const unsigned short* p1, const unsigned short* p2,
                                         const float2* S1a, const float2* S2a, const float* sc, float (&D)[2][4]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  unsigned f1h[NH1], f1l[NH1], f2h[NH2], f2l[NH2];
  {
    float2 v1[NH1], v2[NH2];
    tcq_gather<NH1, 0>(n1, p1, S1a, sc, v1);
    tcq_gather<NH2, 0>(n2, p2, S2a, sc, v2);
#pragma unroll
    for (int h = 0; h < NH1; ++h) split_frag(v1[h], f1h[h], f1l[h]);
#pragma unroll
    for (int h = 0; h < NH2; ++h) split_frag(v2[h], f2h[h], f2l[h]);
  }
  if constexpr (SHAPE == 1 || SHAPE == 2) {  // A = E1 (rows h1 = 0, 1), one B tile per h2
    mma2_bf16x3(D[0], D[1], f1h[0], f1h[1], f1l[0], f1l[1], f1h[0], f1h[1], f1l[0], f1l[1], f2h[0], f2l[0], f2h[1],
                f2l[1]);
  } else if constexpr (SHAPE == 3) {  // A tiles of E1 (h1 = 0, 1 and 2, 3), B = E2
    mma2_bf16x3(D[0], D[1], f1h[0], f1h[1], f1l[0], f1l[1], f1h[2], f1h[3], f1l[2], f1l[3], f2h[0], f2l[0], f2h[0],
                f2l[0]);
  } else {  // A tiles of E2 (h2 = 0, 1 and 2, 3), B = E1
    mma2_bf16x3(D[0], D[1], f2h[0], f2h[1], f2l[0], f2l[1], f2h[2], f2h[3], f2l[2], f2l[3], f1h[0], f1l[0], f1h[0],
                f1l[0]);
  }
}

// P fragments of one shape -> complex F added to the channel slot [alpha1][alpha2][s]
template <int SHAPE>
__device__ __forceinline__ void tcq_flush(float (&D)[2][4], int lane, float2* slot) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int tile = 0; tile < 2; ++tile)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const float x = D[tile][2 * half], y = D[tile][2 * half + 1];  // P[row][2t], P[row][2t + 1]
      const float px = __shfl_xor_sync(0xffffffffu, x, 4);           // same columns, imaginary row
      const float py = __shfl_xor_sync(0xffffffffu, y, 4);
      D[tile][2 * half] = D[tile][2 * half + 1] = 0.f;
      if (g & 1) continue;  // rows 2 alpha + 1 carry the imaginary parts
      const float re = x - py, im = y + px;
      const int ar = g >> 1, ac = t;  // spin of the row side, of the column side
      int a1, a2, s;
      if (SHAPE == 1 || SHAPE == 2) {  // tile = h2, half = h1
        a1 = ar; a2 = ac;
        s = SHAPE == 1 ? half + 2 * tile : tile + 2 * half;
      } else if (SHAPE == 3) {         // rows: h1 = 2 tile + half
        a1 = ar; a2 = ac;
        s = 2 * tile + half;
      } else {                         // rows: E2, h2 = 2 tile + half; columns: E1
        a1 = ac; a2 = ar;
        s = 2 * tile + half;
      }
      float2& o = slot[(a1 * 4 + a2) * 4 + s];
      o.x += re;
      o.y += im;
    }
}

__device__ __forceinline__ void tcq_flush_all(float (&D)[4][2][4], unsigned used, int lane, float2* slot) {
  if (used & 1) tcq_flush<0>(D[0], lane, slot);
  if (used & 2) tcq_flush<1>(D[1], lane, slot);
  if (used & 4) tcq_flush<2>(D[2], lane, slot);
  if (used & 8) tcq_flush<3>(D[3], lane, slot);
}

// TMA: slabs staged by the tensor memory accelerator (tma.cuh); else 16-byte
// cp.async by all threads.  flags: bit 1 is set if a slab wait gave up.
template <int NW, bool TMA>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_tcq(
    const __grid_constant__ CUtensorMap fbmap, const float2* __restrict__ FB, int L, int nchunks, int qb,
    const QuadChunkHdr* __restrict__ chunks, const QuadSeg* __restrict__ segs, const int* __restrict__ group_ch,
    const unsigned short* __restrict__ tab, const float* __restrict__ codes, int max_slot, int max_tab, int max_segs,
    float2* __restrict__ Ft, int* __restrict__ flags) {
  constexpr int NT = NW * 32;
  constexpr int slab = 2 * 2 * TCQ_ST;  // uint4 per buffer: two sides x cells x 32 bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // slabs first, on a 128-byte boundary (TMA destinations), then the rest
  const unsigned pad = (128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u;
  uint4* SB = reinterpret_cast<uint4*>(smem_raw + pad);
  unsigned short* TAB = reinterpret_cast<unsigned short*>(SB + 2 * slab);
  unsigned short* ZROW = TAB + max_tab;  // max_tab % 8 == 0
  float2* OUT = reinterpret_cast<float2*>(ZROW + TCQ_ZROW);
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
  for (int i = threadIdx.x; i < TCQ_ZROW; i += NT) ZROW[i] = (unsigned short)(31u << 11);
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

  // slab: side 1 cells then side 2 cells, 32 bytes (four spins) per cell
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
      if (threadIdx.x == 0)
        tma_issue_slabs(&fbmap, (unsigned)__cvta_generic_to_shared(S), 2 * TCQ_ST * 16, mb0 + (S == SB ? 0u : 8u),
                        base1, n1c, (int)q, base2, n2c, (int)qm);
      return;
    }
    for (int i = threadIdx.x; i < 2 * n1c; i += NT)
      cp_async16t(S + i, reinterpret_cast<const char*>(FB + ((long long)(base1 + (i >> 1)) * V + q) * 4) + 16 * (i & 1));
    uint4* S2 = S + 2 * TCQ_ST;
    for (int i = threadIdx.x; i < 2 * n2c; i += NT)
      cp_async16t(S2 + i, reinterpret_cast<const char*>(FB + ((long long)(base2 + (i >> 1)) * V + qm) * 4) + 16 * (i & 1));
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
  for (int i = threadIdx.x; i < ck.tab_len / 8; i += NT) cp_async16t(TAB + 8 * i, tab + ck.tab_off + 8 * i);
  for (int i = threadIdx.x; i < 2 * nseg; i += NT)
    cp_async16t(reinterpret_cast<uint4*>(SEG) + i, reinterpret_cast<const uint4*>(segs + seg0) + i);
  if (q_begin < q_end) issue_slabs(q_begin, SB);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < ck.nslot * 64; i += NT) OUT[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // a slab wait that gave up: flag it, let thread 0 wait (bounded) for
  // the boxes in flight, and leave together
  auto give_up = [&](unsigned mb, unsigned parity) {
    if (threadIdx.x == 0) {
      atomicOr(flags, 2);
      // the boxes of the buffer given up on may still be in flight: wait for them (up to eight more
      // seconds of the global timer) before the block's shared memory is released
      for (int k = 0; k < 8 && !mbar_wait_timed(mb, parity, 1000000000ull); ++k) {
      }
    }
  };
  if constexpr (TMA) {
    const bool ok = q_begin >= q_end || mbar_wait(mb0, 0);
    if (__syncthreads_or(!ok)) {
      give_up(mb0, 0);
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
    const float2* S2a = reinterpret_cast<const float2*>(S + 2 * TCQ_ST) + a;
    float D[4][2][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y)
#pragma unroll
        for (int z = 0; z < 4; ++z) D[x][y][z] = 0.f;
    unsigned used = 0;  // shapes accumulated since the last flush (warp-uniform)
    int cur = -1;
    for (int si = s_begin;; ++si) {
      // one flush site: on a channel change and after the last run
      const int local = si < s_end ? SEG[si].local : -1;
      if (local != cur) {
        if (cur >= 0) tcq_flush_all(D, used, lane, out_w + cur * 64);
        used = 0;
        cur = local;
      }
      if (si >= s_end) break;
      const QuadSeg sg = SEG[si];
      // a run with exchanged sides (bit 3) is taken back to its own shape and side order
      const bool sw = sg.form & 8;
      const int shape = sw ? (sg.form & 3) ^ 3 : sg.form & 3;
      const int n1 = sw ? sg.n2 : sg.n1, n2 = sw ? sg.n1 : sg.n2;
      used |= 1u << shape;
      const int nh1 = 1 << ((shape & 1) + ((shape >> 1) & 1));
      const int r1 = nh1 * n1, r2 = (4 / nh1) * n2;  // entries per shared index
      const unsigned short* p1 = TAB + (sw ? sg.t2 : sg.t1) + (sg.kbeg + kq) * r1;
      const unsigned short* p2 = TAB + (sw ? sg.t1 : sg.t2) + (sg.kbeg + kq) * r2;
      for (int k0 = sg.kbeg; k0 < sg.kend; k0 += 8, p1 += 8 * r1, p2 += 8 * r2) {
        const bool active = k0 + kq < sg.kend;  // the four lanes of a quad agree
        const unsigned short* q1 = active ? p1 : ZROW;
        const unsigned short* q2 = active ? p2 : ZROW;
        switch (shape) {
          case 0: tcq_step<0>(n1, n2, q1, q2, S1a, S2a, SC, D[0]); break;
          case 1: tcq_step<1>(n1, n2, q1, q2, S1a, S2a, SC, D[1]); break;
          case 2: tcq_step<2>(n1, n2, q1, q2, S1a, S2a, SC, D[2]); break;
          default: tcq_step<3>(n1, n2, q1, q2, S1a, S2a, SC, D[3]); break;
        }
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
        give_up(mb, parity);
        return;
      }
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
    }
  }
}

}  // namespace

size_t tcq_smem_bytes(int max_slot, int max_tab, int max_segs) {
  return 128 + (size_t)2 * 2 * 2 * TCQ_ST * 16 + (size_t)(max_tab + TCQ_ZROW) * 2 +
         (size_t)max_slot * 64 * sizeof(float2) + 64 * sizeof(float) + (size_t)max_segs * sizeof(QuadSeg) +
         (size_t)(3 * max_slot + 1) * sizeof(int) + 8 + 2 * sizeof(unsigned long long);
}

cudaError_t launch_contract_tcq(const float2* FB, long long ncells, int L, int nchunks, int qb, const void* chunks,
                                const void* segs, int max_segs, const int* group_ch, const unsigned short* tab,
                                const float* codes, int max_cells, int max_slot, int max_tab, int max_row, float2* Ft,
                                int* flags, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  if (max_row > TCQ_ZROW || max_tab % 8 || max_cells > TCQ_ST || max_cells > 1024 || max_segs < 0 || !flags)
    return cudaErrorInvalidValue;
  const size_t sm = tcq_smem_bytes(max_slot, max_tab, max_segs);
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL) return cudaErrorInvalidValue;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const bool tma = encode_fb_map(&map, FB, V, ncells);
  auto kern = tma ? k_contract_tcq<NBS_QUAD_WARPS, true> : k_contract_tcq<NBS_QUAD_WARPS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(nqb * nchunks), NBS_QUAD_WARPS * 32, sm, st>>>(map, FB, L, nchunks, qb, (const QuadChunkHdr*)chunks,
                                                                  (const QuadSeg*)segs, group_ch, tab, codes, max_slot,
                                                                  max_tab, max_segs, Ft, flags);
  return cudaGetLastError();
}

}  // namespace nbs
