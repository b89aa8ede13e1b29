// kernels_tc.cu -- the effective-block product of Eq. (4.3) on the tensor cores,
// split-BF16 x 3 with FP32 accumulation (precision mode NBS_BF16X3).
//
// Same work split as the chunk contraction (kernels_contract.cu): a block
// keeps one chunk of channels' compressed gather tables in shared memory and
// sweeps a block of momenta, loading the two momentum slabs of each q with
// cp.async.  For a work item (term, 32 shared indices xi~) lane j builds, in
// FP32, both effective blocks of shared index k0 + j: E1[alpha1, h1] at q and
// E2[alpha2, h2] at -q.  The product sum_k E1[r, k] E2[c, k] is a tiny
// complex GEMM per term: written as real matrices with the real parts in the
// first and the imaginary parts in the second half of the rows (columns),
//   A (rows: E1 re | E1 im) x B (cols: E2 re | E2 im) = P,
//   Re F = P[re, re] - P[im, im],  Im F = P[re, im] + P[im, re].
// Each FP32 value x is split into bf16 hi = rn(x), lo = rn(x - hi); the
// product is hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-16 relative, is
// dropped).  Lanes store their hi/lo rows into a per-warp tile [k][row]
// (k-major), ldmatrix.trans gathers the mma.m16n8k16 fragments, FP32
// accumulators stay in registers for all items of a channel.  The side with
// 16 complex rows (shape 0: E2, shape 3: E1) is the A operand (two m16
// tiles, one n8 tile); shapes 1 and 2 (8 x 8 complex) use one m16 and two n8
// tiles.
#include <cuda_bf16.h>

#include "common.cuh"
#include "plan.h"

namespace nbs {

namespace {

constexpr int TC_WARPS = 8;
// bf16 per tile row (k-major tiles of 32 shared indices): A has up to 32 real rows,
// B up to 16; 8 bf16 of padding make the ldmatrix row addresses conflict-free
constexpr int LD_A = 40, LD_B = 24;
// per-warp staging: hi and lo tiles of A^T and B^T; reused for P (at most 256 floats)
constexpr int STAGE_BYTES = 2 * 32 * LD_A * 2 + 2 * 32 * LD_B * 2;  // 8192

__device__ __forceinline__ void cp_async16c(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x2_trans(unsigned (&r)[2], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// x -> (hi, lo) packed as bf16x2 pairs for two consecutive values
__device__ __forceinline__ void split2(float x0, float x1, __nv_bfloat162& hi, __nv_bfloat162& lo) {
  hi = __floats2bfloat162_rn(x0, x1);
  const float2 h = __bfloat1622float2(hi);
  lo = __floats2bfloat162_rn(x0 - h.x, x1 - h.y);
}

// Build E1 (NH1 x 4 spins) and E2 (NH2 x 4 spins) of shared index k for one term.
template <int SHAPE>
__device__ __forceinline__ void build_blocks(const DevTerm& h, int k, const unsigned short* T1,
                                             const unsigned short* T2, const uint4* S1, int st1, const uint4* S2,
                                             int st2, const float* codes, float2 (&v1)[4][4], float2 (&v2)[4][4]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  // entries of shared index k are ordered [i][h]: the inner loop over h is unrolled
  const unsigned short* p1 = T1 + k * NH1 * h.n1;
  for (int i = 0; i < h.n1; ++i, p1 += NH1) {
#pragma unroll
    for (int hh = 0; hh < NH1; ++hh) {
      const unsigned e = p1[hh];
      const float a = codes[e >> 11];
      const float c = (e & 1024u) ? -a : a;
      const unsigned cell = e & 1023u;
      const float4 x = *reinterpret_cast<const float4*>(S1 + cell);
      const float4 y = *reinterpret_cast<const float4*>(S1 + st1 + cell);
      crfma<float>(v1[hh][0], c, make_float2(x.x, x.y));
      crfma<float>(v1[hh][1], c, make_float2(x.z, x.w));
      crfma<float>(v1[hh][2], c, make_float2(y.x, y.y));
      crfma<float>(v1[hh][3], c, make_float2(y.z, y.w));
    }
  }
  const unsigned short* p2 = T2 + k * NH2 * h.n2;
  for (int i = 0; i < h.n2; ++i, p2 += NH2) {
#pragma unroll
    for (int hh = 0; hh < NH2; ++hh) {
      const unsigned e = p2[hh];
      const float a = codes[e >> 11];
      const float c = (e & 1024u) ? -a : a;
      const unsigned cell = e & 1023u;
      const float4 x = *reinterpret_cast<const float4*>(S2 + cell);
      const float4 y = *reinterpret_cast<const float4*>(S2 + st2 + cell);
      crfma<float>(v2[hh][0], c, make_float2(x.x, x.y));
      crfma<float>(v2[hh][1], c, make_float2(x.z, x.w));
      crfma<float>(v2[hh][2], c, make_float2(y.x, y.y));
      crfma<float>(v2[hh][3], c, make_float2(y.z, y.w));
    }
  }
}

// Store n complex values (index r = alpha * NH + h) of this lane's row k into
// the hi / lo tiles: real part at column r, imaginary part at column n + r.
template <int NH, int LD>
__device__ __forceinline__ void store_row(__nv_bfloat16* hi, __nv_bfloat16* lo, int k, const float2 (&v)[4][4]) {
  constexpr int n = 4 * NH;
  __nv_bfloat162* H = reinterpret_cast<__nv_bfloat162*>(hi + k * LD);
  __nv_bfloat162* Lo = reinterpret_cast<__nv_bfloat162*>(lo + k * LD);
#pragma unroll
  for (int r = 0; r < n; r += 2) {
    const float2 z0 = v[(r) % NH][(r) / NH], z1 = v[(r + 1) % NH][(r + 1) / NH];
    __nv_bfloat162 h, l;
    split2(z0.x, z1.x, h, l);  // real parts of rows r, r + 1
    H[r / 2] = h;
    Lo[r / 2] = l;
    split2(z0.y, z1.y, h, l);  // imaginary parts
    H[(n + r) / 2] = h;
    Lo[(n + r) / 2] = l;
  }
}

template <int SHAPE>
__device__ __forceinline__ void tc_item(const DevTerm& h, int k0, int lane, const unsigned short* T1,
                                        const unsigned short* T2, const uint4* S1, int st1, const uint4* S2, int st2,
                                        const float* codes, unsigned char* stage, float (&acc)[2][4]) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  // A operand: the side with more rows; for shapes 1, 2 (8 x 8 complex) E1
  constexpr bool A_IS_E1 = SHAPE != 0;
  constexpr int RA = A_IS_E1 ? 8 * NH1 : 8 * NH2;  // real rows of A (16 or 32)
  constexpr int MT = RA / 16;                      // m16 tiles (1 or 2); n8 tiles = 2 / MT
  __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(stage);
  __nv_bfloat16* Alo = Ahi + 32 * LD_A;
  __nv_bfloat16* Bhi = Alo + 32 * LD_A;
  __nv_bfloat16* Blo = Bhi + 32 * LD_B;
  float2 v1[4][4], v2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) v1[a][b] = v2[a][b] = make_float2(0.f, 0.f);
  const int k = k0 + lane;
  if (k < h.K) build_blocks<SHAPE>(h, k, T1, T2, S1, st1, S2, st2, codes, v1, v2);
  if (A_IS_E1) {
    store_row<NH1, LD_A>(Ahi, Alo, lane, v1);
    store_row<NH2, LD_B>(Bhi, Blo, lane, v2);
  } else {
    store_row<NH2, LD_A>(Ahi, Alo, lane, v2);
    store_row<NH1, LD_B>(Bhi, Blo, lane, v1);
  }
  __syncwarp();
  const int mat = lane >> 3, rr = lane & 7;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {  // two k16 steps of the 32 shared indices
    const int kb = 16 * ks;
#pragma unroll
    for (int t = 0; t < 2; ++t) {  // the two output tiles
      const int m0 = MT == 2 ? 16 * t : 0;
      const int n0 = MT == 2 ? 0 : 8 * t;
      unsigned ahi[4], alo[4], bhi[2], blo[2];
      // A tile (m0..m0+15, kb..kb+15) from A^T[k][m]: matrices (m lo|hi) x (k lo|hi)
      const int ka = kb + ((mat >> 1) << 3) + rr, ma = m0 + ((mat & 1) << 3);
      ldsm_x4_trans(ahi, Ahi + ka * LD_A + ma);
      ldsm_x4_trans(alo, Alo + ka * LD_A + ma);
      // B tile (kb..kb+15, n0..n0+7) from B^T[k][n]: lanes 0-15 address k rows
      const int kbb = kb + (lane & 15);
      ldsm_x2_trans(bhi, Bhi + kbb * LD_B + n0);
      ldsm_x2_trans(blo, Blo + kbb * LD_B + n0);
      mma_bf16(acc[t], ahi, bhi);
      mma_bf16(acc[t], ahi, blo);
      mma_bf16(acc[t], alo, bhi);
    }
  }
  __syncwarp();
}

// P fragments -> 64 complex products, added to this warp's output slot
template <int SHAPE>
__device__ __forceinline__ void tc_flush(float (&acc)[2][4], int lane, float* P, float2* slot) {
  constexpr int NH1 = 1 << ((SHAPE & 1) + ((SHAPE >> 1) & 1));
  constexpr int NH2 = 4 / NH1;
  constexpr bool A_IS_E1 = SHAPE != 0;
  constexpr int RA = A_IS_E1 ? 8 * NH1 : 8 * NH2;
  constexpr int RB = 256 / RA;  // real columns of B: 16 or 8
  constexpr int MT = RA / 16;
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int m0 = MT == 2 ? 16 * t : 0;
    const int n0 = MT == 2 ? 0 : 8 * t;
    P[(m0 + g) * RB + n0 + 2 * tq] = acc[t][0];
    P[(m0 + g) * RB + n0 + 2 * tq + 1] = acc[t][1];
    P[(m0 + g + 8) * RB + n0 + 2 * tq] = acc[t][2];
    P[(m0 + g + 8) * RB + n0 + 2 * tq + 1] = acc[t][3];
    acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
  }
  __syncwarp();
  constexpr int M1 = 4 * NH1, N2 = 4 * NH2;  // complex rows of E1, E2
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int m = 2 * lane + j;  // (alpha1 * 4 + alpha2) * 4 + s, s = alpha3 + 2 alpha4
    const int a1 = m >> 4, a2 = (m >> 2) & 3, s = m & 3;
    int h1, h2;
    if (SHAPE == 0) { h1 = 0; h2 = s; }
    else if (SHAPE == 3) { h1 = s; h2 = 0; }
    else if (SHAPE == 1) { h1 = s & 1; h2 = s >> 1; }
    else { h1 = s >> 1; h2 = s & 1; }
    const int r1 = a1 * NH1 + h1, c2 = a2 * NH2 + h2;
    float re, im;
    if (A_IS_E1) {
      re = P[r1 * RB + c2] - P[(M1 + r1) * RB + N2 + c2];
      im = P[r1 * RB + N2 + c2] + P[(M1 + r1) * RB + c2];
    } else {
      re = P[c2 * RB + r1] - P[(N2 + c2) * RB + M1 + r1];
      im = P[(N2 + c2) * RB + r1] + P[c2 * RB + M1 + r1];
    }
    slot[m].x += re;
    slot[m].y += im;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(TC_WARPS * 32, 1) k_contract_tc(
    const float2* __restrict__ FB, int L, int nchunks, int qb, const ChunkHdr* __restrict__ chunks,
    const int* __restrict__ group_ch, const int* __restrict__ items, const DevTerm* __restrict__ terms,
    const int* __restrict__ tab_off, const unsigned short* __restrict__ tab, const float* __restrict__ codes,
    int st1, int st2, int max_slot, int max_tab, float2* __restrict__ Ft) {
  constexpr int NT = TC_WARPS * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned short* TAB = reinterpret_cast<unsigned short*>(smem_raw);
  uint4* SB = reinterpret_cast<uint4*>(smem_raw + (size_t)max_tab * 2);
  const int slab = 2 * st1 + 2 * st2;
  unsigned char* STAGE = reinterpret_cast<unsigned char*>(SB + slab);
  float2* OUT = reinterpret_cast<float2*>(STAGE + TC_WARPS * STAGE_BYTES);
  float* CODES = reinterpret_cast<float*>(OUT + max_slot * 64);
  if (threadIdx.x < 32) CODES[threadIdx.x] = codes[threadIdx.x];
  const long long V = (long long)L * L * L;
  const int ci = blockIdx.x % nchunks;
  const long long q_begin = (long long)(blockIdx.x / nchunks) * qb;
  const long long q_end = min(V, q_begin + qb);
  const ChunkHdr& ck = chunks[ci];
  const int base1 = ck.base1, n1 = ck.ncell1, base2 = ck.base2, n2 = ck.ncell2;
  for (int i = threadIdx.x; i < ck.tab_len / 8; i += NT) cp_async16c(TAB + 8 * i, tab + ck.tab_off + 8 * i);
  for (int i = threadIdx.x; i < ck.nslot * 64; i += NT) OUT[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.commit_group;\n" ::: "memory");

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* stage = STAGE + w * STAGE_BYTES;
  const int it0 = ck.item_off + ck.warp_off[w], it1 = ck.item_off + ck.warp_off[w + 1];
  const uint4* S1 = SB;
  const uint4* S2 = SB + 2 * st1;
  for (long long q = q_begin; q < q_end; ++q) {
    // slabs of q (single buffer: every warp finished the previous q at the last barrier)
    const int qx = (int)(q % L), qy = (int)((q / L) % L), qz = (int)(q / ((long long)L * L));
    const long long qm = (L - qx) % L + L * ((L - qy) % L + (long long)L * ((L - qz) % L));
    for (int i = threadIdx.x; i < 2 * n1; i += NT) {
      const int c = i >> 1, p = i & 1;
      cp_async16c(SB + p * st1 + c, reinterpret_cast<const char*>(FB + ((long long)(base1 + c) * V + q) * 4) + 16 * p);
    }
    for (int i = threadIdx.x; i < 2 * n2; i += NT) {
      const int c = i >> 1, p = i & 1;
      cp_async16c(SB + 2 * st1 + p * st2 + c,
                  reinterpret_cast<const char*>(FB + ((long long)(base2 + c) * V + qm) * 4) + 16 * p);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    int cur = -1, cur_shape = 0;
    for (int it = it0; it < it1; ++it) {
      const int term = items[2 * it], k0 = items[2 * it + 1];
      const DevTerm h = terms[term];
      const int local = h.pad - ck.ch_local0;
      if (local != cur || h.shape != cur_shape) {
        if (cur >= 0) {
          float2* slot = OUT + (ck.out_base[w] + cur - ck.cfirst[w]) * 64;
          float* P = reinterpret_cast<float*>(stage);
          switch (cur_shape) {
            case 0: tc_flush<0>(acc, lane, P, slot); break;
            case 1: tc_flush<1>(acc, lane, P, slot); break;
            case 2: tc_flush<2>(acc, lane, P, slot); break;
            default: tc_flush<3>(acc, lane, P, slot); break;
          }
        }
        cur = local;
        cur_shape = h.shape;
      }
      const unsigned short* T1 = TAB + tab_off[2 * term];
      const unsigned short* T2 = TAB + tab_off[2 * term + 1];
      switch (h.shape) {
        case 0: tc_item<0>(h, k0, lane, T1, T2, S1, st1, S2, st2, CODES, stage, acc); break;
        case 1: tc_item<1>(h, k0, lane, T1, T2, S1, st1, S2, st2, CODES, stage, acc); break;
        case 2: tc_item<2>(h, k0, lane, T1, T2, S1, st1, S2, st2, CODES, stage, acc); break;
        default: tc_item<3>(h, k0, lane, T1, T2, S1, st1, S2, st2, CODES, stage, acc); break;
      }
    }
    if (cur >= 0) {
      float2* slot = OUT + (ck.out_base[w] + cur - ck.cfirst[w]) * 64;
      float* P = reinterpret_cast<float*>(stage);
      switch (cur_shape) {
        case 0: tc_flush<0>(acc, lane, P, slot); break;
        case 1: tc_flush<1>(acc, lane, P, slot); break;
        case 2: tc_flush<2>(acc, lane, P, slot); break;
        default: tc_flush<3>(acc, lane, P, slot); break;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ck.nch * 64; i += NT) {
      const int c = i / 64, m = i % 64;
      float2 sum = make_float2(0.f, 0.f);
#pragma unroll
      for (int ww = 0; ww < TC_WARPS; ++ww) {  // fixed order
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
    __syncthreads();
  }
}

}  // namespace

size_t tc_smem_bytes(int st1, int st2, int max_slot, int max_tab) {
  return (size_t)max_tab * 2 + (size_t)(2 * st1 + 2 * st2) * 16 + (size_t)TC_WARPS * STAGE_BYTES +
         (size_t)max_slot * 64 * sizeof(float2) + 128;
}

cudaError_t launch_contract_tc(const float2* FB, int L, int nchunks, int qb, const void* chunks, const int* group_ch,
                               const int* items, const DevTerm* terms, const int* tab_off, const unsigned short* tab,
                               const float* codes, int st1, int st2, int max_slot, int max_tab, float2* Ft,
                               cudaStream_t st) {
  const long long V = (long long)L * L * L;
  const size_t sm = tc_smem_bytes(st1, st2, max_slot, max_tab);
  cudaError_t e = cudaFuncSetAttribute(k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL || max_tab % 8) return cudaErrorInvalidValue;
  k_contract_tc<<<(unsigned)(nqb * nchunks), TC_WARPS * 32, sm, st>>>(FB, L, nchunks, qb, (const ChunkHdr*)chunks,
                                                                     group_ch, items, terms, tab_off, tab, codes, st1,
                                                                     st2, max_slot, max_tab, Ft);
  return cudaGetLastError();
}

}  // namespace nbs
