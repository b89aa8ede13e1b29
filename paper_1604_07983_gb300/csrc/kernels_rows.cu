// kernels_rows.cu -- the effective blocks (Eq. (4.2)) and their product
// (Eq. (4.3)) in two phases per momentum, FP32.
//
// A CTA of 16 warps keeps one chunk's tables in shared memory (plan_rows.cpp)
// and sweeps a block of momenta.  Per momentum q:
//   * the two slabs (B1's stored type at q, B2's at -q; 32 bytes per cell:
//     four sink spins, complex) arrive by TMA into one buffer;
//   * phase A: each thread builds whole effective-block rows, sum of
//     +-1 / +-2 times slab cells, for all four spins at once (one decode per
//     entry, two 16-byte loads, eight FMAs), into the row array;
//   * the slab buffer is free again: one thread issues the next momentum's
//     boxes, which land while phase B runs;
//   * phase B: lane 4 kq + s of a warp takes record (8 step + kq, s): the B1
//     row and B2 row of shared index xi~ for output source-spin pair s and the
//     scale; it forms the 4 x 4 outer product over the sink spins alpha1,
//     alpha2 and accumulates 16 complex values.  At the end of each channel
//     segment a warp sums over its eight kq lanes and adds into its slot;
//   * the slots of each channel are summed in warp order (deterministic) and
//     written to F~[channel][spin][q].
// Waits on the slab mbarrier are bounded (a second of the global timer); a
// wait that gives up sets bit 1 of flags, the CTA leaves once nothing is in
// flight, and every later CTA of the launch leaves at its start.
#include <cstring>

#include "common.cuh"
#include "plan.h"
#include "tma.cuh"

namespace nbs {

namespace {

constexpr unsigned RSLAB_BYTES = 2u * NBS_ROW_SLAB * 32u;
constexpr unsigned long long RWAIT_NS = 1000000000ull;  // slab wait limit (global timer)

struct RowLayout {
  unsigned e, rec, aent, adesc, out, seg, sc, cs, mb, total;
};

// shared-memory layout of one chunk (offsets from a 128-byte aligned base)
__host__ __device__ inline RowLayout row_layout(int nrow, int naent, int nstep, int nslot, int nseg, int nch) {
  RowLayout L;
  unsigned o = RSLAB_BYTES;
  L.e = o;
  o += (unsigned)nrow * 32u;
  L.rec = o;
  o += (unsigned)nstep * 128u;
  L.aent = o;
  o += (unsigned)((naent + 7) / 8) * 16u;
  L.adesc = o;
  o += (unsigned)((nrow + 3) / 4) * 16u;
  L.out = o;
  o += (unsigned)nslot * 512u;
  L.seg = o;
  o += (unsigned)nseg * 16u;
  L.sc = o;
  o += 128u;
  L.cs = o;
  o += (unsigned)((2 * nch + nslot + 1 + 3) / 4) * 16u;
  L.mb = o;
  o += 16u;
  L.total = o;
  return L;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// the site index of -q (componentwise (L - n) mod L)
__device__ __forceinline__ long long minus_q(long long q, int L) {
  const int x = (int)(q % L), y = (int)((q / L) % L), z = (int)(q / ((long long)L * L));
  return (long long)((L - x) % L) + L * ((long long)((L - y) % L) + (long long)L * ((L - z) % L));
}

// sum a lane's 32 floats over the eight lanes of equal s (xor 16, 8, 4),
// halving the kept length at each stage: lane 4 kq + s ends with the floats
// 4 kq .. 4 kq + 3 of its original 32, summed over kq
template <int M>
__device__ __forceinline__ void kq_reduce(float (&acc)[32], int lane) {
  if constexpr (M >= 4) {
    const bool up = lane & M;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float keep = up ? acc[M + j] : acc[j];
      const float give = up ? acc[j] : acc[M + j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, give, M);
    }
    kq_reduce<M / 2>(acc, lane);
  }
}

// acc holds complex 4 alpha1 + alpha2 (floats 2 c, 2 c + 1) for output pair s;
// add the channel's sum into slot[16 alpha1 + 4 alpha2 + s] and clear acc
__device__ __forceinline__ void rows_flush(float (&acc)[32], int lane, float2* slot) {
  kq_reduce<16>(acc, lane);
  const int kq = lane >> 2, s = lane & 3;
  float2* o = slot + 8 * kq + s;  // complex 2 kq: alpha1 = kq >> 1, alpha2 = 2 (kq & 1)
  o[0].x += acc[0];
  o[0].y += acc[1];
  o[4].x += acc[2];
  o[4].y += acc[3];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
}

template <int NW, bool TMA>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_rows(
    const __grid_constant__ CUtensorMap fbmap, const float2* __restrict__ FB, int L, int nchunks, int qb,
    const RowChunkHdr* __restrict__ chunks, const unsigned short* __restrict__ aent,
    const unsigned* __restrict__ adesc, const unsigned* __restrict__ rec, const RowSeg* __restrict__ segs,
    const int* __restrict__ row_ch, const float* __restrict__ scales, float2* __restrict__ Ft,
    int* __restrict__ flags, int skip_first) {
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;
  unsigned char* const sb = smem_raw + pad;
  const RowChunkHdr& ck = chunks[blockIdx.x % nchunks];
  const int nrow1 = ck.nrow1, nrow = ck.nrow1 + ck.nrow2, nstep = ck.nstep, nslot = ck.nslot, nch = ck.nch;
  const int nseg = ck.seg_base[NW];
  const RowLayout lay = row_layout(nrow, ck.naent, nstep, nslot, nseg, nch);
  float4* const SL = reinterpret_cast<float4*>(sb);  // slab: [2][NBS_ROW_SLAB] cells of two float4
  float4* const E = reinterpret_cast<float4*>(sb + lay.e);
  const unsigned* const REC = reinterpret_cast<const unsigned*>(sb + lay.rec);
  const unsigned short* const AE = reinterpret_cast<const unsigned short*>(sb + lay.aent);
  const unsigned* const AD = reinterpret_cast<const unsigned*>(sb + lay.adesc);
  float2* const OUT = reinterpret_cast<float2*>(sb + lay.out);
  const RowSeg* const SEG = reinterpret_cast<const RowSeg*>(sb + lay.seg);
  float* const SC = reinterpret_cast<float*>(sb + lay.sc);
  int* const CS = reinterpret_cast<int*>(sb + lay.cs);  // per chunk channel: its slots SLT[CS[c] .. CS[c + 1])
  int* const SLT = CS + nch + 1;
  int* const GC = SLT + nslot;                          // its request-order channel
  const unsigned mb = smem_u32(sb + lay.mb);

  const long long V = (long long)L * L * L;
  const long long q_begin = (long long)(blockIdx.x / nchunks) * qb;
  const long long q_end = min(V, q_begin + qb);
  const int base1 = ck.base1, n1c = ck.ncell1, base2 = ck.base2, n2c = ck.ncell2;

  if constexpr (TMA) {
    // another CTA of this launch gave up on a slab wait: leave at once
    if (__syncthreads_or(threadIdx.x == 0 && (*reinterpret_cast<volatile int*>(flags) & 2))) return;
    if (threadIdx.x == 0) {
      mbar_init(mb, 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      if (q_begin < q_end) {
        if (skip_first)  // test switch: arm the barrier, issue no box (the wait runs out, nothing in flight)
          mbar_expect_tx(mb, 32u);
        else
          tma_issue_slabs(&fbmap, smem_u32(SL), NBS_ROW_SLAB * 32u, mb, base1, n1c, (int)q_begin, base2, n2c,
                          (int)minus_q(q_begin, L));
      }
    }
  }
  if (threadIdx.x < NBS_ROW_SCALES) SC[threadIdx.x] = scales[threadIdx.x];
  if (threadIdx.x == 0) {
    int n = 0;
    for (int c = 0; c < nch; ++c) {
      CS[c] = n;
      for (int w = 0; w < NW; ++w) {
        const int r = c - ck.cfirst[w];
        if (r >= 0 && r < ck.out_base[w + 1] - ck.out_base[w]) SLT[n++] = ck.out_base[w] + r;
      }
      GC[c] = row_ch[ck.ch_off + c];
    }
    CS[nch] = n;
  }
  {
    const uint4* g = reinterpret_cast<const uint4*>(rec + ck.rec_off);
    for (int i = threadIdx.x; i < nstep * 8; i += NT) cp16((uint4*)REC + i, g + i);
    const uint4* ga = reinterpret_cast<const uint4*>(aent + ck.aent_off);
    for (int i = threadIdx.x; i < (ck.naent + 7) / 8; i += NT) cp16((uint4*)AE + i, ga + i);
    const uint4* gd = reinterpret_cast<const uint4*>(adesc + ck.adesc_off);
    for (int i = threadIdx.x; i < (nrow + 3) / 4; i += NT) cp16((uint4*)AD + i, gd + i);
    const uint4* gs = reinterpret_cast<const uint4*>(segs + ck.seg_off);
    for (int i = threadIdx.x; i < nseg; i += NT) cp16((uint4*)SEG + i, gs + i);
  }
  auto stage_slabs_async = [&](long long q) {  // 16-byte cp.async by all threads (no tensor map)
    const long long qm = minus_q(q, L);
    for (int i = threadIdx.x; i < 2 * n1c; i += NT)
      cp16(SL + i, reinterpret_cast<const char*>(FB + ((long long)(base1 + (i >> 1)) * V + q) * 4) + 16 * (i & 1));
    for (int i = threadIdx.x; i < 2 * n2c; i += NT)
      cp16(SL + 2 * NBS_ROW_SLAB + i,
           reinterpret_cast<const char*>(FB + ((long long)(base2 + (i >> 1)) * V + qm) * 4) + 16 * (i & 1));
  };
  if (!TMA && q_begin < q_end) stage_slabs_async(q_begin);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < nslot * 64; i += NT) OUT[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s_begin = ck.seg_base[w], s_end = ck.seg_base[w + 1];
  float2* const out_w = OUT + (ck.out_base[w] - ck.cfirst[w]) * 64;
  const char* const E1b = reinterpret_cast<const char*>(E);
  const char* const E2b = E1b + (size_t)nrow1 * 32;
  unsigned parity = 0;
  for (long long q = q_begin; q < q_end; ++q, parity ^= 1u) {
    if constexpr (TMA) {
      const bool ok = mbar_wait_timed(mb, parity, RWAIT_NS);
      if (__syncthreads_or(!ok)) {
        // flag the launch; before leaving, wait (bounded) for the one transfer that may be in flight
        if (threadIdx.x == 0) {
          atomicOr(flags, 2);
          if (!skip_first || q != q_begin)
            for (int k = 0; k < 8 && !mbar_wait_timed(mb, parity, RWAIT_NS); ++k) {
            }
        }
        __syncthreads();
        return;
      }
    }
    // ---- phase A: the distinct effective-block rows, all four sink spins ----
    for (int r = threadIdx.x; r < nrow; r += NT) {
      const unsigned d = AD[r];
      const int cnt = (int)(d >> 20);
      const unsigned short* p = AE + (d & 0xFFFFFu);
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
      for (int i = 0; i < cnt; ++i) {
        const unsigned x = p[i];
        float c = (x & 0x1000u) ? 2.f : 1.f;
        c = (x & 0x800u) ? -c : c;
        const float4* sp = SL + 2 * (x & 0x7FFu);
        const float4 v0 = sp[0], v1 = sp[1];
        a0.x = fmaf(c, v0.x, a0.x);
        a0.y = fmaf(c, v0.y, a0.y);
        a0.z = fmaf(c, v0.z, a0.z);
        a0.w = fmaf(c, v0.w, a0.w);
        a1.x = fmaf(c, v1.x, a1.x);
        a1.y = fmaf(c, v1.y, a1.y);
        a1.z = fmaf(c, v1.z, a1.z);
        a1.w = fmaf(c, v1.w, a1.w);
      }
      E[2 * r] = a0;
      E[2 * r + 1] = a1;
    }
    __syncthreads();
    // the slab buffer is free: the next momentum's boxes land during phase B
    if (q + 1 < q_end) {
      if constexpr (TMA) {
        if (threadIdx.x == 0)
          tma_issue_slabs(&fbmap, smem_u32(SL), NBS_ROW_SLAB * 32u, mb, base1, n1c, (int)(q + 1), base2, n2c,
                          (int)minus_q(q + 1, L));
      } else {
        stage_slabs_async(q + 1);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // ---- phase B: products of the rows over the records ----
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    for (int si = s_begin; si < s_end; ++si) {
      const RowSeg sg = SEG[si];
      const unsigned* R = REC + sg.sbeg * 32 + lane;
#pragma unroll 1
      for (int st = sg.sbeg; st < sg.send; ++st, R += 32) {
        const unsigned wd = *R;
        const float sc = SC[wd & 31u];
        const float4* pa = reinterpret_cast<const float4*>(E1b + (wd & 0xFFE0u));
        const float4* pb = reinterpret_cast<const float4*>(E2b + (wd >> 16));
        const float4 a0 = pa[0], a1 = pa[1], b0 = pb[0], b1 = pb[1];
        const float2 a[4] = {make_float2(a0.x * sc, a0.y * sc), make_float2(a0.z * sc, a0.w * sc),
                             make_float2(a1.x * sc, a1.y * sc), make_float2(a1.z * sc, a1.w * sc)};
        const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                             make_float2(b1.z, b1.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 z = make_float2(acc[2 * (4 * i + j)], acc[2 * (4 * i + j) + 1]);
            cfma<float>(z, a[i], b[j]);
            acc[2 * (4 * i + j)] = z.x;
            acc[2 * (4 * i + j) + 1] = z.y;
          }
      }
      rows_flush(acc, lane, out_w + sg.local * 64);
    }
    __syncthreads();
    // ---- the channels' sums, slots in warp order ----
    for (int i = threadIdx.x; i < nch * 64; i += NT) {
      const int c = i >> 6, m = i & 63;
      float2 sum = make_float2(0.f, 0.f);
      for (int k = CS[c]; k < CS[c + 1]; ++k) {
        float2& v = OUT[SLT[k] * 64 + m];
        sum.x += v.x;
        sum.y += v.y;
        v = make_float2(0.f, 0.f);
      }
      const int spin = (m & ~3) | ((m & 1) << 1) | ((m >> 1) & 1);  // [a1][a2][a3 + 2 a4] -> [a1][a2][a3][a4]
      Ft[((long long)GC[c] * 64 + spin) * V + q] = sum;
    }
    if constexpr (!TMA) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
    }
  }
}

}  // namespace

size_t row_chunk_smem(int nrow, int naent, int nstep, int nslot, int nseg, int nch) {
  return 128 + row_layout(nrow, naent, nstep, nslot, nseg, nch).total;
}

cudaError_t launch_contract_rows(const float2* FB, long long ncells, int L, int nchunks, int qb, const void* chunks,
                                 const unsigned short* aent, const unsigned* adesc, const unsigned* rec,
                                 const void* segs, const int* row_ch, const float* scales, int smem, float2* Ft,
                                 int* flags, int skip_first, cudaStream_t st) {
  const long long V = (long long)L * L * L;
  if (nchunks <= 0 || qb <= 0 || smem <= 0 || !flags) return cudaErrorInvalidValue;
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL) return cudaErrorInvalidValue;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const bool tma = encode_fb_map(&map, FB, V, ncells);
  auto kern = tma ? k_contract_rows<NBS_ROW_WARPS, true> : k_contract_rows<NBS_ROW_WARPS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(nqb * nchunks), NBS_ROW_WARPS * 32, smem, st>>>(
      map, FB, L, nchunks, qb, (const RowChunkHdr*)chunks, aent, adesc, rec, (const RowSeg*)segs, row_ch, scales, Ft,
      flags, tma ? skip_first : 0);
  return cudaGetLastError();
}

}  // namespace nbs
