// kernels_rows.cu -- the effective blocks (Eq. (4.2)) and their product
// (Eq. (4.3)) in two phases per momentum, FP32.
//
// A CTA of 16 warps keeps one chunk's row tables in shared memory
// (plan_rows.cpp) and sweeps a block of momenta:
//   * phase A(q): each thread builds whole effective-block rows, sums of
//     +-1 / +-2 times cells of the two staged slabs (B1's stored type at q,
//     B2's at -q; per cell 16 bytes of sink spins 0, 1 and 16 bytes of spins
//     2, 3 in separate planes, staged by 4-D TMA boxes), for all four spins at
//     once (one decode per entry, two 16-byte loads, eight FMAs).
//     The rows live in two planes of 16-byte entries (sink spins 0, 1 and
//     2, 3), double-buffered by the parity of q; row numbers are chosen so
//     that the rows a quarter warp loads together differ mod 8 (no bank
//     conflicts);
//   * phase B(q): lane 4 kq + s of a warp takes record (8 step + kq, s) --
//     read from global memory (L1/L2), four steps ahead -- naming the B1 row
//     and B2 row of shared index xi~ for output source-spin pair s and a
//     scale; it forms the 4 x 4 outer product over the sink spins alpha1,
//     alpha2 and accumulates 16 complex values.  At the end of each channel
//     segment the warp sums over its eight kq lanes into its slot (slots
//     double-buffered by the parity of q);
//   * each warp runs B(q) and then its share of A(q + 1); one barrier per
//     momentum, after which one thread issues the TMA boxes of the slabs of
//     q + 2 (the slab buffer is single) and the slots of q are summed in warp
//     order (deterministic) into F~[channel][spin][q].
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
constexpr int RPREF = 3;                                  // records of a warp's first steps kept in registers

struct RowLayout {
  unsigned e, aent, adesc, out, seg, sc, cs, mb, total;
};

// shared-memory layout of one chunk (offsets from a 128-byte aligned base):
// slab, one or two row buffers of two planes, row tables, two slot buffers, segments, scales, channel lists
__host__ __device__ inline RowLayout row_layout(int nbuf, int nrow, int nadesc, int naent, int nslot, int nseg,
                                                int nch) {
  RowLayout L;
  unsigned o = RSLAB_BYTES;
  L.e = o;
  o += (unsigned)nbuf * (unsigned)nrow * 32u;
  L.aent = o;
  o += (unsigned)((naent + 7) / 8) * 16u;
  L.adesc = o;
  o += (unsigned)((nadesc + 3) / 4) * 16u;
  L.out = o;
  o += 2u * (unsigned)nslot * 512u;
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

// the index of -q in the momentum geometry (componentwise (L - n) mod L; y through the mirror table)
__device__ __forceinline__ long long minus_q(long long q, const MomGeom& g) {
  const int L = g.L, Ly = g.Ly;
  const int x = (int)(q % L), y = (int)((q / L) % Ly), z = (int)(q / ((long long)L * Ly));
  return (long long)((L - x) % L) + L * ((long long)g.ymir[y] + (long long)Ly * ((L - z) % L));
}

__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}

// Stage the planar slabs of one momentum into S with mbarrier mb (one thread, after the block has finished
// reading S): side 1 ncell1 cells from base1 at q, side 2 ncell2 cells from base2 at qm.  The tensor map
// sees the stored blocks as [momentum][half][cell][4 floats] (half = sink spins 0, 1 or 2, 3); a box of
// NBS_ROW_BOX cells and both halves lands as [half][cell][16 bytes], box k of side s at 16-byte unit
// s * 2 NBS_ROW_SLAB + k * 2 NBS_ROW_BOX.  The box's x coordinate is always 0 (16-byte aligned).
__device__ __forceinline__ void tma_issue_planar(const CUtensorMap* map, unsigned S, unsigned mb, int base1, int ncell1,
                                                 int q, int base2, int ncell2, int qm) {
  const int nb1 = (ncell1 + NBS_ROW_BOX - 1) / NBS_ROW_BOX, nb2 = (ncell2 + NBS_ROW_BOX - 1) / NBS_ROW_BOX;
  constexpr unsigned box = 2u * NBS_ROW_BOX * 16u;
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier generic reads of S first
  mbar_expect_tx(mb, (unsigned)(nb1 + nb2) * box);
  for (int k = 0; k < nb1; ++k) tma_load_4d(S + k * box, map, 0, base1 + k * NBS_ROW_BOX, 0, q, mb);
  for (int k = 0; k < nb2; ++k)
    tma_load_4d(S + 2u * NBS_ROW_SLAB * 16u + k * box, map, 0, base2 + k * NBS_ROW_BOX, 0, qm, mb);
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
    const __grid_constant__ CUtensorMap fbmap, const __grid_constant__ MomGeom geom, const float2* __restrict__ FB,
    int nchunks, int qb,
    const RowChunkHdr* __restrict__ chunks, const unsigned short* __restrict__ aent,
    const unsigned* __restrict__ adesc, const unsigned* __restrict__ rec, const RowSeg* __restrict__ segs,
    const int* __restrict__ row_ch, const float* __restrict__ scales, float2* __restrict__ Ft,
    int* __restrict__ flags, int skip_first) {
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;
  unsigned char* const sb = smem_raw + pad;
  const RowChunkHdr& ck = chunks[blockIdx.x % nchunks];
  const int nrow1 = ck.nrow1, nrow = ck.nrow1 + ck.nrow2, nslot = ck.nslot, nch = ck.nch;
  const int nseg = ck.seg_base[NW], nadesc = ck.nadesc, nbuf = ck.nbuf;
  const RowLayout lay = row_layout(nbuf, nrow, nadesc, ck.naent, nslot, nseg, nch);
  float4* const SL = reinterpret_cast<float4*>(sb);  // slab: [2][NBS_ROW_SLAB] cells of two float4
  // row buffer b: E0 + 2 b nrow; plane 0 [nrow] (sink spins 0, 1), plane 1 [nrow] (spins 2, 3); B2's rows
  // from nrow1
  float4* const E0 = reinterpret_cast<float4*>(sb + lay.e);
  const unsigned short* const AE = reinterpret_cast<const unsigned short*>(sb + lay.aent);
  const unsigned* const AD = reinterpret_cast<const unsigned*>(sb + lay.adesc);
  float2* const OUT0 = reinterpret_cast<float2*>(sb + lay.out);  // slot buffer b: OUT0 + b nslot 64
  const RowSeg* const SEG = reinterpret_cast<const RowSeg*>(sb + lay.seg);
  float* const SC = reinterpret_cast<float*>(sb + lay.sc);
  int* const CS = reinterpret_cast<int*>(sb + lay.cs);  // per chunk channel: its slots SLT[CS[c] .. CS[c + 1])
  int* const SLT = CS + nch + 1;
  int* const GC = SLT + nslot;                          // its request-order channel
  const unsigned mb = smem_u32(sb + lay.mb);

  const long long V = (long long)geom.L * geom.Ly * geom.L;  // momenta of this launch
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
          tma_issue_planar(&fbmap, smem_u32(SL), mb, base1, n1c, (int)q_begin, base2, n2c, (int)minus_q(q_begin, geom));
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
    const uint4* ga = reinterpret_cast<const uint4*>(aent + ck.aent_off);
    for (int i = threadIdx.x; i < (ck.naent + 7) / 8; i += NT) cp16((uint4*)AE + i, ga + i);
    const uint4* gd = reinterpret_cast<const uint4*>(adesc + ck.adesc_off);
    for (int i = threadIdx.x; i < (nadesc + 3) / 4; i += NT) cp16((uint4*)AD + i, gd + i);
    const uint4* gs = reinterpret_cast<const uint4*>(segs + ck.seg_off);
    for (int i = threadIdx.x; i < nseg; i += NT) cp16((uint4*)SEG + i, gs + i);
  }
  auto stage_slabs_async = [&](long long q) {  // the same planar slabs by 16-byte cp.async (no tensor map)
    const long long qm = minus_q(q, geom);
    for (int i = threadIdx.x; i < 2 * (n1c + n2c); i += NT) {
      const int side = i >= 2 * n1c, k = side ? i - 2 * n1c : i, c = k >> 1, h = k & 1;
      const long long src = ((long long)((side ? base2 : base1) + c) * V + (side ? qm : q)) * 4 + 2 * h;
      cp16(SL + side * 2 * NBS_ROW_SLAB + (c / NBS_ROW_BOX) * 2 * NBS_ROW_BOX + h * NBS_ROW_BOX + c % NBS_ROW_BOX,
           FB + src);
    }
  };
  // the slabs of momentum qn into the (free) slab buffer
  auto stage_slabs = [&](long long qn) {
    if constexpr (TMA) {
      if (threadIdx.x == 0)
        tma_issue_planar(&fbmap, smem_u32(SL), mb, base1, n1c, (int)qn, base2, n2c, (int)minus_q(qn, geom));
    } else {
      stage_slabs_async(qn);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
  };
  if (!TMA && q_begin < q_end) stage_slabs_async(q_begin);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = threadIdx.x; i < 2 * nslot * 64; i += NT) OUT0[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  // phase A: this thread's share of the distinct rows from the staged slabs, into row buffer Eb
  auto phase_a = [&](float4* Eb) {
    // rows come longest first: deal them to the threads in snake order (reversed every other round)
    for (int r0 = 0, k = 0; r0 < nadesc; r0 += NT, ++k) {
      const int i = (k & 1) ? r0 + NT - 1 - (int)threadIdx.x : r0 + (int)threadIdx.x;
      if (i >= nadesc) continue;
      const unsigned d = AD[i];
      const int cnt = (int)((d >> 14) & 31u), r = (int)(d >> 19);
      const unsigned short* p = AE + (d & 0x3FFFu);
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
      for (int j = 0; j < cnt; ++j) {
        const unsigned x = p[j];
        float c = (x & 0x2000u) ? 2.f : 1.f;
        c = (x & 0x1000u) ? -c : c;
        const float4* sp = SL + (x & 0xFFFu);  // planar slab unit: spins 0, 1; spins 2, 3 one box-half on
        const float4 v0 = sp[0], v1 = sp[NBS_ROW_BOX];
        a0.x = fmaf(c, v0.x, a0.x);
        a0.y = fmaf(c, v0.y, a0.y);
        a0.z = fmaf(c, v0.z, a0.z);
        a0.w = fmaf(c, v0.w, a0.w);
        a1.x = fmaf(c, v1.x, a1.x);
        a1.y = fmaf(c, v1.y, a1.y);
        a1.z = fmaf(c, v1.z, a1.z);
        a1.w = fmaf(c, v1.w, a1.w);
      }
      Eb[r] = a0;
      Eb[nrow + r] = a1;
    }
  };
  // a slab wait gave up: flag the launch; before leaving, wait (bounded) for the transfer that may still
  // be in flight (none when the test switch withheld the first copy)
  auto give_up = [&](unsigned parity, bool in_flight) {
    if (threadIdx.x == 0) {
      atomicOr(flags, 2);
      if (in_flight)
        for (int k = 0; k < 8 && !mbar_wait_timed(mb, parity, RWAIT_NS); ++k) {
        }
    }
    __syncthreads();
  };

  // rows of the first momentum
  {
    bool ok = true;
    if (q_begin < q_end) {
      if constexpr (TMA) ok = mbar_wait_timed(mb, 0u, RWAIT_NS);
      if (ok) phase_a(E0);
    }
    if (__syncthreads_or(!ok)) {
      give_up(0u, !skip_first);
      return;
    }
    if (q_begin + 1 < q_end) stage_slabs(q_begin + 1);
  }

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s_begin = ck.seg_base[w], s_end = ck.seg_base[w + 1];
  // the warp's records: steps [SEG[s_begin].sbeg, SEG[s_end - 1].send), the same for every momentum; the
  // first RPREF of them stay in registers, the rest are read RPREF steps ahead (the table has RPREF
  // padding steps after its last chunk)
  const int st_a = s_begin < s_end ? SEG[s_begin].sbeg : 0, st_b = s_begin < s_end ? SEG[s_end - 1].send : 0;
  const unsigned* const R0 = rec + ck.rec_off + st_a * 32 + lane;
  unsigned first[RPREF];
#pragma unroll
  for (int k = 0; k < RPREF; ++k) first[k] = __ldg(R0 + 32 * k);
  for (long long q = q_begin; q < q_end; ++q) {
    const int b = (int)((q - q_begin) & 1), eb = nbuf == 2 ? b : 0;
    const float4* const E1 = E0 + 2 * eb * nrow;
    const float4* const E2 = E1 + nrow1;
    float2* const out_w = OUT0 + b * nslot * 64 + (ck.out_base[w] - ck.cfirst[w]) * 64;
    // ---- phase B(q): products of the rows over the records ----
    // two steps per iteration with two operand sets: the rows of step st + 1 are loaded while step st's
    // products run (and those of st + 2 during st + 1's); records are read two steps ahead
    {
      float acc[32];  // complex 4 alpha1 + alpha2 as floats 2 c, 2 c + 1
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.f;
      const unsigned* R = R0 + 64;  // record of step st_a + 2
      unsigned recA = first[0], recB = first[1];
      float4 xa0, xa1, ya0, ya1, xb0, xb1, yb0, yb1;
      float sa = 0.f, sb2 = 0.f;
      auto rows_of = [&](unsigned wd, float4& x0, float4& x1, float4& y0, float4& y1, float& scale) {
        scale = SC[wd >> 24];
        const float4* pa = E1 + (wd & 0xFFFu);
        const float4* pb = E2 + ((wd >> 12) & 0xFFFu);
        x0 = pa[0];
        x1 = pa[nrow];
        y0 = pb[0];
        y1 = pb[nrow];
      };
      auto product = [&](const float4& x0, const float4& x1, const float4& y0, const float4& y1, float scale) {
        const float2 a[4] = {make_float2(x0.x * scale, x0.y * scale), make_float2(x0.z * scale, x0.w * scale),
                             make_float2(x1.x * scale, x1.y * scale), make_float2(x1.z * scale, x1.w * scale)};
        const float2 b[4] = {make_float2(y0.x, y0.y), make_float2(y0.z, y0.w), make_float2(y1.x, y1.y),
                             make_float2(y1.z, y1.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 z = make_float2(acc[2 * (4 * i + j)], acc[2 * (4 * i + j) + 1]);
            cfma<float>(z, a[i], b[j]);
            acc[2 * (4 * i + j)] = z.x;
            acc[2 * (4 * i + j) + 1] = z.y;
          }
      };
      int si = s_begin, seg_end = si < s_end ? SEG[si].send : 0, local = si < s_end ? SEG[si].local : 0;
      auto after_step = [&](int st) {
        if (st + 1 == seg_end) {
          rows_flush(acc, lane, out_w + local * 64);
          if (++si < s_end) {
            seg_end = SEG[si].send;
            local = SEG[si].local;
          }
        }
      };
      if (st_a < st_b) {
        rows_of(recA, xa0, xa1, ya0, ya1, sa);
        recA = first[2];
      }
#pragma unroll 1
      for (int st = st_a; st < st_b; st += 2) {
        // step st in set a (loaded); load set b with step st + 1
        const bool more = st + 1 < st_b;
        if (more) {
          rows_of(recB, xb0, xb1, yb0, yb1, sb2);
          recB = __ldg(R + 32);  // step st + 3
        }
        product(xa0, xa1, ya0, ya1, sa);
        after_step(st);
        if (!more) break;
        if (st + 2 < st_b) {
          rows_of(recA, xa0, xa1, ya0, ya1, sa);
          recA = __ldg(R + 64);  // step st + 4
        }
        R += 64;
        product(xb0, xb1, yb0, yb1, sb2);
        after_step(st + 1);
      }
    }
    // ---- phase A(q + 1): this thread's rows, once the slabs of q + 1 have landed ----
    bool ok = true;
    const unsigned parity = (unsigned)((q + 1 - q_begin) & 1);
    if (q + 1 < q_end) {
      if constexpr (TMA) {
        ok = mbar_wait_timed(mb, parity, RWAIT_NS);
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
      // one row buffer (or cp.async staging by all threads): every warp finishes B(q) first
      if (nbuf == 1 || !TMA) __syncthreads();
      if (ok) phase_a(E0 + 2 * (nbuf == 2 ? b ^ 1 : 0) * nrow);
    }
    if (__syncthreads_or(!ok)) {
      give_up(parity, true);
      return;
    }
    // every thread is past B(q) and A(q + 1): the slab buffer is free for q + 2
    if (q + 2 < q_end) stage_slabs(q + 2);
    // ---- the channels' sums of q, slots in warp order ----
    float2* const OUTb = OUT0 + b * nslot * 64;
    for (int i = threadIdx.x; i < nch * 64; i += NT) {
      const int c = i >> 6, m = i & 63;
      float2 sum = make_float2(0.f, 0.f);
      for (int k = CS[c]; k < CS[c + 1]; ++k) {
        float2& v = OUTb[SLT[k] * 64 + m];
        sum.x += v.x;
        sum.y += v.y;
        v = make_float2(0.f, 0.f);
      }
      const int spin = (m & ~3) | ((m & 1) << 1) | ((m >> 1) & 1);  // [a1][a2][a3 + 2 a4] -> [a1][a2][a3][a4]
      Ft[((long long)GC[c] * 64 + spin) * V + q] = sum;
    }
  }
}

}  // namespace

size_t row_chunk_smem(int nbuf, int nrow, int nadesc, int naent, int nslot, int nseg, int nch) {
  return 128 + row_layout(nbuf, nrow, nadesc, naent, nslot, nseg, nch).total;
}

using EncodeTiledRows = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The stored blocks [cell][momentum][8 floats] seen as a 4-D FP32 tensor (4 floats; cells, stride V * 32
// bytes; halves, stride 16; momenta, stride 32) with boxes of 4 x NBS_ROW_BOX x 2 x 1: one box is
// NBS_ROW_BOX cells of one momentum, both halves, landing as [half][cell][16 bytes].  false if TMA is not
// available (the kernel then stages with cp.async).
static bool encode_fb_map_planar(CUtensorMap* map, const float2* FB, long long V, long long ncells) {
  static EncodeTiledRows fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledRows>(p);
  }();
  if (!fn || !FB || (reinterpret_cast<uintptr_t>(FB) & 15) || V <= 0 || ncells <= 0 || V > (1LL << 31)) return false;
  const cuuint64_t dim[4] = {4, (cuuint64_t)ncells, 2, (cuuint64_t)V};
  const cuuint64_t stride[3] = {(cuuint64_t)V * 32, 16, 32};
  const cuuint32_t box[4] = {4, (cuuint32_t)NBS_ROW_BOX, 2, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(FB), dim, stride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_contract_rows(const float2* FB, long long ncells, const MomGeom& geom, int nchunks, int qb,
                                 const void* chunks,
                                 const unsigned short* aent, const unsigned* adesc, const unsigned* rec,
                                 const void* segs, const int* row_ch, const float* scales, int smem, float2* Ft,
                                 int* flags, int skip_first, cudaStream_t st) {
  const long long V = (long long)geom.L * geom.Ly * geom.L;
  if (nchunks <= 0 || qb <= 0 || smem <= 0 || !flags || geom.L < 1 || geom.L > 64 || geom.Ly < 1 || geom.Ly > geom.L)
    return cudaErrorInvalidValue;
  for (int y = 0; y < geom.Ly; ++y)
    if (geom.ymir[y] < 0 || geom.ymir[y] >= geom.Ly) return cudaErrorInvalidValue;
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL) return cudaErrorInvalidValue;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const bool tma = encode_fb_map_planar(&map, FB, V, ncells);
  auto kern = tma ? k_contract_rows<NBS_ROW_WARPS, true> : k_contract_rows<NBS_ROW_WARPS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(nqb * nchunks), NBS_ROW_WARPS * 32, smem, st>>>(
      map, geom, FB, nchunks, qb, (const RowChunkHdr*)chunks, aent, adesc, rec, (const RowSeg*)segs, row_ch, scales, Ft,
      flags, tma ? skip_first : 0);
  return cudaGetLastError();
}

}  // namespace nbs
