// kernels_rows.cu -- the effective blocks (Eq. (4.2)) and their product
// (Eq. (4.3)) in two kernels, FP32.
//
// Over all channels an effective-block row (one shared index xi~ and one held
// source spin of one side: a sum of +-1 / +-2 times stored cells, kept up to a
// scale) depends only on the stored type it sums, a few hundred rows per type
// (plan_rows.cpp).  So:
//   * k_eff_rows (phase A) builds every row of every type at every momentum,
//     all four sink spins at once, into a momentum-major array RQ: the rows
//     of type T at momentum q are one contiguous block (sink spins 0, 1 of all
//     its rows, then spins 2, 3).  A warp takes eight rows at four
//     consecutive momenta, so its loads of a cell are one 128-byte line and
//     its stores of a plane are 128 contiguous bytes: the kernel streams the
//     stored blocks once and writes the rows once (HBM-bound).
//   * k_contract_rows (phase B): a block keeps one chunk's tables (whole
//     channels of one pair of stored types) and sweeps a block of momenta.
//     One helper thread copies the rows of type1 at q and of type2 at -q into
//     a ring of NBS_ROW_STAGES stages (two bulk copies per momentum, completed
//     on the stage's mbarrier); twelve consumer warps form the products: lane
//     8 g + kq takes record (step, g, kq) -- read from global memory
//     (L1/L2), two steps ahead -- naming a B1 row and a B2 row for the output
//     source-spin pair s its segment gives lane group g, and a scale; it forms
//     the 4 x 4 outer product over the sink spins alpha1, alpha2 and
//     accumulates 16 complex values.  At the end of each segment (a run of
//     steps of one channel and one group map) the warp sums over the eight kq
//     lanes of each group into its slot (one slot buffer per stage).  The four helper
//     warps sum the slots of a finished momentum in warp order
//     (deterministic) into F~[ch][spin][q] and then refill that stage.
// Consumers wait on full[stage] (the copies' bytes) and arrive on
// empty[stage]; only the helpers wait on empty[stage].  A consumer never waits
// for another consumer, and the consumer warps run up to NBS_ROW_STAGES - 1
// momenta apart.  Every wait is bounded by the global timer (one second); a
// wait that gives up sets bit 1 of flags, the block finishes without waiting
// again (after letting its copies in flight land) and the call reports the
// timeout.
//
// The blocks run momentum block by momentum block, so the chunks of a momentum
// block share its rows in L2, and within one the chunks come largest first
// (plan order), so the launch ends on the shortest blocks.  Within a block the
// momenta are visited in the order of a list that places -q right after q (as
// (q, -q) pairs): the rows read at -q are the ones other chunks read at q.
#include <vector>

#include "common.cuh"
#include "plan.h"

namespace nbs {

namespace {

constexpr int RPREF = 3;  // records of a warp's first steps kept in registers

struct RowLayout {
  unsigned rows, out, seg, sc, cs, mb, total;
};

// shared-memory layout of one chunk (offsets from a 128-byte aligned base): the row stages (each B1's rows
// then B2's, two planes of 16-byte units each), one slot buffer per stage, segments, scales, channel lists,
// the mbarriers full[stage], empty[stage] and an abort word
__host__ __device__ inline RowLayout row_layout(int nrow1, int nrow2, int nslot, int nseg, int nch) {
  RowLayout L;
  unsigned o = 0;
  L.rows = o;
  o += (unsigned)NBS_ROW_STAGES * 2u * (unsigned)(nrow1 + nrow2) * 16u;
  L.out = o;
  o += (unsigned)NBS_ROW_STAGES * (unsigned)nslot * 512u;
  L.seg = o;
  o += (unsigned)nseg * 16u;
  L.sc = o;
  o += 4u * NBS_ROW_SCALES;
  L.cs = o;
  o += (unsigned)((2 * nch + nslot + 1 + 3) / 4) * 16u;
  L.mb = o;
  o += (unsigned)(2 * NBS_ROW_STAGES * 8 + 16);
  L.total = o;
  return L;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) completing on mbarrier mbar
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mb_expect_tx(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}

// sum a lane's 32 floats over the eight lanes of its group g (xor 4, 2, 1),
// halving the kept length at each stage: lane 8 g + kq ends with the floats
// 4 kq .. 4 kq + 3 of its original 32, summed over the group
template <int M>
__device__ __forceinline__ void kq_reduce(float (&acc)[32], int lane) {
  if constexpr (M >= 4) {
    constexpr int D = M / 4;  // partner distance: kq bit 2, 1, 0 for kept lengths 16, 8, 4
    const bool up = lane & D;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float keep = up ? acc[M + j] : acc[j];
      const float give = up ? acc[j] : acc[M + j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, give, D);
    }
    kq_reduce<M / 2>(acc, lane);
  }
}

// acc holds complex 4 alpha1 + alpha2 (floats 2 c, 2 c + 1) for the output pair s
// of the lane's group g = lane >> 3, s = (map >> 2 g) & 3; add the segment's sum
// into slot[16 alpha1 + 4 alpha2 + s] and clear acc.  Groups that share an s add
// in turn, lowest group first (map bits 8 + 2 g: the group's turn; bits 16..18:
// the number of turns).
__device__ __forceinline__ void rows_flush(float (&acc)[32], int lane, float2* slot, int map) {
  kq_reduce<16>(acc, lane);
  const int kq = lane & 7, g = lane >> 3, s = (map >> (2 * g)) & 3;
  const int rank = (map >> (8 + 2 * g)) & 3, passes = (map >> 16) & 7;  // turn of this group, turns
  float2* o = slot + 8 * kq + s;  // complex 2 kq: alpha1 = kq >> 1, alpha2 = 2 (kq & 1)
  for (int p = 0; p < passes; ++p) {
    if (rank == p) {
      o[0].x += acc[0];
      o[0].y += acc[1];
      o[4].x += acc[2];
      o[4].y += acc[3];
    }
    __syncwarp();
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
}

// named barrier of the four helper warps (0 is __syncthreads)
constexpr int BAR_PROD = 1;
constexpr unsigned long long RWAIT_NS = 1000000000ull;  // hand-off wait limit (global timer)

__device__ __forceinline__ void nb_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
// arrive (release at CTA scope: this thread's earlier shared-memory accesses are ordered before it)
__device__ __forceinline__ void mb_arrive(unsigned a) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// wait (acquire) for the phase of parity `parity` to complete, bounded: after RWAIT_NS of the global timer
// (or once another thread of the CTA has given up, *abort != 0) it sets *abort and bit 1 of flags and
// returns false; the CTA then finishes without waiting again
__device__ __forceinline__ bool mb_wait(unsigned a, unsigned parity, volatile int* abort, int* flags) {
  unsigned long long t0 = 0;
  for (int i = 0; i < (1 << 28); ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      const unsigned long long t = now_ns();
      if (!t0) t0 = t;
      else if (t - t0 > RWAIT_NS) break;
    }
  }
  *abort = 1;
  atomicOr(flags, 2);
  return false;
}

// Phase A: every row of every type at momenta [0, V).  A block takes tiles of (eight consecutive rows of
// one type, 32 consecutive momenta); warp w builds row w of the tile with lane = momentum offset, so the
// loads of a cell are one contiguous 1 KB run (32 momenta x 32 bytes) and a warp walks its row's entries
// in lockstep.  The tile goes through shared memory so that each momentum's eight rows leave as one
// 128-byte line per plane.  Row r (global, of type t) at momentum q: unit q 2 NR + roff_t + r holds sink
// spins 0, 1, that unit + nrow_t spins 2, 3.  The row tables sit in shared memory.
constexpr int EFF_THREADS = 256;  // eight warps: the eight rows of a tile
constexpr int EFF_TILE_BYTES = 2 * 2 * 32 * 8 * 16;  // two tile buffers

__global__ void __launch_bounds__(EFF_THREADS) k_eff_rows(const float4* __restrict__ FB, long long V,
                                                          const RowTypeHdr* __restrict__ types, int ntypes,
                                                          const unsigned* __restrict__ desc,
                                                          const unsigned short* __restrict__ ent, int nent, int NR,
                                                          float4* __restrict__ RQ) {
  extern __shared__ __align__(16) unsigned char eff_smem[];
  // two tile buffers [buffer][plane][32 momenta][8 rows], the row slot k of momentum m at k ^ (m & 7), so
  // that the eight lanes of a quarter-warp (eight momenta, one row) write eight different bank groups
  float4* const TT = reinterpret_cast<float4*>(eff_smem);
  int* const TY = reinterpret_cast<int*>(eff_smem + EFF_TILE_BYTES);                 // [ntypes][3]
  unsigned* const DS = reinterpret_cast<unsigned*>(eff_smem + EFF_TILE_BYTES + 128);  // [NR]
  unsigned short* const ES = reinterpret_cast<unsigned short*>(DS + NR);              // [nent]
  for (int i = threadIdx.x; i < ntypes; i += EFF_THREADS) {
    TY[3 * i] = types[i].base;
    TY[3 * i + 1] = types[i].roff;
    TY[3 * i + 2] = types[i].nrow;
  }
  for (int i = threadIdx.x; i < NR; i += EFF_THREADS) DS[i] = desc[i];
  for (int i = threadIdx.x; i < nent; i += EFF_THREADS) ES[i] = ent[i];
  __syncthreads();

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, noct = NR / 8;
  const long long nq32 = (V + 31) / 32, ntiles = nq32 * noct;
  int buf = 0;
  // one barrier per tile: a warp that reaches the build of tile i + 2 (into this buffer again) has passed
  // the barrier after the build of tile i + 1, which every warp reaches only after its stores of tile i
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const long long qb = tile / noct;
    const int oct = (int)(tile - qb * noct);
    float4* const TB = TT + buf * 512;
    // build: warp w, row 8 oct + w, momentum 32 qb + lane
    {
      const int r = 8 * oct + w;
      const long long q = 32 * qb + lane;
      const unsigned d = DS[r];
      const int cnt = (int)((d >> 24) & 31u), t = (int)(d >> 29);
      const unsigned short* e = ES + (d & 0xFFFFFFu);
      const float4* const col = FB + 2 * min(q, V - 1);  // momentum q of cell 0 (clamped: q >= V is not stored)
      const long long cstride = 2 * V;
      const int base = TY[3 * t];
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
      auto add = [&](unsigned x, const float4& u0, const float4& u1) {
        float c = (x & 0x2000u) ? 2.f : 1.f;
        c = (x & 0x1000u) ? -c : c;
        a0.x = fmaf(c, u0.x, a0.x);
        a0.y = fmaf(c, u0.y, a0.y);
        a0.z = fmaf(c, u0.z, a0.z);
        a0.w = fmaf(c, u0.w, a0.w);
        a1.x = fmaf(c, u1.x, a1.x);
        a1.y = fmaf(c, u1.y, a1.y);
        a1.z = fmaf(c, u1.z, a1.z);
        a1.w = fmaf(c, u1.w, a1.w);
      };
      int j = 0;
      for (; j + 3 < cnt; j += 4) {  // four entries at a time: eight 16-byte loads in flight
        unsigned x[4];
        float4 u[4][2];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          x[k] = e[j + k];
          const float4* p = col + (long long)(base + (int)(x[k] & 0xFFFu)) * cstride;
          u[k][0] = __ldg(p);
          u[k][1] = __ldg(p + 1);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) add(x[k], u[k][0], u[k][1]);
      }
      if (j + 1 < cnt) {  // two more (most rows have two entries): four loads in flight
        const unsigned x0 = e[j], x1 = e[j + 1];
        const float4* p0 = col + (long long)(base + (int)(x0 & 0xFFFu)) * cstride;
        const float4* p1 = col + (long long)(base + (int)(x1 & 0xFFFu)) * cstride;
        const float4 u0 = __ldg(p0), u1 = __ldg(p0 + 1), v0 = __ldg(p1), v1 = __ldg(p1 + 1);
        add(x0, u0, u1);
        add(x1, v0, v1);
        j += 2;
      }
      if (j < cnt) {
        const unsigned x = e[j];
        const float4* p = col + (long long)(base + (int)(x & 0xFFFu)) * cstride;
        add(x, __ldg(p), __ldg(p + 1));
      }
      const int sw = w ^ (lane & 7);
      TB[lane * 8 + sw] = a0;
      TB[256 + lane * 8 + sw] = a1;
    }
    __syncthreads();
    // store: unit u of the tile = (plane h, momentum m, row k), two per thread
    {
      const int t = (int)(DS[8 * oct] >> 29);
      const int roff = TY[3 * t + 1], nrow = TY[3 * t + 2];
      for (int u = threadIdx.x; u < 512; u += EFF_THREADS) {
        const int h = u >> 8, m = (u >> 3) & 31, k = u & 7;
        const long long q = 32 * qb + m;
        if (q < V) RQ[q * 2 * NR + roff + 8 * oct + k + h * nrow] = TB[h * 256 + m * 8 + (k ^ (m & 7))];
      }
    }
  }
}

// Phase B.  qlist: momenta in visiting order as (q, -q) index pairs of the launch's momentum geometry.
__global__ void __launch_bounds__((NBS_ROW_WARPS + NBS_ROW_HELPERS) * 32, 1) k_contract_rows(
    const float4* __restrict__ RQ, long long V, int NR, const int2* __restrict__ qlist, int nchunks, int qb,
    const RowChunkHdr* __restrict__ chunks, const unsigned* __restrict__ rec, const RowSeg* __restrict__ segs,
    const int* __restrict__ row_ch, const float* __restrict__ scales, float2* __restrict__ Ft,
    int* __restrict__ flags) {
  constexpr int NHW = NBS_ROW_HELPERS, NH = NHW * 32, NT = (NBS_ROW_WARPS + NHW) * 32, S = NBS_ROW_STAGES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;
  unsigned char* const sb = smem_raw + pad;
  // blocks momentum-block-major (the chunks of a momentum block share its rows in L2), the chunks of a
  // block largest first (plan order), so the launch ends on the shortest blocks
  const RowChunkHdr& ck = chunks[blockIdx.x % nchunks];
  const int nrow1 = ck.nrow1, nrow2 = ck.nrow2, nslot = ck.nslot, nch = ck.nch;
  const int nseg = ck.seg_base[NBS_ROW_WARPS];
  const RowLayout lay = row_layout(nrow1, nrow2, nslot, nseg, nch);
  // row stage b: RS0 + b stage_units; B1's rows plane 0 [nrow1], plane 1 [nrow1], then B2's likewise
  float4* const RS0 = reinterpret_cast<float4*>(sb + lay.rows);
  const int stage_units = 2 * (nrow1 + nrow2);
  float2* const OUT0 = reinterpret_cast<float2*>(sb + lay.out);  // slot buffer of stage b: OUT0 + b nslot 64
  const RowSeg* const SEG = reinterpret_cast<const RowSeg*>(sb + lay.seg);
  float* const SC = reinterpret_cast<float*>(sb + lay.sc);
  int* const CS = reinterpret_cast<int*>(sb + lay.cs);  // per chunk channel: its slots SLT[CS[c] .. CS[c + 1])
  int* const SLT = CS + nch + 1;
  int* const GC = SLT + nslot;                          // its request-order channel
  // full[b] (the stage's copies: one arrival with their byte count) at MBF + 8 b, empty[b] (the consumers'
  // 384 threads arrive once their products of the stage's momentum are done) at MBE + 8 b
  const unsigned MBF = smem_u32(sb + lay.mb), MBE = MBF + 8u * S;
  volatile int* const ABORT = reinterpret_cast<volatile int*>(sb + lay.mb + 16 * S);

  const long long i0 = (long long)(blockIdx.x / nchunks) * qb;  // this block: qlist[i0 .. i0 + n)
  const int n = (int)(min(V, i0 + qb) - i0);
  const int2* const QL = qlist + i0;

  if (threadIdx.x < NBS_ROW_SCALES) SC[threadIdx.x] = scales[threadIdx.x];
  if (threadIdx.x == 0) {
    for (int b = 0; b < S; ++b) {
      mb_init(MBF + 8u * b, 1);
      mb_init(MBE + 8u * b, NT - NH);
    }
    *ABORT = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    int m = 0;
    for (int c = 0; c < nch; ++c) {
      CS[c] = m;
      for (int w = 0; w < NBS_ROW_WARPS; ++w) {
        const int r = c - ck.cfirst[w];
        if (r >= 0 && r < ck.out_base[w + 1] - ck.out_base[w]) SLT[m++] = ck.out_base[w] + r;
      }
      GC[c] = row_ch[ck.ch_off + c];
    }
    CS[nch] = m;
  }
  {
    const uint4* gs = reinterpret_cast<const uint4*>(segs + ck.seg_off);
    for (int i = threadIdx.x; i < nseg; i += NT) cp16((uint4*)SEG + i, gs + i);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int i = threadIdx.x; i < S * nslot * 64; i += NT) OUT0[i] = make_float2(0.f, 0.f);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  // the rows of momentum index i into stage i % S (one thread): type1 at q, type2 at -q
  auto issue = [&](int i) {
    const int b = i % S;
    const int2 qq = QL[i];
    const unsigned mbar = MBF + 8u * b, dst = smem_u32(RS0 + b * stage_units);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier generic accesses of the stage
    mb_expect_tx(mbar, 32u * (unsigned)(nrow1 + nrow2));
    bulk_g2s(dst, RQ + (long long)qq.x * 2 * NR + 2 * ck.roff1, 32u * (unsigned)nrow1, mbar);
    bulk_g2s(dst + 32u * (unsigned)nrow1, RQ + (long long)qq.y * 2 * NR + 2 * ck.roff2, 32u * (unsigned)nrow2,
             mbar);
  };
  if (threadIdx.x == 0)
    for (int i = 0; i < S && i < n; ++i) issue(i);

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < NHW) {
    // ================= helpers =================
    const int tp = threadIdx.x;
    int last = min(S, n) - 1;  // the latest momentum index whose rows were issued (thread 0)
    for (int i = 0; i < n; ++i) {
      const int b = i % S;
      mb_wait(MBE + 8u * b, (unsigned)((i / S) & 1), ABORT, flags);  // every consumer is done with B(i)
      // the channels' sums of momentum i, slots in warp order; the slots are cleared
      float2* const OUTb = OUT0 + b * nslot * 64;
      const long long q = QL[i].x;
      for (int k = tp; k < nch * 64; k += NH) {
        const int c = k >> 6, m = k & 63;
        float2 sum = make_float2(0.f, 0.f);
        for (int j = CS[c]; j < CS[c + 1]; ++j) {
          float2& v = OUTb[SLT[j] * 64 + m];
          sum.x += v.x;
          sum.y += v.y;
          v = make_float2(0.f, 0.f);
        }
        const int spin = (m & ~3) | ((m & 1) << 1) | ((m >> 1) & 1);  // [a1][a2][a3 + 2 a4] -> [a1][a2][a3][a4]
        Ft[((long long)GC[c] * 64 + spin) * V + q] = sum;
      }
      nb_sync(BAR_PROD, NH);  // the stage's slots are clear before its next momentum can start
      if (tp == 0 && i + S < n && !*ABORT) {
        issue(i + S);
        last = i + S;
      }
    }
    // a wait gave up: let this block's copies in flight land (bounded) before its shared memory goes
    if (tp == 0 && *ABORT)
      for (int i = max(0, last - S + 1); i <= last; ++i)
        for (int k = 0; k < 8; ++k) {
          volatile int never = 0;  // a private flag: these waits run to their own limit
          if (mb_wait(MBF + 8u * (i % S), (unsigned)((i / S) & 1), &never, flags)) break;
        }
    return;
  }

  // ================= consumers =================
  const int wc = w - NHW;
  const int s_begin = ck.seg_base[wc], s_end = ck.seg_base[wc + 1];
  // the warp's records: steps [SEG[s_begin].sbeg, SEG[s_end - 1].send), the same for every momentum; the
  // first RPREF of them stay in registers, the rest are read two steps ahead (the table has padding steps
  // after its last chunk)
  const int st_a = s_begin < s_end ? SEG[s_begin].sbeg : 0, st_b = s_begin < s_end ? SEG[s_end - 1].send : 0;
  const unsigned* const R0 = rec + ck.rec_off + st_a * 32 + lane;
  unsigned first[RPREF];
#pragma unroll
  for (int k = 0; k < RPREF; ++k) first[k] = __ldg(R0 + 32 * k);
  for (int i = 0; i < n; ++i) {
    const int b = i % NBS_ROW_STAGES;
    mb_wait(MBF + 8u * b, (unsigned)((i / NBS_ROW_STAGES) & 1), ABORT, flags);  // the rows of i have landed
    const float4* const E1 = RS0 + b * stage_units;  // B1's rows: plane 0 [nrow1], plane 1 [nrow1]
    const float4* const E2 = E1 + 2 * nrow1;          // B2's rows: plane 0 [nrow2], plane 1 [nrow2]
    float2* const out_w = OUT0 + b * nslot * 64 + (ck.out_base[wc] - ck.cfirst[wc]) * 64;
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
        x1 = pa[nrow1];
        y0 = pb[0];
        y1 = pb[nrow2];
      };
      auto product = [&](const float4& x0, const float4& x1, const float4& y0, const float4& y1, float scale) {
        const float2 a[4] = {make_float2(x0.x * scale, x0.y * scale), make_float2(x0.z * scale, x0.w * scale),
                             make_float2(x1.x * scale, x1.y * scale), make_float2(x1.z * scale, x1.w * scale)};
        const float2 bb[4] = {make_float2(y0.x, y0.y), make_float2(y0.z, y0.w), make_float2(y1.x, y1.y),
                              make_float2(y1.z, y1.w)};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float2 z = make_float2(acc[2 * (4 * u + v)], acc[2 * (4 * u + v) + 1]);
            cfma<float>(z, a[u], bb[v]);
            acc[2 * (4 * u + v)] = z.x;
            acc[2 * (4 * u + v) + 1] = z.y;
          }
      };
      int si = s_begin, seg_end = si < s_end ? SEG[si].send : 0, local = si < s_end ? SEG[si].local : 0;
      int map = si < s_end ? SEG[si].map : 0;
      auto after_step = [&](int st) {
        if (st + 1 == seg_end) {
          rows_flush(acc, lane, out_w + local * 64, map);
          if (++si < s_end) {
            seg_end = SEG[si].send;
            local = SEG[si].local;
            map = SEG[si].map;
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
    mb_arrive(MBE + 8u * b);  // B(i) done: its rows may be overwritten, its slots summed
  }
}

}  // namespace

size_t row_chunk_smem(int nrow1, int nrow2, int nslot, int nseg, int nch) {
  return 128 + row_layout(nrow1, nrow2, nslot, nseg, nch).total;
}

cudaError_t launch_eff_rows(const float2* FB, long long V, const void* types, int ntypes, const unsigned* desc,
                            const unsigned short* ent, int nent, int NR, float2* RQ, int nsm, cudaStream_t st) {
  if (!FB || !RQ || V <= 0 || NR <= 0 || NR % 8 || ntypes < 1 || ntypes > 8 || nent < 0 ||
      (reinterpret_cast<uintptr_t>(FB) & 15) || (reinterpret_cast<uintptr_t>(RQ) & 15))
    return cudaErrorInvalidValue;
  const size_t smem = EFF_TILE_BYTES + 128 + 4 * (size_t)NR + 2 * (size_t)nent;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_eff_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // exactly the blocks that are resident at once (a grid-stride loop: a block queued behind them would
  // start only when one of them has finished all of its tiles)
  int per_sm = 0;
  cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eff_rows, EFF_THREADS, smem);
  if (oe != cudaSuccess) return oe;
  const long long tiles = (V + 31) / 32 * (NR / 8);
  const long long blocks = std::min<long long>(tiles, (long long)std::max(nsm, 1) * std::max(per_sm, 1));
  k_eff_rows<<<(unsigned)blocks, EFF_THREADS, smem, st>>>(reinterpret_cast<const float4*>(FB), V,
                                                           (const RowTypeHdr*)types, ntypes, desc, ent, nent, NR,
                                                           reinterpret_cast<float4*>(RQ));
  return cudaGetLastError();
}

cudaError_t launch_contract_rows(const float2* RQ, const MomGeom& geom, int NR, const int2* qlist, int nchunks, int qb,
                                 const void* chunks, const unsigned* rec, const void* segs, const int* row_ch,
                                 const float* scales, int smem, float2* Ft, int* flags, cudaStream_t st) {
  const long long V = (long long)geom.L * geom.Ly * geom.L;
  if (nchunks <= 0 || qb <= 0 || smem <= 0 || NR <= 0 || !qlist || !RQ || !flags ||
      (reinterpret_cast<uintptr_t>(RQ) & 15) || geom.L < 1 || geom.L > 64 || geom.Ly < 1 || geom.Ly > geom.L)
    return cudaErrorInvalidValue;
  const long long nqb = (V + qb - 1) / qb;
  if (nqb * nchunks > 2147483647LL) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_contract_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_contract_rows<<<(unsigned)(nqb * nchunks), (NBS_ROW_WARPS + NBS_ROW_HELPERS) * 32, smem, st>>>(
      reinterpret_cast<const float4*>(RQ), V, NR, qlist, nchunks, qb, (const RowChunkHdr*)chunks, rec,
      (const RowSeg*)segs, row_ch, scales, Ft, flags);
  return cudaGetLastError();
}

// The momenta of a geometry in the order the row kernel visits them, as (q, -q) pairs of linear indices:
// each q with q <= -q, followed by -q when that differs.  The first members are a permutation of 0 .. V - 1;
// empty if the geometry's mirror table does not make them one.
std::vector<int2> momentum_order(const MomGeom& g) {
  std::vector<int2> out;
  if (g.L < 1 || g.L > 64 || g.Ly < 1 || g.Ly > g.L) return out;
  for (int y = 0; y < g.Ly; ++y)
    if (g.ymir[y] < 0 || g.ymir[y] >= g.Ly || g.ymir[g.ymir[y]] != y) return out;
  const long long V = (long long)g.L * g.Ly * g.L;
  out.reserve((size_t)V);
  for (long long q = 0; q < V; ++q) {
    const int x = (int)(q % g.L), y = (int)((q / g.L) % g.Ly), z = (int)(q / ((long long)g.L * g.Ly));
    const long long m = (long long)((g.L - x) % g.L) + g.L * ((long long)g.ymir[y] + (long long)g.Ly * ((g.L - z) % g.L));
    if (m < q) continue;
    out.push_back(make_int2((int)q, (int)m));
    if (m != q) out.push_back(make_int2((int)m, (int)q));
  }
  std::vector<char> seen((size_t)V, 0);
  for (const int2& p : out) {
    if (p.x < 0 || p.x >= V || p.y < 0 || p.y >= V || seen[(size_t)p.x]) return std::vector<int2>();
    seen[(size_t)p.x] = 1;
  }
  if ((long long)out.size() != V) out.clear();
  return out;
}

}  // namespace nbs
