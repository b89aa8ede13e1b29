// tma.cuh -- TMA staging of the stored-block slabs for the quad-lane
// contractions (kernels_quad.cu, kernels_tcq.cu).
//
// The stored blocks [cell][site][4 spins] (complex FP32) are seen as a 3-D
// FP32 tensor: 8 values (one cell's four spins at one momentum, 32 bytes),
// momenta (stride 32 bytes), cells (stride V * 32 bytes).  One box is 236
// cells of one momentum, so four boxes fill a 944-cell slab side; the box's x
// coordinate is always 0 (16-byte aligned).  An mbarrier per slab buffer
// counts the bytes; waits on it are bounded.
#pragma once
#include <cuda.h>  // CUtensorMap (encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include <cstdint>

namespace nbs {

constexpr int QUAD_BOX = 236;                // cells per TMA box
constexpr int QUAD_BOX_BYTES = QUAD_BOX * 32;
constexpr int QUAD_WAIT_LIMIT = 1 << 20;     // mbarrier polls before a wait gives up

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(addr), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity) {
  for (int i = 0; i < QUAD_WAIT_LIMIT; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// wait bounded in time (limit_ns of the global timer) and in polls; false if it gave up
__device__ __forceinline__ bool mbar_wait_timed(unsigned addr, unsigned parity, unsigned long long limit_ns) {
  unsigned long long t0 = 0;
  for (int i = 0; i < (1 << 28); ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255) == 255) {
      const unsigned long long t = global_ns();
      if (!t0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}

// Stage the slabs of one momentum into buffer S (side 1: ncell1 cells from
// base1 at q; side 2 at the cell offset side2 bytes: ncell2 cells from base2 at
// qm) with mbarrier mb; called by one thread after the block has finished
// reading S.
__device__ __forceinline__ void tma_issue_slabs(const CUtensorMap* map, unsigned S, unsigned side2, unsigned mb,
                                                int base1, int ncell1, int q, int base2, int ncell2, int qm) {
  const int nb1 = (ncell1 + QUAD_BOX - 1) / QUAD_BOX, nb2 = (ncell2 + QUAD_BOX - 1) / QUAD_BOX;
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier generic reads of S first
  mbar_expect_tx(mb, (unsigned)((nb1 + nb2) * QUAD_BOX_BYTES));
  for (int k = 0; k < nb1; ++k) tma_load_3d(S + k * QUAD_BOX_BYTES, map, 0, q, base1 + k * QUAD_BOX, mb);
  for (int k = 0; k < nb2; ++k) tma_load_3d(S + side2 + k * QUAD_BOX_BYTES, map, 0, qm, base2 + k * QUAD_BOX, mb);
}

// Host: encode the map of FB (V momenta, ncells cells); false if TMA is not
// available (the caller then stages with cp.async).
bool encode_fb_map(CUtensorMap* map, const float2* FB, long long V, long long ncells);

}  // namespace nbs
